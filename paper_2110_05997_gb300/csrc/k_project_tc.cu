// First-mode projection of the MLSVD on tensor cores (Sec. 4.1.1 and the
// algorithm "ST-MLSVD" of the thesis: the first truncation step replaces T by
// T x_1 U^(1)T, i.e. every column t_k of the unfolding T_(1) by U^T t_k).
//
// As a matrix product, D(k, r) = sum_j T_(1)(j, k) U(j, r): the columns of
// T_(1) are the rows of the K-major operand A (K = I contiguous floats), U is
// the K-major operand B (row r = column r of U), M = 128 columns per tile,
// ranks padded to 16, K = I.  FP32 accuracy from TF32 tensor cores by the
// split x = hi + lo, hi = x with its 13 low mantissa bits cleared (exact in
// TF32), lo = x - hi (exact in FP32, read by the tensor core to 11
// significant bits), on both operands: with B' = [Bhi; Blo] (N = 32) the two
// MMAs Ahi B' and Alo B' go to two independent accumulators (short dependent
// chains of small MMAs), and D = Ahi Bhi + Ahi Blo + Alo Bhi + Alo Blo; the
// truncation of lo is below 2^-21 of each |x u|.
//
// One CTA per SM takes a contiguous range of 128-column tiles; a tile is
// consumed in chunks of 32 K-floats (one 128-byte swizzled row per column).
// The roles hand chunks over through mbarriers only (no CTA-wide barrier in
// the loop):
//   * thread 256 (the issuer) loads each chunk with a 2D tensor copy (TMA,
//     128-byte swizzle, rows past the end of T and K past I zero-filled) into
//     one of S shared-memory stages, completed on mbarriers, and refills a
//     stage as soon as it has been split (S chunks in flight);
//   * warps 0-7 split the chunk (the 16-byte pieces the MMAs read) into one
//     of three (hi, lo) operand buffers (same swizzled layout), once that
//     buffer's previous MMAs are done, and arrive on the buffer's mbarrier;
//   * the issuer issues the two tcgen05.mma kind::tf32 per K-step of 8 into
//     one of four tile accumulators in tensor memory (M = 128 lanes x 64 FP32
//     columns), commits to the operand buffer's mbarrier and, after a tile's
//     last chunk, to the accumulator's mbarrier;
//   * warps 0-3 read an accumulator back (tcgen05.ld) two tiles later, add
//     its four parts, stage each warp's 32 rows in shared memory and store
//     them as one contiguous run of Y (Y[r + rk k], r < rk), 16-byte stores.
// Every mbarrier wait is bounded and gives up when another role has raised
// the CTA's abort flag; a CTA that timed out poisons Y with NaN, sets the
// error flag, waits a bounded time for its own copies and MMAs, frees its
// tensor memory and returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <stdint.h>

#include <mutex>

#include "kernels.h"
#include "tc_common.cuh"

namespace cpdk {
namespace {

using namespace tc;

constexpr int kM = 128;                       // columns of T_(1) per tile
constexpr int kN = 16;                        // MMA N (ranks padded)
constexpr int kKC = 32;                       // K floats per chunk (128 bytes)
constexpr uint32_t kChunkBytes = kM * kKC * 4;
constexpr uint32_t kBBytes = kN * 128;              // one 16-row operand tile of B
constexpr int kConv = 256;                    // warps 0-7 split; warps 0-3 read tensor memory
constexpr int kIssuer = kConv;                // warp 8, lane 0
constexpr int kThreads = kConv + 32;
constexpr int kMaxStages = 6;                 // FP32 chunks in flight
constexpr int kOpBufs = 3;                    // (hi, lo) operand buffers
constexpr int kAcc = 4;                       // tile accumulators
constexpr int kAccCols = 4 * kN;              // per tile: hi x [Bhi | Blo], lo x [Bhi | Blo]
constexpr int kOutLd = 33;                    // row stride of a warp's output staging (floats)
constexpr long long kDrainBudget = 1ll << 31;

struct PtcArgs {
  float* Y;
  const float* U;             // I x P column-major, rk <= 16 columns used
  const int* dev_rank;
  int I, nch, stages;
  long long c, ntiles;
  int* err;
  long long budget;
  int vec4;                   // Y is 16-byte aligned: float4 stores
};

// kind::tf32 instruction descriptor: FP32 accumulator (bits 4-5 = 1), TF32 A
// and B (bits 7-9 and 10-12 = 2), both K-major, N >> 3 at bit 17, M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
      "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ float tf32_hi(float x) { return __uint_as_float(__float_as_uint(x) & 0xffffe000u); }

// Bounded wait on an mbarrier phase that also gives up once another role has
// raised the CTA's abort flag.
__device__ __forceinline__ bool wait_or_abort(uint32_t bar, uint32_t parity, long long budget,
                                              volatile int* abort_flag) {
  const long long t0 = clock64();
  for (;;) {
    if (mbar_try(bar, parity)) return true;
    if (*abort_flag) return false;
    if (clock64() - t0 > budget) return false;
  }
}

__global__ void __launch_bounds__(kThreads, 1) k_project_tc(const __grid_constant__ CUtensorMap map, PtcArgs a) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const long long t_begin = (long long)blockIdx.x * a.ntiles / gridDim.x;
  const long long t_end = (long long)(blockIdx.x + 1) * a.ntiles / gridDim.x;
  const int ntl = (int)(t_end - t_begin);
  const int nch = a.nch, S = a.stages;
  const int nunits = ntl * nch;

  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t pad = (1024u - (raw & 1023u)) & 1023u;
  unsigned char* sm = smem_raw + pad;
  const uint32_t sb = raw + pad;
  const uint32_t o_op = (uint32_t)S * kChunkBytes;                // kOpBufs x (hi, lo) operand buffers
  const uint32_t o_b = o_op + kOpBufs * 2u * kChunkBytes;          // B tiles: chunk ch at o_b + ch * 2 kBBytes
  const uint32_t o_bar = o_b + (uint32_t)nch * 2u * kBBytes;
  const uint32_t bar_full = sb + o_bar;                           // S barriers: chunk landed
  const uint32_t bar_conv = bar_full + 8u * kMaxStages;           // kOpBufs barriers: buffer split (kConv arrivals)
  const uint32_t bar_done = bar_conv + 8u * kOpBufs;              // kOpBufs barriers: buffer's MMAs done
  const uint32_t bar_acc = bar_done + 8u * kOpBufs;               // kAcc barriers: tile's accumulator ready
  uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + o_bar + 8 * (kMaxStages + 2 * kOpBufs + kAcc));
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tslot + 1);
  float* outs = reinterpret_cast<float*>(sm + o_bar + 8 * (kMaxStages + 2 * kOpBufs + kAcc) + 16);   // 4 x 16 x kOutLd
  const int rk = *a.dev_rank;                                     // <= 16 (launcher's bound)

  // B = U, split, zero beyond rank rk and beyond K = I, K-major swizzled
  for (int e = tid; e < nch * kN * kKC; e += kThreads) {
    const int ch = e / (kN * kKC), rem = e - ch * (kN * kKC), n = rem / kKC, kk = rem - n * kKC;
    const int j = ch * kKC + kk;
    const float u = (n < rk && j < a.I) ? a.U[(size_t)n * a.I + j] : 0.f;
    const float h = tf32_hi(u);
    const uint32_t off = sw128_offset((uint32_t)n, (uint32_t)kk * 4u);
    *reinterpret_cast<float*>(sm + o_b + (uint32_t)ch * 2u * kBBytes + off) = h;
    *reinterpret_cast<float*>(sm + o_b + (uint32_t)ch * 2u * kBBytes + kBBytes + off) = u - h;
  }
  if (tid == 0) {
    *abort_flag = 0;
    for (int s = 0; s < kMaxStages; ++s) mbar_init(bar_full + 8u * s, 1);
    for (int b = 0; b < kOpBufs; ++b) { mbar_init(bar_conv + 8u * b, kConv); mbar_init(bar_done + 8u * b, 1); }
    for (int b = 0; b < kAcc; ++b) mbar_init(bar_acc + 8u * b, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) tmem_alloc(smem_u32(tslot), kAcc * kAccCols);
  fence_async_smem();
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = *tslot;

  // rows of a finished tile: warp w (< 4) holds columns 32 w .. 32 w + 31 of it
  auto epilogue = [&](int tl) -> bool {
    const int b = tl % kAcc;
    if (!wait_or_abort(bar_acc + 8u * (uint32_t)b, (uint32_t)((tl / kAcc) & 1), a.budget, abort_flag)) return false;
    fence_after_sync();
    // columns of accumulator b: [hi Bhi | hi Blo | lo Bhi | lo Blo], 16 each
    float v[4][16];
    const uint32_t t0 = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)b * kAccCols;
#pragma unroll
    for (int p = 0; p < 4; ++p) tmem_ld16(t0 + (uint32_t)p * kN, v[p]);
    tmem_ld_wait();
    fence_before_sync();
    // the warp's 32 columns through its own shared-memory block (row r at
    // r * kOutLd: conflict-free both ways), then out as one contiguous run
    // Y[rk k0 .. rk (k0 + nc)), k0 = the warp's first column; warp-local only
    float* ow = outs + warp * (kN * kOutLd);
    __syncwarp();                                          // the previous copy-out has read ow
#pragma unroll
    for (int r = 0; r < 16; ++r) ow[r * kOutLd + lane] = ((v[3][r] + v[2][r]) + v[1][r]) + v[0][r];
    __syncwarp();
    const long long k0 = (t_begin + tl) * kM + warp * 32;
    const int nc = (int)max(0ll, min(32ll, a.c - k0));
    const int nout = rk * nc;
    float* y = a.Y + (size_t)rk * (size_t)k0;
    if (a.vec4) {                                          // rk k0 is a multiple of 4 (k0 of 32)
      for (int o = 4 * lane; o < nout; o += 128) {
        int mm = o / rk, r = o - mm * rk;
        float f[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          f[u] = (o + u < nout) ? ow[r * kOutLd + mm] : 0.f;
          if (++r == rk) { r = 0; ++mm; }
        }
        if (o + 4 <= nout) {
          *reinterpret_cast<float4*>(y + o) = make_float4(f[0], f[1], f[2], f[3]);
        } else {
          for (int u = 0; u < 4 && o + u < nout; ++u) y[o + u] = f[u];
        }
      }
    } else {
      for (int o = lane; o < nout; o += 32) {
        const int mm = o / rk, r = o - mm * rk;
        y[o] = ow[r * kOutLd + mm];
      }
    }
    return true;
  };

  int issued = 0, committed = 0;         // issuer: chunks copied / whose MMAs were committed
  int acc_tile = -1;                     // issuer: last tile whose accumulator was committed
  if (tid < kConv) {
    // ---- split: stage -> (hi, lo) buffer; warps 0-3 also store finished tiles
    bool ok = true;
    for (int j = 0; j < nunits && ok; ++j) {
      const int s = j % S, ob = j % kOpBufs, ch = j % nch, tl = j / nch;
      if (!wait_or_abort(bar_full + 8u * (uint32_t)s, (uint32_t)((j / S) & 1), a.budget, abort_flag) ||
          (j >= kOpBufs &&
           !wait_or_abort(bar_done + 8u * (uint32_t)ob, (uint32_t)((j / kOpBufs - 1) & 1), a.budget, abort_flag))) {
        ok = false;
        break;
      }
      const float4* x4 = reinterpret_cast<const float4*>(sm + (uint32_t)s * kChunkBytes);
      float4* hi = reinterpret_cast<float4*>(sm + o_op + (uint32_t)ob * 2u * kChunkBytes);
      float4* lo = reinterpret_cast<float4*>(sm + o_op + (uint32_t)ob * 2u * kChunkBytes + kChunkBytes);
      // 16-byte pieces the MMAs read: logical piece (physical piece ^ row % 8) < 2 ks
      const int npieces = 2 * ((min(kKC, a.I - ch * kKC) + 7) >> 3);
#pragma unroll
      for (int q = 0; q < (int)(kChunkBytes / 16) / kConv; ++q) {
        const int e = q * kConv + tid;
        if (((e & 7) ^ ((e >> 3) & 7)) >= npieces) continue;
        const float4 x = x4[e];
        const float4 h = make_float4(tf32_hi(x.x), tf32_hi(x.y), tf32_hi(x.z), tf32_hi(x.w));
        hi[e] = h;
        lo[e] = make_float4(x.x - h.x, x.y - h.y, x.z - h.z, x.w - h.w);
      }
      fence_async_smem();
      asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar_conv + 8u * (uint32_t)ob) : "memory");
      // a tile's rows are stored two tiles later, when its MMAs have long completed
      if (warp < 4 && ch == 0 && tl >= 2) ok = epilogue(tl - 2);
    }
    if (ok && warp < 4)
      for (int tl = ntl - 2 < 0 ? 0 : ntl - 2; tl < ntl && ok; ++tl) ok = epilogue(tl);
    if (!ok) *abort_flag = 1;
  } else if (tid == kIssuer) {
    // ---- copies and MMAs
    auto issue = [&](int j) {             // chunk j of this CTA into stage j % S
      const uint32_t bar = bar_full + 8u * (uint32_t)(j % S);
      const uint32_t dst = sb + (uint32_t)(j % S) * kChunkBytes;
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(kChunkBytes) : "memory");
      tma_load_2d(dst, &map, (j % nch) * kKC, (int)((t_begin + j / nch) * kM), bar);
    };
    for (; issued < S && issued < nunits; ++issued) issue(issued);
    const uint32_t idesc = idesc_tf32(kM, 2 * kN);
    for (int j = 0; j < nunits; ++j) {
      const int ob = j % kOpBufs, ch = j % nch, tl = j / nch;
      if (!wait_or_abort(bar_conv + 8u * (uint32_t)ob, (uint32_t)((j / kOpBufs) & 1), a.budget, abort_flag)) {
        *abort_flag = 1;
        break;
      }
      if (issued < nunits) { issue(issued); ++issued; }   // chunk j's stage has been read: chunk j + S
      fence_after_sync();
      const int kv = min(kKC, a.I - ch * kKC);
      const int ks = (kv + 7) >> 3;
      const uint32_t ahi = sb + o_op + (uint32_t)ob * 2u * kChunkBytes, alo = ahi + kChunkBytes;
      const uint32_t bb = sb + o_b + (uint32_t)ch * 2u * kBBytes;      // 32 rows: Bhi, then Blo
      const uint32_t dt = tmem + (uint32_t)(tl % kAcc) * kAccCols;
      for (int kk = 0; kk < ks; ++kk) {
        const uint32_t ko = (uint32_t)kk * 32u, acc = (ch > 0 || kk > 0) ? 1u : 0u;
        mma_tf32(dt, sw128_desc(ahi + ko), sw128_desc(bb + ko), idesc, acc);
        mma_tf32(dt + 2 * kN, sw128_desc(alo + ko), sw128_desc(bb + ko), idesc, acc);
      }
      mma_commit(bar_done + 8u * (uint32_t)ob);
      if (ch == nch - 1) { mma_commit(bar_acc + 8u * (uint32_t)(tl % kAcc)); acc_tile = tl; }
      committed = j + 1;
    }
  }
  __syncthreads();
  if (tid == kIssuer) {
    const bool failed = *abort_flag != 0;
    if (failed) {
      a.Y[0] = __int_as_float(0x7fc00000);
      if (a.err) atomicExch(a.err, CPD_ERR_TIMEOUT);
      // the last copy issued into each stage (earlier ones were consumed)
      for (int j = issued - S < 0 ? 0 : issued - S; j < issued; ++j)
        (void)mbar_wait_cycles(bar_full + 8u * (uint32_t)(j % S), (uint32_t)((j / S) & 1), kDrainBudget);
    }
    if (committed > 0) {                   // every MMA of this CTA has completed
      const int jl = committed - 1;
      (void)mbar_wait_cycles(bar_done + 8u * (uint32_t)(jl % kOpBufs), (uint32_t)((jl / kOpBufs) & 1),
                             failed ? kDrainBudget : a.budget);
    }
    if (failed && acc_tile >= 0)           // and its last accumulator arrive has landed
      (void)mbar_wait_cycles(bar_acc + 8u * (uint32_t)(acc_tile % kAcc), (uint32_t)((acc_tile / kAcc) & 1),
                             kDrainBudget);
  }
  fence_before_sync();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, kAcc * kAccCols);
}

size_t ptc_smem(int nch, int S) {
  return 1024 + (size_t)S * kChunkBytes + (size_t)kOpBufs * 2 * kChunkBytes + (size_t)nch * 2 * kBBytes +
         8 * (kMaxStages + 2 * kOpBufs + kAcc) + 16 + (size_t)4 * kN * kOutLd * 4;
}

struct PtcCache {
  std::mutex mu;
  int dev = -1, sms = 0, lim = 0;
  size_t have = 0;
};
PtcCache g_ptc;

}  // namespace

bool project_tc_supported(long long I, long long c, int rmax, const float* T) {
  return I >= 32 && I <= 256 && (I % 4) == 0 && c >= kM && c < (1ll << 31) && rmax >= 1 && rmax <= kN &&
         (reinterpret_cast<uintptr_t>(T) & 15u) == 0 && tensor_map_encoder() != nullptr;
}

cudaError_t launch_project_tc(const float* T, long long I, long long c, const float* U, const int* dev_rank,
                              int rmax, float* Y, cudaStream_t st, int* err, long long budget) {
  if (!project_tc_supported(I, c, rmax, T)) return cudaErrorNotSupported;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  PtcArgs a{};
  a.Y = Y; a.U = U; a.dev_rank = dev_rank; a.I = (int)I; a.c = c;
  a.nch = (int)((I + kKC - 1) / kKC);
  a.ntiles = (c + kM - 1) / kM;
  a.err = err;
  a.budget = budget > 0 ? budget : (1ll << 31);
  a.vec4 = (reinterpret_cast<uintptr_t>(Y) & 15u) == 0 ? 1 : 0;
  int sms = 0;
  size_t smem = 0;
  {
    std::lock_guard<std::mutex> lk(g_ptc.mu);
    if (g_ptc.dev != dev) {
      g_ptc.dev = dev; g_ptc.have = 0;
      if ((e = cudaDeviceGetAttribute(&g_ptc.sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
      if ((e = cudaDeviceGetAttribute(&g_ptc.lim, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) != cudaSuccess)
        return e;
    }
    int S = kMaxStages;
    while (S > 2 && ptc_smem(a.nch, S) > (size_t)g_ptc.lim) --S;
    smem = ptc_smem(a.nch, S);
    if (smem > (size_t)g_ptc.lim) return cudaErrorNotSupported;
    a.stages = S;
    if (g_ptc.have < smem) {
      if ((e = cudaFuncSetAttribute(k_project_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) !=
          cudaSuccess)
        return e;
      g_ptc.have = smem;
    }
    sms = g_ptc.sms;
  }
  // T_(1) as a 2D tensor: I floats per column (inner), c columns; boxes of 32 x 128
  CUtensorMap map;
  cuuint64_t gdim[2] = {(cuuint64_t)I, (cuuint64_t)c};
  cuuint64_t gstride[1] = {(cuuint64_t)I * 4};
  cuuint32_t box[2] = {(cuuint32_t)kKC, (cuuint32_t)kM};
  cuuint32_t estr[2] = {1, 1};
  if (tensor_map_encoder()(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(T), gdim, gstride, box, estr,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return cudaErrorInvalidValue;
  const long long grid = a.ntiles < sms ? a.ntiles : sms;
  k_project_tc<<<(unsigned)grid, kThreads, smem, st>>>(map, a);
  count_launch();
  return cudaGetLastError();
}

}  // namespace cpdk
