// Generic BF16 tensor-core GEMM with FP32 operands in global memory, for the
// learned initialiser's network (forward and backward passes):
//   D(m, n) = epilogue( sum_k A(m, k) B(n, k) ),  A(m, k) = A[m sam + k sak],
//   B(n, k) = B[n sbn + k sbk]  (any strides, so transposed operands need no copy),
// epilogue: + bias[n], ReLU, times [mask(m, n) > 0], and D = or D +=.
//
// One CTA per 128 x 128 output tile.  Each 64-wide K step, the CTA's threads
// read both 128 x 64 operand tiles (coalesced along whichever of the two
// strides is 1), round them to BF16 and store them K-major in the 128-byte-
// swizzled layout; one thread issues four tcgen05.mma (M = N = 128, K = 16)
// accumulating in tensor memory and commits to an mbarrier that releases the
// double-buffered tile two steps later.  Warps 0-3 read the accumulator rows
// back (tcgen05.ld) for the epilogue.  All mbarrier waits are bounded; on a
// timeout the CTA writes NaN into its output tile, waits (bounded) for its
// MMAs, frees its tensor memory and returns.
#include <cuda_bf16.h>
#include <stdint.h>

#include "kernels.h"
#include "tc_common.cuh"

namespace cpdk {
namespace {

using namespace tc;

constexpr int kTile = 128;
constexpr int kKT = 64;
constexpr int kThreads = 256;
constexpr uint32_t kTileBytes = kTile * 128;      // 128 rows x 64 BF16

// One 128 x 64 operand tile: rows r0.., K columns k0.. of X(r, k) = X[r sr + k sk]
// (zero outside rows < nr, k < nk), BF16, K-major, 128-byte swizzle.
__device__ __forceinline__ void load_tile(const float* __restrict__ X, long long sr, long long sk, int nr, int nk,
                                          int r0, int k0, unsigned char* dst) {
  if (sk == 1) {
    // items (row, 8-value chunk), chunks fastest: 8 threads read 256 contiguous bytes
    for (int e = threadIdx.x; e < kTile * 8; e += kThreads) {
      const int rl = e >> 3, c = e & 7, r = r0 + rl, k = k0 + 8 * c;
      float f[8];
      const float* p = X + (long long)r * sr + k;
      if (r < nr && k + 8 <= nk && ((reinterpret_cast<uintptr_t>(p) & 15u) == 0)) {
        const float4 a = *reinterpret_cast<const float4*>(p), b = *reinterpret_cast<const float4*>(p + 4);
        f[0] = a.x; f[1] = a.y; f[2] = a.z; f[3] = a.w; f[4] = b.x; f[5] = b.y; f[6] = b.z; f[7] = b.w;
      } else {
#pragma unroll
        for (int u = 0; u < 8; ++u) f[u] = (r < nr && k + u < nk) ? p[u] : 0.f;
      }
      const int sw = rl & 7;
      *reinterpret_cast<uint4*>(dst + (rl >> 3) * 1024 + sw * 128 + ((c ^ sw) << 4)) = pack_bf16x8(f);
    }
  } else {
    // items (chunk, row), rows fastest: a warp reads 32 consecutive rows per value
    // (coalesced when sr == 1), and its 16-byte stores hit eight distinct chunks
    for (int e = threadIdx.x; e < kTile * 8; e += kThreads) {
      const int c = e >> 7, rl = e & 127, r = r0 + rl, k = k0 + 8 * c;
      float f[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) f[u] = (r < nr && k + u < nk) ? X[(long long)r * sr + (long long)(k + u) * sk] : 0.f;
      const int sw = rl & 7;
      *reinterpret_cast<uint4*>(dst + (rl >> 3) * 1024 + sw * 128 + ((c ^ sw) << 4)) = pack_bf16x8(f);
    }
  }
}

__global__ void __launch_bounds__(kThreads, 1) k_gemm_tc(GemmArgs a) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t pad = (1024u - (raw & 1023u)) & 1023u;
  unsigned char* sm = smem_raw + pad;
  const uint32_t sb = raw + pad;
  // layout: A0 | A1 | B0 | B1 (16 KB each) | 2 mbarriers | tensor-memory address
  const uint32_t bar = sb + 4 * kTileBytes;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + 4 * kTileBytes + 16);
  const int m0 = blockIdx.x * kTile, n0 = blockIdx.y * kTile;
  const int nsteps = (a.K + kKT - 1) / kKT;

  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar + 8u) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"(128u)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tslot;
  const uint32_t idesc = mma_idesc(kTile, kTile);

  bool ok = true;
  int committed = 0;
  for (int j = 0; j < nsteps; ++j) {
    const int b = j & 1;
    bool fail = false;
    if (j >= 2) fail = !mbar_wait(bar + 8u * b, (uint32_t)(((j - 2) >> 1) & 1));
    if (__syncthreads_or(fail)) { ok = false; break; }
    unsigned char* ta = sm + (uint32_t)b * kTileBytes;
    unsigned char* tb = sm + (uint32_t)(2 + b) * kTileBytes;
    load_tile(a.A, a.sam, a.sak, a.M, a.K, m0, j * kKT, ta);
    load_tile(a.B, a.sbn, a.sbk, a.N, a.K, n0, j * kKT, tb);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    committed = j + 1;
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t sa = sb + (uint32_t)b * kTileBytes, sbb = sb + (uint32_t)(2 + b) * kTileBytes;
#pragma unroll
      for (int kk = 0; kk < kKT / 16; ++kk) {
        const uint64_t ad = sw128_desc(sa + kk * 32u), bd = sw128_desc(sbb + kk * 32u);
        const uint32_t acc = (j > 0 || kk > 0) ? 1u : 0u;
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
            "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
            : "memory");
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar + 8u * b)
                   : "memory");
    }
  }
  if (committed > 0) {
    const int jl = committed - 1;
    const bool fail = !mbar_wait(bar + 8u * (jl & 1), (uint32_t)((jl >> 1) & 1));
    if (__syncthreads_or(fail)) ok = false;
  }
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp < 4) {
    const int m = m0 + warp * 32 + lane;
    const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
    for (int c0 = 0; c0 < kTile; c0 += 16) {
      uint32_t r[16];
      if (committed > 0 && ok) {
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
            "[%16];"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
              "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
              "=r"(r[15])
            : "r"(tmem + lane_base + (uint32_t)c0));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      } else {
#pragma unroll
        for (int u = 0; u < 16; ++u) r[u] = (committed > 0) ? 0x7fc00000u : 0u;   // K == 0: zero; failure: NaN
      }
      if (m >= a.M) continue;
#pragma unroll
      for (int u = 0; u < 16; ++u) {
        const int n = n0 + c0 + u;
        if (n >= a.N) break;
        float v = __uint_as_float(r[u]);
        if (a.bias) v += a.bias[n];
        if (a.relu) v = fmaxf(v, 0.f);
        if (a.mask && !(a.mask[(long long)m * a.ldm + n] > 0.f)) v = 0.f;
        float* d = a.D + (long long)m * a.ldd + n;
        *d = a.accumulate ? *d + v : v;
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(128u) : "memory");
}

constexpr size_t kSmem = 1024 + 4 * (size_t)kTileBytes + 64;

}  // namespace

cudaError_t launch_gemm_tc(const GemmArgs& a, cudaStream_t st) {
  if (a.M < 0 || a.N < 0 || a.K < 0) return cudaErrorInvalidValue;
  if (a.M == 0 || a.N == 0) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(k_gemm_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem);
  if (e != cudaSuccess) return e;
  dim3 grid((unsigned)((a.M + kTile - 1) / kTile), (unsigned)((a.N + kTile - 1) / kTile));
  k_gemm_tc<<<grid, kThreads, kSmem, st>>>(a);
  count_launch();
  return cudaGetLastError();
}

}  // namespace cpdk
