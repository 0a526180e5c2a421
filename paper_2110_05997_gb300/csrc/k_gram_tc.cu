// BF16 tensor-core Gram of the first-mode unfolding (Sec. 4.1.1 and App. A of
// the thesis: the left singular vectors of T_(1) come from the eigenpairs of
// G = T_(1) T_(1)^T).  A = T_(1) is the column-major I x C matrix whose
// columns are contiguous in T, so a run of 64 columns is one contiguous block
// of 64*I floats.
//
// One CTA per SM takes a contiguous range of 64-column steps:
//   * thread 0 streams each step's FP32 block into a shared-memory stage with a
//     bulk asynchronous copy completed on an mbarrier (several stages in flight);
//   * the warpgroup converts the stage to BF16, writing it K-major (row i holds
//     the step's 64 values of row i of A, 128 bytes) in the 128-byte-swizzled
//     layout the tensor core reads;
//   * thread 0 issues tcgen05.mma (M = 128, N = ceil16(I), K = 16 each) into
//     FP32 accumulators in tensor memory: D_m += X[128m : 128m+128] X^T for the
//     one or two 128-row tiles m of X, and commits to an mbarrier that frees
//     the BF16 buffer (double-buffered) for the step after next;
//   * finally each thread reads its accumulator row back (tcgen05.ld) and adds
//     it into G with vector atomics; G is symmetric, so row i of D goes to the
//     contiguous column i of G.
// Every mbarrier wait is bounded; on a timeout the CTA poisons G with NaN
// (the solve then ends with a numeric status), waits a bounded time for its
// own copies, frees its tensor memory and returns.
#include <cuda_bf16.h>
#include <stdint.h>

#include "kernels.h"

namespace cpdk {
namespace {

constexpr int kKT = 64;                   // unfolding columns per step
constexpr int kThreads = 128;             // one warpgroup
constexpr int kMaxStages = 4;
constexpr int kSpinLimit = 1 << 21;       // bounded mbarrier polling

struct TcArgs {
  const float* A;       // I x C column-major
  float* G;             // I x I, accumulated into (zeroed by the caller)
  long long C;
  int I, N, nM, stages;
  int nk_full, nk;      // full steps, all steps (a ragged tail step last)
  int vec4;             // G rows may be added as float4
  unsigned tmem_cols;
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  for (int it = 0; it < kSpinLimit; ++it) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

// tcgen05 shared-memory matrix descriptor for a K-major tile whose rows are
// 128 bytes, stored as 8-row groups of 1024 bytes with the 128-byte swizzle.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);     // start address
  d |= (uint64_t)1 << 16;                        // leading byte offset (unused here)
  d |= (uint64_t)(1024u >> 4) << 32;             // stride byte offset: one 8-row group
  d |= (uint64_t)1 << 46;                        // descriptor version
  d |= (uint64_t)2 << 61;                        // 128-byte swizzle
  return d;
}

// tcgen05 instruction descriptor, kind::f16: BF16 A and B (both K-major),
// FP32 accumulator, M x N tile.
__host__ __device__ constexpr uint32_t mma_idesc(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__global__ void __launch_bounds__(kThreads, 1) k_gram_tc(TcArgs a) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const long long k_begin = (long long)blockIdx.x * a.nk / gridDim.x;
  const long long k_end = (long long)(blockIdx.x + 1) * a.nk / gridDim.x;
  const int nsteps = (int)(k_end - k_begin);
  if (nsteps <= 0) return;

  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t pad = (1024u - (raw & 1023u)) & 1023u;
  unsigned char* sm = smem_raw + pad;
  const uint32_t sb = raw + pad;
  const int I = a.I, S = a.stages, nM = a.nM;
  const uint32_t bf_bytes = (uint32_t)nM * 128u * 128u;
  const uint32_t st_bytes = (uint32_t)I * kKT * 4u;
  const uint32_t o_bf = 0, o_st = 2 * bf_bytes;
  const uint32_t o_bar = (o_st + (uint32_t)S * st_bytes + 7u) & ~7u;
  const uint32_t bar_full = sb + o_bar;                 // S barriers
  const uint32_t bar_mma = bar_full + 8u * kMaxStages;  // 2 barriers
  uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + o_bar + 8 * kMaxStages + 16);

  // zero both BF16 buffers: rows >= I stay zero for the whole kernel
  for (uint32_t e = tid * 16u; e < 2 * bf_bytes; e += kThreads * 16u)
    *reinterpret_cast<uint4*>(sm + o_bf + e) = make_uint4(0, 0, 0, 0);
  if (tid == 0) {
    for (int s = 0; s < S; ++s)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar_full + 8u * s) : "memory");
    for (int b = 0; b < 2; ++b)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar_mma + 8u * b) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"(a.tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tslot;

  auto issue = [&](int j) {            // bulk copy of step k_begin + j into stage j % S
    const long long k = k_begin + j;
    const uint32_t bar = bar_full + 8u * (uint32_t)(j % S);
    const uint32_t dst = sb + o_st + (uint32_t)(j % S) * st_bytes;
    const float* src = a.A + (size_t)k * kKT * (size_t)I;
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(st_bytes) : "memory");
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
        "l"(src), "r"(st_bytes), "r"(bar)
        : "memory");
  };
  int issued = 0;                      // steps whose copy has been issued
  if (tid == 0) {
    for (int j = 0; j < S && j < nsteps; ++j) {
      if (k_begin + j >= a.nk_full) break;
      issue(j);
      issued = j + 1;
    }
  }

  const uint32_t idesc = mma_idesc(128, a.N);
  bool ok = true;
  int done = 0;                        // steps whose copy has been consumed
  int committed = 0;                   // steps whose MMAs have been committed
  for (int j = 0; j < nsteps; ++j) {
    const long long k = k_begin + j;
    const int s = j % S, b = j & 1;
    const bool tail = k >= a.nk_full;
    bool fail = false;
    if (!tail) fail = !mbar_wait(bar_full + 8u * s, (uint32_t)((j / S) & 1));
    if (!fail && j >= 2) fail = !mbar_wait(bar_mma + 8u * b, (uint32_t)(((j - 2) >> 1) & 1));
    if (__syncthreads_or(fail)) { ok = false; break; }
    // FP32 stage -> BF16, K-major, 128-byte swizzle: element (i, kk) of the
    // step sits at (i/8)*1024 + (i%8)*128 + (((kk/8) ^ (i%8)) * 16) + (kk%8)*2.
    unsigned char* bf = sm + o_bf + (uint32_t)b * bf_bytes;
    const float* stg = reinterpret_cast<const float*>(sm + o_st + (uint32_t)s * st_bytes);
    const int cols = tail ? (int)(a.C - k * kKT) : kKT;
    for (int q = tid; q < I * 8; q += kThreads) {
      const int c = q / I, i = q - c * I;
      float v[8];
      if (!tail) {
#pragma unroll
        for (int u = 0; u < 8; ++u) v[u] = stg[(c * 8 + u) * I + i];
      } else {
#pragma unroll
        for (int u = 0; u < 8; ++u)
          v[u] = (c * 8 + u < cols) ? a.A[((size_t)k * kKT + c * 8 + u) * (size_t)I + i] : 0.f;
      }
      uint4 w;
      __nv_bfloat162 h0 = __floats2bfloat162_rn(v[0], v[1]), h1 = __floats2bfloat162_rn(v[2], v[3]);
      __nv_bfloat162 h2 = __floats2bfloat162_rn(v[4], v[5]), h3 = __floats2bfloat162_rn(v[6], v[7]);
      w.x = *reinterpret_cast<uint32_t*>(&h0); w.y = *reinterpret_cast<uint32_t*>(&h1);
      w.z = *reinterpret_cast<uint32_t*>(&h2); w.w = *reinterpret_cast<uint32_t*>(&h3);
      const int r = i & 7;
      *reinterpret_cast<uint4*>(bf + (i >> 3) * 1024 + r * 128 + ((c ^ r) << 4)) = w;
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (!tail) ++done;
    committed = j + 1;
    if (tid == 0) {
      // stage s is consumed: refill it with step j + S
      if (j + S < nsteps && k + S < a.nk_full) { issue(j + S); issued = j + S + 1; }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t bfa = sb + o_bf + (uint32_t)b * bf_bytes;
      for (int m = 0; m < nM; ++m) {
#pragma unroll
        for (int kk = 0; kk < kKT / 16; ++kk) {
          const uint64_t ad = sw128_desc(bfa + (uint32_t)m * 16384u + kk * 32u);
          const uint64_t bd = sw128_desc(bfa + kk * 32u);
          const uint32_t acc = (j > 0 || kk > 0) ? 1u : 0u;
          asm volatile(
              "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
              "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem + (uint32_t)m * 256u),
              "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
              : "memory");
        }
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       bar_mma + 8u * b)
                   : "memory");
    }
  }
  if (ok) {
    const int jl = nsteps - 1;
    const bool fail = !mbar_wait(bar_mma + 8u * (jl & 1), (uint32_t)((jl >> 1) & 1));
    if (__syncthreads_or(fail)) ok = false;
  }
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (ok) {
    const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
    for (int m = 0; m < nM; ++m) {
      const int i = m * 128 + warp * 32 + lane;
      for (int c0 = 0; c0 < a.N; c0 += 16) {
        uint32_t r[16];
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
            "[%16];"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
              "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
              "=r"(r[15])
            : "r"(tmem + lane_base + (uint32_t)(m * 256 + c0)));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (i < I) {
          float* g = a.G + (size_t)i * I;        // column i of G (= row i by symmetry)
          if (a.vec4) {
#pragma unroll
            for (int u = 0; u < 16; u += 4) {
              const int jj = c0 + u;
              if (jj < I)
                atomicAdd(reinterpret_cast<float4*>(g + jj),
                          make_float4(__uint_as_float(r[u]), __uint_as_float(r[u + 1]),
                                      __uint_as_float(r[u + 2]), __uint_as_float(r[u + 3])));
            }
          } else {
#pragma unroll
            for (int u = 0; u < 16; ++u)
              if (c0 + u < I) atomicAdd(g + c0 + u, __uint_as_float(r[u]));
          }
        }
      }
    }
  } else if (tid == 0) {
    a.G[0] = __int_as_float(0x7fc00000);           // NaN: the solve reports a numeric failure
    // bounded waits for this CTA's copies and MMAs still in flight
    for (int j = done; j < issued; ++j) (void)mbar_wait(bar_full + 8u * (uint32_t)(j % S), (uint32_t)((j / S) & 1));
    if (committed > 0) {
      const int jl = committed - 1;
      (void)mbar_wait(bar_mma + 8u * (jl & 1), (uint32_t)((jl >> 1) & 1));
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(a.tmem_cols) : "memory");
}

size_t tc_smem_bytes(int I, int nM, int S) {
  const size_t bf = (size_t)nM * 128 * 128;
  return 1024 + 2 * bf + (size_t)S * I * kKT * 4 + 8 * kMaxStages + 16 + 16 + 64;
}

}  // namespace

size_t gram_bf16_tc_scratch_bytes(long long I, long long C) { (void)I; (void)C; return 0; }

bool gram_bf16_tc_supported(long long I, const float* T) {
  return I >= 1 && I <= 256 && (reinterpret_cast<uintptr_t>(T) & 15u) == 0;
}

cudaError_t launch_gram_bf16_tc(const float* T, long long I, long long C, float* G, float* scratch,
                                size_t scratch_bytes, cudaStream_t st) {
  (void)scratch; (void)scratch_bytes;
  if (!gram_bf16_tc_supported(I, T) || C < 1) return cudaErrorNotSupported;
  TcArgs a{};
  a.A = T; a.G = G; a.C = C; a.I = (int)I;
  a.nM = I > 128 ? 2 : 1;
  a.N = (int)((I + 15) / 16 * 16);
  if (a.N < 16) a.N = 16;
  unsigned cols = 32;
  while (cols < (unsigned)(a.nM == 2 ? 512 : a.N)) cols <<= 1;
  a.tmem_cols = cols;
  a.nk_full = (int)(C / kKT);
  a.nk = a.nk_full + (C % kKT ? 1 : 0);
  a.vec4 = (I % 4 == 0 && (reinterpret_cast<uintptr_t>(G) & 15u) == 0) ? 1 : 0;
  int dev = 0, lim = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&lim, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  int S = kMaxStages;
  while (S > 2 && tc_smem_bytes(a.I, a.nM, S) > (size_t)lim) --S;
  const size_t smem = tc_smem_bytes(a.I, a.nM, S);
  if (smem > (size_t)lim) return cudaErrorNotSupported;
  a.stages = S;
  int grid = nsm > 0 ? nsm : 1;
  if (grid > a.nk) grid = a.nk;
  cudaError_t e = cudaFuncSetAttribute(k_gram_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_gram_tc<<<grid, kThreads, smem, st>>>(a);
  count_launch();
  return cudaGetLastError();
}

}  // namespace cpdk
