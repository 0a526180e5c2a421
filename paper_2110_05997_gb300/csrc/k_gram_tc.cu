// BF16 tensor-core Gram of the first-mode unfolding (Sec. 4.1.1 and App. A of
// the thesis: the left singular vectors of T_(1) come from the eigenpairs of
// G = T_(1) T_(1)^T).  A = T_(1) is the column-major I x C matrix whose
// columns are contiguous in T, so a run of 64 columns is one contiguous block
// of 64*I floats.
//
// One CTA per SM takes a contiguous range of 64-column steps:
//   * an issuer thread (warp 8) streams each step's FP32 block into a
//     shared-memory stage with a bulk asynchronous copy completed on an
//     mbarrier (several stages in flight);
//   * eight warps convert the stage to BF16, writing it K-major (row i holds
//     the step's 64 values of row i of A, 128 bytes) in the 128-byte-swizzled
//     layout the tensor core reads;
//   * the issuer issues tcgen05.mma (M = 128, N = ceil16(I), K = 16 each) into
//     FP32 accumulators in tensor memory: D_m += X[128m : 128m+128] X^T for the
//     one or two 128-row tiles m of X, and commits to an mbarrier that frees
//     the BF16 buffer (double-buffered) for the step after next;
//   * finally warps 0-3 read the accumulator rows back (tcgen05.ld) into
//     shared memory, the CTAs of a thread-block cluster sum their partial
//     Grams through distributed shared memory (each CTA a slice of rows), and
//     add the sums into G with vector atomics; G is symmetric, so row i of D
//     goes to the contiguous column i of G.
// Every mbarrier wait is bounded; on a timeout the CTA poisons G with NaN
// (the solve then ends with a numeric status), waits a bounded time for its
// own copies, frees its tensor memory and returns.
#include <cuda_bf16.h>
#include <stdint.h>

#include <map>
#include <mutex>
#include <utility>

#include "kernels.h"
#include "tc_common.cuh"

namespace cpdk {
namespace {

using namespace tc;

constexpr int kKT = 64;                   // unfolding columns per step
constexpr int kConv = 256;                // converting threads (warps 0-7; warps 0-3 read tensor memory back)
constexpr int kIssuer = 256;              // thread issuing the bulk copies and the MMAs (warp 8)
constexpr int kThreads = kConv + 32;
constexpr int kMaxStages = 4;
constexpr int kCluster = 8;               // CTAs whose partial Grams are summed on chip

struct TcArgs {
  const float* A;       // I x C column-major
  float* G;             // I x I, accumulated into (zeroed by the caller)
  long long C;
  int I, N, nM, stages;
  int nk_full, nk;      // full steps, all steps (a ragged tail step last)
  int vec4;             // G rows may be added as float4
  unsigned tmem_cols;
  int* err;             // set to CPD_ERR_TIMEOUT when a pipeline wait runs out (or nullptr)
  long long budget;     // bound of every pipeline wait in SM clock cycles
};

__global__ void __launch_bounds__(kThreads, 1) k_gram_tc(TcArgs a) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const long long k_begin = (long long)blockIdx.x * a.nk / gridDim.x;
  const long long k_end = (long long)(blockIdx.x + 1) * a.nk / gridDim.x;
  const int nsteps = (int)(k_end - k_begin);      // >= 1 when gridDim.x <= nk

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
  int issued = 0;                      // steps whose copy has been issued (issuer thread)
  if (tid == kIssuer) {
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
    if (!tail) fail = !mbar_wait_cycles(bar_full + 8u * s, (uint32_t)((j / S) & 1), a.budget);
    if (!fail && j >= 2) fail = !mbar_wait_cycles(bar_mma + 8u * b, (uint32_t)(((j - 2) >> 1) & 1), a.budget);
    if (__syncthreads_or(fail)) { ok = false; break; }
    // FP32 stage -> BF16, K-major, 128-byte swizzle: element (i, kk) of the
    // step sits at (i/8)*1024 + (i%8)*128 + (((kk/8) ^ (i%8)) * 16) + (kk%8)*2.
    unsigned char* bf = sm + o_bf + (uint32_t)b * bf_bytes;
    const float* stg = reinterpret_cast<const float*>(sm + o_st + (uint32_t)s * st_bytes);
    const int cols = tail ? (int)(a.C - k * kKT) : kKT;
    if (!tail && (I & 3) == 0) {
      // item (g, c): rows 4g..4g+3, values 8c..8c+7 of the step, read as
      // float4 along the rows.  Items go to threads by diagonals of 8 x 8
      // blocks: in quarter-warp t of block b, lane k takes c = k and
      // g = 8b + (k + t) % 8, so that (with I % 4 == 0) the eight lanes of
      // every quarter-warp hit eight different 16-byte bank groups both in
      // the loads and in the swizzled stores.
      const float4* stg4 = reinterpret_cast<const float4*>(stg);
      const int I4 = I >> 2, nb = (I4 + 7) >> 3;
      for (int e = tid; tid < kConv && e < nb * 64; e += kConv) {
        const int k = e & 7, t = (e >> 3) & 7, bb = e >> 6;
        const int c = k, g = 8 * bb + ((k + t) & 7);
        if (g >= I4) continue;
        float4 v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) v[u] = stg4[(c * 8 + u) * I4 + g];
#pragma unroll
        for (int x = 0; x < 4; ++x) {
          const int i = 4 * g + x, r = i & 7;
          float f[8];
#pragma unroll
          for (int u = 0; u < 8; ++u) f[u] = x == 0 ? v[u].x : x == 1 ? v[u].y : x == 2 ? v[u].z : v[u].w;
          *reinterpret_cast<uint4*>(bf + (i >> 3) * 1024 + r * 128 + ((c ^ r) << 4)) = pack_bf16x8(f);
        }
      }
    } else {
      for (int c = 0; c < 8; ++c) {
        for (int i = tid; tid < kConv && i < I; i += kConv) {
          float f[8];
          if (!tail) {
#pragma unroll
            for (int u = 0; u < 8; ++u) f[u] = stg[(c * 8 + u) * I + i];
          } else {
#pragma unroll
            for (int u = 0; u < 8; ++u)
              f[u] = (c * 8 + u < cols) ? a.A[((size_t)k * kKT + c * 8 + u) * (size_t)I + i] : 0.f;
          }
          const int r = i & 7;
          *reinterpret_cast<uint4*>(bf + (i >> 3) * 1024 + r * 128 + ((c ^ r) << 4)) = pack_bf16x8(f);
        }
      }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (!tail) ++done;
    committed = j + 1;
    if (tid == kIssuer) {
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
  if (ok && nsteps > 0) {
    const int jl = nsteps - 1;
    const bool fail = !mbar_wait_cycles(bar_mma + 8u * (jl & 1), (uint32_t)((jl >> 1) & 1), a.budget);
    if (__syncthreads_or(fail)) ok = false;
  }
  const bool has_d = ok && nsteps > 0;             // this CTA holds a valid partial D
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (!ok && tid == kIssuer) {
    a.G[0] = __int_as_float(0x7fc00000);           // NaN: the eigen-solve cannot use G
    if (a.err) atomicExch(a.err, CPD_ERR_TIMEOUT);   // the solve reports the timeout
    // bounded waits for this CTA's copies and MMAs still in flight
    for (int j = done; j < issued; ++j) (void)mbar_wait(bar_full + 8u * (uint32_t)(j % S), (uint32_t)((j / S) & 1));
    if (committed > 0) {
      const int jl = committed - 1;
      (void)mbar_wait(bar_mma + 8u * (jl & 1), (uint32_t)((jl >> 1) & 1));
    }
  }
  // Epilogue, by column passes of at most 128 columns: every CTA of the
  // cluster moves its partial D (rows < I) from tensor memory into its own
  // shared memory (the stages are free now), the cluster synchronises, and
  // CTA r sums rows [r I / cs, (r + 1) I / cs) over the cluster's CTAs through
  // distributed shared memory and adds them into G.  Every CTA takes part in
  // every cluster barrier, whatever its state, so a failed CTA cannot block
  // its peers.
  uint32_t crank, csize;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(crank));
  asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(csize));
  float* dsm = reinterpret_cast<float*>(sm + o_bf);
  const uint32_t dsm_s = sb + o_bf;
  const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
  const int r0 = (int)(crank * (uint32_t)I / csize), r1 = (int)((crank + 1) * (uint32_t)I / csize);
  // widest pass (a multiple of 16 columns) whose I x (W + 4) floats fit below the barriers
  const int wp = min(a.N, (((int)(o_bar / (4u * (uint32_t)I)) - 4) / 16) * 16);
  for (int h = 0; h * wp < a.N; ++h) {
    const int W = min(wp, a.N - h * wp), ld = W + 4;
    if (!has_d) {                                  // contribute zeros
      for (int e = tid; e < I * (W >> 2); e += kThreads) {
        const int i = e / (W >> 2), c = e - i * (W >> 2);
        *reinterpret_cast<float4*>(dsm + (size_t)i * ld + 4 * c) = make_float4(0.f, 0.f, 0.f, 0.f);
      }
    } else if (warp < 4) {
      for (int m = 0; m < nM; ++m) {
        const int i = m * 128 + warp * 32 + lane;
        for (int c0 = 0; c0 < W; c0 += 16) {
          uint32_t r[16];
          asm volatile(
              "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
              "[%16];"
              : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                "=r"(r[15])
              : "r"(tmem + lane_base + (uint32_t)(m * 256 + h * wp + c0)));
          asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
          if (i < I) {
            float4* d = reinterpret_cast<float4*>(dsm + (size_t)i * ld + c0);
#pragma unroll
            for (int u = 0; u < 4; ++u)
              d[u] = make_float4(__uint_as_float(r[4 * u]), __uint_as_float(r[4 * u + 1]),
                                 __uint_as_float(r[4 * u + 2]), __uint_as_float(r[4 * u + 3]));
          }
        }
      }
    }
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
    {
      // two items per thread and iteration: 2 x cs remote loads in flight
      const int w4 = W >> 2, n = (r1 - r0) * w4;
      for (int e0 = tid; e0 < n; e0 += 2 * kThreads) {
        float4 v[2][kCluster];
        int ii[2], jj[2];
#pragma unroll
        for (int x = 0; x < 2; ++x) {
          const int e = e0 + x * kThreads;
          const int row = e / w4;
          ii[x] = r0 + row;
          const int jl = (e - row * w4) * 4;
          jj[x] = (e < n) ? h * wp + jl : I;          // I marks an idle slot
          const uint32_t off = dsm_s + (uint32_t)(((size_t)ii[x] * ld + jl) * 4);
#pragma unroll
          for (int q = 0; q < kCluster; ++q) {
            v[x][q] = make_float4(0.f, 0.f, 0.f, 0.f);
            if (q < (int)csize && jj[x] < I) {
              uint32_t ra;
              asm("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(off), "r"(q));
              asm volatile("ld.shared::cluster.v4.f32 {%0,%1,%2,%3}, [%4];"
                           : "=f"(v[x][q].x), "=f"(v[x][q].y), "=f"(v[x][q].z), "=f"(v[x][q].w)
                           : "r"(ra));
            }
          }
        }
#pragma unroll
        for (int x = 0; x < 2; ++x) {
          const int i = ii[x], j = jj[x];
          if (j >= I) continue;
          float4 acc = v[x][0];
#pragma unroll
          for (int q = 1; q < kCluster; ++q) {
            acc.x += v[x][q].x; acc.y += v[x][q].y; acc.z += v[x][q].z; acc.w += v[x][q].w;
          }
          float* g = a.G + (size_t)i * I + j;        // column i of G (= row i by symmetry)
          if (a.vec4) {
            atomicAdd(reinterpret_cast<float4*>(g), acc);
          } else {
            atomicAdd(g, acc.x);
            if (j + 1 < I) atomicAdd(g + 1, acc.y);
            if (j + 2 < I) atomicAdd(g + 2, acc.z);
            if (j + 3 < I) atomicAdd(g + 3, acc.w);
          }
        }
      }
    }
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(a.tmem_cols) : "memory");
}

// Co-resident clusters of the configuration's cluster size for a dynamic
// shared-memory size, queried once per (device, size, cluster size).
int max_clusters(int dev, size_t smem, int cs, const cudaLaunchConfig_t& cfg) {
  static std::mutex mu;
  static std::map<std::pair<int, std::pair<size_t, int>>, int> cache;
  std::lock_guard<std::mutex> lk(mu);
  const auto key = std::make_pair(dev, std::make_pair(smem, cs));
  auto it = cache.find(key);
  if (it != cache.end()) return it->second;
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, k_gram_tc, &cfg) != cudaSuccess) {
    (void)cudaGetLastError();
    n = 0;
  }
  cache[key] = n;
  return n;
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
                                size_t scratch_bytes, cudaStream_t st, int* err, long long budget) {
  (void)scratch; (void)scratch_bytes;
  if (!gram_bf16_tc_supported(I, T) || C < 1) return cudaErrorNotSupported;
  TcArgs a{};
  a.err = err;
  a.budget = budget > 0 ? budget : (1ll << 31);
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
  cudaError_t e = cudaFuncSetAttribute(k_gram_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  // The cluster size (8, 4 or 2) that keeps the most SMs busy: clusters are
  // placed within a GPC, so clusters of 8 leave the SMs of a GPC beyond a
  // multiple of 8 idle (120 of 152 on GB300).  Larger clusters sum more of
  // the partial Grams on chip, so ties go to the larger size; single-CTA
  // clusters when none fits.  Every CTA must get at least one step.
  cudaLaunchConfig_t cfg{};
  cudaLaunchAttribute attr[1];
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.y = 1; attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr; cfg.numAttrs = 1;
  int cs = 1, grid = (nsm > 0 ? nsm : 1);
  for (int c = kCluster; c >= 2; c >>= 1) {
    if (a.nk < 2 * c) continue;
    attr[0].val.clusterDim.x = c;
    cfg.gridDim = dim3(c * ((nsm + c - 1) / c));
    const int ncl = max_clusters(dev, smem, c, cfg);
    if (ncl * c > (cs == 1 ? 0 : grid)) { cs = c; grid = ncl * c; }
  }
  while (grid > a.nk && grid > cs) grid -= cs;
  if (cs == 1 && grid > a.nk) grid = a.nk;
  attr[0].val.clusterDim.x = cs;
  cfg.gridDim = dim3(grid);
  e = cudaLaunchKernelEx(&cfg, k_gram_tc, a);
  if (e != cudaSuccess) return e;
  count_launch();
  return cudaGetLastError();
}

}  // namespace cpdk
