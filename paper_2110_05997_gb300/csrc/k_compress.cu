// Compression kernels (thesis Sec. 2.2, 4.1.1, App. A): mode Gram matrices
// T_(l) T_(l)^T on CUDA cores (FP32), their leading eigenpairs (one CTA:
// subspace iteration with CholQR orthonormalisation and a Jacobi
// Rayleigh-Ritz step), the truncation rank of Algorithm "Compression", and
// the mode-l projection Y = T x_l U^T.
#include "kernels.h"
#include "common.cuh"
#include "eig_cta.cuh"

namespace cpdk {

__device__ __forceinline__ long long view_a(const View3& v) {
  long long a = v.a_host;
  if (v.dev_ranks)
    for (int j = 0; j < v.nr; ++j) a *= v.dev_ranks[j];
  return a;
}

// ---- Gram on CUDA cores --------------------------------------------------------
// G[j, j'] += sum_q X[q, j] X[q, j'], q = (i, k) over the (a, c) indices of
// the (a, b, c) view, X[q, j] = T[i + a j + a b k].  CTA = one 64x64 tile of
// the upper triangle x one K-split; 256 threads, 4x4 outputs each; the
// K-step's 16 rows q are loaded along the contiguous index.
constexpr int kGT = 64, kGK = 16;

__global__ void __launch_bounds__(256) k_gram_simt(const float* __restrict__ T, View3 v,
                                                   long long chunk, int ntile, float* G) {
  __shared__ float As[kGK][kGT + 4];
  __shared__ float Bs[kGK][kGT + 4];
  // tile pair (ti <= tj) from blockIdx.x
  int pair = blockIdx.x, ti = 0;
  while (pair >= ntile - ti) { pair -= ntile - ti; ++ti; }
  const int tj = ti + pair;
  const long long a = view_a(v), b = v.b, K = a * v.c;
  const long long q0 = (long long)blockIdx.y * chunk;
  const long long q1 = q0 + chunk < K ? q0 + chunk : K;
  if (q0 >= q1) return;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  // offsets i + a b k of the K-step's kGK rows q = (i, k), one division each
  // (by kGK threads) instead of one per loaded element; -1 past the chunk
  __shared__ long long qoff[kGK];
  float acc[4][4] = {};
  for (long long qb = q0; qb < q1; qb += kGK) {
    if (threadIdx.x < kGK) {
      const long long q = qb + threadIdx.x;
      qoff[threadIdx.x] = q < q1 ? (q % a) + a * b * (q / a) : -1;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < kGK * kGT; e += 256) {
      // consecutive threads on the contiguous index: j when a = 1, else q
      // (runs of a consecutive i)
      const int kk = a == 1 ? e / kGT : e % kGK, jj = a == 1 ? e - kk * kGT : e / kGK;
      const long long base = qoff[kk];
      float xa = 0.f, xb = 0.f;
      if (base >= 0) {
        const long long ja = (long long)ti * kGT + jj, jb = (long long)tj * kGT + jj;
        if (ja < b) xa = __ldg(T + base + a * ja);
        if (jb < b) xb = __ldg(T + base + a * jb);
      }
      As[kk][jj] = xa; Bs[kk][jj] = xb;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < kGK; ++kk) {
      const float4 av = *reinterpret_cast<const float4*>(&As[kk][ty * 4]);
      const float4 bv = *reinterpret_cast<const float4*>(&Bs[kk][tx * 4]);
      const float ar[4] = {av.x, av.y, av.z, av.w}, br[4] = {bv.x, bv.y, bv.z, bv.w};
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int w = 0; w < 4; ++w) acc[u][w] = fmaf(ar[u], br[w], acc[u][w]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int w = 0; w < 4; ++w) {
      const long long r = (long long)ti * kGT + ty * 4 + u, c = (long long)tj * kGT + tx * 4 + w;
      if (r < b && c < b) {
        atomicAdd(G + r + b * c, acc[u][w]);
        if (ti != tj) atomicAdd(G + c + b * r, acc[u][w]);
      }
    }
}

// Gram of a mode with b <= 128 columns: one CTA forms the whole b x b Gram
// over a contiguous range of rows q (split K), NT x NT threads with an 8 x 8
// register block each (tile width W = 8 NT >= b): per row q one 16-byte pair
// of loads for the block's rows and one for its columns feed 64 FMAs.  The
// K-step's 16 rows are loaded along the contiguous index (j when a = 1, else
// q), the next step's loads in flight in registers during this step's FMAs
// (double-buffered shared memory); the partial Gram is added into G with
// float4 atomics (b % 4 == 0 and a 16-byte aligned G) or scalar ones.  Both
// triangles are formed directly.
constexpr int kSqK = 16;

template <int NT>
__global__ void __launch_bounds__(NT * NT) k_gram_sq(const float* __restrict__ T, View3 v, long long chunk,
                                                      float* G, int vec4) {
  constexpr int W = 8 * NT, LD = W + 4, NTH = NT * NT;
  constexpr int PER = (kSqK * W + NTH - 1) / NTH;       // elements a thread loads per K-step
  __shared__ __align__(16) float Xs[2][kSqK][LD];
  const unsigned a = (unsigned)view_a(v), b = (unsigned)v.b;
  const unsigned K = a * (unsigned)v.c;                // < 2^32: tensors hold at most 4e9 entries
  const unsigned q0 = (unsigned)((long long)blockIdx.x * chunk);
  const unsigned q1 = (unsigned)min((long long)q0 + chunk, (long long)K);
  if (q0 >= q1) return;
  const int tx = threadIdx.x % NT, ty = threadIdx.x / NT;
  // element e of a K-step: row kk, column jj, along the contiguous index
  auto load = [&](unsigned qb, float (&x)[PER]) {
#pragma unroll
    for (int t = 0; t < PER; ++t) {
      const int e = threadIdx.x + t * NTH;
      const int kk = a == 1 ? e / W : e % kSqK, jj = a == 1 ? e - kk * W : e / kSqK;
      const unsigned q = qb + (unsigned)kk;
      float val = 0.f;
      if (e < kSqK * W && q < q1 && (unsigned)jj < b) {
        const unsigned k = q / a, i = q - k * a;
        val = __ldg(T + (size_t)i + (size_t)a * b * k + (size_t)a * jj);
      }
      x[t] = val;
    }
  };
  auto store = [&](int buf, const float (&x)[PER]) {
#pragma unroll
    for (int t = 0; t < PER; ++t) {
      const int e = threadIdx.x + t * NTH;
      if (e < kSqK * W) {
        const int kk = a == 1 ? e / W : e % kSqK, jj = a == 1 ? e - kk * W : e / kSqK;
        Xs[buf][kk][jj] = x[t];
      }
    }
  };
  float acc[8][8];
#pragma unroll
  for (int u = 0; u < 8; ++u)
#pragma unroll
    for (int w = 0; w < 8; ++w) acc[u][w] = 0.f;
  float x[PER];
  load(q0, x);
  store(0, x);
  __syncthreads();
  int buf = 0;
  for (unsigned qb = q0; qb < q1; qb += kSqK) {
    const bool more = qb + kSqK < q1;
    if (more) load(qb + kSqK, x);                       // in flight during this step's FMAs
#pragma unroll 4
    for (int kk = 0; kk < kSqK; ++kk) {
      const float4 r0 = *reinterpret_cast<const float4*>(&Xs[buf][kk][ty * 8]);
      const float4 r1 = *reinterpret_cast<const float4*>(&Xs[buf][kk][ty * 8 + 4]);
      const float4 c0 = *reinterpret_cast<const float4*>(&Xs[buf][kk][tx * 8]);
      const float4 c1 = *reinterpret_cast<const float4*>(&Xs[buf][kk][tx * 8 + 4]);
      const float rv[8] = {r0.x, r0.y, r0.z, r0.w, r1.x, r1.y, r1.z, r1.w};
      const float cv[8] = {c0.x, c0.y, c0.z, c0.w, c1.x, c1.y, c1.z, c1.w};
#pragma unroll
      for (int u = 0; u < 8; ++u)
#pragma unroll
        for (int w = 0; w < 8; ++w) acc[u][w] = fmaf(rv[u], cv[w], acc[u][w]);
    }
    if (more) store(buf ^ 1, x);
    __syncthreads();
    buf ^= 1;
  }
  const int r0 = ty * 8;
#pragma unroll
  for (int w = 0; w < 8; ++w) {
    const unsigned c = (unsigned)(tx * 8 + w);
    if (c >= b) continue;
    float* g = G + (size_t)b * c;
    if (vec4 && (unsigned)(r0 + 8) <= b) {
      atomicAdd(reinterpret_cast<float4*>(g + r0), make_float4(acc[0][w], acc[1][w], acc[2][w], acc[3][w]));
      atomicAdd(reinterpret_cast<float4*>(g + r0 + 4), make_float4(acc[4][w], acc[5][w], acc[6][w], acc[7][w]));
    } else {
#pragma unroll
      for (int u = 0; u < 8; ++u)
        if ((unsigned)(r0 + u) < b) atomicAdd(g + r0 + u, acc[u][w]);
    }
  }
}

template <int NT>
cudaError_t launch_gram_sq_t(const float* T, View3 v, long long a_max, float* G, cudaStream_t st) {
  const long long K = a_max * v.c;
  long long grid = 2 * 152;                          // two CTAs per SM, each a K range
  const long long maxg = (K + 4 * kSqK - 1) / (4 * kSqK);
  if (grid > maxg) grid = maxg;
  if (grid < 1) grid = 1;
  long long chunk = (K + grid - 1) / grid;
  chunk = (chunk + kSqK - 1) / kSqK * kSqK;
  grid = (K + chunk - 1) / chunk;
  const int vec4 = (v.b % 4 == 0 && (reinterpret_cast<uintptr_t>(G) & 15u) == 0) ? 1 : 0;
  k_gram_sq<NT><<<(unsigned)grid, NT * NT, 0, st>>>(T, v, chunk, G, vec4);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_gram_simt(const float* T, View3 v, long long a_max, float* G, cudaStream_t st) {
  if (v.b <= 32) return launch_gram_sq_t<4>(T, v, a_max, G, st);
  if (v.b <= 56) return launch_gram_sq_t<7>(T, v, a_max, G, st);
  if (v.b <= 80) return launch_gram_sq_t<10>(T, v, a_max, G, st);
  if (v.b <= 104) return launch_gram_sq_t<13>(T, v, a_max, G, st);
  if (v.b <= 128) return launch_gram_sq_t<16>(T, v, a_max, G, st);
  const int ntile = (int)((v.b + kGT - 1) / kGT);
  const int npair = ntile * (ntile + 1) / 2;
  const long long K = a_max * v.c;
  long long splits = (8 * 152 + npair - 1) / npair;     // eight CTAs per SM hide the load latency
  const long long maxs = (K + 255) / 256;
  if (splits > maxs) splits = maxs;
  if (splits < 1) splits = 1;
  if (splits > 65535) splits = 65535;
  long long chunk = (K + splits - 1) / splits;
  chunk = (chunk + kGK - 1) / kGK * kGK;
  k_gram_simt<<<dim3(npair, (unsigned)splits), 256, 0, st>>>(T, v, chunk, ntile, G);
  count_launch();
  return cudaGetLastError();
}

constexpr int kEigThreads = 512;

size_t eig_work_floats(int I, int P) {
  (void)P;
  return (size_t)I * I + 64;
}

__global__ void __launch_bounds__(kEigThreads, 1) k_eig(EigArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  eig_run(a, smem_raw);
}

cudaError_t launch_eig(const EigArgs& a_in, cudaStream_t st) {
  EigArgs a = a_in;
  const size_t base = eig_smem_bytes(a.I, a.P, false);
  const size_t with_g = eig_smem_bytes(a.I, a.P, true);
  int dev = 0, lim = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&lim, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  size_t smem = with_g;
  if (with_g > (size_t)lim) { smem = base; } else { a.work = nullptr; }
  if (smem > (size_t)lim) return cudaErrorInvalidValue;
  if (smem == base && a.work == nullptr) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(k_eig, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_eig<<<1, kEigThreads, smem, st>>>(a);
  count_launch();
  return cudaGetLastError();
}

// ---- projection Y = T x_l U^T --------------------------------------------------
// First mode (a = 1): one warp per column of T_(1) (contiguous b floats), lanes
// over j, a register block of 16 outputs, warp reductions.
__global__ void __launch_bounds__(256) k_project_first(const float* __restrict__ T, long long b,
                                                       long long c, const float* __restrict__ U,
                                                       const int* dev_rank, float* Y) {
  extern __shared__ float Us[];
  const int rk = *dev_rank;
  for (long long e = threadIdx.x; e < b * rk; e += blockDim.x) Us[e] = U[e];
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const long long warp = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const long long nwarps = (long long)gridDim.x * (blockDim.x >> 5);
  for (long long k = warp; k < c; k += nwarps) {
    const float* col = T + b * k;
    for (int r0 = 0; r0 < rk; r0 += 16) {
      float acc[16];
#pragma unroll
      for (int t = 0; t < 16; ++t) acc[t] = 0.f;
      for (long long j = lane; j < b; j += 32) {
        const float x = __ldg(col + j);
#pragma unroll
        for (int t = 0; t < 16; ++t)
          if (r0 + t < rk) acc[t] = fmaf(Us[(r0 + t) * b + j], x, acc[t]);
      }
#pragma unroll
      for (int t = 0; t < 16; ++t) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc[t] += __shfl_xor_sync(0xffffffffu, acc[t], o);
      }
      if (lane < 16 && r0 + lane < rk) {
        float mine = 0.f;
#pragma unroll
        for (int t = 0; t < 16; ++t) mine = (t == lane) ? acc[t] : mine;
        Y[(r0 + lane) + (long long)rk * k] = mine;
      }
    }
  }
}

// First mode (a = 1), tiled: a CTA copies kPC consecutive columns of T_(1)
// (contiguous, b floats each) into shared memory with a row stride of b + 1
// (asynchronous 4-byte copies; odd stride, so the column reads below are free
// of bank conflicts), thread t takes column t and forms its rk outputs from a
// j-major copy of U (RP floats per row j, zero beyond rk; 16-byte broadcast
// loads), summing over j in order.
constexpr int kPC = 128;

template <int RP>
__global__ void __launch_bounds__(kPC) k_project_tiled(const float* __restrict__ T, int b, long long c,
                                                        const float* __restrict__ U, const int* dev_rank,
                                                        float* Y) {
  extern __shared__ __align__(16) float sm[];
  float* Ut = sm;                                   // b x RP, j-major
  float* tile = Ut + (size_t)b * RP;                // kPC x (b + 1)
  const int rk = *dev_rank;                         // <= RP (checked by the launcher's bound)
  const long long k0 = (long long)blockIdx.x * kPC;
  const int nc = (int)((c - k0) < kPC ? (c - k0) : kPC);
  const float* src = T + (size_t)k0 * b;
  for (int col = 0; col < nc; ++col) {
    for (int j = threadIdx.x; j < b; j += kPC) {
      const unsigned dst = (unsigned)__cvta_generic_to_shared(tile + (size_t)col * (b + 1) + j);
      asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(dst), "l"(src + (size_t)col * b + j) : "memory");
    }
  }
  for (int e = threadIdx.x; e < b * RP; e += kPC) {
    const int j = e / RP, p = e - j * RP;
    Ut[e] = p < rk ? U[(size_t)p * b + j] : 0.f;
  }
  asm volatile("cp.async.wait_all;" ::: "memory");
  __syncthreads();
  const int t = threadIdx.x;
  if (t < nc) {
    float acc[RP];
#pragma unroll
    for (int p = 0; p < RP; ++p) acc[p] = 0.f;
    const float* x = tile + (size_t)t * (b + 1);
    const float4* u4 = reinterpret_cast<const float4*>(Ut);
#pragma unroll 4
    for (int j = 0; j < b; ++j) {
      const float xv = x[j];
#pragma unroll
      for (int q = 0; q < RP / 4; ++q) {
        const float4 u = u4[j * (RP / 4) + q];
        acc[4 * q] = fmaf(u.x, xv, acc[4 * q]);
        acc[4 * q + 1] = fmaf(u.y, xv, acc[4 * q + 1]);
        acc[4 * q + 2] = fmaf(u.z, xv, acc[4 * q + 2]);
        acc[4 * q + 3] = fmaf(u.w, xv, acc[4 * q + 3]);
      }
    }
    float* y = Y + (size_t)rk * (k0 + t);
#pragma unroll
    for (int p = 0; p < RP; ++p)
      if (p < rk) y[p] = acc[p];
  }
}

template <int RP>
cudaError_t launch_project_tiled(const float* T, int b, long long c, const float* U, const int* dev_rank,
                                 float* Y, size_t smem, cudaStream_t st) {
  cudaError_t e = cudaFuncSetAttribute(k_project_tiled<RP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_project_tiled<RP><<<(unsigned)((c + kPC - 1) / kPC), kPC, smem, st>>>(T, b, c, U, dev_rank, Y);
  count_launch();
  return cudaGetLastError();
}

// General mode: one warp per (i, k) of the (a, c) indices; lanes stride j,
// 16 outputs per pass, warp reductions.
__global__ void __launch_bounds__(256) k_project_gen(const float* __restrict__ T, View3 v,
                                                     const float* __restrict__ U, const int* dev_rank,
                                                     float* Y) {
  const long long a = view_a(v), b = v.b, c = v.c;
  const int rk = *dev_rank;
  const long long n = a * c;
  const int lane = threadIdx.x & 31;
  const long long warp = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const long long nwarps = (long long)gridDim.x * (blockDim.x >> 5);
  for (long long q = warp; q < n; q += nwarps) {
    const long long i = q % a, k = q / a;
    const float* t = T + i + a * b * k;
    for (int r0 = 0; r0 < rk; r0 += 16) {
      float acc[16];
#pragma unroll
      for (int u = 0; u < 16; ++u) acc[u] = 0.f;
      for (long long j = lane; j < b; j += 32) {
        const float x = __ldg(t + a * j);
#pragma unroll
        for (int u = 0; u < 16; ++u)
          if (r0 + u < rk) acc[u] = fmaf(__ldg(U + (r0 + u) * b + j), x, acc[u]);
      }
#pragma unroll
      for (int u = 0; u < 16; ++u) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc[u] += __shfl_xor_sync(0xffffffffu, acc[u], o);
      }
      if (lane < 16 && r0 + lane < rk) {
        float mine = 0.f;
#pragma unroll
        for (int u = 0; u < 16; ++u) mine = (u == lane) ? acc[u] : mine;
        Y[i + a * (r0 + lane) + a * rk * k] = mine;
      }
    }
  }
}

// Later modes (a > 1): one thread per (i, k), consecutive threads on
// consecutive i, so that the loads T(i, j, k) and the stores Y(i, r, k) of a
// warp are contiguous runs.  A CTA of 256 threads holds Q = 256 / JS pairs
// and splits the j range JS ways (each warp 32 consecutive pairs of one
// split); the JS partial sums of a pair are added in shared memory, split
// order.  U is held j-major (RP floats per j, zero beyond the rank).
template <int RP, int JS>
__global__ void __launch_bounds__(256) k_project_mid(const float* __restrict__ T, View3 v,
                                                     const float* __restrict__ U, const int* dev_rank,
                                                     float* Y) {
  constexpr int Q = 256 / JS;
  extern __shared__ __align__(16) float sm[];
  const long long a = view_a(v), b = v.b, c = v.c;
  float* Ut = sm;                                   // b x RP
  float* part = Ut + (size_t)b * RP;                // JS x RP x Q partial sums
  const int rk = *dev_rank;
  for (long long e = threadIdx.x; e < b * RP; e += 256) {
    const long long j = e / RP;
    const int p = (int)(e - j * RP);
    Ut[e] = p < rk ? U[(size_t)p * b + j] : 0.f;
  }
  __syncthreads();
  const int split = threadIdx.x / Q, qq = threadIdx.x - split * Q;
  const long long n = a * c, q = (long long)blockIdx.x * Q + qq;
  const long long k = q / a, i = q - k * a;
  float acc[RP];
#pragma unroll
  for (int p = 0; p < RP; ++p) acc[p] = 0.f;
  if (q < n) {
    const float* t = T + i + a * b * k;
    const long long j1 = (split + 1) * b / JS;
#pragma unroll 4
    for (long long j = split * b / JS; j < j1; ++j) {
      const float x = __ldg(t + a * j);
      const float4* u4 = reinterpret_cast<const float4*>(Ut + j * RP);
#pragma unroll
      for (int g = 0; g < RP / 4; ++g) {
        const float4 u = u4[g];
        acc[4 * g] = fmaf(u.x, x, acc[4 * g]);
        acc[4 * g + 1] = fmaf(u.y, x, acc[4 * g + 1]);
        acc[4 * g + 2] = fmaf(u.z, x, acc[4 * g + 2]);
        acc[4 * g + 3] = fmaf(u.w, x, acc[4 * g + 3]);
      }
    }
  }
  if constexpr (JS > 1) {
#pragma unroll
    for (int p = 0; p < RP; ++p) part[(split * RP + p) * Q + qq] = acc[p];
    __syncthreads();
    if (split == 0) {
#pragma unroll
      for (int p = 0; p < RP; ++p)
        for (int s = 1; s < JS; ++s) acc[p] += part[(s * RP + p) * Q + qq];
    }
  }
  if (split == 0 && q < n) {
    float* y = Y + i + a * (long long)rk * k;
#pragma unroll
    for (int p = 0; p < RP; ++p)
      if (p < rk) y[a * p] = acc[p];
  }
}

template <int RP>
cudaError_t launch_project_mid_rp(const float* T, View3 v, long long n_max, const float* U, const int* dev_rank,
                                  float* Y, cudaStream_t st) {
  int js = 1;
  while (js < 8 && n_max * js < 152ll * 1024) js *= 2;
  const size_t smem = ((size_t)v.b * RP + (size_t)256 * RP) * sizeof(float);
  const long long q = 256 / js, blocks = (n_max + q - 1) / q;
  if (blocks < 1 || blocks >= (1ll << 31)) return cudaErrorInvalidValue;
  auto run = [&](auto kern) -> cudaError_t {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<(unsigned)blocks, 256, smem, st>>>(T, v, U, dev_rank, Y);
    count_launch();
    return cudaGetLastError();
  };
  if (js == 1) return run(k_project_mid<RP, 1>);
  if (js == 2) return run(k_project_mid<RP, 2>);
  if (js == 4) return run(k_project_mid<RP, 4>);
  return run(k_project_mid<RP, 8>);
}

cudaError_t launch_project(const float* T, View3 v, long long a_max, const float* U,
                           const int* dev_rank, int rmax, float* Y, cudaStream_t st, int* err,
                           long long budget) {
  if (v.a_host == 1 && v.dev_ranks == nullptr && project_tc_supported(v.b, v.c, rmax, T))
    return launch_project_tc(T, v.b, v.c, U, dev_rank, rmax, Y, st, err, budget);
  if (v.a_host == 1 && v.dev_ranks == nullptr && rmax <= 16) {
    const int rp = rmax <= 4 ? 4 : rmax <= 8 ? 8 : rmax <= 12 ? 12 : 16;
    const size_t smem = ((size_t)v.b * rp + (size_t)kPC * (v.b + 1)) * sizeof(float);
    if (smem <= 112 * 1024 + 512 && v.c < (1ll << 40)) {     // two CTAs per SM
      if (rp == 4) return launch_project_tiled<4>(T, (int)v.b, v.c, U, dev_rank, Y, smem, st);
      if (rp == 8) return launch_project_tiled<8>(T, (int)v.b, v.c, U, dev_rank, Y, smem, st);
      if (rp == 12) return launch_project_tiled<12>(T, (int)v.b, v.c, U, dev_rank, Y, smem, st);
      return launch_project_tiled<16>(T, (int)v.b, v.c, U, dev_rank, Y, smem, st);
    }
  }
  if (v.a_host == 1 && v.dev_ranks == nullptr) {
    const size_t smem = (size_t)v.b * rmax * sizeof(float);
    if (smem <= 200 * 1024) {
      cudaError_t e = cudaFuncSetAttribute(k_project_first, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
      long long blocks = (v.c + 7) / 8;
      if (blocks > 4 * 152) blocks = 4 * 152;
      if (blocks < 1) blocks = 1;
      k_project_first<<<(unsigned)blocks, 256, smem, st>>>(T, v.b, v.c, U, dev_rank, Y);
      count_launch();
      return cudaGetLastError();
    }
  }
  if (rmax <= 16 && (size_t)v.b * 16 * sizeof(float) <= 160 * 1024) {
    const long long n_max = a_max * v.c;
    if (rmax <= 4) return launch_project_mid_rp<4>(T, v, n_max, U, dev_rank, Y, st);
    if (rmax <= 8) return launch_project_mid_rp<8>(T, v, n_max, U, dev_rank, Y, st);
    if (rmax <= 12) return launch_project_mid_rp<12>(T, v, n_max, U, dev_rank, Y, st);
    return launch_project_mid_rp<16>(T, v, n_max, U, dev_rank, Y, st);
  }
  long long n = a_max * v.c;             // one warp per (i, k)
  long long blocks = (n + 7) / 8;
  if (blocks > 16 * 152) blocks = 16 * 152;
  if (blocks < 1) blocks = 1;
  k_project_gen<<<(unsigned)blocks, 256, 0, st>>>(T, v, U, dev_rank, Y);
  count_launch();
  return cudaGetLastError();
}

__global__ void k_copy(const float* s, float* d, long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) d[i] = s[i];
}
cudaError_t launch_copy_f32(const float* src, float* dst, long long n, cudaStream_t st) {
  k_copy<<<64, 256, 0, st>>>(src, dst, n);
  count_launch();
  return cudaGetLastError();
}

// BF16 tcgen05 Gram: provided by k_gram_tc.cu.

}  // namespace cpdk
