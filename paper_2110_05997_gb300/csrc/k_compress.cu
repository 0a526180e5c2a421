// Compression kernels (thesis Sec. 2.2, 4.1.1, App. A): mode Gram matrices
// T_(l) T_(l)^T on CUDA cores (FP32), their leading eigenpairs (one CTA:
// subspace iteration with CholQR orthonormalisation and a Jacobi
// Rayleigh-Ritz step), the truncation rank of Algorithm "Compression", and
// the mode-l projection Y = T x_l U^T.
#include "kernels.h"
#include "common.cuh"

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
// the upper triangle x one K-split; 256 threads, 4x4 outputs each.
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
  float acc[4][4] = {};
  for (long long qb = q0; qb < q1; qb += kGK) {
    for (int e = threadIdx.x; e < kGK * kGT; e += 256) {
      const int kk = e / kGT, jj = e - kk * kGT;
      const long long q = qb + kk;
      float xa = 0.f, xb = 0.f;
      if (q < q1) {
        const long long i = q % a, k = q / a;
        const long long base = i + a * b * k;
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

cudaError_t launch_gram_simt(const float* T, View3 v, long long a_max, float* G, cudaStream_t st) {
  const int ntile = (int)((v.b + kGT - 1) / kGT);
  const int npair = ntile * (ntile + 1) / 2;
  const long long K = a_max * v.c;
  long long splits = (2 * 152 + npair - 1) / npair;
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

// ---- leading eigenpairs of a Gram matrix ---------------------------------------
constexpr int kEigThreads = 512;
constexpr int kMaxM = 72;            // subspace width cap (P + oversampling)

__host__ __device__ inline int eig_m(int I, int P) {
  int m = P + 6;
  if (m > I) m = I;
  if (m > kMaxM) m = kMaxM;
  return m;
}

size_t eig_work_floats(int I, int P) {
  (void)P;
  return (size_t)I * I + 64;
}

// Cyclic Jacobi with a round-robin parallel ordering on the m x m symmetric H
// (Golub & Van Loan, Algorithm "cyclic Jacobi" with the 2x2 symmetric Schur
// rotation); V accumulates the rotations.  FP64 throughout: H is the small
// Rayleigh-Ritz matrix (m <= P + 6), whose eigenvalues span the signal and the
// noise floor; FP32 rotations lose ~1e-5 of the signal subspace there.
__device__ void jacobi_eig(double* H, double* V, int m, double* red) {
  __shared__ double cs[kMaxM], sn[kMaxM];
  __shared__ int pp[kMaxM / 2 + 1], qq[kMaxM / 2 + 1];
  __shared__ double s_off, s_diag;
  for (int e = threadIdx.x; e < m * m; e += blockDim.x) V[e] = (e % (m + 1) == 0) ? 1.0 : 0.0;
  __syncthreads();
  const int me = m + (m & 1), np = me / 2;
  for (int sweep = 0; sweep < 20; ++sweep) {
    if (threadIdx.x < 32) {
      double o = 0.0, d = 0.0;
      for (int e = threadIdx.x; e < m * m; e += 32) {
        const int r = e / m, c2 = e - r * m;
        if (r == c2) d = fma(H[e], H[e], d); else o = fma(H[e], H[e], o);
      }
#pragma unroll
      for (int k = 16; k > 0; k >>= 1) { o += __shfl_xor_sync(0xffffffffu, o, k); d += __shfl_xor_sync(0xffffffffu, d, k); }
      if (threadIdx.x == 0) { s_off = o; s_diag = d; }
    }
    __syncthreads();
    if (s_off <= 1e-26 * s_diag || s_diag == 0.0) break;
    for (int t = 0; t < me - 1; ++t) {
      if (threadIdx.x < np) {
        const int k = threadIdx.x;
        int p, q;
        if (k == 0) { p = 0; q = (t % (me - 1)) + 1; }
        else { p = ((t + k) % (me - 1)) + 1; q = ((t - k + me - 1) % (me - 1)) + 1; }
        if (p > q) { const int x = p; p = q; q = x; }
        double c = 1.0, s = 0.0;
        if (q < m) {
          // tangent of the Schur rotation in FP32 (it only has to reduce H_pq),
          // then (c, s) renormalised in FP64 by one Newton step for
          // 1/sqrt(c^2 + s^2), so the rotation is orthogonal to FP64 precision.
          const float apq = (float)H[p * m + q];
          if (fabsf(apq) > 1e-35f) {
            const float tau = ((float)H[q * m + q] - (float)H[p * m + p]) / (2.f * apq);
            const float tt = (tau >= 0.f ? 1.f : -1.f) / (fabsf(tau) + sqrtf(fmaf(tau, tau, 1.f)));
            const float c0 = rsqrtf(fmaf(tt, tt, 1.f));
            const double cd = (double)c0, sd = (double)(tt * c0);
            const double nrm = fma(cd, cd, sd * sd);
            const double kf = fma(-0.5, nrm, 1.5);
            c = cd * kf; s = sd * kf;
          }
        } else { p = q = -1; }
        pp[k] = p; qq[k] = q; cs[k] = c; sn[k] = s;
      }
      __syncthreads();
      for (int e = threadIdx.x; e < np * m; e += blockDim.x) {     // rows: J^T H
        const int k = e / m, j = e - k * m, p = pp[k], q = qq[k];
        if (p < 0) continue;
        const double hp = H[p * m + j], hq = H[q * m + j];
        H[p * m + j] = cs[k] * hp - sn[k] * hq;
        H[q * m + j] = sn[k] * hp + cs[k] * hq;
      }
      __syncthreads();
      for (int e = threadIdx.x; e < np * m; e += blockDim.x) {     // columns: H J, V J
        const int k = e / m, i = e - k * m, p = pp[k], q = qq[k];
        if (p < 0) continue;
        const double hp = H[i * m + p], hq = H[i * m + q];
        H[i * m + p] = cs[k] * hp - sn[k] * hq;
        H[i * m + q] = sn[k] * hp + cs[k] * hq;
        const double vp = V[i * m + p], vq = V[i * m + q];
        V[i * m + p] = cs[k] * vp - sn[k] * vq;
        V[i * m + q] = sn[k] * vp + cs[k] * vq;
      }
      __syncthreads();
    }
  }
}

// Z (I x m, column-major, ld I) -> orthonormal Q with span(Q) = span(Z) by
// Cholesky QR on column-normalised Z (FP32; C = Z^T Z has unit diagonal, and
// a pivot below 1e-5 marks a column as dependent on the previous ones).
// Dependent columns are replaced by pseudo-random +-1 vectors and the
// factorisation is repeated.  Warp-parallel dots; Cholesky by warp 0;
// row-wise forward substitution.  Returns false if it did not succeed.
__device__ bool cholqr(float* Z, float* Q, int I, int m, float* Lf, float* Cf, uint64_t seed, int salt) {
  __shared__ int bad;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  for (int attempt = 0; attempt < 6; ++attempt) {
    for (int j = warp; j < m; j += nwarp) {
      float s = 0.f;
      for (int i = lane; i < I; i += 32) s = fmaf(Z[j * I + i], Z[j * I + i], s);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (lane == 0) Cf[j] = s > 0.f ? rsqrtf(s) : 0.f;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < I * m; e += blockDim.x) Z[e] *= Cf[e / I];
    __syncthreads();
    // C = Z^T Z: one warp per upper-triangle entry
    const int ntri = m * (m + 1) / 2;
    for (int t = warp; t < ntri; t += nwarp) {
      int r = 0, rem = t;
      while (rem >= m - r) { rem -= m - r; ++r; }
      const int c = r + rem;
      float s = 0.f;
      for (int i = lane; i < I; i += 32) s = fmaf(Z[r * I + i], Z[c * I + i], s);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (lane == 0) { Lf[r * m + c] = s; Lf[c * m + r] = s; }
    }
    if (threadIdx.x == 0) bad = -1;
    __syncthreads();
    // Cholesky C = L L^T by warp 0, L in the lower triangle of Lf
    if (warp == 0) {
      for (int j = 0; j < m; ++j) {
        float s = 0.f;
        for (int k = lane; k < j; k += 32) s = fmaf(Lf[j * m + k], Lf[j * m + k], s);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        const float piv = Lf[j * m + j] - s;
        __syncwarp();
        if (!(piv > 1e-5f)) { if (lane == 0) bad = j; break; }
        const float ljj = sqrtf(piv);
        const float inv = 1.f / ljj;
        for (int i = j + 1 + lane; i < m; i += 32) {
          float t = Lf[i * m + j];
          for (int k = 0; k < j; ++k) t = fmaf(-Lf[i * m + k], Lf[j * m + k], t);
          Lf[i * m + j] = t * inv;
        }
        __syncwarp();
        if (lane == 0) Lf[j * m + j] = ljj;
        __syncwarp();
      }
    }
    __syncthreads();
    if (bad >= 0) {
      const int from = bad;
      for (int e = threadIdx.x; e < I * (m - from); e += blockDim.x) {
        const int j = from + e / I, i = e % I;
        const uint64_t h = splitmix64(seed, kStreamEig,
                                      ((uint64_t)(salt * 131 + attempt) * 1000003ull + j) * 65536ull + i);
        Z[j * I + i] = (h >> 63) ? 1.f : -1.f;
      }
      __syncthreads();
      continue;
    }
    // Q = Z L^{-T}: row-wise forward substitution L q^T = z^T
    for (int i = threadIdx.x; i < I; i += blockDim.x) {
      float q[kMaxM];
      for (int j = 0; j < m; ++j) {
        float t = Z[j * I + i];
        for (int k = 0; k < j; ++k) t = fmaf(-Lf[j * m + k], q[k], t);
        q[j] = t / Lf[j * m + j];
      }
      for (int j = 0; j < m; ++j) Q[j * I + i] = q[j];
    }
    __syncthreads();
    return true;
  }
  return false;
}

// Z = G Q (G symmetric I x I, column-major; Q I x m): a thread computes four
// columns of one row with independent accumulators.
__device__ void gram_times(const float* G, const float* Q, float* Z, int I, int m) {
  const int mq = (m + 3) >> 2;
  for (int e = threadIdx.x; e < I * mq; e += blockDim.x) {
    const int i = e % I, j0 = (e / I) * 4;
    float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
    const float* q0 = Q + (size_t)j0 * I;
    const bool h1 = j0 + 1 < m, h2 = j0 + 2 < m, h3 = j0 + 3 < m;
    for (int k = 0; k < I; ++k) {
      const float g = G[i + (size_t)I * k];
      a0 = fmaf(g, q0[k], a0);
      if (h1) a1 = fmaf(g, q0[I + k], a1);
      if (h2) a2 = fmaf(g, q0[2 * I + k], a2);
      if (h3) a3 = fmaf(g, q0[3 * I + k], a3);
    }
    Z[(size_t)j0 * I + i] = a0;
    if (h1) Z[(size_t)(j0 + 1) * I + i] = a1;
    if (h2) Z[(size_t)(j0 + 2) * I + i] = a2;
    if (h3) Z[(size_t)(j0 + 3) * I + i] = a3;
  }
  __syncthreads();
}

// H = (Q^T Z + Z^T Q) / 2 (m x m, row-major) by one warp per upper-triangle entry.
__device__ void rayleigh(const float* Q, const float* Z, double* H, int I, int m) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  const int ntri = m * (m + 1) / 2;
  for (int t = warp; t < ntri; t += nwarp) {
    int r = 0, rem = t;
    while (rem >= m - r) { rem -= m - r; ++r; }
    const int c = r + rem;
    float s = 0.f;
    for (int i = lane; i < I; i += 32) s += Q[r * I + i] * Z[c * I + i] + Q[c * I + i] * Z[r * I + i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) { H[r * m + c] = 0.5 * (double)s; H[c * m + r] = 0.5 * (double)s; }
  }
  __syncthreads();
}

__global__ void __launch_bounds__(kEigThreads) k_eig(EigArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int I = a.I, P = a.P, m = eig_m(I, P);
  // layout: red(128 d) | H(m*m d) | V(m*m d) | Lf(m*m) | Cf(m) | Q(I*m) | Z(I*m) | G(I*I if it fits)
  double* red = reinterpret_cast<double*>(smem_raw);
  double* H = red + 128;
  double* V = H + m * m;
  float* Lf = reinterpret_cast<float*>(V + m * m);
  float* Cf = Lf + m * m;
  float* Q = Cf + ((m + 3) & ~3);
  float* Z = Q + (size_t)I * m;
  float* Gs = Z + (size_t)I * m;
  const bool g_in_smem = a.work == nullptr;
  const float* G = a.G;
  if (g_in_smem) {
    for (int e = threadIdx.x; e < I * I; e += blockDim.x) Gs[e] = a.G[e];
    G = Gs;
  }
  __syncthreads();
  __shared__ float lam[kMaxM];
  __shared__ int order[kMaxM];
  if (m == I) {
    // the whole space: Jacobi on G itself (m = I <= P + 6)
    for (int e = threadIdx.x; e < I * I; e += blockDim.x) H[e] = (double)G[e];
    __syncthreads();
    jacobi_eig(H, V, I, red);
    for (int e = threadIdx.x; e < I * m; e += blockDim.x) {
      const int j = e / I, i = e - j * I;
      Q[j * I + i] = (float)V[i * m + j];
    }
  } else {
    // subspace iteration from G * Omega (Omega random +-1)
    for (int e = threadIdx.x; e < I * m; e += blockDim.x) {
      const int j = e / I, i = e - j * I;
      Q[e] = (splitmix64(a.seed, kStreamEig, (uint64_t)j * 1000003ull + i) >> 63) ? 1.f : -1.f;
    }
    __syncthreads();
    gram_times(G, Q, Z, I, m);
    double prev = -1.0;
    for (int it = 0; it < 30; ++it) {
      cholqr(Z, Q, I, m, Lf, Cf, a.seed, it);
      for (int e = threadIdx.x; e < I * m; e += blockDim.x) Z[e] = Q[e];
      __syncthreads();
      cholqr(Z, Q, I, m, Lf, Cf, a.seed, 1000 + it);
      gram_times(G, Q, Z, I, m);
      float vf[1] = {0.f};
      for (int e = threadIdx.x; e < I * m; e += blockDim.x) vf[0] = fmaf(Q[e], Z[e], vf[0]);
      double v[1];
      block_sum<1>(vf, v, red);
      if (prev > 0.0 && fabs(v[0] - prev) <= 1e-6 * fabs(v[0])) break;
      prev = v[0];
    }
    // Rayleigh-Ritz: H = Q^T G Q, eig, U = Q V
    rayleigh(Q, Z, H, I, m);
    jacobi_eig(H, V, m, red);
    for (int e = threadIdx.x; e < I * m; e += blockDim.x) {
      const int j = e / I, i = e - j * I;
      float s = 0.f;
      for (int k = 0; k < m; ++k) s = fmaf(Q[k * I + i], (float)V[k * m + j], s);
      Z[e] = s;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < I * m; e += blockDim.x) Q[e] = Z[e];
  }
  for (int j = threadIdx.x; j < m; j += blockDim.x) lam[j] = (float)H[j * m + j];
  __syncthreads();
  // order by |lambda| descending (stable)
  for (int j = threadIdx.x; j < m; j += blockDim.x) {
    int p = 0;
    const float lj = fabsf(lam[j]);
    for (int t = 0; t < m; ++t) { const float lt = fabsf(lam[t]); p += (lt > lj || (lt == lj && t < j)) ? 1 : 0; }
    order[p] = j;
  }
  __syncthreads();
  // output: top P, signs with the largest-|.| entry positive (first on ties)
  for (int r = threadIdx.x >> 5; r < P; r += blockDim.x >> 5) {
    const int j = order[r];
    const float* q = Q + j * I;
    float best = -1.f; int bi = 0x7fffffff;
    for (int i = threadIdx.x & 31; i < I; i += 32) {
      const float x = fabsf(q[i]);
      if (x > best || (x == best && i < bi)) { best = x; bi = i; }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float ob = __shfl_xor_sync(0xffffffffu, best, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
    }
    const float sg = q[bi] < 0.f ? -1.f : 1.f;
    for (int i = threadIdx.x & 31; i < I; i += 32) a.U[(size_t)r * I + i] = sg * q[i];
    if ((threadIdx.x & 31) == 0) a.sigma[r] = sqrtf(fmaxf(fabsf(lam[j]), 0.f));
  }
  __syncthreads();
  // truncation rank (Algorithm "Compression"): smallest i in 1..P with
  // sum_{r>i} sigma_r^2 / sum_{r<=P} sigma_r^2 < mlsvd_tol / L
  if (threadIdx.x == 0) {
    double tot = 0.0;
    for (int r = 0; r < P; ++r) tot += fabs((double)lam[order[r]]);
    int rk = P;
    if (tot <= 0.0) rk = 1;
    else {
      for (int i = 1; i <= P; ++i) {
        double tail = 0.0;
        for (int r = i; r < P; ++r) tail += fabs((double)lam[order[r]]);
        if (tail / tot < a.mlsvd_tol / a.L) { rk = i; break; }
      }
    }
    *a.rank_out = rk;
  }
}

cudaError_t launch_eig(const EigArgs& a_in, cudaStream_t st) {
  EigArgs a = a_in;
  const int m = eig_m(a.I, a.P);
  size_t base = 128 * sizeof(double) + 2 * (size_t)m * m * sizeof(double) + (size_t)m * m * sizeof(float) +
                (size_t)((m + 3) & ~3) * sizeof(float) + 2 * (size_t)a.I * m * sizeof(float);
  size_t with_g = base + (size_t)a.I * a.I * sizeof(float);
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

cudaError_t launch_project(const float* T, View3 v, long long a_max, const float* U,
                           const int* dev_rank, int rmax, float* Y, cudaStream_t st) {
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
