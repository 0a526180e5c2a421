// CTA-level leading eigenpairs of a mode Gram matrix (App. A of the thesis:
// left singular vectors of an unfolding from the eigenpairs of its Gram
// matrix), and the truncation rank of Algorithm "Compression" (Sec. 4.1.1).
// Subspace iteration (FP32 products, Cholesky-QR orthonormalisation) and a
// Rayleigh-Ritz step whose small symmetric eigenproblem is solved by cyclic
// Jacobi in FP64.  Shared by the single-tensor eigen kernel and the batched
// solver.
#pragma once

#include "kernels.h"
#include "common.cuh"

namespace cpdk {

// ---- leading eigenpairs of a Gram matrix ---------------------------------------
constexpr int kMaxM = 72;            // subspace width cap (P + oversampling)

__host__ __device__ inline int eig_m(int I, int P) {
  int m = P + 6;
  if (m > I) m = I;
  if (m > kMaxM) m = kMaxM;
  return m;
}


// Cyclic Jacobi with a round-robin parallel ordering on the m x m symmetric H
// (Golub & Van Loan, Algorithm "cyclic Jacobi" with the 2x2 symmetric Schur
// rotation); V accumulates the rotations.  FP64 throughout: H is the small
// Rayleigh-Ritz matrix (m <= P + 6), whose eigenvalues span the signal and the
// noise floor; FP32 rotations lose ~1e-5 of the signal subspace there.
static __device__ void jacobi_eig(double* H, double* V, int m, double* red) {
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
static __device__ bool cholqr(float* Z, float* Q, int I, int m, float* Lf, float* Cf, uint64_t seed, int salt) {
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
static __device__ void gram_times(const float* G, const float* Q, float* Z, int I, int m) {
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
static __device__ void rayleigh(const float* Q, const float* Z, double* H, int I, int m) {
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


__host__ __device__ inline size_t eig_smem_bytes(int I, int P, bool with_g) {
  const int m = eig_m(I, P);
  size_t base = 128 * sizeof(double) + 2 * (size_t)m * m * sizeof(double) + (size_t)m * m * sizeof(float) +
                (size_t)((m + 3) & ~3) * sizeof(float) + 2 * (size_t)I * m * sizeof(float);
  return with_g ? base + (size_t)I * I * sizeof(float) : base;
}

// Leading P eigenpairs of the symmetric I x I Gram matrix a.G (column-major),
// by the whole CTA, with `smem_raw` as shared-memory workspace of
// eig_smem_bytes(I, P, g_in_smem) bytes.  a.work == nullptr means: copy G into
// that workspace first (it fits); otherwise G is read where it is.
static __device__ void eig_run(const EigArgs& a, unsigned char* smem_raw) {
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

}  // namespace cpdk
