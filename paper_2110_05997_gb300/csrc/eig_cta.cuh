// CTA-level leading eigenpairs of a mode Gram matrix (App. A of the thesis:
// left singular vectors of an unfolding from the eigenpairs of its Gram
// matrix), and the truncation rank of Algorithm "Compression" (Sec. 4.1.1).
// Subspace iteration (FP32 products, Cholesky-QR orthonormalisation) and a
// Rayleigh-Ritz step whose small symmetric eigenproblem is solved by cyclic
// Jacobi (FP32 sweeps, then an FP64 polish).  Shared by the single-tensor
// eigen kernel and the batched solver.
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


// The 2x2 symmetric Schur rotation (c, s) that zeroes h_pq (Golub & Van Loan,
// "symmetric Schur decomposition"); identity (returns false) when q is the
// padding index or |h_pq| <= skip * (|h_pp| + |h_qq|).  The tangent is formed
// in FP32 (the rotation only has to reduce h_pq) from the difference
// h_qq - h_pp taken in the working precision, and (c, s) is renormalised by
// one Newton step for 1/sqrt(c^2 + s^2) in the working precision, so that the
// rotation is orthogonal to that precision.
template <typename Real>
__device__ __forceinline__ bool jacobi_rot(const Real* H, int m, int p, int q, float skip, Real& c, Real& s) {
  c = 1; s = 0;
  if (q >= m) return false;
  const Real hpq = H[p * m + q], hpp = H[p * m + p], hqq = H[q * m + q];
  const float apq = (float)hpq;
  if (!(fabsf(apq) > 1e-35f) || !(fabs(hpq) > (Real)skip * (fabs(hpp) + fabs(hqq)))) return false;
  const float tau = __fdividef((float)(hqq - hpp), 2.f * apq);
  float tt;
  if (fabsf(tau) > 1e18f) {
    tt = __fdividef(0.5f, tau);
  } else {
    const float r = fmaf(tau, tau, 1.f);
    tt = copysignf(__fdividef(1.f, fabsf(tau) + r * rsqrtf(r)), tau);
  }
  const float c0 = rsqrtf(fmaf(tt, tt, 1.f)), s0 = tt * c0;
  if (sizeof(Real) == sizeof(double)) {
    const double cd = (double)c0, sd = (double)s0;
    const double kf = fma(-0.5, fma(cd, cd, sd * sd), 1.5);
    c = (Real)(cd * kf); s = (Real)(sd * kf);
  } else {
    const float kf = fmaf(-0.5f, fmaf(c0, c0, s0 * s0), 1.5f);
    c = (Real)(c0 * kf); s = (Real)(s0 * kf);
  }
  return true;
}

// Pair k of round t of the round-robin parallel ordering on me = m + (m & 1)
// indices (Golub & Van Loan, "parallel Jacobi"): index 0 stays, the others
// rotate; p < q, q == m is the padding index of odd m.
__device__ __forceinline__ void jacobi_pair(int t, int k, int nr, int& p, int& q) {
  p = 0; q = t + 1;
  if (k != 0) {
    int x = t + k, y = t - k + nr;
    if (x >= nr) x -= nr;
    if (y >= nr) y -= nr;
    p = x + 1; q = y + 1;
  }
  if (p > q) { const int x = p; p = q; q = x; }
}

// One cyclic sweep of Jacobi with the round-robin parallel ordering on the
// m x m symmetric H (row-major); V accumulates the rotations.  Per round: one
// thread per pair forms its rotation (the identity (1, 0) when skipped);
// then the round's m/2 disjoint rotations J are applied as H <- J^T H J into
// the other buffer, one 2x2 block (pair k1 rows, pair k2 columns) per work
// item, and V <- V J in place, one (row, pair) per item.  The work items
// recompute the pairs' indices instead of reading them, so that their loads
// of H and of the rotations issue together.  H and Hn swap roles after each
// round.
template <typename Real>
static __device__ void jacobi_sweep(Real*& H, Real*& Hn, Real* V, int m, float skip) {
  __shared__ Real r_c[kMaxM / 2], r_s[kMaxM / 2];
  const int me = m + (m & 1), np = me / 2, nr = me - 1;
  const int nblk = np * np;
  // integer quotients of the work-item index by np and m through FP32
  // reciprocals: exact here, as (e + 0.5) / np stays 0.5 / np away from an
  // integer and e < 2^12
  const float inv_np = 1.f / (float)np, inv_m = 1.f / (float)m;
  for (int t = 0; t < nr; ++t) {
    if (threadIdx.x < np) {
      const int k = threadIdx.x;
      int p, q;
      jacobi_pair(t, k, nr, p, q);
      Real c, s;
      jacobi_rot(H, m, p, q, skip, c, s);
      r_c[k] = c; r_s[k] = s;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < nblk + np * m; e += blockDim.x) {
      if (e < nblk) {
        const int k1 = __float2int_rd(((float)e + 0.5f) * inv_np), k2 = e - k1 * np;
        int p1, q1, p2, q2;
        jacobi_pair(t, k1, nr, p1, q1);
        jacobi_pair(t, k2, nr, p2, q2);
        const bool r1 = q1 < m, r2 = q2 < m;
        const Real c1 = r_c[k1], s1 = r_s[k1], c2 = r_c[k2], s2 = r_s[k2];
        const Real a = H[p1 * m + p2];
        const Real b = r2 ? H[p1 * m + q2] : (Real)0;
        const Real cc = r1 ? H[q1 * m + p2] : (Real)0;
        const Real d = (r1 && r2) ? H[q1 * m + q2] : (Real)0;
        // rows (pair k1), then columns (pair k2)
        const Real o00 = c1 * a - s1 * cc, o01 = c1 * b - s1 * d;
        const Real o10 = s1 * a + c1 * cc, o11 = s1 * b + c1 * d;
        Hn[p1 * m + p2] = c2 * o00 - s2 * o01;
        if (r2) Hn[p1 * m + q2] = s2 * o00 + c2 * o01;
        if (r1) Hn[q1 * m + p2] = c2 * o10 - s2 * o11;
        if (r1 && r2) Hn[q1 * m + q2] = s2 * o10 + c2 * o11;
      } else {
        const int f = e - nblk, k = __float2int_rd(((float)f + 0.5f) * inv_m), i = f - k * m;
        int p, q;
        jacobi_pair(t, k, nr, p, q);
        if (q >= m) continue;
        const Real c = r_c[k], s = r_s[k];
        const Real vp = V[i * m + p], vq = V[i * m + q];
        V[i * m + p] = c * vp - s * vq;
        V[i * m + q] = s * vp + c * vq;
      }
    }
    __syncthreads();
    Real* x = H; H = Hn; Hn = x;
  }
}

// Off-diagonal and diagonal squared masses of H (warp 0, FP32 partial sums of
// the working-precision squares), broadcast through shared memory.
template <typename Real>
static __device__ void jacobi_masses(const Real* H, int m, float& off, float& diag) {
  __shared__ float s_off, s_diag;
  if (threadIdx.x < 32) {
    float o = 0.f, d = 0.f;
    for (int e = threadIdx.x; e < m * m; e += 32) {
      const int r = e / m, c2 = e - r * m;
      const float h = (float)H[e];
      if (r == c2) d = fmaf(h, h, d); else o = fmaf(h, h, o);
    }
#pragma unroll
    for (int k = 16; k > 0; k >>= 1) { o += __shfl_xor_sync(0xffffffffu, o, k); d += __shfl_xor_sync(0xffffffffu, d, k); }
    if (threadIdx.x == 0) { s_off = o; s_diag = d; }
  }
  __syncthreads();
  off = s_off; diag = s_diag;
  __syncthreads();
}

// Y = op(A) * B for m x m row-major FP64 matrices, op(A) = A or A^T; when
// `ns` is set, Y = 1.5 I - 0.5 A^T B instead (the Newton-Schulz factor).
static __device__ void small_gemm(const double* A, bool at, const double* B, double* Y, int m, bool ns) {
  for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
    const int i = e / m, j = e - i * m;
    double s0 = 0.0, s1 = 0.0;
    int k = 0;
    for (; k + 1 < m; k += 2) {
      s0 = fma(at ? A[k * m + i] : A[i * m + k], B[k * m + j], s0);
      s1 = fma(at ? A[(k + 1) * m + i] : A[i * m + k + 1], B[(k + 1) * m + j], s1);
    }
    if (k < m) s0 = fma(at ? A[k * m + i] : A[i * m + k], B[k * m + j], s0);
    const double s = s0 + s1;
    Y[e] = ns ? ((i == j ? 1.5 : 0.0) - 0.5 * s) : s;
  }
  __syncthreads();
}

// Eigen-decomposition H = V diag(h) V^T of the m x m symmetric Rayleigh-Ritz
// (or small Gram) matrix, to FP64 accuracy.  H's eigenvalues span the signal
// and the noise floor, so an FP32-only decomposition loses ~1e-5 of the signal
// subspace; FP64 rotations throughout are bound by the FP64 pipe.  Three
// stages instead:
//   1. cyclic Jacobi in FP32 on a copy of H until the off-diagonal mass stops
//      falling (it ends at FP32 rounding level, ~1e-7 relative);
//   2. the FP32 eigenvectors V0 made orthonormal to FP64 precision by two
//      Newton-Schulz steps X <- X (3I - X^T X) / 2 (Higham, "Functions of
//      Matrices", the Newton-Schulz iteration for the polar factor), and
//      H <- V1^T H V1, now diagonal up to ~1e-7 relative;
//   3. FP64 cyclic Jacobi sweeps on that H accumulating into V1; rotations
//      below FP64 resolution are skipped, so the sweeps after the first only
//      work inside clusters of close eigenvalues.
// W1, W2: m x m FP64 scratch each.  On return H is diagonal (the eigenvalues)
// and the columns of V are the eigenvectors.
static __device__ void jacobi_eig(double* H, double* V, int m, double* W1, double* W2, bool polish = true) {
  float* Hf = reinterpret_cast<float*>(W1);
  float* Vf = Hf + m * m;
  float* Hf2 = reinterpret_cast<float*>(W2);
  for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
    Hf[e] = (float)H[e];
    Vf[e] = (e % (m + 1) == 0) ? 1.f : 0.f;
  }
  __syncthreads();
  float off, diag, prev = 3.4e38f;
  for (int sweep = 0; sweep < 16; ++sweep) {
    jacobi_masses(Hf, m, off, diag);
    if (!(off > 1e-13f * diag) || diag == 0.f) break;
    if (off <= 1e-9f * diag && off > 0.25f * prev) break;      // at FP32 rounding level
    prev = off;
    jacobi_sweep<float>(Hf, Hf2, Vf, m, 0.f);
  }
  for (int e = threadIdx.x; e < m * m; e += blockDim.x) V[e] = (double)Vf[e];
  if (!polish) {
    // the FP32 decomposition is as accurate as the (BF16-rounded) Gram
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) H[e] = (double)Hf[e];
    __syncthreads();
    return;
  }
  __syncthreads();
  small_gemm(V, true, V, W2, m, true);          // W2 = (3I - V0^T V0) / 2
  small_gemm(V, false, W2, W1, m, false);       // W1 = V0 W2
  small_gemm(W1, true, W1, W2, m, true);        // second step: W2 = (3I - W1^T W1) / 2
  small_gemm(W1, false, W2, V, m, false);       // V = V1 = W1 W2
  small_gemm(H, false, V, W2, m, false);        // W2 = H V1
  small_gemm(V, true, W2, H, m, false);         // H = V1^T H V1
  double* Hc = H;
  double* Hn = W1;
  for (int sweep = 0; sweep < 12; ++sweep) {
    __shared__ double s_o, s_d;
    if (threadIdx.x < 32) {
      // masses in FP64 (the stop test is far below FP32 rounding)
      double o = 0.0, d = 0.0;
      for (int e = threadIdx.x; e < m * m; e += 32) {
        const int r = e / m, c2 = e - r * m;
        if (r == c2) d = fma(Hc[e], Hc[e], d); else o = fma(Hc[e], Hc[e], o);
      }
#pragma unroll
      for (int k = 16; k > 0; k >>= 1) { o += __shfl_xor_sync(0xffffffffu, o, k); d += __shfl_xor_sync(0xffffffffu, d, k); }
      if (threadIdx.x == 0) { s_o = o; s_d = d; }
    }
    __syncthreads();
    const double o = s_o, d = s_d;
    __syncthreads();
    if (o <= 1e-26 * d || d == 0.0) break;
    jacobi_sweep<double>(Hc, Hn, V, m, 1e-17f);
  }
  if (Hc != H) {
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) H[e] = Hc[e];
    __syncthreads();
  }
}

// These routines run a handful of times per call, so their code is kept
// compact (loops, not full unrolls: straight-line code executed once is bound
// by instruction fetch), with eight-wide register batches so that the loads
// of a batch are in flight together.

// Q = Z L^{-T} (Q[:, j] of row i from L q^T = z^T, forward substitution), one
// thread per row, the row's unknowns read back from Q; dinv[j] = 1 / L_jj.
static __device__ void fwd_subst(const float* Z, float* Q, int I, int m, const float* Lf, const float* dinv) {
  for (int i = threadIdx.x; i < I; i += blockDim.x) {
    for (int j = 0; j < m; ++j) {
      float t = Z[j * I + i];
      for (int k0 = 0; k0 < j; k0 += 8) {
        float lv[8], qv[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const bool in = k0 + u < j;
          lv[u] = in ? Lf[j * m + k0 + u] : 0.f;
          qv[u] = in ? Q[(k0 + u) * I + i] : 0.f;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) t = fmaf(-lv[u], qv[u], t);
      }
      Q[j * I + i] = t * dinv[j];
    }
  }
}

// Right-looking Cholesky C = L L^T of the symmetric m x m matrix in Lf
// (row-major) by one warp in shared memory: step j takes the pivot, scales
// column j below it (one row per lane) and updates the trailing lower
// triangle, lane i row i.  On exit the lower triangle of Lf holds L and
// dinv[j] = 1 / L_jj; `bad` gets the first column whose pivot is not above
// 1e-5 (the factor is then incomplete).
static __device__ void chol_warp(float* Lf, float* dinv, int m, int lane, int& bad) {
  for (int j = 0; j < m; ++j) {
    const float piv = Lf[j * m + j];
    if (!(piv > 1e-5f)) {
      if (lane == 0) bad = j;
      return;
    }
    const float ljj = sqrtf(piv), inv = 1.f / ljj;
    for (int i = j + 1 + lane; i < m; i += 32) Lf[i * m + j] *= inv;
    __syncwarp();
    if (lane == 0) { Lf[j * m + j] = ljj; dinv[j] = inv; }
    for (int i = j + 1 + lane; i < m; i += 32) {
      const float lij = Lf[i * m + j];
      for (int k0 = j + 1; k0 <= i; k0 += 8) {
        float lk[8], cv[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const bool in = k0 + u <= i;
          lk[u] = in ? Lf[(k0 + u) * m + j] : 0.f;
          cv[u] = in ? Lf[i * m + k0 + u] : 0.f;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u)
          if (k0 + u <= i) Lf[i * m + k0 + u] = fmaf(-lij, lk[u], cv[u]);
      }
    }
    __syncwarp();
  }
}

// Z (I x m, column-major, ld I) -> orthonormal Q with span(Q) = span(Z) by
// Cholesky QR on column-normalised Z (FP32; C = Z^T Z has unit diagonal, and
// a pivot below 1e-5 marks a column as dependent on the previous ones).
// Dependent columns are replaced by pseudo-random +-1 vectors and the
// factorisation is repeated.  Warp-parallel dots; Cholesky by warp 0 in
// shared memory; row-wise forward substitution.  Cf: m floats of scratch
// (the column scales, then 1 / L_jj).  Returns false if it did not succeed.
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
    // C = Z^T Z: one thread per upper-triangle entry (r, c), four partial
    // sums.  For even I the thread starts its pass over the rows at row c
    // (cyclically), so that a warp's 32 consecutive columns c fall in
    // distinct banks; for odd I the column stride already does.
    const int ntri = m * (m + 1) / 2;
    for (int t = threadIdx.x; t < ntri; t += blockDim.x) {
      int r = 0, rem = t;
      while (rem >= m - r) { rem -= m - r; ++r; }
      const int c = r + rem;
      const float* zr = Z + r * I;
      const float* zc = Z + c * I;
      int i = (I & 1) ? 0 : c % I;
      float acc[4] = {0.f, 0.f, 0.f, 0.f};
      int q = 0;
      for (; q + 4 <= I; q += 4) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          acc[u] = fmaf(zr[i], zc[i], acc[u]);
          if (++i == I) i = 0;
        }
      }
      for (; q < I; ++q) {
        acc[0] = fmaf(zr[i], zc[i], acc[0]);
        if (++i == I) i = 0;
      }
      const float s = (acc[0] + acc[1]) + (acc[2] + acc[3]);
      Lf[r * m + c] = s;
      Lf[c * m + r] = s;
    }
    if (threadIdx.x == 0) bad = -1;
    __syncthreads();
    // Cholesky C = L L^T by warp 0, L in the lower triangle of Lf, 1 / L_jj in Cf
    if (warp == 0) chol_warp(Lf, Cf, m, lane, bad);
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
    fwd_subst(Z, Q, I, m, Lf, Cf);
    __syncthreads();
    return true;
  }
  return false;
}

// Z = G Q (G symmetric I x I, column-major; Q I x m, column-major).
// Shared-memory wavefronts, not FMAs, bound this product, so each thread
// takes a 4 x 4 tile of Z: per k one 16-byte load of G's rows 4b..4b+3 and
// one 16-byte broadcast load of Q's row k from the k-major copy Qt (stride
// mp = m rounded up to 4, zero-padded) feed 16 FMAs.  Needs I % 4 == 0, a
// 16-byte aligned G and TILED (the batched solver's small Grams keep the
// scalar form and its registers); otherwise a thread computes four columns
// of two rows (i and i + ceil(I/2)) with scalar loads.  Both forms sum over
// k in the same order, so they give the same Z.
template <bool TILED>
static __device__ void gram_times(const float* G, const float* Q, float* Z, float* Qt, int I, int m) {
  const int mp = (m + 3) & ~3, mq = mp >> 2;
  if (TILED && (I & 3) == 0 && (reinterpret_cast<uintptr_t>(G) & 15) == 0) {
    for (int e = threadIdx.x; e < I * mp; e += blockDim.x) {
      const int k = e / mp, j = e - k * mp;
      Qt[e] = j < m ? Q[(size_t)j * I + k] : 0.f;
    }
    __syncthreads();
    const int Ib = I >> 2;
    const float4* G4 = reinterpret_cast<const float4*>(G);
    const float4* Q4 = reinterpret_cast<const float4*>(Qt);
    for (int e = threadIdx.x; e < Ib * mq; e += blockDim.x) {
      const int bi = e % Ib, c = e / Ib;
      float acc[4][4];
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = 0.f;
#pragma unroll 4
      for (int k = 0; k < I; ++k) {
        const float4 g = G4[(size_t)k * Ib + bi];
        const float4 q = Q4[(size_t)k * mq + c];
        const float gv[4] = {g.x, g.y, g.z, g.w}, qv[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int v = 0; v < 4; ++v) acc[u][v] = fmaf(gv[u], qv[v], acc[u][v]);
      }
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        const int j = 4 * c + v;
        if (j < m) {
#pragma unroll
          for (int u = 0; u < 4; ++u) Z[(size_t)j * I + 4 * bi + u] = acc[u][v];
        }
      }
    }
    __syncthreads();
    return;
  }
  const int Ih = (I + 1) >> 1;
  for (int e = threadIdx.x; e < Ih * mq; e += blockDim.x) {
    const int i = e % Ih, j0 = (e / Ih) * 4, i2 = i + Ih;
    const bool two = i2 < I;
    const int i2c = two ? i2 : i;
    float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f, b0 = 0.f, b1 = 0.f, b2 = 0.f, b3 = 0.f;
    const float* q0 = Q + (size_t)j0 * I;
    const bool h1 = j0 + 1 < m, h2 = j0 + 2 < m, h3 = j0 + 3 < m;
    const float* q1 = h1 ? q0 + I : q0;
    const float* q2 = h2 ? q0 + 2 * I : q0;
    const float* q3 = h3 ? q0 + 3 * I : q0;
#pragma unroll 4
    for (int k = 0; k < I; ++k) {
      const float g = G[i + (size_t)I * k], g2 = G[i2c + (size_t)I * k];
      const float x0 = q0[k], x1 = q1[k], x2 = q2[k], x3 = q3[k];
      a0 = fmaf(g, x0, a0); a1 = fmaf(g, x1, a1); a2 = fmaf(g, x2, a2); a3 = fmaf(g, x3, a3);
      b0 = fmaf(g2, x0, b0); b1 = fmaf(g2, x1, b1); b2 = fmaf(g2, x2, b2); b3 = fmaf(g2, x3, b3);
    }
    Z[(size_t)j0 * I + i] = a0;
    if (h1) Z[(size_t)(j0 + 1) * I + i] = a1;
    if (h2) Z[(size_t)(j0 + 2) * I + i] = a2;
    if (h3) Z[(size_t)(j0 + 3) * I + i] = a3;
    if (two) {
      Z[(size_t)j0 * I + i2] = b0;
      if (h1) Z[(size_t)(j0 + 1) * I + i2] = b1;
      if (h2) Z[(size_t)(j0 + 2) * I + i2] = b2;
      if (h3) Z[(size_t)(j0 + 3) * I + i2] = b3;
    }
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


// tiled: room for the k-major copy of Q that the tiled G Q product reads
// (the eigen kernel, MMAX > 32; the batched solver's eig_run<32> has none).
__host__ __device__ inline size_t eig_smem_bytes(int I, int P, bool with_g, bool tiled = true) {
  const int m = eig_m(I, P);
  const size_t mp = (size_t)((m + 3) & ~3);
  size_t base = 128 * sizeof(double) + 4 * (size_t)m * m * sizeof(double) +
                (((size_t)m * m + 3) & ~(size_t)3) * sizeof(float) + mp * sizeof(float) +
                (tiled ? (size_t)I * mp * sizeof(float) : 0) + 2 * (size_t)I * m * sizeof(float);
  return with_g ? base + (size_t)I * I * sizeof(float) : base;
}

// Leading P eigenpairs of the symmetric I x I Gram matrix a.G (column-major),
// by the whole CTA, with `smem_raw` as shared-memory workspace of
// eig_smem_bytes(I, P, g_in_smem) bytes.  a.work == nullptr means: copy G into
// that workspace first (it fits); otherwise G is read where it is.
// MMAX: the largest subspace width the caller needs (72 for the eigen
// kernel, 32 for the batched solver's modes of at most 64).
template <int MMAX = kMaxM>
static __device__ void eig_run(const EigArgs& a, unsigned char* smem_raw) {
  const int I = a.I, P = a.P, m = eig_m(I, P);
  // layout: red(128 d) | H, V, W1, W2 (m*m d each) | Lf(m*m, to 4) | Cf(m, to 4) | Qt(I*mp)
  //         | Q(I*m) | Z(I*m) | G(I*I if it fits); Lf, Qt and G start on 16 bytes
  const int mp = (m + 3) & ~3;
  double* red = reinterpret_cast<double*>(smem_raw);
  double* H = red + 128;
  double* V = H + m * m;
  double* W1 = V + m * m;
  double* W2 = W1 + m * m;
  float* Lf = reinterpret_cast<float*>(W2 + m * m);
  float* Cf = Lf + ((m * m + 3) & ~3);
  float* Qt = Cf + mp;
  float* Q = Qt + (MMAX > 32 ? (size_t)I * mp : 0);
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
    jacobi_eig(H, V, I, W1, W2, a.fp32_only == 0);
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
    gram_times<(MMAX > 32)>(G, Q, Z, Qt, I, m);
    double prev = -1.0;
    for (int it = 0; it < 30; ++it) {
      cholqr(Z, Q, I, m, Lf, Cf, a.seed, it);
      for (int e = threadIdx.x; e < I * m; e += blockDim.x) Z[e] = Q[e];
      __syncthreads();
      cholqr(Z, Q, I, m, Lf, Cf, a.seed, 1000 + it);
      gram_times<(MMAX > 32)>(G, Q, Z, Qt, I, m);
      float vf[1] = {0.f};
      for (int e = threadIdx.x; e < I * m; e += blockDim.x) vf[0] = fmaf(Q[e], Z[e], vf[0]);
      double v[1];
      block_sum<1>(vf, v, red);
      if (prev > 0.0 && fabs(v[0] - prev) <= 1e-6 * fabs(v[0])) break;
      prev = v[0];
    }
    // Rayleigh-Ritz: H = Q^T G Q, eig, U = Q V
    rayleigh(Q, Z, H, I, m);
    jacobi_eig(H, V, m, W1, W2, a.fp32_only == 0);
    // U = Q V with V rounded to FP32 once (W1 is free again): a conversion
    // from FP64 inside every FMA would run on the narrow FP64 pipe
    float* Vs = reinterpret_cast<float*>(W1);
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) Vs[e] = (float)V[e];
    __syncthreads();
    for (int e = threadIdx.x; e < I * m; e += blockDim.x) {
      const int j = e / I, i = e - j * I;
      float s = 0.f;
      for (int k = 0; k < m; ++k) s = fmaf(Q[k * I + i], Vs[k * m + j], s);
      Z[e] = s;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < I * m; e += blockDim.x) Q[e] = Z[e];
  }
  for (int j = threadIdx.x; j < m; j += blockDim.x) lam[j] = (float)H[j * m + j];
  __syncthreads();
  // order by |lambda| descending (stable); a NaN ranks below every number, so
  // that the positions are a permutation whatever the input (a poisoned Gram)
  auto key = [](float x) { const float v = fabsf(x); return v == v ? v : -1.f; };
  for (int j = threadIdx.x; j < m; j += blockDim.x) {
    int p = 0;
    const float lj = key(lam[j]);
    for (int t = 0; t < m; ++t) { const float lt = key(lam[t]); p += (lt > lj || (lt == lj && t < j)) ? 1 : 0; }
    order[p] = j;
  }
  __syncthreads();
  // output: top P, signs with the largest-|.| entry positive (first on ties)
  for (int r = threadIdx.x >> 5; r < P; r += blockDim.x >> 5) {
    const int j = order[r];
    const float* q = Q + j * I;
    float best = -1.f; int bi = 0x7fffffff;
    for (int i = threadIdx.x & 31; i < I; i += 32) {
      float x = fabsf(q[i]);
      if (!(x == x)) x = -0.5f;                 // a NaN still yields a valid index
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
  // (the tails by one backward pass: tail_i = tail_{i+1} + sigma_{i+1}^2)
  if (threadIdx.x == 0) {
    double* tail = red;                         // P + 1 <= 128 doubles, free here
    tail[P] = 0.0;
    for (int r = P - 1; r >= 0; --r) tail[r] = tail[r + 1] + fabs((double)lam[order[r]]);
    const double tot = tail[0];
    int rk = P;
    if (tot <= 0.0) rk = 1;
    else {
      const double lim = tot * (a.mlsvd_tol / a.L);
      for (int i = 1; i <= P; ++i)
        if (tail[i] < lim) { rk = i; break; }
    }
    *a.rank_out = rk;
  }
}

}  // namespace cpdk
