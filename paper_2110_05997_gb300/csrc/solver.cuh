// CTA-level damped Gauss-Newton building blocks (thesis Sec. 3.5, 4.1.3, 4.7).
//
// Every function here is executed by ALL threads of one CTA; vectors of the
// parameter space (length n = R * sum I_l, stacked vec blocks of Sec. 3.1)
// live in shared memory (or in global memory when they do not fit), R x R
// matrices always in shared memory.  FP32 data, FP64 scalars (CG alpha/beta,
// ||r||^2, F, mu, gain ratio) as the precision contract asks.
#pragma once

#include "common.cuh"

namespace cpdk {

struct Shape {
  int L, R, n, N;
  int d[kMaxL];
  int off[kMaxL + 1];   // start of block l in the stacked vector; off[L] = n
  float dinv[kMaxL];    // 1 / d[l], for index decoding without integer division
};

__host__ __device__ inline void make_shape(Shape& s, int L, const int* d, int R) {
  s.L = L; s.R = R; s.N = 1; s.off[0] = 0;
  for (int l = 0; l < kMaxL; ++l) { s.d[l] = 1; s.dinv[l] = 1.f; }
  for (int l = 0; l < L; ++l) {
    s.d[l] = d[l]; s.dinv[l] = 1.f / (float)d[l];
    s.N *= d[l]; s.off[l + 1] = s.off[l] + R * d[l];
  }
  s.n = s.off[L];
}

// Working buffers of the solver.  Pi2 holds Pi^(a,b) for a != b and, on its
// diagonal blocks (a, a), Pi^(a) (the same Hadamard product over j != a).
struct Bufs {
  const float* S;  float* F;  float* Kb;  float* Bb;          // tensor-sized (core pass)
  float* W; float* G; float* X; float* Rr; float* P; float* Z; float* Tmp;  // n each
  float* gram; float* Pi2; float* Xm; float* Ym;              // L*R*R, L*L*R*R, L*R*R, L*R*R
  float* msq; float* gam; float* sc;                          // L*R each
  double* red;                                                // >= 128 doubles, shared
  float* Minv = nullptr;      // block preconditioner: (Pi^(l) + mu diag gamma^(l))^{-1}, L*R*R
  double* Bd = nullptr;       // its FP64 Cholesky workspace, L*R*R
};

// Floats of the solver's small buffers (R x R Grams and Pi matrices, the
// Hv intermediates, L x R vectors), plus with the block preconditioner its
// inverse blocks and their FP64 workspace (two floats per double).
__host__ __device__ inline size_t small_buf_floats(int L, int R, int blk) {
  const size_t RR = (size_t)R * R;
  auto up = [](size_t x) { return (x + 3) & ~(size_t)3; };
  size_t f = up(L * RR) + up((size_t)L * L * RR) + 2 * up(L * RR) + 3 * up((size_t)L * R);
  if (blk) f += up(L * RR) + 2 * up(L * RR);
  return f;
}

// Carve the small buffers from p (16-byte aligned); returns the end.
__device__ inline float* carve_small(Bufs& b, float* p, int L, int R, int blk) {
  const size_t RR = (size_t)R * R;
  auto up = [](size_t x) { return (x + 3) & ~(size_t)3; };
  b.gram = p; p += up(L * RR);
  b.Pi2 = p; p += up((size_t)L * L * RR);
  b.Xm = p; p += up(L * RR);
  b.Ym = p; p += up(L * RR);
  b.msq = p; p += up((size_t)L * R);
  b.gam = p; p += up((size_t)L * R);
  b.sc = p; p += up((size_t)L * R);
  b.Minv = nullptr; b.Bd = nullptr;
  if (blk) {
    b.Minv = p; p += up(L * RR);
    b.Bd = reinterpret_cast<double*>(p); p += 2 * up(L * RR);
  }
  return p;
}

// Iteration state, kept in shared memory by the single-CTA solvers and in
// global memory between the kernels of the refinement loop.
struct State {
  double mu, F, normS, pred_drop, step, grad_inf, rel_err;
  int k, kglob, cg_total, stop, status, iters;
};

struct DevResult {
  int status, iters, stop, cg_total, kglob, pad0;   // pad0: start taken (1 = learned factors)
  double rel_err, mu, grad_inf, normS;
};

template <int L>
__device__ __forceinline__ void decode_j(const Shape& s, int j, int& l, int& i, int& r) {
  l = 0;
#pragma unroll
  for (int t = 1; t < L; ++t) l += (j >= s.off[t]) ? 1 : 0;
  // q = r d + i with i < d: (q + 0.5) / d is at least 0.5 / d away from an
  // integer, far more than the FP32 rounding of (q + 0.5) * (1/d) for
  // q < R d <= 2^16 d, so the floor is exact
  const int q = j - s.off[l];
  r = __float2int_rd(((float)q + 0.5f) * s.dinv[l]);
  i = q - r * s.d[l];
}

// pi^(l) = W^(l)T W^(l) and the Pi matrices as Hadamard products of the
// other modes' Grams (Sec. 3.5.3, the display defining Pi^(l',l'') and Pi^(l')).
template <int L>
__device__ void grams_pi(const Shape& s, const Bufs& b) {
  const int R = s.R, RR = R * R;
  for (int q = threadIdx.x; q < L * RR; q += blockDim.x) {
    const int l = q / RR, rs = q - l * RR, r = rs / R, c = rs - r * R;
    if (c < r) continue;
    const float* wr = b.W + s.off[l] + r * s.d[l];
    const float* wc = b.W + s.off[l] + c * s.d[l];
    float acc = 0.f;
    for (int i = 0; i < s.d[l]; ++i) acc = fmaf(wr[i], wc[i], acc);
    b.gram[l * RR + r * R + c] = acc;
    b.gram[l * RR + c * R + r] = acc;
  }
  __syncthreads();
  for (int q = threadIdx.x; q < L * L * RR; q += blockDim.x) {
    const int ab = q / RR, rs = q - ab * RR, a = ab / L, bb = ab - a * L;
    float p = 1.f;
#pragma unroll
    for (int j = 0; j < L; ++j)
      if (j != a && j != bb) p *= b.gram[j * RR + rs];
    b.Pi2[q] = p;
  }
  __syncthreads();
}

// Diagonal regulariser D (gamma) and Jacobi preconditioner M of Sec. 4.8:
// gamma_r^(l) = prod_{j!=l}||w_r^(j)|| * max_m max_r' prod_{j!=m}||w_r'^(j)||,
// M_(l,r) = prod_{j!=l}||w_r^(j)||^2 + mu * gamma_r^(l); msq = M^{-1/2}.
template <int L>
__device__ void regularize(const Shape& s, const Bufs& b, double mu) {
  const int R = s.R, RR = R * R;
  float mx = 0.f;
  for (int q = threadIdx.x; q < L * R; q += blockDim.x) {
    const int l = q / R, r = q - l * R;
    float p = 1.f;
#pragma unroll
    for (int j = 0; j < L; ++j)
      if (j != l) p *= sqrtf(fmaxf(b.gram[j * RR + r * R + r], 0.f));
    b.gam[q] = p;
    mx = fmaxf(mx, p);
  }
  const float gmax = block_max(mx, b.red);
  const float muf = (float)mu;
  for (int q = threadIdx.x; q < L * R; q += blockDim.x) {
    const int l = q / R, r = q - l * R;
    const float g = b.gam[q] * gmax;
    const float a = b.Pi2[(l * L + l) * RR + r * R + r];
    b.gam[q] = g;
    const float m = fmaf(muf, g, a);
    b.msq[q] = m > 0.f ? rsqrtf(m) : 1.f;
  }
  __syncthreads();
}

// Block-Jacobi preconditioner (the diagonal blocks of J^T J + mu D; by the
// theorem on J^T J of Sec. 3.5.3 block l is Pi^(l) (x) I_{I_l}, D's block
// diag(gamma^(l)) (x) I): gamma as in regularize(), then per mode the R x R
// matrix B_l = Pi^(l) + mu diag(gamma^(l)) in FP64, its Cholesky factor C
// (one warp per mode, right-looking), C^{-1} by forward substitution (lane j
// column j) and Minv_l = C^{-T} C^{-1} rounded to FP32.  msq is set to 1:
// the block PCG works in the original variables.  R <= 32; needs L warps.
template <int L>
__device__ void regularize_block(const Shape& s, const Bufs& b, double mu) {
  const int R = s.R, RR = R * R;
  float mx = 0.f;
  for (int q = threadIdx.x; q < L * R; q += blockDim.x) {
    const int l = q / R, r = q - l * R;
    float p = 1.f;
#pragma unroll
    for (int j = 0; j < L; ++j)
      if (j != l) p *= sqrtf(fmaxf(b.gram[j * RR + r * R + r], 0.f));
    b.gam[q] = p;
    mx = fmaxf(mx, p);
  }
  const float gmax = block_max(mx, b.red);
  for (int q = threadIdx.x; q < L * R; q += blockDim.x) { b.gam[q] *= gmax; b.msq[q] = 1.f; }
  __syncthreads();
  for (int q = threadIdx.x; q < L * RR; q += blockDim.x) {
    const int l = q / RR, rc = q - l * RR, r = rc / R, c = rc - r * R;
    double v = (double)b.Pi2[(l * L + l) * RR + rc];
    if (r == c) v += mu * (double)b.gam[l * R + r];
    b.Bd[q] = v;
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (warp < L) {
    double* B = b.Bd + warp * RR;
    for (int k = 0; k < R; ++k) {                  // lower Cholesky factor in place
      if (lane == 0) B[k * R + k] = sqrt(fmax(B[k * R + k], 1e-300));
      __syncwarp();
      const double dk = B[k * R + k];
      for (int i = k + 1 + lane; i < R; i += 32) B[i * R + k] /= dk;
      __syncwarp();
      for (int e = lane; e < (R - k - 1) * (R - k - 1); e += 32) {
        const int i = k + 1 + e / (R - k - 1), j = k + 1 + e % (R - k - 1);
        if (j <= i) B[i * R + j] -= B[i * R + k] * B[j * R + k];
      }
      __syncwarp();
    }
    // C^{-1}: column j = lane by forward substitution, kept in the lane until
    // every lane has read C, then written over C's lower triangle
    float* Mi = b.Minv + warp * RR;
    double ci[32];
    const int j = lane;
    if (j < R) {
      for (int i = 0; i < R; ++i) {
        if (i < j) { ci[i] = 0.0; continue; }
        double v = (i == j) ? 1.0 : 0.0;
        for (int t = j; t < i; ++t) v -= B[i * R + t] * ci[t];
        ci[i] = v / B[i * R + i];
      }
    }
    __syncwarp();
    if (j < R)
      for (int i = j; i < R; ++i) B[i * R + j] = ci[i];
    __syncwarp();
    // Minv = C^{-T} C^{-1}: Minv[r][c] = sum_{t >= max(r, c)} Ci[t][r] Ci[t][c]
    for (int e = lane; e < RR; e += 32) {
      const int r = e / R, c = e - r * R;
      double v = 0.0;
      for (int t = (r > c ? r : c); t < R; ++t) v += B[t * R + r] * B[t * R + c];
      Mi[e] = (float)v;
    }
  }
  __syncthreads();
}

// First two phases of Theorem "Hv": Xm^(l) = V^(l)T W^(l) and
// Ym^(l') = sum_{l''!=l'} Pi^(l',l'') * Xm^(l'').
template <int L>
__device__ void hv_xy(const Shape& s, const Bufs& b, const float* V) {
  const int R = s.R, RR = R * R;
  for (int q = threadIdx.x; q < L * RR; q += blockDim.x) {
    const int l = q / RR, rs = q - l * RR, t = rs / R, r = rs - t * R;
    const float* vt = V + s.off[l] + t * s.d[l];
    const float* wr = b.W + s.off[l] + r * s.d[l];
    float acc = 0.f;
    for (int i = 0; i < s.d[l]; ++i) acc = fmaf(vt[i], wr[i], acc);
    b.Xm[q] = acc;
  }
  __syncthreads();
  for (int q = threadIdx.x; q < L * RR; q += blockDim.x) {
    const int a = q / RR, rs = q - a * RR;
    float y = 0.f;
#pragma unroll
    for (int bb = 0; bb < L; ++bb)
      if (bb != a) y = fmaf(b.Pi2[(a * L + bb) * RR + rs], b.Xm[bb * RR + rs], y);
    b.Ym[q] = y;
  }
  __syncthreads();
}

// Last phase of Theorem "Hv" for entry (l, i, r):
// (V^(l) Pi^(l) + W^(l) Ym^(l))[i, r].
template <int L>
__device__ __forceinline__ float hv_entry(const Shape& s, const Bufs& b, const float* V,
                                          int l, int i, int r) {
  const int R = s.R, RR = R * R;
  const float* P1 = b.Pi2 + (l * L + l) * RR;
  const float* Y = b.Ym + l * RR;
  const float* Vl = V + s.off[l] + i;
  const float* Wl = b.W + s.off[l] + i;
  const int d = s.d[l];
  float z = 0.f;
  for (int t = 0; t < R; ++t) {
    z = fmaf(Vl[t * d], P1[t * R + r], z);
    z = fmaf(Wl[t * d], Y[t * R + r], z);
  }
  return z;
}

// The CG stop test ||r||^2 < tol in FP32: the smallest float >= tol (rounded
// up), so that rr < tolf exactly when (double)rr < tol, with one conversion
// per call instead of an FP64 compare per thread and iteration.
__device__ __forceinline__ float stop_threshold_f(double tol) { return __double2float_ru(tol); }

// Algorithm "Conjugate gradient - dGN" (Sec. 4.1.3) on
// B = M^{-1/2}(J^T J + mu D)M^{-1/2}, x0 = 0, r0 = M^{-1/2} A^T b, stop on
// ||r||^2 < tol or maxit; x_hat is left in b.X.  Returns the iterations run.
template <int L>
__device__ int pcg(const Shape& s, const Bufs& b, double mu, int maxit, double tol) {
  const float tolf = stop_threshold_f(tol);
  // The inner products are FP32 block sums; alpha and beta are FP32 quotients
  // of them (the updates use FP32 alpha and beta, and the correctly rounded
  // FP32 quotient is what an FP64 quotient rounded to FP32 gives, barring
  // double rounding), so no warp repeats FP64 scalar work; the stop test
  // compares ||r||^2 with tol in FP64.
  const int n = s.n, R = s.R;
  float v[1] = {0.f};
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    int l, i, r; decode_j<L>(s, j, l, i, r);
    const float m = b.msq[l * R + r];
    const float rv = m * b.G[j];
    b.Rr[j] = rv; b.P[j] = rv; b.X[j] = 0.f; b.Tmp[j] = m * rv;
    v[0] = fmaf(rv, rv, v[0]);
  }
  float rr0[1];
  block_sum_f<1>(v, rr0, b.red);
  float rr = rr0[0];
  int its = 0;
  for (int it = 0; it < maxit; ++it) {
    hv_xy<L>(s, b, b.Tmp);
    float pzf[1] = {0.f};
    const float muf = (float)mu;
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
      int l, i, r; decode_j<L>(s, j, l, i, r);
      const int q = l * R + r;
      const float z = b.msq[q] * (hv_entry<L>(s, b, b.Tmp, l, i, r) + muf * b.gam[q] * b.Tmp[j]);
      b.Z[j] = z;
      pzf[0] = fmaf(b.P[j], z, pzf[0]);
    }
    float pz[1];
    block_sum_f<1>(pzf, pz, b.red);
    if (!(pz[0] > 0.f)) break;
    const float af = rr / pz[0];
    float rnf[1] = {0.f};
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
      b.X[j] = fmaf(af, b.P[j], b.X[j]);
      const float rv = fmaf(-af, b.Z[j], b.Rr[j]);
      b.Rr[j] = rv;
      rnf[0] = fmaf(rv, rv, rnf[0]);
    }
    float rn[1];
    block_sum_f<1>(rnf, rn, b.red);
    const float bf = rr > 0.f ? rn[0] / rr : 0.f;
    rr = rn[0];
    its = it + 1;
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
      int l, i, r; decode_j<L>(s, j, l, i, r);
      const float pv = fmaf(bf, b.P[j], b.Rr[j]);
      b.P[j] = pv;
      b.Tmp[j] = b.msq[l * R + r] * pv;
    }
    __syncthreads();
    if (rr < tolf) break;
  }
  return its;
}

// Preconditioned CG (App. A, the standard form) on (J^T J + mu D) x = A^T b
// with the block-Jacobi preconditioner of regularize_block(): z = M^{-1} r is,
// per mode, Z^(l) = R^(l) Minv_l.  Vectors: x in b.X, r in b.Rr, z in b.Tmp,
// p in b.P, q = (J^T J + mu D) p in b.Z.  Stop on r^T z < tol (the split
// form's ||M^{-1/2} r||^2) or maxit; x is left in b.X in the original
// variables (msq = 1).  Returns the iterations run.
template <int L>
__device__ int pcg_block(const Shape& s, const Bufs& b, double mu, int maxit, double tol) {
  const float tolf = stop_threshold_f(tol);
  const int n = s.n, R = s.R, RR = R * R;
  auto minv = [&](int j, const float* v) {          // (V^(l) Minv_l)[i, r] for entry j = (l, i, r)
    int l, i, r; decode_j<L>(s, j, l, i, r);
    const float* vr = v + s.off[l] + i;
    const float* M = b.Minv + l * RR + r;
    const int d = s.d[l];
    float z = 0.f;
    for (int t = 0; t < R; ++t) z = fmaf(vr[t * d], M[t * R], z);
    return z;
  };
  for (int j = threadIdx.x; j < n; j += blockDim.x) { b.Rr[j] = b.G[j]; b.X[j] = 0.f; }
  __syncthreads();
  float v[1] = {0.f};
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    const float z = minv(j, b.Rr);
    b.Tmp[j] = z; b.P[j] = z;
    v[0] = fmaf(b.Rr[j], z, v[0]);
  }
  float rz0[1];
  block_sum_f<1>(v, rz0, b.red);
  float rz = rz0[0];
  int its = 0;
  const float muf = (float)mu;
  for (int it = 0; it < maxit; ++it) {
    hv_xy<L>(s, b, b.P);
    float pqf[1] = {0.f};
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
      int l, i, r; decode_j<L>(s, j, l, i, r);
      const float q = hv_entry<L>(s, b, b.P, l, i, r) + muf * b.gam[l * R + r] * b.P[j];
      b.Z[j] = q;
      pqf[0] = fmaf(b.P[j], q, pqf[0]);
    }
    float pq[1];
    block_sum_f<1>(pqf, pq, b.red);
    if (!(pq[0] > 0.f)) break;
    const float af = rz / pq[0];
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
      b.X[j] = fmaf(af, b.P[j], b.X[j]);
      b.Rr[j] = fmaf(-af, b.Z[j], b.Rr[j]);
    }
    __syncthreads();
    float rzf[1] = {0.f};
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
      const float z = minv(j, b.Rr);
      b.Tmp[j] = z;
      rzf[0] = fmaf(b.Rr[j], z, rzf[0]);
    }
    float rzn[1];
    block_sum_f<1>(rzf, rzn, b.red);
    const float bf = rz > 0.f ? rzn[0] / rz : 0.f;
    rz = rzn[0];
    its = it + 1;
    for (int j = threadIdx.x; j < n; j += blockDim.x) b.P[j] = fmaf(bf, b.P[j], b.Tmp[j]);
    __syncthreads();
    if (rz < tolf) break;
  }
  return its;
}

// The PCG of pcg() with the last phase of Theorem "Hv" taken row by row: a
// thread forms the R entries (l, i, 0..R-1) of one row of block l together
// (RP >= R accumulators), loading V^(l)[i, t] and W^(l)[i, t] once per t and
// the rows t of Pi^(l) and Ym^(l) as broadcasts, half the shared-memory loads
// of one entry at a time.  Every entry sums in the order of hv_entry, so z is
// the same as in pcg(); the partial sums of p^T z are taken per thread over
// its rows (another order).  For blocks with long columns (the refinement
// step on the full tensor).
template <int L, int RP>
__device__ int pcg_rows(const Shape& s, const Bufs& b, double mu, int maxit, double tol) {
  const float tolf = stop_threshold_f(tol);
  const int n = s.n, R = s.R, RR = R * R;
  int nrows = 0;
#pragma unroll
  for (int l = 0; l < L; ++l) nrows += s.d[l];
  float v[1] = {0.f};
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    int l, i, r; decode_j<L>(s, j, l, i, r);
    const float m = b.msq[l * R + r];
    const float rv = m * b.G[j];
    b.Rr[j] = rv; b.P[j] = rv; b.X[j] = 0.f; b.Tmp[j] = m * rv;
    v[0] = fmaf(rv, rv, v[0]);
  }
  float rr0[1];
  block_sum_f<1>(v, rr0, b.red);
  float rr = rr0[0];
  int its = 0;
  for (int it = 0; it < maxit; ++it) {
    hv_xy<L>(s, b, b.Tmp);
    float pzf[1] = {0.f};
    const float muf = (float)mu;
    for (int row = threadIdx.x; row < nrows; row += blockDim.x) {
      int l = 0, i = row;
      while (l < L - 1 && i >= s.d[l]) { i -= s.d[l]; ++l; }
      const float* P1 = b.Pi2 + (l * L + l) * RR;
      const float* Y = b.Ym + l * RR;
      const int d = s.d[l], base = s.off[l] + i;
      float z[RP];
#pragma unroll
      for (int r = 0; r < RP; ++r) z[r] = 0.f;
      for (int t = 0; t < R; ++t) {
        const float vt = b.Tmp[base + t * d], wt = b.W[base + t * d];
        const float* p1 = P1 + t * R;
        const float* y = Y + t * R;
#pragma unroll
        for (int r = 0; r < RP; ++r) {
          if (r < R) {
            z[r] = fmaf(vt, p1[r], z[r]);
            z[r] = fmaf(wt, y[r], z[r]);
          }
        }
      }
#pragma unroll
      for (int r = 0; r < RP; ++r) {
        if (r < R) {
          const int j = base + r * d, q = l * R + r;
          const float zz = b.msq[q] * (z[r] + muf * b.gam[q] * b.Tmp[j]);
          b.Z[j] = zz;
          pzf[0] = fmaf(b.P[j], zz, pzf[0]);
        }
      }
    }
    float pz[1];
    block_sum_f<1>(pzf, pz, b.red);
    if (!(pz[0] > 0.f)) break;
    const float af = rr / pz[0];
    float rnf[1] = {0.f};
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
      b.X[j] = fmaf(af, b.P[j], b.X[j]);
      const float rv = fmaf(-af, b.Z[j], b.Rr[j]);
      b.Rr[j] = rv;
      rnf[0] = fmaf(rv, rv, rnf[0]);
    }
    float rn[1];
    block_sum_f<1>(rnf, rn, b.red);
    const float bf = rr > 0.f ? rn[0] / rr : 0.f;
    rr = rn[0];
    its = it + 1;
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
      int l, i, r; decode_j<L>(s, j, l, i, r);
      const float pv = fmaf(bf, b.P[j], b.Rr[j]);
      b.P[j] = pv;
      b.Tmp[j] = b.msq[l * R + r] * pv;
    }
    __syncthreads();
    if (rr < tolf) break;
  }
  return its;
}

// The same PCG when every thread owns at most one unknown (n <= blockDim.x):
// x, r, p, the preconditioner entry and the decoded index stay in registers
// and only M^{-1/2} p (the vector J^T J is applied to) goes through shared
// memory.  Same operations in the same order as pcg(), so the same results
// (FP32 scalars as described there).
template <int L>
__device__ int pcg_owned(const Shape& s, const Bufs& b, double mu, int maxit, double tol) {
  const float tolf = stop_threshold_f(tol);
  const int n = s.n, R = s.R;
  const int j = threadIdx.x;
  const bool own = j < n;
  int l = 0, i = 0, r = 0;
  float m = 0.f, mg = 0.f, x = 0.f, rj = 0.f, pj = 0.f;
  const float muf = (float)mu;
  float v[1] = {0.f};
  if (own) {
    decode_j<L>(s, j, l, i, r);
    m = b.msq[l * R + r];
    mg = muf * b.gam[l * R + r];
    rj = m * b.G[j];
    pj = rj;
    b.Tmp[j] = m * rj;
    v[0] = rj * rj;
  }
  float rr0[1];
  block_sum_f<1>(v, rr0, b.red);
  float rr = rr0[0];
  int its = 0;
  for (int it = 0; it < maxit; ++it) {
    hv_xy<L>(s, b, b.Tmp);
    float pzf[1] = {0.f};
    float z = 0.f;
    if (own) {
      z = m * (hv_entry<L>(s, b, b.Tmp, l, i, r) + mg * (m * pj));
      pzf[0] = pj * z;
    }
    float pz[1];
    block_sum_f<1>(pzf, pz, b.red);
    if (!(pz[0] > 0.f)) break;
    const float af = rr / pz[0];
    float rnf[1] = {0.f};
    if (own) {
      x = fmaf(af, pj, x);
      rj = fmaf(-af, z, rj);
      rnf[0] = rj * rj;
    }
    float rn[1];
    block_sum_f<1>(rnf, rn, b.red);
    const float bf = rr > 0.f ? rn[0] / rr : 0.f;
    rr = rn[0];
    its = it + 1;
    if (own) {
      pj = fmaf(bf, pj, rj);
      b.Tmp[j] = m * pj;
    }
    __syncthreads();
    if (rr < tolf) break;
  }
  if (own) b.X[j] = x;
  __syncthreads();
  return its;
}

// Norm-balancing (Sec. 4.1.3 "Updates"): ||w_r^(1)|| = ... = ||w_r^(L)||,
// common value the geometric mean, signs kept.
template <int L>
__device__ void balance(const Shape& s, const Bufs& b) {
  const int R = s.R;
  for (int q = threadIdx.x; q < L * R; q += blockDim.x) {
    const int l = q / R, r = q - l * R;
    const float* w = b.W + s.off[l] + r * s.d[l];
    float acc = 0.f;
    for (int i = 0; i < s.d[l]; ++i) acc = fmaf(w[i], w[i], acc);
    b.sc[q] = sqrtf(acc);
  }
  __syncthreads();
  for (int q = threadIdx.x; q < L * R; q += blockDim.x) {
    const int l = q / R, r = q - l * R;
    float lg = 0.f; bool ok = true;
#pragma unroll
    for (int j = 0; j < L; ++j) {
      const float nj = b.sc[j * R + r];
      ok = ok && (nj > 0.f);
      lg += ok ? logf(nj) : 0.f;
    }
    b.gam[q] = ok ? expf(lg / L) / b.sc[q] : 1.f;   // gam reused as scratch
  }
  __syncthreads();
  for (int j = threadIdx.x; j < s.n; j += blockDim.x) {
    int l, i, r; decode_j<L>(s, j, l, i, r);
    b.W[j] *= b.gam[l * R + r];
  }
  __syncthreads();
}

// After the PCG: x = M^{-1/2} x_hat (into b.X), the predicted decrease
// F - ½||f + Jx||^2 = <g, x> - ½<x, J^T J x> (g = A^T b) and the squared step
// norm ||x||^2 (both in thread 0), then w += x and balancing.
template <int L>
__device__ void finish_step(const Shape& s, const Bufs& b, double& pred_drop, double& step) {
  const int R = s.R;
  for (int j = threadIdx.x; j < s.n; j += blockDim.x) {
    int l, i, r; decode_j<L>(s, j, l, i, r);
    b.X[j] *= b.msq[l * R + r];
  }
  __syncthreads();
  hv_xy<L>(s, b, b.X);
  float vf[3] = {0.f, 0.f, 0.f};
  for (int j = threadIdx.x; j < s.n; j += blockDim.x) {
    int l, i, r; decode_j<L>(s, j, l, i, r);
    const float x = b.X[j];
    vf[0] = fmaf(b.G[j], x, vf[0]);
    vf[1] = fmaf(x, hv_entry<L>(s, b, b.X, l, i, r), vf[1]);
    vf[2] = fmaf(x, x, vf[2]);
  }
  float v[3];
  block_sum_f<3>(vf, v, b.red);
  // FP64 only in thread 0, the callers' bookkeeping thread (the FP64 pipe is
  // too slow for a conversion in every thread); other threads get 0
  pred_drop = 0.0; step = 0.0;
  if (threadIdx.x == 0) {
    pred_drop = (double)v[0] - 0.5 * (double)v[1];
    step = (double)v[2];            // squared here; the caller takes the root
  }
  for (int j = threadIdx.x; j < s.n; j += blockDim.x) b.W[j] += b.X[j];
  __syncthreads();
  balance<L>(s, b);
}

// Residual and gradient of a tensor held by the CTA (Sec. 4.1.3 "Computing the
// residual", "Computing the gradient"): f = S - [[W]], fsq = ||f||^2 (FP32
// block sum) and ginf = ||G||_inf, both returned in thread 0 (0 elsewhere),
// G = A^T b = -grad F, blockwise f_(l) (Khatri-Rao of the other factors).
// The MTTKRPs share two contractions of f: over the last mode (serving modes
// 1..L-1) and over the first mode (serving mode L).
template <int L>
__device__ void core_pass(const Shape& s, const Bufs& b, double& fsq, double& ginf) {
  const int R = s.R, N = s.N;
  const int dl = s.d[L - 1], NL = N / dl, d0 = s.d[0], N0 = N / d0;
  const float* WL = b.W + s.off[L - 1];
  // K[r][e'] = prod_{j<L-1} W_j[i_j, r] over the first L-1 modes
  for (int q = threadIdx.x; q < NL; q += blockDim.x) {
    int idx[kMaxL];
    int rem = q;
#pragma unroll
    for (int j = 0; j < L - 1; ++j) { idx[j] = rem % s.d[j]; rem /= s.d[j]; }
    for (int r = 0; r < R; ++r) {
      float p = 1.f;
#pragma unroll
      for (int j = 0; j < L - 1; ++j) p *= b.W[s.off[j] + r * s.d[j] + idx[j]];
      b.Kb[r * NL + q] = p;
    }
  }
  __syncthreads();
  float accf[1] = {0.f};
  for (int e = threadIdx.x; e < N; e += blockDim.x) {
    const int iL = e / NL, q = e - iL * NL;
    float t = 0.f;
    for (int r = 0; r < R; ++r) t = fmaf(b.Kb[r * NL + q], WL[r * dl + iL], t);
    const float f = b.S[e] - t;
    b.F[e] = f;
    accf[0] = fmaf(f, f, accf[0]);
  }
  float acc[1];
  block_sum_f<1>(accf, acc, b.red);
  fsq = threadIdx.x == 0 ? (double)acc[0] : 0.0;   // valid in thread 0 (see the end)
  // A[r][e'] = sum_{iL} f[e', iL] W_L[iL, r];  B[r][e''] = sum_{i0} f[i0, e''] W_0[i0, r]
  for (int q = threadIdx.x; q < R * NL; q += blockDim.x) {
    const int r = q / NL, e = q - r * NL;
    const float* w = WL + r * dl;
    float a = 0.f;
    for (int iL = 0; iL < dl; ++iL) a = fmaf(b.F[e + NL * iL], w[iL], a);
    b.Kb[q] = a;
  }
  for (int q = threadIdx.x; q < R * N0; q += blockDim.x) {
    const int r = q / N0, e = q - r * N0;
    const float* w = b.W + r * d0;
    const float* f = b.F + d0 * e;
    float a = 0.f;
    for (int i0 = 0; i0 < d0; ++i0) a = fmaf(f[i0], w[i0], a);
    b.Bb[q] = a;
  }
  __syncthreads();
  float gm = 0.f;
  for (int j = threadIdx.x; j < s.n; j += blockDim.x) {
    int l, i, r; decode_j<L>(s, j, l, i, r);
    // source buffer, its strides per mode, and the free modes to sum over
    const float* src;
    int base, fm[2], fstride[2], nf = 0;
    if (l < L - 1) {
      src = b.Kb + r * NL;
      int st = 1; base = 0;
#pragma unroll
      for (int t = 0; t < L - 1; ++t) {
        if (t == l) base = i * st; else { fm[nf] = t; fstride[nf] = st; ++nf; }
        st *= s.d[t];
      }
    } else {
      src = b.Bb + r * N0;
      int st = 1; base = 0;
#pragma unroll
      for (int t = 1; t < L; ++t) {
        if (t == l) base = i * st; else { fm[nf] = t; fstride[nf] = st; ++nf; }
        st *= s.d[t];
      }
    }
    float g = 0.f;
    if (nf == 1) {
      const float* w = b.W + s.off[fm[0]] + r * s.d[fm[0]];
      for (int u = 0; u < s.d[fm[0]]; ++u) g = fmaf(src[base + u * fstride[0]], w[u], g);
    } else {
      const float* w0 = b.W + s.off[fm[0]] + r * s.d[fm[0]];
      const float* w1 = b.W + s.off[fm[1]] + r * s.d[fm[1]];
      for (int u1 = 0; u1 < s.d[fm[1]]; ++u1) {
        float h = 0.f;
        const float* sp = src + base + u1 * fstride[1];
        for (int u0 = 0; u0 < s.d[fm[0]]; ++u0) h = fmaf(sp[u0 * fstride[0]], w0[u0], h);
        g = fmaf(h, w1[u1], g);
      }
    }
    b.G[j] = g;
    gm = fmaxf(gm, fabsf(g));
  }
  const float gmax = block_max(gm, b.red);
  ginf = 0.0;
  if (threadIdx.x == 0) ginf = (double)gmax;
}

// Stop tests of Sec. 4.1.3 in the printed order (reading: windows as printed,
// checked when k is a multiple of c = 1 + ceil(maxiter/10) and k > 2c).
// hist[j] = relative error after iteration j (hist[0] the starting point).
__device__ inline int stop_test(int k, int maxiter, double tol, double e, double step,
                                double ginf, double div_thresh, const double* hist) {
  const int c = 1 + (maxiter + 9) / 10;
  if (e < tol) return CPD_STOP_REL_ERR;
  if (step < tol) return CPD_STOP_STEP;
  if (fabs(hist[k - 1] - e) < tol) return CPD_STOP_IMPROVEMENT;
  if (ginf < tol) return CPD_STOP_GRAD;
  if (k % c == 0 && k > 2 * c) {
    double a1 = 0.0, a2 = 0.0, imp = 0.0;
    for (int j = k - 2 * c; j <= k - c; ++j) a1 += hist[j];
    for (int j = k - c; j <= k; ++j) { a2 += hist[j]; imp += fabs(hist[j - 1] - hist[j]); }
    a1 /= c; a2 /= c; imp /= c;
    if (a1 - a2 < tol) return CPD_STOP_AVG_ERR;
    if (imp < 1e-3 * a2) return CPD_STOP_AVG_IMPROVEMENT;
  }
  if (e > div_thresh) return CPD_STOP_DIVERGENCE;     // max(1, ||S||^2) / (1e-16 + tol)
  if (k == maxiter) return CPD_STOP_MAXITER;
  return CPD_STOP_NONE;
}

// Divergence threshold of stop test 7: max(1, ||S||^2) / (1e-16 + tol), capped
// at a relative error of 1e4 for the FP32 iteration: a trajectory that far
// off has diverged, and the printed bound (>= 1e6 with tol = 1e-6) lies where
// FP32 residuals overflow; the cap keeps the last iterate finite.
constexpr double kFp32DivergenceCap = 1e4;
__device__ inline double divergence_threshold(double normS, double tol) {
  return fmin(fmax(1.0, normS * normS) / (1e-16 + tol), kFp32DivergenceCap);
}

// cg_maxiter(k) for k = 1..len into tab[k] by all threads of the CTA (the FP64
// powers are computed once per solve, in parallel).  Ends with a barrier.
__device__ inline void fill_cg_table(int* tab, int len, uint64_t seed, double ca, double cb) {
  for (int k = threadIdx.x + 1; k <= len; k += blockDim.x) tab[k] = cg_maxiter(k, seed, ca, cb);
  __syncthreads();
}

// Gain ratio (Sec. 3.5.2 / 4.1.3) and the damping update x3 below 0.25,
// /3 above 0.75 (the rule Sec. 4.1.3 settles on), then the FP32 floor mu_min:
// the CG runs in FP32, and with mu far below the FP32 unit roundoff the
// rounding of J^T J v is amplified by ~1/mu along the scaling null space of
// J^T J (Sec. 3.5, "J^T J is singular"), which can overflow the step.
__device__ inline double gain_update(double F_old, double F_new, double pred_drop, double& mu,
                                     double mu_min) {
  const double g = pred_drop > 0.0 ? quick_div(F_old - F_new, pred_drop) : 0.0;
  if (g < 0.25) mu *= 3.0;
  else if (g > 0.75) mu /= 3.0;
  if (mu < mu_min) mu = mu_min;
  return g;
}

__device__ inline void write_trace(double* trace, int cap, int slot, int k, double e, double mu,
                                   double gain, int cg, double step, double ginf, int stage) {
  if (trace == nullptr || slot < 0 || slot >= cap) return;
  double* t = trace + (size_t)slot * CPD_TRACE_FIELDS;
  t[0] = k; t[1] = e; t[2] = mu; t[3] = gain; t[4] = cg; t[5] = step; t[6] = ginf; t[7] = stage;
}

}  // namespace cpdk
