// Uncompression (Sec. 4.1.4), projection of a given starting CPD on the
// truncated bases, and the output normalisation of Fig. "tensorfox-flow"
// (unit columns, weights lambda, sorted descending).
#include "kernels.h"
#include "common.cuh"

namespace cpdk {

// W~^(l) = U^(l) W^(l): U^(l) is I_l x P_l (ld I_l) with its first R~_l columns
// used; W^(l) is R~_l x R (the core solver's stacked layout, dims from the
// device); the result is I_l x R in the original-space stacked layout.
__global__ void k_uncompress(int L, Dims4 dims, int R, const float* U, const int* core_dims,
                             Dims4 P, const float* Wc, float* Wf) {
  int offU = 0, offC = 0, offF = 0;
  for (int l = 0; l < L; ++l) {
    const int I = (int)dims.v[l], rk = core_dims[l];
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < I * R; q += gridDim.x * blockDim.x) {
      const int r = q / I, i = q - r * I;
      float acc = 0.f;
      for (int t = 0; t < rk; ++t) acc = fmaf(U[offU + t * I + i], Wc[offC + r * rk + t], acc);
      Wf[offF + q] = acc;
    }
    offU += I * (int)P.v[l];
    offC += rk * R;
    offF += I * R;
  }
}

// W_core^(l) = U^(l)T W0^(l) for a caller-given starting CPD in the original space.
__global__ void k_project_given(int L, Dims4 dims, int R, const float* U, const int* core_dims,
                                Dims4 P, const float* W0, float* Wc) {
  int offU = 0, offC = 0, offF = 0;
  for (int l = 0; l < L; ++l) {
    const int I = (int)dims.v[l], rk = core_dims[l];
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < rk * R; q += gridDim.x * blockDim.x) {
      const int r = q / rk, t = q - r * rk;
      float acc = 0.f;
      for (int i = 0; i < I; ++i) acc = fmaf(U[offU + t * I + i], W0[offF + r * I + i], acc);
      Wc[offC + q] = acc;
    }
    offU += I * (int)P.v[l];
    offC += rk * R;
    offF += I * R;
  }
}

// Output normalisation: lambda_r = prod_l ||w_r^(l)||, unit columns; the
// largest-|.| entry of every column of modes 1..L-1 is made positive (first
// on ties) and the sign moves to mode L; terms sorted by lambda, descending
// (stable).  One CTA.
__global__ void k_normalize(int L, Dims4 dims, int R, const float* W, float* W_out, float* lam_out) {
  __shared__ double lam[kMaxR];
  __shared__ float inv[kMaxL * kMaxR];
  __shared__ float sgn[kMaxL * kMaxR];
  __shared__ int pos[kMaxR];
  int off[kMaxL + 1]; off[0] = 0;
  for (int l = 0; l < L; ++l) off[l + 1] = off[l] + (int)dims.v[l] * R;
  for (int q = threadIdx.x; q < L * R; q += blockDim.x) {
    const int l = q / R, r = q - l * R, I = (int)dims.v[l];
    const float* w = W + off[l] + r * I;
    double s = 0.0; float best = -1.f; int bi = 0;
    for (int i = 0; i < I; ++i) {
      s += (double)w[i] * (double)w[i];
      if (fabsf(w[i]) > best) { best = fabsf(w[i]); bi = i; }
    }
    const double nr = sqrt(s);
    inv[q] = nr > 0.0 ? (float)(1.0 / nr) : 1.f;
    sgn[q] = (w[bi] < 0.f) ? -1.f : 1.f;
    lam[r] = 0.0;  // filled below
    (void)nr;
  }
  __syncthreads();
  for (int r = threadIdx.x; r < R; r += blockDim.x) {
    double p = 1.0; float last = 1.f;
    for (int l = 0; l < L; ++l) p *= 1.0 / (double)inv[l * R + r];
    for (int l = 0; l < L - 1; ++l) last *= sgn[l * R + r];
    sgn[(L - 1) * R + r] = last;
    lam[r] = p;
  }
  __syncthreads();
  for (int r = threadIdx.x; r < R; r += blockDim.x) {
    int p = 0;
    for (int t = 0; t < R; ++t) p += (lam[t] > lam[r] || (lam[t] == lam[r] && t < r)) ? 1 : 0;
    pos[r] = p;
    lam_out[p] = (float)lam[r];
  }
  __syncthreads();
  for (int l = 0; l < L; ++l) {
    const int I = (int)dims.v[l];
    for (int q = threadIdx.x; q < I * R; q += blockDim.x) {
      const int r = q / I, i = q - r * I;
      W_out[off[l] + pos[r] * I + i] = W[off[l] + q] * inv[l * R + r] * sgn[l * R + r];
    }
  }
}

static Dims4 to_dims4(int L, const long long* d) {
  Dims4 x; for (int l = 0; l < CPD_MAX_ORDER; ++l) x.v[l] = (l < L) ? d[l] : 1; return x;
}
static Dims4 to_dims4i(int L, const int* d) {
  Dims4 x; for (int l = 0; l < CPD_MAX_ORDER; ++l) x.v[l] = (l < L) ? d[l] : 1; return x;
}

cudaError_t launch_uncompress(int L, const long long* dims, int R, const float* U, const int* core_dims,
                              const int* Pdims, const float* Wc, float* Wfull, cudaStream_t st) {
  k_uncompress<<<8, 256, 0, st>>>(L, to_dims4(L, dims), R, U, core_dims, to_dims4i(L, Pdims), Wc, Wfull);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_project_given(int L, const long long* dims, int R, const float* U,
                                 const int* core_dims, const int* Pdims, const float* W0,
                                 float* Wc, cudaStream_t st) {
  k_project_given<<<1, 256, 0, st>>>(L, to_dims4(L, dims), R, U, core_dims, to_dims4i(L, Pdims), W0, Wc);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_normalize(int L, const long long* dims, int R, const float* W, float* W_out,
                             float* lam_out, cudaStream_t st) {
  k_normalize<<<1, 256, 0, st>>>(L, to_dims4(L, dims), R, W, W_out, lam_out);
  count_launch();
  return cudaGetLastError();
}

}  // namespace cpdk
