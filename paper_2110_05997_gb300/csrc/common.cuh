// Device helpers shared by the CPD kernels: reductions, SplitMix64, the
// cg_maxiter draw, and small index utilities.  sm_103a only.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <math.h>

#include "../../include/cpd.h"

namespace cpdk {

constexpr int kMaxL = CPD_MAX_ORDER;
constexpr int kMaxR = CPD_MAX_RANK;

// ---- SplitMix64 (Steele, Lea & Flood, 2014) --------------------------------
// The counter-th output (counter >= 1) of SplitMix64 started at state
// seed + stream * 0xD1B54A32D192ED03.
__host__ __device__ inline uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
__host__ __device__ inline uint64_t splitmix64(uint64_t seed, uint64_t stream, uint64_t counter) {
  return mix64(seed + stream * 0xD1B54A32D192ED03ull + counter * 0x9E3779B97F4A7C15ull);
}
constexpr uint64_t kStreamCG = 1;
constexpr uint64_t kStreamInit = 2;
constexpr uint64_t kStreamEig = 3;

// cg_maxiter of dGN iteration k (Sec. 4.1.3): uniform integer in
// [1 + ceil(k^a), 2 + ceil(k^b)], inclusive; ceilings of x - 1e-9 so that
// powers that are integers in exact arithmetic do not round up.
__host__ __device__ inline int cg_maxiter(int k, uint64_t seed, double a, double b) {
  int lo = 1 + (int)ceil(pow((double)k, a) - 1e-9);
  int hi = 2 + (int)ceil(pow((double)k, b) - 1e-9);
  if (hi < lo) hi = lo;
  uint64_t w = (uint64_t)(hi - lo + 1);
  return lo + (int)(splitmix64(seed, kStreamCG, (uint64_t)k) % w);
}

// N(0,1) entry j of the stacked starting vector (Box-Muller on outputs 2j+1, 2j+2).
__device__ inline double normal_draw(uint64_t seed, uint64_t j) {
  double u1 = (double)((splitmix64(seed, kStreamInit, 2 * j + 1) >> 11) + 1) * 0x1.0p-53;
  double u2 = (double)(splitmix64(seed, kStreamInit, 2 * j + 2) >> 11) * 0x1.0p-53;
  return sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
}

// ---- block reductions (every thread receives the result) --------------------
// FP32 partial sums per thread, across the warp (shuffles) and across the
// warps (every thread adds the <= 32 per-warp partials from shared memory);
// the result is returned as FP64 for the scalar recurrences.  No FP64
// instruction is issued: on sm_103a the FP64 pipe runs at ~1/64 of FP32 and
// a single FP64 add per warp costs more than the whole FP32 reduction.
// `red` must hold 32 * NV floats (it is declared as doubles by the callers).
// Contains two barriers.
template <int NV>
__device__ inline void block_sum(const float (&in)[NV], double (&out)[NV], double* red) {
  float v[NV];
#pragma unroll
  for (int i = 0; i < NV; ++i) {
    v[i] = in[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[i] += __shfl_xor_sync(0xffffffffu, v[i], o);
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  float* r = reinterpret_cast<float*>(red);
  __syncthreads();
  if (lane == 0)
#pragma unroll
    for (int i = 0; i < NV; ++i) r[i * 32 + wid] = v[i];
  __syncthreads();
#pragma unroll
  for (int i = 0; i < NV; ++i) {
    float s = lane < nw ? r[i * 32 + lane] : 0.f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    out[i] = (double)s;
  }
}

// As block_sum, the totals left in FP32 (no FP64 conversion in every warp).
template <int NV>
__device__ inline void block_sum_f(const float (&in)[NV], float (&out)[NV], double* red) {
  float v[NV];
#pragma unroll
  for (int i = 0; i < NV; ++i) {
    v[i] = in[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[i] += __shfl_xor_sync(0xffffffffu, v[i], o);
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  float* r = reinterpret_cast<float*>(red);
  __syncthreads();
  if (lane == 0)
#pragma unroll
    for (int i = 0; i < NV; ++i) r[i * 32 + wid] = v[i];
  __syncthreads();
#pragma unroll
  for (int i = 0; i < NV; ++i) {
    float s = lane < nw ? r[i * 32 + lane] : 0.f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    out[i] = s;
  }
}

// a / b and sqrt(x) to ~FP64 accuracy from an FP32 estimate and one step of
// Newton's method in FP64 (2-3 FP64 FMAs instead of a full FP64 division /
// square root sequence).
//   quotient: q1 = q0 + (a - q0 b) / b with the residual a - q0 b formed by one
//     FMA and the division by b taken with the FP32 reciprocal; the relative
//     error of q0 (~2^-22) is squared, giving ~2^-46;
//   square root: s1 = s0 + (x - s0^2) / (2 s0), Newton's (Heron's) step for
//     s^2 = x from the FP32 root s0, again squaring its relative error.
// Valid while a, b, x and the results are within the FP32 exponent range.
__host__ __device__ __forceinline__ double quick_div(double a, double b) {
  const float rb = 1.f / (float)b;
  const double q0 = (double)((float)a * rb);
  return fma(fma(-q0, b, a), (double)rb, q0);
}
__host__ __device__ __forceinline__ double quick_sqrt(double x) {
  if (!(x > 0.0)) return x == 0.0 ? 0.0 : sqrt(x);
  const float s0 = sqrtf((float)x);
  const double s = (double)s0;
  return fma(fma(-s, s, x), 0.5 / s, s);
}

__device__ inline float block_max(float v, double* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  float* r = reinterpret_cast<float*>(red);
  __syncthreads();
  if (lane == 0) r[wid] = v;
  __syncthreads();
  float m = lane < nw ? r[lane] : r[0];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  return m;
}

// argmax of (value, index) with ties to the smaller index; every thread gets it.
__device__ inline void block_argmax(float& v, int& idx, double* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    float ov = __shfl_xor_sync(0xffffffffu, v, o);
    int oi = __shfl_xor_sync(0xffffffffu, idx, o);
    if (ov > v || (ov == v && oi < idx)) { v = ov; idx = oi; }
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  __syncthreads();
  if (lane == 0) { red[2 * wid] = v; red[2 * wid + 1] = (double)idx; }
  __syncthreads();
  v = (float)red[0]; idx = (int)red[1];
  for (int w = 1; w < nw; ++w) {
    float ov = (float)red[2 * w]; int oi = (int)red[2 * w + 1];
    if (ov > v || (ov == v && oi < idx)) { v = ov; idx = oi; }
  }
}

__device__ inline bool finite_d(double x) { return isfinite(x); }

// a / b (quick_div) computed once per warp (lane 0) and broadcast.
__device__ __forceinline__ double warp_div(double a, double b) {
  double q = 0.0;
  if ((threadIdx.x & 31) == 0) q = quick_div(a, b);
  return __shfl_sync(0xffffffffu, q, 0);
}

}  // namespace cpdk
