// The pass over T of a refinement iteration (dGN on the full tensor after
// uncompression): residual e = T - [[W]], ||e||^2 (and ||T||^2) in FP64, and
// the MTTKRP of e for every mode (= -grad F; the Sec. 4.1.3 formulas applied
// to T).  Included by one translation unit per tensor order.
#pragma once

#include "kernels.h"
#include "solver.cuh"

namespace cpdk {

// Mode-1 fibers (I1 contiguous floats) in batches of kNB.  Thread i owns row
// i1 = i of every fiber: with kr_r = prod_{l>=2} W_l[i_l, r] (shared, float4
// broadcast loads) it forms t~ = sum_r W1[i1, r] kr_r (W1 row in registers),
// e = t - t~, ||e||^2, and accumulates G1[i1, :] += e kr in registers for the
// whole kernel.  Then Q = E^T W1 per fiber (float4 broadcast of W1 rows) and
// G_l[i_l, r] += q_r prod_{j>=2, j!=l} W_j[i_j, r] for l >= 2 (shared atomics).
constexpr int kNB = 32;
static_assert(kNB == 32, "the Q product maps fibres of a batch to the lanes of a warp");


template <int L, int RMAX, int SLOTS>
__global__ void __launch_bounds__(256) k_refine_pass(RefinePassArgs a) {
  if (a.done && *a.done) return;
  extern __shared__ __align__(16) float sm[];
  const int R = a.R, R4 = (R + 3) & ~3;
  const int I1 = (int)a.dims[0];
  int d[kMaxL], off[kMaxL + 1];
  off[0] = 0;
#pragma unroll
  for (int l = 0; l < kMaxL; ++l) d[l] = (l < L) ? (int)a.dims[l] : 1;
#pragma unroll
  for (int l = 0; l < L; ++l) off[l + 1] = off[l] + d[l] * R;
  const int n = off[L];
  long long nf = 1;
#pragma unroll
  for (int l = 1; l < L; ++l) nf *= d[l];
  // shared: Ws (n) | W1r (I1 x R4, row-major) | Gs (n) | E (I1 x (kNB+1)) | KR (kNB x R4)
  //         | Qs (2 x kNB x R4, double-buffered)
  float* Ws = sm;
  float* W1r = Ws + ((n + 3) & ~3);
  float* Gs = W1r + (size_t)I1 * R4;
  float* E = Gs + ((n + 3) & ~3);
  float* KR = E + (((size_t)I1 * (kNB + 1) + 3) & ~(size_t)3);
  float* Qs2 = KR + kNB * R4;
#pragma unroll 8
  for (int j = threadIdx.x; j < n; j += blockDim.x) { Ws[j] = a.W[j]; Gs[j] = 0.f; }
#pragma unroll 4
  for (int j = threadIdx.x; j < I1 * R; j += blockDim.x) {      // W1 (I1 x R, column-major) -> rows
    const int r = j / I1, i = j - r * I1;
    W1r[i * R4 + r] = a.W[j];
  }
  for (int j = threadIdx.x; j < I1 * (R4 - R); j += blockDim.x) {
    const int r = R + j / I1, i = j % I1;
    W1r[i * R4 + r] = 0.f;
  }
  __syncthreads();
  // thread owns rows i1 = threadIdx.x + s * blockDim.x, s < SLOTS
  float w[SLOTS][RMAX], g1[SLOTS][RMAX];
#pragma unroll
  for (int sl = 0; sl < SLOTS; ++sl) {
    const int i = threadIdx.x + sl * blockDim.x;
#pragma unroll
    for (int r = 0; r < RMAX; ++r) { w[sl][r] = (i < I1 && r < R) ? W1r[i * R4 + r] : 0.f; g1[sl][r] = 0.f; }
  }
  double esq = 0.0, tsq = 0.0;
  const long long nbatch = (nf + kNB - 1) / kNB;
  constexpr int kHalf = kNB / 2;
  float xa[kHalf], xb[kHalf];                 // register double buffers (one row per thread)
  if constexpr (SLOTS == 1) {
    const long long b0 = blockIdx.x;
    const int i = threadIdx.x;
    if (b0 < nbatch && i < I1) {
      const long long fb = b0 * kNB;
      const int nb0 = (int)((nf - fb) < kNB ? (nf - fb) : kNB);
      const float* tb = a.T + (size_t)I1 * fb + i;
#pragma unroll
      for (int u = 0; u < kHalf; ++u) xa[u] = (u < nb0) ? __ldg(tb + (size_t)I1 * u) : 0.f;
    }
  }
  int par = 0;
  for (long long bt = blockIdx.x; bt < nbatch; bt += gridDim.x, par ^= 1) {
    const long long f0 = bt * kNB;
    const int nb = (int)((nf - f0) < kNB ? (nf - f0) : kNB);
    float* Qs = Qs2 + par * kNB * R4;          // read by this batch's scatter only
    for (int e = threadIdx.x; e < kNB * R4; e += blockDim.x) {
      const int f = e / R4, r = e - f * R4;
      float p = 0.f;
      if (f < nb && r < R) {
        unsigned rem = (unsigned)(f0 + f);     // fibre index < 2^31 (checked at launch)
        p = 1.f;
#pragma unroll
        for (int l = 1; l < L; ++l) {
          const unsigned il = rem % (unsigned)d[l];
          rem /= (unsigned)d[l];
          p *= Ws[off[l] + r * d[l] + (int)il];
        }
      }
      KR[e] = p;
      Qs[e] = 0.f;
    }
    __syncthreads();
    // one entry (row i, fibre f): t~ = W1[i,:] . kr_f, e = t - t~, ||e||^2,
    // ||t||^2, G1[i,:] += e kr_f, and e into E for the Q product
    auto entry = [&](int sl, int i, int f, float x, float& esqf, float& tsqf) {
      const float4* k4 = reinterpret_cast<const float4*>(KR + f * R4);
      float kr[RMAX];
#pragma unroll
      for (int q = 0; q < RMAX / 4; ++q) {
        if (4 * q < R) {
          const float4 v = k4[q];
          kr[4 * q] = v.x; kr[4 * q + 1] = v.y; kr[4 * q + 2] = v.z; kr[4 * q + 3] = v.w;
        } else {
          kr[4 * q] = kr[4 * q + 1] = kr[4 * q + 2] = kr[4 * q + 3] = 0.f;
        }
      }
      // four partial sums: a 4-long dependency chain instead of an R-long one
      float tq[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int r = 0; r < RMAX; ++r) tq[r & 3] = fmaf(w[sl][r], kr[r], tq[r & 3]);
      const float ev = x - ((tq[0] + tq[1]) + (tq[2] + tq[3]));
      esqf = fmaf(ev, ev, esqf);
      tsqf = fmaf(x, x, tsqf);
#pragma unroll
      for (int r = 0; r < RMAX; ++r) g1[sl][r] = fmaf(ev, kr[r], g1[sl][r]);
      E[i * (kNB + 1) + f] = ev;
    };
    if constexpr (SLOTS == 1) {
      // one row per thread: the batch's two chunks of kHalf values are
      // register double buffers; chunk 1 is requested before chunk 0 is used,
      // and the next batch's chunk 0 before chunk 1 is used, so HBM latency
      // overlaps the arithmetic
      const int i = threadIdx.x;
      if (i < I1) {
        float esqf = 0.f, tsqf = 0.f;
        const float* tp = a.T + (size_t)I1 * f0 + i;
#pragma unroll
        for (int u = 0; u < kHalf; ++u) xb[u] = (kHalf + u < nb) ? __ldg(tp + (size_t)I1 * (kHalf + u)) : 0.f;
#pragma unroll
        for (int u = 0; u < kHalf; ++u)
          if (u < nb) entry(0, i, u, xa[u], esqf, tsqf);
        const long long bn = bt + gridDim.x;
        if (bn < nbatch) {
          const long long fn = bn * kNB;
          const int nbn = (int)((nf - fn) < kNB ? (nf - fn) : kNB);
          const float* tn = a.T + (size_t)I1 * fn + i;
#pragma unroll
          for (int u = 0; u < kHalf; ++u) xa[u] = (u < nbn) ? __ldg(tn + (size_t)I1 * u) : 0.f;
        }
#pragma unroll
        for (int u = 0; u < kHalf; ++u)
          if (kHalf + u < nb) entry(0, i, kHalf + u, xb[u], esqf, tsqf);
        for (int f = nb; f < kNB; ++f) E[i * (kNB + 1) + f] = 0.f;
        esq += (double)esqf;
        tsq += (double)tsqf;
      }
    } else {
#pragma unroll
      for (int sl = 0; sl < SLOTS; ++sl) {
        const int i = threadIdx.x + sl * blockDim.x;
        if (i >= I1) continue;
        float esqf = 0.f, tsqf = 0.f;
        const float* tp = a.T + (size_t)I1 * f0 + i;
        // the batch's values of row i in chunks of kPF fibres, all loads of a
        // chunk issued before any is used
        constexpr int kPF = kNB / 4;
        for (int c0 = 0; c0 < nb; c0 += kPF) {
          float xv[kPF];
#pragma unroll
          for (int u = 0; u < kPF; ++u) xv[u] = (c0 + u < nb) ? __ldg(tp + (size_t)I1 * (c0 + u)) : 0.f;
#pragma unroll
          for (int u = 0; u < kPF; ++u)
            if (c0 + u < nb) entry(sl, i, c0 + u, xv[u], esqf, tsqf);
        }
        for (int f = nb; f < kNB; ++f) E[i * (kNB + 1) + f] = 0.f;
        esq += (double)esqf;
        tsq += (double)tsqf;
      }
    }
    __syncthreads();
    // Q = E^T W1: warp w takes a slice of the rows, lane f the fibre f; the
    // row of W1 is a broadcast load shared by all fibres, and the slices'
    // partial sums meet in Qs through shared atomics
    {
      const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
      const int r0 = (int)((long long)wid * I1 / nw), r1 = (int)((long long)(wid + 1) * I1 / nw);
      float acc[RMAX];
#pragma unroll
      for (int r = 0; r < RMAX; ++r) acc[r] = 0.f;
      for (int ii = r0; ii < r1; ++ii) {
        const float e = E[ii * (kNB + 1) + lane];
        const float4* wr = reinterpret_cast<const float4*>(W1r + (size_t)ii * R4);
#pragma unroll
        for (int q = 0; q < RMAX / 4; ++q) {
          if (4 * q < R) {
            const float4 wv = wr[q];
            acc[4 * q] = fmaf(e, wv.x, acc[4 * q]); acc[4 * q + 1] = fmaf(e, wv.y, acc[4 * q + 1]);
            acc[4 * q + 2] = fmaf(e, wv.z, acc[4 * q + 2]); acc[4 * q + 3] = fmaf(e, wv.w, acc[4 * q + 3]);
          }
        }
      }
      if (lane < nb) {
#pragma unroll
        for (int r = 0; r < RMAX; ++r)
          if (r < R) atomicAdd(Qs + lane * R4 + r, acc[r]);
      }
    }
    __syncthreads();
    // scatter q into the other modes
    for (int o = threadIdx.x; o < nb * R; o += blockDim.x) {
      const int f = o / R, r = o - f * R;
      int idx[kMaxL];
      unsigned rem = (unsigned)(f0 + f);
#pragma unroll
      for (int l = 1; l < L; ++l) { idx[l] = (int)(rem % (unsigned)d[l]); rem /= (unsigned)d[l]; }
      const float q = Qs[f * R4 + r];
#pragma unroll
      for (int l = 1; l < L; ++l) {
        float p = q;
#pragma unroll
        for (int j = 1; j < L; ++j)
          if (j != l) p *= Ws[off[j] + r * d[j] + idx[j]];
        atomicAdd(Gs + off[l] + r * d[l] + idx[l], p);
      }
    }
    // no barrier: the next batch's first writes (KR, the other Qs buffer)
    // are not read here, and E and this Qs are rewritten only after two more
    // barriers
  }
#pragma unroll
  for (int sl = 0; sl < SLOTS; ++sl) {
    const int i = threadIdx.x + sl * blockDim.x;
    if (i >= I1) continue;
#pragma unroll
    for (int r = 0; r < RMAX; ++r)
      if (r < R && g1[sl][r] != 0.f) atomicAdd(a.G + r * I1 + i, g1[sl][r]);
  }
  __syncthreads();
  for (int j = off[1] + threadIdx.x; j < n; j += blockDim.x)
    if (Gs[j] != 0.f) atomicAdd(a.G + j, Gs[j]);
  // per-thread FP64 partials -> per-warp FP64 sums -> global FP64 atomics
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    esq += __shfl_xor_sync(0xffffffffu, esq, o);
    tsq += __shfl_xor_sync(0xffffffffu, tsq, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(a.esq, esq);
    if (a.want_tsq) atomicAdd(a.esq + 1, tsq);
  }
}

inline size_t pass_smem(int L, const long long* dims, int R) {
  size_t n = 0;
  for (int l = 0; l < L; ++l) n += (size_t)dims[l] * R;
  const size_t R4 = (R + 3) & ~3;
  const size_t n4 = (n + 3) & ~(size_t)3;
  return (2 * n4 + (size_t)dims[0] * R4 + (((size_t)dims[0] * (kNB + 1) + 3) & ~(size_t)3) +
          3 * (size_t)kNB * R4) * sizeof(float);
}


template <int L, int RMAX, int SLOTS>
inline cudaError_t launch_pass_t(const RefinePassArgs& a, size_t smem, int threads, long long blocks,
                                 cudaStream_t st) {
  cudaError_t e = cudaFuncSetAttribute(k_refine_pass<L, RMAX, SLOTS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_refine_pass<L, RMAX, SLOTS><<<(unsigned)blocks, threads, smem, st>>>(a);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_refine_pass3(const RefinePassArgs& a, size_t smem, int threads, long long blocks,
                                cudaStream_t st);
cudaError_t launch_refine_pass4(const RefinePassArgs& a, size_t smem, int threads, long long blocks,
                                cudaStream_t st);

// Instantiations for one order: the rank padded to 8, 12, 16, 32 or 64, and
// SLOTS rows per thread (I1 <= 256 * SLOTS).
template <int L>
inline cudaError_t launch_pass_l(const RefinePassArgs& a, size_t smem, int threads, long long blocks,
                                 cudaStream_t st) {
  const int slots = (int)((a.dims[0] + 255) / 256);
#define CPD_PASS_SLOTS3(RM)                                                        \
  if (slots <= 1) return launch_pass_t<L, RM, 1>(a, smem, threads, blocks, st);    \
  if (slots <= 2) return launch_pass_t<L, RM, 2>(a, smem, threads, blocks, st);    \
  return launch_pass_t<L, RM, 4>(a, smem, threads, blocks, st);
  if (a.R <= 8) { CPD_PASS_SLOTS3(8) }
  if (a.R <= 12) { CPD_PASS_SLOTS3(12) }
  if (a.R <= 16) { CPD_PASS_SLOTS3(16) }
#undef CPD_PASS_SLOTS3
  if (a.R <= 32) {
    if (slots <= 1) return launch_pass_t<L, 32, 1>(a, smem, threads, blocks, st);
    return launch_pass_t<L, 32, 2>(a, smem, threads, blocks, st);
  }
  return launch_pass_t<L, 64, 1>(a, smem, threads, blocks, st);
}

}  // namespace cpdk
