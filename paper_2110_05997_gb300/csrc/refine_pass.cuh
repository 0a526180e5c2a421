// The pass over T of a refinement iteration (dGN on the full tensor after
// uncompression): residual e = T - [[W]], ||e||^2 (and ||T||^2) in FP64, and
// the MTTKRP of e for every mode (= -grad F; the Sec. 4.1.3 formulas applied
// to T).  Included by one translation unit per tensor order.
#pragma once

#include <mutex>

#include "kernels.h"
#include "solver.cuh"

namespace cpdk {

// Mode-1 fibers (I1 contiguous floats) in batches of kNB.  Thread i owns row
// i1 = i of every fiber: with kr_r = prod_{l>=2} W_l[i_l, r] (shared, float4
// broadcast loads) it forms t~ = sum_r W1[i1, r] kr_r (W1 row in registers),
// e = t - t~, ||e||^2, and accumulates G1[i1, :] += e kr in registers for the
// whole kernel.  Then Q = E^T W1 per fiber (float4 broadcast of W1 rows; each
// warp's partial sums over its slice of rows in its own shared slice) and
// G_l[i_l, r] += q_r prod_{j>=2, j!=l} W_j[i_j, r] for l >= 2: lane f takes
// fibre f, lanes with the same i_l in a run are summed by a segmented warp
// reduction, and one shared atomic per run adds the sum.
constexpr int kNB = 32;
static_assert(kNB == 32, "the Q product and the scatter map fibres of a batch to the lanes of a warp");
constexpr int kPassWarps = 8;                  // 256 threads at most

// Q partials per warp (plain stores, summed in the scatter) while they fit;
// above, shared atomics into one Q buffer per batch
template <int RP>
constexpr bool pass_q_slices() { return RP <= 16; }

// Padded rank of the pass: the shared rows of the Khatri-Rao products, of W1
// and of Q have this many floats (zero beyond R), so the inner loops run over
// a compile-time length with no rank tests.
inline __host__ __device__ int pass_rank_pad(int R) {
  return R <= 8 ? 8 : R <= 12 ? 12 : R <= 16 ? 16 : R <= 32 ? 32 : 64;
}

// Small ranks with one row per thread are held to 128 registers, so that two
// CTAs of up to 8 warps share an SM (each SM sub-partition holds 4 such warps).
template <int L, int RP, int SLOTS>
__global__ void __launch_bounds__(256, (RP <= 16 && SLOTS == 1) ? 2 : 1) k_refine_pass(RefinePassArgs a) {
  if (a.done && *a.done) return;
  extern __shared__ __align__(16) float sm[];
  const int R = a.R;
  const int I1 = (int)a.dims[0];
  // d[l] for modes 2..L; off[l]: start of mode l (l >= 1) in the modes-2..L
  // part of the stacked vectors, which begins after W1's I1 x R floats
  int d[kMaxL], off[kMaxL + 1];
#pragma unroll
  for (int l = 0; l < kMaxL; ++l) d[l] = (l < L) ? (int)a.dims[l] : 1;
  off[0] = 0;
  off[1] = 0;
#pragma unroll
  for (int l = 1; l < L; ++l) off[l + 1] = off[l] + d[l] * R;
  const int n2 = off[L];
  const int w1n = I1 * R;
  unsigned nf = 1;                             // < 2^31 (checked at launch)
#pragma unroll
  for (int l = 1; l < L; ++l) nf *= (unsigned)d[l];
  // shared: Ws (modes 2..L) | Gs (modes 2..L) | W1r (I1 x RP, row-major)
  //         | E (I1 x (kNB+1)) | KR (kNB x RP) | Q (per-warp slices 8 x RP x kNB, or 2 x kNB x RP)
  //         | fibre indices (2 x (L-1) x kNB)
  constexpr bool kSlices = pass_q_slices<RP>();
  constexpr int kQFloats = kSlices ? kPassWarps * RP * kNB : 2 * kNB * RP;
  const int n24 = (n2 + 3) & ~3;
  float* Ws = sm;
  float* Gs = Ws + n24;
  float* W1r = Gs + n24;
  float* E = W1r + (size_t)I1 * RP;
  float* KR = E + (((size_t)I1 * (kNB + 1) + 3) & ~(size_t)3);
  float* Qs2 = KR + kNB * RP;
  int* fidx2 = reinterpret_cast<int*>(Qs2 + kQFloats);
  for (int j = threadIdx.x; j < n2; j += blockDim.x) { Ws[j] = a.W[w1n + j]; Gs[j] = 0.f; }
  for (int j = threadIdx.x; j < I1 * RP; j += blockDim.x) {     // W1 (I1 x R, column-major) -> rows
    const int i = j / RP, r = j - i * RP;
    W1r[j] = r < R ? a.W[r * I1 + i] : 0.f;
  }
  __syncthreads();
  // thread owns rows i1 = threadIdx.x + s * blockDim.x, s < SLOTS
  float w[SLOTS][RP], g1[SLOTS][RP];
#pragma unroll
  for (int sl = 0; sl < SLOTS; ++sl) {
    const int i = threadIdx.x + sl * blockDim.x;
    const float4* w4 = reinterpret_cast<const float4*>(W1r + (size_t)i * RP);
#pragma unroll
    for (int q = 0; q < RP / 4; ++q) {
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (i < I1) v = w4[q];
      w[sl][4 * q] = v.x; w[sl][4 * q + 1] = v.y; w[sl][4 * q + 2] = v.z; w[sl][4 * q + 3] = v.w;
    }
#pragma unroll
    for (int r = 0; r < RP; ++r) g1[sl][r] = 0.f;
  }
  double esq = 0.0, tsq = 0.0;
  const unsigned nbatch = (nf + kNB - 1) / kNB;
  constexpr int kHalf = kNB / 2;
  float xa[kHalf], xb[kHalf];                 // register double buffers (one row per thread)
  if constexpr (SLOTS == 1) {
    const unsigned b0 = blockIdx.x;
    const int i = threadIdx.x;
    if (b0 < nbatch && i < I1) {
      const unsigned fb = b0 * kNB;
      const int nb0 = (int)((nf - fb) < kNB ? (nf - fb) : kNB);
      const float* tb = a.T + (size_t)I1 * fb + i;
#pragma unroll
      for (int u = 0; u < kHalf; ++u) xa[u] = (u < nb0) ? __ldg(tb + (size_t)I1 * u) : 0.f;
    }
  }
  int par = 0;
  for (unsigned bt = blockIdx.x; bt < nbatch; bt += gridDim.x, par ^= 1) {
    const unsigned f0 = bt * kNB;
    const int nb = (int)((nf - f0) < kNB ? (nf - f0) : kNB);
    // atomics variant: this batch's Q buffer, read by its scatter only; the
    // per-warp slices are rewritten only after two more barriers
    float* Qs = kSlices ? Qs2 : Qs2 + par * kNB * RP;
    int* fidx = fidx2 + par * (L - 1) * kNB;   // (L-1) x kNB indices i_2.., by mode
    // Khatri-Rao rows: item (chunk q of four ranks, fibre f = lane)
    for (int e = threadIdx.x; e < kNB * (RP / 4); e += blockDim.x) {
      const int f = e & (kNB - 1), q = e / kNB;
      float4 p = make_float4(0.f, 0.f, 0.f, 0.f);
      if (f < nb) {
        int il[kMaxL];
        unsigned rem = f0 + f;
#pragma unroll
        for (int l = 1; l < L; ++l) { il[l] = (int)(rem % (unsigned)d[l]); rem /= (unsigned)d[l]; }
        if (q == 0) {
#pragma unroll
          for (int l = 1; l < L; ++l) fidx[(l - 1) * kNB + f] = il[l];
        }
        float pv[4] = {1.f, 1.f, 1.f, 1.f};
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int r = 4 * q + u;
          if (r < R) {
#pragma unroll
            for (int l = 1; l < L; ++l) pv[u] *= Ws[off[l] + r * d[l] + il[l]];
          } else {
            pv[u] = 0.f;
          }
        }
        p = make_float4(pv[0], pv[1], pv[2], pv[3]);
      }
      reinterpret_cast<float4*>(KR + f * RP)[q] = p;
      if constexpr (!kSlices) reinterpret_cast<float4*>(Qs + f * RP)[q] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    __syncthreads();
    // one entry (row i, fibre f): t~ = W1[i,:] . kr_f, e = t - t~, ||e||^2,
    // ||t||^2, G1[i,:] += e kr_f, and e into E for the Q product
    auto entry = [&](int sl, int i, int f, float x, float& esqf, float& tsqf) {
      const float4* k4 = reinterpret_cast<const float4*>(KR + f * RP);
      float kr[RP];
#pragma unroll
      for (int q = 0; q < RP / 4; ++q) {
        const float4 v = k4[q];
        kr[4 * q] = v.x; kr[4 * q + 1] = v.y; kr[4 * q + 2] = v.z; kr[4 * q + 3] = v.w;
      }
      // four partial sums: a 4-long dependency chain instead of an R-long one
      float tq[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int r = 0; r < RP; ++r) tq[r & 3] = fmaf(w[sl][r], kr[r], tq[r & 3]);
      const float ev = x - ((tq[0] + tq[1]) + (tq[2] + tq[3]));
      esqf = fmaf(ev, ev, esqf);
      tsqf = fmaf(x, x, tsqf);
#pragma unroll
      for (int r = 0; r < RP; ++r) g1[sl][r] = fmaf(ev, kr[r], g1[sl][r]);
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
        const unsigned bn = bt + gridDim.x;
        const unsigned fn = bn * kNB;
        const int nbn = bn < nbatch ? (int)((nf - fn) < kNB ? (nf - fn) : kNB) : 0;
        const float* tn = a.T + (size_t)I1 * fn + i;
        if (nb == kNB) {                       // whole batch: no per-entry tests
#pragma unroll
          for (int u = 0; u < kHalf; ++u) xb[u] = __ldg(tp + (size_t)I1 * (kHalf + u));
#pragma unroll
          for (int u = 0; u < kHalf; ++u) entry(0, i, u, xa[u], esqf, tsqf);
          if (nbn == kNB) {
#pragma unroll
            for (int u = 0; u < kHalf; ++u) xa[u] = __ldg(tn + (size_t)I1 * u);
          } else {
#pragma unroll
            for (int u = 0; u < kHalf; ++u) xa[u] = (u < nbn) ? __ldg(tn + (size_t)I1 * u) : 0.f;
          }
#pragma unroll
          for (int u = 0; u < kHalf; ++u) entry(0, i, kHalf + u, xb[u], esqf, tsqf);
        } else {                               // the ragged last batch
#pragma unroll
          for (int u = 0; u < kHalf; ++u) xb[u] = (kHalf + u < nb) ? __ldg(tp + (size_t)I1 * (kHalf + u)) : 0.f;
#pragma unroll
          for (int u = 0; u < kHalf; ++u)
            if (u < nb) entry(0, i, u, xa[u], esqf, tsqf);
#pragma unroll
          for (int u = 0; u < kHalf; ++u) xa[u] = (u < nbn) ? __ldg(tn + (size_t)I1 * u) : 0.f;
#pragma unroll
          for (int u = 0; u < kHalf; ++u)
            if (kHalf + u < nb) entry(0, i, kHalf + u, xb[u], esqf, tsqf);
          for (int f = nb; f < kNB; ++f) E[i * (kNB + 1) + f] = 0.f;
        }
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
    // row of W1 is a broadcast load shared by all fibres, two rows per step
    {
      const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
      const int r0 = (int)((long long)wid * I1 / nw), r1 = (int)((long long)(wid + 1) * I1 / nw);
      float acc[RP], acc2[RP];
#pragma unroll
      for (int r = 0; r < RP; ++r) { acc[r] = 0.f; acc2[r] = 0.f; }
      int ii = r0;
      for (; ii + 2 <= r1; ii += 2) {
        const float e0 = E[ii * (kNB + 1) + lane];
        const float e1 = E[(ii + 1) * (kNB + 1) + lane];
        const float4* wr0 = reinterpret_cast<const float4*>(W1r + (size_t)ii * RP);
        const float4* wr1 = reinterpret_cast<const float4*>(W1r + (size_t)(ii + 1) * RP);
#pragma unroll
        for (int q = 0; q < RP / 4; ++q) {
          const float4 u = wr0[q], v = wr1[q];
          acc[4 * q] = fmaf(e0, u.x, acc[4 * q]); acc[4 * q + 1] = fmaf(e0, u.y, acc[4 * q + 1]);
          acc[4 * q + 2] = fmaf(e0, u.z, acc[4 * q + 2]); acc[4 * q + 3] = fmaf(e0, u.w, acc[4 * q + 3]);
          acc2[4 * q] = fmaf(e1, v.x, acc2[4 * q]); acc2[4 * q + 1] = fmaf(e1, v.y, acc2[4 * q + 1]);
          acc2[4 * q + 2] = fmaf(e1, v.z, acc2[4 * q + 2]); acc2[4 * q + 3] = fmaf(e1, v.w, acc2[4 * q + 3]);
        }
      }
      if (ii < r1) {
        const float e0 = E[ii * (kNB + 1) + lane];
        const float4* wr0 = reinterpret_cast<const float4*>(W1r + (size_t)ii * RP);
#pragma unroll
        for (int q = 0; q < RP / 4; ++q) {
          const float4 u = wr0[q];
          acc[4 * q] = fmaf(e0, u.x, acc[4 * q]); acc[4 * q + 1] = fmaf(e0, u.y, acc[4 * q + 1]);
          acc[4 * q + 2] = fmaf(e0, u.z, acc[4 * q + 2]); acc[4 * q + 3] = fmaf(e0, u.w, acc[4 * q + 3]);
        }
      }
      if constexpr (kSlices) {
#pragma unroll
        for (int r = 0; r < RP; ++r) Qs[(wid * RP + r) * kNB + lane] = acc[r] + acc2[r];
      } else if (lane < nb && r1 > r0) {
#pragma unroll
        for (int r = 0; r < RP; ++r)
          if (r < R) atomicAdd(Qs + lane * RP + r, acc[r] + acc2[r]);
      }
    }
    __syncthreads();
    // scatter q into the other modes: warp w takes ranks w, w + nw, ...,
    // lane f the fibre f; runs of lanes with the same index i_l are summed
    // (segmented suffix sums by shuffles) and their first lane adds the sum
    {
      const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
      const bool act = lane < nb;
      const unsigned le = lane == 31 ? 0xffffffffu : ((2u << lane) - 1u);
      int idx[kMaxL], seg[kMaxL];
      bool head[kMaxL];
#pragma unroll
      for (int l = 1; l < L; ++l) {
        idx[l] = act ? fidx[(l - 1) * kNB + lane] : -1 - lane;
        const int prev = __shfl_up_sync(0xffffffffu, idx[l], 1);
        head[l] = lane == 0 || prev != idx[l];
        seg[l] = __popc(__ballot_sync(0xffffffffu, head[l]) & le);
      }
      for (int r = wid; r < R; r += nw) {
        float q = 0.f;
        if constexpr (kSlices) {
          for (int w2 = 0; w2 < nw; ++w2) q += Qs[(w2 * RP + r) * kNB + lane];
        } else {
          q = Qs[lane * RP + r];
        }
        float wv[kMaxL];
#pragma unroll
        for (int l = 1; l < L; ++l) wv[l] = act ? Ws[off[l] + r * d[l] + idx[l]] : 0.f;
#pragma unroll
        for (int l = 1; l < L; ++l) {
          float p = q;
#pragma unroll
          for (int j = 1; j < L; ++j)
            if (j != l) p *= wv[j];
#pragma unroll
          for (int o = 1; o < 32; o <<= 1) {
            const float pv = __shfl_down_sync(0xffffffffu, p, o);
            const int sv = __shfl_down_sync(0xffffffffu, seg[l], o);
            if (lane + o < 32 && sv == seg[l]) p += pv;
          }
          if (act && head[l]) atomicAdd(Gs + off[l] + r * d[l] + idx[l], p);
        }
      }
    }
    // no barrier: the next batch's first writes (KR, the other index buffer
    // and Q buffer) are not read here, and E and the Q slices are rewritten
    // only after two more barriers
  }
#pragma unroll
  for (int sl = 0; sl < SLOTS; ++sl) {
    const int i = threadIdx.x + sl * blockDim.x;
    if (i >= I1) continue;
#pragma unroll
    for (int r = 0; r < RP; ++r)
      if (r < R && g1[sl][r] != 0.f) atomicAdd(a.G + r * I1 + i, g1[sl][r]);
  }
  __syncthreads();
  for (int j = threadIdx.x; j < n2; j += blockDim.x)
    if (Gs[j] != 0.f) atomicAdd(a.G + w1n + j, Gs[j]);
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
  size_t n2 = 0;
  for (int l = 1; l < L; ++l) n2 += (size_t)dims[l] * R;
  const size_t RP = (size_t)pass_rank_pad(R);
  const size_t n24 = (n2 + 3) & ~(size_t)3;
  const size_t q = RP <= 16 ? (size_t)kPassWarps * RP * kNB : 2 * (size_t)kNB * RP;
  return (2 * n24 + (size_t)dims[0] * RP + (((size_t)dims[0] * (kNB + 1) + 3) & ~(size_t)3) +
          (size_t)kNB * RP + q) * sizeof(float) + 2 * (size_t)(L - 1) * kNB * sizeof(int);
}


// Grid: every CTA resident at once (CTAs per SM by registers, shared memory
// and threads, times the SM count), capped at the number of fibre batches
// `nbatch`; each CTA strides over the batches.
// The attributes and the resident-CTA count of the last (device, shared
// memory, threads) an instantiation was launched with are kept, so repeated
// launches of one shape make no host queries.
struct PassLaunchCache {
  std::mutex mu;
  int dev = -1, threads = 0;
  size_t smem = 0;
  long long resident = 0;
};

template <int L, int RP, int SLOTS>
inline cudaError_t launch_pass_t(const RefinePassArgs& a, size_t smem, int threads, long long nbatch,
                                 cudaStream_t st) {
  static PassLaunchCache cache;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  long long resident = 0;
  {
    std::lock_guard<std::mutex> lk(cache.mu);
    if (cache.dev == dev && cache.smem == smem && cache.threads == threads) resident = cache.resident;
  }
  if (resident == 0) {
    e = cudaFuncSetAttribute(k_refine_pass<L, RP, SLOTS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    // all of the unified L1 as shared memory, so that CTAs can share an SM
    e = cudaFuncSetAttribute(k_refine_pass<L, RP, SLOTS>, cudaFuncAttributePreferredSharedMemoryCarveout,
                             cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
    int per_sm = 0, sms = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_refine_pass<L, RP, SLOTS>, threads, smem)) != cudaSuccess)
      return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    resident = (long long)per_sm * sms;
    std::lock_guard<std::mutex> lk(cache.mu);
    cache.dev = dev; cache.smem = smem; cache.threads = threads; cache.resident = resident;
  }
  long long blocks = resident;
  if (blocks > nbatch) blocks = nbatch;
  if (blocks < 1) blocks = 1;
  k_refine_pass<L, RP, SLOTS><<<(unsigned)blocks, threads, smem, st>>>(a);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_refine_pass3(const RefinePassArgs& a, size_t smem, int threads, long long nbatch,
                                cudaStream_t st);
cudaError_t launch_refine_pass4(const RefinePassArgs& a, size_t smem, int threads, long long nbatch,
                                cudaStream_t st);

// Instantiations for one order: the rank padded to 8, 12, 16, 32 or 64, and
// SLOTS rows per thread (I1 <= 256 * SLOTS).
template <int L>
inline cudaError_t launch_pass_l(const RefinePassArgs& a, size_t smem, int threads, long long nbatch,
                                 cudaStream_t st) {
  const int slots = (int)((a.dims[0] + 255) / 256);
  const int rp = pass_rank_pad(a.R);
#define CPD_PASS_SLOTS3(RM)                                                        \
  if (slots <= 1) return launch_pass_t<L, RM, 1>(a, smem, threads, nbatch, st);    \
  if (slots <= 2) return launch_pass_t<L, RM, 2>(a, smem, threads, nbatch, st);    \
  return launch_pass_t<L, RM, 4>(a, smem, threads, nbatch, st);
  if (rp == 8) { CPD_PASS_SLOTS3(8) }
  if (rp == 12) { CPD_PASS_SLOTS3(12) }
  if (rp == 16) { CPD_PASS_SLOTS3(16) }
#undef CPD_PASS_SLOTS3
  if (rp == 32) {
    if (slots <= 1) return launch_pass_t<L, 32, 1>(a, smem, threads, nbatch, st);
    return launch_pass_t<L, 32, 2>(a, smem, threads, nbatch, st);
  }
  return launch_pass_t<L, 64, 1>(a, smem, threads, nbatch, st);
}

}  // namespace cpdk
