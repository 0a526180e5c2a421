// Batched solver for many small, unevenly shaped third-order CPDs: one
// persistent launch; every CTA takes items from a device work queue (items
// sorted longest-first by the host) and runs the whole method on each:
// ST-MLSVD compression (Gram, leading eigenpairs and truncation, projection;
// Sec. 2.2 and 4.1.1), initialisation and damped Gauss-Newton on the core
// (Sec. 4.1.2-4.1.3, the same device code as the single-tensor solver),
// uncompression (Sec. 4.1.4) and output normalisation.
#include <algorithm>
#include <map>
#include <mutex>
#include <string.h>
#include <vector>

#include "kernels.h"
#include "solver.cuh"
#include "dgn_cta.cuh"
#include "eig_cta.cuh"

namespace cpdk {

constexpr int kBatchThreadChoices[3] = {64, 128, 256};   // CTA sizes the autotuner times
constexpr int kBatchMaxDim = 64;
constexpr int kBatchMaxRank = 16;
constexpr int kGTile = 16;           // rows of the Gram's staging tile
constexpr int kGLd = 68;             // padded row length of the staging tile

// G (b x b, column-major) = sum_q X[q,:]^T X[q,:] with X[q, j] = T[i + a j + a b k],
// q = i + a k over the a*c "other" indices.  b <= 64; TH threads, each a
// TM x TN block of the 64 x 64 output (TH = 64: 8 x 8, 128: 4 x 8, 256: 4 x 4,
// the tile shapes the batch autotuner chooses between); rows of X staged in
// shared memory.
template <int TH>
__device__ void cta_gram(const float* __restrict__ T, int a, int b, int c, float* G, float* tile) {
  constexpr int TN = TH == 256 ? 4 : 8, NCG = 64 / TN, TM = 64 / (TH / NCG);
  const int tx = threadIdx.x % NCG, ty = threadIdx.x / NCG;
  float acc[TM][TN];
#pragma unroll
  for (int u = 0; u < TM; ++u)
#pragma unroll
    for (int v = 0; v < TN; ++v) acc[u][v] = 0.f;
  const long long K = (long long)a * c;
  for (long long qb = 0; qb < K; qb += kGTile) {
    for (int e = threadIdx.x; e < kGTile * 64; e += blockDim.x) {
      const int kk = e >> 6, jj = e & 63;
      const long long q = qb + kk;
      float x = 0.f;
      if (q < K && jj < b) {
        const long long i = q % a, k = q / a;
        x = __ldg(T + i + (long long)a * jj + (long long)a * b * k);
      }
      tile[kk * kGLd + jj] = x;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < kGTile; ++kk) {
      float av[TM], bv[TN];
#pragma unroll
      for (int u = 0; u < TM; u += 4) {
        const float4 ar = *reinterpret_cast<const float4*>(tile + kk * kGLd + ty * TM + u);
        av[u] = ar.x; av[u + 1] = ar.y; av[u + 2] = ar.z; av[u + 3] = ar.w;
      }
#pragma unroll
      for (int v = 0; v < TN; v += 4) {
        const float4 bb = *reinterpret_cast<const float4*>(tile + kk * kGLd + tx * TN + v);
        bv[v] = bb.x; bv[v + 1] = bb.y; bv[v + 2] = bb.z; bv[v + 3] = bb.w;
      }
#pragma unroll
      for (int u = 0; u < TM; ++u)
#pragma unroll
        for (int v = 0; v < TN; ++v) acc[u][v] = fmaf(av[u], bv[v], acc[u][v]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int u = 0; u < TM; ++u)
#pragma unroll
    for (int v = 0; v < TN; ++v) {
      const int r = ty * TM + u, cc = tx * TN + v;
      if (r < b && cc < b) G[r + b * cc] = acc[u][v];
    }
  __syncthreads();
}

// Y[i + a r + a rk k] = sum_j U[j + b r] T[i + a j + a b k], r < rk <= 16.
__device__ void cta_project(const float* __restrict__ T, int a, int b, int c, const float* U, int rk,
                            float* Y) {
  const long long n = (long long)a * c;
  for (long long q = threadIdx.x; q < n; q += blockDim.x) {
    const long long i = q % a, k = q / a;
    const float* t = T + i + (long long)a * b * k;
    float acc[kBatchMaxRank];
#pragma unroll
    for (int u = 0; u < kBatchMaxRank; ++u) acc[u] = 0.f;
    for (int j = 0; j < b; ++j) {
      const float x = t[(long long)a * j];
#pragma unroll
      for (int u = 0; u < kBatchMaxRank; ++u)
        if (u < rk) acc[u] = fmaf(U[u * b + j], x, acc[u]);
    }
#pragma unroll
    for (int u = 0; u < kBatchMaxRank; ++u)
      if (u < rk) Y[i + (long long)a * u + (long long)a * rk * k] = acc[u];
  }
  __syncthreads();
}

struct BatchLayout {           // per-CTA global scratch, offsets in floats
  size_t U, sig, Y1, Y2, S, Wc, Wf, res, cg, total;
};

__host__ __device__ inline BatchLayout batch_layout(int dmax, int Rmax, int maxiter) {
  const size_t P = (size_t)(Rmax < dmax ? Rmax : dmax);
  auto up = [](size_t x) { return (x + 63) & ~(size_t)63; };
  BatchLayout l{};
  size_t o = 0;
  l.U = o; o += up(3 * (size_t)dmax * P);
  l.sig = o; o += up(3 * P);
  l.Y1 = o; o += up(P * dmax * dmax);
  l.Y2 = o; o += up(P * P * dmax);
  l.S = o; o += up(P * P * P);
  l.Wc = o; o += up(3 * (size_t)dmax * Rmax);          // core factors (or T's, uncompressed)
  l.Wf = o; o += up(3 * (size_t)dmax * Rmax);
  l.res = o; o += 64;                                  // DevResult
  l.cg = o; o += up((size_t)maxiter + 1);              // cg_maxiter table (ints)
  l.total = o;
  return l;
}

__host__ __device__ inline int g_floats(int dmax) { return (dmax * dmax + 3) & ~3; }   // 16-byte multiple

// Per-item store between the phases of a phased run (offsets in floats):
// core (P^3) | U blocks (3 x dmax x P, block l at dmax * P * l) | meta
// (core dims as ints, ||S||, eligibility for the learned start).
struct StoreLayout { size_t core, U, meta, total; };
__host__ __device__ inline StoreLayout store_layout(int dmax, int Rmax) {
  const size_t P = (size_t)(Rmax < dmax ? Rmax : dmax);
  auto up = [](size_t x) { return (x + 63) & ~(size_t)63; };
  StoreLayout l{};
  l.core = 0;
  l.U = up(P * P * P);
  l.meta = l.U + up(3 * (size_t)dmax * P);
  l.total = l.meta + 64;
  return l;
}

__host__ __device__ inline size_t batch_compress_smem(int dmax, int Rmax) {
  const int P = Rmax < dmax ? Rmax : dmax;
  return (size_t)g_floats(dmax) * 4 + (size_t)kGTile * kGLd * 4 + (size_t)dmax * P * 4 + 256 +
         eig_smem_bytes(dmax, P, false, false);
}

// Resident blocks per SM the register allocation must allow (170 registers a
// thread for 64- and 128-thread blocks); without the bound the allocator
// caps registers for an occupancy target of its own and spills.
template <int TH>
constexpr int kBatchMinBlocks = TH == 64 ? 6 : TH == 128 ? 3 : 1;

template <int TH>
__global__ void __launch_bounds__(TH, kBatchMinBlocks<TH>) k_batch(BatchArgs a, int dmax, int Rmax, size_t smem_bytes) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_idx;
  __shared__ int s_rank[3];
  const BatchLayout lay = batch_layout(dmax, Rmax, a.maxiter);
  float* gs = a.scratch + (size_t)blockIdx.x * a.scratch_floats_per_cta;
  double* hist = a.hist + (size_t)blockIdx.x * (a.maxiter + 1);
  int* cgtab = reinterpret_cast<int*>(gs + lay.cg);
  DevResult* dres = reinterpret_cast<DevResult*>(gs + lay.res);
  const int P0 = Rmax < dmax ? Rmax : dmax;
  // compression shared layout: G | tile | Us | eig workspace
  float* G = reinterpret_cast<float*>(smem_raw);
  float* tile = G + g_floats(dmax);
  float* Us = tile + kGTile * kGLd;
  unsigned char* eigw = reinterpret_cast<unsigned char*>(Us + dmax * P0) + 256 -
                        (reinterpret_cast<size_t>(Us + dmax * P0) & 255);
  for (int guard = 0; guard < a.B + 1; ++guard) {     // at most B items per CTA
    if (threadIdx.x == 0) s_idx = atomicAdd(a.queue, 1);
    __syncthreads();
    const int idx = s_idx;
    __syncthreads();
    if (idx >= a.B) break;
    const BatchItem it = a.items[idx];
    const int d[3] = {it.d[0], it.d[1], it.d[2]};
    const int R = it.R;
    const uint64_t seed = a.seed + (uint64_t)it.b;
    const float* T = a.T + it.t_off;
    int core[3] = {d[0], d[1], d[2]};
    const float* S = T;
    float* U = gs + lay.U;
    const StoreLayout sl = store_layout(dmax, Rmax);
    float* slot = a.store ? a.store + (size_t)it.b * a.store_floats : nullptr;
    int* meta_i = slot ? reinterpret_cast<int*>(slot + sl.meta) : nullptr;
    if (a.phase == 2) {
      // the core and bases stored by phase 1; U blocks sit at dmax * P0 * l
      core[0] = meta_i[0]; core[1] = meta_i[1]; core[2] = meta_i[2];
      S = slot + sl.core;
      U = slot + sl.U;
    } else if (a.compress) {
      // ST-MLSVD: mode by mode on the partially projected tensor
      const float* cur = T;
      float* outs[3] = {gs + lay.Y1, gs + lay.Y2, gs + lay.S};
      long long ah = 1;
      size_t offU = 0;
      for (int l = 0; l < 3; ++l) {
        long long c = 1;
        for (int j = l + 1; j < 3; ++j) c *= d[j];
        const int P = R < d[l] ? R : d[l];
        cta_gram<TH>(cur, (int)ah, d[l], (int)c, G, tile);
        EigArgs ea{};
        ea.G = G; ea.I = d[l]; ea.P = P; ea.U = U + offU; ea.sigma = gs + lay.sig + l * P0;
        ea.rank_out = &s_rank[l]; ea.mlsvd_tol = a.mlsvd_tol; ea.L = 3;
        ea.seed = seed + 7919ull * (uint64_t)l;
        ea.work = G;                                   // non-null: G is read in place
        eig_run<32>(ea, eigw);
        __syncthreads();
        const int rk = s_rank[l];
        for (int e = threadIdx.x; e < d[l] * rk; e += blockDim.x) Us[e] = U[offU + e];
        __syncthreads();
        cta_project(cur, (int)ah, d[l], (int)c, Us, rk, outs[l]);
        core[l] = rk;
        cur = outs[l];
        ah *= rk;
        offU += (size_t)d[l] * P;
      }
      S = gs + lay.S;
    }
    if (a.phase == 1) {
      // store the core, the bases and the network's input row; no solve
      const int nc = core[0] * core[1] * core[2];
      float* dst = slot + sl.core;
      double sq = 0.0;
      for (int e = threadIdx.x; e < nc; e += blockDim.x) {
        const float v = S[e];
        dst[e] = v;
        sq += (double)v * (double)v;
      }
      {
        int offU = 0;
        for (int l = 0; l < 3; ++l) {
          const int P = R < d[l] ? R : d[l];
          for (int e = threadIdx.x; e < d[l] * P; e += blockDim.x) slot[sl.U + (size_t)dmax * P0 * l + e] = U[offU + e];
          offU += d[l] * P;
        }
      }
      __shared__ double s_sq;
      {
        float sqf[1] = {(float)sq};
        double o[1];
        block_sum<1>(sqf, o, reinterpret_cast<double*>(smem_raw));
        if (threadIdx.x == 0) s_sq = o[0];
      }
      __syncthreads();
      const float nrm = (float)sqrt(s_sq);
      const bool elig = R <= CPD_INITNET_RANK && core[0] <= CPD_INITNET_CORE && core[1] <= CPD_INITNET_CORE &&
                        core[2] <= CPD_INITNET_CORE && nrm > 0.f;
      if (threadIdx.x == 0) {
        meta_i[0] = core[0]; meta_i[1] = core[1]; meta_i[2] = core[2];
        slot[sl.meta + 3] = nrm;
        meta_i[4] = elig ? 1 : 0;
      }
      if (a.X) {
        float* x = a.X + (size_t)it.b * CPD_INITNET_IN_PAD;
        const float inv = nrm > 0.f ? 1.f / nrm : 0.f;
        for (int e = threadIdx.x; e < CPD_INITNET_IN_PAD; e += blockDim.x) {
          float v = 0.f;
          if (elig) {
            if (e < 4096) {
              const int i = e & 15, j = (e >> 4) & 15, k = e >> 8;
              if (i < core[0] && j < core[1] && k < core[2]) v = S[i + core[0] * (j + core[1] * k)] * inv;
            } else if (e == 4096 + R - 1) {
              v = 1.f;
            }
          }
          x[e] = v;
        }
      }
      __syncthreads();
      continue;
    }
    // damped Gauss-Newton on the core (the single-CTA solver); an item whose
    // tensor would not fit the launched shared memory is refused, not run
    {
      int cd[CPD_MAX_ORDER] = {core[0], core[1], core[2], 1};
      if (dgn_smem_bytes(3, cd, R, 1) > smem_bytes) {
        if (threadIdx.x == 0) {
          cpd_info inf;
          memset(&inf, 0, sizeof(inf));
          inf.status = CPD_ERR_UNSUPPORTED;
          a.infos[it.b] = inf;
        }
        __syncthreads();
        continue;
      }
    }
    DgnArgs da{};
    da.R = R;
    da.dims[0] = core[0]; da.dims[1] = core[1]; da.dims[2] = core[2]; da.dims[3] = 1;
    da.dev_dims = nullptr;
    da.S = S; da.s_f64 = 0; da.W0 = nullptr; da.init = a.init; da.seed = seed;
    if (a.phase == 2 && a.init == CPD_INIT_LEARNED) {
      // the network's proposal, scaled back by ||S||^(1/3), as stacked core-space
      // blocks; the MLSVD start when the item is not eligible
      if (meta_i[4] && a.Y) {
        float* W0 = gs + lay.Wf;
        const float* y = a.Y + (size_t)it.b * CPD_INITNET_OUT;
        const float sc = cbrtf(slot[sl.meta + 3]);
        int offC = 0;
        for (int l = 0; l < 3; ++l) {
          for (int q = threadIdx.x; q < core[l] * R; q += blockDim.x) {
            const int r = q / core[l], i = q - r * core[l];
            W0[offC + q] = y[l * 128 + r * 16 + i] * sc;
          }
          offC += core[l] * R;
        }
        da.W0 = W0;
      } else {
        da.init = CPD_INIT_MLSVD;
      }
    }
    da.tol = a.tol; da.tau = a.tau; da.cg_a = a.cg_a; da.cg_b = a.cg_b; da.maxiter = a.maxiter;
    da.mu0 = -1.0; da.mu_min = a.mu_min; da.k0 = 0; da.big_in_smem = 1; da.gscratch = nullptr;
    da.hist = hist; da.trace = nullptr; da.trace_cap = 0; da.trace_slot0 = 0;
    da.W_out = gs + lay.Wc; da.res = dres; da.cgtab = cgtab; da.cgtab_len = a.maxiter;
    __syncthreads();
    dgn_run<3>(da, smem_raw);
    __syncthreads();
    // uncompression W~ = U W (or the factors themselves)
    const float* Wc = gs + lay.Wc;
    float* Wf = gs + lay.Wf;
    {
      int offU = 0, offC = 0, offF = 0;
      for (int l = 0; l < 3; ++l) {
        const int I = d[l], rk = core[l], P = R < d[l] ? R : d[l];
        for (int q = threadIdx.x; q < I * R; q += blockDim.x) {
          const int r = q / I, i = q - r * I;
          float acc;
          if (a.compress) {
            acc = 0.f;
            for (int t = 0; t < rk; ++t) acc = fmaf(U[offU + t * I + i], Wc[offC + r * rk + t], acc);
          } else {
            acc = Wc[offC + r * rk + i];
          }
          Wf[offF + q] = acc;
        }
        offU += (a.phase == 2) ? dmax * P0 : I * P;
        offC += rk * R;
        offF += I * R;
      }
    }
    __syncthreads();
    if (a.phase == 2 && a.target) {
      // the core CPD as a training target: terms by decreasing weight, the
      // outputs' sign rule, column (l, r) scaled to (lambda_r / ||S||)^(1/3)
      float* tn = reinterpret_cast<float*>(smem_raw);              // 3 * R norms
      float* ts = tn + 3 * kBatchMaxRank;                           // 3 * R signs
      double* tl = reinterpret_cast<double*>(ts + 3 * kBatchMaxRank);
      int* tp = reinterpret_cast<int*>(tl + kBatchMaxRank);
      int offc[3] = {0, core[0] * R, (core[0] + core[1]) * R};
      for (int q = threadIdx.x; q < 3 * R; q += blockDim.x) {
        const int l = q / R, r = q - l * R, I = core[l];
        const float* w = Wc + offc[l] + r * I;
        double s2 = 0.0; float best = -1.f; int bi = 0;
        for (int i = 0; i < I; ++i) {
          s2 += (double)w[i] * (double)w[i];
          if (fabsf(w[i]) > best) { best = fabsf(w[i]); bi = i; }
        }
        tn[q] = (float)sqrt(s2);
        ts[q] = w[bi] < 0.f ? -1.f : 1.f;
      }
      __syncthreads();
      for (int r = threadIdx.x; r < R; r += blockDim.x) {
        tl[r] = (double)tn[r] * (double)tn[R + r] * (double)tn[2 * R + r];
        ts[2 * R + r] = ts[r] * ts[R + r];
      }
      __syncthreads();
      for (int r = threadIdx.x; r < R; r += blockDim.x) {
        int p = 0;
        for (int t = 0; t < R; ++t) p += (tl[t] > tl[r] || (tl[t] == tl[r] && t < r)) ? 1 : 0;
        tp[r] = p;
      }
      __syncthreads();
      // only converged, non-degenerate core CPDs make targets: the solve
      // reached rel_err < 1e-3 and no term outweighs the core 8 times
      // (diverging, cancelling terms appear near swamps)
      const float snrm = slot[sl.meta + 3];
      __shared__ int s_tgt_ok;
      if (threadIdx.x == 0) {
        bool okc = meta_i[4] != 0 && dres->status == CPD_OK && dres->rel_err < 1e-3;
        for (int r = 0; r < R; ++r) okc = okc && tl[r] <= 8.0 * (double)snrm;
        s_tgt_ok = okc ? 1 : 0;
      }
      __syncthreads();
      const bool elig = meta_i[4] != 0;             // the mask marks the entries that exist
      const bool tgt_ok = s_tgt_ok != 0;
      float* tg = a.target + (size_t)it.b * CPD_INITNET_OUT;
      float* tm = a.tmask ? a.tmask + (size_t)it.b * CPD_INITNET_OUT : nullptr;
      for (int e = threadIdx.x; e < CPD_INITNET_OUT; e += blockDim.x) { tg[e] = 0.f; if (tm) tm[e] = 0.f; }
      __syncthreads();
      if (elig) {
        for (int l = 0; l < 3; ++l) {
          const int I = core[l];
          for (int q = threadIdx.x; q < I * R; q += blockDim.x) {
            const int r = q / I, i = q - r * I;
            const float nr = tn[l * R + r];
            const float colscale = (float)cbrt(snrm > 0.f ? tl[r] / (double)snrm : 0.0);
            const float v = nr > 0.f ? Wc[offc[l] + q] / nr * ts[l * R + r] * colscale : 0.f;
            tg[l * 128 + tp[r] * 16 + i] = tgt_ok ? v : 0.f;
            if (tm) tm[l * 128 + tp[r] * 16 + i] = 1.f;
          }
        }
      }
      __syncthreads();
    }
    // output normalisation (unit columns, lambda, signs, descending lambda)
    float* nrm = reinterpret_cast<float*>(smem_raw);          // 3 * R
    float* sgn = nrm + 3 * kBatchMaxRank;                      // 3 * R
    double* lamd = reinterpret_cast<double*>(sgn + 3 * kBatchMaxRank);
    int* pos = reinterpret_cast<int*>(lamd + kBatchMaxRank);
    {
      int off[4] = {0, d[0] * R, (d[0] + d[1]) * R, (d[0] + d[1] + d[2]) * R};
      for (int q = threadIdx.x; q < 3 * R; q += blockDim.x) {
        const int l = q / R, r = q - l * R, I = d[l];
        const float* w = Wf + off[l] + r * I;
        double s = 0.0; float best = -1.f; int bi = 0;
        for (int i = 0; i < I; ++i) {
          s += (double)w[i] * (double)w[i];
          if (fabsf(w[i]) > best) { best = fabsf(w[i]); bi = i; }
        }
        nrm[q] = (float)sqrt(s);
        sgn[q] = w[bi] < 0.f ? -1.f : 1.f;
      }
      __syncthreads();
      for (int r = threadIdx.x; r < R; r += blockDim.x) {
        lamd[r] = (double)nrm[r] * (double)nrm[R + r] * (double)nrm[2 * R + r];
        sgn[2 * R + r] = sgn[r] * sgn[R + r];
      }
      __syncthreads();
      float* lam_out = a.lam + it.l_off;
      for (int r = threadIdx.x; r < R; r += blockDim.x) {
        int p = 0;
        for (int t = 0; t < R; ++t) p += (lamd[t] > lamd[r] || (lamd[t] == lamd[r] && t < r)) ? 1 : 0;
        pos[r] = p;
        lam_out[p] = (float)lamd[r];
      }
      __syncthreads();
      float* W_out = a.W + it.w_off;
      for (int l = 0; l < 3; ++l) {
        const int I = d[l];
        for (int q = threadIdx.x; q < I * R; q += blockDim.x) {
          const int r = q / I, i = q - r * I;
          const float nr = nrm[l * R + r];
          W_out[off[l] + pos[r] * I + i] = Wf[off[l] + q] * (nr > 0.f ? 1.f / nr : 1.f) * sgn[l * R + r];
        }
      }
    }
    if (threadIdx.x == 0) {
      cpd_info inf;
      memset(&inf, 0, sizeof(inf));
      inf.status = dres->status; inf.iters = dres->iters; inf.stop_reason = dres->stop;
      inf.cg_total = dres->cg_total; inf.rel_err = dres->rel_err; inf.mu = dres->mu;
      inf.grad_inf = dres->grad_inf;
      inf.core_dims[0] = core[0]; inf.core_dims[1] = core[1]; inf.core_dims[2] = core[2];
      inf.init_used = dres->pad0;
      a.infos[it.b] = inf;
    }
    __syncthreads();
  }
}

// Shared memory of one batch CTA: the larger of the compression phase and
// the dGN phase; the dGN holds the core (P^3, P = min(Rmax, dmax)) or, without
// compression, the whole item tensor (dmax^3).
size_t batch_store_floats(int dmax, int Rmax) { return store_layout(dmax, Rmax).total; }

size_t batch_smem_bytes(int dmax, int Rmax, int compress) {
  const int P = compress ? (Rmax < dmax ? Rmax : dmax) : dmax;
  int cd[CPD_MAX_ORDER] = {P, P, P, 1};
  size_t s1 = compress ? batch_compress_smem(dmax, Rmax) : 0;
  size_t s2 = dgn_smem_bytes(3, cd, Rmax, 1);
  size_t s3 = 2048;                                 // normalisation scratch
  size_t s = s1 > s2 ? s1 : s2;
  return s > s3 ? s : s3;
}

}  // namespace cpdk

using namespace cpdk;

namespace {
size_t smem_cap() {
  int dev = 0, v = 0;
  if (cudaGetDevice(&dev) == cudaSuccess &&
      cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) == cudaSuccess && v > 0)
    return (size_t)v;
  return 227 * 1024;
}

int batch_validate(int B, const int* dims, const int* ranks, const cpd_options& o, int* dmax, int* Rmax) {
  if (B < 1 || dims == nullptr || ranks == nullptr) return CPD_ERR_INVALID_ARG;
  if (o.maxiter < 1 || o.maxiter > 100000 || !(o.tol >= 0.0) || !(o.tau >= 0.0)) return CPD_ERR_INVALID_ARG;
  if (o.init != CPD_INIT_MLSVD && o.init != CPD_INIT_RANDOM) return CPD_ERR_UNSUPPORTED;
  if (o.refine_maxiter != 0 || o.gram_precision != CPD_GRAM_FP32) return CPD_ERR_UNSUPPORTED;
  int dm = 1, rm = 1;
  for (int b = 0; b < B; ++b) {
    const int R = ranks[b];
    if (R < 1) return CPD_ERR_INVALID_ARG;
    if (R > kBatchMaxRank) return CPD_ERR_UNSUPPORTED;
    double N = 1.0;
    for (int l = 0; l < 3; ++l) {
      const int x = dims[3 * b + l];
      if (x < 1) return CPD_ERR_INVALID_ARG;
      if (x > kBatchMaxDim || x < 2) return CPD_ERR_UNSUPPORTED;
      dm = x > dm ? x : dm;
      N *= x;
    }
    if ((double)R > N) return CPD_ERR_INVALID_ARG;
    rm = R > rm ? R : rm;
  }
  *dmax = dm; *Rmax = rm;
  if (!o.compress) {
    // the uncompressed solve keeps T in shared memory
    int cd[CPD_MAX_ORDER] = {dm, dm, dm, 1};
    if (dgn_smem_bytes(3, cd, rm, 1) > smem_cap()) return CPD_ERR_UNSUPPORTED;
  }
  return CPD_OK;
}

struct BatchPlan {
  size_t items, queue, infos, scratch, hist, total;
  int ctas;
  size_t per_cta;
};

// The CTA count follows from the shared-memory and thread budget of an SM
// (analytically, so the workspace size does not depend on runtime state);
// CTAs that cannot be resident at once simply start later and drain the queue.
int batch_ctas(int TH, size_t smem, int B) {
  int per_sm = (int)((228 * 1024) / (smem + 1024));
  if (per_sm > 2048 / TH) per_sm = 2048 / TH;
  if (per_sm > 32) per_sm = 32;
  if (per_sm < 1) per_sm = 1;
  const int sms = 152;
  return per_sm * sms < B ? per_sm * sms : B;
}

BatchPlan batch_plan(int B, int dmax, int Rmax, const cpd_options& o, size_t smem) {
  BatchPlan p{};
  p.ctas = 0;                         // capacity: the most CTAs any candidate CTA size launches
  for (int TH : kBatchThreadChoices) { const int c = batch_ctas(TH, smem, B); p.ctas = c > p.ctas ? c : p.ctas; }
  const BatchLayout lay = batch_layout(o.compress ? dmax : dmax, Rmax, o.maxiter);
  p.per_cta = lay.total;
  auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
  size_t off = 0;
  p.items = off; off += up(sizeof(BatchItem) * B);
  p.queue = off; off += 256;
  p.infos = off; off += up(sizeof(cpd_info) * B);
  p.hist = off; off += up(sizeof(double) * (size_t)(o.maxiter + 1) * p.ctas);
  p.scratch = off; off += up(sizeof(float) * p.per_cta * p.ctas);
  p.total = off;
  return p;
}
}  // namespace

namespace {

// Workspace of a phased run: the plain plan, then the per-item store, the
// network's inputs and outputs and its activation scratch.
struct ExLayout { BatchPlan p; size_t store, X, Y, act, total; size_t store_floats; };
ExLayout batch_ex_layout(int B, int dmax, int Rmax, const cpd_options& o, size_t smem) {
  ExLayout e{};
  e.p = batch_plan(B, dmax, Rmax, o, smem);
  auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
  e.store_floats = store_layout(dmax, Rmax).total;
  size_t off = e.p.total;
  e.store = off; off += up(sizeof(float) * e.store_floats * (size_t)B);
  e.X = off; off += up(sizeof(float) * (size_t)CPD_INITNET_IN_PAD * B);
  e.Y = off; off += up(sizeof(float) * (size_t)CPD_INITNET_OUT * B);
  e.act = off; off += up(initnet_act_bytes(B));
  e.total = off;
  return e;
}

template <int TH>
cudaError_t launch_th(BatchArgs a, int dmax, int Rmax, size_t smem, cudaStream_t st) {
  const int ctas = batch_ctas(TH, smem, a.B);
  a.ctas = ctas;
  cudaError_t e = cudaFuncSetAttribute(k_batch<TH>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_batch<TH><<<ctas, TH, smem, st>>>(a, dmax, Rmax, smem);
  count_launch();
  return cudaGetLastError();
}

// Queue reset and one persistent launch with CTAs of TH threads.
int launch_k_batch(const BatchArgs& a, int dmax, int Rmax, size_t smem, int TH, cudaStream_t st) {
  if (cudaMemsetAsync(a.queue, 0, 256, st) != cudaSuccess) return CPD_ERR_CUDA;
  cudaError_t e = TH == 64 ? launch_th<64>(a, dmax, Rmax, smem, st)
                           : TH == 256 ? launch_th<256>(a, dmax, Rmax, smem, st)
                                       : launch_th<128>(a, dmax, Rmax, smem, st);
  return e == cudaSuccess ? CPD_OK : CPD_ERR_CUDA;
}

// Autotuner of the batched solver's CTA size (and with it the Gram tile shape
// and the CTAs per SM): on the first call for a shape class (device, largest
// mode, largest rank, compression, batch size rounded to a power of two) it
// runs the whole batch once per candidate, timed with CUDA events on the
// stream, and keeps the fastest for later calls.  Not while the stream is
// being captured (the default, 128, is used then).  opts->block_threads of
// 64, 128 or 256 fixes the choice.
std::mutex g_tune_mu;
std::map<std::vector<long long>, int> g_tuned;

template <class Run>
int batch_threads(const cpd_options& o, int dmax, int Rmax, int B, cudaStream_t st, Run run, int* rc) {
  *rc = CPD_OK;
  if (o.block_threads == 64 || o.block_threads == 128 || o.block_threads == 256) return o.block_threads;
  int dev = 0;
  cudaGetDevice(&dev);
  int bb = 1;
  while ((1 << bb) < B) ++bb;
  const std::vector<long long> key = {dev, dmax, Rmax, o.compress, bb};
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tuned.find(key);
    if (it != g_tuned.end()) return it->second;
  }
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cap) != cudaSuccess || cap != cudaStreamCaptureStatusNone) {
    cudaGetLastError();
    return 128;
  }
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) { *rc = CPD_ERR_CUDA; return 128; }
  int best = 128;
  float best_ms = 3.4e38f;
  for (int TH : kBatchThreadChoices) {
    cudaEventRecord(e0, st);
    const int r = run(TH);
    cudaEventRecord(e1, st);
    if (r != CPD_OK || cudaEventSynchronize(e1) != cudaSuccess) { *rc = r != CPD_OK ? r : CPD_ERR_CUDA; break; }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best_ms) { best_ms = ms; best = TH; }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (*rc == CPD_OK) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tuned[key] = best;
  }
  return best;
}

std::vector<BatchItem> sorted_items(int B, const int64_t* t_off, const int* dims, const int* ranks,
                                    const int64_t* w_off, const int64_t* l_off) {
  std::vector<BatchItem> items((size_t)B);
  for (int b = 0; b < B; ++b) {
    BatchItem& it = items[(size_t)b];
    it.t_off = t_off[b]; it.w_off = w_off[b]; it.l_off = l_off[b];
    it.d[0] = dims[3 * b]; it.d[1] = dims[3 * b + 1]; it.d[2] = dims[3 * b + 2];
    it.R = ranks[b]; it.b = b; it.pad = 0;
  }
  std::stable_sort(items.begin(), items.end(), [](const BatchItem& x, const BatchItem& y) {
    const double cx = (double)x.d[0] * x.d[1] * x.d[2] * (x.d[0] + x.d[1] + x.d[2]) + 4e3 * x.R * x.R;
    const double cy = (double)y.d[0] * y.d[1] * y.d[2] * (y.d[0] + y.d[1] + y.d[2]) + 4e3 * y.R * y.R;
    return cx > cy;
  });
  return items;
}

// Graphs of the plain batched solve, per argument set (pointers, options,
// CTA size and a hash of the items), least recently used first out.  Each
// keeps the pinned host copy of the sorted items its upload node reads.
struct BatchGraphKey {
  int dev, B, TH, pad;
  unsigned long long h;
  cpd_options o;
  const float* T; float* W; float* lam; void* ws; size_t ws_bytes;
};
struct BatchGraphEntry { BatchGraphKey k; cudaGraphExec_t exec; BatchItem* pinned; unsigned long long used; };
std::mutex g_bgraph_mu;
std::vector<BatchGraphEntry> g_bgraphs;
unsigned long long g_bgraph_clock = 0;
constexpr size_t kMaxBatchGraphs = 8;

unsigned long long fnv1a(unsigned long long h, const void* p, size_t n) {
  const unsigned char* c = static_cast<const unsigned char*>(p);
  for (size_t i = 0; i < n; ++i) { h ^= c[i]; h *= 1099511628211ull; }
  return h;
}

unsigned long long batch_hash(int B, const int64_t* t_off, const int* dims, const int* ranks, const int64_t* w_off,
                              const int64_t* l_off) {
  unsigned long long h = 1469598103934665603ull;
  h = fnv1a(h, t_off, sizeof(int64_t) * B);
  h = fnv1a(h, dims, sizeof(int) * 3 * B);
  h = fnv1a(h, ranks, sizeof(int) * B);
  h = fnv1a(h, w_off, sizeof(int64_t) * B);
  h = fnv1a(h, l_off, sizeof(int64_t) * B);
  return h;
}

cudaGraphExec_t batch_graph_get(const BatchGraphKey& k) {
  std::lock_guard<std::mutex> lk(g_bgraph_mu);
  for (auto& e : g_bgraphs)
    if (memcmp(&e.k, &k, sizeof(k)) == 0) { e.used = ++g_bgraph_clock; return e.exec; }
  return nullptr;
}

void batch_graph_put(const BatchGraphKey& k, cudaGraphExec_t exec, BatchItem* pinned) {
  std::lock_guard<std::mutex> lk(g_bgraph_mu);
  if (g_bgraphs.size() >= kMaxBatchGraphs) {
    size_t victim = 0;
    for (size_t i = 1; i < g_bgraphs.size(); ++i)
      if (g_bgraphs[i].used < g_bgraphs[victim].used) victim = i;
    cudaGraphExecDestroy(g_bgraphs[victim].exec);
    cudaFreeHost(g_bgraphs[victim].pinned);
    g_bgraphs.erase(g_bgraphs.begin() + victim);
  }
  g_bgraphs.push_back(BatchGraphEntry{k, exec, pinned, ++g_bgraph_clock});
}

// mode 0: plain method + network inputs and training targets; mode 1: learned start.
int batch_ex(int mode, int B, const float* T_packed, const int64_t* t_off, const int* dims, const int* ranks,
             const cpd_options* opts, const float* params, float* W_packed, const int64_t* w_off,
             float* lam_packed, const int64_t* l_off, float* X, float* target, float* tmask, cpd_info* infos,
             void* workspace, size_t ws_bytes, void* stream) {
  cpd_options o; cpd_default_options(&o);
  if (opts) o = *opts;
  o.compress = 1; o.init = CPD_INIT_MLSVD;
  int dmax = 0, Rmax = 0;
  int v = batch_validate(B, dims, ranks, o, &dmax, &Rmax);
  if (v != CPD_OK) return v;
  if (!T_packed || !t_off || !W_packed || !w_off || !lam_packed || !l_off || !workspace)
    return CPD_ERR_INVALID_ARG;
  const size_t smem = batch_smem_bytes(dmax, Rmax, 1);
  if (smem > smem_cap()) return CPD_ERR_UNSUPPORTED;
  const ExLayout e = batch_ex_layout(B, dmax, Rmax, o, smem);
  if (ws_bytes < e.total) return CPD_ERR_WORKSPACE;
  const std::vector<BatchItem> items = sorted_items(B, t_off, dims, ranks, w_off, l_off);
  char* ws = static_cast<char*>(workspace);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (cudaMemcpyAsync(ws + e.p.items, items.data(), sizeof(BatchItem) * B, cudaMemcpyHostToDevice, st) != cudaSuccess)
    return CPD_ERR_CUDA;
  BatchArgs a{};
  a.T = T_packed; a.W = W_packed; a.lam = lam_packed;
  a.items = reinterpret_cast<const BatchItem*>(ws + e.p.items);
  a.B = B;
  a.queue = reinterpret_cast<int*>(ws + e.p.queue);
  a.infos = reinterpret_cast<cpd_info*>(ws + e.p.infos);
  a.scratch = reinterpret_cast<float*>(ws + e.p.scratch);
  a.scratch_floats_per_cta = e.p.per_cta;
  a.hist = reinterpret_cast<double*>(ws + e.p.hist);
  a.maxiter = o.maxiter; a.tol = o.tol; a.tau = o.tau; a.cg_a = o.cg_a; a.cg_b = o.cg_b; a.mu_min = o.mu_min;
  a.mlsvd_tol = o.mlsvd_tol; a.compress = 1; a.seed = o.seed; a.ctas = e.p.ctas;
  a.store = reinterpret_cast<float*>(ws + e.store);
  a.store_floats = e.store_floats;
  float* Xw = (mode == 1 || X == nullptr) ? reinterpret_cast<float*>(ws + e.X) : X;
  float* Yw = reinterpret_cast<float*>(ws + e.Y);
  auto run = [&](int TH) -> int {
    int r;
    {
      ProfScope ps(st, "batch_compress");
      a.phase = 1; a.X = Xw; a.init = CPD_INIT_MLSVD; a.Y = nullptr; a.target = nullptr; a.tmask = nullptr;
      if ((r = launch_k_batch(a, dmax, Rmax, smem, TH, st)) != CPD_OK) return r;
    }
    if (mode == 1) {
      ProfScope ps(st, "initnet_forward");
      if (initnet_forward(params, Xw, B, ws + e.act, Yw, st) != cudaSuccess) return CPD_ERR_CUDA;
    }
    ProfScope ps(st, "batch_solve");
    a.phase = 2; a.X = nullptr;
    a.init = mode == 1 ? CPD_INIT_LEARNED : CPD_INIT_MLSVD;
    a.Y = mode == 1 ? Yw : nullptr;
    a.target = mode == 0 ? target : nullptr;
    a.tmask = mode == 0 ? tmask : nullptr;
    return launch_k_batch(a, dmax, Rmax, smem, TH, st);
  };
  int trc = CPD_OK;
  const int TH = batch_threads(o, dmax, Rmax, B, st, run, &trc);
  if (trc != CPD_OK) return trc;
  if ((v = run(TH)) != CPD_OK) return v;
  if (infos) {
    if (cudaMemcpyAsync(infos, ws + e.p.infos, sizeof(cpd_info) * B, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return CPD_ERR_CUDA;
  }
  return cudaGetLastError() == cudaSuccess ? CPD_OK : CPD_ERR_CUDA;
}

}  // namespace

extern "C" {

size_t cpd_batch_workspace_size(int B, const int* dims, const int* ranks, const cpd_options* opts) {
  cpd_options o; cpd_default_options(&o);
  if (opts) o = *opts;
  int dmax = 0, Rmax = 0;
  if (batch_validate(B, dims, ranks, o, &dmax, &Rmax) != CPD_OK) return 0;
  const size_t smem = batch_smem_bytes(dmax, Rmax, o.compress);
  return batch_plan(B, dmax, Rmax, o, smem).total;
}

int cpd_batch_solve(int B, const float* T_packed, const int64_t* t_off, const int* dims,
                    const int* ranks, const cpd_options* opts, float* W_packed,
                    const int64_t* w_off, float* lam_packed, const int64_t* l_off,
                    cpd_info* infos, void* workspace, size_t ws_bytes, void* stream) {
  cpd_options o; cpd_default_options(&o);
  if (opts) o = *opts;
  int dmax = 0, Rmax = 0;
  int v = batch_validate(B, dims, ranks, o, &dmax, &Rmax);
  if (v != CPD_OK) return v;
  if (!T_packed || !t_off || !W_packed || !w_off || !lam_packed || !l_off || !workspace)
    return CPD_ERR_INVALID_ARG;
  const size_t smem = batch_smem_bytes(dmax, Rmax, o.compress);
  if (smem > smem_cap()) return CPD_ERR_UNSUPPORTED;
  const BatchPlan p = batch_plan(B, dmax, Rmax, o, smem);
  if (ws_bytes < p.total) return CPD_ERR_WORKSPACE;
  // items, longest first (cost ~ entries x mode sizes)
  const std::vector<BatchItem> items = sorted_items(B, t_off, dims, ranks, w_off, l_off);
  char* ws = static_cast<char*>(workspace);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  BatchArgs a{};
  a.T = T_packed; a.W = W_packed; a.lam = lam_packed;
  a.items = reinterpret_cast<const BatchItem*>(ws + p.items);
  a.B = B;
  a.queue = reinterpret_cast<int*>(ws + p.queue);
  a.infos = reinterpret_cast<cpd_info*>(ws + p.infos);
  a.scratch = reinterpret_cast<float*>(ws + p.scratch);
  a.scratch_floats_per_cta = p.per_cta;
  a.hist = reinterpret_cast<double*>(ws + p.hist);
  a.maxiter = o.maxiter; a.tol = o.tol; a.tau = o.tau; a.cg_a = o.cg_a; a.cg_b = o.cg_b; a.mu_min = o.mu_min;
  a.mlsvd_tol = o.mlsvd_tol; a.compress = o.compress; a.init = o.init; a.seed = o.seed; a.ctas = p.ctas;
  auto direct = [&](int TH) -> int {
    if (cudaMemcpyAsync(ws + p.items, items.data(), sizeof(BatchItem) * B, cudaMemcpyHostToDevice, st) != cudaSuccess)
      return CPD_ERR_CUDA;
    ProfScope ps(st, "batch");
    return launch_k_batch(a, dmax, Rmax, smem, TH, st);
  };
  int trc = CPD_OK;
  const int TH = batch_threads(o, dmax, Rmax, B, st, direct, &trc);
  if (trc != CPD_OK) return trc;
  // replay a captured graph (item upload from a pinned copy, queue reset, the
  // persistent launch) when the stream allows it; graphs are cached per
  // argument set
  bool launched = false;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (st != nullptr && !profile_enabled() && cudaStreamIsCapturing(st, &cap) == cudaSuccess &&
      cap == cudaStreamCaptureStatusNone) {
    BatchGraphKey k;
    memset(&k, 0, sizeof(k));
    cudaGetDevice(&k.dev);
    k.B = B; k.TH = TH; k.o = o; k.T = T_packed; k.W = W_packed; k.lam = lam_packed;
    k.ws = workspace; k.ws_bytes = ws_bytes;
    k.h = batch_hash(B, t_off, dims, ranks, w_off, l_off);
    cudaGraphExec_t exec = batch_graph_get(k);
    if (exec == nullptr) {
      BatchItem* pinned = nullptr;
      if (cudaMallocHost(reinterpret_cast<void**>(&pinned), sizeof(BatchItem) * B) == cudaSuccess) {
        memcpy(pinned, items.data(), sizeof(BatchItem) * B);
        cudaGraph_t g = nullptr;
        if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
          int rc = CPD_OK;
          if (cudaMemcpyAsync(ws + p.items, pinned, sizeof(BatchItem) * B, cudaMemcpyHostToDevice, st) != cudaSuccess)
            rc = CPD_ERR_CUDA;
          if (rc == CPD_OK) rc = launch_k_batch(a, dmax, Rmax, smem, TH, st);
          count_launch(-1);                  // captured, not launched: counted when replayed
          const cudaError_t ec = cudaStreamEndCapture(st, &g);
          if (rc == CPD_OK && ec == cudaSuccess && g != nullptr && cudaGraphInstantiate(&exec, g, 0) == cudaSuccess) {
            batch_graph_put(k, exec, pinned);
            pinned = nullptr;
          } else {
            exec = nullptr;
          }
          if (g) cudaGraphDestroy(g);
          cudaGetLastError();
        }
        if (pinned) cudaFreeHost(pinned);
      }
    }
    if (exec != nullptr) {
      if (cudaGraphLaunch(exec, st) != cudaSuccess) return CPD_ERR_CUDA;
      count_launch(1);
      launched = true;
    }
  }
  if (!launched) {
    const int rc = direct(TH);
    if (rc != CPD_OK) return rc;
  }
  if (infos) {
    if (cudaMemcpyAsync(infos, ws + p.infos, sizeof(cpd_info) * B, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return CPD_ERR_CUDA;
  }
  return cudaGetLastError() == cudaSuccess ? CPD_OK : CPD_ERR_CUDA;
}

size_t cpd_batch_ex_workspace_size(int B, const int* dims, const int* ranks, const cpd_options* opts) {
  cpd_options o; cpd_default_options(&o);
  if (opts) o = *opts;
  o.compress = 1; o.init = CPD_INIT_MLSVD;
  int dmax = 0, Rmax = 0;
  if (batch_validate(B, dims, ranks, o, &dmax, &Rmax) != CPD_OK) return 0;
  const size_t smem = batch_smem_bytes(dmax, Rmax, 1);
  return batch_ex_layout(B, dmax, Rmax, o, smem).total;
}

int cpd_batch_initnet_data(int B, const float* T_packed, const int64_t* t_off, const int* dims,
                           const int* ranks, const cpd_options* opts, float* W_packed,
                           const int64_t* w_off, float* lam_packed, const int64_t* l_off,
                           float* X, float* target, float* mask, cpd_info* infos,
                           void* workspace, size_t ws_bytes, void* stream) {
  return batch_ex(0, B, T_packed, t_off, dims, ranks, opts, nullptr, W_packed, w_off, lam_packed, l_off, X,
                  target, mask, infos, workspace, ws_bytes, stream);
}

int cpd_batch_solve_learned(int B, const float* T_packed, const int64_t* t_off, const int* dims,
                            const int* ranks, const cpd_options* opts, const float* params,
                            float* W_packed, const int64_t* w_off, float* lam_packed,
                            const int64_t* l_off, cpd_info* infos, void* workspace,
                            size_t ws_bytes, void* stream) {
  if (params == nullptr) return CPD_ERR_INVALID_ARG;
  return batch_ex(1, B, T_packed, t_off, dims, ranks, opts, params, W_packed, w_off, lam_packed, l_off, nullptr,
                  nullptr, nullptr, infos, workspace, ws_bytes, stream);
}

}  // extern "C"
