// The pass over T of a refinement iteration on the tensor cores: residual
// e = T - [[W]], ||e||^2 (and ||T||^2) with FP64 accumulation, and the MTTKRP
// of e for every mode (= -grad F, the gradient formulas of Sec. 4.1.3 applied
// to the full tensor) in one read of T.
//
// T is viewed as the I1 x nf matrix X of its mode-1 fibres (nf = I2 ... IL),
// cut into tiles of 128 consecutive fibres; fibres longer than 128 are cut
// into nch row chunks of IC rows.  Per tile and chunk:
//   * a tensor-map bulk copy brings the FP32 block X[chunk rows, 128 fibres]
//     into a shared-memory stage (zero-filled beyond the tensor);
//   * the compute warps form the tile's Khatri-Rao rows kr_f = prod_{l>=2}
//     W_l[i_l(f), :] (the other modes' factor rows, in shared memory) and
//     split each entry into three BF16 parts (hi + mid + lo carry 24 bits);
//   * the tensor core forms X~^T = KR W1^T from the six products of parts
//     whose exponents sum to at most 2^-16 of the leading one (FP32-accurate
//     model entries, accumulated in FP32 in tensor memory, one lane per fibre);
//   * the compute warps read X~ back, form e = x - x~ (FP32), accumulate
//     ||e||^2, and store e in BF16 as the tile E^T (fibre rows, 128-byte
//     swizzle) over the stage the block came in (it is no longer needed);
//   * the tensor core forms Q = E^T W1 (fibre x rank, K-major operands) and
//     accumulates G1 += E KR (mode-1 gradient; both operands read MN-major
//     from the same two tiles), BF16 products with FP32 accumulation;
//   * the compute warps scatter Q into modes 2..L: G_l[i_l, r] += q_fr
//     prod_{j>=2, j!=l} W_j[i_j, r], the mode-2 term per fibre and the slower
//     modes once per run of fibres that share their indices.
// The MTTKRP of e is in BF16 (relative error ~2^-9 per product, as the
// compression Grams): it perturbs the refined optimum by ~2^-9 of the noise
// level's effect, far below the parity tolerances; the residual itself, the
// quantity that decides the fit, is FP32-accurate.
//
// The compute warps build tile k+1's Khatri-Rao rows (double-buffered) before
// tile k's residual, and scatter tile k-1's Q after it (Q double-buffered in
// tensor memory), so the X~ MMAs of the next tile and the Q / G1 MMAs of the
// current one run while the compute warps work.
//
// Roles: warps 0-7 compute (warp w owns TMEM lanes / fibres 32 (w % 4) + lane
// and, with the other warp of its lane quarter, half of the columns and of
// the ranks), warp 8 issues the copies, warp 9 the MMAs.  Every mbarrier wait
// is bounded in SM clock cycles; a wait that runs out sets the shared abort
// flag and the global error word.  The copy and MMA threads then stop
// issuing; the compute warps keep their control flow (so that every warp
// reaches every named barrier) with the waits failing at once and the work
// skipped; the copies and MMAs still in flight are waited for (bounded) and
// the tensor memory is freed before the CTA exits.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <stdint.h>

#include <mutex>
#include <type_traits>

#include "kernels.h"
#include "tc_common.cuh"

namespace cpdk {
namespace {

using namespace tc;

constexpr int kFB = 128;                  // fibres per tile (TMEM lanes, MMA M)
constexpr int kNG = 4;                    // compute warp groups (4 warps each)
constexpr int kCW = 4 * kNG;              // compute warps
constexpr int kThreads = 32 * (kCW + 2);  // + copy warp + MMA warp
constexpr int kRP = 16;                   // padded rank (MMA N of Q and G1, K of X~)
constexpr int kRG = kRP / kNG;            // ranks per warp group in the Khatri-Rao rows / scatter
constexpr int kStages = 2;
constexpr uint32_t kTmemCols = 512;
constexpr uint32_t kColQ = 256, kColG1 = 288;   // D_q[2], D_g1[c] (16 columns each); X~[2] in 0..255

struct TcPassArgs {
  const float* W;           // stacked factors
  float* G;                 // stacked MTTKRP of the residual (accumulated into, zeroed by the launcher)
  double* esq;              // [0] ||e||^2, [1] ||T||^2
  const int* done;          // skip when *done != 0
  int* err;                 // set to CPD_ERR_TIMEOUT when a bounded wait runs out
  int L, R, I1, IC, ICP, nch, want_tsq;
  int d[CPD_MAX_ORDER];     // dims (d[0] = I1)
  long long nf;             // fibres (product of dims 2..L)
  long long nft;            // fibre tiles
  int n2;                   // R * (I2 + ... + IL)
  int rows;                 // I2 + ... + IL (rows of the shared factor and accumulator blocks)
  int roff[CPD_MAX_ORDER];  // first row of mode l (l >= 1) in those blocks
  long long budget;         // wait budget in SM clock cycles
  // division of fibre indices (< 2^31) by d[l] as (x * dm[l]) >> dk[l] (exact; see div_magic)
  unsigned long long dm[CPD_MAX_ORDER];
  int dk[CPD_MAX_ORDER];
  // shared-memory layout (bytes from the 1024-aligned base)
  uint32_t o_kr, o_w1s, o_w1q, o_t, stage, o_w, o_g, o_bar;   // stage: bytes per stage
};

// Longest suspension of a waiting thread per try (it resumes when the phase
// completes); also the delay with which a waiter notices another role's abort.
constexpr uint32_t kSuspendNs = 20000;

// Bounded wait on phase `parity`: false when the wait took more than `budget`
// SM clock cycles (also when the phase completed during the suspension that
// overran the budget) or another role has aborted (pass a flag that stays zero
// to ignore aborts, as the teardown's drains do).
__device__ __forceinline__ bool wait_bar(uint32_t bar, uint32_t parity, long long budget,
                                         volatile int* abort_flag) {
  const long long t0 = clock64();
  for (;;) {
    const bool done = mbar_try_hint(bar, parity, kSuspendNs);
    if (clock64() - t0 > budget) return false;
    if (done) return true;
    if (*abort_flag) return false;
  }
}

// Bound of the teardown's waits for copies and MMAs still in flight: never the
// caller's (possibly tiny) budget, so that no copy lands in a CTA that has exited.
constexpr long long kDrainBudget = 1ll << 31;

__device__ __forceinline__ void arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// x = hi + mid + lo, each BF16 (round to nearest): 24 significant bits.
__device__ __forceinline__ void split3(float x, float& h, float& m, float& l) {
  h = __bfloat162float(__float2bfloat16_rn(x));
  const float r1 = x - h;
  m = __bfloat162float(__float2bfloat16_rn(r1));
  l = r1 - m;
}

__device__ __forceinline__ uint32_t pack2(float a, float b) {
  __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<uint32_t*>(&h);
}

// x / d[l] for x < 2^31 by a multiply and a shift: with k = 31 + ceil(log2 d)
// and m = ceil(2^k / d), floor(x m / 2^k) = floor(x / d) since x (m d - 2^k)
// < 2^31 d <= 2^k (Granlund and Montgomery, "Division by invariant integers
// using multiplication", 1994); x m < 2^64.
__device__ __forceinline__ unsigned div_l(const TcPassArgs& a, unsigned x, int l) {
  return (unsigned)(((unsigned long long)x * a.dm[l]) >> a.dk[l]);
}

// Indices (i_2, ..., i_L) of fibre F < 2^31 (F = i_2 + I_2 (i_3 + I_3 i_4));
// returns F / I_2 (the index of the run of fibres sharing i_3, ..., i_L).
template <int L>
__device__ __forceinline__ unsigned fibre_index(const TcPassArgs& a, unsigned F, int (&il)[CPD_MAX_ORDER]) {
  unsigned rem = F, q1 = 0;
#pragma unroll
  for (int l = 1; l < L; ++l) {
    const unsigned q = div_l(a, rem, l);
    il[l] = (int)(rem - q * (unsigned)a.d[l]);
    if (l == 1) q1 = q;
    rem = q;
  }
  return q1;
}

// The factor rows of modes 2..L and their gradient accumulators sit in shared
// memory rank-minor, 16 floats (kRP ranks) per row, rows of mode l after those
// of modes 2..l-1.  Factor rows are read as four-rank float4 groups by lanes of
// consecutive rows: group g of row i is stored at group g ^ ((i >> 1) & 3), so
// that the eight rows of a quarter warp hit eight distinct 16-byte bank groups.
// Accumulators take single-rank atomics from lanes of consecutive rows: rank r
// of row i is stored at position r ^ ((i >> 1) & 15), 32 distinct banks.
__device__ __forceinline__ int ws_quad(int row, int g) { return row * kRP + ((g ^ ((row >> 1) & 3)) << 2); }
__device__ __forceinline__ int ws_at(int row, int r) { return ws_quad(row, r >> 2) + (r & 3); }
__device__ __forceinline__ int gs_at(int row, int r) { return row * kRP + (r ^ ((row >> 1) & 15)); }


// barrier slots (8 bytes each) after o_bar
enum : uint32_t {
  kBarFull = 0,                 // kStages: copy of a stage landed
  kBarEmpty = kStages,          // kStages: the Q / G1 MMAs reading a stage's E^T completed
  kBarKr = 2 * kStages,         // a Khatri-Rao tile written (once per tile)
  kBarTtFull = kBarKr + 1,      // 2: X~ of a unit in tensor memory
  kBarTtFree = kBarTtFull + 2,  // 2: X~ buffer read back
  kBarEFull = kBarTtFree + 2,   // E^T of a unit written
  kBarQg = kBarEFull + 1,       // every MMA of a tile completed (once per tile)
  kBarDrain = kBarQg + 1,       // every MMA of the CTA completed (teardown)
  kNumBars = kBarDrain + 1
};

template <int L>
__global__ void __launch_bounds__(kThreads, 1) k_refine_tc(const __grid_constant__ CUtensorMap tmap, TcPassArgs a) {
  if (a.done && *a.done) return;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t pad = (1024u - (raw & 1023u)) & 1023u;
  unsigned char* sm = smem_raw + pad;
  const uint32_t sb = raw + pad;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int R = a.R, I1 = a.I1, IC = a.IC, ICP = a.ICP, nch = a.nch;
  const uint32_t bar0 = sb + a.o_bar;
  auto BAR = [&](uint32_t i) { return bar0 + 8u * i; };
  uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + a.o_bar + 8 * kNumBars);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(sm + a.o_bar + 8 * kNumBars + 4);
  float* Ws = reinterpret_cast<float*>(sm + a.o_w);      // factor rows of modes 2..L (ws_at)
  float* Gs = reinterpret_cast<float*>(sm + a.o_g);      // their gradient accumulators (gs_at)

  // ---- prologue: operand tiles, factor blocks, barriers, tensor memory ------
  for (uint32_t o = (uint32_t)tid * 16u; o < a.o_t; o += kThreads * 16u)   // KR[2], W1s, W1q zeroed
    *reinterpret_cast<uint4*>(sm + o) = make_uint4(0, 0, 0, 0);
  for (int j = tid; j < a.rows * kRP; j += kThreads) {
    const int row = j / kRP, r = j - row * kRP;
    int l = 1;
    while (l + 1 < L && row >= a.roff[l + 1]) ++l;
    const int i = row - a.roff[l];
    Ws[ws_at(row, r)] = r < R ? a.W[(size_t)I1 * R + (size_t)R * (a.roff[l] - a.roff[1]) + (size_t)r * a.d[l] + i] : 0.f;
    Gs[j] = 0.f;
  }
  if (tid == 0) {
    *abort_flag = 0;
    for (int s = 0; s < kStages; ++s) { mbar_init(BAR(kBarFull + s), 1); mbar_init(BAR(kBarEmpty + s), 1); }
    mbar_init(BAR(kBarKr), kCW);
    for (int b = 0; b < 2; ++b) { mbar_init(BAR(kBarTtFull + b), 1); mbar_init(BAR(kBarTtFree + b), kCW); }
    mbar_init(BAR(kBarEFull), kCW);
    mbar_init(BAR(kBarQg), 1);
    mbar_init(BAR(kBarDrain), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == kCW + 1) tmem_alloc(smem_u32(tslot), kTmemCols);
  __syncthreads();
  // W1 in split parts (X~'s B operand: rows i1 of the chunk, K = rank: hi at
  // bytes 0-31, mid 32-63, lo 64-95) and in BF16 (Q's B operand: rows = rank,
  // K = i1 of the chunk in 64-wide atoms of 2 KB)
  for (int e = tid; e < nch * ICP * kRP; e += kThreads) {
    const int c = e / (ICP * kRP), rem = e - c * ICP * kRP, row = rem / kRP, r = rem - row * kRP;
    const int i1 = c * IC + row;
    const float w = (row < IC && i1 < I1 && r < R) ? a.W[(size_t)r * I1 + i1] : 0.f;
    float h, m, l;
    split3(w, h, m, l);
    unsigned char* t = sm + a.o_w1s + (uint32_t)c * (uint32_t)ICP * 128u;
    *reinterpret_cast<__nv_bfloat16*>(t + sw128_offset(row, 2 * r)) = __float2bfloat16_rn(h);
    *reinterpret_cast<__nv_bfloat16*>(t + sw128_offset(row, 32 + 2 * r)) = __float2bfloat16_rn(m);
    *reinterpret_cast<__nv_bfloat16*>(t + sw128_offset(row, 64 + 2 * r)) = __float2bfloat16_rn(l);
    unsigned char* q = sm + a.o_w1q + (uint32_t)c * 4096u + (uint32_t)(row >> 6) * 2048u;
    *reinterpret_cast<__nv_bfloat16*>(q + sw128_offset(r, 2 * (row & 63))) = __float2bfloat16_rn(w);
  }
  fence_async_smem();
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = *tslot;

  const long long nk = (a.nft - blockIdx.x + gridDim.x - 1) / gridDim.x;   // tiles of this CTA
  const long long nunits = nk * nch;
  const long long budget = a.budget;
  const uint32_t tile_bytes = (uint32_t)kFB * (uint32_t)IC * 4u;
  bool failed = false;
  int zero_flag_storage = 0;
  volatile int* no_abort = &zero_flag_storage;

  if (warp == kCW) {
    // ---- copy issuer -------------------------------------------------------
    if (lane == 0) {
      long long issued = 0;
      for (long long u = 0; u < nunits; ++u) {
        const int s = (int)(u % kStages);
        if (u >= kStages &&
            !wait_bar(BAR(kBarEmpty + s), (uint32_t)(((u / kStages) - 1) & 1), budget, abort_flag)) {
          failed = true;
          break;
        }
        const long long k = u / nch;
        const int c = (int)(u - k * nch);
        const long long ft = (long long)blockIdx.x + k * (long long)gridDim.x;
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(BAR(kBarFull + s)),
                     "r"(tile_bytes)
                     : "memory");
        tma_load_2d(sb + a.o_t + (uint32_t)s * a.stage, &tmap, c * IC, (int)(ft * kFB), BAR(kBarFull + s));
        issued = u + 1;
      }
      if (failed) { *abort_flag = 1; if (a.err) atomicExch(a.err, CPD_ERR_TIMEOUT); }
      // drain: the last copy issued into each stage has landed (bounded, aborts ignored)
      for (int s = 0; s < kStages; ++s) {
        long long ul = -1;
        for (long long u = issued - 1; u >= 0 && u >= issued - kStages; --u)
          if (u % kStages == s) { ul = u; break; }
        if (ul >= 0) wait_bar(BAR(kBarFull + s), (uint32_t)((ul / kStages) & 1), kDrainBudget, no_abort);
      }
    }
  } else if (warp == kCW + 1) {
    // ---- MMA issuer --------------------------------------------------------
    if (lane == 0) {
      const uint32_t id_tt = mma_idesc(128, ICP);
      const uint32_t id_q = mma_idesc(128, kRP);
      const uint32_t id_g1 = mma_idesc_major(128, kRP, true, true);
      const int pa[6] = {0, 0, 1, 0, 2, 1}, pb[6] = {0, 1, 0, 2, 0, 1};
      bool g1_started[2] = {false, false};
      long long tt_issued = 0;
      // X~ of unit u = KR(tile) W1(chunk)^T from the six products of parts
      auto issue_tt = [&](long long u) -> bool {
        const long long k = u / nch;
        const int c = (int)(u - k * nch), b = (int)(u & 1);
        if (c == 0 && !wait_bar(BAR(kBarKr), (uint32_t)(k & 1), budget, abort_flag)) return false;
        if (u >= 2 && !wait_bar(BAR(kBarTtFree + b), (uint32_t)(((u >> 1) - 1) & 1), budget, abort_flag))
          return false;
        fence_after_sync();
        const uint32_t kr = sb + a.o_kr + (uint32_t)(k & 1) * 16384u;
        const uint32_t w1 = sb + a.o_w1s + (uint32_t)c * (uint32_t)ICP * 128u;
#pragma unroll
        for (int j = 0; j < 6; ++j)
          mma_f16(tmem + (uint32_t)b * 128u, sw128_desc(kr + 32u * pa[j]), sw128_desc(w1 + 32u * pb[j]), id_tt,
                  j > 0 ? 1u : 0u);
        mma_commit(BAR(kBarTtFull + b));
        return true;
      };
      for (long long u = 0; u < nunits && !failed; ++u) {
        // X~ one unit ahead, so that it runs while the compute warps work on unit u
        while (tt_issued < nunits && tt_issued <= u + 1) {
          if (!issue_tt(tt_issued)) { failed = true; break; }
          ++tt_issued;
        }
        if (failed) break;
        if (!wait_bar(BAR(kBarEFull), (uint32_t)(u & 1), budget, abort_flag)) { failed = true; break; }
        fence_after_sync();
        const long long k = u / nch;
        const int c = (int)(u - k * nch), s = (int)(u % kStages);
        const uint32_t et = sb + a.o_t + (uint32_t)s * a.stage;
        const uint32_t kr = sb + a.o_kr + (uint32_t)(k & 1) * 16384u;
        const uint32_t dq = tmem + kColQ + 16u * (uint32_t)(k & 1);
        for (int kk = 0; kk < ICP / 16; ++kk)
          mma_f16(dq, sw128_desc(et + (uint32_t)(kk >> 2) * 16384u + (uint32_t)(kk & 3) * 32u),
                  sw128_desc(sb + a.o_w1q + (uint32_t)c * 4096u + (uint32_t)(kk >> 2) * 2048u + (uint32_t)(kk & 3) * 32u),
                  id_q, (c > 0 || kk > 0) ? 1u : 0u);
#pragma unroll
        for (int ks = 0; ks < kFB / 16; ++ks)
          mma_f16(tmem + kColG1 + 16u * (uint32_t)c, sw128_desc_mn(et + (uint32_t)ks * 2048u, 16384u, 1024u),
                  sw128_desc_mn(kr + (uint32_t)ks * 2048u, 16384u, 1024u), id_g1, (g1_started[c] || ks > 0) ? 1u : 0u);
        g1_started[c] = true;
        mma_commit(BAR(kBarEmpty + s));            // the stage (its E^T) can be refilled
        if (c == nch - 1) mma_commit(BAR(kBarQg));  // the tile's Q is complete, its KR buffer free
      }
      if (failed) { *abort_flag = 1; if (a.err) atomicExch(a.err, CPD_ERR_TIMEOUT); }
      // drain: every MMA issued has completed (bounded, aborts ignored)
      mma_commit(BAR(kBarDrain));
      wait_bar(BAR(kBarDrain), 0u, kDrainBudget, no_abort);
    }
  } else {
    // ---- compute warps -----------------------------------------------------
    static_assert(kRG == 4, "a warp group writes 4 ranks (8 bytes of each BF16 part)");
    constexpr int kMaxChunks = 128 / 8 / kNG;          // 8-column chunks of X~ per thread
    const int q4 = warp & 3, g = warp >> 2;
    const int fl = 32 * q4 + lane;                       // fibre of the tile = tensor-memory lane
    const uint32_t lane_base = (uint32_t)(32 * q4) << 16;
    const int nchunk = ICP / 8;
    const bool rank_group = kRG * g < R;                 // this warp's ranks hold any of the R
    // ||e||^2 and ||x||^2 of this thread's elements: per-unit FP32 partials
    // summed across units with Neumaier's compensation (FP64 instructions in
    // the tile loop would cost more than the loop's arithmetic)
    float esq_s = 0.f, esq_c = 0.f, tsq_s = 0.f, tsq_c = 0.f;
    auto acc2 = [](float& sum, float& comp, float x) {
      const float t = sum + x;
      comp += fabsf(sum) >= fabsf(x) ? (sum - t) + x : (x - t) + sum;
      sum = t;
    };
    auto cbar = []() { asm volatile("bar.sync 1, %0;" ::"n"(32 * kCW) : "memory"); };
    auto wwait = [&](uint32_t bar, uint32_t parity) {
      const bool ok = failed ? false : wait_bar(bar, parity, budget, abort_flag);
      if (!__all_sync(0xffffffffu, ok) && !failed) { failed = true; *abort_flag = 1; }
    };
    // ranks 4g .. 4g + 3 of factor row i of mode l (zero beyond R)
    auto wrow = [&](int l, int i) {
      return *reinterpret_cast<const float4*>(Ws + ws_quad(a.roff[l] + i, g));
    };

    // Khatri-Rao row of fibre fl of tile ft into buffer kb: ranks 4g .. 4g + 3
    // in three BF16 parts
    auto khatri_rao = [&](long long ft, int kb) {
      const long long F = ft * kFB + fl;
      float kr[kRG] = {0.f, 0.f, 0.f, 0.f};
      if (F < a.nf && rank_group) {
        int il[CPD_MAX_ORDER];
        fibre_index<L>(a, (unsigned)F, il);
        float4 p = wrow(1, il[1]);
#pragma unroll
        for (int l = 2; l < L; ++l) {
          const float4 w = wrow(l, il[l]);
          p.x *= w.x; p.y *= w.y; p.z *= w.z; p.w *= w.w;
        }
        kr[0] = p.x; kr[1] = p.y; kr[2] = p.z; kr[3] = p.w;
      }
      float hp[kRG], mp[kRG], lp[kRG];
#pragma unroll
      for (int j = 0; j < kRG; ++j) split3(kr[j], hp[j], mp[j], lp[j]);
      unsigned char* t = sm + a.o_kr + (uint32_t)kb * 16384u;
      const uint32_t b0 = 2u * kRG * (uint32_t)g;
      *reinterpret_cast<uint2*>(t + sw128_offset(fl, b0)) = make_uint2(pack2(hp[0], hp[1]), pack2(hp[2], hp[3]));
      *reinterpret_cast<uint2*>(t + sw128_offset(fl, 32u + b0)) = make_uint2(pack2(mp[0], mp[1]), pack2(mp[2], mp[3]));
      *reinterpret_cast<uint2*>(t + sw128_offset(fl, 64u + b0)) = make_uint2(pack2(lp[0], lp[1]), pack2(lp[2], lp[3]));
    };

    // residual of unit (stage s, X~ buffer b) into registers: e = x - x~ in
    // BF16 pairs, ||e||^2 (and with TSQ ||x||^2) accumulated; two chunks per
    // tensor-memory wait
    auto residual = [&](int s, int b, uint4 (&pk)[kMaxChunks], auto tsq_tag) {
      constexpr bool TSQ = decltype(tsq_tag)::value;
      const float* xr = reinterpret_cast<const float*>(sm + a.o_t + (uint32_t)s * a.stage) + (size_t)fl * IC;
      const uint32_t dtt = tmem + lane_base + (uint32_t)b * 128u;
      float esf = 0.f, tsf = 0.f;
#pragma unroll
      for (int m = 0; m < kMaxChunks; m += 2) {
        const int j0 = g + kNG * m, j1 = g + kNG * (m + 1);
        if (j0 < nchunk) {                     // the same for every lane of the warp
          float tt[2][8];
          tmem_ld8(dtt + 8u * (uint32_t)j0, tt[0]);
          if (j1 < nchunk) tmem_ld8(dtt + 8u * (uint32_t)j1, tt[1]);
          float4 x[2][2];
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int i0 = 8 * (h == 0 ? j0 : j1);
            const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
            x[h][0] = i0 < IC ? *reinterpret_cast<const float4*>(xr + i0) : z4;
            x[h][1] = i0 + 4 < IC ? *reinterpret_cast<const float4*>(xr + i0 + 4) : z4;
          }
          tmem_ld_wait();
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            if (h == 1 && j1 >= nchunk) break;
            const float xv[8] = {x[h][0].x, x[h][0].y, x[h][0].z, x[h][0].w,
                                 x[h][1].x, x[h][1].y, x[h][1].z, x[h][1].w};
            float e[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
              e[u] = xv[u] - tt[h][u];
              esf = fmaf(e[u], e[u], esf);
              if (TSQ) tsf = fmaf(xv[u], xv[u], tsf);
            }
            pk[m + h] = make_uint4(pack2(e[0], e[1]), pack2(e[2], e[3]), pack2(e[4], e[5]), pack2(e[6], e[7]));
          }
        }
      }
      acc2(esq_s, esq_c, esf);
      if (TSQ) acc2(tsq_s, tsq_c, tsf);
    };

    // scatter Q of tile ft (tensor-memory buffer qb) into the modes 2..L
    // accumulators.  Mode 2: each fibre adds its term q_fr prod_{l>=3}
    // W_l[i_l, r] with a shared atomic (the fibres of one i2 in a tile are
    // I2 apart, so the atomics of a warp rarely collide).  Modes 3..L: the
    // values q_fr W_2[i2, r] of a run of fibres with the same (i3, ..., iL)
    // (consecutive lanes) are summed over the warp and added once per run.
    // With at most two runs in the warp (I2 >= 31, or the warp inside one
    // run) the eight sums (two runs x four ranks) come out of one transposing
    // butterfly (9 shuffles, lane 4v ends with sum v); otherwise a segmented
    // shuffle reduction per rank.
    auto scatter = [&](long long ft, int qb) {
      if (!rank_group || failed) return;                 // warp-uniform
      float qv[kRG];
      tmem_ld4(tmem + lane_base + kColQ + 16u * (uint32_t)qb + (uint32_t)(kRG * g), qv);
      tmem_ld_wait();
      const long long F = ft * kFB + fl;
      const bool valid = F < a.nf;
      int il[CPD_MAX_ORDER] = {0, 0, 0, 0};
      unsigned run = 0;
      if (valid) run = fibre_index<L>(a, (unsigned)F, il);
      float sv[kRG] = {0.f, 0.f, 0.f, 0.f};
      if (valid) {
        const float4 w2 = wrow(1, il[1]);
        float4 p = wrow(2, il[2]);
        if constexpr (L == 4) {
          const float4 w4 = wrow(3, il[3]);
          p.x *= w4.x; p.y *= w4.y; p.z *= w4.z; p.w *= w4.w;
        }
        const int row2 = a.roff[1] + il[1];
        atomicAdd(&Gs[gs_at(row2, kRG * g + 0)], qv[0] * p.x);
        atomicAdd(&Gs[gs_at(row2, kRG * g + 1)], qv[1] * p.y);
        atomicAdd(&Gs[gs_at(row2, kRG * g + 2)], qv[2] * p.z);
        atomicAdd(&Gs[gs_at(row2, kRG * g + 3)], qv[3] * p.w);
        sv[0] = qv[0] * w2.x; sv[1] = qv[1] * w2.y; sv[2] = qv[2] * w2.z; sv[3] = qv[3] * w2.w;
      }
      // runs of the warp: lanes past the end form one run of their own (their values are 0)
      const unsigned key = valid ? run : 0xffffffffu;
      const unsigned prevk = __shfl_up_sync(0xffffffffu, key, 1);
      const bool head = lane == 0 || prevk != key;
      const unsigned heads = __ballot_sync(0xffffffffu, head);
      // add a run's sum s (rank r) into G_3 .. G_L; (i3, i4) are the run's
      auto add_run = [&](float s, int r, int i3, int i4) {
        if constexpr (L == 3) {
          atomicAdd(&Gs[gs_at(a.roff[2] + i3, r)], s);
        } else {
          atomicAdd(&Gs[gs_at(a.roff[2] + i3, r)], s * Ws[ws_at(a.roff[3] + i4, r)]);
          atomicAdd(&Gs[gs_at(a.roff[3] + i4, r)], s * Ws[ws_at(a.roff[2] + i3, r)]);
        }
      };
      if (__popc(heads) <= 2) {
        const int h1 = heads == 1u ? 32 : __ffs(heads & ~1u) - 1;   // first lane of the second run
        const bool first = lane < h1;
        float v[8];
#pragma unroll
        for (int j = 0; j < kRG; ++j) { v[j] = first ? sv[j] : 0.f; v[kRG + j] = first ? 0.f : sv[j]; }
        const bool b4 = (lane & 16) != 0, b3 = (lane & 8) != 0, b2 = (lane & 4) != 0;
        float w[4], x[2];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const float send = b4 ? v[i] : v[i + 4], keep = b4 ? v[i + 4] : v[i];
          w[i] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
        }
#pragma unroll
        for (int i = 0; i < 2; ++i) {
          const float send = b3 ? w[i] : w[i + 2], keep = b3 ? w[i + 2] : w[i];
          x[i] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
        }
        float y;
        {
          const float send = b2 ? x[0] : x[1], keep = b2 ? x[1] : x[0];
          y = keep + __shfl_xor_sync(0xffffffffu, send, 4);
        }
        y += __shfl_xor_sync(0xffffffffu, y, 2);
        y += __shfl_xor_sync(0xffffffffu, y, 1);
        // lane 4v holds the sum of value v = 4 * run + rank-in-group
        const int src = b4 ? (h1 & 31) : 0;
        const int i3 = __shfl_sync(0xffffffffu, il[2], src);
        const int i4 = __shfl_sync(0xffffffffu, L == 4 ? il[3] : 0, src);
        const bool run_valid = __shfl_sync(0xffffffffu, (int)valid, src) != 0 && (!b4 || h1 < 32);
        const int r = kRG * g + ((lane >> 2) & 3);
        if ((lane & 3) == 0 && run_valid && r < R) add_run(y, r, i3, i4);
      } else {
        const unsigned le = lane == 31 ? 0xffffffffu : ((2u << lane) - 1u);
        const int seg = __popc(heads & le);
#pragma unroll
        for (int j = 0; j < kRG; ++j) {
          float s = sv[j];
#pragma unroll
          for (int o = 1; o < 32; o <<= 1) {
            const float pv = __shfl_down_sync(0xffffffffu, s, o);
            const int ps = __shfl_down_sync(0xffffffffu, seg, o);
            if (lane + o < 32 && ps == seg) s += pv;
          }
          const int r = kRG * g + j;
          if (valid && head && r < R) add_run(s, r, il[2], L == 4 ? il[3] : 0);
        }
      }
    };

    // tile k: the next tile's Khatri-Rao rows (once every MMA of tile k-1 is
    // done), the residual of each chunk of tile k, then tile k-1's scatter
    auto tile = [&](long long k) { return (long long)blockIdx.x + k * (long long)gridDim.x; };
    if (nk > 0) {
      khatri_rao(tile(0), 0);
      fence_async_smem();
      __syncwarp();
      if (lane == 0) arrive(BAR(kBarKr));
    }
    for (long long k = 0; k < nk; ++k) {
      if (k >= 1) {
        wwait(BAR(kBarQg), (uint32_t)((k - 1) & 1));
        fence_after_sync();
      }
      if (k + 1 < nk) {
        khatri_rao(tile(k + 1), (int)((k + 1) & 1));
        fence_async_smem();
        __syncwarp();
        if (lane == 0) arrive(BAR(kBarKr));
      }
      for (int c = 0; c < nch; ++c) {
        const long long u = k * nch + c;
        const int s = (int)(u % kStages), b = (int)(u & 1);
        wwait(BAR(kBarFull + s), (uint32_t)((u / kStages) & 1));
        wwait(BAR(kBarTtFull + b), (uint32_t)((u >> 1) & 1));
        fence_after_sync();
        uint4 pk[kMaxChunks];
        if (a.want_tsq) residual(s, b, pk, std::true_type{});
        else residual(s, b, pk, std::false_type{});
        fence_before_sync();
        cbar();                                   // the stage's block has been read by every warp
        unsigned char* et = sm + a.o_t + (uint32_t)s * a.stage;
#pragma unroll
        for (int m = 0; m < kMaxChunks; ++m) {
          const int j = g + kNG * m;
          if (j < nchunk) {
            const int i0 = 8 * j;
            *reinterpret_cast<uint4*>(et + (uint32_t)(i0 >> 6) * 16384u + sw128_offset(fl, 2u * (uint32_t)(i0 & 63))) = pk[m];
          }
        }
        fence_async_smem();
        __syncwarp();
        if (lane == 0) {
          arrive(BAR(kBarTtFree + b));
          arrive(BAR(kBarEFull));
        }
      }
      if (k >= 1) scatter(tile(k - 1), (int)((k - 1) & 1));
    }
    if (nk > 0) {
      wwait(BAR(kBarQg), (uint32_t)((nk - 1) & 1));
      fence_after_sync();
      scatter(tile(nk - 1), (int)((nk - 1) & 1));
    }

    // ---- epilogue: G1 from tensor memory, G_2..G_L from shared memory, norms
    cbar();
    const bool aborted = *abort_flag != 0;
    if (!aborted && nk > 0) {
      for (int c = 0; c < nch; ++c) {
        float v[kRG];
        tmem_ld4(tmem + lane_base + kColG1 + 16u * (uint32_t)c + (uint32_t)(kRG * g), v);
        tmem_ld_wait();
        const int i1 = c * IC + fl;
        if (fl < IC && i1 < I1) {
#pragma unroll
          for (int j = 0; j < kRG; ++j) {
            const int r = kRG * g + j;
            if (r < R && v[j] != 0.f) atomicAdd(a.G + (size_t)r * I1 + i1, v[j]);
          }
        }
      }
    }
    if (!aborted)
      for (int j = tid; j < a.rows * kRP; j += 32 * kCW) {
        const int row = j / kRP, r = j - row * kRP;
        if (r >= R) continue;
        const float v = Gs[gs_at(row, r)];
        if (v == 0.f) continue;
        int l = 1;
        while (l + 1 < L && row >= a.roff[l + 1]) ++l;
        atomicAdd(a.G + (size_t)I1 * R + (size_t)R * a.roff[l] + (size_t)r * a.d[l] + (row - a.roff[l]), v);
      }
    double esq_d = (double)esq_s + (double)esq_c, tsq_d = (double)tsq_s + (double)tsq_c;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      esq_d += __shfl_xor_sync(0xffffffffu, esq_d, o);
      tsq_d += __shfl_xor_sync(0xffffffffu, tsq_d, o);
    }
    if (lane == 0 && !aborted) {
      atomicAdd(a.esq, esq_d);
      if (a.want_tsq) atomicAdd(a.esq + 1, tsq_d);
    }
    if (failed && a.err) atomicExch(a.err, CPD_ERR_TIMEOUT);
  }
  fence_before_sync();
  __syncthreads();
  if (warp == kCW + 1) tmem_dealloc(tmem, kTmemCols);
}

}  // namespace

// ---- host side ----------------------------------------------------------------

namespace {

struct TcPlan {
  int IC = 0, ICP = 0, nch = 0, n2 = 0, rows = 0;
  long long nf = 0;
  uint32_t o_kr = 0, o_w1s = 0, o_w1q = 0, o_t = 0, stage = 0, o_w = 0, o_g = 0, o_bar = 0;
  size_t smem = 0;
};

// Row chunks of at most 128 rows (one tensor-memory lane per row for G1),
// chunk length a multiple of 4 (16-byte rows of the copy); with two or more
// chunks an odd number of 16-byte groups per stage row, so that the residual's
// row reads (one fibre per lane) fall in distinct bank groups.  A stage holds
// the copied block and then the unit's E^T (two 16 KB atoms).
bool tc_plan(int L, const long long* dims, int R, TcPlan& p) {
  if ((L != 3 && L != 4) || R < 1 || R > kRP) return false;
  const long long I1 = dims[0];
  if (I1 < 4 || I1 % 4 != 0 || I1 > 256) return false;
  p.nch = (int)((I1 + 127) / 128);
  p.IC = (int)(((I1 + p.nch - 1) / p.nch + 3) / 4 * 4);
  if (p.nch > 1 && p.IC % 8 == 0 && p.IC + 4 <= 128) p.IC += 4;
  if (p.IC > 128 || (long long)(p.nch - 1) * p.IC >= I1) return false;
  p.ICP = (p.IC + 15) / 16 * 16;
  p.nf = 1;
  p.n2 = 0;
  for (int l = 1; l < L; ++l) {
    if (dims[l] < 1) return false;
    p.nf *= dims[l];
    p.n2 += (int)dims[l] * R;
    p.rows += (int)dims[l];
  }
  if (p.nf >= (1ll << 31) - kFB) return false;
  auto up = [](size_t x, size_t a) { return (x + a - 1) / a * a; };
  size_t o = 0;
  p.o_kr = (uint32_t)o; o += 2 * 16384;
  p.o_w1s = (uint32_t)o; o += (size_t)p.nch * p.ICP * 128;
  p.o_w1q = (uint32_t)o; o += (size_t)p.nch * 4096;
  o = up(o, 1024);
  p.o_t = (uint32_t)o;
  const size_t tile = (size_t)kFB * p.IC * 4;
  p.stage = (uint32_t)up(tile > 32768 ? tile : 32768, 1024);
  o += (size_t)kStages * p.stage;
  p.o_w = (uint32_t)o; o += (size_t)p.rows * kRP * 4;
  p.o_g = (uint32_t)o; o += (size_t)p.rows * kRP * 4;
  p.o_bar = (uint32_t)up(o, 8); o = p.o_bar + 8 * kNumBars + 16;
  p.smem = up(o, 16) + 1024;                 // + the alignment of the base to 1024 bytes
  return p.smem <= (size_t)227 * 1024;
}

struct TcLaunchCache {
  std::mutex mu;
  int dev = -1;
  size_t smem3 = 0, smem4 = 0;
  int sms = 0;
};
TcLaunchCache g_tc_cache;

template <int L>
cudaError_t launch_tc_t(const CUtensorMap& map, const TcPassArgs& a, size_t smem, int grid, cudaStream_t st) {
  k_refine_tc<L><<<grid, kThreads, smem, st>>>(map, a);
  count_launch();
  return cudaGetLastError();
}

}  // namespace

bool refine_tc_supported(int L, const long long* dims, int R, const float* T) {
  TcPlan p;
  if (!tc_plan(L, dims, R, p)) return false;
  if ((reinterpret_cast<uintptr_t>(T) & 15u) != 0) return false;
  return tensor_map_encoder() != nullptr;
}

cudaError_t launch_refine_tc(const RefinePassArgs& a, cudaStream_t st) {
  TcPlan p;
  if (!tc_plan(a.L, a.dims, a.R, p)) return cudaErrorInvalidValue;
  auto enc = tensor_map_encoder();
  if (enc == nullptr) return cudaErrorNotSupported;
  // the fibre matrix X (I1 x nf, column stride I1 floats), boxes of IC rows x 128 fibres
  CUtensorMap map;
  cuuint64_t gdim[2] = {(cuuint64_t)a.dims[0], (cuuint64_t)p.nf};
  cuuint64_t gstride[1] = {(cuuint64_t)a.dims[0] * 4};
  cuuint32_t box[2] = {(cuuint32_t)p.IC, (cuuint32_t)kFB};
  cuuint32_t estr[2] = {1, 1};
  if (enc(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(a.T), gdim, gstride, box, estr,
          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return cudaErrorInvalidValue;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  int sms = 0;
  {
    std::lock_guard<std::mutex> lk(g_tc_cache.mu);
    if (g_tc_cache.dev != dev) { g_tc_cache.dev = dev; g_tc_cache.smem3 = g_tc_cache.smem4 = 0; g_tc_cache.sms = 0; }
    size_t& have = a.L == 3 ? g_tc_cache.smem3 : g_tc_cache.smem4;
    if (have < p.smem) {
      e = a.L == 3 ? cudaFuncSetAttribute(k_refine_tc<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p.smem)
                   : cudaFuncSetAttribute(k_refine_tc<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p.smem);
      if (e != cudaSuccess) return e;
      have = p.smem;
    }
    if (g_tc_cache.sms == 0) {
      e = cudaDeviceGetAttribute(&g_tc_cache.sms, cudaDevAttrMultiProcessorCount, dev);
      if (e != cudaSuccess) return e;
    }
    sms = g_tc_cache.sms;
  }
  TcPassArgs t{};
  t.W = a.W; t.G = a.G; t.esq = a.esq; t.done = a.done; t.err = a.err;
  t.L = a.L; t.R = a.R; t.I1 = (int)a.dims[0]; t.IC = p.IC; t.ICP = p.ICP; t.nch = p.nch; t.want_tsq = a.want_tsq;
  for (int l = 0; l < CPD_MAX_ORDER; ++l) t.d[l] = l < a.L ? (int)a.dims[l] : 1;
  t.nf = p.nf;
  t.nft = (p.nf + kFB - 1) / kFB;
  t.n2 = p.n2;
  t.budget = a.budget > 0 ? a.budget : (1ll << 31);
  for (int l = 0; l < CPD_MAX_ORDER; ++l) {
    const unsigned long long d = (unsigned long long)t.d[l];
    int s = 0;
    while ((1ull << s) < d) ++s;                       // ceil(log2 d)
    t.dk[l] = 31 + s;
    t.dm[l] = ((1ull << t.dk[l]) + d - 1) / d;
  }
  t.o_kr = p.o_kr; t.o_w1s = p.o_w1s; t.o_w1q = p.o_w1q; t.o_t = p.o_t; t.stage = p.stage;
  t.o_w = p.o_w; t.o_g = p.o_g; t.o_bar = p.o_bar;
  t.rows = p.rows;
  for (int l = 0, acc = 0; l < CPD_MAX_ORDER; ++l) {
    t.roff[l] = l >= 1 ? acc : 0;
    if (l >= 1 && l < a.L) acc += (int)a.dims[l];
  }
  const long long grid = t.nft < sms ? t.nft : sms;     // one CTA per SM, persistent over the tiles
  return a.L == 3 ? launch_tc_t<3>(map, t, p.smem, (int)grid, st) : launch_tc_t<4>(map, t, p.smem, (int)grid, st);
}

}  // namespace cpdk
