/*
 * cpd.h — C ABI of the GB300 (sm_103a) CPD library: truncated MLSVD
 * compression followed by damped Gauss-Newton (dGN) on the compressed core,
 * after F. Bottega Diniz, "Tensor decompositions and algorithms, with
 * applications to tensor learning" (thesis, 2019; arXiv 2110.05997).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Tensors are dense and column-major: entry (i1, ..., iL) (0-based) sits at
 *    i1 + I1*(i2 + I2*(i3 + ...)), i.e. i1 fastest, the order in which the
 *    thesis unfolds tensors (Sec. 2.1.1, Algorithm "Unfolding").
 *  - A CPD with factors W^(l) (I_l x R, column-major) is passed as ONE buffer
 *    holding vec(W^(1)), ..., vec(W^(L)) back to back: the stacked parameter
 *    vector w of Sec. 3.1.  Block l starts at R * (I_1 + ... + I_{l-1}).
 *  - Every tensor / factor / output pointer is a DEVICE pointer owned by the
 *    caller; the library never allocates, frees or retains caller memory.
 *    Scratch memory is the caller's `workspace` of at least the number of
 *    bytes cpd_workspace_size() returns (256-byte aligned).
 *  - Work is enqueued on `stream` (a cudaStream_t passed as void*; NULL = the
 *    legacy default stream).  Calls that fill a host `cpd_info` synchronise
 *    that stream before returning; everything else is stream-ordered.
 *  - Arguments are validated before anything is launched; a validation
 *    failure returns CPD_ERR_INVALID_ARG or CPD_ERR_UNSUPPORTED and touches
 *    nothing.  A CUDA error returns CPD_ERR_CUDA.  Non-convergence is not an
 *    error: it is stop_reason CPD_STOP_MAXITER.  NaN/Inf met during the
 *    iteration ends it with info.status = CPD_ERR_NUMERIC.
 *  - Distinct workspaces make concurrent calls on distinct streams safe.
 *  - Supported orders: L = 3 and L = 4.  Ranks 1 <= R <= 64.
 */
#ifndef CPD_H_
#define CPD_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define CPD_MAX_ORDER 4
#define CPD_MAX_RANK 64

typedef enum {
  CPD_OK = 0,
  CPD_ERR_INVALID_ARG = -1,
  CPD_ERR_CUDA = -2,
  CPD_ERR_WORKSPACE = -3,
  CPD_ERR_NUMERIC = -4,
  CPD_ERR_TIMEOUT = -5,
  CPD_ERR_UNSUPPORTED = -6
} cpd_status;

/* Stop tests of Sec. 4.1.3 ("Stopping conditions"), in the printed order. */
typedef enum {
  CPD_STOP_NONE = 0,
  CPD_STOP_REL_ERR = 1,          /* ||S - S_k|| / ||S|| < tol               */
  CPD_STOP_STEP = 2,             /* ||w_{k-1} - w_k|| < tol                 */
  CPD_STOP_IMPROVEMENT = 3,      /* |e_{k-1} - e_k| < tol                   */
  CPD_STOP_GRAD = 4,             /* ||grad F||_inf < tol                    */
  CPD_STOP_AVG_ERR = 5,          /* windowed average error stalls           */
  CPD_STOP_AVG_IMPROVEMENT = 6,  /* windowed improvement < 1e-3 * error     */
  CPD_STOP_DIVERGENCE = 7,       /* e_k > max(1,||S||^2) / (1e-16 + tol)    */
  CPD_STOP_MAXITER = 8
} cpd_stop_reason;

/* Initialisation (Sec. 4.1.2). */
typedef enum {
  CPD_INIT_MLSVD = 0,   /* R core entries of largest |s| as rank-one terms          */
  CPD_INIT_RANDOM = 1,  /* N(0,1) by Box-Muller on SplitMix64 stream 2 of `seed`    */
  CPD_INIT_GIVEN = 2,   /* caller's W0 in the ORIGINAL space (projected under compression) */
  CPD_INIT_LEARNED = 3  /* the learned initialiser's factors for the core when their
                           residual is below half the MLSVD start's, else the MLSVD
                           start (batched solver only: cpd_batch_solve_learned; no
                           counterpart in the thesis) */
} cpd_init;

/* Arithmetic of the compression Gram matrices. */
typedef enum {
  CPD_GRAM_FP32 = 0,    /* FP32 CUDA-core Gram                                   */
  CPD_GRAM_BF16 = 1     /* BF16 tcgen05 tensor-core Gram, FP32 accumulate (mode 1,
                           I_1 <= 256, T 16-byte aligned, else CPD_ERR_UNSUPPORTED);
                           accuracy is won back by refinement in the original space */
} cpd_gram_precision;

/* Preconditioner of the CG inside each dGN iteration. */
typedef enum {
  CPD_PRECOND_JACOBI = 0,  /* the diagonal M of Sec. 4.8 (the thesis's choice)              */
  CPD_PRECOND_BLOCK = 1    /* block-Jacobi: the exact diagonal blocks (Pi^(l) + mu diag
                              gamma^(l)) (x) I of J^T J + mu D (Sec. 3.5.3, corollary on the
                              diagonal blocks), inverted per mode by an FP64 R x R Cholesky
                              factorisation; R <= 32, else CPD_ERR_UNSUPPORTED.  The batched
                              solver always uses the diagonal one. */
} cpd_precond;

/* Element type of the input tensor. */
typedef enum { CPD_F32 = 0, CPD_F64 = 1 } cpd_dtype;

/* Options; cpd_default_options() fills the thesis's defaults. */
typedef struct {
  int maxiter;          /* 200: dGN iteration cap (Sec. 4.1.3 "Main parameters")   */
  double tol;           /* 1e-6: every stop test and the CG test ||r||^2 < tol    */
  double tau;           /* 1.0: mu0 = tau * mean|S| (Sec. 4.1.3)                  */
  double cg_a, cg_b;    /* 0.4, 0.9: cg_maxiter ~ U[1+ceil(k^a), 2+ceil(k^b)] (Sec. 4.1.3, 4.4) */
  double mlsvd_tol;     /* 1e-6: truncation tolerance (Algorithm "Compression") */
  int st_mlsvd;         /* 1: sequentially truncated MLSVD; 0: classic MLSVD     */
  int compress;         /* 1: compress then dGN on the core; 0: dGN on T itself  */
  int init;             /* cpd_init                                              */
  int gram_precision;   /* cpd_gram_precision                                    */
  int refine_maxiter;   /* dGN iterations on T after uncompression (0 = none)   */
  uint64_t seed;        /* SplitMix64 seed for cg_maxiter (stream 1) and init    */
  int block_threads;    /* threads of the single-CTA solver kernels (0 = auto)   */
  double mu_min;        /* 1e-5: floor of the damping parameter after each update.
                           The solvers run the CG in FP32; once mu falls far below
                           the FP32 unit roundoff (~6e-8) relative to J^T J, the
                           rounding of J^T J v is amplified by ~1/mu along the
                           scaling null space of J^T J (Theorem "J^T J is
                           singular", Sec. 3.5) and the step overflows.  The floor
                           keeps that amplification below ~1e-2.  0 = the thesis's
                           rule alone (mu x3 / mu /3, Sec. 4.1.3 "Updates"). */
  long long timeout_cycles;  /* bound of every device-side wait on an mbarrier of
                           the tensor-core kernels, in SM clock cycles (0 = the
                           default of 2^31 cycles, about one second); a wait that
                           runs out ends the call with CPD_ERR_TIMEOUT */
  int precond;          /* cpd_precond: CPD_PRECOND_JACOBI                        */
} cpd_options;

/* Outcome of one CPD. */
typedef struct {
  int status;           /* cpd_status of this item                               */
  int iters;            /* dGN iterations on the core (or on T if compress = 0)  */
  int stop_reason;      /* cpd_stop_reason of that stage                         */
  int cg_total;         /* CG iterations of that stage                           */
  double rel_err;       /* last ||S - S_k|| / ||S|| of that stage                */
  double mu;            /* damping parameter after the last iteration            */
  double grad_inf;      /* ||grad F||_inf at the last iterate                    */
  int core_dims[CPD_MAX_ORDER];  /* truncated multilinear rank (or dims of T)    */
  int refine_iters;     /* refinement iterations run                             */
  int refine_stop_reason;
  int refine_cg_total;
  int init_used;        /* 1 when dGN started from the learned initialiser's factors */
  double refine_rel_err;  /* ||T - T_k|| / ||T|| after refinement (FP64-accumulated) */
} cpd_info;

/* Per-iteration trace record (optional, device memory, 8 doubles each):
 * {k, rel_err, mu, gain_ratio, cg_iterations, ||x||, ||grad F||_inf, stage}
 * stage 0 = core dGN, 1 = refinement. */
#define CPD_TRACE_FIELDS 8

void cpd_default_options(cpd_options* opts);
const char* cpd_status_string(int status);

/* Bytes of workspace cpd_compress / cpd_dgn_solve need for this problem. */
size_t cpd_workspace_size(int L, const int64_t* dims, int R, const cpd_options* opts);

/*
 * cpd_compress — truncated MLSVD of T (Algorithm "Compression", Sec. 4.1.1,
 * on Algorithm "MLSVD" or "ST-MLSVD", Sec. 2.2), through the Gram matrices
 * T_(l) T_(l)^T and their leading eigenpairs (App. A).
 *   T           device, FP32, column-major I1 x ... x IL
 *   U_out       device, FP32: L blocks, block l is I_l x P_l column-major,
 *               P_l = min(I_l, R); only the first R~_l columns are meaningful
 *   core_out    device, FP32, prod(P_l) entries: the core, column-major with
 *               the TRUNCATED dims R~_1 x ... x R~_L packed at the start
 *   sigma_out   device, FP32, sum(P_l): leading singular values per mode
 *               (of the sequential unfoldings under ST-MLSVD)
 *   core_dims_out host, L ints: R~_l (synchronises the stream)
 * Singular vectors are sign-normalised (largest-|.| entry positive).
 * Arithmetic: the Grams in FP32 (the first mode's in BF16 on tensor cores
 * with opts->gram_precision = CPD_GRAM_BF16, FP32 accumulation); the first
 * mode's projection on TF32 tensor cores with both operands split into two
 * TF32 parts (FP32-accurate: |error| <= 2^-21 sum |t u|) when 32 <= I1 <= 256,
 * I1 % 4 == 0, N / I1 >= 128, P_1 <= 16 and T is 16-byte aligned, else and
 * for the other modes on the CUDA cores in FP32.  A bounded pipeline wait of
 * a tensor-core kernel that runs out (opts->timeout_cycles) leaves NaN in
 * its output.
 */
int cpd_compress(const float* T, int L, const int64_t* dims, int R, const cpd_options* opts,
                 float* U_out, float* core_out, float* sigma_out, int* core_dims_out,
                 void* workspace, size_t ws_bytes, void* stream);

/*
 * cpd_dgn_solve — the whole method of Fig. "tensorfox-flow" (Sec. 4.1):
 * compression (if opts->compress), initialisation, damped Gauss-Newton on the
 * core (Sec. 4.1.3: residual, MTTKRP gradient, Hadamard-of-Gram Pi matrices,
 * matrix-free J^T J v of Theorem "Hv" inside Jacobi- or block-Jacobi-
 * preconditioned CG with the diagonal regulariser of Sec. 4.8), uncompression
 * (Sec. 4.1.4), optional refinement iterations on T, and output normalisation.
 * Without compression, an FP32 tensor of at least 2^20 entries with a random
 * or given start runs every dGN iteration as one pass over T plus a
 * single-CTA step (the refinement machinery; same limits as refinement).
 *   T          device, element type `dtype` (CPD_F64 only with compress = 0)
 *   W0         device, FP32, stacked I_l x R blocks (INIT_GIVEN), else NULL
 *   W_out      device, FP32, stacked I_l x R blocks with unit columns
 *   lambda_out device, FP32, R weights, descending: T ~ sum_r lambda_r w_r^(1) o ... o w_r^(L)
 *   info       host (synchronises the stream); may be NULL (no sync)
 *   trace      device, CPD_TRACE_FIELDS doubles per iteration, capacity
 *              (maxiter + refine_maxiter) records, or NULL
 * Refinement (refine_maxiter > 0) needs I_1 <= 1024 for R <= 16, <= 512 for
 * R <= 32, <= 256 for R <= 64, a product of I_2..I_L below 2^31, and its
 * pass's shared memory (two copies of the factor blocks of modes 2..L plus
 * I_1 x (33 + padded R) floats) within 227 KB; else CPD_ERR_UNSUPPORTED.
 * On a non-default stream the launch sequence is captured once per argument
 * set into a CUDA graph and replayed; its refinement iterations are the body
 * of a conditional while node, so only the iterations the stop tests allow
 * are launched.
 */
int cpd_dgn_solve(const void* T, int dtype, int L, const int64_t* dims, int R,
                  const cpd_options* opts, const float* W0, float* W_out, float* lambda_out,
                  cpd_info* info, double* trace, void* workspace, size_t ws_bytes,
                  void* stream);

/*
 * cpd_dgn_solve_noalloc — cpd_dgn_solve for callers that cannot give the
 * library a workspace because they may not allocate device memory when they
 * need a CPD: a plugin inside a framework whose allocator owns all device
 * memory, or a latency-critical loop where a cudaMalloc (which can synchronise
 * the device) is not acceptable.  The thesis has no counterpart: this is a
 * packaging of the uncompressed dGN solve.  It allocates nothing; its scratch
 * is a 128 KiB array inside the library, held on every GPU that loads the
 * library until the process exits.
 * Limits: opts->compress = 0 and opts->refine_maxiter = 0, maxiter <= 4096,
 * R * (I_1 + ... + I_L) <= 16384, and T must fit the solver CTA's shared
 * memory; a larger problem returns CPD_ERR_WORKSPACE.  Other arguments and the
 * results are those of cpd_dgn_solve (no trace).  The first call on each
 * device looks up the array's device address (cudaGetSymbolAddress) and must
 * come before any stream capture on that device.  Every call uses the same
 * array and leaves its contents behind: calls whose GPU work can overlap (on
 * different streams or from different host threads) race and must be
 * serialised by the caller.  Launch failures are returned directly; a
 * failure inside the solve (info.status) is only seen when `info` is given,
 * since only then does the call wait for the GPU.
 */
int cpd_dgn_solve_noalloc(const void* T, int dtype, int L, const int64_t* dims, int R,
                          const cpd_options* opts, const float* W0, float* W_out,
                          float* lambda_out, cpd_info* info, void* stream);

/*
 * cpd_batch_solve — B independent third-order CPDs of uneven shapes, each
 * compressed, solved and uncompressed by one CTA of one persistent launch
 * that takes items from a device work queue ordered longest-first.
 *   T_packed   device, FP32: the B tensors back to back, item b at element
 *              offset t_off[b] (host array, B entries)
 *   dims       host, B x 3 ints (I1, I2, I3 per item), each in [2, 64]
 *   ranks      host, B ints in [1, 16]
 *   W_packed   device, FP32 outputs: item b's stacked factors at element
 *              offset w_off[b] (host), R_b * (I1+I2+I3) floats
 *   lam_packed device, FP32 outputs: item b's R_b weights at offset l_off[b]
 *   infos      host, B records (synchronises the stream) or NULL
 * The per-item options are `opts` (compress, init MLSVD/RANDOM, tolerances);
 * item b uses seed opts->seed + b.  opts->block_threads of 64, 128 or 256
 * fixes the CTA size (and with it the Gram tile shape and CTAs per SM);
 * otherwise an autotuner times the three on the first call for a shape class
 * (device, largest mode, largest rank, compression, batch size rounded to a
 * power of two), keeps the fastest, and later calls use it (the first call
 * therefore runs the batch four times).  On a non-default stream that is not
 * being captured, the item upload, queue reset and launch are captured once
 * per argument set into a CUDA graph and replayed.
 */
size_t cpd_batch_workspace_size(int B, const int* dims, const int* ranks, const cpd_options* opts);
int cpd_batch_solve(int B, const float* T_packed, const int64_t* t_off, const int* dims,
                    const int* ranks, const cpd_options* opts, float* W_packed,
                    const int64_t* w_off, float* lam_packed, const int64_t* l_off,
                    cpd_info* infos, void* workspace, size_t ws_bytes, void* stream);

/* ---- learned initialiser ---------------------------------------------------
 * No counterpart in the thesis, which starts dGN from random factors or from
 * the compressed core (Sec. 4.1.2): a multilayer perceptron proposes the
 * initial factors for dGN on a compressed core, and the solver keeps the
 * MLSVD start unless the proposal's residual is below half of its residual.
 *
 *   input row x (CPD_INITNET_IN_PAD floats): S / ||S|| with S the core
 *     (I1 x I2 x I3 <= 16^3) zero-padded into a 16 x 16 x 16 column-major
 *     block (entries 0..4095), then the rank one-hot (entry 4096 + R - 1,
 *     R <= 8), then zeros;
 *   hidden layers: h1 = relu(W1 x + b1), h2 = relu(W2 h1 + b2) (512 each);
 *   output row y (CPD_INITNET_OUT floats): y[l*128 + r*16 + i] is entry
 *     (i, r) of the mode-l factor divided by ||S||^(1/3) (i < 16, r < 8).
 *   parameters, one FP32 vector of cpd_initnet_param_count() floats:
 *     W1 (512 x 4160, row-major) | b1 (512) | W2 (512 x 512) | b2 | W3 (384 x 512) | b3 (384).
 * Products run on BF16 tensor cores (operands rounded to BF16, FP32
 * accumulation).  Matrices are row-major, one sample per row.
 */
#define CPD_INITNET_CORE 16
#define CPD_INITNET_RANK 8
#define CPD_INITNET_IN 4104
#define CPD_INITNET_IN_PAD 4160
#define CPD_INITNET_HIDDEN 512
#define CPD_INITNET_OUT 384

size_t cpd_initnet_param_count(void);
/* Workspace bytes of cpd_initnet_forward / cpd_initnet_grad for B samples. */
size_t cpd_initnet_workspace_size(int B);
/* Y (B x 384, device) = network(X) for X (B x 4160, device, padding zero). */
int cpd_initnet_forward(const float* params, const float* X, int B, float* Y, void* workspace,
                        size_t ws_bytes, void* stream);
/*
 * Gradient of a training loss with respect to all parameters, into grad
 * (param_count floats, device; overwritten), and the loss into *loss_dev
 * (device double).  With a target (B x 384, device): the masked mean
 * squared error  loss = sum_{b,o} mask[b,o] (y[b,o] - target[b,o])^2 / sum mask.
 * With target == NULL: the reconstruction error of the input cores by the
 * proposed factors (the CP objective on each core, Sec. 3.1),
 *   loss = (1/B) sum_b ||S_b / ||S_b|| - sum_r a_r (x) b_r (x) c_r||^2,
 * factors taken from y_b where mask[b] is 1 (the entries that exist).
 */
int cpd_initnet_grad(const float* params, const float* X, const float* target, const float* mask,
                     int B, float* grad, double* loss_dev, void* workspace, size_t ws_bytes,
                     void* stream);
/* One Adam step (Kingma & Ba) on params with moments m, v (device), step >= 1. */
int cpd_initnet_adam(float* params, float* m, float* v, const float* grad, int step, double lr,
                     double beta1, double beta2, double eps, void* stream);

/*
 * Batched solves that feed and use the learned initialiser (same items,
 * limits and outputs as cpd_batch_solve; compression is always on; items
 * with R > 8 or a core mode above 16 always start from the MLSVD start).
 *  cpd_batch_initnet_data: the plain method (MLSVD start) on every item, plus
 *    per item b the network input row X[b] (4160 floats) and the solver's
 *    core CPD as a training target[b] (384 floats, the output layout above;
 *    terms by decreasing weight, signs as in the outputs, each column scaled
 *    to (lambda_r / ||S||)^(1/3); a zero row when the core solve did not
 *    reach rel_err < 1e-3 or a term's weight exceeds 8 ||S||: no target from
 *    a stalled or degenerate CPD) and mask[b] (1 on the factor entries that
 *    exist: rows below the core dims, columns below R; all 0 for ineligible items).
 *    X, target, mask: device, row-major; any of them may be NULL.
 *  cpd_batch_solve_learned: the network (params) proposes each eligible
 *    item's start, taken when its residual is below half the MLSVD start's;
 *    cpd_info.init_used tells which start dGN took.
 */
size_t cpd_batch_ex_workspace_size(int B, const int* dims, const int* ranks, const cpd_options* opts);
int cpd_batch_initnet_data(int B, const float* T_packed, const int64_t* t_off, const int* dims,
                           const int* ranks, const cpd_options* opts, float* W_packed,
                           const int64_t* w_off, float* lam_packed, const int64_t* l_off,
                           float* X, float* target, float* mask, cpd_info* infos,
                           void* workspace, size_t ws_bytes, void* stream);
int cpd_batch_solve_learned(int B, const float* T_packed, const int64_t* t_off, const int* dims,
                            const int* ranks, const cpd_options* opts, const float* params,
                            float* W_packed, const int64_t* w_off, float* lam_packed,
                            const int64_t* l_off, cpd_info* infos, void* workspace,
                            size_t ws_bytes, void* stream);

/* ---- component calls (the same device code the solvers run), for testing
 *      and for callers that compose the steps themselves ---------------------- */

/*
 * cpd_gemm_bf16 — the tensor-core GEMM the learned initialiser runs on:
 *   D[m*ldd + n] (=, or += when accumulate) epi(sum_k A[m*sam + k*sak] B[n*sbn + k*sbk])
 * for m < M, n < N, k < K; epi adds bias[n] (if non-NULL), applies ReLU (if
 * relu), and zeroes entries where mask[m*ldm + n] <= 0 (if mask non-NULL).
 * A, B, D, bias, mask: device FP32; operands rounded to BF16, FP32 accumulation.
 */
int cpd_gemm_bf16(int M, int N, int K, const float* A, int64_t sam, int64_t sak, const float* B,
                  int64_t sbn, int64_t sbk, float* D, int64_t ldd, const float* bias, int relu,
                  const float* mask, int64_t ldm, int accumulate, void* stream);

/*
 * cpd_core_eval — residual and gradient on a small tensor by one CTA
 * (Sec. 4.1.3 "Computing the residual" and "Computing the gradient"):
 *   f = S - [[W]]; fsq = ||f||^2 (FP64 accumulation); g = A^T b = -grad F,
 *   block l of g = f_(l) (W^(L) ⊙ .. ⊙ W^(l+1) ⊙ W^(l-1) ⊙ .. ⊙ W^(1)).
 *   S, W device FP32; f_out (prod dims, may be NULL), g_out (stacked blocks)
 *   device FP32; fsq_out device double[1].
 */
int cpd_core_eval(const float* S, int L, const int64_t* dims, int R, const float* W,
                  float* f_out, float* g_out, double* fsq_out, void* workspace,
                  size_t ws_bytes, void* stream);

/*
 * cpd_jtj_apply — out = J^T J v for the CPD W (Theorem "Hv", Sec. 3.5.3):
 *   block l' of out = V^(l') Pi^(l') + sum_{l''≠l'} W^(l') (Pi^(l',l'') * (V^(l'')^T W^(l''))).
 *   W, V, out device FP32 stacked blocks.
 */
int cpd_jtj_apply(int L, const int64_t* dims, int R, const float* W, const float* V,
                  float* out, void* workspace, size_t ws_bytes, void* stream);

/*
 * cpd_mode_gram — G = T_(l) T_(l)^T (I_l x I_l, FP32, column-major), the Gram
 * route to the left singular vectors of the unfolding (App. A).  precision is
 * a cpd_gram_precision (BF16 supported for mode l = 0 with I_1 <= 256 and a
 * 16-byte-aligned T only; otherwise CPD_ERR_UNSUPPORTED).
 */
int cpd_mode_gram(const float* T, int L, const int64_t* dims, int mode, int precision,
                  float* G_out, void* workspace, size_t ws_bytes, void* stream);

/*
 * cpd_refine_eval — one pass over a large tensor T (FP32): residual
 * e = T - [[W]], esq = ||e||^2 (FP64 accumulation, device double[1]) and the
 * MTTKRP of e for every mode into g_out (stacked blocks, = -grad F).
 * Same shape limits as refinement in cpd_dgn_solve (else CPD_ERR_UNSUPPORTED).
 */
int cpd_refine_eval(const float* T, int L, const int64_t* dims, int R, const float* W,
                    float* g_out, double* esq_out, void* workspace, size_t ws_bytes,
                    void* stream);


/* ---- diagnostics ------------------------------------------------------------ */

/* Number of kernels this library has launched in this process (all streams). */
long long cpd_launch_count(void);

/*
 * Per-stage device timing.  While enabled (on != 0), every launch site of the
 * solvers records a CUDA event pair on the stream it launches on; stage names
 * are the launcher names ("gram_fp32", "gram_bf16_tc", "eig", "project",
 * "dgn_core", "uncompress", "refine_pass", "refine_step", "normalize", ...).
 * cpd_profile_read synchronises the recorded events, returns up to
 * max_entries stages (names: 32 chars each, NUL-terminated; ms: total device
 * milliseconds; launches: launch count) and clears the record.  Returns the
 * number of stages written, or a negative cpd_status.  Not thread-safe.
 */
int cpd_profile_enable(int on);
int cpd_profile_read(int max_entries, char* names, double* ms, long long* launches);

#ifdef __cplusplus
}
#endif
#endif /* CPD_H_ */
