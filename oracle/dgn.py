"""Damped Gauss-Newton CPD (thesis Ch. 3, Sec. 4.1.2-4.1.4, Sec. 4.8), FP64.

Notation follows the thesis: W^(l) (I_l × R) factor matrices, w their stacked
vec (Sec. 3.1), f the residual (eq. (residual_function)), F = ½||f||^2,
A = J_f, b = -f, pi^(l) = W^(l)T W^(l) (Sec. 3.5.3), Pi^(l',l'') and Pi^(l')
Hadamard products of the other modes' Grams, D the diagonal regulariser and
M the Jacobi preconditioner (Sec. 4.8).

Readings of passages that are silent, garbled or inconsistent (each is
listed with its justification in the design notes):
  R1  the CG system matrix applies mu·D (the system (dGN-eq)); the three-step
      product display of Sec. 4.1.3 writes mu·I, which contradicts M's definition;
  R2  the PCG returns x = M^{-1/2} x_hat (x_hat = M^{1/2} x, App. A eq. (precond4));
  R3  cg_maxiter at iteration k is uniform on the integers of
      [1 + ceil(k^a), 2 + ceil(k^b)], inclusive, drawn from a counter-based
      SplitMix64 stream (Steele, Lea & Flood 2014) so that two
      implementations draw the same integers; ceilings are taken of x - 1e-9
      so that powers that are integers in exact arithmetic do not round up;
  R4  the CG stop test is ||r||^2 < tol, absolute, tol the dGN tolerance;
  R5  the gain ratio uses ½||f + Jx||^2 = F - <g, x> + ½<x, J^T J x>, g = -grad F
      (exact; Sec. 3.5.2 gain ratio with consistent ½ factors);
  R6  per iteration: solve -> w += x -> norm-balance (keeps column signs; the
      common norm is the geometric mean) -> new residual and gradient ->
      gain ratio -> mu update (x3 below 0.25, /3 above 0.75) -> stop tests;
      the starting point is balanced too;
  R7  D and M are rebuilt every iteration from the current balanced factors;
      for general L, gamma_r^(l) = prod_{j≠l}||w_r^(j)|| ·
      max_m max_r' prod_{j≠m}||w_r'^(j)|| (the L = 3 formulas of Sec. 4.8);
  R8  stop tests in the printed order; the gradient-norm test uses the
      gradient at the new iterate; tests 5 and 6 run when k is a multiple of
      c = 1 + ceil(maxiter/10) and k > 2c, with the printed windows; the
      divergence test uses the norm of the tensor being decomposed;
  R9  mu0 = tau·mean|S| over the tensor being decomposed (Sec. 4.1.3);
  R10 refinement in the original space continues mu and the iteration
      counter k of cg_maxiter from the core stage; its stop tests start a
      fresh error history.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, replace

import numpy as np

from .tensor import cpd_tensor, unfold, kr_others
from .mlsvd import compress as _compress

MASK64 = (1 << 64) - 1
GOLDEN_GAMMA = 0x9E3779B97F4A7C15
STREAM_STRIDE = 0xD1B54A32D192ED03
STREAM_CG = 1
STREAM_INIT = 2

STOP_NAMES = {1: "rel_err", 2: "step", 3: "improvement", 4: "grad", 5: "avg_err",
              6: "avg_improvement", 7: "divergence", 8: "maxiter"}


@dataclass
class Options:
    maxiter: int = 200          # Sec. 4.1.3 "Main parameters"
    tol: float = 1e-6           # one tolerance for every stop test (Sec. 4.1.3)
    tau: float = 1.0            # mu0 = tau·mean|S|
    cg_a: float = 0.4           # cg_maxiter interval exponents (Sec. 4.4 result)
    cg_b: float = 0.9
    mlsvd_tol: float = 1e-6     # no default printed; chosen
    st_mlsvd: bool = True       # Algorithm ST-MLSVD (True) or MLSVD (False)
    compress: bool = True       # False: dGN directly on T
    init: str = "mlsvd"         # "mlsvd" (Sec. 4.1.2 second approach), "random", "given"
    refine_maxiter: int = 0     # dGN iterations in the original space after uncompression
    seed: int = 0
    precond: str = "jacobi"     # "jacobi": diagonal M (Sec. 4.8); "block": the exact
                                # diagonal blocks of J^T J + mu D (Sec. 3.5.3 corollary)


# --- SplitMix64 (Steele, Lea & Flood 2014) -----------------------------------

def _mix64(z: int) -> int:
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    return z ^ (z >> 31)


def splitmix64(seed: int, stream: int, counter: int) -> int:
    """The counter-th output (counter >= 1) of SplitMix64 started at state
    seed + stream·0xD1B54A32D192ED03 (mod 2^64)."""
    state = (int(seed) + int(stream) * STREAM_STRIDE + int(counter) * GOLDEN_GAMMA) & MASK64
    return _mix64(state)


def _ceil_guard(x: float) -> int:
    return int(math.ceil(x - 1e-9))


def cg_maxiter(k: int, seed: int, a: float = 0.4, b: float = 0.9) -> int:
    """Reading R3 of Sec. 4.1.3: uniform integer in [1+ceil(k^a), 2+ceil(k^b)]."""
    lo = 1 + _ceil_guard(float(k) ** a)
    hi = 2 + _ceil_guard(float(k) ** b)
    if hi < lo:
        hi = lo
    return lo + splitmix64(seed, STREAM_CG, k) % (hi - lo + 1)


# --- residual, gradient, Grams, Hv (Sec. 3.5, Sec. 4.1.3) --------------------

def residual(T: np.ndarray, Ws) -> np.ndarray:
    """f_{i1..iL} = t_{i1..iL} - sum_r prod_l w_{il r}^(l)  (eq. (residual_function))."""
    return T - cpd_tensor(Ws)


def neg_gradient(f: np.ndarray, Ws):
    """A^T b = -grad F, blockwise f_(l) · (W^(L) ⊙ .. ⊙ W^(l+1) ⊙ W^(l-1) ⊙ .. ⊙ W^(1))
    (theorem of Kolda, Acar and Dunlavy quoted in Sec. 4.1.3, applied to the
    residual: -dF/dW^(l) = T_(l)·KR - W^(l)Pi^(l) = f_(l)·KR)."""
    return [unfold(f, l) @ kr_others(Ws, l) for l in range(len(Ws))]


def grams(Ws):
    """pi^(l) = W^(l)T W^(l)  (Sec. 3.5.3)."""
    return [W.T @ W for W in Ws]


def pi_matrices(gr):
    """Pi^(l',l'') = Hadamard product of pi^(l) over l ∉ {l', l''}, and
    Pi^(l') = Hadamard product over l ≠ l'  (Sec. 3.5.3)."""
    L = len(gr)
    R = gr[0].shape[0]
    Pi1 = []
    for a in range(L):
        P = np.ones((R, R))
        for j in range(L):
            if j != a:
                P = P * gr[j]
        Pi1.append(P)
    Pi2 = [[None] * L for _ in range(L)]
    for a in range(L):
        for b in range(L):
            if a == b:
                continue
            P = np.ones((R, R))
            for j in range(L):
                if j != a and j != b:
                    P = P * gr[j]
            Pi2[a][b] = P
    return Pi1, Pi2


def jtj_apply(Ws, Pi1, Pi2, Vs):
    """Theorem "Hv" (Sec. 3.5.3): block l' of J^T J·v is
    V^(l')Pi^(l') + sum_{l''≠l'} W^(l')·(Pi^(l',l'') * (V^(l'')T W^(l'')))."""
    L = len(Ws)
    out = []
    for a in range(L):
        Z = Vs[a] @ Pi1[a]
        for b in range(L):
            if b != a:
                Z = Z + Ws[a] @ (Pi2[a][b] * (Vs[b].T @ Ws[b]))
        out.append(Z)
    return out


def column_norms(Ws):
    return [np.sqrt(np.sum(W * W, axis=0)) for W in Ws]


def regularizer(Ws):
    """gamma_r^(l) of Sec. 4.8 (reading R7 for general L)."""
    L = len(Ws)
    nr = column_norms(Ws)
    prod_other = []
    for l in range(L):
        p = np.ones_like(nr[0])
        for j in range(L):
            if j != l:
                p = p * nr[j]
        prod_other.append(p)
    gmax = max(float(np.max(p)) for p in prod_other)
    return [p * gmax for p in prod_other]


def preconditioner(Ws, gamma, mu: float):
    """M = diag(a_ii + mu·d_ii): block (l, r) is prod_{j≠l}||w_r^(j)||^2 + mu·gamma_r^(l)
    (Sec. 4.8, D_X, D_Y, D_Z and the general-L diagonal of J^T J)."""
    L = len(Ws)
    nr = column_norms(Ws)
    out = []
    for l in range(L):
        p = np.ones_like(nr[0])
        for j in range(L):
            if j != l:
                p = p * nr[j] ** 2
        out.append(p + mu * gamma[l])
    return out


def block_preconditioner(Pi1, gamma, mu: float):
    """Block-Jacobi preconditioner: the diagonal blocks of J^T J + mu D.  By the
    theorem on J^T J (Sec. 3.5.3) the block of mode l is Pi^(l) (x) I_{I_l}, and
    D's block is diag(gamma^(l)) (x) I, so the block of mode l acts on vec(V^(l))
    as V^(l) -> V^(l) (Pi^(l) + mu diag(gamma^(l))); returns the R x R matrices
    B_l = Pi^(l) + mu diag(gamma^(l)) and their Cholesky factors."""
    Bs = [P + mu * np.diag(g) for P, g in zip(Pi1, gamma)]
    return Bs, [np.linalg.cholesky(B) for B in Bs]


def pcg_block(Ws, Pi1, Pi2, g, gamma, chol, mu: float, maxit: int, tol: float):
    """Preconditioned CG (App. A) on (J^T J + mu D) x = A^T b with the
    block-Jacobi preconditioner: z = M^{-1} r is, per mode, the solve
    Z^(l) B_l = R^(l) by the Cholesky factor of B_l.  The stop test is the
    split form's ||M^{-1/2} r||^2 = r^T M^{-1} r < tol; returns (x, iterations)."""
    def apply_A(P):
        H = jtj_apply(Ws, Pi1, Pi2, P)
        return [H[l] + mu * gamma[l][None, :] * P[l] for l in range(len(P))]

    def precond(Rm):
        out = []
        for l, C in enumerate(chol):
            # Z B = R with B = C C^T:  Z = R C^{-T} C^{-1}
            Y = np.linalg.solve(C, Rm[l].T)          # C Y = R^T
            out.append(np.linalg.solve(C.T, Y).T)    # C^T Z^T = Y
        return out

    x = [np.zeros_like(v) for v in g]
    r = [v.copy() for v in g]
    z = precond(r)
    p = [v.copy() for v in z]
    rz = _dot(r, z)
    its = 0
    for i in range(maxit):
        q = apply_A(p)
        pq = _dot(p, q)
        if pq <= 0.0:
            break
        alpha = rz / pq
        x = [xi + alpha * pi for xi, pi in zip(x, p)]
        r = [ri - alpha * qi for ri, qi in zip(r, q)]
        z = precond(r)
        rz_new = _dot(r, z)
        beta = rz_new / rz if rz > 0 else 0.0
        p = [zi + beta * pi for zi, pi in zip(z, p)]
        rz = rz_new
        its = i + 1
        if rz_new < tol:
            break
    return x, its


def _dot(A, B) -> float:
    return float(sum(np.sum(a * b) for a, b in zip(A, B)))


def pcg(Ws, Pi1, Pi2, g, gamma, Mdiag, mu: float, maxit: int, tol: float):
    """Algorithm "Conjugate gradient - dGN" (Sec. 4.1.3) with the three-step
    product B·p = M^{-1/2}(J^T J + mu D)M^{-1/2}·p; returns (x, iterations)
    with x = M^{-1/2} x_hat (reading R2)."""
    msq = [1.0 / np.sqrt(m) for m in Mdiag]

    def apply_B(P):
        Z = [P[l] * msq[l][None, :] for l in range(len(P))]
        H = jtj_apply(Ws, Pi1, Pi2, Z)
        return [(H[l] + mu * gamma[l][None, :] * Z[l]) * msq[l][None, :]
                for l in range(len(P))]

    r = [g[l] * msq[l][None, :] for l in range(len(g))]
    p = [x.copy() for x in r]
    x = [np.zeros_like(v) for v in r]
    rr = _dot(r, r)
    its = 0
    for i in range(maxit):
        z = apply_B(p)
        pz = _dot(p, z)
        if pz <= 0.0:
            break
        alpha = rr / pz
        x = [xi + alpha * pi for xi, pi in zip(x, p)]
        r = [ri - alpha * zi for ri, zi in zip(r, z)]
        rr_new = _dot(r, r)
        beta = rr_new / rr if rr > 0 else 0.0
        p = [ri + beta * pi for ri, pi in zip(r, p)]
        rr = rr_new
        its = i + 1
        if rr_new < tol:
            break
    return [x[l] * msq[l][None, :] for l in range(len(x))], its


def balance(Ws):
    """Norm-balance each rank-one term so ||w_r^(1)|| = ... = ||w_r^(L)||
    (Sec. 4.1.3 "Updates"); signs are kept, the common norm is the geometric
    mean of the L column norms."""
    L = len(Ws)
    Ws = [W.copy() for W in Ws]
    nr = column_norms(Ws)
    R = Ws[0].shape[1]
    for r in range(R):
        ns = [float(nr[l][r]) for l in range(L)]
        if min(ns) <= 0.0:
            continue
        target = math.exp(sum(math.log(n) for n in ns) / L)
        for l in range(L):
            Ws[l][:, r] *= target / ns[l]
    return Ws


# --- initialisation (Sec. 4.1.2) ---------------------------------------------

def init_mlsvd_energy(S: np.ndarray, R: int):
    """Second approach of Sec. 4.1.2: the R core entries of largest |s| give
    rank-one terms s·e_{j1} ⊗ ... ⊗ e_{jL}; s goes on mode 1 (balancing
    spreads it).  Ties go to the smaller column-major index.  If the core
    has fewer than R entries the extra terms repeat the largest entries."""
    dims = S.shape
    flat = S.ravel(order="F")
    order = np.argsort(-np.abs(flat), kind="stable")
    Ws = [np.zeros((d, R)) for d in dims]
    for r in range(R):
        idx = int(order[r % flat.size])
        mi = np.unravel_index(idx, dims, order="F")
        Ws[0][mi[0], r] = flat[idx]
        for l in range(1, len(dims)):
            Ws[l][mi[l], r] = 1.0
    return Ws


def init_random(seed: int, dims, R: int):
    """First approach of Sec. 4.1.2: N(0,1) entries, drawn by Box-Muller from
    the SplitMix64 stream STREAM_INIT so that the CUDA path draws the same
    numbers: entry j of the stacked vec w uses outputs 2j+1 and 2j+2."""
    Ws = []
    j = 0
    for I in dims:
        W = np.empty((I, R))
        for r in range(R):
            for i in range(I):
                u1 = ((splitmix64(seed, STREAM_INIT, 2 * j + 1) >> 11) + 1) * 2.0 ** -53
                u2 = (splitmix64(seed, STREAM_INIT, 2 * j + 2) >> 11) * 2.0 ** -53
                W[i, r] = math.sqrt(-2.0 * math.log(u1)) * math.cos(2.0 * math.pi * u2)
                j += 1
        Ws.append(W)
    return Ws


# --- updates and stopping conditions (Sec. 4.1.3) -----------------------------

def window_constant(maxiter: int) -> int:
    """c = 1 + ceil(maxiter/10), the batch length of stop tests 5 and 6."""
    return 1 + math.ceil(maxiter / 10)


def gain_ratio(F_old: float, F_new: float, pred_drop: float) -> float:
    """Gain ratio of Sec. 3.5.2 / Sec. 4.1.3 "Updates": actual over predicted
    decrease, pred_drop = F_old - ½||f + Jx||^2 (reading R5).  A
    non-positive predicted decrease gives gain 0 (the step is not trusted)."""
    return (F_old - F_new) / pred_drop if pred_drop > 0 else 0.0


def update_mu(mu: float, gain: float) -> float:
    """Damping update chosen in Sec. 4.1.3 "Updates": mu <- 3 mu when the
    gain is below 0.25, mu <- mu/3 when it is above 0.75, else unchanged."""
    if gain < 0.25:
        return 3.0 * mu
    if gain > 0.75:
        return mu / 3.0
    return mu


def stop_reason(errs, k: int, step: float, grad_inf: float, norm: float, tol: float,
                maxiter: int) -> int:
    """The seven stopping conditions of Sec. 4.1.3, in the printed order, plus
    the iteration cap; returns the number of the first that holds (0: none).

    errs[j] is the relative error ||S - S^(j)|| / ||S|| after iteration j
    (errs[0] at the start), k >= 1 the current iteration, step = ||w^(k-1) -
    w^(k)||, grad_inf = ||grad F(w^(k))||_inf, norm = ||S|| of the tensor
    being decomposed.  Conditions 5 and 6 are evaluated only when k is a
    multiple of c = 1 + ceil(maxiter/10) and k > 2c, with the printed sums
    over j = k-2c..k-c and j = k-c..k (c + 1 terms each), divided by c."""
    e = errs[k]
    c = window_constant(maxiter)
    if e < tol:
        return 1
    if step < tol:
        return 2
    if abs(errs[k - 1] - errs[k]) < tol:
        return 3
    if grad_inf < tol:
        return 4
    batch = k % c == 0 and k > 2 * c
    if batch:
        avg_old = sum(errs[j] for j in range(k - 2 * c, k - c + 1)) / c
        avg_new = sum(errs[j] for j in range(k - c, k + 1)) / c
        if avg_old - avg_new < tol:
            return 5
        avg_impr = sum(abs(errs[j - 1] - errs[j]) for j in range(k - c, k + 1)) / c
        if avg_impr < 1e-3 * avg_new:
            return 6
    if e > max(1.0, norm ** 2) / (1e-16 + tol):
        return 7
    if k == maxiter:
        return 8
    return 0


# --- the dGN loop (Sec. 4.1.3) -------------------------------------------------

def dgn(T: np.ndarray, W0, opts: Options, mu0: float | None = None, k0: int = 0,
        trace: list | None = None):
    """Damped Gauss-Newton on T from W0.  Returns (W, info) where info holds
    iters, stop, rel_err, mu, grad_inf, cg_total, k (last global iteration)."""
    L = T.ndim
    tol = opts.tol
    normT = float(np.linalg.norm(T))
    Ws = balance([np.array(W, dtype=np.float64) for W in W0])
    mu = opts.tau * float(np.mean(np.abs(T))) if mu0 is None else float(mu0)
    f = residual(T, Ws)
    F = 0.5 * float(np.sum(f * f))
    g = neg_gradient(f, Ws)
    errs = [math.sqrt(2.0 * F) / normT if normT > 0 else 0.0]
    stop, k, cg_total = 8, 0, 0
    grad_inf = max(float(np.max(np.abs(x))) for x in g)
    for k in range(1, opts.maxiter + 1):
        gr = grams(Ws)
        Pi1, Pi2 = pi_matrices(gr)
        gamma = regularizer(Ws)
        maxit = cg_maxiter(k0 + k, opts.seed, opts.cg_a, opts.cg_b)
        if opts.precond == "block":
            _, chol = block_preconditioner(Pi1, gamma, mu)
            x, its = pcg_block(Ws, Pi1, Pi2, g, gamma, chol, mu, maxit, tol)
        else:
            Mdiag = preconditioner(Ws, gamma, mu)
            x, its = pcg(Ws, Pi1, Pi2, g, gamma, Mdiag, mu, maxit, tol)
        cg_total += its
        Hx = jtj_apply(Ws, Pi1, Pi2, x)
        pred_drop = _dot(g, x) - 0.5 * _dot(x, Hx)     # F - ½||f + Jx||^2
        step = math.sqrt(_dot(x, x))
        Ws = balance([W + X for W, X in zip(Ws, x)])
        f = residual(T, Ws)
        F_new = 0.5 * float(np.sum(f * f))
        g = neg_gradient(f, Ws)
        gain = gain_ratio(F, F_new, pred_drop)
        mu = update_mu(mu, gain)
        e = math.sqrt(2.0 * F_new) / normT if normT > 0 else 0.0
        errs.append(e)
        grad_inf = max(float(np.max(np.abs(v))) for v in g)
        F = F_new
        if trace is not None:
            trace.append(dict(k=k0 + k, rel_err=e, mu=mu, gain=gain, cg=its,
                              step=step, grad_inf=grad_inf))
        stop = stop_reason(errs, k, step, grad_inf, normT, tol, opts.maxiter)
        if stop:
            break
    info = dict(iters=k, stop=stop, rel_err=errs[-1], mu=mu, grad_inf=grad_inf,
                cg_total=cg_total, k=k0 + k)
    return Ws, info


# --- uncompression and output (Sec. 4.1.4, Fig. tensorfox-flow) ---------------

def uncompress(Us, Ws):
    """W~^(l) = U^(l) W^(l)  (Sec. 4.1.4)."""
    return [U @ W for U, W in zip(Us, Ws)]


def normalize(Ws):
    """Unit columns and weights lambda_r = prod_l ||w_r^(l)|| (output box of
    Fig. tensorfox-flow).  The largest-|.| entry of each column of modes
    1..L-1 is made positive, the sign goes to mode L; terms are sorted by
    lambda, descending."""
    L = len(Ws)
    nr = column_norms(Ws)
    lam = np.ones_like(nr[0])
    for n in nr:
        lam = lam * n
    Wn = [W / np.where(n > 0, n, 1.0)[None, :] for W, n in zip(Ws, nr)]
    R = Wn[0].shape[1]
    for r in range(R):
        for l in range(L - 1):
            i = int(np.argmax(np.abs(Wn[l][:, r])))
            if Wn[l][i, r] < 0:
                Wn[l][:, r] *= -1.0
                Wn[L - 1][:, r] *= -1.0
    order = np.argsort(-lam, kind="stable")
    return [np.asfortranarray(W[:, order]) for W in Wn], lam[order]


def cpd(T: np.ndarray, R: int, opts: Options | None = None, W0=None):
    """The whole method of Fig. tensorfox-flow: compression, initialisation,
    dGN, uncompression (and optional refinement), output normalisation.

    Returns (W unit-column factors, lambda, info).  With init "given", W0 is in
    the original space and, under compression, is projected on the bases."""
    opts = opts or Options()
    T = np.asarray(T, dtype=np.float64)
    L = T.ndim
    info = {}
    if opts.compress:
        Us, sigmas, S, ranks = _compress(T, R, opts.mlsvd_tol, opts.st_mlsvd)
        info.update(core_dims=list(S.shape), sigmas=sigmas)
    else:
        Us, S = None, T
        info.update(core_dims=list(T.shape))
    if opts.init == "given":
        Wi = [np.asarray(W, dtype=np.float64) for W in W0]
        if Us is not None:
            Wi = [U.T @ W for U, W in zip(Us, Wi)]
    elif opts.init == "random":
        Wi = init_random(opts.seed, S.shape, R)
    else:
        Wi = init_mlsvd_energy(S, R)
    W, core_info = dgn(S, Wi, opts)
    info["core"] = core_info
    if Us is not None:
        W = uncompress(Us, W)
    if opts.refine_maxiter > 0:
        W, ref_info = dgn(T, W, replace(opts, maxiter=opts.refine_maxiter),
                          mu0=core_info["mu"], k0=core_info["k"])
        info["refine"] = ref_info
    Wn, lam = normalize(W)
    return Wn, lam, info
