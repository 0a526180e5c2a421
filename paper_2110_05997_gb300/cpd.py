"""Thin Python binding of libcpd (the C ABI declared in include/cpd.h).

Argument marshalling only: tensors are torch CUDA tensors whose data pointers
are handed to the library, workspaces are allocated with torch, and the
current torch CUDA stream is passed through.  Every step of the method runs
in the library's kernels; nothing here computes.  The functions carry the C
entry points' names.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libcpd.so")

MAX_ORDER = 4
MAX_RANK = 64
TRACE_FIELDS = 8

STATUS = {0: "ok", -1: "invalid argument", -2: "CUDA error", -3: "workspace too small",
          -4: "non-finite value in the iteration", -5: "bounded wait expired",
          -6: "unsupported configuration"}
STOP = {0: "none", 1: "rel_err", 2: "step", 3: "improvement", 4: "grad", 5: "avg_err",
        6: "avg_improvement", 7: "divergence", 8: "maxiter"}
INIT = {"mlsvd": 0, "random": 1, "given": 2, "learned": 3}
INITNET_CORE, INITNET_RANK, INITNET_IN, INITNET_IN_PAD, INITNET_HIDDEN, INITNET_OUT = 16, 8, 4104, 4160, 512, 384
GRAM = {"fp32": 0, "bf16": 1}
PRECOND = {"jacobi": 0, "block": 1}
F32, F64 = 0, 1

EXPORTS = ["cpd_default_options", "cpd_status_string", "cpd_workspace_size", "cpd_compress",
           "cpd_dgn_solve", "cpd_batch_workspace_size", "cpd_batch_solve", "cpd_core_eval",
           "cpd_jtj_apply", "cpd_mode_gram", "cpd_refine_eval", "cpd_launch_count",
           "cpd_profile_enable", "cpd_profile_read", "cpd_dgn_solve_noalloc",
           "cpd_initnet_param_count", "cpd_initnet_workspace_size", "cpd_initnet_forward",
           "cpd_initnet_grad", "cpd_initnet_adam", "cpd_batch_ex_workspace_size",
           "cpd_batch_initnet_data", "cpd_batch_solve_learned", "cpd_gemm_bf16"]


class CpdError(RuntimeError):
    def __init__(self, fn: str, status: int):
        super().__init__(f"{fn} failed: {STATUS.get(status, status)} ({status})")
        self.status = status


class cpd_options(C.Structure):
    _fields_ = [("maxiter", C.c_int), ("tol", C.c_double), ("tau", C.c_double),
                ("cg_a", C.c_double), ("cg_b", C.c_double), ("mlsvd_tol", C.c_double),
                ("st_mlsvd", C.c_int), ("compress", C.c_int), ("init", C.c_int),
                ("gram_precision", C.c_int), ("refine_maxiter", C.c_int),
                ("seed", C.c_uint64), ("block_threads", C.c_int), ("mu_min", C.c_double),
                ("timeout_cycles", C.c_longlong), ("precond", C.c_int)]


class cpd_info(C.Structure):
    _fields_ = [("status", C.c_int), ("iters", C.c_int), ("stop_reason", C.c_int),
                ("cg_total", C.c_int), ("rel_err", C.c_double), ("mu", C.c_double),
                ("grad_inf", C.c_double), ("core_dims", C.c_int * MAX_ORDER),
                ("refine_iters", C.c_int), ("refine_stop_reason", C.c_int),
                ("refine_cg_total", C.c_int), ("init_used", C.c_int), ("refine_rel_err", C.c_double)]

    def as_dict(self):
        return dict(status=self.status, iters=self.iters, stop=self.stop_reason,
                    stop_name=STOP.get(self.stop_reason), cg_total=self.cg_total,
                    rel_err=self.rel_err, mu=self.mu, grad_inf=self.grad_inf,
                    core_dims=list(self.core_dims), refine_iters=self.refine_iters,
                    refine_stop=self.refine_stop_reason, refine_cg_total=self.refine_cg_total,
                    refine_rel_err=self.refine_rel_err, init_used=self.init_used)


_lib = None


def lib():
    """Load libcpd.so; fails loudly if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "paper_2110_05997_gb300.build.build()")
        L = C.CDLL(LIB_PATH)
        vp, i64p, fp, dp, ip = C.c_void_p, C.POINTER(C.c_int64), C.c_void_p, C.c_void_p, C.POINTER(C.c_int)
        optp, infop = C.POINTER(cpd_options), C.POINTER(cpd_info)
        L.cpd_default_options.argtypes = [optp]
        L.cpd_default_options.restype = None
        L.cpd_status_string.argtypes = [C.c_int]
        L.cpd_status_string.restype = C.c_char_p
        L.cpd_workspace_size.argtypes = [C.c_int, i64p, C.c_int, optp]
        L.cpd_workspace_size.restype = C.c_size_t
        L.cpd_compress.argtypes = [vp, C.c_int, i64p, C.c_int, optp, fp, fp, fp, ip, vp, C.c_size_t, vp]
        L.cpd_compress.restype = C.c_int
        L.cpd_dgn_solve.argtypes = [vp, C.c_int, C.c_int, i64p, C.c_int, optp, vp, fp, fp, infop, dp,
                                    vp, C.c_size_t, vp]
        L.cpd_dgn_solve.restype = C.c_int
        L.cpd_batch_workspace_size.argtypes = [C.c_int, ip, ip, optp]
        L.cpd_batch_workspace_size.restype = C.c_size_t
        L.cpd_batch_solve.argtypes = [C.c_int, vp, i64p, ip, ip, optp, fp, i64p, fp, i64p, infop, vp,
                                      C.c_size_t, vp]
        L.cpd_batch_solve.restype = C.c_int
        L.cpd_core_eval.argtypes = [vp, C.c_int, i64p, C.c_int, vp, fp, fp, dp, vp, C.c_size_t, vp]
        L.cpd_core_eval.restype = C.c_int
        L.cpd_jtj_apply.argtypes = [C.c_int, i64p, C.c_int, vp, vp, fp, vp, C.c_size_t, vp]
        L.cpd_jtj_apply.restype = C.c_int
        L.cpd_mode_gram.argtypes = [vp, C.c_int, i64p, C.c_int, C.c_int, fp, vp, C.c_size_t, vp]
        L.cpd_mode_gram.restype = C.c_int
        L.cpd_refine_eval.argtypes = [vp, C.c_int, i64p, C.c_int, vp, fp, dp, vp, C.c_size_t, vp]
        L.cpd_refine_eval.restype = C.c_int
        L.cpd_dgn_solve_noalloc.argtypes = [vp, C.c_int, C.c_int, i64p, C.c_int, optp, vp, fp, fp, infop, vp]
        L.cpd_dgn_solve_noalloc.restype = C.c_int
        L.cpd_initnet_param_count.argtypes = []
        L.cpd_initnet_param_count.restype = C.c_size_t
        L.cpd_initnet_workspace_size.argtypes = [C.c_int]
        L.cpd_initnet_workspace_size.restype = C.c_size_t
        L.cpd_initnet_forward.argtypes = [vp, vp, C.c_int, fp, vp, C.c_size_t, vp]
        L.cpd_initnet_forward.restype = C.c_int
        L.cpd_initnet_grad.argtypes = [vp, vp, vp, vp, C.c_int, fp, dp, vp, C.c_size_t, vp]
        L.cpd_initnet_grad.restype = C.c_int
        L.cpd_initnet_adam.argtypes = [fp, fp, fp, vp, C.c_int, C.c_double, C.c_double, C.c_double,
                                       C.c_double, vp]
        L.cpd_initnet_adam.restype = C.c_int
        L.cpd_batch_ex_workspace_size.argtypes = [C.c_int, ip, ip, optp]
        L.cpd_batch_ex_workspace_size.restype = C.c_size_t
        L.cpd_batch_initnet_data.argtypes = [C.c_int, vp, i64p, ip, ip, optp, fp, i64p, fp, i64p, fp, fp,
                                             fp, infop, vp, C.c_size_t, vp]
        L.cpd_batch_initnet_data.restype = C.c_int
        L.cpd_batch_solve_learned.argtypes = [C.c_int, vp, i64p, ip, ip, optp, vp, fp, i64p, fp, i64p,
                                              infop, vp, C.c_size_t, vp]
        L.cpd_batch_solve_learned.restype = C.c_int
        L.cpd_gemm_bf16.argtypes = [C.c_int, C.c_int, C.c_int, vp, C.c_int64, C.c_int64, vp, C.c_int64,
                                    C.c_int64, fp, C.c_int64, vp, C.c_int, vp, C.c_int64, C.c_int, vp]
        L.cpd_gemm_bf16.restype = C.c_int
        L.cpd_launch_count.argtypes = []
        L.cpd_launch_count.restype = C.c_longlong
        L.cpd_profile_enable.argtypes = [C.c_int]
        L.cpd_profile_enable.restype = C.c_int
        L.cpd_profile_read.argtypes = [C.c_int, C.c_char_p, C.POINTER(C.c_double), C.POINTER(C.c_longlong)]
        L.cpd_profile_read.restype = C.c_int
        _lib = L
    return _lib


def _check(fn, status):
    if status != 0:
        raise CpdError(fn, status)


def _dims(dims):
    return (C.c_int64 * len(dims))(*[int(d) for d in dims])


def _ptr(t):
    return C.c_void_p(0 if t is None else t.data_ptr())


def _stream(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def cpd_default_options(**kw) -> cpd_options:
    o = cpd_options()
    lib().cpd_default_options(C.byref(o))
    for k, v in kw.items():
        if k == "init" and isinstance(v, str):
            v = INIT[v]
        if k == "gram_precision" and isinstance(v, str):
            v = GRAM[v]
        if k == "precond" and isinstance(v, str):
            v = PRECOND[v]
        setattr(o, k, int(v) if isinstance(getattr(o, k), int) else float(v))
    return o


def cpd_status_string(status: int) -> str:
    return lib().cpd_status_string(int(status)).decode()


def cpd_workspace_size(dims, R: int, opts: cpd_options | None = None) -> int:
    opts = opts or cpd_default_options()
    return int(lib().cpd_workspace_size(len(dims), _dims(dims), int(R), C.byref(opts)))


def _workspace(nbytes: int, device):
    import torch
    return torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device)


def _stacked_split(w, dims, R):
    out, o = [], 0
    for d in dims:
        out.append(w[o:o + d * R].reshape(R, d).t())   # column-major I x R view
        o += d * R
    return out


def stack_factors(Ws):
    """Stacked vec layout [vec W1; ...; vec WL] (column-major blocks) of a list of I_l x R tensors."""
    import torch
    return torch.cat([W.t().contiguous().reshape(-1) for W in Ws])


def flat_tensor(T):
    """Column-major flat view (i1 fastest) of a tensor given as torch / numpy array."""
    import torch
    if not isinstance(T, torch.Tensor):
        T = torch.from_numpy(T)
    return T.permute(*reversed(range(T.ndim))).contiguous().reshape(-1)


def cpd_dgn_solve(T_flat, dims, R: int, opts: cpd_options | None = None, W0_flat=None,
                  trace: bool = False, stream=None, workspace=None, want_info: bool = True):
    """Run the whole method on the device tensor ``T_flat`` (column-major flat,
    FP32 or FP64).  Returns (W list of I_l x R unit-column tensors, lambda,
    info dict, trace tensor or None).  With want_info=False no info record is
    read (the call does not synchronise the stream) and the info is None."""
    import torch
    opts = opts or cpd_default_options()
    dev = T_flat.device
    dtype = F64 if T_flat.dtype == torch.float64 else F32
    n = R * sum(int(d) for d in dims)
    W = torch.empty(n, dtype=torch.float32, device=dev)
    lam = torch.empty(R, dtype=torch.float32, device=dev)
    tr = None
    if trace:
        tr = torch.zeros((opts.maxiter + opts.refine_maxiter) * TRACE_FIELDS, dtype=torch.float64, device=dev)
    if workspace is None:
        workspace = _workspace(cpd_workspace_size(dims, R, opts), dev)
    info = cpd_info()
    st = lib().cpd_dgn_solve(_ptr(T_flat), dtype, len(dims), _dims(dims), int(R), C.byref(opts),
                             _ptr(W0_flat), _ptr(W), _ptr(lam), C.byref(info) if want_info else None,
                             _ptr(tr), _ptr(workspace), workspace.numel(), _stream(stream))
    _check("cpd_dgn_solve", st)
    trv = None
    if tr is not None:
        trv = tr.reshape(-1, TRACE_FIELDS)
    return _stacked_split(W, dims, R), lam, (info.as_dict() if want_info else None), trv


def cpd_compress(T_flat, dims, R: int, opts: cpd_options | None = None, stream=None):
    """Truncated MLSVD.  Returns (U list of I_l x R~_l, core tensor (R~ dims, as
    a column-major flat tensor), sigma list, core dims)."""
    import torch
    opts = opts or cpd_default_options()
    dev = T_flat.device
    P = [min(int(d), R) for d in dims]
    U = torch.empty(sum(int(d) * p for d, p in zip(dims, P)), dtype=torch.float32, device=dev)
    n_core = 1
    for p in P:
        n_core *= p
    core = torch.empty(n_core, dtype=torch.float32, device=dev)
    sig = torch.empty(sum(P), dtype=torch.float32, device=dev)
    cd = (C.c_int * len(dims))()
    ws = _workspace(cpd_workspace_size(dims, R, opts), dev)
    st = lib().cpd_compress(_ptr(T_flat), len(dims), _dims(dims), int(R), C.byref(opts), _ptr(U),
                            _ptr(core), _ptr(sig), cd, _ptr(ws), ws.numel(), _stream(stream))
    _check("cpd_compress", st)
    ranks = list(cd)
    Us, o, so, sigs = [], 0, 0, []
    for d, p, k in zip(dims, P, ranks):
        Us.append(U[o:o + d * p].reshape(p, d).t()[:, :k])
        sigs.append(sig[so:so + p])
        o += d * p
        so += p
    nc = 1
    for k in ranks:
        nc *= k
    return Us, core[:nc], sigs, ranks


def cpd_core_eval(S_flat, dims, R: int, W_flat, stream=None):
    """Residual, ||f||^2 and A^T b = -grad F of a small tensor by the solver's code."""
    import torch
    dev = S_flat.device
    N = 1
    for d in dims:
        N *= int(d)
    f = torch.empty(N, dtype=torch.float32, device=dev)
    g = torch.empty(W_flat.numel(), dtype=torch.float32, device=dev)
    fsq = torch.empty(1, dtype=torch.float64, device=dev)
    ws = _workspace(8 * (2 * N + 4 * N * R // max(1, min(int(d) for d in dims)) + 4096), dev)
    st = lib().cpd_core_eval(_ptr(S_flat), len(dims), _dims(dims), int(R), _ptr(W_flat), _ptr(f),
                             _ptr(g), _ptr(fsq), _ptr(ws), ws.numel(), _stream(stream))
    _check("cpd_core_eval", st)
    return f, g, fsq


def cpd_jtj_apply(dims, R: int, W_flat, V_flat, stream=None):
    import torch
    out = torch.empty_like(V_flat)
    st = lib().cpd_jtj_apply(len(dims), _dims(dims), int(R), _ptr(W_flat), _ptr(V_flat), _ptr(out),
                             None, 0, _stream(stream))
    _check("cpd_jtj_apply", st)
    return out


def cpd_mode_gram(T_flat, dims, mode: int, precision: str = "fp32", stream=None):
    import torch
    I = int(dims[mode])
    G = torch.empty(I * I, dtype=torch.float32, device=T_flat.device)
    ws = _workspace(1 << 20, T_flat.device)
    st = lib().cpd_mode_gram(_ptr(T_flat), len(dims), _dims(dims), int(mode), GRAM[precision],
                             _ptr(G), _ptr(ws), ws.numel(), _stream(stream))
    _check("cpd_mode_gram", st)
    return G.reshape(I, I).t()


def cpd_refine_eval(T_flat, dims, R: int, W_flat, stream=None):
    """One pass over a large tensor: ||e||^2, ||T||^2 and the MTTKRP of e."""
    import torch
    g = torch.empty(W_flat.numel(), dtype=torch.float32, device=T_flat.device)
    esq = torch.zeros(2, dtype=torch.float64, device=T_flat.device)
    st = lib().cpd_refine_eval(_ptr(T_flat), len(dims), _dims(dims), int(R), _ptr(W_flat), _ptr(g),
                               _ptr(esq), None, 0, _stream(stream))
    _check("cpd_refine_eval", st)
    return g, esq


@dataclass
class BatchResult:
    W: list
    lam: list
    infos: list


def cpd_batch_workspace_size(dims, ranks, opts: cpd_options | None = None) -> int:
    opts = opts or cpd_default_options()
    B = len(ranks)
    d = (C.c_int * (3 * B))(*[int(x) for row in dims for x in row])
    r = (C.c_int * B)(*[int(x) for x in ranks])
    return int(lib().cpd_batch_workspace_size(B, d, r, C.byref(opts)))


def cpd_batch_ex_workspace_size(dims, ranks, opts: cpd_options | None = None) -> int:
    """Workspace bytes of cpd_batch_initnet_data / cpd_batch_solve_learned
    (also enough for cpd_batch_solve on the same items)."""
    opts = opts or cpd_default_options()
    B = len(ranks)
    d = (C.c_int * (3 * B))(*[int(x) for row in dims for x in row])
    r = (C.c_int * B)(*[int(x) for x in ranks])
    return int(lib().cpd_batch_ex_workspace_size(B, d, r, C.byref(opts)))


def cpd_batch_solve(T_packed, t_off, dims, ranks, opts: cpd_options | None = None, stream=None,
                    workspace=None, want_infos: bool = True):
    """B third-order CPDs in one persistent launch.  ``T_packed`` holds the
    column-major tensors back to back at element offsets ``t_off``."""
    import torch
    opts = opts or cpd_default_options()
    B = len(ranks)
    dev = T_packed.device
    w_off, l_off, wo, lo = [], [], 0, 0
    for b in range(B):
        w_off.append(wo)
        l_off.append(lo)
        wo += int(ranks[b]) * sum(int(x) for x in dims[b])
        lo += int(ranks[b])
    W = torch.empty(max(wo, 1), dtype=torch.float32, device=dev)
    lam = torch.empty(max(lo, 1), dtype=torch.float32, device=dev)
    d = (C.c_int * (3 * B))(*[int(x) for row in dims for x in row])
    r = (C.c_int * B)(*[int(x) for x in ranks])
    to = (C.c_int64 * B)(*[int(x) for x in t_off])
    wof = (C.c_int64 * B)(*w_off)
    lof = (C.c_int64 * B)(*l_off)
    infos = (cpd_info * B)() if want_infos else None
    if workspace is None:
        workspace = _workspace(int(lib().cpd_batch_workspace_size(B, d, r, C.byref(opts))), dev)
    st = lib().cpd_batch_solve(B, _ptr(T_packed), to, d, r, C.byref(opts), _ptr(W), wof, _ptr(lam),
                               lof, infos, _ptr(workspace), workspace.numel(), _stream(stream))
    _check("cpd_batch_solve", st)
    return W, lam, w_off, l_off, ([i.as_dict() for i in infos] if infos is not None else None)


def _batch_marshal(T_packed, t_off, dims, ranks):
    import torch
    B = len(ranks)
    dev = T_packed.device
    w_off, l_off, wo, lo = [], [], 0, 0
    for b in range(B):
        w_off.append(wo)
        l_off.append(lo)
        wo += int(ranks[b]) * sum(int(x) for x in dims[b])
        lo += int(ranks[b])
    W = torch.empty(max(wo, 1), dtype=torch.float32, device=dev)
    lam = torch.empty(max(lo, 1), dtype=torch.float32, device=dev)
    d = (C.c_int * (3 * B))(*[int(x) for row in dims for x in row])
    r = (C.c_int * B)(*[int(x) for x in ranks])
    to = (C.c_int64 * B)(*[int(x) for x in t_off])
    return B, dev, W, lam, w_off, l_off, d, r, to, (C.c_int64 * B)(*w_off), (C.c_int64 * B)(*l_off)


def cpd_batch_initnet_data(T_packed, t_off, dims, ranks, opts: cpd_options | None = None, stream=None,
                           workspace=None):
    """The plain method (MLSVD start) on every item, plus the network input rows
    X (B x 4160), the core CPDs as training targets (B x 384) and their masks."""
    import torch
    opts = opts or cpd_default_options()
    B, dev, W, lam, w_off, l_off, d, r, to, wof, lof = _batch_marshal(T_packed, t_off, dims, ranks)
    X = torch.empty(B, INITNET_IN_PAD, dtype=torch.float32, device=dev)
    tgt = torch.empty(B, INITNET_OUT, dtype=torch.float32, device=dev)
    msk = torch.empty(B, INITNET_OUT, dtype=torch.float32, device=dev)
    infos = (cpd_info * B)()
    if workspace is None:
        workspace = _workspace(cpd_batch_ex_workspace_size(dims, ranks, opts), dev)
    st = lib().cpd_batch_initnet_data(B, _ptr(T_packed), to, d, r, C.byref(opts), _ptr(W), wof, _ptr(lam), lof,
                                      _ptr(X), _ptr(tgt), _ptr(msk), infos, _ptr(workspace), workspace.numel(),
                                      _stream(stream))
    _check("cpd_batch_initnet_data", st)
    return X, tgt, msk, W, lam, w_off, l_off, [i.as_dict() for i in infos]


def cpd_batch_solve_learned(T_packed, t_off, dims, ranks, params, opts: cpd_options | None = None,
                            stream=None, workspace=None, want_infos: bool = True):
    """Batched solves whose dGN starts from the learned initialiser's factors
    (or the MLSVD start when that has the smaller residual)."""
    opts = opts or cpd_default_options()
    B, dev, W, lam, w_off, l_off, d, r, to, wof, lof = _batch_marshal(T_packed, t_off, dims, ranks)
    infos = (cpd_info * B)() if want_infos else None
    if workspace is None:
        workspace = _workspace(cpd_batch_ex_workspace_size(dims, ranks, opts), dev)
    st = lib().cpd_batch_solve_learned(B, _ptr(T_packed), to, d, r, C.byref(opts), _ptr(params), _ptr(W), wof,
                                       _ptr(lam), lof, infos, _ptr(workspace), workspace.numel(),
                                       _stream(stream))
    _check("cpd_batch_solve_learned", st)
    return W, lam, w_off, l_off, ([i.as_dict() for i in infos] if infos is not None else None)


def cpd_initnet_param_count() -> int:
    return int(lib().cpd_initnet_param_count())


def cpd_initnet_workspace_size(B: int) -> int:
    return int(lib().cpd_initnet_workspace_size(int(B)))


def cpd_initnet_forward(params, X, stream=None, workspace=None):
    import torch
    B = X.shape[0]
    Y = torch.empty(B, INITNET_OUT, dtype=torch.float32, device=X.device)
    if workspace is None:
        workspace = _workspace(cpd_initnet_workspace_size(B), X.device)
    _check("cpd_initnet_forward", lib().cpd_initnet_forward(_ptr(params), _ptr(X), B, _ptr(Y), _ptr(workspace),
                                                            workspace.numel(), _stream(stream)))
    return Y


def cpd_initnet_grad(params, X, target, mask, grad=None, loss=None, stream=None, workspace=None):
    """Gradient of the masked mean squared error (into ``grad``) and the loss (device double)."""
    import torch
    B = X.shape[0]
    if grad is None:
        grad = torch.empty_like(params)
    if loss is None:
        loss = torch.zeros(1, dtype=torch.float64, device=X.device)
    if workspace is None:
        workspace = _workspace(cpd_initnet_workspace_size(B), X.device)
    _check("cpd_initnet_grad", lib().cpd_initnet_grad(_ptr(params), _ptr(X), _ptr(target), _ptr(mask), B, _ptr(grad),
                                                      _ptr(loss), _ptr(workspace), workspace.numel(),
                                                      _stream(stream)))
    return grad, loss


def cpd_initnet_adam(params, m, v, grad, step: int, lr: float = 1e-3, beta1: float = 0.9,
                     beta2: float = 0.999, eps: float = 1e-8, stream=None) -> None:
    _check("cpd_initnet_adam", lib().cpd_initnet_adam(_ptr(params), _ptr(m), _ptr(v), _ptr(grad), int(step),
                                                      float(lr), float(beta1), float(beta2), float(eps),
                                                      _stream(stream)))


def cpd_gemm_bf16(M, N, K, A, sam, sak, B, sbn, sbk, D, ldd, bias=None, relu=False, mask=None, ldm=0,
                  accumulate=False, stream=None) -> None:
    _check("cpd_gemm_bf16", lib().cpd_gemm_bf16(int(M), int(N), int(K), _ptr(A), int(sam), int(sak), _ptr(B),
                                                int(sbn), int(sbk), _ptr(D), int(ldd), _ptr(bias), int(bool(relu)),
                                                _ptr(mask), int(ldm), int(bool(accumulate)), _stream(stream)))


def cpd_launch_count() -> int:
    return int(lib().cpd_launch_count())


def cpd_profile_enable(on: bool = True) -> None:
    _check("cpd_profile_enable", lib().cpd_profile_enable(1 if on else 0))


def cpd_profile_read(max_entries: int = 64) -> dict:
    """Per-stage device milliseconds and launch counts recorded since the last read."""
    names = C.create_string_buffer(32 * max_entries)
    ms = (C.c_double * max_entries)()
    cnt = (C.c_longlong * max_entries)()
    n = lib().cpd_profile_read(max_entries, names, ms, cnt)
    if n < 0:
        raise CpdError("cpd_profile_read", n)
    raw = names.raw
    out = {}
    for i in range(n):
        nm = raw[32 * i:32 * (i + 1)].split(b"\0", 1)[0].decode()
        out[nm] = dict(ms=float(ms[i]), launches=int(cnt[i]))
    return out


def cpd_dgn_solve_noalloc(T_flat, dims, R: int, opts: cpd_options | None = None, W0_flat=None,
                          stream=None, W_out=None, lam_out=None):
    """cpd_dgn_solve without a workspace: for callers that may not allocate
    device memory at solve time.  The library keeps the scratch in a fixed
    128 KiB device array; the caller still provides (or here, this binding
    allocates once) the output buffers.  Uncompressed solves only; problems
    beyond the array's capacity raise CpdError (workspace too small)."""
    import torch
    opts = opts or cpd_default_options(compress=0)
    dtype = F64 if T_flat.dtype == torch.float64 else F32
    n = R * sum(int(d) for d in dims)
    W = W_out if W_out is not None else torch.empty(n, dtype=torch.float32, device=T_flat.device)
    lam = lam_out if lam_out is not None else torch.empty(R, dtype=torch.float32, device=T_flat.device)
    info = cpd_info()
    st = lib().cpd_dgn_solve_noalloc(_ptr(T_flat), dtype, len(dims), _dims(dims), int(R), C.byref(opts),
                                     _ptr(W0_flat), _ptr(W), _ptr(lam), C.byref(info), _stream(stream))
    _check("cpd_dgn_solve_noalloc", st)
    return _stacked_split(W, dims, R), lam, info.as_dict()
