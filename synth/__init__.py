"""Seeded synthetic inputs for the CPD hot path.

This module is the only code shared by the CUDA path's callers (tests, bench)
and the FP64 oracle.  It draws random numbers and assembles planted tensors;
it holds none of the method's arithmetic (no compression, no residuals, no
Gauss-Newton).  Every generator is deterministic in its seed.

Layout contract: a tensor T with dims (I1, ..., IL) is an ``np.ndarray`` of
that shape whose memory order is column-major (Fortran), i.e. i1 fastest, as
the thesis fixes for unfoldings and vec (Sec. 2.1.1, Algorithm "Unfolding";
Sec. 3.1 for vec of factor matrices).  Factor matrices are Iℓ×R, column-major.

Workload recipes (Sec. 4.3.5 "Collinear factors" and the noise model of Sec. 4.9.2):
  * planted rank-R tensor T0 = sum_r w_r^(1) ⊗ ... ⊗ w_r^(L) with factor
    columns drawn i.i.d. N(0, I);
  * "pairwise collinearity rho": w_r = sqrt(rho)·s + sqrt(1-rho)·g_r with s, g_r
    i.i.d. N(0, I) per mode, so E[cos(w_r, w_r')] = rho (Sec. 4.3 builds swamps
    by mixing every column toward one shared direction; this is the same
    construction with a Gaussian shared direction);
  * relative noise eta: T = T0 + eta·||T0||·E/||E||, E i.i.d. N(0,1).
"""
from __future__ import annotations

import numpy as np

SEED_BASE = 2110_05997


def rng(seed: int) -> np.random.Generator:
    return np.random.default_rng(np.random.PCG64(int(seed) & ((1 << 63) - 1)))


def gaussian_factors(g: np.random.Generator, dims, R: int, rho: float = 0.0):
    """Factor matrices Iℓ×R (FP64, column-major) with pairwise collinearity rho."""
    Ws = []
    for I in dims:
        G = g.standard_normal((I, R))
        if rho > 0.0:
            s = g.standard_normal((I, 1))
            G = np.sqrt(rho) * s + np.sqrt(1.0 - rho) * G
        Ws.append(np.asfortranarray(G))
    return Ws


def planted_tensor(Ws) -> np.ndarray:
    """T0 = sum_r outer products of the factor columns, FP64, column-major.

    Assembled as mode-1 rows times the column-major Khatri-Rao product of the
    remaining factors (i2 fastest, matching the unfolding order).
    """
    dims = [W.shape[0] for W in Ws]
    R = Ws[0].shape[1]
    rest = np.ones((1, R))
    for W in Ws[1:]:
        # rows of `rest` run over (i2, ..., i_ell) with i2 fastest
        rest = np.einsum("ar,br->abr", rest, W).reshape(-1, R, order="F")
    T1 = Ws[0] @ rest.T                      # I1 x prod(rest)
    return np.asfortranarray(T1.reshape(dims, order="F"))


def add_noise(g: np.random.Generator, T0: np.ndarray, eta: float, dtype=np.float64):
    """T = T0 + eta·||T0||·E/||E|| (relative noise level eta)."""
    if eta <= 0.0:
        return np.asfortranarray(T0.astype(dtype))
    E = g.standard_normal(T0.shape).astype(np.float64)
    T = T0 + (eta * np.linalg.norm(T0) / np.linalg.norm(E)) * E
    return np.asfortranarray(T.astype(dtype))


def planted(seed: int, dims, R: int, rho: float = 0.0, eta: float = 0.0,
            dtype=np.float64):
    """A planted CPD problem: returns (T, true factors)."""
    g = rng(seed)
    Ws = gaussian_factors(g, dims, R, rho)
    T = add_noise(g, planted_tensor(Ws), eta, dtype)
    return T, Ws


def initial_factors(seed: int, dims, R: int, dtype=np.float64):
    """Random N(0,1) starting factors (Sec. 4.1.2, first approach), passed to
    both the CUDA path and the oracle as an input."""
    g = rng(seed ^ 0x5EED_1217)
    return [np.asfortranarray(g.standard_normal((I, R)).astype(dtype)) for I in dims]


# --- named workloads -------------------------------------------------------

def c1_plain_dgn(seed: int = SEED_BASE + 1):
    """20×20×20 FP64, rank 5 Gaussian factors, noise 1e-6 relative, N(0,1)
    starting factors; dGN on T directly (no compression)."""
    dims, R = (20, 20, 20), 5
    T, Wt = planted(seed, dims, R, 0.0, 1e-6, np.float64)
    W0 = initial_factors(seed, dims, R)
    return dict(T=T, R=R, W0=W0, W_true=Wt, name="dgn_20x20x20_r5_fp64")


def c2_compressed(seed: int = SEED_BASE + 2, n: int = 200):
    """n×n×n FP32 (n=200), rank 10, pairwise collinearity 0.5, noise 1e-4."""
    dims, R = (n, n, n), 10
    T, Wt = planted(seed, dims, R, 0.5, 1e-4, np.float32)
    return dict(T=T, R=R, W_true=Wt, name=f"mlsvd_dgn_{n}x{n}x{n}_r10_rho0.5_fp32")


def c3_order4(seed: int = SEED_BASE + 3, n: int = 100):
    """n^4 FP32 (n=100: 400 MB), rank 15 Gaussian factors, noise 1e-5."""
    dims, R = (n, n, n, n), 15
    T, Wt = planted(seed, dims, R, 0.0, 1e-5, np.float32)
    return dict(T=T, R=R, W_true=Wt, name=f"mlsvd_dgn_{n}^4_r15_fp32")


def c4_batch_specs(seed: int = SEED_BASE + 4, B: int = 4096, lo: int = 8, hi: int = 48,
                   rlo: int = 2, rhi: int = 8):
    """Shapes of the uneven batch: each mode size uniform in [lo, hi], rank
    uniform in [rlo, rhi]."""
    g = rng(seed)
    dims = g.integers(lo, hi + 1, size=(B, 3))
    Rs = g.integers(rlo, rhi + 1, size=B)
    return dims, Rs


def c4_batch(seed: int = SEED_BASE + 4, B: int = 4096, lo: int = 8, hi: int = 48,
             rlo: int = 2, rhi: int = 8, eta: float = 1e-6):
    """B third-order FP32 tensors with uneven shapes and ranks, Gaussian
    factors, noise eta relative."""
    dims, Rs = c4_batch_specs(seed, B, lo, hi, rlo, rhi)
    items = []
    for b in range(B):
        T, Wt = planted(seed * 7919 + b, tuple(int(d) for d in dims[b]), int(Rs[b]),
                        0.0, eta, np.float32)
        items.append(dict(T=T, R=int(Rs[b]), W_true=Wt))
    return items


def c5_initnet(seed: int = SEED_BASE + 5, B: int = 4096, n: int = 16, rlo: int = 1, rhi: int = 8,
               rho_max: float = 0.9, eta: float = 1e-6):
    """B planted n x n x n FP32 tensors for the learned initialiser: rank
    uniform in [rlo, rhi], pairwise collinearity rho uniform in [0, rho_max]
    per item, noise eta relative.  Returns the packed column-major tensors
    (B x n^3), ranks and rhos.  Items of one rank are drawn together."""
    g = rng(seed)
    Rs = g.integers(rlo, rhi + 1, size=B)
    rhos = g.uniform(0.0, rho_max, size=B)
    out = np.empty((B, n ** 3), dtype=np.float32)
    for R in range(rlo, rhi + 1):
        idx = np.nonzero(Rs == R)[0]
        if idx.size == 0:
            continue
        Bg = idx.size
        sr = np.sqrt(rhos[idx])[:, None, None]
        cr = np.sqrt(1.0 - rhos[idx])[:, None, None]
        F = [sr * g.standard_normal((Bg, n, 1)) + cr * g.standard_normal((Bg, n, R)) for _ in range(3)]
        # column-major flattening: entry (i, j, k) at i + n j + n^2 k
        T0 = np.einsum("bkr,bjr,bir->bkji", F[2], F[1], F[0]).reshape(Bg, -1)
        E = g.standard_normal(T0.shape)
        scale = eta * np.linalg.norm(T0, axis=1) / np.linalg.norm(E, axis=1)
        out[idx] = (T0 + scale[:, None] * E).astype(np.float32)
    return out, Rs.astype(int), rhos


def warming_up_tensor() -> np.ndarray:
    """The 6×5×4 tensor t_ijk = phi(x_i, y_j, z_k) of Sec. 4.2 ("Warming up"),
    phi(x,y,z) = cos(1-x)sin(1+y^2) - sin(1+x^2)e^{x^2+y^2+z^2} - cos(x)ln(1+z),
    on uniform grids of [0,1] with 6, 5 and 4 samples."""
    x = np.linspace(0.0, 1.0, 6)
    y = np.linspace(0.0, 1.0, 5)
    z = np.linspace(0.0, 1.0, 4)
    X, Y, Z = np.meshgrid(x, y, z, indexing="ij")
    T = (np.cos(1 - X) * np.sin(1 + Y**2)
         - np.sin(1 + X**2) * np.exp(X**2 + Y**2 + Z**2)
         - np.cos(X) * np.log(1 + Z))
    return np.asfortranarray(T)


def warming_up_separable():
    """The three separable rank-one terms of the warming-up tensor (Sec. 4.2):
    returns factor matrices X (6×3), Y (5×3), Z (4×3) with T = [[X, Y, Z]]."""
    x = np.linspace(0.0, 1.0, 6)
    y = np.linspace(0.0, 1.0, 5)
    z = np.linspace(0.0, 1.0, 4)
    X = np.stack([np.cos(1 - x), -np.sin(1 + x**2) * np.exp(x**2), -np.cos(x)], axis=1)
    Y = np.stack([np.sin(1 + y**2), np.exp(y**2), np.ones_like(y)], axis=1)
    Z = np.stack([np.ones_like(z), np.exp(z**2), np.log(1 + z)], axis=1)
    return [np.asfortranarray(X), np.asfortranarray(Y), np.asfortranarray(Z)]


def flat(T: np.ndarray) -> np.ndarray:
    """Column-major flattening (the device layout)."""
    return np.ascontiguousarray(T.ravel(order="F"))
