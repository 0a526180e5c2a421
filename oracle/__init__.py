"""FP64 CPU oracle for the MLSVD + damped Gauss-Newton CPD method.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code
with the CUDA path (the C-ABI library under ``paper_2110_05997_gb300``); the
only common module is ``synth`` (seeded inputs, no method arithmetic).

The oracle is plain numpy in FP64: each function follows one passage of the
thesis (F. Bottega Diniz, "Tensor decompositions and algorithms, with
applications to tensor learning", 2019) and names it.  Library routines used
as single steps: matrix product, ``numpy.linalg.eigh`` (symmetric eigensolver,
standing in for the SVD of an unfolding through its Gram matrix, App. A),
sorting, and ``scipy.optimize.linear_sum_assignment`` (only for aligning two
CPDs in tests).

Every function here is pinned by a ``-m "not gpu"`` test against something
other than itself (worked examples printed in the thesis, closed forms,
brute force, finite differences); see ``tests/test_oracle_*.py``.
"""
from .tensor import (unfold, fold, mode_product, multilinear, khatri_rao, kron,
                     cpd_tensor)
from .mlsvd import (gram_left_singular, mlsvd_classic, mlsvd_st, truncation_rank,
                    compress)
from .dgn import (Options, splitmix64, cg_maxiter, residual, neg_gradient, grams,
                  pi_matrices, jtj_apply, regularizer, preconditioner, pcg, balance,
                  init_mlsvd_energy, init_random, dgn, uncompress, normalize, cpd,
                  window_constant, gain_ratio, update_mu, stop_reason, block_preconditioner, pcg_block,
                  STOP_NAMES)
from .evaluate import fit, align, compare_cpd

__all__ = [n for n in dir() if not n.startswith("_")]
