"""CPU FP64 oracle for the composite-polynomial PSD-cone projection.

TEST INFRASTRUCTURE ONLY.  This package is the independent checker of the
CUDA library, written from the paper (Factorization-free Orthogonal
Projection onto the PSD Cone with Composite Polynomial Filtering):

* ``eigh_jacobi``      cyclic Jacobi eigen-decomposition (C + OpenMP);
* ``project_from_eig`` the exact projection Q max(L,0) Q^T (Sec. 1, Higham);
* ``filter_from_eig``  the exact filter output Q diag(l (1+g(l/lam~))/2) Q^T,
                       what Algorithm 2 computes in exact arithmetic;
* ``lanczos_bound``    the norm bound of Sec. 3.4 / Theorem 2 (FP64 Lanczos);
* ``chain_fp64``       Algorithm 2 stage by stage in FP64;
* ``composite``, ``efloat``, ``stage_image``  scalar checks (Sec. 3.1-3.3);
* ``rel_err``, ``band_errors``  the FP64 error metrics (Sec. 4.1);
* ``deflate_project``  deflation of the dominant Ritz pairs, then the filter
                       (the remedy of Sec. 6, in this library's reading);
* ``remez.sequential_remez``  Stage I of the coefficient design (Algorithm 1).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s
``cpu_baseline`` / ``--impl reference`` leg may import, call, link or run
anything under ``oracle/``.  It shares no code with the CUDA path and never
imports it.  Every function here is pinned, against closed forms, invariants
and the values the paper prints, by ``tests/test_oracle_*.py``.
"""
from . import schedules
from .deflate import DEFLATE_TOL, deflate_project, ritz_pairs
from ._clib import build as build_clib
from .core import (BANDS, LANCZOS_SEED, band_errors, chain_fp64, composite, efloat,
                   eigh_jacobi, filter_from_eig, lanczos_bound, lanczos_start, phi,
                   project_from_eig, rel_err, relu_approx, spectral, splitmix64, stage_image)


def num_threads():
    """Threads the C part of the oracle uses (OpenMP)."""
    from . import _clib
    return int(_clib.lib().oracle_num_threads())


def oracle_project(X, precision="half", lam_tilde=None):
    """Reference results for one input X (FP64 promotion of its FP32 bits).

    Returns dict(pi=Pi(X), F=F(X), lam_tilde, bound=lanczos dict, lam, Q).
    ``precision``: "half" (f~*_half, T=7) or "single" (f~*_single, T=10).
    """
    import numpy as np
    X = np.asarray(X, dtype=np.float64)
    coefs, scales = schedules.schedule(precision)
    bound = lanczos_bound(X)
    lt = bound["lam_tilde"] if lam_tilde is None else float(lam_tilde)
    lam, Q = eigh_jacobi(X)
    return dict(pi=project_from_eig(lam, Q), F=filter_from_eig(lam, Q, lt, coefs, scales),
                lam_tilde=lt, bound=bound, lam=lam, Q=Q)
