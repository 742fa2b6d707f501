"""The reference values bench.py reports accuracy against (Pi and the filter
output F from a known eigendecomposition, computed in bench.py itself with the
library's schedule) agree with the oracle's."""
import numpy as np

import bench
import oracle
from oracle import schedules as S
from paper_2507_09165_gb300 import synth


def test_bench_exact_references_match_oracle():
    X32, Q, lam = synth.spectral_matrix("uniform", 64, 11)
    lt = 1.0123
    for name in ("half", "single"):
        coefs, post = S.schedule(name)
        P, F = bench.exact_references(lam, Q, lt, coefs, post)
        assert np.allclose(P, oracle.project_from_eig(lam, Q), rtol=0, atol=1e-13)
        assert np.allclose(F, oracle.filter_from_eig(lam, Q, lt, coefs, post), rtol=0, atol=1e-13)
    A = P + 1e-3
    assert abs(bench.rel_fro(A, P) - oracle.rel_err(A, P)) < 1e-15
