"""Pins of the oracle's filter output F(X) (what Algorithm 2 computes).

Two independent routes to F are compared (eigen-decomposition + scalar map,
and Algorithm 2's GEMM chain in FP64), then each is tied to closed forms and to
the paper's error bound: the spectral operator inherits the scalar error of the
composite polynomial (Sec. 1, polynomial filtering).
"""
import numpy as np
import pytest

import oracle
from oracle import schedules as S
from paper_2507_09165_gb300 import synth


@pytest.mark.parametrize("prec", ["half", "single"])
@pytest.mark.parametrize("n", [1, 2, 7, 40, 128])
def test_chain_equals_eigen_route(prec, n):
    X = synth.gaussian_symmetric(n, 20 + n).astype(np.float64)
    coefs, scales = S.schedule(prec)
    lt = oracle.lanczos_bound(X)["lam_tilde"]
    lam, Q = oracle.eigh_jacobi(X)
    F = oracle.filter_from_eig(lam, Q, lt, coefs, scales)
    C, _ = oracle.chain_fp64(X, lt, coefs, scales)
    assert oracle.rel_err(C, F) < 1e-12


def test_identity_schedule_closed_form():
    # With one stage f(x) = x, Algorithm 2 returns lam~ X0 (I + X0) / 2
    # = (X + X^2 / lam~) / 2.
    X = synth.gaussian_symmetric(30, 31).astype(np.float64)
    lt = 7.5
    want = 0.5 * (X + X @ X / lt)
    lam, Q = oracle.eigh_jacobi(X)
    F = oracle.filter_from_eig(lam, Q, lt, [(1.0, 0.0, 0.0)], [1.0])
    C, _ = oracle.chain_fp64(X, lt, [(1.0, 0.0, 0.0)], [1.0])
    assert np.max(np.abs(F - want)) < 1e-13 * np.max(np.abs(want))
    assert np.max(np.abs(C - want)) < 1e-13 * np.max(np.abs(want))


def test_quintic_stage_closed_form():
    # One quintic stage f(x) = a x + b x^3 + c x^5 and divisor s:
    # X_1 = (a X0 + b X0^3 + c X0^5) / s, output (X + lam~ X0 X_1) / 2.
    X = synth.gaussian_symmetric(25, 32).astype(np.float64)
    lt = 9.0
    a, b, c, s = 1.5, -0.7, 0.2, 1.01
    X0 = X / lt
    X1 = (a * X0 + b * np.linalg.matrix_power(X0, 3) + c * np.linalg.matrix_power(X0, 5)) / s
    want = 0.5 * (X + lt * X0 @ X1)
    lam, Q = oracle.eigh_jacobi(X)
    F = oracle.filter_from_eig(lam, Q, lt, [(a, b, c)], [s])
    C, XT = oracle.chain_fp64(X, lt, [(a, b, c)], [s])
    assert np.max(np.abs(F - want)) < 1e-13 * np.max(np.abs(want))
    assert np.max(np.abs(C - want)) < 1e-13 * np.max(np.abs(want))
    assert np.max(np.abs(XT - X1)) < 1e-13


@pytest.mark.parametrize("prec,scalar_bound", [("half", 6e-5), ("single", 1e-5)])
def test_filter_within_scalar_error_of_projection(prec, scalar_bound):
    # All eigenvalues lie in [-lam~, lam~] (Theorem 2), so
    # ||F - Pi||_2 = max_i |phi(l_i) - relu(l_i)| <= lam~ * e, with e the
    # ReLU error of x (1 + g(x)) / 2 on [-1, 1] (dense grid, Sec. 3.2).
    coefs, scales = S.schedule(prec)
    x = np.linspace(-1, 1, 400001)
    e = float(np.max(np.abs(oracle.relu_approx(x, coefs, scales) - np.maximum(x, 0))))
    assert e < scalar_bound
    X = synth.wigner(200, 33).astype(np.float64)
    lt = oracle.lanczos_bound(X)["lam_tilde"]
    lam, Q = oracle.eigh_jacobi(X)
    F = oracle.filter_from_eig(lam, Q, lt, coefs, scales)
    P = oracle.project_from_eig(lam, Q)
    assert np.linalg.norm(F - P, 2) <= lt * e * (1 + 1e-6) + 1e-14


def test_filter_moreau_analogue():
    # g odd => phi(l) - phi(-l) = l, so F(X) - F(-X) = X (lam~ is the same for
    # X and -X: the bound only sees X^2).
    X = synth.gaussian_symmetric(50, 34).astype(np.float64)
    coefs, scales = S.schedule("half")
    lt = oracle.lanczos_bound(X)["lam_tilde"]
    C1, _ = oracle.chain_fp64(X, lt, coefs, scales)
    C2, _ = oracle.chain_fp64(-X, lt, coefs, scales)
    assert np.max(np.abs(C1 - C2 - X)) < 1e-12 * np.max(np.abs(X))


def test_positive_homogeneity():
    X = synth.gaussian_symmetric(40, 35).astype(np.float64)
    coefs, scales = S.schedule("half")
    b1 = oracle.lanczos_bound(X)
    b2 = oracle.lanczos_bound(3.0 * X)
    C1, _ = oracle.chain_fp64(X, b1["lam_tilde"], coefs, scales)
    C2, _ = oracle.chain_fp64(3.0 * X, b2["lam_tilde"], coefs, scales)
    assert oracle.rel_err(C2, 3.0 * C1) < 1e-12


def test_zero_and_scalar_inputs():
    coefs, scales = S.schedule("half")
    C, _ = oracle.chain_fp64(np.zeros((4, 4)), 0.0, coefs, scales)
    assert not np.any(C)
    for x in (2.0, -3.0):
        X = np.array([[x]])
        lt = oracle.lanczos_bound(X)["lam_tilde"]
        assert lt == abs(x)
        C, _ = oracle.chain_fp64(X, lt, coefs, scales)
        g1 = float(oracle.composite(np.sign(x), coefs, scales))
        assert C[0, 0] == pytest.approx(0.5 * x * (1 + g1), rel=1e-15)


def test_rel_err_conventions():
    A = np.eye(3)
    assert oracle.rel_err(2 * A, A) == pytest.approx(1.0)
    # reference zero (projection of an NSD matrix): relative to ||X||_F
    X = -np.eye(3)
    assert oracle.rel_err(0.5 * A, 0 * A, X) == pytest.approx(0.5)


def test_band_errors_partition():
    # the bands partition the eigenvectors, so the squared band numerators
    # add up to ||A - ref||_F^2.
    X, Q, lam = synth.spectral_matrix("powerlaw", 120, 40)
    rng = np.random.default_rng(1)
    D = rng.standard_normal((120, 120))
    D = D + D.T
    rows = oracle.band_errors(D, np.zeros_like(D), lam, Q)
    tot = 0.0
    for sign, lo, hi, k, err in rows:
        if k:
            sel_lam = lam[(np.abs(lam) / np.max(np.abs(lam)) >= lo) & (np.abs(lam) / np.max(np.abs(lam)) < hi)
                          & ((lam > 0) if sign > 0 else (lam <= 0))]
            tot += (err * np.linalg.norm(sel_lam)) ** 2
    assert sum(k for *_, k, _ in rows) == 120
    assert tot == pytest.approx(np.linalg.norm(D) ** 2, rel=1e-10)
