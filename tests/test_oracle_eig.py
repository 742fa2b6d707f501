"""Pins of the oracle's eigen-decomposition and exact projection.

Closed forms (diagonal, rank-one, 2x2), a matrix built from a known spectrum,
the defining properties of the projection onto a closed convex cone
(Sec. 1: Pi(X) is the nearest PSD matrix) and an independent library
eigensolver.
"""
import numpy as np
import pytest

import oracle
from paper_2507_09165_gb300 import synth


def _sym(rng, n):
    G = rng.standard_normal((n, n))
    return 0.5 * (G + G.T)


def test_diagonal_closed_form():
    d = np.array([3.0, -1.0, 0.0, 2.5, -7.0, 1e-3])
    lam, Q = oracle.eigh_jacobi(np.diag(d))
    assert np.array_equal(lam, np.sort(d))
    P = oracle.project_from_eig(lam, Q)
    assert np.allclose(P, np.diag(np.maximum(d, 0)), atol=0, rtol=0)


@pytest.mark.parametrize("s", [2.5, -0.75])
def test_rank_one_closed_form(s):
    rng = np.random.default_rng(3)
    v = rng.standard_normal(9)
    v /= np.linalg.norm(v)
    X = s * np.outer(v, v)
    lam, Q = oracle.eigh_jacobi(X)
    P = oracle.project_from_eig(lam, Q)
    want = X if s > 0 else np.zeros_like(X)
    assert np.max(np.abs(P - want)) < 1e-14


def test_two_by_two_closed_form():
    rng = np.random.default_rng(4)
    for _ in range(50):
        a, b, c = rng.standard_normal(3)
        lam, Q = oracle.eigh_jacobi(np.array([[a, b], [b, c]]))
        r = np.hypot(0.5 * (a - c), b)
        want = np.array([0.5 * (a + c) - r, 0.5 * (a + c) + r])
        assert np.allclose(lam, want, rtol=1e-14, atol=1e-15)


def test_known_spectrum():
    # X = Q diag(l) Q^T with a Haar-random Q (QR of a Gaussian): eigenvalues
    # come back to rounding.
    n = 96
    Q = synth.haar_orthogonal(n, seed=11)
    lam0 = np.linspace(-1, 1, n) ** 3
    X = (Q * lam0) @ Q.T
    lam, V = oracle.eigh_jacobi(X)
    assert np.max(np.abs(lam - np.sort(lam0))) < 1e-13
    assert np.max(np.abs(V.T @ V - np.eye(n))) < 1e-13
    P = oracle.project_from_eig(lam, V)
    assert np.max(np.abs(P - (Q * np.maximum(lam0, 0)) @ Q.T)) < 1e-13


@pytest.mark.parametrize("n", [1, 2, 5, 31, 64, 130])
def test_against_library_eigensolver(n):
    rng = np.random.default_rng(n)
    X = _sym(rng, n)
    lam, Q = oracle.eigh_jacobi(X)
    ref = np.linalg.eigvalsh(X)
    scale = max(1.0, float(np.max(np.abs(ref))))
    assert np.max(np.abs(lam - ref)) < 1e-13 * scale * max(1, n)
    assert np.linalg.norm(Q @ np.diag(lam) @ Q.T - X) < 1e-13 * np.linalg.norm(X) * max(1, n)


@pytest.mark.parametrize("n", [17, 80])
def test_projection_invariants(n):
    rng = np.random.default_rng(100 + n)
    X = _sym(rng, n)
    lam, Q = oracle.eigh_jacobi(X)
    P = oracle.project_from_eig(lam, Q)
    nx = np.linalg.norm(X, 2)
    # Pi(X) is PSD, X - Pi(X) is NSD
    assert np.min(np.linalg.eigvalsh(P)) >= -1e-12 * nx
    assert np.max(np.linalg.eigvalsh(X - P)) <= 1e-12 * nx
    # complementarity <Pi(X), X - Pi(X)> = 0
    assert abs(np.sum(P * (X - P))) <= 1e-12 * np.linalg.norm(X) ** 2
    # idempotence Pi(Pi(X)) = Pi(X)
    l2, Q2 = oracle.eigh_jacobi(P)
    assert np.max(np.abs(oracle.project_from_eig(l2, Q2) - P)) < 1e-12 * nx
    # Moreau decomposition X = Pi(X) - Pi(-X)
    l3, Q3 = oracle.eigh_jacobi(-X)
    assert np.max(np.abs(P - oracle.project_from_eig(l3, Q3) - X)) < 1e-12 * nx
    # nearest PSD matrix: no random PSD matrix is closer
    for _ in range(20):
        B = rng.standard_normal((n, n // 2 + 1))
        Z = P + 1e-2 * (B @ B.T) / n
        assert np.linalg.norm(X - P) <= np.linalg.norm(X - Z)
    # non-expansive ||Pi(X) - Pi(Y)|| <= ||X - Y||
    Y = X + 0.3 * _sym(rng, n)
    l4, Q4 = oracle.eigh_jacobi(Y)
    assert np.linalg.norm(P - oracle.project_from_eig(l4, Q4)) <= np.linalg.norm(X - Y) * (1 + 1e-12)


def test_empty_and_scalar():
    lam, Q = oracle.eigh_jacobi(np.zeros((0, 0)))
    assert lam.shape == (0,)
    lam, Q = oracle.eigh_jacobi(np.array([[-2.0]]))
    assert lam[0] == -2.0 and Q[0, 0] == 1.0
