"""CPU tests of the ADMM workload driver's update equations (Sec. 5, the
three-step scheme with A = diag, b = 1), with an exact eigendecomposition as
the projection.  Pinned to closed forms: the max-cut SDP of the 5-cycle has
value (25 + 5 sqrt 5) / 8 (Goemans-Williamson), and with C = L (a graph
Laplacian, PSD) the optimum is 0 at X = 1 1^T."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2507_09165_gb300.admm import Solve  # noqa: E402


def exact_projection(V):
    w, Q = np.linalg.eigh(V.double().numpy())
    return torch.from_numpy((Q * np.maximum(w, 0.0)) @ Q.T).to(V.dtype)


def cycle_laplacian(n):
    A = np.zeros((n, n))
    for i in range(n):
        A[i, (i + 1) % n] = A[(i + 1) % n, i] = 1.0
    return np.diag(A.sum(1)) - A


def run(C, sigma, iters):
    sv = Solve(torch.from_numpy(C).double(), sigma, iters)
    while True:
        V = sv.make_input()
        sv.S.copy_(exact_projection(V))
        if sv.finish_iteration():
            return sv


@pytest.mark.parametrize("sigma", [0.5, 1.0, 3.0])
def test_maxcut_5_cycle_value(sigma):
    sv = run(-cycle_laplacian(5) / 4.0, sigma, 3000)
    eta, parts = sv.surrogate()
    assert eta < 1e-6
    assert abs(parts["pobj"] + (25 + 5 * math.sqrt(5)) / 8) < 1e-5
    assert abs(parts["dobj"] + (25 + 5 * math.sqrt(5)) / 8) < 1e-5
    np.testing.assert_allclose(sv.X.diagonal().numpy(), 1.0, atol=1e-8)


def test_laplacian_objective_reaches_zero_at_all_ones():
    L = cycle_laplacian(7)
    sv = run(L, 1.0, 2000)
    eta, parts = sv.surrogate()
    assert eta < 1e-6 and abs(parts["pobj"]) < 1e-6
    np.testing.assert_allclose(sv.X.numpy(), np.ones((7, 7)), atol=1e-4)


def test_first_projection_input():
    # X_0 = S_0 = 0, y_0 = 0: y_1 = 1/sigma + diag(C), V_1 = C - Diag(y_1)
    C = cycle_laplacian(6)
    sv = Solve(torch.from_numpy(C), 2.0, 1)
    V = sv.make_input().numpy()
    np.testing.assert_allclose(sv.y.numpy(), 0.5 + np.diag(C))
    np.testing.assert_allclose(V, C - np.diag(0.5 + np.diag(C)))


def test_solver_switches_precision_and_converges():
    # a deliberately coarse "low" projection (the exact one rounded to 3
    # significant digits) stalls above the switch threshold's neighbourhood; the
    # solver must switch to the exact "high" projection once the surrogate drops
    # below 1e-2 and then converge to 1e-6
    from paper_2507_09165_gb300.admm import solve

    def project(V, S, prec):
        P = exact_projection(V)
        if prec == "low":
            P = torch.from_numpy(np.round(P.numpy(), 3))
        S.copy_(P)

    C = torch.from_numpy(-cycle_laplacian(5) / 4.0)
    r = solve(C, project, sigma=1.0, max_iters=4000, eta_switch=1e-2, eta_tol=1e-6, check_every=5,
              low="low", high="high")
    assert r["switch_iter"] is not None
    assert all(p == "low" for k, p, _ in r["history"] if k <= r["switch_iter"])
    assert r["history"][-1][2] < 1e-6
    pobj = float((C * r["X"]).sum())
    assert abs(pobj + (25 + 5 * math.sqrt(5)) / 8) < 1e-5
