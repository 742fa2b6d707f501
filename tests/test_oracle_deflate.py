"""Pins of the oracle's deflated projection (the remedy of Sec. 6 for spectra
with a few dominant eigenvalues), against closed forms that do not go through
the deflation code: the eigen-decomposition of X, Pi(X), and the scalar map phi.
"""
import numpy as np
import pytest

import oracle
from oracle import schedules as S
from paper_2507_09165_gb300 import synth

COEFS, SCALES = S.schedule("half")


def spectral64(kind, n, seed):
    _, Q, lam = synth.spectral_matrix(kind, n, seed)
    return (Q * lam[None, :]) @ Q.T, Q, lam


def test_kmax_zero_is_the_plain_filter():
    X, Q, lam = spectral64("powerlaw", 150, 3)
    r = oracle.deflate_project(X, 0, COEFS, SCALES)
    assert r["k"] == 0
    lt = oracle.lanczos_bound(X)["lam_tilde"]
    F = oracle.filter_from_eig(lam, Q, lt, COEFS, SCALES)
    assert np.max(np.abs(r["out"] - F)) < 1e-12 * np.max(np.abs(F))
    assert r["lam_tilde_defl"] == pytest.approx(lt, rel=1e-12)


def test_ritz_values_are_the_dominant_eigenvalues():
    # Converged Ritz pairs are eigenpairs of X: each kept mu_j equals an
    # eigenvalue, the kept ones are the k of largest modulus, and v_j is the
    # eigenvector up to sign.
    X, Q, lam = spectral64("powerlaw", 200, 5)
    mu, V, resid, _ = oracle.ritz_pairs(X)
    order = np.argsort(-np.abs(lam))
    conv = [j for j in range(len(mu)) if resid[j] < 1e-10]
    assert len(conv) >= 5
    assert conv == list(range(len(conv)))  # the dominant ones converge first
    for j in conv:
        i = order[j]
        assert mu[j] == pytest.approx(lam[i], abs=1e-10)
        assert abs(abs(V[:, j] @ Q[:, i]) - 1.0) < 1e-10
    assert np.all(np.abs(mu[:-1]) >= np.abs(mu[1:]))


def test_closed_form_with_converged_pairs():
    # With pairs converged to 1e-11 lam~ the deflated subspace is invariant to
    # that accuracy, so the result is Q diag(psi) Q^T: max(lam, 0) on the
    # deflated eigenvalues, phi(lam; lam~') on the rest, lam~' >= the largest
    # remaining |lam| (Theorem 2 for X').
    X, Q, lam = spectral64("powerlaw", 200, 7)
    r = oracle.deflate_project(X, 16, COEFS, SCALES, tol=1e-11)
    k = r["k"]
    assert 4 <= k <= 16
    order = np.argsort(-np.abs(lam))
    defl = set(order[:k].tolist())
    assert any(lam[i] < 0 for i in defl) and any(lam[i] > 0 for i in defl)
    rest = np.array([i not in defl for i in range(len(lam))])
    top_rest = np.max(np.abs(lam[rest]))
    lt2 = r["lam_tilde_defl"]
    assert top_rest <= lt2 <= 1.01 * top_rest
    psi = np.maximum(lam, 0.0)
    psi[rest] = oracle.phi(lam[rest], lt2, COEFS, SCALES)
    want = oracle.spectral(lam, Q, psi)
    assert np.linalg.norm(r["out"] - want) <= 1e-9 * np.linalg.norm(want)


def test_low_rank_input_gives_the_exact_projection():
    # rank 6 with distinct |lam|: K_m(X^2, q_0) = span(q_0) + range(X) after 7
    # steps (breakdown), every nonzero eigenpair is deflated (plus, possibly,
    # the null-space direction of q_0 with mu ~ 1e-17) and X' = 0, so the
    # result is Pi(X) itself (no filter error at all).
    n, r = 120, 6
    rng = np.random.default_rng(11)
    U, _ = np.linalg.qr(rng.standard_normal((n, r)))
    lam = np.array([3.0, -2.5, 1.7, -1.1, 0.6, 0.25])
    X = (U * lam[None, :]) @ U.T
    res = oracle.deflate_project(X, 16, COEFS, SCALES)
    assert res["k"] in (r, r + 1)
    np.testing.assert_allclose(res["mu"][:r], lam, atol=1e-13)
    assert res["k"] == r or abs(res["mu"][r]) < 1e-14
    P = (U * np.maximum(lam, 0)[None, :]) @ U.T
    assert np.linalg.norm(res["out"] - P) <= 1e-12 * np.linalg.norm(P)


def test_kmax_bounds_the_deflated_set():
    X, _, _ = spectral64("powerlaw", 150, 9)
    full = oracle.deflate_project(X, 16, COEFS, SCALES)
    for kmax in (1, 3):
        r = oracle.deflate_project(X, kmax, COEFS, SCALES)
        assert r["k"] <= kmax
        assert r["keep"] == [j for j in full["keep"] if j < kmax]


def test_deflation_improves_powerlaw_and_leaves_uniform():
    # The Sec. 6 failure mode: the power-law spectrum's small eigenvalues sit
    # in the composite's unresolved band around 0; deflating the dominant
    # pairs rescales the rest and cuts the error by orders of magnitude.  A
    # uniform spectrum has no converged dominant pair: nothing changes.
    X, Q, lam = spectral64("powerlaw", 300, 11)
    P = oracle.project_from_eig(lam, Q)
    r = oracle.deflate_project(X, 16, COEFS, SCALES)
    F0 = oracle.filter_from_eig(lam, Q, oracle.lanczos_bound(X)["lam_tilde"], COEFS, SCALES)
    e0 = np.linalg.norm(F0 - P) / np.linalg.norm(P)
    e1 = np.linalg.norm(r["out"] - P) / np.linalg.norm(P)
    assert r["k"] >= 8 and e1 < e0 / 10
    Xu, Qu, lamu = spectral64("uniform", 300, 11)
    ru = oracle.deflate_project(Xu, 16, COEFS, SCALES)
    assert ru["k"] == 0
