"""Deflation of the dominant eigenpairs before the composite filter.

TEST INFRASTRUCTURE ONLY: part of the CPU FP64 oracle (only ``tests/``,
``__graft_entry__.smoke()`` and the cpu_baseline / reference leg of
``bench.py`` may import it).

Sec. 6 (Limitations) names deflation of dominant eigenvalues as the remedy for
spectra in which a few eigenvalues of large modulus push the rest into the
band around 0 that the composite resolves poorly; the paper gives no
algorithm.  The library's reading, taken here step by step:

  1. the norm bound of X (``lanczos_bound``: 20 Lanczos steps on X^2) and its
     orthonormal basis Q_m of the Krylov space K_m(X^2, q_0);
  2. Rayleigh-Ritz with X on span(Q_m): H = Q_m^T X Q_m = W diag(mu) W^T,
     Ritz vectors v_j = Q_m w_j ordered by |mu_j| descending;
  3. of the first kmax pairs, those with ||X v_j - mu_j v_j||_2 <= tol lam~
     (and mu_j != 0) are deflated: X' = X - V diag(mu) V^T;
  4. F(X') with X''s own norm bound lam~' (what Algorithm 2 returns for X' in
     exact arithmetic);
  5. the result F(X') + V diag(max(mu, 0)) V^T.

If span(V) is invariant under X (residuals 0), X' annihilates span(V) and the
result is Q diag(psi) Q^T with psi = max(lam, 0) on the deflated eigenpairs and
psi = phi(lam; lam~') on the others: the closed form the tests pin it to.
"""
import numpy as np

from .core import eigh_jacobi, filter_from_eig, lanczos_bound

DEFLATE_TOL = 1e-6


def ritz_pairs(X, bound=None):
    """Steps 1-2: Ritz pairs of X on the norm bound's Lanczos basis.

    Returns (mu, V, resid, bound): mu (m,), V (n, m) columns v_j, resid (m,)
    = ||X v_j - mu_j v_j||_2, ordered by |mu| descending (ties keep the
    ascending eigenvalue order of the decomposition).
    """
    X = np.asarray(X, dtype=np.float64)
    if bound is None:
        bound = lanczos_bound(X)
    Qm = bound["Q"]
    Z = X @ Qm
    H = Qm.T @ Z
    H = 0.5 * (H + H.T)
    mu, W = eigh_jacobi(H)
    order = np.argsort(-np.abs(mu), kind="stable")
    mu, W = mu[order], W[:, order]
    V = Qm @ W
    R = Z @ W - V * mu[None, :]
    resid = np.linalg.norm(R, axis=0)
    return mu, V, resid, bound


def deflate_project(X, kmax, coefs, scales, tol=DEFLATE_TOL):
    """Steps 1-5 for a symmetric X (FP64).  Returns dict(out, k, keep (indices
    into the Ritz order), mu, resid, lam_tilde (of X), lam_tilde_defl (of X'),
    X_defl)."""
    X = np.asarray(X, dtype=np.float64)
    mu, V, resid, bound = ritz_pairs(X)
    lt = bound["lam_tilde"]
    keep = [j for j in range(min(kmax, len(mu))) if mu[j] != 0.0 and resid[j] <= tol * lt]
    Vk, Mk = V[:, keep], mu[keep]
    Xd = X - (Vk * Mk[None, :]) @ Vk.T
    Xd = 0.5 * (Xd + Xd.T)
    bd = lanczos_bound(Xd)
    lam, Q = eigh_jacobi(Xd)
    F = filter_from_eig(lam, Q, bd["lam_tilde"], coefs, scales)
    out = F + (Vk * np.maximum(Mk, 0.0)[None, :]) @ Vk.T
    return dict(out=out, k=len(keep), keep=keep, mu=mu, resid=resid, lam_tilde=lt,
                lam_tilde_defl=bd["lam_tilde"], X_defl=Xd)
