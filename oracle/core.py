"""Plain CPU FP64 oracle of the composite-polynomial PSD-cone projection.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  Slow and direct on purpose:
each function states the passage of the paper it follows.  No blocking, no
fusion, no reordering beyond what the definition or algorithm states; numpy's
matmul is used as a library primitive for matrix products.
"""
import math

import numpy as np

from . import _clib
from .schedules import LANCZOS_STEPS

# ---------------------------------------------------------------------------
# Eigen-decomposition (cyclic Jacobi in C) and the two spectral operators.
# ---------------------------------------------------------------------------


def eigh_jacobi(X, max_sweeps=40, tol=1e-14):
    """Eigen-decomposition X = Q diag(lam) Q^T of a symmetric matrix, FP64.

    Cyclic Jacobi (Golub & Van Loan Sec. 8.5) in oracle.c.  Returns lam in
    ascending order and Q with the matching columns.  Ties may come in any
    order; Pi(X) and F(X) do not depend on the basis inside an eigenspace.
    """
    A = np.array(X, dtype=np.float64, order="C", copy=True)
    n = A.shape[0]
    if A.shape != (n, n):
        raise ValueError("square matrix expected")
    if n == 0:
        return np.zeros(0), np.zeros((0, 0))
    w = np.zeros(n)
    V = np.zeros((n, n))
    sweeps = _clib.lib().oracle_jacobi_eig(n, _clib.dptr(A), _clib.dptr(w), _clib.dptr(V),
                                           int(max_sweeps), float(tol))
    if sweeps >= max_sweeps:
        raise RuntimeError("Jacobi did not converge in %d sweeps" % max_sweeps)
    order = np.argsort(w, kind="stable")
    return w[order], V[:, order]


def spectral(lam, Q, values):
    """Spectral operator Q diag(values) Q^T (Sec. 1, spectral operator)."""
    return (Q * np.asarray(values, dtype=np.float64)[None, :]) @ Q.T


def project_from_eig(lam, Q):
    """Exact PSD projection Pi(X) = Q diag(max(lam, 0)) Q^T (Sec. 1, Higham)."""
    return spectral(lam, Q, np.maximum(lam, 0.0))


# ---------------------------------------------------------------------------
# The scalar composite polynomial.
# ---------------------------------------------------------------------------


def composite(x, coefs, scales=None):
    """g(x) = s_T^-1 f_T( ... s_1^-1 f_1(x)), f_t(x) = a_t x + b_t x^3 + c_t x^5.

    Sec. 1 (composite filter p = f_T o ... o f_1), Sec. 3.3 (d_t = 5, odd),
    Sec. 3.4 (the 1/s_t rescale after stage t).  FP64, elementwise; each
    quintic is evaluated as x (a + x^2 (b + x^2 c)), which is odd bit for bit.
    """
    x = np.array(x, dtype=np.float64, copy=True)
    T = len(coefs)
    if scales is None:
        scales = (1.0,) * T
    for (a, b, c), s in zip(coefs, scales):
        x2 = x * x
        x = x * (a + x2 * (b + x2 * c))
        x = x / s
    return x


def relu_approx(x, coefs, scales=None):
    """f~(x) = x (1 + g(x)) / 2, the ReLU approximation of Sec. 3.2."""
    x = np.asarray(x, dtype=np.float64)
    return 0.5 * x * (1.0 + composite(x, coefs, scales))


def phi(lam, lam_tilde, coefs, scales):
    """The scalar map the run-time algorithm applies to each eigenvalue.

    Algorithm 2 scales by lam_tilde, runs the T stages and returns
    lam_tilde * X0 (I + X_T) / 2, so eigenvalue l becomes
    lam_tilde * (l / lam_tilde) * (1 + g(l / lam_tilde)) / 2 = l (1 + g(l/lam_tilde)) / 2.
    For lam_tilde == 0 (X == 0) the result is 0.
    """
    lam = np.asarray(lam, dtype=np.float64)
    if lam_tilde == 0.0:
        return np.zeros_like(lam)
    return 0.5 * lam * (1.0 + composite(lam / lam_tilde, coefs, scales))


def filter_from_eig(lam, Q, lam_tilde, coefs, scales):
    """F(X) = Q diag(phi(lam_i)) Q^T: what Algorithm 2 returns in exact arithmetic."""
    return spectral(lam, Q, phi(lam, lam_tilde, coefs, scales))


# ---------------------------------------------------------------------------
# Norm bound: 20-step Lanczos on X^2 and Theorem 2.
# ---------------------------------------------------------------------------

_MASK64 = (1 << 64) - 1
_GOLDEN = 0x9E3779B97F4A7C15
LANCZOS_SEED = 0x243F6A8885A308D3  # fixed seed of the start vector


def splitmix64(seed, count):
    """Counter-based SplitMix64 (Steele, Lea & Flood, OOPSLA 2014).

    Element i is the SplitMix64 output for state seed + (i + 1) * golden-gamma.
    """
    i = np.arange(1, count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & _MASK64) + i * np.uint64(_GOLDEN)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return z


def lanczos_start(n, seed=LANCZOS_SEED):
    """Start vector: v_i = 2 u_i - 1 with u_i = (SplitMix64_i >> 11) * 2^-53, then unit length."""
    z = splitmix64(seed, n)
    u = (z >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
    v = 2.0 * u - 1.0
    return v / np.linalg.norm(v)


def lanczos_bound(X, steps=LANCZOS_STEPS, seed=LANCZOS_SEED, breakdown=1e-12):
    """Upper bound lam_tilde of ||X||_2 (Sec. 3.4, Theorem 2; Algorithm 2 steps 1-2).

    Lanczos (Parlett, The Symmetric Eigenvalue Problem, Ch. 13) on A = X^2 with
    A q computed as X (X q), FP64, full re-orthogonalisation against all
    previous Lanczos vectors (classical Gram-Schmidt applied twice).  The
    largest Ritz pair (sigma, q) of the m x m tridiagonal T_m gives
        lam_tilde = sqrt(sigma + ||X^2 q - sigma q||_2).
    Readings (the paper gives no more detail):
      * start vector: lanczos_start(n) (SplitMix64, fixed seed);
      * stop early when beta_j <= breakdown * ||X||_F^2 (an invariant Krylov
        space, e.g. n < 20 or low rank; ||X||_F^2 >= ||X^2||_2 sets the scale);
      * lam_tilde is raised to max(., ||X||_F / sqrt(n), max_i |X_ii|): both are
        lower bounds of ||X||_2, so a Lanczos value below them is certainly not
        an upper bound.
    Returns a dict with lam_tilde, sigma, resid, m, alpha, beta, beta_m (the
    norm of the m-th residual vector), y (Ritz vector in the Lanczos basis),
    fro, maxdiag, Q (the n x m Lanczos basis).
    """
    X = np.asarray(X, dtype=np.float64)
    n = X.shape[0]
    fro = float(np.sqrt(np.sum(X * X)))
    maxdiag = float(np.max(np.abs(np.diag(X)))) if n else 0.0
    if n == 0:
        return dict(lam_tilde=0.0, sigma=0.0, resid=0.0, m=0, alpha=[], beta=[], beta_m=0.0,
                    y=np.zeros(0), fro=0.0, maxdiag=0.0, Q=np.zeros((0, 0)))
    Qv = np.zeros((n, steps))
    alpha = []
    beta = []
    q = lanczos_start(n, seed)
    q_prev = np.zeros(n)
    b_prev = 0.0
    m = 0
    for j in range(steps):
        Qv[:, j] = q
        w = X @ (X @ q)
        a = float(q @ w)
        w = w - a * q - b_prev * q_prev
        for _ in range(2):  # full re-orthogonalisation, twice
            h = Qv[:, : j + 1].T @ w
            w = w - Qv[:, : j + 1] @ h
        b = float(np.linalg.norm(w))
        alpha.append(a)
        m = j + 1
        beta_m = b
        if b <= breakdown * fro * fro or j == steps - 1:
            break
        beta.append(b)
        q_prev, q, b_prev = q, w / b, b
    T = np.diag(alpha) + np.diag(beta[: m - 1], 1) + np.diag(beta[: m - 1], -1)
    theta, Y = eigh_jacobi(T)
    sigma = float(theta[-1])
    y = Y[:, -1]
    qr = Qv[:, :m] @ y
    qr = qr / np.linalg.norm(qr)
    r = X @ (X @ qr) - sigma * qr
    resid = float(np.linalg.norm(r))
    lam = math.sqrt(max(sigma + resid, 0.0))
    lam = max(lam, fro / math.sqrt(n), maxdiag)
    return dict(lam_tilde=lam, sigma=sigma, resid=resid, m=m, alpha=alpha, beta=beta[: m - 1],
                beta_m=beta_m, y=y, fro=fro, maxdiag=maxdiag, Q=Qv[:, :m].copy())


# ---------------------------------------------------------------------------
# Algorithm 2 evaluated step by step in FP64 (a second route to F(X)).
# ---------------------------------------------------------------------------


def chain_fp64(X, lam_tilde, coefs, scales):
    """Algorithm 2 after the bound, in FP64 with library matmuls.

    X0 = X / lam_tilde; for t = 1..T: X_t = f_t(X_{t-1}) / s_t with
    f_t(Z) = Z (a I + b Z^2 + c Z^4) formed from the three products Z^2,
    (Z^2)^2 and Z (.) (Sec. 3.3: 3 GEMMs per quintic); return
    lam_tilde * X0 (I + X_T) / 2.  Returns (result, X_T).
    """
    X = np.asarray(X, dtype=np.float64)
    n = X.shape[0]
    if lam_tilde == 0.0:
        return np.zeros_like(X), np.zeros_like(X)
    I = np.eye(n)
    X0 = X / lam_tilde
    Xt = X0
    for (a, b, c), s in zip(coefs, scales):
        Y = Xt @ Xt
        P = a * I + b * Y + c * (Y @ Y)
        Xt = (Xt @ P) / s
    out = lam_tilde * 0.5 * (X0 @ (I + Xt))
    return out, Xt


# ---------------------------------------------------------------------------
# Metrics (Sec. 4.1: relative Frobenius error, FP64).
# ---------------------------------------------------------------------------


def rel_err(A, ref, X=None):
    """||A - ref||_F / ||ref||_F in FP64 (Sec. 4.1).

    When ||ref||_F == 0 (the projection of an NSD matrix) the error is taken
    relative to ||X||_F instead (absolute error if X is not given).
    """
    A = np.asarray(A, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    num = float(np.linalg.norm(A - ref))
    den = float(np.linalg.norm(ref))
    if den == 0.0:
        den = float(np.linalg.norm(X)) if X is not None else 1.0
        if den == 0.0:
            den = 1.0
    return num / den


BANDS = ((0.0, 1e-4), (1e-4, 1e-3), (1e-3, 1e-2), (1e-2, 1e-1), (1e-1, 1.0 + 1e-12))


def band_errors(A, ref, lam, Q):
    """Error per eigenvalue band: ||(A - ref) Q_B||_F / ||X Q_B||_F.

    Bands of |lam| / ||X||_2 (BANDS), split by sign; Q_B are the eigenvectors
    of X in the band, X Q_B = Q_B diag(lam_B).  Returns a list of
    (sign, lo, hi, count, error).
    """
    A = np.asarray(A, dtype=np.float64)
    D = A - np.asarray(ref, dtype=np.float64)
    top = float(np.max(np.abs(lam))) if len(lam) else 1.0
    rel = np.abs(lam) / (top if top > 0 else 1.0)
    out = []
    for sign in (1, -1):
        for lo, hi in BANDS:
            sel = (rel >= lo) & (rel < hi) & ((lam > 0) if sign > 0 else (lam <= 0))
            k = int(np.sum(sel))
            if k == 0:
                out.append((sign, lo, hi, 0, float("nan")))
                continue
            QB = Q[:, sel]
            den = float(np.linalg.norm(lam[sel]))
            num = float(np.linalg.norm(D @ QB))
            out.append((sign, lo, hi, k, num / den if den > 0 else float("nan")))
    return out


def efloat(coefs, scales=None):
    """Discretised error over all float32 x in [-1, 1] (Sec. 3.2, e_float).

    Returns dict(relu=max |x(1+g)/2 - relu(x)|, doubled=max |x g - |x||,
    argmax=x of the ReLU maximum, count=number of float32 values in [0, 1]).
    """
    T = len(coefs)
    if scales is None:
        scales = (1.0,) * T
    coef = np.ascontiguousarray(np.array(coefs, dtype=np.float64).reshape(-1))
    inv_s = np.ascontiguousarray(1.0 / np.array(scales, dtype=np.float64))
    out = np.zeros(4)
    _clib.lib().oracle_efloat_scan(T, _clib.dptr(coef), _clib.dptr(inv_s), _clib.dptr(out))
    return dict(relu=out[0], doubled=out[1], argmax=out[2], count=int(out[3]))


def stage_image(coef, a, b):
    """Image [min f, max f] of f(x) = a1 x + b1 x^3 + c1 x^5 over [a, b].

    Algorithm 1 step (2): the next interval is the image of the current one.
    Extrema are at the end points or at the real roots of f'(x) in [a, b].
    """
    a1, b1, c1 = coef
    cands = [a, b]
    # f'(x) = a1 + 3 b1 x^2 + 5 c1 x^4, a quadratic in y = x^2
    for y in np.roots([5.0 * c1, 3.0 * b1, a1]):
        if abs(y.imag) < 1e-14 and y.real > 0:
            x = math.sqrt(y.real)
            if a <= x <= b:
                cands.append(x)
    vals = [a1 * x + b1 * x ** 3 + c1 * x ** 5 for x in cands]
    return min(vals), max(vals), cands
