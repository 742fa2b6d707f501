"""Stage I of the coefficient design: the sequential Remez construction of the
composite sign approximation (Algorithm 1, Sec. 3.1) with the Remez algorithm
of the appendix ("Remez Algorithm", Algorithm 3).

TEST INFRASTRUCTURE ONLY: part of the CPU FP64 oracle (only ``tests/``,
``__graft_entry__.smoke()`` and the cpu_baseline / reference leg of
``bench.py`` may import it).  It regenerates the f* columns of Tables 1 and 2
from (eps, T, d_t = 5), independently of their transcription in
``schedules.py``.

Problem of stage t (Algorithm 1): f*_t is the minimax odd polynomial of degree
d_t for sign(x) on [-b_t, -a_t] U [a_t, b_t]; by oddness (Eq. remez-1) it is the
minimax approximation of the constant 1 on [a_t, b_t] in the basis
Phi = {x, x^3, ..., x^d}, which is a Haar space on [a_t, b_t] since a_t > 0.  The
next interval is the image [a_{t+1}, b_{t+1}] = f*_t([a_t, b_t]) (Eq.
update-interval).

Remez steps (appendix), for m = (d + 1) / 2 basis functions:
  0. start from m + 1 Chebyshev nodes x_1 < ... < x_{m+1} on [a, b];
  1. solve sum_l c_l phi_l(x_i) - g(x_i) = (-1)^i E for (c, E);
  2. find the m roots z_1 < ... < z_m of e(x) = sum_l c_l phi_l(x) - g(x), one
     between consecutive nodes;
  3. on each sub-interval [z_{i-1}, z_i] (z_0 = a, z_{m+1} = b) take the point
     where e attains its maximum if e(x_i) > 0, its minimum otherwise;
  4. stop when the new points agree with the old ones, else exchange.
Step 3 evaluates e at the sub-interval's end points and at the critical points
of e inside it; e'(x) is an even polynomial, so its critical points are the
square roots of the positive roots of a polynomial in u = x^2 (numpy.roots).
"""
import numpy as np


def _basis(x, m):
    """phi_l(x) = x^(2l - 1), l = 1..m, as columns."""
    x = np.asarray(x, dtype=np.float64)
    return np.stack([x ** (2 * l - 1) for l in range(1, m + 1)], axis=-1)


def _poly(c, x):
    return _basis(x, len(c)) @ np.asarray(c, dtype=np.float64)


def _critical_points(c, lo, hi):
    """Points of (lo, hi) where d/dx sum_l c_l x^(2l-1) = 0."""
    m = len(c)
    # derivative sum_l (2l - 1) c_l u^(l - 1), u = x^2; numpy.roots wants the
    # highest power first
    coef = [(2 * l - 1) * c[l - 1] for l in range(m, 0, -1)]
    while len(coef) > 1 and coef[0] == 0.0:
        coef = coef[1:]
    out = []
    if len(coef) > 1:
        for u in np.roots(coef):
            if abs(u.imag) <= 1e-12 * max(1.0, abs(u.real)) and u.real > 0:
                x = float(np.sqrt(u.real))
                if lo < x < hi:
                    out.append(x)
    return out


def _bisect_root(f, lo, hi, iters=200):
    flo = f(lo)
    for _ in range(iters):
        mid = 0.5 * (lo + hi)
        fm = f(mid)
        if fm == 0.0:
            return mid
        if (fm > 0) == (flo > 0):
            lo, flo = mid, fm
        else:
            hi = mid
        if hi - lo <= 4 * np.finfo(float).eps * max(abs(lo), abs(hi)):
            break
    return 0.5 * (lo + hi)


def limit_odd(d=5):
    """The confluent limit of remez_odd(1 - h, 1 + h, d) as h -> 0: the odd
    polynomial of degree d with f(1) = 1 and f^(k)(1) = 0 for k = 1..m-1
    (m = (d + 1) / 2 conditions); for d = 5, (15 x - 10 x^3 + 3 x^5) / 8."""
    m = (d + 1) // 2
    A = np.zeros((m, m))
    rhs = np.zeros(m)
    for k in range(m):          # k-th derivative at x = 1 of x^(2l - 1)
        for l in range(1, m + 1):
            p = 2 * l - 1
            coef = 1.0
            for q in range(k):
                coef *= (p - q)
            A[k, l - 1] = coef if p >= k else 0.0
    rhs[0] = 1.0
    return tuple(float(v) for v in np.linalg.solve(A, rhs))


# Below this interval width the alternation system of remez_odd is too
# ill-conditioned in FP64 (x, x^3, x^5 are nearly dependent near x = 1) and the
# stage is the confluent limit, which the minimax polynomial approaches as
# O(width^2): the printed f*_single stages 9 and 10 are exactly that limit.
COLLAPSED_WIDTH = 1e-4


def remez_odd(a, b, d=5, g=lambda x: np.ones_like(np.asarray(x, dtype=np.float64)), max_iter=100, tol=1e-12):
    """Minimax odd polynomial of degree d approximating g on [a, b] (0 < a < b).

    Returns dict(coef=(c_1, ..., c_m) for x, x^3, ..., E=|error| levelled,
    nodes=alternation points, iters=Remez iterations).
    """
    if not (0 < a < b):
        raise ValueError("need 0 < a < b")
    m = (d + 1) // 2
    k = np.arange(m + 1)
    # step 0: Chebyshev nodes of [a, b] in increasing order
    x = 0.5 * (a + b) - 0.5 * (b - a) * np.cos(np.pi * k / m)
    sign = (-1.0) ** (k + 1)  # (-1)^i for i = 1..m+1
    c, E = None, None
    for it in range(1, max_iter + 1):
        # step 1: alternation system
        A = np.concatenate([_basis(x, m), -sign[:, None]], axis=1)
        sol = np.linalg.solve(A, g(x))
        c, E = sol[:m], sol[m]
        e = lambda t: _poly(c, t) - g(t)
        # step 2: one root of e between consecutive nodes
        z = [_bisect_root(e, x[i], x[i + 1]) for i in range(m)]
        edges = [a] + z + [b]
        # step 3: the extremum of e on each sub-interval, of the sign e(x_i) has
        y = np.empty_like(x)
        for i in range(m + 1):
            lo, hi = edges[i], edges[i + 1]
            cand = np.array([lo, hi] + _critical_points(c, lo, hi))
            vals = e(cand)
            y[i] = cand[np.argmax(vals)] if e(x[i]) > 0 else cand[np.argmin(vals)]
        # step 4: convergence
        done = np.max(np.abs(y - x)) <= tol * (b - a)
        x = y
        if done:
            break
    return dict(coef=tuple(float(v) for v in c), E=abs(float(E)), nodes=tuple(float(v) for v in x), iters=it)


def sequential_remez(eps, T, degrees=5):
    """Algorithm 1: returns dict(coef=[(a_t, b_t, c_t), ...], intervals=[(a_t, b_t), ...], E=[E_t, ...])."""
    degs = [degrees] * T if np.isscalar(degrees) else list(degrees)
    lo, hi = float(eps), 1.0
    coefs, intervals, errs = [], [], []
    for t in range(T):
        if hi - lo < COLLAPSED_WIDTH:
            c = limit_odd(degs[t])
            cand = np.array([lo, hi] + _critical_points(c, lo, hi))
            r = dict(coef=c, E=float(np.max(np.abs(_poly(c, cand) - 1.0))))
        else:
            r = remez_odd(lo, hi, degs[t])
        coefs.append(r["coef"])
        intervals.append((lo, hi))
        errs.append(r["E"])
        # image of [lo, hi] under f*_t: the extrema over the end points and the
        # critical points (for the minimax polynomial, [1 - E_t, 1 + E_t])
        cand = np.array([lo, hi] + _critical_points(r["coef"], lo, hi))
        vals = _poly(r["coef"], cand)
        lo, hi = float(np.min(vals)), float(np.max(vals))
    return dict(coef=coefs, intervals=intervals, E=errs)
