"""Pins of the oracle's scalar composite polynomial against what the paper prints.

The composite g and the scan over every float32 value are checked against the
e_float values printed in Tables 1 and 2, the Stage-I construction of
Algorithm 1 (equioscillation of each Remez polynomial on its interval), the
closed-form limit polynomial of Table 1, and the count of Sec. 3.2.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import schedules as S
from oracle.core import stage_image

TABLES = {
    "single_fstar": S.SINGLE_FSTAR,
    "single_ftilde": S.SINGLE_FTILDE,
    "half_fstar": S.HALF_FSTAR,
    "half_ftilde": S.HALF_FTILDE,
}


@pytest.fixture(scope="module")
def scans():
    return {k: oracle.efloat(v) for k, v in TABLES.items()}


def test_table_shapes():
    # Sec. 3.3: T = 10 (single), T = 7 (half); 3T + 1 GEMMs = 31 and 22.
    assert len(S.SINGLE_FSTAR) == len(S.SINGLE_FTILDE) == 10
    assert len(S.HALF_FSTAR) == len(S.HALF_FTILDE) == 7
    assert 3 * len(S.SINGLE_FTILDE) + 1 == 31
    assert 3 * len(S.HALF_FTILDE) + 1 == 22


def test_s_float_count(scans, golden):
    # Sec. 3.2: |S_float| float32 values in [-1, 1]; the scan visits [0, 1]
    # (the errors are even in x), so 2 * count - 1 (zero counted once).
    want = int(golden("e_float.txt")["s_float_count"])
    for r in scans.values():
        assert 2 * r["count"] - 1 == want


@pytest.mark.parametrize("key", ["single_ftilde", "half_fstar", "half_ftilde"])
def test_efloat_matches_printed(scans, golden, key):
    # The printed e_float reproduces as max |x g(x) - |x||, i.e. twice the
    # ReLU error of x (1 + g) / 2 (reading recorded with the oracle).
    printed = float(golden("e_float.txt")[key])
    got = scans[key]["doubled"]
    assert abs(got - printed) / printed < 1e-2, (key, got, printed)
    assert scans[key]["relu"] * 2 == pytest.approx(got, rel=1e-12)


def test_efloat_single_fstar_not_above_printed(scans, golden):
    # The one table whose printed e_float does not reproduce: the recomputed
    # value is smaller than the printed one (see the stage-I check below: this
    # column equioscillates from x = 1e-4, not from eps = 1e-3).
    printed = float(golden("e_float.txt")["single_fstar"])
    assert scans["single_fstar"]["doubled"] <= printed


def test_refinement_lowers_error(scans):
    # Sec. 3.2: Stage II lowers the ReLU error of the Stage-I initialisation.
    assert scans["half_ftilde"]["relu"] < scans["half_fstar"]["relu"]


def _alternation(coef, a, b):
    lo, hi, cands = stage_image(coef, a, b)
    xs = sorted(cands)
    errs = [coef[0] * x + coef[1] * x ** 3 + coef[2] * x ** 5 - 1.0 for x in xs]
    return lo, hi, xs, errs


@pytest.mark.parametrize("name,eps1", [("half", 1e-3), ("single", 1e-4)])
def test_stage1_equioscillation(name, eps1):
    # Algorithm 1: f*_t is the minimax odd quintic for sign on [a_t, b_t], so
    # f*_t - 1 equioscillates at 4 points (Chebyshev alternation in the Haar
    # space span{x, x^3, x^5}) and [a_{t+1}, b_{t+1}] = f*_t([a_t, b_t]).
    # A wrong digit or sign in a coefficient breaks the alternation.  The
    # tolerance (1e-4 E + 2e-6) covers the drift of the intervals propagated here
    # with the printed 10-digit coefficients.
    table = S.HALF_FSTAR if name == "half" else S.SINGLE_FSTAR
    a, b = eps1, 1.0
    for t, coef in enumerate(table):
        lo, hi, xs, errs = _alternation(coef, a, b)
        E = 0.5 * (hi - lo)
        if E > 1e-6:
            assert len(errs) == 4
            for k, e in enumerate(errs):
                assert abs(abs(e) - E) <= 1e-4 * E + 2e-6, (name, t + 1, errs)
                if k:
                    assert np.sign(e) == -np.sign(errs[k - 1])
        # the image interval is centred on 1 (both ends at distance E)
        assert abs(0.5 * (lo + hi) - 1.0) < 1e-5
        a, b = lo, hi
    assert abs(a - 1.0) < 1e-8 and abs(b - 1.0) < 1e-8


def test_single_fstar_first_stage_uses_eps_1e4():
    # Reading recorded with the oracle: with eps = 1e-3 the error of f*_1 at
    # the left end (about 0.9915) is below the alternation level E = 0.99915,
    # i.e. the polynomial is not the minimax on [1e-3, 1]; at eps = 1e-4 it is.
    coef = S.SINGLE_FSTAR[0]
    lo, hi, xs, errs = _alternation(coef, 1e-3, 1.0)
    E = 0.5 * (hi - lo)
    assert abs(errs[0]) < E - 5e-3
    lo, hi, xs, errs = _alternation(coef, 1e-4, 1.0)
    E = 0.5 * (hi - lo)
    assert all(abs(abs(e) - E) < 1e-6 for e in errs)


def test_limit_polynomial_closed_form():
    # Table 1: f*_9 = f*_10 = (15 x - 10 x^3 + 3 x^5) / 8, with f(1) = 1 and
    # f'(1) = f''(1) = 0 (the fixed point 1 is of third order).
    for coef in S.SINGLE_FSTAR[8:]:
        assert coef == (15 / 8, -10 / 8, 3 / 8)
    a, b, c = S.SINGLE_FSTAR[9]
    assert a + b + c == pytest.approx(1.0, abs=1e-15)
    assert a + 3 * b + 5 * c == pytest.approx(0.0, abs=1e-15)
    assert 6 * b + 20 * c == pytest.approx(0.0, abs=1e-15)


def test_composite_is_odd_bitwise():
    x = np.linspace(0, 1, 10001)
    for tab in TABLES.values():
        assert np.array_equal(oracle.composite(-x, tab), -oracle.composite(x, tab))


def test_composite_slope_at_zero():
    # g'(0) = prod_t a_t / s_t (chain rule; only the linear terms survive).
    for name in ("half", "single"):
        coefs, scales = S.schedule(name)
        h = 1e-9
        slope = (oracle.composite(h, coefs, scales) - oracle.composite(-h, coefs, scales)) / (2 * h)
        want = math.prod(c[0] / s for c, s in zip(coefs, scales))
        assert slope == pytest.approx(want, rel=1e-5)


def test_rescale_reading():
    # Sec. 3.4 rescale.  Dividing after stages 1..T-1 keeps the ReLU error of
    # the half filter at the level of e_float; dividing the final iterate too
    # would bias every positive eigenvalue by (1 - 1/1.01) / 2 ~ 0.5 %.
    x = np.linspace(-1, 1, 400001)
    relu = np.maximum(x, 0)
    err = {}
    for kind in ("none", "half", "half_all"):
        sc = S.post_scale(kind, 7)
        err[kind] = float(np.max(np.abs(oracle.relu_approx(x, S.HALF_FTILDE, sc) - relu)))
    assert err["none"] < 2.5e-5
    assert err["half"] < 6e-5
    assert err["half_all"] > 4e-3
    # single: 1/1.001 after the first eight stages
    sc = S.post_scale("single", 10)
    es = float(np.max(np.abs(oracle.relu_approx(x, S.SINGLE_FTILDE, sc) - relu)))
    assert es < 1e-5


def test_composite_bounded_beyond_one():
    # Overshoot margin used by the bound check: a spectrum slightly above the
    # bound (|x| <= 1.02 for half, 1.01 for single) stays bounded by 1.05.
    for name, top in (("half", 1.02), ("single", 1.01)):
        coefs, scales = S.schedule(name)
        x = np.linspace(-top, top, 200001)
        assert float(np.max(np.abs(oracle.composite(x, coefs, scales)))) < 1.05
