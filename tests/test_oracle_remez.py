"""Stage I coefficient design (Algorithm 1 with the appendix's Remez
algorithm) against what the paper prints and closed forms.

Pins: the f* columns of Table 2 (half, eps = 1e-3, T = 7) and Table 1
(single, T = 10) to their printed 10 decimals; the degree-1 minimax of the
constant 1 on [a, b] (c = 2 / (a + b), E = (b - a) / (b + a)); the confluent
limit (15 x - 10 x^3 + 3 x^5) / 8; equioscillation of every stage; the stage
images [1 - E_t, 1 + E_t] (Eq. update-interval)."""
import numpy as np
import pytest

from oracle import remez
from oracle import schedules as S


def max_diff(gen, ref):
    return max(abs(a - b) for c1, c2 in zip(gen, ref) for a, b in zip(c1, c2))


def test_half_fstar_column_reproduced():
    r = remez.sequential_remez(1e-3, 7)
    assert max_diff(r["coef"], S.HALF_FSTAR) < 1e-9


def test_single_fstar_column_reproduced_from_eps_1e4():
    # The single column is the Algorithm-1 output for eps = 1e-4, not the
    # stated 1e-3 (reading R2); its last two stages are the confluent limit.
    r = remez.sequential_remez(1e-4, 10)
    assert max_diff(r["coef"], S.SINGLE_FSTAR) < 1e-9
    r3 = remez.sequential_remez(1e-3, 10)
    assert max_diff(r3["coef"][:6], S.SINGLE_FSTAR[:6]) > 1e-2


@pytest.mark.parametrize("a,b", [(1e-3, 1.0), (0.2, 0.9), (0.5, 3.0)])
def test_degree_one_closed_form(a, b):
    r = remez.remez_odd(a, b, d=1)
    assert r["coef"][0] == pytest.approx(2.0 / (a + b), rel=1e-13)
    assert r["E"] == pytest.approx((b - a) / (b + a), rel=1e-12)


def test_confluent_limit_closed_form():
    c = remez.limit_odd(5)
    assert np.allclose(c, (15 / 8, -10 / 8, 3 / 8), rtol=0, atol=1e-15)
    # and it is what the minimax polynomial approaches on shrinking intervals
    for h in (1e-2, 3e-3):
        r = remez.remez_odd(1 - h, 1 + h, 5)
        assert max(abs(x - y) for x, y in zip(r["coef"], c)) < 10 * h * h


@pytest.mark.parametrize("eps,T", [(1e-3, 7), (1e-4, 10)])
def test_every_stage_equioscillates_and_maps_to_its_image(eps, T):
    r = remez.sequential_remez(eps, T)
    for t, ((lo, hi), c, E) in enumerate(zip(r["intervals"], r["coef"], r["E"])):
        if hi - lo < remez.COLLAPSED_WIDTH:
            continue
        out = remez.remez_odd(lo, hi, 5)
        x = np.array(out["nodes"])
        e = remez._poly(out["coef"], x) - 1.0
        assert np.all(np.sign(e[1:]) == -np.sign(e[:-1]))          # alternation
        assert np.allclose(np.abs(e), E, rtol=1e-9, atol=1e-15)     # equal ripple
        assert x[0] == lo and x[-1] == hi                          # end points are extremal
        # the error never exceeds E on a dense grid of the interval
        g = np.linspace(lo, hi, 20001)
        assert np.max(np.abs(remez._poly(out["coef"], g) - 1.0)) <= E * (1 + 1e-9) + 1e-15  # FP64 evaluation near 1
        if t + 1 < T:
            nlo, nhi = r["intervals"][t + 1]
            assert nlo == pytest.approx(1 - E, abs=1e-12) and nhi == pytest.approx(1 + E, abs=1e-12)
