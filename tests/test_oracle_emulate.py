"""Pins of the rounding model of the product chain (oracle/emulate.py), and the
storage-format findings it supports: FP8 (e4m3) stages cannot come first, and
BF16 storage cannot meet rel_F <= 2e-3 at the cost of the FP16 mixed scheme.

CPU only.  The model is Algorithm 2 with explicit roundings of every stored
matrix; the exact reference is oracle.chain_fp64 (equal to F(X) to ~1e-12,
tests/test_oracle_filter.py).
"""
import numpy as np
import pytest

import oracle
from oracle import emulate as em
from paper_2507_09165_gb300 import synth

torch = pytest.importorskip("torch")

COEFS, SCALES = oracle.schedules.schedule("half")
T = len(COEFS)


# ---------------------------------------------------------------------------
# The storage roundings, against an independent implementation (torch's casts)
# and against values written out by hand.
# ---------------------------------------------------------------------------


def test_bf16_rounding_matches_torch():
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.standard_normal(20000) * 10.0 ** rng.integers(-6, 6, 20000),
                        [0.0, -0.0, 1.0, -1.0, 3.0e38]])
    x32 = x.astype(np.float32)
    ref = torch.from_numpy(x32).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(em.round_bf16(x32.astype(np.float64)), ref)
    # ties to even: 1 + 2^-8 lies halfway between 1 and 1 + 2^-7 -> 1;
    # 1 + 3 * 2^-8 halfway between 1 + 2^-7 and 1 + 2^-6 -> 1 + 2^-6
    assert em.round_bf16(np.array([1.0 + 2.0 ** -8]))[0] == 1.0
    assert em.round_bf16(np.array([1.0 + 3 * 2.0 ** -8]))[0] == 1.0 + 2.0 ** -6


def test_f16_rounding_matches_torch():
    rng = np.random.default_rng(1)
    x = (rng.standard_normal(20000) * 10.0 ** rng.integers(-8, 4, 20000)).astype(np.float32)
    ref = torch.from_numpy(x).to(torch.float16).to(torch.float64).numpy()
    assert np.array_equal(em.round_f16(x.astype(np.float64)), ref)
    assert em.round_f16(np.array([1.0 + 2.0 ** -11]))[0] == 1.0  # tie to even
    assert em.round_f16(np.array([2.0 ** -24]))[0] == 2.0 ** -24  # smallest subnormal


def test_e4m3_rounding():
    # OCP E4M3: 1 + k/8 in [1, 2); subnormals k * 2^-9; max 448, saturating here
    vals = {1.0: 1.0, 1.0625: 1.0, 1.1875: 1.25, 0.3: 0.3125, 2.0 ** -9: 2.0 ** -9,
            3 * 2.0 ** -10: 2.0 ** -8, 448.0: 448.0, 1000.0: 448.0, -1.3: -1.25, 0.0: 0.0}
    for x, r in vals.items():
        assert em.round_e4m3(np.array([x]))[0] == r, x
    rng = np.random.default_rng(2)
    x = (rng.uniform(-440.0, 440.0, 20000) * 10.0 ** rng.integers(-3, 1, 20000)).astype(np.float32)
    if hasattr(torch, "float8_e4m3fn"):
        ref = torch.from_numpy(x).to(torch.float8_e4m3fn).to(torch.float64).numpy()
        assert np.array_equal(em.round_e4m3(x.astype(np.float64)), ref)


def test_pair_storage_is_the_rounded_remainder():
    rng = np.random.default_rng(3)
    v = rng.standard_normal(1000)
    s = em.store(v, "f16x2")
    hi, lo = s.parts
    assert np.array_equal(hi, em.round_f16(v))
    assert np.array_equal(lo, em.round_f16(em.round_f32(v) - hi))
    # about 22 significant bits while the lo part is a normal FP16 number
    # (|lo| >= 2^-14, so |v| above about 2^-2)
    big = np.abs(v) >= 0.25
    assert np.max(np.abs(s.value() - em.round_f32(v))[big] / np.abs(v[big])) < 2.0 ** -20


def test_unrounded_plan_is_the_exact_chain():
    X = synth.gaussian_symmetric(64, 5).astype(np.float64)
    lt = oracle.lanczos_bound(X)["lam_tilde"]
    ref, XT = oracle.chain_fp64(X, lt, COEFS, SCALES)
    out, XT2, ok = em.chain_rounded(X, lt, COEFS, SCALES, em.Plan.uniform(T, "f64"))
    assert ok
    # the model rounds only the two FP32 quantities the GPU writes in FP32 (the
    # accumulators and the output): FP32 level of agreement
    assert oracle.rel_err(out, ref) < 1e-6
    assert oracle.rel_err(XT2, XT) < 1e-5


def test_product_counts():
    assert em.Plan.uniform(T, "f16").products() == 22
    assert em.Plan.uniform(T, "bf16x2").products() == 66
    # the FP16 mixed scheme of the library: P pairs in stages 1-4, Y pairs in stages 2-3
    y = ["f16", "f16x2", "f16x2"] + ["f16"] * 4
    p = ["f16x2"] * 4 + ["f16"] * 3
    assert em.Plan(T, "f16", y, p, ["f16"] * T).products() == 30
    assert em.named_plan("mixed").y == y and em.named_plan("mixed").p == p
    # the earlier scheme with Y pairs in stage 1 too
    assert em.Plan(T, "f16", ["f16x2"] * 3 + ["f16"] * 4, p, ["f16"] * T).products() == 32


# ---------------------------------------------------------------------------
# Storage findings (rounding model on five spectrum families).
# ---------------------------------------------------------------------------


def _families(n):
    out = {"gaussian": synth.gaussian_symmetric(n, 11), "wigner": synth.wigner(n, 12)}
    for i, k in enumerate(("uniform", "clustered", "powerlaw")):
        out[k] = synth.spectral_matrix(k, n, 13 + 2 * i)[0]
    cases = {}
    for k, X in out.items():
        X = X.astype(np.float64)
        lt = oracle.lanczos_bound(X)["lam_tilde"]
        cases[k] = (X, lt, oracle.chain_fp64(X, lt, COEFS, SCALES)[0])
    return cases


@pytest.fixture(scope="module")
def fam():
    return _families(192)


def _err(case, plan):
    X, lt, ref = case
    return em.chain_error(X, lt, COEFS, SCALES, plan, ref)


def _fp8_plan(first, last):
    """e4m3 for every matrix of stages first..last (1-based) and for their input
    iterate; FP16 elsewhere (the FP8_LATE precision is first = 6, last = 7)."""
    x0 = "e4m3" if first == 1 else "f16"
    y = ["e4m3" if first <= t + 1 <= last else "f16" for t in range(T)]
    x = ["e4m3" if first <= t + 2 <= last else "f16" for t in range(T)]
    return em.Plan(T, x0, y, list(y), x)


def test_fp8_first_stage_leaves_the_basin(fam):
    # Stage 1 in e4m3 (u = 2^-4): a_1 = 8.29, b_1 = -22.6, c_1 = 15.8 amplify the
    # rounding of X_0 and Y past the composite's basin of about +-1.03, and the
    # iterates diverge on spectra with mass near +-1.
    plan = _fp8_plan(1, 1)
    for k in ("gaussian", "wigner", "uniform"):
        assert _err(fam[k], plan) == float("inf"), k
    # the same e4m3 rounding in the last two stages stays within the FP8 bar
    # (power-law spectra excepted: there ||F(X)||_F can be far below ||X||_2 --
    # when the largest eigenvalues are negative -- and every rounding counts
    # relative to ||X||_2; see the FP16 test below)
    late = _fp8_plan(6, 7)
    for k in ("gaussian", "wigner", "uniform", "clustered"):
        e = _err(fam[k], late)
        assert e <= 5e-2, (k, e)


def test_bf16_storage_misses_2e3_below_the_mixed_cost(fam):
    plain = em.Plan.uniform(T, "bf16")
    for k, case in fam.items():
        assert _err(case, plain) > 2e-3, k
    # The plan a greedy search (add the pair that removes most error per tensor
    # product, from plain BF16) holds at 32 products, more than the FP16 mixed
    # scheme's 30: still above 2e-3.
    pairs = {"p0", "p1", "p2", "y0", "y1", "y2", "p3"}
    pl = em.Plan(T, "bf16", ["bf16x2" if "y%d" % t in pairs else "bf16" for t in range(T)],
                 ["bf16x2" if "p%d" % t in pairs else "bf16" for t in range(T)], ["bf16"] * T)
    assert pl.products() == 32
    assert max(_err(c, pl) for c in fam.values()) > 2e-3
    # BF16 pairs for every matrix meet it with a wide margin, at 3x the products
    allp = em.Plan.uniform(T, "bf16x2")
    assert max(_err(c, allp) for c in fam.values()) < 2e-4
    # the FP16 mixed scheme meets the 1e-3 headline bar at 30 products (2e-3 on
    # the power-law spectrum, whose two largest eigenvalues are negative here);
    # its stage-1 Y pair, dropped from the earlier 32-product scheme, costs 2
    # products and buys ~1e-4 on spread spectra, nothing on dominated ones
    mixed = em.named_plan("mixed")
    old = em.Plan(T, "f16", ["f16x2"] * 3 + ["f16"] * 4, mixed.p, ["f16"] * T)
    for k, case in fam.items():
        e = _err(case, mixed)
        assert e < (2e-3 if k == "powerlaw" else 1e-3), k
        assert e < 1.3 * _err(case, old), k


def test_fp16_plain_misses_2e3_on_dominated_spectra(fam):
    # Plain FP16 storage (the paper's half-precision chain) meets 2e-3 on spread
    # spectra but not where a few eigenvalues dominate ||X||_F: the rounding of
    # the iterates, relative to ||X||_2, is large against ||F(X)||_F there.
    plain = em.Plan.uniform(T, "f16")
    for k in ("gaussian", "wigner", "uniform"):
        assert _err(fam[k], plain) < 2e-3, k
    for k in ("clustered", "powerlaw"):
        assert _err(fam[k], plain) > 2e-3, k



def test_fp16_with_early_polynomial_pairs_is_a_partial_remedy(fam):
    # Plain FP16 except P of stages 2 and 3, stored as FP16 pairs (X P then
    # costs two products, Y^2 with a pair output one): 24 tensor products.  It
    # brings the clustered spectrum under 2e-3 and cuts every family's error,
    # but not on this power-law instance, whose largest eigenvalues are
    # negative (||F(X)||_F far below ||X||_2): there the roundings of the
    # iterates themselves count, which only pairs for X_t (mixed-like costs)
    # remove.  Not built as a precision for that reason.
    pp = em.Plan(T, "f16", ["f16"] * T, ["f16", "f16x2", "f16x2", "f16", "f16", "f16", "f16"], ["f16"] * T)
    plain = em.Plan.uniform(T, "f16")
    assert pp.products() == 24
    for k, case in fam.items():
        assert _err(case, pp) < 0.85 * _err(case, plain), k
    for k in ("gaussian", "wigner", "uniform", "clustered"):
        assert _err(fam[k], pp) < 2e-3, k
    assert _err(fam["clustered"], plain) > 2e-3
    assert _err(fam["powerlaw"], pp) > 2e-3
