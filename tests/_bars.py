"""Accuracy bars of the GPU parity tests and the record of their known misses.

rel_F = ||out - F||_F / ||F||_F against the oracle's exact filter output F(X),
what Algorithm 2 computes in exact arithmetic.  Bars: FP16 and BF16 2e-3, FP8
stages 5e-2, FP32 1e-5; the FP16 mixed scheme 1e-3 (the accuracy target of the
n = 10,000 projection).

Where a precision cannot meet its bar on an input, the test records an
expected failure with the measured value instead of a wider bar:
  * BF16 storage: every rounding at unit roundoff 2^-9 adds ~3-4e-4, and the
    chain stores 22 matrices; the rounding model (oracle/emulate.py) puts the
    plain BF16 chain at ~1.3e-2 on spread spectra and ~3e-2 on dominated ones,
    and no BF16 storage plan gets below 2e-3 with fewer than ~56 tensor products
    (tests/test_oracle_emulate.py);
  * plain FP16 storage on spectra where a few eigenvalues dominate ||X||_F
    (clustered around 0 with +-1 anchors, power law): the roundings, relative
    to ||X||_2, are large against ||F(X)||_F.
An expected failure is only taken when the rounding model of the same chain on
the same input (for orders above 1024: on the order-1024 matrix of the same
spectrum family and seed, the model's error does not grow with n) is itself
above the bar, and the measured error must stay within 1.5x the model's, so a
kernel defect cannot hide behind it.
"""
import numpy as np
import pytest

import oracle
from oracle import emulate

TOL_F = {"fp16": 2e-3, "bf16": 2e-3, "fp8_late": 5e-2, "fp32": 1e-5, "mixed": 1e-3}
SCHED = {"fp16": "half", "bf16": "half", "mixed": "half", "fp8_late": "half", "fp32": "single"}
MODEL_MAX_ORDER = 1024


def model_error(prec, X, lam_tilde):
    """rel_F of the rounding model of `prec`'s chain on X (FP64 array) with the
    given norm bound."""
    coefs, scales = oracle.schedules.schedule(SCHED[prec])
    return emulate.chain_error(np.asarray(X, dtype=np.float64), lam_tilde, coefs, scales,
                               emulate.named_plan(prec, len(coefs)))


def _assess(prec, rel_f, what, model_fn):
    """None if rel_f meets the bar; the known-miss message if the miss is
    covered by the rounding model (model_fn() -> the model's error in the same
    metric); a failed assertion otherwise."""
    tol = TOL_F[prec]
    if rel_f <= tol:
        return None
    if prec not in ("fp16", "bf16", "mixed", "fp8_late") or model_fn is None:
        pytest.fail("%s %s: rel_F = %.3e above the %g bar" % (prec, what, rel_f, tol))
    model = model_fn()
    assert model > tol, ("%s %s: rel_F = %.3e above the %g bar, but the rounding model of the chain "
                         "meets it (%.3e)" % (prec, what, rel_f, tol, model))
    assert rel_f <= 1.5 * model, ("%s %s: rel_F = %.3e, more than 1.5x the rounding model's %.3e"
                                  % (prec, what, rel_f, model))
    return "%s: measured rel_F = %.3e, rounding model %.3e" % (what, rel_f, model)


def _model_fn(prec, X, lam_tilde, model_input):
    if model_input is None and X is None:
        return None

    def fn():
        if model_input is not None:
            Xm, lm = model_input()
        else:
            assert X.shape[0] <= MODEL_MAX_ORDER, "give a model_input for orders above %d" % MODEL_MAX_ORDER
            Xm, lm = X, lam_tilde
        return model_error(prec, Xm, lm)
    return fn


def check_rel_f(prec, rel_f, X=None, lam_tilde=None, what="", model_input=None, model_fn=None):
    """Assert rel_f <= TOL_F[prec], or record the known miss (see the module doc).

    X, lam_tilde: the input and the bound the GPU used; model_input: a callable
    returning (X, lam_tilde) of a smaller stand-in for the model when X is
    larger than MODEL_MAX_ORDER; model_fn: a callable returning the model's
    error directly (for another metric).  Call it last in a test (an expected
    failure ends the test)."""
    check_all(prec, [(rel_f, X, lam_tilde, what, model_input, model_fn)])


def check_all(prec, results):
    """check_rel_f over several results (rel_f, X, lam_tilde, what[, model_input[, model_fn]]):
    every result is assessed, then one expected failure lists the known misses."""
    misses = []
    for r in results:
        rel_f, X, lam_tilde, what = r[:4]
        mi = r[4] if len(r) > 4 else None
        fn = r[5] if len(r) > 5 and r[5] is not None else _model_fn(prec, X, lam_tilde, mi)
        m = _assess(prec, rel_f, what, fn)
        if m:
            misses.append(m)
    if misses:
        pytest.xfail("%s misses the %g bar on %d case(s): %s" % (prec, TOL_F[prec], len(misses),
                                                                 "; ".join(misses)))
