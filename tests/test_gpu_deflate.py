"""GPU parity of the deflated projection (psd_project_deflate) with the oracle's
deflate_project, through the C ABI.

Both sides run the same steps (norm bound with its Lanczos basis, Rayleigh-Ritz
with X, residual test, deflation, filter of the deflated matrix with its own
norm bound, add-back); the number of deflated pairs is an integer decision and
must agree exactly, so the inputs are checked to keep every residual of the
candidate pairs at least 1.5x away from the threshold.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from oracle import emulate  # noqa: E402
from paper_2507_09165_gb300 import binding as b  # noqa: E402
from paper_2507_09165_gb300 import synth  # noqa: E402

DEV = torch.device("cuda")
from _bars import SCHED, TOL_F, check_rel_f  # noqa: E402
KMAX = 16


def to_dev(X, ld=None):
    n = X.shape[0]
    ld = ld or n
    Xt = torch.zeros((n, ld), dtype=torch.float32)
    Xt[:, :n] = torch.from_numpy(np.asarray(X, dtype=np.float32))
    return Xt.to(DEV)


def run_deflate(X, prec, kmax=KMAX, ld=None, ld_out=None, inplace=False):
    n = X.shape[0]
    ld = ld or n
    Xd = to_dev(X, ld)
    info = torch.zeros(b.INFO_BYTES, dtype=torch.uint8, device=DEV)
    kused = torch.full((1,), -1, dtype=torch.int32, device=DEV)
    if inplace:
        out, ld_out = Xd, ld
    else:
        ld_out = ld_out or n
        out = torch.full((n, ld_out), float("nan"), dtype=torch.float32, device=DEV)
    b.psd_project_deflate(n, Xd, ld, out, ld_out, prec, kmax, info, kused)
    torch.cuda.synchronize()
    return out.cpu().numpy()[:, :n].astype(np.float64), int(kused.item()), b.info_from_bytes(info.cpu().numpy())


def run_plain(X, prec):
    n = X.shape[0]
    Xd = to_dev(X)
    out = torch.full_like(Xd, float("nan"))
    b.psd_project_ex(n, Xd, n, out, n, prec)
    torch.cuda.synchronize()
    return out.cpu().numpy().astype(np.float64)


def oracle_deflate(X, prec, kmax=KMAX):
    coefs, scales = oracle.schedules.schedule(SCHED[prec])
    r = oracle.deflate_project(np.asarray(X, dtype=np.float64), kmax, coefs, scales)
    rel = r["resid"][:kmax] / r["lam_tilde"] / oracle.DEFLATE_TOL
    near = [j for j in range(len(rel)) if 1 / 1.5 < rel[j] < 1.5]
    assert not near, "residuals too close to the deflation threshold: %s" % rel[near]
    return r


def _model_deflated(prec, ref):
    coefs, scales = oracle.schedules.schedule(SCHED[prec])
    Xd = ref["X_defl"].astype(np.float32).astype(np.float64)
    lt = ref["lam_tilde_defl"]
    out_m, _, _ = emulate.chain_rounded(Xd, lt, coefs, scales, emulate.named_plan(prec))
    return np.linalg.norm(out_m - oracle.chain_fp64(Xd, lt, coefs, scales)[0]) / np.linalg.norm(ref["out"])


def rel(A, B):
    return np.linalg.norm(A - B) / np.linalg.norm(B)


@pytest.fixture(scope="module")
def spectra():
    out = {}
    for kind, n, seed in (("powerlaw", 700, 11), ("clustered", 300, 11), ("powerlaw", 257, 9)):
        X, Q, lam = synth.spectral_matrix(kind, n, seed)
        out[(kind, n)] = (X, oracle.project_from_eig(lam, Q))
    return out


@pytest.mark.parametrize("prec", ["fp16", "bf16", "mixed", "fp32"])
@pytest.mark.parametrize("case", [("powerlaw", 700), ("clustered", 300), ("powerlaw", 257)])
def test_deflate_parity(spectra, case, prec):
    X, _ = spectra[case]
    ref = oracle_deflate(X, prec)
    out, k, info = run_deflate(X, prec)
    assert info["status"] == 0
    assert k == ref["k"], (k, ref["k"])
    assert abs(info["lambda_bound"] - ref["lam_tilde_defl"]) <= 1e-6 * ref["lam_tilde_defl"]
    assert np.array_equal(out, out.T)
    e = rel(out, ref["out"])

    # the rounding model of the filter of the deflated matrix, in the same metric
    check_rel_f(prec, e, what="deflated %s n = %d" % case,
                model_fn=(lambda: _model_deflated(prec, ref)) if prec != "fp32" else None)


@pytest.mark.parametrize("prec", ["fp16", "mixed", "fp32"])
def test_deflation_cuts_the_powerlaw_error(spectra, prec):
    X, P = spectra[("powerlaw", 700)]
    out, k, _ = run_deflate(X, prec)
    e1 = rel(out, P)
    e0 = rel(run_plain(X, prec), P)
    assert k >= 8
    assert e1 < e0 / 5, (e0, e1)


def test_low_rank_plus_rounding():
    # rank 6 in FP32: the deflated matrix is the FP32 rounding noise, so the
    # result is Pi(X) up to that noise, far below the plain filter's error
    n, r = 300, 6
    rng = np.random.default_rng(21)
    U, _ = np.linalg.qr(rng.standard_normal((n, r)))
    lam = np.array([3.0, -2.5, 1.7, -1.1, 0.6, 0.25])
    X = ((U * lam[None, :]) @ U.T).astype(np.float32)
    P = (U * np.maximum(lam, 0)[None, :]) @ U.T
    out, k, info = run_deflate(X, "fp16")
    assert info["status"] == 0 and k >= r
    assert rel(out, P) < 1e-5
    assert rel(run_plain(X, "fp16"), P) > 10 * rel(out, P)


@pytest.mark.parametrize("prec", ["fp16", "fp32"])
def test_nothing_deflated_is_the_plain_projection(prec):
    # kmax = 0, and a uniform spectrum (no converged dominant pair): the
    # result is bit-identical to psd_project_ex
    X, _, _ = synth.spectral_matrix("uniform", 300, 11)
    plain = run_plain(X, prec)
    for kmax in (0, KMAX):
        out, k, info = run_deflate(X, prec, kmax=kmax)
        assert k == 0 and info["status"] == 0
        assert np.array_equal(out, plain), kmax


def test_leading_dims_and_inplace(spectra):
    X, _ = spectra[("powerlaw", 257)]
    ref, k, _ = run_deflate(X, "fp16")
    o2, k2, _ = run_deflate(X, "fp16", ld=263, ld_out=260)
    o3, k3, _ = run_deflate(X, "fp16", ld=261, inplace=True)
    assert k == k2 == k3 > 0
    assert np.array_equal(ref, o2) and np.array_equal(ref, o3)


@pytest.mark.parametrize("n", [1, 2, 17, 65, 129])
def test_small_orders(n):
    X = synth.gaussian_symmetric(n, 700 + n)
    ref = oracle_deflate(X, "fp16")
    out, k, info = run_deflate(X, "fp16")
    assert info["status"] == 0
    assert k == ref["k"]
    nx = np.linalg.norm(X.astype(np.float64))
    if np.linalg.norm(ref["out"]) < 1e-6 * nx:  # X negative semidefinite: Pi(X) = 0
        # every pair deflated, X' is the FP32 rounding of X - V M V^T (~1e-7 ||X||)
        assert np.linalg.norm(out - ref["out"]) <= 1e-6 * nx
    else:
        check_rel_f("fp16", rel(out, ref["out"]), what="deflated Gaussian n = %d" % n,
                    model_fn=lambda: _model_deflated("fp16", ref))


def test_nonfinite_and_bad_arguments():
    n = 100
    X = synth.gaussian_symmetric(n, 3)
    X[7, 5] = np.nan  # row 7, column 5 of the row-major copy: the upper triangle column-major
    out, k, info = run_deflate(X, "fp16")
    assert k == 0 and info["status"] == 4
    Xd = to_dev(synth.gaussian_symmetric(n, 4))
    o = torch.empty_like(Xd)
    with pytest.raises(b.PsdError) as e:
        b.psd_project_deflate(n, Xd, n, o, n, "fp16", 17)
    assert e.value.status == 1
    with pytest.raises(b.PsdError) as e:  # partial overlap of X and out
        b.psd_project_deflate(n - 1, Xd, n, Xd[1:], n, "fp16", 4)
    assert e.value.status == 1
    b.psd_project_deflate(0, None, 0, None, 0, "fp16", 4)
