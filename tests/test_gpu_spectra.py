"""GPU parity on spectrum-controlled inputs of order 4096, every precision.

X = Q diag(l) Q^T with Haar Q and three spectra: uniform on [-1, 1]; clustered
(n - 2 eigenvalues in +-1e-3 around 0, anchors +-1); power law |l_i| = i^-1.5
with random signs.  The oracle's filter output is known from the spectrum:
F = Q diag(phi(l)) Q^T with phi(l) = l (1 + g(l / lam~)) / 2, lam~ the GPU's
bound (checked against max |l| first), so the whole output is compared with it
(the Sec. 4.1 relative Frobenius error), and the error per band of |l| / ||X||_2
is printed against F and against Pi(X) = Q diag(max(l, 0)) Q^T.

These are the spectra on which the composite filter is weakest (Sec. 6:
eigenvalues crowded into the band around 0, or a few dominating the rest), and
where the plain FP16 and BF16 chains miss their bar (recorded as expected
failures with the measured value, tests/_bars.py).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from paper_2507_09165_gb300 import binding as b  # noqa: E402
from paper_2507_09165_gb300 import synth  # noqa: E402

from _bars import SCHED, check_rel_f  # noqa: E402

DEV = torch.device("cuda")
N = 4096
KINDS = {"uniform": 4, "clustered": 5, "powerlaw": 6}
PRECS = ["fp16", "bf16", "mixed", "fp8_late", "fp32"]


@pytest.fixture(scope="module")
def spectra():
    out = {}
    for kind, seed in KINDS.items():
        X32, Q, lam = synth.spectral_matrix(kind, N, seed)
        out[kind] = (X32, Q, lam, seed)
    return out


def _model_input(kind, seed):
    # the rounding model on the order-1024 matrix of the same family and seed
    def fn():
        Xm = synth.spectral_matrix(kind, 1024, seed)[0].astype(np.float64)
        return Xm, oracle.lanczos_bound(Xm)["lam_tilde"]
    return fn


def _bands(E, lam, vals, top):
    """||D Q_B||_F / ||X Q_B||_F per band of |l| / top, split by sign, given
    E = D Q (D = output - reference)."""
    rel = np.abs(lam) / top
    res = {}
    for sign in (1, -1):
        for lo, hi in oracle.BANDS:
            sel = (rel >= lo) & (rel < hi) & ((lam > 0) if sign > 0 else (lam <= 0))
            if not np.any(sel):
                continue
            den = np.linalg.norm(lam[sel])
            res["%s[%g,%g)" % ("+" if sign > 0 else "-", lo, min(hi, 1.0))] = np.linalg.norm(E[:, sel]) / den
    return res


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("kind", list(KINDS))
def test_spectrum_controlled_order_4096(spectra, kind, prec):
    X32, Q, lam, seed = spectra[kind]
    Xd = torch.from_numpy(X32).to(DEV)
    out = torch.full_like(Xd, float("nan"))
    info = torch.zeros(b.INFO_BYTES, dtype=torch.uint8, device=DEV)
    b.psd_project_ex(N, Xd, N, out, N, prec, info)
    torch.cuda.synchronize()
    info = b.info_from_bytes(info.cpu().numpy())
    assert info["status"] == 0, info
    assert torch.equal(out, out.T)
    o = out.cpu().numpy().astype(np.float64)
    del out, Xd
    lt = info["lambda_bound"]
    top = float(np.max(np.abs(lam)))
    assert top * (1 - 1e-6) <= lt <= 1.01 * top  # Theorem 2, and a tight bound
    coefs, scales = oracle.schedules.schedule(SCHED[prec])
    phi = oracle.phi(lam, lt, coefs, scales)
    F = oracle.spectral(lam, Q, phi)
    D = o - F
    rel_f = float(np.linalg.norm(D) / np.linalg.norm(F))
    relu = np.maximum(lam, 0.0)
    rel_pi = float(np.linalg.norm(o - oracle.spectral(lam, Q, relu)) / np.linalg.norm(relu))
    E = D @ Q
    bf = _bands(E, lam, phi, top)
    bp = _bands(E + Q * (phi - relu)[None, :], lam, relu, top)  # (out - Pi) Q = D Q + Q diag(phi - relu)
    print("\n%s %s n=%d rel_F=%.3e rel_Pi=%.3e lam~=%.6g" % (kind, prec, N, rel_f, rel_pi, lt))
    print("  bands vs F : " + " ".join("%s %.2e" % kv for kv in bf.items()))
    print("  bands vs Pi: " + " ".join("%s %.2e" % kv for kv in bp.items()))
    check_rel_f(prec, rel_f, what="%s n = %d" % (kind, N), model_input=_model_input(kind, seed))
