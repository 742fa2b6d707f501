"""Failure detection, driven from the host (psd_debug_set), on the GPU.

Nothing here faults, traps or hangs the GPU: the injected conditions are a
norm bound scaled below ||X||_2 (the filter then sees a spectrum beyond its
basin, which the overshoot report must catch) and a zero wait limit for the
persistent norm bound's grid barriers (every barrier that is not already
complete gives up at once; the CTAs leave at their next barrier and the status
word carries PSD_ERR_TIMEOUT; the batched bound's dependency waits give up the
same way and every block of the batch reports it).  After each, the defaults
are restored and a normal call on the same context must give the usual
result, bit for bit.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from paper_2507_09165_gb300 import binding as b  # noqa: E402
from paper_2507_09165_gb300 import synth  # noqa: E402

DEV = torch.device("cuda")
PSD_ERR_NONFINITE, PSD_ERR_BOUND, PSD_ERR_TIMEOUT = 4, 5, 6


def _project(X, n, prec="fp16"):
    out = torch.full_like(X, float("nan"))
    info = torch.zeros(b.INFO_BYTES, dtype=torch.uint8, device=DEV)
    b.psd_project_ex(n, X, n, out, n, prec, info)
    torch.cuda.synchronize()
    return out.cpu(), b.info_from_bytes(info.cpu().numpy())


@pytest.fixture(scope="module")
def wigner():
    n = 1500
    return n, torch.from_numpy(synth.wigner(n, 31)).to(DEV)


def test_debug_knobs_reject_bad_values():
    for knob, value in ((0, 1.0), (3, 1.0), (b.DEBUG_BOUND_SCALE, 0.0), (b.DEBUG_BOUND_SCALE, -1.0),
                        (b.DEBUG_BOUND_SCALE, float("nan")), (b.DEBUG_BARRIER_LIMIT_NS, -1.0),
                        (b.DEBUG_BARRIER_LIMIT_NS, 1e12)):
        with pytest.raises(b.PsdError):
            b.psd_debug_set(knob, value)


def test_bound_below_the_norm_is_reported_as_overshoot(wigner):
    n, X = wigner
    ref, info0 = _project(X, n)
    assert info0["status"] == 0
    try:
        b.psd_debug_set(b.DEBUG_BOUND_SCALE, 0.5)
        _, info = _project(X, n)
    finally:
        b.psd_debug_set(b.DEBUG_BOUND_SCALE, 1.0)
    # lam~ halved: the top of the spectrum lies at 2 on the filter's scale, far
    # outside the composite's basin (about +-1.03)
    assert info["lambda_bound"] == pytest.approx(0.5 * info0["lambda_bound"], rel=1e-12)
    assert info["status"] in (PSD_ERR_BOUND, PSD_ERR_NONFINITE), info
    assert not (info["overshoot_max"] <= 1.01)  # above the limit, or NaN
    again, info1 = _project(X, n)
    assert info1["status"] == 0
    assert info1["lambda_bound"] == info0["lambda_bound"]
    assert torch.equal(again.view(torch.int32), ref.view(torch.int32))


def test_barrier_timeout_is_reported_and_the_context_stays_usable(wigner):
    n, X = wigner
    ref, info0 = _project(X, n, "mixed")
    assert info0["status"] == 0
    try:
        b.psd_debug_set(b.DEBUG_BARRIER_LIMIT_NS, 0)
        _, info = _project(X, n, "mixed")
        nb_info = torch.zeros(b.INFO_BYTES, dtype=torch.uint8, device=DEV)
        b.psd_norm_bound(n, X, n, nb_info)
        torch.cuda.synchronize()
    finally:
        b.psd_debug_set(b.DEBUG_BARRIER_LIMIT_NS, 4e9)
    assert info["status"] == PSD_ERR_TIMEOUT, info
    again, info1 = _project(X, n, "mixed")
    assert info1["status"] == 0
    assert info1["lambda_bound"] == info0["lambda_bound"]
    assert torch.equal(again.view(torch.int32), ref.view(torch.int32))


def test_batched_wait_timeout_is_reported_for_every_block():
    # the batched bound's one-launch form waits on per-block counters
    sizes = [700, 33, 256, 5, 1024, 129]
    mats = [torch.from_numpy(synth.wigner(n, 3100 + i)).to(DEV) for i, n in enumerate(sizes)]
    outs = [torch.full_like(M, float("nan")) for M in mats]
    infos = [torch.zeros(b.INFO_BYTES, dtype=torch.uint8, device=DEV) for _ in mats]
    descs = b.block_descs([(n, M, n, o, n, i) for n, M, o, i in zip(sizes, mats, outs, infos)])

    def run():
        for i in infos:
            i.zero_()
        b.psd_project_batched(len(sizes), descs, "fp16")
        torch.cuda.synchronize()
        return [o.cpu().clone() for o in outs], [b.info_from_bytes(i.cpu().numpy()) for i in infos]

    prev = b.psd_batched_force_bound(1)
    try:
        ref, info0 = run()
        assert all(i["status"] == 0 for i in info0)
        try:
            b.psd_debug_set(b.DEBUG_BARRIER_LIMIT_NS, 0)
            _, info = run()
        finally:
            b.psd_debug_set(b.DEBUG_BARRIER_LIMIT_NS, 4e9)
        again, info1 = run()
    finally:
        b.psd_batched_force_bound(prev)
    assert all(i["status"] == PSD_ERR_TIMEOUT for i in info), [i["status"] for i in info]
    assert all(i["status"] == 0 for i in info1)
    for r, a, i0, i1 in zip(ref, again, info0, info1):
        assert torch.equal(a.view(torch.int32), r.view(torch.int32))
        assert i1 == i0
