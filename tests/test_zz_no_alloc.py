"""GPU test of psd_norm_bound_noalloc, the norm bound for callers that cannot
allocate device memory (its scratch is a static device array), through the
C ABI.  It must report what the allocating psd_norm_bound reports, on calls in
a row and across different orders (the shared array keeps the previous call's
contents), and reject orders beyond its fixed capacity.

This file is collected last on purpose: it also passes alone in a fresh
process, where its first call performs the per-device set-up.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from paper_2507_09165_gb300 import binding as b  # noqa: E402
from paper_2507_09165_gb300 import synth  # noqa: E402

FIELDS = ("lambda_bound", "lanczos_sigma", "lanczos_resid", "fro_X", "max_diag")


def bound(fn, X):
    n = X.shape[0]
    Xd = torch.from_numpy(X).cuda()
    info = torch.zeros(b.INFO_BYTES, dtype=torch.uint8, device="cuda")
    fn(n, Xd, n, info)
    torch.cuda.synchronize()
    return b.info_from_bytes(info.cpu().numpy())


def same(got, ref):
    assert got["status"] == 0
    assert got["lanczos_steps"] == ref["lanczos_steps"]
    for k in FIELDS:
        assert got[k] == pytest.approx(ref[k], rel=1e-6, abs=1e-300), k


@pytest.mark.parametrize("n", [1, 300, 4096])
def test_noalloc_matches_allocating_entry_point_twice(n):
    X = synth.gaussian_symmetric(n, 500 + n)
    ref = bound(b.psd_norm_bound, X)
    same(bound(b.psd_norm_bound_noalloc, X), ref)
    same(bound(b.psd_norm_bound_noalloc, X), ref)


def test_noalloc_different_orders_in_a_row():
    X1 = synth.wigner(4096, 11)
    X2 = synth.lowrank_plus_noise(777, 12, rank=10)
    r1, r2 = bound(b.psd_norm_bound, X1), bound(b.psd_norm_bound, X2)
    same(bound(b.psd_norm_bound_noalloc, X1), r1)
    same(bound(b.psd_norm_bound_noalloc, X2), r2)
    same(bound(b.psd_norm_bound_noalloc, X1), r1)


def test_noalloc_rejects_orders_beyond_capacity():
    n = 4097
    Xd = torch.zeros((n, n), dtype=torch.float32, device="cuda")
    info = torch.zeros(b.INFO_BYTES, dtype=torch.uint8, device="cuda")
    with pytest.raises(b.PsdError) as e:
        b.psd_norm_bound_noalloc(n, Xd, n, info)
    assert e.value.status == 1  # PSD_ERR_INVALID_ARG, nothing launched
    torch.cuda.synchronize()
    assert not np.any(info.cpu().numpy())
