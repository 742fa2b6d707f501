"""GPU test of psd_norm_bound_noalloc, the norm bound for callers that cannot
allocate device memory (its scratch is a static device array), through the
C ABI.  It runs the same kernels in the same order as the allocating
psd_norm_bound, so its report must be bit-identical to that one, on calls in a
row and across different orders (the shared array keeps the previous call's
contents); a call after the first must leave the device's free memory as it
was; orders beyond its fixed capacity are rejected.

This file is collected last on purpose: it also passes alone in a fresh
process, where its first call performs the per-device set-up.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from paper_2507_09165_gb300 import binding as b  # noqa: E402
from paper_2507_09165_gb300 import synth  # noqa: E402


def bound(fn, X):
    """The raw psd_info_t bytes one call writes (a report filled with 0xFF first,
    so every field the call leaves alone shows up too)."""
    n = X.shape[0]
    Xd = torch.from_numpy(X).cuda()
    info = torch.full((b.INFO_BYTES,), 255, dtype=torch.uint8, device="cuda")
    fn(n, Xd, n, info)
    torch.cuda.synchronize()
    return info.cpu().numpy()


def same(got, ref):
    assert b.info_from_bytes(got)["status"] == 0
    assert np.array_equal(got, ref), (b.info_from_bytes(got), b.info_from_bytes(ref))


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


def test_noalloc_call_leaves_free_memory_unchanged():
    n = 2048
    Xd = torch.from_numpy(synth.wigner(n, 13)).cuda()
    info = torch.zeros(b.INFO_BYTES, dtype=torch.uint8, device="cuda")
    b.psd_norm_bound_noalloc(n, Xd, n, info)  # first call: set-up, kernels loaded
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        b.psd_norm_bound_noalloc(n, Xd, n, info)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)
    assert b.info_from_bytes(info.cpu().numpy())["status"] == 0


def test_noalloc_rejects_orders_beyond_capacity():
    n = 4097
    Xd = torch.zeros((n, n), dtype=torch.float32, device="cuda")
    info = torch.zeros(b.INFO_BYTES, dtype=torch.uint8, device="cuda")
    with pytest.raises(b.PsdError) as e:
        b.psd_norm_bound_noalloc(n, Xd, n, info)
    assert e.value.status == 1  # PSD_ERR_INVALID_ARG, nothing launched
    torch.cuda.synchronize()
    assert not np.any(info.cpu().numpy())
