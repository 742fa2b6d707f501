"""Parity at the full sizes of the workloads, in the launch configuration
bench.py times (the library's default plans and graphs).

* One matrix of order 10,000 with a known spectrum (Q diag(l) Q^T, Haar Q,
  semicircle l: the laws of the timed Wigner matrix): the oracle's scalar map
  phi gives the exact filter output F and Pi at any entry, F_ij = sum_k Q_ik
  phi(l_k) Q_jk, so the GPU output is compared with them on sampled entries.
* The headline metric itself, rel err of the mixed path against the FP32 path,
  on the Wigner and the low-rank-plus-noise inputs of order 10,000, with the
  properties that hold at any size (exact symmetry, status, the report).
* The 512-block batch: sampled blocks against the oracle, every block's
  properties.
* The request server at order 8000: a served result is bit-identical to the
  direct call.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from paper_2507_09165_gb300 import binding as b  # noqa: E402
from paper_2507_09165_gb300 import synth  # noqa: E402

DEV = torch.device("cuda")
N = 10000
from _bars import SCHED, TOL_F, check_all  # noqa: E402
GB = 1 << 30


def project(Xd, prec):
    n = Xd.shape[0]
    out = torch.empty_like(Xd)
    info = torch.zeros(b.INFO_BYTES, dtype=torch.uint8, device=DEV)
    b.psd_project_ex(n, Xd, n, out, n, prec, info)
    torch.cuda.synchronize()
    return out, b.info_from_bytes(info.cpu().numpy())


def sampled_pairs(n, count, seed):
    rng = np.random.default_rng(seed)
    i = rng.integers(0, n, size=count)
    j = rng.integers(0, n, size=count)
    d = rng.integers(0, n, size=count // 8)  # diagonal entries too
    return np.concatenate([i, d]), np.concatenate([j, d])


def spectral_entries(Q, values, I, J, chunk=512):
    """(Q diag(values) Q^T)_{I_s, J_s} in FP64, one sample at a time in chunks."""
    out = np.empty(len(I))
    for s in range(0, len(I), chunk):
        qi = Q[I[s:s + chunk]]
        qj = Q[J[s:s + chunk]]
        out[s:s + chunk] = np.einsum("sk,k,sk->s", qi, values, qj)
    return out


@pytest.fixture(scope="module")
def known_spectrum():
    X32, Q, lam = synth.spectral_matrix("semicircle", N, 20)
    return X32, Q, lam


@pytest.mark.parametrize("prec", ["mixed", "fp16", "fp32"])
def test_n10000_known_spectrum_sampled_entries(known_spectrum, prec):
    X32, Q, lam = known_spectrum
    Xd = torch.from_numpy(X32).to(DEV)
    out, info = project(Xd, prec)
    assert info["status"] == 0
    lt = info["lambda_bound"]
    top = float(np.max(np.abs(lam)))
    assert top * (1 - 1e-6) <= lt <= 1.01 * top  # Theorem 2, and a tight bound
    I, J = sampled_pairs(N, 4096, 5)
    got = out.cpu().numpy()[I, J].astype(np.float64)
    del out, Xd
    coefs, scales = oracle.schedules.schedule(SCHED[prec])
    F = spectral_entries(Q, oracle.phi(lam, lt, coefs, scales), I, J)
    P = spectral_entries(Q, np.maximum(lam, 0.0), I, J)
    rel_f = np.linalg.norm(got - F) / np.linalg.norm(F)
    rel_p = np.linalg.norm(got - P) / np.linalg.norm(P)
    assert rel_f <= TOL_F[prec], rel_f
    if prec == "mixed":
        assert rel_p <= 1e-3, rel_p  # the headline accuracy against the true projection
    # the report's residual <out, X - out> / ||X||^2 against the exact filter output's
    phi = oracle.phi(lam, lt, coefs, scales)
    c_f = float(np.sum(phi * (lam - phi)) / np.sum(lam * lam))
    assert abs(info["compl_resid"] - c_f) <= 5 * TOL_F[prec], (info["compl_resid"], c_f)


@pytest.mark.parametrize("kind", ["wigner", "lowrank"])
def test_n10000_mixed_against_the_fp32_path(kind):
    X = synth.wigner(N, 2) if kind == "wigner" else synth.lowrank_plus_noise(N, 3)
    Xd = torch.from_numpy(X).to(DEV)
    o_mix, i_mix = project(Xd, "mixed")
    o_32, i_32 = project(Xd, "fp32")
    assert i_mix["status"] == 0 and i_32["status"] == 0
    assert i_mix["lambda_bound"] == i_32["lambda_bound"]  # the same norm bound
    assert torch.equal(o_mix, o_mix.T) and torch.equal(o_32, o_32.T)
    rel = float(torch.linalg.norm((o_mix - o_32).double()) / torch.linalg.norm(o_32.double()))
    assert rel <= 1e-3, rel
    # the lower bound ||X v|| / ||v|| of ||X||_2 from a few power steps never exceeds lam~
    v = torch.randn(N, 1, device=DEV, dtype=torch.float64, generator=torch.Generator(DEV).manual_seed(1))
    X64 = Xd.double()
    for _ in range(30):
        v = X64 @ v
        v /= torch.linalg.norm(v)
    est = float(torch.linalg.norm(X64 @ v))
    assert est <= i_mix["lambda_bound"] * (1 + 1e-9)
    assert abs(i_mix["compl_resid"]) < 1e-2 and abs(i_32["compl_resid"]) < 1e-3


def test_512_block_batch_sampled_blocks_and_all_properties():
    sizes = synth.block_sizes(512, 7)
    mats = [synth.wigner(n, 7000 + i) for i, n in enumerate(sizes)]
    X = [torch.from_numpy(m).to(DEV) for m in mats]
    O = [torch.full_like(x, float("nan")) for x in X]
    infos = [torch.zeros(b.INFO_BYTES, dtype=torch.uint8, device=DEV) for _ in sizes]
    d = b.block_descs([(n, x, n, o, n, i) for n, x, o, i in zip(sizes, X, O, infos)])
    # the block-diagonal workload runs in FP16, which meets the 2e-3 bar on it
    b.psd_project_batched(len(sizes), d, "fp16")
    torch.cuda.synchronize()
    reps = [b.info_from_bytes(i.cpu().numpy()) for i in infos]
    for n, o, r in zip(sizes, O, reps):
        assert r["status"] == 0, (n, r)
        assert torch.equal(o, o.T)
        assert np.isfinite(r["compl_resid"]) and abs(r["compl_resid"]) < 0.01
    order = np.argsort(sizes)
    picks = sorted({int(order[0]), int(order[len(order) // 4]), int(order[len(order) // 2]),
                    int(order[3 * len(order) // 4]), int(order[-1])})
    results = []
    for k in picks:
        X64 = mats[k].astype(np.float64)
        ref = oracle.oracle_project(X64, "half")
        assert reps[k]["lambda_bound"] == pytest.approx(ref["lam_tilde"], rel=1e-6)
        rel = oracle.rel_err(O[k].cpu().numpy().astype(np.float64), ref["F"])
        results.append((rel, X64, reps[k]["lambda_bound"], "block %d, n = %d" % (k, sizes[k])))
    check_all("fp16", results)


def test_server_order_8000_served_equals_direct():
    n = 8000
    L = synth.er_laplacian(n, 8)
    V = torch.from_numpy((L - np.eye(n)).astype(np.float32)).to(DEV)  # an ADMM projection input
    ref, r_info = project(V, "fp16")
    h = b.psd_server_create(4 * GB, 0, n, 4)
    try:
        out = torch.full_like(V, float("nan"))
        info, lat = b.psd_server_wait(h, b.psd_server_submit(h, n, V, n, out, n, "fp16"))
        assert info["status"] == 0 and lat > 0
        assert torch.equal(out, ref)
        for k in ("lambda_bound", "lanczos_sigma", "lanczos_resid", "fro_X", "overshoot_max", "compl_resid"):
            assert info[k] == r_info[k], k
    finally:
        b.psd_server_destroy(h)
