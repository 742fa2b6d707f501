"""GPU tests of the request server (continuous batching of projections).

The server's promise: a request's output and report are bit-identical to a
psd_project call with the same precision on the same input, whether it runs
alone or shares every launch with other requests at other stages.  Parity of
psd_project itself with the oracle is covered in test_gpu_project.py; one
oracle check here ties the served result to the oracle directly.
"""
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from paper_2507_09165_gb300 import binding as b, synth  # noqa: E402

GB = 1 << 30
INFO_KEYS = ("status", "lanczos_steps", "lambda_bound", "lanczos_sigma", "lanczos_resid", "fro_X", "max_diag",
             "overshoot_max", "compl_resid")


def make(n, seed, ld=None):
    ld = ld or n
    X = torch.zeros((n, ld), dtype=torch.float32)
    X[:, :n] = torch.from_numpy(synth.wigner(n, seed))
    return X.cuda()


def single(n, X, ld, prec):
    out = torch.full_like(X, float("nan"))
    info = torch.zeros(b.INFO_BYTES, dtype=torch.uint8, device="cuda")
    b.psd_project_ex(n, X, ld, out, ld, prec, info)
    torch.cuda.synchronize()
    return out, b.info_from_bytes(info.cpu().numpy().tobytes())


def same_info(a, c):
    # compl_resid: the final product's per-tile shares, summed in the same order
    return all(a[k] == c[k] for k in INFO_KEYS) and np.isfinite(a["compl_resid"])


@pytest.fixture
def server():
    h = b.psd_server_create(2 * GB, 0, 2048, 32)
    yield h
    b.psd_server_destroy(h)


@pytest.mark.parametrize("prec", ["bf16", "fp16"])
def test_served_equals_single_alone_and_in_mix(server, prec):
    sizes = [1, 17, 100, 255, 256, 300, 513, 1000, 2048, 64, 777]
    Xs = [make(n, 9100 + i) for i, n in enumerate(sizes)]
    ref = [single(n, X, n, prec) for n, X in zip(sizes, Xs)]
    # alone: one request at a time
    for n, X, (r_out, r_info) in zip(sizes, Xs, ref):
        out = torch.full_like(X, float("nan"))
        t = b.psd_server_submit(server, n, X, n, out, n, prec)
        info, lat = b.psd_server_wait(server, t)
        assert lat > 0
        assert torch.equal(out, r_out), n
        assert same_info(info, r_info), (n, info, r_info)
    # in the mix: all at once, then again with staggered arrivals so that
    # requests join while others are at different stages
    for stagger in (0.0, 0.0007):
        outs = [torch.full_like(X, float("nan")) for X in Xs]
        tickets = []
        for n, X, o in zip(sizes, Xs, outs):
            tickets.append(b.psd_server_submit(server, n, X, n, o, n, prec))
            if stagger:
                time.sleep(stagger)
        for n, t, o, (r_out, r_info) in zip(sizes, tickets, outs, ref):
            info, _ = b.psd_server_wait(server, t)
            assert torch.equal(o, r_out), (n, stagger)
            assert same_info(info, r_info), n
    st = b.psd_server_stats(server)
    assert st["completed"] == 3 * len(sizes)
    assert st["max_running"] > 1  # the mix did share launches
    assert 0 < st["p50_ms"] <= st["p99_ms"] <= st["max_ms"]


def test_served_matches_oracle(server):
    oracle = pytest.importorskip("oracle")
    n = 300
    Xh, Q, lam = synth.spectral_matrix("semicircle", n, 31)
    X = torch.from_numpy(Xh).cuda()
    out = torch.empty_like(X)
    info, _ = b.psd_server_wait(server, b.psd_server_submit(server, n, X, n, out, n, "fp16"))
    assert info["status"] == 0
    ref = oracle.oracle_project(Xh.astype(np.float64), "half")
    assert abs(info["lambda_bound"] - ref["lam_tilde"]) <= 1e-6 * ref["lam_tilde"]
    F = ref["F"]
    rel = np.linalg.norm(out.cpu().double().numpy() - F) / np.linalg.norm(F)
    assert rel < 2e-3, rel
    # the report's <out, X - out> / ||X||_F^2 against the exact filter output's
    coefs, scales = oracle.schedules.schedule("half")
    phi = oracle.phi(lam, info["lambda_bound"], coefs, scales)
    c_f = float(np.sum(phi * (lam - phi)) / np.sum(lam * lam))
    assert abs(info["compl_resid"] - c_f) <= 1e-2, (info["compl_resid"], c_f)


def test_tight_budget_admission_and_reuse():
    # room for about two requests of order 1024 at a time: the rest wait in
    # the queue, and every result still equals the single-call result
    n_max = 1024
    row_bytes = n_max * 2
    budget = (2 << 20) + 9 * n_max * row_bytes  # ~1 MB of records and scratch, then rows
    h = b.psd_server_create(budget, 0, n_max, 8)
    try:
        sizes = [1024, 700, 1000, 333, 1024, 64, 900, 1024, 513, 128, 1000, 1024]
        Xs = [make(n, 9300 + i) for i, n in enumerate(sizes)]
        ref = [single(n, X, n, "bf16")[0] for n, X in zip(sizes, Xs)]
        outs = [torch.full_like(X, float("nan")) for X in Xs]
        tickets = [b.psd_server_submit(h, n, X, n, o, n, "bf16") for n, X, o in zip(sizes, Xs, outs)]
        for n, t, o, r in zip(sizes, tickets, outs, ref):
            info, _ = b.psd_server_wait(h, t)
            assert info["status"] == 0
            assert torch.equal(o, r), n
        st = b.psd_server_stats(h)
        assert st["peak_rows"] <= st["arena_rows"]
        assert 2 * 4 * 1024 <= st["arena_rows"] < 3 * 4 * 1024  # two order-1024 requests fit, three do not
        assert st["completed"] == len(sizes)
    finally:
        b.psd_server_destroy(h)


def test_ld_and_inplace(server):
    n, ld = 300, 311
    X = make(n, 77, ld)
    ref, _ = single(n, X, ld, "bf16")
    out = torch.full((n, ld + 5), float("nan"), device="cuda")
    info, _ = b.psd_server_wait(server, b.psd_server_submit(server, n, X, ld, out, ld + 5, "bf16"))
    assert torch.equal(out[:, :n], ref[:, :n])
    assert torch.isnan(out[:, n:]).all()  # padding of out untouched
    Xi = X.clone()
    b.psd_server_wait(server, b.psd_server_submit(server, n, Xi, ld, Xi, ld, "bf16"))
    assert torch.equal(Xi[:, :n], ref[:, :n])


def test_ready_event_orders_the_input(server):
    n = 1000
    X = make(n, 5)
    ref, _ = single(n, X, n, "bf16")
    s = torch.cuda.Stream()
    Xw = torch.zeros_like(X)
    ev = torch.cuda.Event()
    with torch.cuda.stream(s):
        torch.cuda._sleep(20_000_000)  # the input is written well after the submit
        Xw.copy_(X)
        ev.record(s)
    out = torch.empty_like(X)
    info, _ = b.psd_server_wait(server, b.psd_server_submit(server, n, Xw, n, out, n, "bf16", ready=ev))
    assert torch.equal(out, ref)


def test_cancel_queued_request():
    h = b.psd_server_create(2 * GB, 0, 4096, 1)  # one request admitted at a time
    try:
        Xs = [make(4096, 1), make(512, 2), make(512, 3), make(512, 4)]
        outs = [torch.full_like(X, float("nan")) for X in Xs]
        ts = [b.psd_server_submit(h, X.shape[0], X, X.shape[0], o, X.shape[0], "bf16") for X, o in zip(Xs, outs)]
        b.psd_server_cancel(h, ts[2])
        infos = [b.psd_server_wait(h, t)[0] for t in ts]
        assert infos[2]["status"] == 8  # PSD_ERR_CANCELED
        assert torch.isnan(outs[2]).all()
        for k in (0, 1, 3):
            assert infos[k]["status"] == 0
            assert not torch.isnan(outs[k]).any()
        assert b.psd_server_stats(h)["canceled"] == 1
    finally:
        b.psd_server_destroy(h)


def test_wait_timeout_keeps_ticket(server):
    n = 2048
    X = make(n, 8)
    out = torch.empty_like(X)
    t = b.psd_server_submit(server, n, X, n, out, n, "bf16")
    with pytest.raises(b.PsdError) as e:
        b.psd_server_wait(server, t, timeout_ms=1)
    assert e.value.status == 6
    info, _ = b.psd_server_wait(server, t)
    assert info["status"] == 0
    with pytest.raises(b.PsdError):  # retired
        b.psd_server_poll(server, t)


def test_nonfinite_input_reported(server):
    n = 200
    X = make(n, 3)
    X[7, 5] = float("nan")  # upper triangle of the column-major matrix: row >= col in torch
    _, r_info = single(n, X, n, "bf16")
    out = torch.empty_like(X)
    info, _ = b.psd_server_wait(server, b.psd_server_submit(server, n, X, n, out, n, "bf16"))
    assert info["status"] == 4 and r_info["status"] == 4


def test_zero_order_and_bad_arguments(server):
    t = b.psd_server_submit(server, 0, None, 0, None, 0, "bf16")
    done, info, lat = b.psd_server_poll(server, t)
    assert done and info["status"] == 0
    X = make(64, 1)
    with pytest.raises(b.PsdError) as e:
        b.psd_server_submit(server, 4096, X, 4096, X, 4096, "bf16")  # above max_order
    assert e.value.status == 1
    with pytest.raises(b.PsdError) as e:
        b.psd_server_submit(server, 64, X, 64, X, 64, "fp32")
    assert e.value.status == 7
    with pytest.raises(b.PsdError) as e:
        b.psd_server_submit(server, 64, X, 63, X, 64, "bf16")  # ld < n
    assert e.value.status == 1
    with pytest.raises(b.PsdError) as e:
        b.psd_server_create(1 << 20, 0, 8192, 4)  # budget below one request
    assert e.value.status == 3
