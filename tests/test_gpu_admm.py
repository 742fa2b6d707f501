"""GPU test of the ADMM serving workload: interleaved solves through the
request server follow exactly the trajectory of the same solves run with
direct psd_project calls (every projection is bit-identical, and the y- and
X-updates are deterministic), and they make progress on the SDP."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from paper_2507_09165_gb300 import admm, binding as b, synth  # noqa: E402


def test_served_admm_matches_direct_calls():
    graphs = {n: torch.from_numpy(synth.er_laplacian(n, 8 + i, p=0.05).astype(np.float32)).cuda()
              for i, n in enumerate((64, 200, 333))}
    iters = 12
    server = b.psd_server_create(1 << 30, 0, 512, 16)
    try:
        res = admm.run_serving(server, graphs, "bf16", solve_rate=400.0, arrival_seconds=0.02, iters=iters,
                               think_ms=0.2, seed=3, max_solves=6)
    finally:
        b.psd_server_destroy(server)
    assert len(res["solves"]) == res["arrivals"] >= 2
    assert all(r["status"] == 0 for r in res["records"])
    assert len(res["records"]) == iters * len(res["solves"])
    # replay each solve with direct calls on one stream
    for sd in res["solves"]:
        C = graphs[sd["n"]]
        sv = admm.Solve(C, sd["sigma"], iters)
        for _ in range(iters):
            V = sv.make_input()
            torch.cuda.synchronize()
            b.psd_project(sv.n, V, sv.n, sv.S, "bf16")
            torch.cuda.synchronize()
            sv.finish_iteration()
        eta, _ = sv.surrogate()
        assert eta == sd["eta"], (sd, eta)
    summary = admm.summarize(res)
    assert summary["bad_status"] == 0 and summary["requests"] == len(res["records"])
