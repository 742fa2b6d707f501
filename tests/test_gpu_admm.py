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
        res = admm.run_serving(server, graphs, "fp16", solve_rate=400.0, arrival_seconds=0.02, iters=iters,
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
            b.psd_project(sv.n, V, sv.n, sv.S, "fp16")
            torch.cuda.synchronize()
            sv.finish_iteration()
        eta, _ = sv.surrogate()
        assert eta == sd["eta"], (sd, eta)
    summary = admm.summarize(res)
    assert summary["bad_status"] == 0 and summary["requests"] == len(res["records"])


def test_solver_warm_start_matches_exact_admm():
    # max-cut SDP of a small random graph: the GPU solver (mixed projections,
    # then FP32 ones once the surrogate is below 1e-2) reaches the optimum the
    # same ADMM finds with exact (eigendecomposition) projections on the CPU
    n = 120
    L = synth.er_laplacian(n, 21, p=0.1)
    C64 = -L / 4.0
    C = torch.from_numpy(C64.astype(np.float32)).cuda()

    def project_gpu(V, S, prec):
        b.psd_project(n, V, n, S, prec)

    r = admm.solve(C, project_gpu, sigma=1.0, max_iters=3000, eta_switch=1e-2, eta_tol=1e-4, check_every=10)
    assert r["switch_iter"] is not None and r["history"][-1][1] == "fp32"
    assert r["history"][-1][2] < 1e-4, r["history"][-5:]
    pobj = float((C.double() * r["X"].double()).sum())

    def project_cpu(V, S, prec):
        w, Q = np.linalg.eigh(V.double().numpy())
        S.copy_(torch.from_numpy((Q * np.maximum(w, 0.0)) @ Q.T))

    ref = admm.solve(torch.from_numpy(C64), project_cpu, sigma=1.0, max_iters=6000, eta_switch=1e-2,
                     eta_tol=1e-7, check_every=50)
    pref = float((torch.from_numpy(C64) * ref["X"]).sum())
    assert abs(pobj - pref) <= 1e-3 * abs(pref), (pobj, pref)
