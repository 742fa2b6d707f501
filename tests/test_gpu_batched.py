"""GPU tests of the batched projection of a block-diagonal cone (grouped
launches over all blocks), through the C ABI: parity of every block against
the CPU FP64 oracle's filter output, bit-identity of a block alone and in the
batch, caller leading dimensions and in-place outputs, argument checks."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from oracle import emulate  # noqa: E402
from paper_2507_09165_gb300 import binding as b  # noqa: E402
from paper_2507_09165_gb300 import synth  # noqa: E402

DEV = torch.device("cuda")
from _bars import SCHED, TOL_F, check_all  # noqa: E402
SIZES = [1, 7, 33, 64, 100, 128, 129, 200, 256, 300, 513, 1024]


class Batch:
    def __init__(self, mats, ld_pad=0, out_pad=0, inplace=()):
        self.n = [m.shape[0] for m in mats]
        self.X, self.out, self.info, self.ld, self.ldo = [], [], [], [], []
        for i, M in enumerate(mats):
            n = M.shape[0]
            ld = n + ld_pad
            t = torch.zeros((n, ld), dtype=torch.float32)
            t[:, :n] = torch.from_numpy(M)
            Xd = t.to(DEV)
            if i in inplace:
                out, ldo = Xd, ld
            else:
                ldo = n + out_pad
                out = torch.full((n, ldo), float("nan"), dtype=torch.float32, device=DEV)
            self.X.append(Xd)
            self.out.append(out)
            self.ld.append(ld)
            self.ldo.append(ldo)
            self.info.append(torch.zeros(b.INFO_BYTES, dtype=torch.uint8, device=DEV))

    def run(self, prec):
        descs = b.block_descs([(n, X, ld, out, ldo, inf) for n, X, ld, out, ldo, inf in
                               zip(self.n, self.X, self.ld, self.out, self.ldo, self.info)])
        b.psd_project_batched(len(self.n), descs, prec)
        torch.cuda.synchronize()
        outs = [o.cpu().numpy()[:, :n].astype(np.float64) for o, n in zip(self.out, self.n)]
        infos = [b.info_from_bytes(i.cpu().numpy()) for i in self.info]
        return outs, infos


@pytest.fixture(scope="module")
def mats():
    out = []
    for i, n in enumerate(SIZES):
        X = synth.gaussian_symmetric(n, 900 + i) if i % 2 else synth.wigner(n, 900 + i)
        ref = oracle.oracle_project(X.astype(np.float64), "half")
        coefs, scales = oracle.schedules.schedule("single")
        ref["F_single"] = oracle.filter_from_eig(ref["lam"], ref["Q"], ref["lam_tilde"], coefs, scales)
        out.append((X, ref))
    return out


@pytest.mark.parametrize("prec", ["fp16", "bf16", "mixed", "fp32"])
def test_batched_matches_oracle(mats, prec):
    B = Batch([m for m, _ in mats])
    outs, infos = B.run(prec)
    results = []
    for (X, ref), o, inf, n in zip(mats, outs, infos, SIZES):
        assert inf["status"] == 0, (n, inf)
        assert inf["lambda_bound"] == pytest.approx(ref["lam_tilde"], rel=1e-6)
        assert np.array_equal(o, o.T)
        F = ref["F_single"] if SCHED[prec] == "single" else ref["F"]
        X64 = X.astype(np.float64)
        if n == 1:
            # n = 1: the error relative to |x| (F = phi(x) can be ~0)
            err = abs(o[0, 0] - F[0, 0]) / abs(X64[0, 0])
            coefs, scales = oracle.schedules.schedule(SCHED[prec])

            def model(X64=X64, F=F, lt=inf["lambda_bound"]):
                out_m, _, _ = emulate.chain_rounded(X64, lt, coefs, scales, emulate.named_plan(prec))
                return abs(out_m[0, 0] - F[0, 0]) / abs(X64[0, 0])
            results.append((err, None, None, "n = 1", None, model if prec != "fp32" else None))
            continue
        results.append((oracle.rel_err(o, F), X64, inf["lambda_bound"], "n = %d" % n))
        c_ref = float(np.sum(o * (X64 - o))) / float(np.sum(X64 * X64))
        assert abs(inf["compl_resid"] - c_ref) <= 1e-7, (n, inf["compl_resid"], c_ref)
    check_all(prec, results)


@pytest.mark.parametrize("prec", ["bf16", "mixed"])
def test_block_alone_and_in_batch_bitwise(mats, prec):
    B = Batch([m for m, _ in mats])
    outs, _ = B.run(prec)
    for k in (0, 5, 8, 11):
        A = Batch([mats[k][0]])
        alone, _ = A.run(prec)
        assert np.array_equal(alone[0], outs[k]), SIZES[k]
    # a different batch composition (reversed order, some blocks dropped)
    sub = [mats[k][0] for k in (11, 8, 5, 0)]
    C = Batch(sub)
    outs2, _ = C.run(prec)
    for k, o in zip((11, 8, 5, 0), outs2):
        assert np.array_equal(o, outs[k])


def test_batched_leading_dims_and_inplace(mats):
    sub = [mats[k][0] for k in (2, 7, 9)]
    B1 = Batch(sub)
    ref, _ = B1.run("fp16")
    B2 = Batch(sub, ld_pad=5, out_pad=3, inplace=(1,))
    got, infos = B2.run("fp16")
    for a, c, inf in zip(ref, got, infos):
        assert inf["status"] == 0
        assert np.array_equal(a, c)


@pytest.mark.parametrize("prec", ["fp16", "bf16"])
def test_batched_config_workload_sampled(prec):
    # 512 Wigner blocks, orders log-uniform in [16, 1024] (seed 7); parity on a
    # sample.  The block-diagonal workload runs in FP16, which meets the 2e-3
    # bar on it; BF16 is checked against the same bar (a known miss).
    sizes = synth.block_sizes(512, 7)
    rng = np.random.default_rng(0)
    mats = [synth.wigner(n, 7000 + i) for i, n in enumerate(sizes)]
    B = Batch(mats)
    outs, infos = B.run(prec)
    assert all(inf["status"] == 0 for inf in infos)
    results = []
    for i in rng.choice(512, size=6, replace=False):
        X = mats[i].astype(np.float64)
        ref = oracle.oracle_project(X, "half")
        results.append((oracle.rel_err(outs[i], ref["F"]), X, infos[i]["lambda_bound"], "block %d, n = %d" % (i, sizes[i])))
    check_all(prec, results)


def test_batched_rejects_bad_blocks():
    X = torch.zeros((1025, 1025), device=DEV)
    with pytest.raises(b.PsdError):
        b.psd_project_batched(1, b.block_descs([(1025, X, 1025, X, 1025, None)]), "bf16")
    Y = torch.zeros((8, 8), device=DEV)
    with pytest.raises(b.PsdError):
        b.psd_project_batched(1, b.block_descs([(8, Y, 7, Y, 8, None)]), "bf16")
    with pytest.raises(b.PsdError):
        b.psd_project_batched(1, b.block_descs([(8, Y, 8, Y, 8, None)]), "fp8_early")


@pytest.mark.parametrize("prec", ["bf16", "mixed"])
def test_every_schedule_gives_the_same_bits_and_autotune_picks_one(prec):
    # The autotuner only reorders which persistent CTA takes which tile of a
    # grouped product: every candidate schedule must give bit-identical
    # outputs and reports.  A batch with a signature of its own, so the
    # autotuned run below times all candidates instead of reusing a choice.
    # BF16 plans have a seventh candidate, the 256 x 256 tiles on SM pairs,
    # whose final product sums the complementarity residual from 16 shares per
    # tile instead of 4 (the same value to rounding).
    sizes = [900, 17, 640, 256, 1000, 3, 450, 128, 777, 64, 300 + (prec == "mixed")]
    mats = [synth.wigner(n, 4400 + i) for i, n in enumerate(sizes)]
    ncand = 7 if prec == "bf16" else 6
    ref = None
    try:
        for idx in range(ncand):
            b.psd_batched_force_schedule(idx)
            b.psd_release_workspaces()
            outs, infos = Batch(mats).run(prec)
            chosen, _ = b.psd_batched_last_tuning()
            assert chosen == idx
            assert all(i["status"] == 0 for i in infos)
            if ref is None:
                ref = (outs, infos)
            else:
                for o, r in zip(outs, ref[0]):
                    assert np.array_equal(o, r), idx
                for i, r in zip(infos, ref[1]):
                    assert {k: v for k, v in i.items() if k != "compl_resid"} == \
                        {k: v for k, v in r.items() if k != "compl_resid"}, idx
                    assert abs(i["compl_resid"] - r["compl_resid"]) <= 1e-12 + 1e-9 * abs(r["compl_resid"])
        b.psd_batched_force_schedule(-1)
        b.psd_release_workspaces()
        outs, _ = Batch(mats).run(prec)
        chosen, ms = b.psd_batched_last_tuning()
        assert 0 <= chosen < ncand and len(ms) == ncand
        assert all(t > 0 for t in ms) and ms[chosen] == min(ms)
        for o, r in zip(outs, ref[0]):
            assert np.array_equal(o, r)
    finally:
        b.psd_batched_force_schedule(-1)


@pytest.mark.parametrize("prec", ["fp16", "bf16"])
@pytest.mark.parametrize("workload", ["orders", "512 blocks"])
def test_product_shapes_and_forms_give_the_same_bits(mats, prec, workload):
    # FP16 / BF16 plans can run their products as 128-row tiles with one
    # launch per product (schedule 0), as 256 x 256 tiles on SM pairs
    # (schedule 6), or as the chain form (all products in one persistent launch,
    # a block's next product waiting on counters of its previous product's
    # tiles).  Per element the arithmetic is the same: outputs and bounds are
    # bit-identical, the complementarity residual (4, 16 or 8 shares per tile)
    # agrees to rounding.
    if workload == "orders":
        ms = [m for m, _ in mats]
    else:
        ms = [synth.wigner(n, 7000 + i) for i, n in enumerate(synth.block_sizes(512, 7))]
    res = []
    try:
        for sched, form in ((0, 0), (6, 0), (0, 1)):
            b.psd_batched_force_schedule(sched)
            b.psd_batched_force_form(form)
            b.psd_release_workspaces()
            res.append(Batch(ms).run(prec))
            assert b.psd_batched_last_tuning()[0] == sched
    finally:
        b.psd_batched_force_schedule(-1)
        b.psd_batched_force_form(-1)
    o0, i0 = res[0]
    for o1, i1 in res[1:]:
        for k in range(len(ms)):
            assert i1[k]["status"] == i0[k]["status"] == 0, k
            assert np.array_equal(o0[k], o1[k]), (k, ms[k].shape[0])
            assert i1[k]["lambda_bound"] == i0[k]["lambda_bound"]
            assert i1[k]["overshoot_max"] == i0[k]["overshoot_max"]
            assert abs(i1[k]["compl_resid"] - i0[k]["compl_resid"]) <= 1e-12 + 1e-9 * abs(i0[k]["compl_resid"])


@pytest.mark.parametrize("workload", ["orders", "512 blocks"])
def test_norm_bound_forms_give_the_same_bits(mats, workload):
    # The batched norm bound runs as ONE launch whose CTAs claim work items
    # (start vectors, mat-vec tiles, reductions, Lanczos steps, Ritz vectors,
    # bounds) and wait only on their own block's earlier items, or as one
    # grouped launch per phase.  Each item runs the same arithmetic in the same
    # order, so outputs and whole reports must agree bit for bit; the orders
    # include blocks below 20 (Lanczos breakdown: their later items do no work).
    if workload == "orders":
        ms = [m for m, _ in mats]
    else:
        ms = [synth.wigner(n, 7000 + i) for i, n in enumerate(synth.block_sizes(512, 7))]
    res = []
    try:
        for form in (0, 1):
            b.psd_batched_force_bound(form)
            b.psd_release_workspaces()
            res.append(Batch(ms).run("fp16"))
    finally:
        b.psd_batched_force_bound(-1)
    (o0, i0), (o1, i1) = res
    for k in range(len(ms)):
        assert i0[k]["status"] == 0, k
        assert np.array_equal(o0[k], o1[k]), (k, ms[k].shape[0])
        assert i1[k] == i0[k], (k, ms[k].shape[0])
