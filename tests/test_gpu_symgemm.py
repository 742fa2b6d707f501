"""GPU tests of the tensor-core symmetric product (the building block of every
stage of Algorithm 2), called through the C ABI.

Expected values are FP64 products of the same 16-bit operands computed on the
CPU with numpy; the kernel accumulates in FP32 and rounds the result once to
16 bits (or writes FP32 for the final epilogue).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from paper_2507_09165_gb300 import binding as b  # noqa: E402

SIZES = [16, 100, 128, 255, 256, 300, 513, 1000]
DT = {"fp16": torch.float16, "bf16": torch.bfloat16}
EPS = {"fp16": 2.0 ** -11, "bf16": 2.0 ** -8}


def sym16(n, ld, seed, prec, scale=1.0):
    rng = np.random.default_rng(seed)
    G = rng.standard_normal((n, n)) * (scale / np.sqrt(n))
    A = 0.5 * (G + G.T)
    t = torch.zeros((n, ld), dtype=DT[prec])
    t[:, :n] = torch.from_numpy(A).to(DT[prec])
    return t


def as64(t, n):
    return t[:, :n].double().numpy()


def check_upper(C, D, n, prec, absA, absB):
    # |C - D| <= one rounding of D plus the FP32 accumulation error bound
    acc = n * 2.0 ** -23 * (absA @ absB)
    tol = EPS[prec] * np.abs(D) + 2 * acc + 1e-30
    err = np.abs(C - D)
    iu = np.triu_indices(n)
    bad = err[iu] > tol[iu]
    assert not np.any(bad), (np.max(err[iu] / tol[iu]), int(np.sum(bad)))


@pytest.mark.parametrize("prec", ["fp16", "bf16"])
@pytest.mark.parametrize("n", SIZES)
def test_product_copy(n, prec):
    ld = (n + 7) // 8 * 8
    A = sym16(n, ld, 1 + n, prec)
    B = sym16(n, ld, 2 + n, prec)
    dev = torch.device("cuda")
    Ad, Bd = A.to(dev), B.to(dev)
    Cd = torch.full((n, ld), float("nan"), dtype=DT[prec], device=dev)
    b.psd_symm_product(n, Ad, Bd, ld, Cd, 0, prec, 0)
    torch.cuda.synchronize()
    C = as64(Cd.cpu(), n)
    A64, B64 = as64(A, n), as64(B, n)
    D = A64 @ B64.T
    assert np.all(np.isfinite(C))
    assert np.array_equal(C, C.T)  # exactly symmetric
    check_upper(C, D, n, prec, np.abs(A64), np.abs(B64))
    # the padding columns are never written
    if ld > n:
        assert torch.isnan(Cd[:, n:].float()).all()


@pytest.mark.parametrize("n", [64, 300, 700])
def test_product_poly_scale_and_absmax(n):
    prec = "fp16"
    ld = (n + 7) // 8 * 8
    dev = torch.device("cuda")
    Y = sym16(n, ld, 10 + n, prec)
    Yd = Y.to(dev)
    P = torch.zeros((n, ld), dtype=torch.float16, device=dev)
    a, bb, c = 2.7632556383, -2.0607754898, 0.4695405857
    amax = torch.zeros(1, dtype=torch.float32, device=dev)
    b.psd_symm_product(n, Yd, Yd, ld, P, 0, prec, 1, (a, bb, c), Yd, ld, amax)
    S = torch.zeros((n, ld), dtype=torch.float16, device=dev)
    b.psd_symm_product(n, Yd, Yd, ld, S, 0, prec, 2, (1 / 1.01,))
    torch.cuda.synchronize()
    Y64 = as64(Y, n)
    D = Y64 @ Y64
    # FP32 epilogue arithmetic on the FP32 accumulator, one rounding to fp16
    Dp = a * np.eye(n) + bb * Y64 + c * D
    Pc = as64(P.cpu(), n)
    assert np.array_equal(Pc, Pc.T)
    absY = np.abs(Y64)
    acc = n * 2.0 ** -23 * (absY @ absY)
    tol = EPS[prec] * np.abs(Dp) + 2 * abs(c) * acc + 1e-6 * (abs(a) + abs(bb) * absY)
    assert np.all(np.abs(Pc - Dp) <= tol)
    assert float(amax.item()) == float(np.max(np.abs(Pc)))
    Sc = as64(S.cpu(), n)
    Ds = D / 1.01
    assert np.all(np.abs(Sc - Ds) <= EPS[prec] * np.abs(Ds) + 2 * acc)


@pytest.mark.parametrize("n", [33, 256, 517])
def test_product_final_reads_upper_triangle_only(n):
    # out = (Xf + lam A B) / 2 in FP32; Xf's other triangle holds NaN and must
    # never be read.  In a row-major tensor the library's (column-major) upper
    # triangle X[i + j ld], i <= j, is T[j][i]: the row >= col part.
    prec = "fp16"
    ld = (n + 7) // 8 * 8
    dev = torch.device("cuda")
    A = sym16(n, ld, 20 + n, prec)
    B = sym16(n, ld, 21 + n, prec)
    rng = np.random.default_rng(n)
    Xs = rng.standard_normal((n, n)).astype(np.float32)
    Xs = np.tril(Xs) + np.tril(Xs, -1).T
    Xpoison = Xs.copy()
    Xpoison[np.triu_indices(n, 1)] = np.nan
    ldx = n + 3
    Xt = torch.zeros((n, ldx), dtype=torch.float32)
    Xt[:, :n] = torch.from_numpy(Xpoison)
    ldo = n + 5
    out = torch.full((n, ldo), -7.0, dtype=torch.float32, device=dev)
    lam = 3.25
    b.psd_symm_product(n, A.to(dev), B.to(dev), ld, out, ldo, prec, 3, (lam,), Xt.to(dev), ldx)
    torch.cuda.synchronize()
    o = out.cpu().numpy().astype(np.float64)
    assert np.all(o[:, n:] == -7.0)
    o = o[:, :n]
    assert np.all(np.isfinite(o))
    assert np.array_equal(o, o.T)
    A64, B64 = as64(A, n), as64(B, n)
    D = 0.5 * (Xs.astype(np.float64) + lam * (A64 @ B64.T))
    acc = n * 2.0 ** -23 * (np.abs(A64) @ np.abs(B64))
    tol = 2.0 ** -22 * (np.abs(D) + np.abs(Xs)) + lam * acc
    iu = np.triu_indices(n)
    assert np.all(np.abs(o - D)[iu] <= tol[iu] + 1e-6)


def test_product_is_deterministic():
    n, prec = 777, "bf16"
    ld = 784
    dev = torch.device("cuda")
    A = sym16(n, ld, 5, prec).to(dev)
    outs = []
    for _ in range(3):
        C = torch.zeros((n, ld), dtype=DT[prec], device=dev)
        b.psd_symm_product(n, A, A, ld, C, 0, prec, 0)
        outs.append(C)
    torch.cuda.synchronize()
    assert torch.equal(outs[0], outs[1]) and torch.equal(outs[1], outs[2])


def test_product_rejects_bad_arguments():
    dev = torch.device("cuda")
    A = torch.zeros((8, 8), dtype=torch.float16, device=dev)
    with pytest.raises(b.PsdError):
        b.psd_symm_product(8, A, A, 7, A, 0, "fp16", 0)  # ld not a multiple of 8
    with pytest.raises(b.PsdError):
        b.psd_symm_product(8, A, A, 8, A, 0, "fp8_early", 0)  # no product for this precision
    with pytest.raises(b.PsdError):
        b.psd_symm_product(8, A, A, 8, A, 0, "fp16", 9)  # unknown epilogue


def split_pair(A64, prec, n, ld):
    """(hi, lo) storage of A64 as FP16 pairs (mixed) or TF32 pairs (fp32), rows of ld elements."""
    if prec == "mixed":
        hi = torch.from_numpy(A64).to(torch.float16)
        lo = (torch.from_numpy(A64) - hi.double()).to(torch.float16)
        dt = torch.float16
    else:
        a = torch.from_numpy(A64.astype(np.float32)).view(torch.int32).numpy().astype(np.int64)
        hb = ((a + 0x1000) & 0xFFFFE000).astype(np.uint32).view(np.float32)
        rem = (A64.astype(np.float32) - hb).astype(np.float32).view(np.int32).astype(np.int64)
        lb = ((rem + 0x1000) & 0xFFFFE000).astype(np.uint32).view(np.float32)
        hi, lo = torch.from_numpy(hb.copy()), torch.from_numpy(lb.copy())
        dt = torch.float32
    t = torch.zeros((2, n, ld), dtype=dt)
    t[0, :, :n] = hi
    t[1, :, :n] = lo
    return t


@pytest.mark.parametrize("prec", ["mixed", "fp32"])
@pytest.mark.parametrize("n", [64, 255, 300, 513, 1500])
def test_split_product(n, prec):
    # value = hi + lo; product = A_hi B_hi + A_hi B_lo + A_lo B_hi, FP32 accumulation,
    # output split again: FP16 pairs keep ~22 bits (fewer where lo is subnormal),
    # TF32 pairs ~22 bits.
    ld = (n + 7) // 8 * 8
    rng = np.random.default_rng(n)
    G = rng.standard_normal((n, n)) / np.sqrt(n)
    A64 = 0.5 * (G + G.T)
    G = rng.standard_normal((n, n)) / np.sqrt(n)
    B64 = 0.5 * (G + G.T)
    A, B = split_pair(A64, prec, n, ld), split_pair(B64, prec, n, ld)
    dev = torch.device("cuda")
    Ad, Bd = A.to(dev), B.to(dev)
    Cd = torch.full_like(Ad, float("nan"))
    b.psd_symm_product(n, Ad, Bd, ld, Cd, 0, prec, 0)
    torch.cuda.synchronize()
    Cc = Cd.cpu().double().numpy()
    C = Cc[0, :, :n] + Cc[1, :, :n]
    Av = A.double().numpy()[0, :, :n] + A.double().numpy()[1, :, :n]
    Bv = B.double().numpy()[0, :, :n] + B.double().numpy()[1, :, :n]
    D = Av @ Bv
    assert np.array_equal(C, C.T)
    # A B of two different symmetric matrices is not symmetric: the kernel forms
    # the upper triangle and mirrors it, so compare the upper triangle
    iu = np.triu_indices(n)
    rel = 2.0 ** -18 if prec == "mixed" else 2.0 ** -20
    acc = 4 * n * 2.0 ** -24 * (np.abs(Av) @ np.abs(Bv))
    err, tol = np.abs(C - D)[iu], (rel * np.abs(D) + acc)[iu]
    assert np.all(err <= tol), np.max(err / tol)
    # far more accurate than one 16-bit product.  TF32 pairs: the tensor cores
    # add into FP32 without rounding to nearest; the kernel folds K-chunks of
    # 128 into a round-to-nearest running sum, so the error does not grow with n
    # (without folding: 1.8e-6 at n = 255, 3.7e-6 at n = 513).
    bound = 2e-5 if prec == "mixed" else 1.5e-6
    assert np.linalg.norm(err) / np.linalg.norm(D[iu]) < bound


@pytest.mark.parametrize("prec", ["mixed", "fp32"])
@pytest.mark.parametrize("n", [97, 300, 513])
def test_split_product_poly_and_scale_epilogues(n, prec):
    # The stage epilogues of the split product on pair operands, ld a multiple of 8
    # (not of 64) and n not a multiple of 32, so the Y chunks have ragged edges:
    # P = a I + b Y + c Y^2 (polynomial, Y read as a pair in the epilogue) and
    # s A B (scale), both split into pairs again.
    ld = (n + 7) // 8 * 8
    rng = np.random.default_rng(1000 + n)
    G = rng.standard_normal((n, n)) / np.sqrt(n)
    Y64 = 0.5 * (G + G.T)
    G = rng.standard_normal((n, n)) / np.sqrt(n)
    B64 = 0.5 * (G + G.T)
    Y, B = split_pair(Y64, prec, n, ld), split_pair(B64, prec, n, ld)
    dev = torch.device("cuda")
    Yd, Bd = Y.to(dev), B.to(dev)
    Yv = Y.double().numpy()[0, :, :n] + Y.double().numpy()[1, :, :n]
    Bv = B.double().numpy()[0, :, :n] + B.double().numpy()[1, :, :n]
    a, bb, c, sc = 1.5, -0.7, 0.3, 1.0 / 1.01
    iu = np.triu_indices(n)
    rel = 2.0 ** -18 if prec == "mixed" else 2.0 ** -20
    for epi, params, B_d, Bval in ((1, (a, bb, c), Yd, Yv), (2, (sc,), Bd, Bv)):
        Cd = torch.full_like(Yd, float("nan"))
        if epi == 1:
            b.psd_symm_product(n, Yd, B_d, ld, Cd, 0, prec, 1, params=params, aux=Yd, ld_aux=ld)
        else:
            b.psd_symm_product(n, Yd, B_d, ld, Cd, 0, prec, 2, params=params)
        torch.cuda.synchronize()
        Cc = Cd.cpu().double().numpy()
        C = Cc[0, :, :n] + Cc[1, :, :n]
        prod = Yv @ Bval
        acc = 4 * n * 2.0 ** -24 * (np.abs(Yv) @ np.abs(Bval))
        if epi == 1:
            D = a * np.eye(n) + bb * Yv + c * prod
            tol = abs(c) * (rel * np.abs(prod) + acc) + rel * np.abs(D) + 2.0 ** -22 * (abs(bb) * np.abs(Yv) + a)
        else:
            D = sc * prod
            tol = sc * (rel * np.abs(prod) + acc) + rel * np.abs(D)
        assert np.array_equal(C, C.T), epi
        err = np.abs(C - D)[iu]
        assert np.all(err <= tol[iu]), (epi, np.max(err / tol[iu]))


F8 = getattr(torch, "float8_e4m3fn", None)


def e4m3_sym(n, ld, seed, scale):
    """(device bytes, decoded FP64 values) of a symmetric matrix stored as RN_e4m3(value * scale)."""
    rng = np.random.default_rng(seed)
    G = rng.standard_normal((n, n)) / np.sqrt(n)
    A = 0.5 * (G + G.T)
    q = torch.from_numpy(A * scale).to(F8)  # round to nearest, values far below 448
    t = torch.zeros((n, ld), dtype=torch.uint8)
    t[:, :n] = q.view(torch.uint8)
    return t.cuda(), q.double().numpy() / scale


@pytest.mark.skipif(F8 is None, reason="torch without float8_e4m3fn")
@pytest.mark.parametrize("n", [16, 130, 255, 300, 700])
def test_fp8_products(n):
    # e4m3 operands (kind::f8f6f4), FP32 accumulation, e4m3 output with power-of-two scales
    ld = (n + 15) // 16 * 16
    sA, sB, sC, sY = 256.0, 128.0, 64.0, 256.0
    Ad, A = e4m3_sym(n, ld, 40 + n, sA)
    Bd, B = e4m3_sym(n, ld, 41 + n, sB)
    Yd, Y = e4m3_sym(n, ld, 42 + n, sY)
    absAB = np.abs(A) @ np.abs(B)
    acc = 2 * n * 2.0 ** -23 * absAB

    def run(epi, params):
        C = torch.full((n, ld), 0x7F, dtype=torch.uint8, device="cuda")  # e4m3 NaN poison
        b.psd_symm_product(n, Ad, Bd, ld, C, 0, "fp8_late", epi, params, Yd if epi == 1 else None, ld)
        torch.cuda.synchronize()
        Cb = C.cpu()
        assert (Cb[:, n:] == 0x7F).all()  # padding never written
        v = Cb[:, :n].contiguous().view(F8).double().numpy() / sC
        return v

    D = A @ B
    iu = np.triu_indices(n)
    # epi 0: C = A B
    C0 = run(0, (1.0 / (sA * sB), 1.0, sC))
    assert np.all(np.isfinite(C0)) and np.array_equal(C0, C0.T)
    tol = 2.0 ** -4 * np.abs(D) + 2.0 ** -10 / sC + acc
    assert np.all(np.abs(C0 - D)[iu] <= tol[iu])
    # epi 1: C = a I + b Y + c A B  (Y read as e4m3 / sY)
    a, bb, c = 0.75, -0.5, 0.25
    C1 = run(1, (a, bb, c, 1.0 / (sA * sB), 1.0 / sY, sC))
    D1 = a * np.eye(n) + bb * Y + c * D
    tol1 = 2.0 ** -4 * np.abs(D1) + 2.0 ** -10 / sC + abs(c) * acc + 1e-6
    assert np.all(np.abs(C1 - D1)[iu] <= tol1[iu])
    # epi 2: C = (A B) s
    C2 = run(2, (0.5, 1.0 / (sA * sB), 1.0, sC))
    D2 = 0.5 * D
    tol2 = 2.0 ** -4 * np.abs(D2) + 2.0 ** -10 / sC + acc
    assert np.all(np.abs(C2 - D2)[iu] <= tol2[iu])


@pytest.mark.parametrize("n", [97, 300, 513])
@pytest.mark.parametrize("epi,out", [(e, o) for o in ("fp16", "bf16", "fp16 pair") for e in (0, 1, 2)
                                     if not (o == "fp16 pair" and e == 2)])
def test_grouped_instance_gives_the_same_bits(n, epi, out):
    # The grouped launches over many small matrices (block-diagonal cones) run
    # an instance with 8 epilogue warps, each taking every second 32-column
    # chunk of its quarter of the tile, and a 3-stage ring; the single-matrix
    # launches run 4 warps and a 4-stage ring.  Same arithmetic per element:
    # the outputs must be bit-identical, for every stage epilogue, the 16-bit
    # and the FP16-pair outputs, and orders whose chunk counts are odd.
    prec = "bf16" if out == "bf16" else "fp16"
    ld = (n + 7) // 8 * 8
    dev = torch.device("cuda")
    A = sym16(n, ld, 40 + n, prec).to(dev)
    B = sym16(n, ld, 41 + n, prec).to(dev)
    Y = sym16(n, ld, 42 + n, prec).to(dev)
    flag = b.EPI_F16_PAIR_OUT if out == "fp16 pair" else 0
    params = {0: (), 1: (4.0611848147, -2.9698947955, 0.5492133813), 2: (1 / 1.01,)}[epi]
    rows = 2 * n if flag else n
    outs = []
    for grouped in (0, b.EPI_GROUPED):
        C = torch.full((rows, ld), float("nan"), dtype=DT[prec], device=dev)
        b.psd_symm_product(n, A, B if epi != 1 else Y, ld, C, 0, prec, epi | flag | grouped, params,
                           Y if epi == 1 else None, ld if epi == 1 else 0)
        torch.cuda.synchronize()
        outs.append(C.cpu())
    c4, c8 = outs
    assert torch.isfinite(c4[:, :n]).all()
    assert torch.equal(c4.view(torch.int16), c8.view(torch.int16))
    if flag:  # the pair carries more than the single FP16 rounding: lo is not all zero
        assert torch.count_nonzero(c4[n:, :n]) > n


@pytest.mark.parametrize("n", [16, 97, 255, 256, 300, 513, 1000])
@pytest.mark.parametrize("epi,out", [(e, o) for o in ("fp16", "bf16", "fp16 pair") for e in (0, 1, 2)
                                     if not (o == "fp16 pair" and e == 2)])
def test_cta_pair_form_gives_the_same_bits(n, epi, out):
    # The projection's 16-bit stage products run on pairs of SMs: one M = 256
    # tensor-core product per 256 x 256 tile, A's rows split between the two
    # SMs and B's rows split between their shared memories.  Per element it is
    # the same dot product in the same K order as the one-SM form, so the two
    # outputs must be bit-identical, also where a 256-row tile is ragged
    # (n = 97, 255, 300, 513, 1000) or the pair owns a single tile (n = 16).
    prec = "bf16" if out == "bf16" else "fp16"
    ld = (n + 7) // 8 * 8
    dev = torch.device("cuda")
    A = sym16(n, ld, 50 + n, prec).to(dev)
    B = sym16(n, ld, 51 + n, prec).to(dev)
    Y = sym16(n, ld, 52 + n, prec).to(dev)
    flag = b.EPI_F16_PAIR_OUT if out == "fp16 pair" else 0
    params = {0: (), 1: (4.0611848147, -2.9698947955, 0.5492133813), 2: (1 / 1.01,)}[epi]
    rows = 2 * n if flag else n
    outs = []
    for form in (0, b.EPI_CTA_PAIR):
        C = torch.full((rows, ld), float("nan"), dtype=DT[prec], device=dev)
        b.psd_symm_product(n, A, B if epi != 1 else Y, ld, C, 0, prec, epi | flag | form, params,
                           Y if epi == 1 else None, ld if epi == 1 else 0)
        torch.cuda.synchronize()
        outs.append(C.cpu())
    c1, c2 = outs
    assert torch.isfinite(c1[:, :n]).all()
    assert torch.equal(c1.view(torch.int16), c2.view(torch.int16))


@pytest.mark.parametrize("prec", ["fp16", "bf16"])
@pytest.mark.parametrize("n", [16, 97, 255, 300, 513, 1000])
def test_cta_pair_form_final_product_gives_the_same_bits(n, prec):
    # The final product out = (X + lam~ A B) / 2 in FP32, on pairs of SMs and
    # on one: the same accumulator bits, so the same output, both triangles.
    ld = (n + 7) // 8 * 8
    dev = torch.device("cuda")
    A = sym16(n, ld, 60 + n, prec).to(dev)
    B = sym16(n, ld, 61 + n, prec).to(dev)
    rng = np.random.default_rng(62 + n)
    G = rng.standard_normal((n, n))
    X = torch.from_numpy((0.5 * (G + G.T)).astype(np.float32)).to(dev)
    outs = []
    for form in (0, b.EPI_CTA_PAIR):
        C = torch.full((n, n), float("nan"), dtype=torch.float32, device=dev)
        b.psd_symm_product(n, A, B, ld, C, n, prec, 3 | form, (1.37,), X, n)
        torch.cuda.synchronize()
        outs.append(C.cpu())
    assert torch.isfinite(outs[0]).all()
    assert torch.equal(outs[0].view(torch.int32), outs[1].view(torch.int32))


def test_cta_pair_form_rejects_what_it_does_not_run():
    n, ld = 64, 64
    dev = torch.device("cuda")
    A = sym16(n, ld, 1, "fp16").to(dev)
    C = torch.zeros((2 * n, ld), dtype=torch.float16, device=dev)
    for epi in (b.EPI_CTA_PAIR | b.EPI_GROUPED, b.EPI_CTA_PAIR | 2 | b.EPI_F16_PAIR_OUT):
        with pytest.raises(RuntimeError):
            b.psd_symm_product(n, A, A, ld, C, 0, "fp16", epi, (1.0,))


@pytest.mark.parametrize("n", [16, 97, 255, 300, 513, 1000])
@pytest.mark.parametrize("epi", [0, 1, 2])
def test_cta_pair_form_of_the_split_product_gives_the_same_bits(n, epi):
    # The mixed precision's products of FP16 pairs (A_hi B_hi + A_hi B_lo +
    # A_lo B_hi) on SM pairs and on one SM: the same three tensor products in
    # the same K order per element, so the same output pair, bit for bit.
    ld = (n + 7) // 8 * 8
    rng = np.random.default_rng(70 + n)
    G = rng.standard_normal((n, n)) / np.sqrt(n)
    A = split_pair(0.5 * (G + G.T), "mixed", n, ld)
    G = rng.standard_normal((n, n)) / np.sqrt(n)
    B = split_pair(0.5 * (G + G.T), "mixed", n, ld)
    dev = torch.device("cuda")
    Ad, Bd = A.to(dev), B.to(dev)
    params = {0: (), 1: (1.5, -0.7, 0.3), 2: (1.0 / 1.01,)}[epi]
    outs = []
    for form in (0, b.EPI_CTA_PAIR):
        Cd = torch.full_like(Ad, float("nan"))
        if epi == 1:
            b.psd_symm_product(n, Ad, Ad, ld, Cd, 0, "mixed", 1 | form, params=params, aux=Ad, ld_aux=ld)
        else:
            b.psd_symm_product(n, Ad, Bd, ld, Cd, 0, "mixed", epi | form, params=params)
        torch.cuda.synchronize()
        outs.append(Cd.cpu())
    assert torch.isfinite(outs[0][:, :, :n]).all()
    assert torch.equal(outs[0].view(torch.int16), outs[1].view(torch.int16))
