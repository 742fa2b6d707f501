"""Rounding model of Algorithm 2's product chain in low-precision storage.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  numpy, FP64 arithmetic
with explicit roundings: every matrix the chain stores (X_0, and per stage
Y = X^2, the stage polynomial P and the next iterate) is rounded to a chosen
storage format exactly where a tensor-core path would store it, and every
product is formed from the stored values as a tensor-core product of them
would (hi/lo pairs: hi*hi + hi*lo + lo*hi, the lo*lo term dropped).  Products
are accumulated in FP64 and rounded to FP32 before the storage rounding, the
accumulator type the paper's half-precision runs use (Sec. 4, FP16 tensor
cores with FP32 accumulation).

It answers one question the paper leaves to the implementer: which storage
formats keep the chain within a given distance of the exact filter output
F(X) (Algorithm 2 in exact arithmetic, computed by ``core.chain_fp64``).  The
stage equations are those of Algorithm 2 and Sec. 3.3-3.4:
    X_0 = X / lam~
    Y   = X_{t-1} X_{t-1}
    P   = a_t I + b_t Y + c_t Y Y
    X_t = X_{t-1} P / s_t
    out = (X + lam~ X_0 X_T) / 2
The model shares no code with the CUDA library.

Storage formats:
  "f64"     no rounding;            "f32"  IEEE binary32, round to nearest even;
  "f16"     IEEE binary16, RN-even; "bf16" bfloat16 (8-bit significand), RN-even;
  "e4m3"    OCP FP8 E4M3 (3 fraction bits, bias 7, max 448, saturating), RN-even,
            of the value times a power-of-two scale;
  "f16x2", "bf16x2"  hi/lo pairs: hi = RN(v), lo = RN(v - hi), value hi + lo.
"""
import numpy as np

from .core import chain_fp64, rel_err

FORMATS = ("f64", "f32", "f16", "bf16", "e4m3", "f16x2", "bf16x2")


def round_f32(x):
    return np.asarray(x, dtype=np.float64).astype(np.float32).astype(np.float64)


def round_f16(x):
    """binary16, RN-even, from an FP32 value (numpy's float32 -> float16 cast rounds to nearest even)."""
    with np.errstate(over="ignore"):
        return np.asarray(x, dtype=np.float64).astype(np.float32).astype(np.float16).astype(np.float64)


def round_bf16(x):
    """bfloat16, RN-even on the FP32 bit pattern: keep the top 16 bits after adding
    0x7FFF plus the lowest kept bit (ties to even).  Non-finite values pass through."""
    f = np.asarray(x, dtype=np.float64).astype(np.float32)
    bits = f.view(np.uint32).astype(np.uint64)
    rounded = ((bits + 0x7FFF + ((bits >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)
    out = rounded.view(np.float32).astype(np.float64)
    bad = ~np.isfinite(f)
    if np.any(bad):
        out = np.where(bad, f.astype(np.float64), out)
    return out


_E4M3_MAX = 448.0


def round_e4m3(x):
    """OCP E4M3: normals 2^-6 .. 448 with 3 fraction bits, subnormals k * 2^-9,
    RN-even, saturating at +-448 (the conversion the tensor-core path uses)."""
    v = np.asarray(x, dtype=np.float64).astype(np.float32).astype(np.float64)
    a = np.abs(v)
    with np.errstate(divide="ignore", invalid="ignore"):
        e = np.floor(np.log2(np.where(a > 0, a, 1.0)))
    e = np.maximum(e, -6.0)           # below 2^-6 the spacing stays 2^-9 (subnormals)
    q = np.exp2(e - 3.0)              # spacing of the binade
    r = np.round(a / q) * q           # numpy rounds halves to even
    r = np.minimum(r, _E4M3_MAX)
    r = np.where(np.isnan(v), np.nan, r)
    return np.copysign(r, v)


_ROUND = {"f64": lambda x: np.asarray(x, dtype=np.float64), "f32": round_f32, "f16": round_f16,
          "bf16": round_bf16}


class Stored:
    """A matrix in a storage format: `parts` are the stored matrices (one, or
    hi and lo), `scale` the power of two an e4m3 matrix is stored times."""

    def __init__(self, parts, scale=1.0):
        self.parts = parts
        self.scale = scale

    def value(self):
        v = self.parts[0] if len(self.parts) == 1 else self.parts[0] + self.parts[1]
        return v / self.scale


def store(v, fmt, scale=1.0):
    """Round the FP32 value v (FP64 array) into format `fmt`."""
    v = round_f32(v)
    if fmt in _ROUND:
        return Stored([_ROUND[fmt](v)])
    if fmt == "e4m3":
        return Stored([round_e4m3(v * scale)], scale)
    if fmt in ("f16x2", "bf16x2"):
        r = _ROUND[fmt[:-2]]
        hi = r(v)
        lo = r(round_f32(v - hi))
        return Stored([hi, lo])
    raise ValueError(fmt)


def product(A, B):
    """FP32-accumulated product of two stored matrices: for pairs the three
    products hi*hi + hi*lo + lo*hi (the lo*lo term is not formed)."""
    a, b = A.parts, B.parts
    acc = a[0] @ b[0]
    if len(b) == 2:
        acc = acc + a[0] @ b[1]
    if len(a) == 2:
        acc = acc + a[1] @ b[0]
    return round_f32(acc / (A.scale * B.scale))


def tensor_products(fa, fb):
    """Tensor-core products one product of formats fa x fb costs."""
    pa, pb = fa.endswith("x2"), fb.endswith("x2")
    return 3 if (pa and pb) else 2 if (pa or pb) else 1


class Plan:
    """Storage formats of one run of the chain.

    x0: format of X_0; per stage t (0-based) y[t], p[t], x[t] (the format of
    X_t, the iterate stage t produces); scales of e4m3 matrices: power of two
    per matrix kind (X_t, Y) and for P a power of two from the stage's
    coefficients (largest |a + b y + c y^2| over y in [0, 1.25]).
    """

    def __init__(self, T, x0, y, p, x, name=""):
        assert len(y) == len(p) == len(x) == T
        self.T, self.x0, self.y, self.p, self.x, self.name = T, x0, list(y), list(p), list(x), name

    @classmethod
    def uniform(cls, T, fmt, name=""):
        return cls(T, fmt, [fmt] * T, [fmt] * T, [fmt] * T, name or fmt)

    def products(self):
        """Tensor-core products of the whole chain (3 per stage, 1 final; pairs cost more)."""
        n = 0
        cur = self.x0
        for t in range(self.T):
            n += tensor_products(cur, cur) + tensor_products(self.y[t], self.y[t])
            n += tensor_products(cur, self.p[t])
            cur = self.x[t]
        return n + tensor_products(self.x0, cur)


E4M3_SCALE_X = 256.0
E4M3_SCALE_Y = 256.0


def _poly_scale(a, b, c):
    ys = [0.0, 1.25] + ([-b / (2 * c)] if c != 0 else [])
    m = max(abs(a + b * y + c * y * y) for y in ys if 0.0 <= y <= 1.25)
    s = 1.0
    while s * 2.0 * m < 400.0:
        s *= 2.0
    while s > 1.0 / 1024 and s * m >= 400.0:
        s *= 0.5
    return s


def chain_rounded(X, lam_tilde, coefs, scales, plan):
    """Algorithm 2 after the bound, with every stored matrix rounded per `plan`.

    Returns (out, X_T value, finite): out = (X + lam~ X_0 X_T) / 2 with the
    final product accumulated in FP32 and X added in FP32.
    """
    X = np.asarray(X, dtype=np.float64)
    n = X.shape[0]
    I = np.eye(n)
    X0 = store(X * (1.0 / lam_tilde), plan.x0, E4M3_SCALE_X)
    cur = X0
    with np.errstate(over="ignore", invalid="ignore"):
        for t, ((a, b, c), s) in enumerate(zip(coefs, scales)):
            Y = store(product(cur, cur), plan.y[t], E4M3_SCALE_Y)
            YY = product(Y, Y)
            P = store(a * I + b * Y.value() + c * YY, plan.p[t], _poly_scale(a, b, c))
            cur = store(product(cur, P) * (1.0 / s), plan.x[t], E4M3_SCALE_X)
            if not np.all(np.isfinite(cur.value())):
                return np.full_like(X, np.nan), cur.value(), False
        XT = cur.value()
        out = round_f32(0.5 * (X + lam_tilde * product(X0, cur)))
    return out, XT, bool(np.all(np.isfinite(out)))


def chain_error(X, lam_tilde, coefs, scales, plan, ref=None):
    """rel_F of the rounded chain against the exact chain (chain_fp64 equals F(X) to
    ~1e-12, pinned in tests/test_oracle_filter.py).  inf when the chain left the
    filter's basin (non-finite iterates, or |X_T| entries beyond 2)."""
    if ref is None:
        ref, _ = chain_fp64(X, lam_tilde, coefs, scales)
    out, XT, finite = chain_rounded(X, lam_tilde, coefs, scales, plan)
    if not finite or np.max(np.abs(XT)) > 2.0:
        return float("inf")
    return rel_err(out, ref, X)


def named_plan(name, T=7):
    """Storage plans of the half-precision chain (T = 7) by precision name:
    "fp16" / "bf16": every matrix in that format (the paper's half-precision
    chain); "mixed": FP16 iterates, P as an FP16 pair in stages 1-4 and Y too
    in stages 2-3; "fp8_late": FP16, with stages 6-7 and their input iterate
    in e4m3 (X_T in FP16)."""
    if name in ("fp16", "bf16"):
        return Plan.uniform(T, {"fp16": "f16", "bf16": "bf16"}[name], name)
    if name == "mixed":
        y = ["f16x2" if 1 <= t <= 2 else "f16" for t in range(T)]
        p = ["f16x2" if t < 4 else "f16" for t in range(T)]
        return Plan(T, "f16", y, p, ["f16"] * T, name)
    if name == "fp8_late":
        y = ["e4m3" if t >= T - 2 else "f16" for t in range(T)]
        x = ["e4m3" if T - 3 <= t < T - 1 else "f16" for t in range(T)]
        return Plan(T, "f16", y, list(y), x, name)
    raise ValueError(name)
