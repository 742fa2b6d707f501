"""Seeded synthetic inputs for the PSD-cone projection (numpy only).

The paper measures on Matrix Depot matrices and Mittelmann SDP instances,
which are not available here; these generators stand in for them with the
structures the paper discusses (dense symmetric matrices with a spread
spectrum, a few dominant eigenvalues over a bulk, clustered spectra near 0,
block-diagonal cones, and the iterates of the ADMM solver of Sec. 4.2).

This module holds none of the projection's arithmetic.  It is the one module
both the CUDA path's callers and the oracle's callers use: every matrix is
produced in FP64 from numpy's PCG64 stream for ``seed`` and rounded once to
FP32, so both sides see identical FP32 bits.
"""
import math

import numpy as np


def _rng(seed):
    return np.random.default_rng(np.random.PCG64(int(seed)))


def to_f32(X):
    """Round to FP32 (round-to-nearest-even) and symmetrise exactly."""
    X = np.asarray(X, dtype=np.float64)
    X = 0.5 * (X + X.T)
    return np.ascontiguousarray(X.astype(np.float32))


def gaussian_symmetric(n, seed):
    """X = (G + G^T) / 2, G iid N(0, 1)  (n = 256 single-matrix workload)."""
    G = _rng(seed).standard_normal((n, n))
    return to_f32(0.5 * (G + G.T))


def wigner(n, seed):
    """Wigner matrix (G + G^T) / (2 sqrt(n)): semicircle spectrum on [-sqrt2, sqrt2]."""
    G = _rng(seed).standard_normal((n, n))
    G += G.T
    G *= 0.5 / math.sqrt(n)
    return to_f32(G)


def haar_orthogonal(n, seed):
    """Haar-random orthogonal Q: QR of a Gaussian matrix with diag(R) > 0."""
    G = _rng(seed).standard_normal((n, n))
    Q, R = np.linalg.qr(G)
    d = np.sign(np.diag(R))
    d[d == 0] = 1.0
    return Q * d[None, :]


def lowrank_plus_noise(n, seed, rank=50, noise=1e-2):
    """Rank-`rank` PSD + rank-`rank` NSD + noise * (G + G^T) / 2.

    U = first 2*rank columns of the Q factor of a Gaussian n x 2rank matrix;
    the 2*rank magnitudes are uniform in [1, 10]; the first half enter with +,
    the second with -.  The noise bulk has radius about noise * sqrt(2 n).
    """
    rng = _rng(seed)
    k = 2 * rank
    U, _ = np.linalg.qr(rng.standard_normal((n, k)))
    s = rng.uniform(1.0, 10.0, size=k)
    s[rank:] *= -1.0
    G = rng.standard_normal((n, n))
    X = (U * s[None, :]) @ U.T + noise * 0.5 * (G + G.T)
    return to_f32(X)


def spectrum(kind, n, seed):
    """Eigenvalue sets for the spectrum-controlled workload (sorted ascending).

    "uniform":   iid uniform on [-1, 1];
    "clustered": l_1 = 1, l_2 = -1 (they fix the scale), the other n-2 iid
                 uniform in [-1e-3, 1e-3];
    "powerlaw":  |l_i| = i^-1.5 (i = 1..n), random signs, so max |l| = 1;
    "semicircle": iid from the semicircle law on [-sqrt2, sqrt2] (the
                 eigenvalue law of a large Wigner matrix).
    """
    rng = _rng(seed)
    if kind == "uniform":
        lam = rng.uniform(-1.0, 1.0, size=n)
    elif kind == "clustered":
        lam = rng.uniform(-1e-3, 1e-3, size=n)
        if n >= 1:
            lam[0] = 1.0
        if n >= 2:
            lam[1] = -1.0
    elif kind == "powerlaw":
        mag = np.arange(1, n + 1, dtype=np.float64) ** -1.5
        sign = np.where(rng.uniform(size=n) < 0.5, -1.0, 1.0)
        lam = mag * sign
    elif kind == "semicircle":
        # rejection sampling of the density (2 / (pi R^2)) sqrt(R^2 - x^2), R = sqrt 2
        R = math.sqrt(2.0)
        out = []
        while len(out) < n:
            x = rng.uniform(-R, R, size=2 * n)
            y = rng.uniform(0.0, 1.0, size=2 * n)
            keep = x[y * R <= np.sqrt(R * R - x * x)]
            out.extend(keep.tolist())
        lam = np.array(out[:n])
    else:
        raise ValueError(kind)
    return np.sort(lam)


def spectral_matrix(kind, n, seed):
    """X = Q diag(l) Q^T with Haar Q (seed) and spectrum(kind, n, seed + 1).

    Returns (X32, Q, lam): the FP32 input and the FP64 factors it was built
    from.  Pi(X64) and F(X64) are known in closed form from (Q, lam); the FP32
    rounding moves them by at most the Lipschitz constant of the scalar map
    times ||X32 - X64||_F.
    """
    Q = haar_orthogonal(n, seed)
    lam = spectrum(kind, n, seed + 1)
    X = (Q * lam[None, :]) @ Q.T
    return to_f32(X), Q, lam


def spectral_matrix_device(kind, n, seed, device):
    """X = Q diag(l) Q^T built on a CUDA device (for orders where the CPU QR is
    slow): Q Haar from the QR of a Gaussian drawn by torch's generator seeded
    with `seed` on `device` (diag R > 0), l = spectrum(kind, n, seed + 1).

    Returns (X32, Q, lam) as device tensors: the FP32 input (exactly
    symmetric) and the FP64 factors.  The bits differ from spectral_matrix's
    (another random stream); the spectrum is the same.
    """
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    G = torch.randn(n, n, generator=g, dtype=torch.float64, device=device)
    Q, R = torch.linalg.qr(G)
    del G
    Q *= torch.sign(torch.diagonal(R))[None, :]
    del R
    lam = torch.from_numpy(spectrum(kind, n, seed + 1)).to(device)
    X = (Q * lam[None, :]) @ Q.T
    X = 0.5 * (X + X.T)
    return X.float().contiguous(), Q, lam


def block_sizes(count=512, seed=7, lo=16, hi=1024):
    """Block orders n_i = round(exp(U[ln lo, ln hi])) for a block-diagonal cone."""
    u = _rng(seed).uniform(math.log(lo), math.log(hi), size=count)
    return [int(v) for v in np.clip(np.rint(np.exp(u)), lo, hi)]


def wigner_blocks(count=512, seed=7):
    """Block-diagonal workload: `count` Wigner blocks, block i seeded seed*1000 + i."""
    return [wigner(n, seed * 1000 + i) for i, n in enumerate(block_sizes(count, seed))]


def er_laplacian(n, seed, p=0.01):
    """Laplacian L = D - A of an Erdos-Renyi G(n, p) graph with unit weights (FP64)."""
    rng = _rng(seed)
    U = rng.uniform(size=(n, n)) < p
    A = np.triu(U, 1)
    A = (A | A.T).astype(np.float64)
    return np.diag(A.sum(axis=1)) - A
