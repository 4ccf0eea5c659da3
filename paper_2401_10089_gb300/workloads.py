"""Seeded synthetic inputs for the matrix-logarithm workloads.

This module holds no arithmetic of the method: it only draws matrices. It is
the one module that both the CUDA path's tests/benchmarks and the CPU oracle's
tests take inputs from. The paper's own test sets (Sec. 7, matrix sets 1-3)
are not available, so these seeded families stand in for them:

* ``dense_32``        -- one 32x32 A = Q diag(lam) Q^T + 0.1 N / sqrt(32), Q from
                         the QR of a Gaussian matrix, lam log-uniform in [0.1, 10].
* ``identity_plus``   -- a batch of A = I + E, E Gaussian rescaled so that
                         ||E||_1 is uniform in [0.2, 5].
* ``triangular_similar`` -- A = Q T Q^T with T upper triangular, diag(T)
                         log-uniform in [1e-2, 1e2] and Gaussian off-diagonal
                         entries of standard deviation ``offdiag_std``
                         (0.1 literally, 0.1/n for the well-conditioned variant).
* ``spd``             -- A = Q diag(lam) Q^T with lam log-uniform in a range.
* ``ragged_spd``      -- many SPD matrices with n drawn from a size set
                         (``ragged_spd_device``: the same recipe drawn on a
                         torch device).
"""
from __future__ import annotations

import numpy as np


def _orthogonal(rng: np.random.Generator, n: int, count: int | None = None) -> np.ndarray:
    if count is None:
        q, r = np.linalg.qr(rng.standard_normal((n, n)))
        return q * np.sign(np.diag(r))[None, :]
    g = rng.standard_normal((count, n, n))
    q, r = np.linalg.qr(g)
    d = np.sign(np.diagonal(r, axis1=1, axis2=2))
    return q * d[:, None, :]


def _log_uniform(rng, lo, hi, size):
    return np.exp(rng.uniform(np.log(lo), np.log(hi), size))


def dense_32(seed: int = 0, n: int = 32) -> np.ndarray:
    rng = np.random.default_rng(seed)
    q = _orthogonal(rng, n)
    lam = _log_uniform(rng, 0.1, 10.0, n)
    return q @ np.diag(lam) @ q.T + 0.1 * rng.standard_normal((n, n)) / np.sqrt(n)


def identity_plus(count: int, n: int, seed: int = 1, lo: float = 0.2, hi: float = 5.0) -> np.ndarray:
    rng = np.random.default_rng(seed)
    e = rng.standard_normal((count, n, n))
    target = rng.uniform(lo, hi, count)
    cur = np.abs(e).sum(axis=1).max(axis=1)
    e *= (target / cur)[:, None, None]
    return e + np.eye(n)[None]


def triangular_similar(n: int, seed: int = 2, offdiag_std: float | None = None) -> np.ndarray:
    """A = Q T Q^T; ``offdiag_std`` defaults to the well-conditioned 0.1/n."""
    rng = np.random.default_rng(seed)
    std = 0.1 / n if offdiag_std is None else offdiag_std
    t = np.triu(rng.standard_normal((n, n)) * std, 1)
    t[np.diag_indices(n)] = _log_uniform(rng, 1e-2, 1e2, n)
    q = _orthogonal(rng, n)
    return q @ t @ q.T


def spd(count: int, n: int, seed: int = 3, lo: float = 1e-2, hi: float = 1e2) -> np.ndarray:
    rng = np.random.default_rng(seed)
    q = _orthogonal(rng, n, count)
    lam = _log_uniform(rng, lo, hi, (count, n))
    a = (q * lam[:, None, :]) @ np.swapaxes(q, 1, 2)
    return 0.5 * (a + np.swapaxes(a, 1, 2))


def ragged_sizes(count: int, sizes=(4, 8, 16, 32, 64, 128, 256), seed: int = 4) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return np.asarray(sizes, dtype=np.int32)[rng.integers(0, len(sizes), count)]


def ragged_spd(count: int, sizes=(4, 8, 16, 32, 64, 128, 256), seed: int = 4,
               lo: float = 1e-3, hi: float = 1e3, dtype=np.float32):
    """(packed values, n per matrix, element offset per matrix)."""
    ns = ragged_sizes(count, sizes, seed)
    offs = np.zeros(count, dtype=np.int64)
    offs[1:] = np.cumsum(ns.astype(np.int64) ** 2)[:-1]
    total = int((ns.astype(np.int64) ** 2).sum())
    out = np.empty(total, dtype=dtype)
    rng = np.random.default_rng(seed + 1000)
    for n in np.unique(ns):
        idx = np.nonzero(ns == n)[0]
        mats = spd(len(idx), int(n), seed=int(rng.integers(1 << 31)), lo=lo, hi=hi)
        for j, b in enumerate(idx):
            out[offs[b]:offs[b] + n * n] = mats[j].ravel()
    return out, ns, offs


def ragged_spd_device(count: int, device, sizes=(4, 8, 16, 32, 64, 128, 256), seed: int = 4,
                      lo: float = 1e-3, hi: float = 1e3):
    """The ``ragged_spd`` recipe drawn on a torch device (for the 20,000-matrix
    batch, whose host generation takes half a minute): n per matrix from
    ``ragged_sizes``, A = Q diag(lam) Q^T with Q from the QR of a seeded
    Gaussian matrix and lam log-uniform in [lo, hi], FP32 storage. Returns
    (packed values, n per matrix, element offsets) as device tensors. The
    matrices differ from ``ragged_spd``'s (another generator), the recipe is
    the same."""
    import torch
    ns = ragged_sizes(count, sizes, seed)
    offs = np.zeros(count, dtype=np.int64)
    offs[1:] = np.cumsum(ns.astype(np.int64) ** 2)[:-1]
    total = int((ns.astype(np.int64) ** 2).sum())
    out = torch.empty(total, dtype=torch.float32, device=device)
    gen = torch.Generator(device=device)
    gen.manual_seed(seed + 1000)
    offs_d = torch.from_numpy(offs).to(device)
    for n in np.unique(ns):
        n = int(n)
        idx = np.nonzero(ns == n)[0]
        g = torch.randn((len(idx), n, n), generator=gen, device=device, dtype=torch.float64)
        q, r = torch.linalg.qr(g)
        q = q * torch.sign(torch.diagonal(r, dim1=1, dim2=2))[:, None, :]
        u = torch.rand((len(idx), n), generator=gen, device=device, dtype=torch.float64)
        lam = torch.exp(np.log(lo) + (np.log(hi) - np.log(lo)) * u)
        a = (q * lam[:, None, :]) @ q.transpose(1, 2)
        a = (0.5 * (a + a.transpose(1, 2))).to(torch.float32).reshape(len(idx), n * n)
        pos = offs_d[torch.from_numpy(idx).to(device)][:, None] + torch.arange(n * n, device=device)[None, :]
        out[pos.reshape(-1)] = a.reshape(-1)
    return out, torch.from_numpy(ns).to(device), offs_d


def gaussian(shape, seed: int = 5) -> np.ndarray:
    return np.random.default_rng(seed).standard_normal(shape)


def diag_from_eigs(lam, seed: int = 6) -> np.ndarray:
    """V diag(lam) V^{-1} with a seeded, well-conditioned V (returns A, V)."""
    lam = np.asarray(lam, dtype=np.float64)
    n = lam.shape[0]
    rng = np.random.default_rng(seed)
    v = np.eye(n) + 0.3 * rng.standard_normal((n, n)) / np.sqrt(n)
    return v @ np.diag(lam) @ np.linalg.inv(v), v
