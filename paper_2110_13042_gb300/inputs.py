"""Seeded synthetic inputs for low(A^T A) -- shared by the tests, the oracle
checks and the benchmark.  Holds none of the method's arithmetic.

Every value is a pure function of (seed, element index): a counter-based
splitmix64 stream (Steele, Lea & Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014: the 64-bit finaliser with increments of the golden
gamma 0x9E3779B97F4A7C15).  Element (i, j) of an m x n matrix uses counter
i * n + j, so any subset of columns can be regenerated without the rest (the
sampled-tile checks of very large inputs rely on this).

Recipes (the paper tests on randomly generated dense square and tall matrices,
Section 5.1; the shapes and distributions below are those of the workloads the
library is measured on):

* ``uniform(m, n, seed)``            i.i.d. U[-1, 1)
* ``integer_valued(m, n, seed, lo, hi)`` i.i.d. integers in [lo, hi] (exact in
                                     every precision the library offers)
* ``column_scaled_normal(m, n, seed)`` N(0,1) entries, each column scaled by
                                     10^U(-3,3)  (precision stress)
* ``low_rank_stressed(m, n, seed)``  U[-1,1) + 1e4 * (G1 G2^T)/4, G1 m x 16,
                                     G2 n x 16 i.i.d. N(0,1)  (cancellation)
* ``batch_shapes(count, seed)``      m ~ log-uniform[64, 4096],
                                     n ~ log-uniform[32, 1024]
* ``hadamard(m, n)``                 first n columns of the Sylvester-Hadamard
                                     matrix of order m = 4^k scaled by 2^-k
                                     (orthonormal columns, dyadic entries)
"""
from __future__ import annotations

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_S30, _S27, _S31, _S11 = (np.uint64(s) for s in (30, 27, 31, 11))
_TWO_M53 = 2.0 ** -53


def _mix64(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> _S30)) * _M1
    z = (z ^ (z >> _S27)) * _M2
    return z ^ (z >> _S31)


def _key(seed: int, stream: int = 0) -> np.uint64:
    with np.errstate(over="ignore"):
        s = np.array([(seed * 0x9E3779B97F4A7C15 + stream * 0xD1B54A32D192ED03
                       + 0x632BE59BD9B4E019) % (1 << 64)], dtype=np.uint64)
        return _mix64(s)[0]


def u64(seed: int, idx: np.ndarray, stream: int = 0) -> np.ndarray:
    """Raw 64-bit outputs for counters ``idx`` (uint64 array)."""
    idx = np.asarray(idx, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return _mix64(_key(seed, stream) + (idx + np.uint64(1)) * _GAMMA)


def unit(seed: int, idx: np.ndarray, stream: int = 0) -> np.ndarray:
    """Uniform doubles in [0, 1) with 53 random bits."""
    return (u64(seed, idx, stream) >> _S11).astype(np.float64) * _TWO_M53


def _grid(m: int, n: int, cols=None) -> np.ndarray:
    cols = np.arange(n, dtype=np.uint64) if cols is None else np.asarray(cols, np.uint64)
    rows = np.arange(m, dtype=np.uint64)
    return rows[:, None] * np.uint64(n) + cols[None, :]


def uniform(m: int, n: int, seed: int, cols=None, dtype=np.float64,
            block_rows: int = 4096) -> np.ndarray:
    """i.i.d. U[-1, 1) entries; ``cols`` selects a subset of columns (the
    values equal those of the same columns of the full matrix)."""
    ncols = n if cols is None else len(cols)
    out = np.empty((m, ncols), dtype=dtype)
    for r0 in range(0, m, block_rows):
        r1 = min(m, r0 + block_rows)
        idx = _grid(r1 - r0, n, cols) + np.uint64(r0 * n)
        out[r0:r1] = 2.0 * unit(seed, idx) - 1.0
    return out


def integer_valued(m: int, n: int, seed: int, lo: int = -8, hi: int = 8,
                   dtype=np.float64) -> np.ndarray:
    """i.i.d. integers uniform in [lo, hi]."""
    idx = _grid(m, n)
    v = np.floor(unit(seed, idx) * (hi - lo + 1)) + lo
    return v.astype(dtype)


def normal(m: int, n: int, seed: int, cols=None, stream: int = 1) -> np.ndarray:
    """i.i.d. N(0,1) by Box-Muller on two counter-based uniforms."""
    idx = _grid(m, n, cols)
    u1 = 1.0 - unit(seed, idx * np.uint64(2), stream)          # (0, 1]
    u2 = unit(seed, idx * np.uint64(2) + np.uint64(1), stream)  # [0, 1)
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)


def column_scaled_normal(m: int, n: int, seed: int, cols=None) -> np.ndarray:
    """N(0,1) entries with column j scaled by 10^{U(-3,3)} (one factor per
    column, drawn from stream 2 with counter j)."""
    cols_idx = np.arange(n, dtype=np.uint64) if cols is None else np.asarray(cols, np.uint64)
    expo = 6.0 * unit(seed, cols_idx, stream=2) - 3.0
    return normal(m, n, seed, cols) * (10.0 ** expo)[None, :]


def low_rank_stressed(m: int, n: int, seed: int, rank: int = 16,
                      magnitude: float = 1e4, cols=None) -> np.ndarray:
    """U[-1,1) + magnitude * (G1 @ G2^T) / 4 with G1 (m x rank), G2 (n x rank)
    i.i.d. N(0,1) (streams 3 and 4)."""
    G1 = normal(m, rank, seed, stream=3)
    G2 = normal(n, rank, seed, stream=4)
    if cols is not None:
        G2 = G2[np.asarray(cols)]
    return uniform(m, n, seed, cols) + magnitude * (G1 @ G2.T) / 4.0


def batch_shapes(count: int, seed: int, m_range=(64, 4096), n_range=(32, 1024)):
    """Shapes (m_i, n_i) with log-uniform m and n (streams 5 and 6)."""
    i = np.arange(count, dtype=np.uint64)
    lm = np.log(m_range[0]) + unit(seed, i, 5) * (np.log(m_range[1]) - np.log(m_range[0]))
    ln = np.log(n_range[0]) + unit(seed, i, 6) * (np.log(n_range[1]) - np.log(n_range[0]))
    ms = np.clip(np.rint(np.exp(lm)), m_range[0], m_range[1]).astype(np.int64)
    ns = np.clip(np.rint(np.exp(ln)), n_range[0], n_range[1]).astype(np.int64)
    return ms, ns


def hadamard(m: int, n: int) -> np.ndarray:
    """First n columns of the order-m Sylvester-Hadamard matrix, m = 4^k,
    scaled by 2^-k so the columns are orthonormal (every entry is +-2^-k)."""
    k = 0
    while 4 ** k < m:
        k += 1
    if 4 ** k != m or n > m:
        raise ValueError("hadamard: m must be a power of 4 and n <= m")
    H = np.array([[1.0]])
    while H.shape[0] < m:
        H = np.block([[H, H], [H, -H]])
    return H[:, :n] * 2.0 ** (-k)


# ------------------------------------------------------------ on-device --
# Inputs of several GB are drawn on the GPU from torch's seeded Philox
# generator (same distributions as above, different streams): the parity
# tests pull the sampled columns back from the device copy, so the oracle
# sees exactly the values the library saw.

def _torch_gen(seed: int, device):
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    return g


def device_uniform(m: int, n: int, seed: int, device, dtype=None):
    """i.i.d. U[-1, 1) entries on ``device``."""
    import torch
    g = _torch_gen(seed, device)
    return torch.rand((m, n), generator=g, device=device, dtype=dtype or torch.float64) * 2 - 1


def device_column_scaled_normal(m: int, n: int, seed: int, device, dtype=None):
    """N(0,1) entries with column j scaled by 10^U(-3,3), on ``device``."""
    import torch
    dt = dtype or torch.float64
    g = _torch_gen(seed, device)
    scale = 10.0 ** (torch.rand(n, generator=g, device=device, dtype=torch.float64) * 6 - 3)
    A = torch.randn((m, n), generator=g, device=device, dtype=torch.float64)
    A.mul_(scale[None, :])
    return A.to(dt)


def device_low_rank_stressed(m: int, n: int, seed: int, device, rank: int = 16, magnitude: float = 1e4,
                             dtype=None):
    """U[-1,1) + magnitude * (G1 G2^T) / 4 with G1 (m x rank), G2 (n x rank)
    i.i.d. N(0,1), on ``device``."""
    import torch
    g = _torch_gen(seed, device)
    A = torch.rand((m, n), generator=g, device=device, dtype=torch.float64) * 2 - 1
    G1 = torch.randn((m, rank), generator=g, device=device, dtype=torch.float64)
    G2 = torch.randn((n, rank), generator=g, device=device, dtype=torch.float64)
    A.addmm_(G1, G2.T, alpha=magnitude / 4.0)
    return A.to(dtype or torch.float64)
