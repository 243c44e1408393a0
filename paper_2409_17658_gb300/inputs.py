"""Seeded synthetic operands, shared by the tests, the benchmark and the oracle checks.

Holds no arithmetic of the method: it only draws int16 matrices in the
library's encoding (0x3FFF = infinity).  The generator is SplitMix64 (Steele,
Lea and Flood, 2014) used as a counter-based stream: entry e of a matrix drawn
with seed s is mix(s * 2^32 + e), so any entry can be regenerated alone and
the result does not depend on chunking.

Distributions:
  "u32"   value uniform in [0, 32], replaced by infinity with probability 1/2
          (the synthetic (min,+) GEMM workload);
  "wide"  value uniform in [0, 0x1FFF], infinity with probability 1/2;
  "dense" value uniform in [0, 0x1FFF], never infinity.
"""
from __future__ import annotations

import numpy as np

INF16 = 0x3FFF
_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(counter: np.ndarray) -> np.ndarray:
    """Output function of SplitMix64 at state (counter + 1) * golden gamma."""
    with np.errstate(over="ignore"):
        z = (counter.astype(np.uint64) + np.uint64(1)) * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def _values(x: np.ndarray, dist: str) -> np.ndarray:
    lo = x & np.uint64(0xFFFFFFFF)
    if dist == "u32":
        v = (lo * np.uint64(33)) >> np.uint64(32)
        inf = (x >> np.uint64(63)) == 1
    elif dist == "wide":
        v = (lo * np.uint64(0x2000)) >> np.uint64(32)
        inf = (x >> np.uint64(63)) == 1
    elif dist == "dense":
        v = (lo * np.uint64(0x2000)) >> np.uint64(32)
        inf = np.zeros(x.shape, dtype=bool)
    else:
        raise ValueError(dist)
    return np.where(inf, INF16, v).astype(np.int16)


def matrix(rows: int, cols: int, seed: int, dist: str = "u32", ld: int | None = None,
           chunk_rows: int = 1024) -> np.ndarray:
    """A rows x ld int16 matrix; columns >= cols (padding) are infinity."""
    ld = cols if ld is None else ld
    out = np.full((rows, ld), INF16, dtype=np.int16)
    base = np.uint64(seed) << np.uint64(32)
    for r0 in range(0, rows, chunk_rows):
        r1 = min(rows, r0 + chunk_rows)
        idx = (np.arange(r0, r1, dtype=np.uint64)[:, None] * np.uint64(cols)
               + np.arange(cols, dtype=np.uint64)[None, :])
        out[r0:r1, :cols] = _values(splitmix64(base + idx), dist)
    return out


def entries(rows_idx, cols_idx, cols: int, seed: int, dist: str = "u32") -> np.ndarray:
    """Selected entries of matrix(..., cols, seed, dist) without drawing the rest."""
    idx = np.asarray(rows_idx, dtype=np.uint64) * np.uint64(cols) + np.asarray(cols_idx, dtype=np.uint64)
    return _values(splitmix64((np.uint64(seed) << np.uint64(32)) + idx), dist)


def rows_of(row_idx, cols: int, seed: int, dist: str = "u32") -> np.ndarray:
    """Whole rows of matrix(..., cols, seed, dist)."""
    r = np.asarray(row_idx, dtype=np.uint64)[:, None]
    idx = r * np.uint64(cols) + np.arange(cols, dtype=np.uint64)[None, :]
    return _values(splitmix64((np.uint64(seed) << np.uint64(32)) + idx), dist)


def cols_of(col_idx, rows: int, cols: int, seed: int, dist: str = "u32") -> np.ndarray:
    """Whole columns of matrix(rows, cols, seed, dist), shape (rows, len(col_idx))."""
    c = np.asarray(col_idx, dtype=np.uint64)[None, :]
    idx = np.arange(rows, dtype=np.uint64)[:, None] * np.uint64(cols) + c
    return _values(splitmix64((np.uint64(seed) << np.uint64(32)) + idx), dist)


# ---------------------------------------------------------------- the same stream with torch (CPU or CUDA)

def _s64(u: int) -> int:
    return u - (1 << 64) if u >= (1 << 63) else u


def _srl(z, s: int):
    """Logical right shift of an int64 tensor holding uint64 bits."""
    return (z >> s) & ((1 << (64 - s)) - 1)


def splitmix64_torch(counter):
    """splitmix64() on an int64 torch tensor (uint64 bits, wrapping arithmetic)."""
    z = (counter + 1) * _s64(0x9E3779B97F4A7C15)
    z = (z ^ _srl(z, 30)) * _s64(0xBF58476D1CE4E5B9)
    z = (z ^ _srl(z, 27)) * _s64(0x94D049BB133111EB)
    return z ^ _srl(z, 31)


def _values_torch(x, dist: str):
    import torch

    lo = x & 0xFFFFFFFF
    if dist == "u32":
        v = (lo * 33) >> 32
        inf = x < 0
    elif dist == "wide":
        v = (lo * 0x2000) >> 32
        inf = x < 0
    elif dist == "dense":
        v = (lo * 0x2000) >> 32
        inf = torch.zeros_like(x, dtype=torch.bool)
    else:
        raise ValueError(dist)
    return torch.where(inf, torch.full_like(v, INF16), v).to(torch.int16)


def matrix_torch(rows: int, cols: int, seed: int, dist: str = "u32", ld: int | None = None, device="cpu",
                 chunk_rows: int = 2048):
    """Same values as matrix(), drawn with torch on `device` (a rows x ld int16 tensor)."""
    import torch

    ld = cols if ld is None else ld
    out = torch.full((rows, ld), INF16, dtype=torch.int16, device=device)
    base = seed << 32
    col = torch.arange(cols, dtype=torch.int64, device=device)[None, :]
    for r0 in range(0, rows, chunk_rows):
        r1 = min(rows, r0 + chunk_rows)
        idx = torch.arange(r0, r1, dtype=torch.int64, device=device)[:, None] * cols + col
        out[r0:r1, :cols] = _values_torch(splitmix64_torch(idx + base), dist)
    return out


def log_uniform_sizes(count: int, lo: int, hi: int, seed: int) -> list[int]:
    """count sizes round(exp(U[ln lo, ln hi])) from the same counter-based stream."""
    x = splitmix64((np.uint64(seed) << np.uint64(32)) + np.arange(count, dtype=np.uint64))
    u = (x >> np.uint64(11)).astype(np.float64) / float(1 << 53)
    return [int(round(np.exp(np.log(lo) + ui * (np.log(hi) - np.log(lo))))) for ui in u]
