"""Plain CPU oracle for the (min,+) transfer-matrix method of arXiv 2409.17658.

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only permitted users.  The library's
product path never imports this package.

The arithmetic lives in ``rd_oracle.c`` (plain C, int64, no normalisation);
this module only compiles it with gcc and marshals numpy arrays through ctypes.
Every function cites the paper passage it restates in the C source.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rd_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "librdoracle.so")

INF = 0x3FFFFFFFFFFFFFFF  # the oracle's own infinity for int64 matrices
I16_INF = 0x3FFF  # the library interface's int16 encoding of infinity

_lib = None
_lock = threading.Lock()


def build(force: bool = False) -> str:
    """Compile rd_oracle.c into a shared library with gcc (OpenMP over output rows)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.run(["gcc", "-O2", "-std=c11", "-fopenmp", "-shared", "-fPIC", "-o", tmp, _SRC], check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            i64, i32, u32, vp = ctypes.c_int64, ctypes.c_int32, ctypes.c_uint32, ctypes.c_void_p
            lib.rdo_threads.restype = ctypes.c_int
            lib.rdo_num_words.argtypes = [ctypes.c_int]
            lib.rdo_num_words.restype = i64
            lib.rdo_words.argtypes = [ctypes.c_int, vp, vp, i64]
            lib.rdo_words.restype = i64
            lib.rdo_follows.argtypes = [ctypes.c_int, u32, u32]
            lib.rdo_follows.restype = ctypes.c_int
            lib.rdo_transfer.argtypes = [ctypes.c_int, vp, i64]
            lib.rdo_transfer.restype = ctypes.c_int
            lib.rdo_minplus.argtypes = [vp, vp, vp, i64, i64, i64]
            lib.rdo_minplus.restype = None
            lib.rdo_minplus_i16.argtypes = [vp, i64, vp, i64, vp, i64, i64, i64, i64]
            lib.rdo_minplus_i16.restype = None
            lib.rdo_minplus_i16_entries.argtypes = [vp, i64, vp, i64, i64, vp, vp, i64, vp]
            lib.rdo_minplus_i16_entries.restype = None
            lib.rdo_power_step.argtypes = [vp, vp, i64, vp]
            lib.rdo_power_step.restype = ctypes.c_int
            lib.rdo_power_until_periodic.argtypes = [ctypes.c_int, vp, i64, ctypes.c_int, vp, vp, vp, vp, vp]
            lib.rdo_power_until_periodic.restype = ctypes.c_int
            lib.rdo_power_rows.argtypes = [ctypes.c_int, vp, ctypes.c_int, ctypes.c_int, vp]
            lib.rdo_power_rows.restype = ctypes.c_int
            lib.rdo_power_until_periodic_rows.argtypes = [ctypes.c_int, ctypes.c_int, vp, vp, vp, vp, vp]
            lib.rdo_power_until_periodic_rows.restype = ctypes.c_int
            lib.rdo_brute_force.argtypes = [ctypes.c_int, ctypes.c_int]
            lib.rdo_brute_force.restype = i64
            lib.rdo_row_dp.argtypes = [ctypes.c_int, ctypes.c_int]
            lib.rdo_row_dp.restype = i64
            lib.rdo_gamma_direct.argtypes = [ctypes.c_int, ctypes.c_int, vp]
            lib.rdo_gamma_direct.restype = ctypes.c_int
            lib.rdo_follows_loss.argtypes = [ctypes.c_int, u32, u32]
            lib.rdo_follows_loss.restype = ctypes.c_int
            lib.rdo_nd.argtypes = [ctypes.c_int, u32, u32]
            lib.rdo_nd.restype = ctypes.c_int
            lib.rdo_transfer_loss.argtypes = [ctypes.c_int, vp, i64]
            lib.rdo_transfer_loss.restype = ctypes.c_int
            lib.rdo_brute_force_loss.argtypes = [ctypes.c_int, ctypes.c_int]
            lib.rdo_brute_force_loss.restype = i64
            lib.rdo_transfer_rows.argtypes = [ctypes.c_int, vp, ctypes.c_int, vp]
            lib.rdo_transfer_rows.restype = ctypes.c_int
            _ = i32
            _lib = lib
    return _lib


def _ptr(a: np.ndarray) -> int:
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data


def threads() -> int:
    """OpenMP threads the oracle's parallel loops use."""
    return _load().rdo_threads()


def num_words(m: int) -> int:
    """C_m, the number of correct words of length m (Definition 4, Table 1)."""
    n = _load().rdo_num_words(m)
    if n < 0:
        raise ValueError(f"m={m} out of range")
    return n


def words(m: int):
    """Correct words in increasing code order, and their weights 2 p(a) + p(b)."""
    n = num_words(m)
    code = np.zeros(n, dtype=np.uint32)
    wt = np.zeros(n, dtype=np.int32)
    got = _load().rdo_words(m, _ptr(code), _ptr(wt), n)
    assert got == n
    return code, wt


def follows(m: int, q: int, p: int) -> bool:
    """True when word p can follow word q (Sec. 4.A rules)."""
    return bool(_load().rdo_follows(m, q, p))


def transfer(m: int) -> np.ndarray:
    """A(G) of Corollary 6 as an N x N int64 matrix, INF for non-arcs."""
    n = num_words(m)
    a = np.empty((n, n), dtype=np.int64)
    rc = _load().rdo_transfer(m, _ptr(a), n)
    assert rc == 0
    return a


def transfer_rows(m: int, rows) -> np.ndarray:
    """Rows `rows` of A(G), int64 with INF, without building the whole matrix."""
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    out = np.empty((len(rows), num_words(m)), dtype=np.int64)
    assert _load().rdo_transfer_rows(m, _ptr(rows), len(rows), _ptr(out)) == 0
    return out


def minplus(x: np.ndarray, y: np.ndarray) -> np.ndarray:
    """Textbook (min,+) product of int64 matrices with INF (Sec. 3)."""
    x = np.ascontiguousarray(x, dtype=np.int64)
    y = np.ascontiguousarray(y, dtype=np.int64)
    assert x.shape[1] == y.shape[0]
    z = np.empty((x.shape[0], y.shape[1]), dtype=np.int64)
    _load().rdo_minplus(_ptr(x), _ptr(y), _ptr(z), x.shape[0], x.shape[1], y.shape[1])
    return z


def minplus_i16(x: np.ndarray, y: np.ndarray) -> np.ndarray:
    """(min,+) product of int16 operands in the library encoding (0x3FFF = INF); int32 result, INF = 0x3FFF."""
    x = np.ascontiguousarray(x, dtype=np.int16)
    y = np.ascontiguousarray(y, dtype=np.int16)
    rows, inner = x.shape
    inner2, cols = y.shape
    assert inner == inner2
    z = np.empty((rows, cols), dtype=np.int32)
    _load().rdo_minplus_i16(_ptr(x), inner, _ptr(y), cols, _ptr(z), cols, rows, inner, cols)
    return z


def minplus_i16_entries(x: np.ndarray, y: np.ndarray, ri, cj) -> np.ndarray:
    """Entries (ri[e], cj[e]) of the int16-encoded product, each by its own O(K) minimum."""
    x = np.ascontiguousarray(x, dtype=np.int16)
    y = np.ascontiguousarray(y, dtype=np.int16)
    ri = np.ascontiguousarray(ri, dtype=np.int64)
    cj = np.ascontiguousarray(cj, dtype=np.int64)
    out = np.empty(len(ri), dtype=np.int32)
    _load().rdo_minplus_i16_entries(_ptr(x), x.shape[1], _ptr(y), y.shape[1], x.shape[1], _ptr(ri), _ptr(cj),
                                    len(ri), _ptr(out))
    return out


def power_step(x: np.ndarray, a: np.ndarray) -> np.ndarray:
    """X (x) A through the arc lists of A (same value as minplus)."""
    x = np.ascontiguousarray(x, dtype=np.int64)
    a = np.ascontiguousarray(a, dtype=np.int64)
    n = a.shape[0]
    z = np.empty((n, n), dtype=np.int64)
    assert _load().rdo_power_step(_ptr(x), _ptr(a), n, _ptr(z)) == 0
    return z


def power_until_periodic(m: int = 0, a: np.ndarray | None = None, kmax: int = 64) -> dict:
    """Algorithm 2 with the first-repeat rule.

    Returns dict(found, k, p, q, j, gamma) where gamma[k'] = min diag A^k' for
    k' = 1..j (gamma[0] unused) and, when found, A^(k+p) = q (x) A^k.
    """
    if m >= 1:
        a_ptr, n = None, 0
    else:
        a = np.ascontiguousarray(a, dtype=np.int64)
        a_ptr, n = _ptr(a), a.shape[0]
    gamma = np.zeros(kmax + 1, dtype=np.int64)
    k = np.zeros(1, dtype=np.int32)
    p = np.zeros(1, dtype=np.int32)
    q = np.zeros(1, dtype=np.int64)
    j = np.zeros(1, dtype=np.int32)
    rc = _load().rdo_power_until_periodic(m, a_ptr, n, kmax, _ptr(gamma), _ptr(k), _ptr(p), _ptr(q), _ptr(j))
    if rc not in (0, 5):
        raise RuntimeError(f"oracle power_until_periodic failed rc={rc}")
    jj = int(j[0])
    return dict(found=(rc == 0), k=int(k[0]) if rc == 0 else None, p=int(p[0]) if rc == 0 else None,
                q=int(q[0]) if rc == 0 else None, j=jj, gamma=gamma[: jj + 1].copy())


def power_until_periodic_rows(m: int, kmax: int = 40) -> dict:
    """Algorithm 2 with the first-repeat rule, streamed one start word at a time (no dense power kept).

    Same rule and results as power_until_periodic(m); gamma is filled for k = 1..kmax whether or
    not a repeat was found (index 0 unused), and j is the repeat's j (kmax when none).
    """
    gamma = np.zeros(kmax + 1, dtype=np.int64)
    k = np.zeros(1, dtype=np.int32)
    p = np.zeros(1, dtype=np.int32)
    q = np.zeros(1, dtype=np.int64)
    j = np.zeros(1, dtype=np.int32)
    rc = _load().rdo_power_until_periodic_rows(m, kmax, _ptr(gamma), _ptr(k), _ptr(p), _ptr(q), _ptr(j))
    if rc not in (0, 5):
        raise RuntimeError(f"oracle power_until_periodic_rows failed rc={rc}")
    return dict(found=(rc == 0), k=int(k[0]) if rc == 0 else None, p=int(p[0]) if rc == 0 else None,
                q=int(q[0]) if rc == 0 else None, j=int(j[0]), gamma=gamma)


def power_rows(m: int, rows, kmax: int) -> np.ndarray:
    """Rows `rows` of A^1..A^kmax (raw int64, INF): array [kmax, len(rows), N]."""
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    n = num_words(m)
    out = np.empty((kmax, len(rows), n), dtype=np.int64)
    assert _load().rdo_power_rows(m, _ptr(rows), len(rows), kmax, _ptr(out)) == 0
    return out


def brute_force(m: int, n: int) -> int:
    """gamma_R(P_m box C_n) by exhaustive search over f: V -> {0,1,2} (the RDF definition)."""
    r = _load().rdo_brute_force(m, n)
    if r < 0:
        raise ValueError("size out of range")
    return int(r)


def row_dp(m: int, n: int) -> int:
    """gamma_R(P_m box C_n) by dynamic programming along the path (independent of the column words)."""
    r = _load().rdo_row_dp(m, n)
    if r < 0:
        raise ValueError("size out of range")
    return int(r)


def transfer_loss(m: int) -> np.ndarray:
    """The Appendix variant's matrix: labels 10 p(a) + 5 p(b) - 2 nd(q,p) (raw, may be negative), INF off arcs."""
    n = num_words(m)
    a = np.empty((n, n), dtype=np.int64)
    assert _load().rdo_transfer_loss(m, _ptr(a), n) == 0
    return a


def nd(m: int, q: int, p: int) -> int:
    """Algorithm 3: vertices newly dominated by column p after column q."""
    return int(_load().rdo_nd(m, q, p))


def follows_loss(m: int, q: int, p: int) -> bool:
    return bool(_load().rdo_follows_loss(m, q, p))


def brute_force_loss(m: int, n: int) -> int:
    """2 L_a(n) on the m-row strip by exhaustive search over the Appendix's definition (mn <= 20)."""
    r = _load().rdo_brute_force_loss(m, n)
    if r == -(2 ** 63):
        raise ValueError("size out of range")
    return int(r)


def gamma_direct(m: int, nmax: int) -> np.ndarray:
    """Algorithm 1 for n = 1..nmax: gamma[n] = min diag A^n, straight powering (index 0 unused)."""
    g = np.zeros(nmax + 1, dtype=np.int64)
    assert _load().rdo_gamma_direct(m, nmax, _ptr(g)) == 0
    return g


def gamma_from_period(gamma, k: int, p: int, q: int, n: int) -> int:
    """Solution of the finite-difference equation of Prop. 7 from its boundary values."""
    if n < k + p:
        return int(gamma[n])
    t = (n - k) // p
    return int(gamma[k + (n - k) % p]) + q * t
