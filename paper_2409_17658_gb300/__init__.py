"""Python binding of the rd C ABI (include/rd.h): argument marshalling only.

Every step of the computation runs in the CUDA library ``_build/librd.so``;
this module converts torch tensors to pointers, sizes and the current CUDA
stream, and converts status codes to exceptions.  It fails loudly when the
library has not been built -- there is no fallback path.
"""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "librd.so")
HEADER = os.path.join(os.path.dirname(_HERE), "include", "rd.h")

RD_OK, RD_ERR_ARG, RD_ERR_RANGE, RD_ERR_NOMEM, RD_ERR_CUDA, RD_NOT_FOUND, RD_ERR_TIMEOUT = range(7)
STATUS_NAMES = {0: "RD_OK", 1: "RD_ERR_ARG", 2: "RD_ERR_RANGE", 3: "RD_ERR_NOMEM", 4: "RD_ERR_CUDA",
                5: "RD_NOT_FOUND", 6: "RD_ERR_TIMEOUT"}
RD_INF = 0x3FFF
RD_MAX_FINITE = 0x1FFF
RD_MAX_M = 15
RD_GAMMA_UNSET = -(2 ** 63)
RD_GAMMA_INF = 2 ** 63 - 1


class RdError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        msg = f"{where}: {STATUS_NAMES.get(status, status)}"
        if status == RD_ERR_CUDA:
            msg += f" ({_lib().rd_last_cuda_error().decode()})"
        super().__init__(msg)


_LIB = None


def _lib():
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2409_17658_gb300.build.build()")
        _LIB = _configure(ctypes.CDLL(LIB_PATH))
    return _LIB


def use_library(path: str):
    """Route every call of this binding to the library at `path` (for example the checked build,
    build.build(checked=True)); returns the library used before, for restoring with use_library_handle."""
    global _LIB
    prev = _LIB
    _LIB = _configure(ctypes.CDLL(path))
    return prev


def use_library_handle(lib) -> None:
    """Restore a library returned by use_library (None: the default librd.so on next use)."""
    global _LIB
    _LIB = lib


def _configure(lib):
    """Declares the argument and result types of every entry point of a loaded library."""
    i64, i32, vp, sz = ctypes.c_int64, ctypes.c_int32, ctypes.c_void_p, ctypes.c_size_t
    st = ctypes.c_int
    lib.rd_last_cuda_error.restype = ctypes.c_char_p
    lib.rd_last_cuda_error.argtypes = []
    lib.rd_state_count.argtypes = [ctypes.c_int, vp]
    lib.rd_padded_dim.argtypes = [i64, vp]
    lib.rd_enumerate_states.argtypes = [ctypes.c_int, vp, vp, vp]
    lib.rd_build_transfer.argtypes = [ctypes.c_int, vp, i64, vp]
    lib.rd_build_transfer_loss.argtypes = [ctypes.c_int, vp, i64, vp]
    lib.rd_minplus_gemm_batched.argtypes = [vp, ctypes.c_int, vp]
    lib.rd_minplus_gemv.argtypes = [vp, vp, i64, vp, i64, i64, vp, vp]
    lib.rd_power_until_periodic_multi.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, vp]
    lib.rd_power_until_periodic_multi_bounded.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                          ctypes.c_uint32, ctypes.c_int32, vp]
    lib.rd_power_until_periodic_multi_bounded.restype = st
    lib.rd_server_create.argtypes = [sz, ctypes.c_int, vp]
    lib.rd_server_submit.argtypes = [vp, ctypes.c_int, vp, vp, vp]
    lib.rd_server_wait.argtypes = [vp, ctypes.c_int, vp, ctypes.c_double, vp, vp, vp]
    lib.rd_server_stats.argtypes = [vp, vp]
    lib.rd_server_destroy.argtypes = [vp]
    lib.rd_minplus_gemm.argtypes = [vp, i64, vp, i64, vp, i64, i64, i64, i64, vp, vp]
    lib.rd_power_work_bytes.argtypes = [i64, i64, ctypes.c_int, ctypes.c_int, vp]
    lib.rd_power_until_periodic.argtypes = [vp, i64, i64, ctypes.c_int, vp, sz, vp, vp, vp, vp, vp]
    lib.rd_gamma_R.argtypes = [ctypes.c_int, i64, vp]
    lib.rd_power_slot.argtypes = [i64, i64, ctypes.c_int, sz, ctypes.c_int, vp]
    lib.rd_power_until_periodic_noalloc.argtypes = [vp, i64, i64, ctypes.c_int, vp, vp, vp, vp, vp]
    lib.rd_sparse_count.argtypes = [vp, i64, i64, i64, ctypes.c_int, vp, vp, vp]
    lib.rd_sparse_record_words.argtypes = [ctypes.c_int]
    lib.rd_sparse_record_words.restype = ctypes.c_int
    lib.rd_sparse_build.argtypes = [vp, i64, i64, i64, ctypes.c_int, vp, vp, vp]
    lib.rd_sparse_minplus.argtypes = [ctypes.c_int, i64, vp, vp, vp, i64, i64, vp, i64, vp, vp]
    lib.rd_power_until_periodic_sparse.argtypes = [vp, i64, i64, ctypes.c_int, vp, vp, ctypes.c_int, vp, sz, vp,
                                                   vp, vp, vp, vp]
    lib.rd_sparse_tune.argtypes = [vp, i64, i64, vp, sz, vp, vp, vp]
    lib.rd_sparse_minplus_tma.argtypes = [ctypes.c_int, i64, vp, vp, vp, i64, i64, vp, i64, vp, vp, vp]
    lib.rd_sparse_minplus_tma_bounded.argtypes = [ctypes.c_int, i64, vp, vp, vp, i64, i64, vp, i64, vp, vp,
                                                  ctypes.c_uint32, ctypes.c_int32, vp]
    lib.rd_sparse_minplus_tma_bounded.restype = st
    lib.rd_split_default_j.argtypes = [ctypes.c_int]
    lib.rd_split_default_j.restype = ctypes.c_int
    lib.rd_split_plan_bytes.argtypes = [ctypes.c_int, ctypes.c_int, vp]
    lib.rd_split_plan.argtypes = [ctypes.c_int, ctypes.c_int, vp, sz, vp, vp]
    lib.rd_split_minplus.argtypes = [vp, vp, vp, i64, vp, i64, vp, i64, vp, vp]
    lib.rd_power_until_periodic_split.argtypes = [vp, i64, vp, vp, vp, i64, ctypes.c_int, vp, sz, vp, vp, vp,
                                                  vp, vp]
    lib.rd_tune_bucket.argtypes = [i64]
    lib.rd_tune_bucket.restype = ctypes.c_int
    lib.rd_tune_set.argtypes = [vp, ctypes.c_int]
    lib.rd_tune_get.argtypes = [vp, ctypes.c_int, vp]
    lib.rd_tune_lookup.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, vp]
    lib.rd_tune_gemm.argtypes = [vp, i64, vp, i64, vp, i64, i64, i64, i64, ctypes.c_int, vp, vp]
    lib.rd_tune_split.argtypes = [vp, vp, vp, i64, vp, i64, vp, i64, ctypes.c_int, vp, vp]
    for name in ("rd_tune_set", "rd_tune_get", "rd_tune_lookup", "rd_tune_gemm", "rd_tune_split"):
        getattr(lib, name).restype = st
    for name in ("rd_state_count", "rd_padded_dim", "rd_enumerate_states", "rd_build_transfer",
                 "rd_minplus_gemm", "rd_power_work_bytes", "rd_power_until_periodic", "rd_gamma_R",
                 "rd_power_slot", "rd_power_until_periodic_noalloc", "rd_sparse_count", "rd_sparse_build",
                 "rd_sparse_minplus", "rd_power_until_periodic_sparse", "rd_sparse_tune",
                 "rd_build_transfer_loss", "rd_minplus_gemm_batched", "rd_power_until_periodic_multi",
                 "rd_server_create", "rd_server_submit", "rd_server_wait", "rd_server_stats",
                 "rd_server_destroy", "rd_sparse_minplus_tma", "rd_minplus_gemv", "rd_split_plan_bytes",
                 "rd_split_plan", "rd_split_minplus", "rd_power_until_periodic_split",
                 "rd_measure_addmin_peak"):
        getattr(lib, name).restype = st
    lib.rd_measure_addmin_peak.argtypes = [vp, sz, i64, vp, vp]
    lib.rd_gamma_R_clear.argtypes = []
    lib.rd_gamma_R_clear.restype = st
    lib.rd_minplus_gemm_streamk_work_bytes.argtypes = [i64, i64, i64, vp]
    lib.rd_minplus_gemm_streamk_work_bytes.restype = st
    lib.rd_minplus_gemm_streamk.argtypes = [vp, i64, vp, i64, vp, i64, i64, i64, i64, vp, sz, vp, vp]
    lib.rd_minplus_gemm_streamk.restype = st
    lib.rd_minplus_gemm_host_work_bytes.argtypes = [i64, i64, i64, vp]
    lib.rd_minplus_gemm_host_work_bytes.restype = st
    lib.rd_minplus_gemm_host.argtypes = [vp, i64, vp, i64, vp, i64, i64, i64, i64, vp, sz, vp, vp]
    lib.rd_minplus_gemm_host.restype = st
    lib.rd_gamma_R_export.argtypes = [ctypes.c_int, vp, vp, i64]
    lib.rd_gamma_R_import.argtypes = [vp, vp]
    lib.rd_server_export.argtypes = [vp, ctypes.c_int, vp, vp, i64]
    lib.rd_server_import.argtypes = [vp, vp, vp]
    for name in ("rd_gamma_R_export", "rd_gamma_R_import", "rd_server_export", "rd_server_import"):
        getattr(lib, name).restype = st
    lib.rd_split_check_flags.argtypes = [vp, ctypes.c_int]
    lib.rd_split_check_flags.restype = st
    _ = i32
    return lib


def declared_symbols() -> list[str]:
    """Names of the functions include/rd.h declares."""
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:rd_status|const char \*)\s*(rd_\w+)\s*\(", text, re.M)))


def _check(status: int, where: str, ok=(RD_OK,)):
    if status not in ok:
        raise RdError(status, where)
    return status


def _stream(stream):
    import torch

    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _dptr(t) -> ctypes.c_void_p:
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


# ---------------------------------------------------------------- entry points (same names as the ABI)

def state_count(m: int) -> int:
    """C_m, the number of correct words of length m (Definition 4)."""
    n = ctypes.c_int64()
    _check(_lib().rd_state_count(m, ctypes.byref(n)), "rd_state_count")
    return n.value


def padded_dim(n: int) -> int:
    """Smallest accepted leading dimension >= n."""
    out = ctypes.c_int64()
    _check(_lib().rd_padded_dim(n, ctypes.byref(out)), "rd_padded_dim")
    return out.value


def enumerate_states(m: int, codes, weights, stream=None) -> None:
    """codes (int32/uint32, C_m) and weights (uint8, C_m) on the device."""
    _check(_lib().rd_enumerate_states(m, _dptr(codes), _dptr(weights), _stream(stream)), "rd_enumerate_states")


def build_transfer(m: int, A, stream=None) -> None:
    """Fill A (int16, C_m x ld, row-major, ld = A.stride(0)) with A(G)."""
    assert A.dim() == 2 and A.stride(1) == 1
    _check(_lib().rd_build_transfer(m, _dptr(A), A.stride(0), _stream(stream)), "rd_build_transfer")


def build_transfer_loss(m: int, A, stream=None) -> None:
    """Fill A with the Appendix variant's matrix, labels shifted by loss_shift(m)."""
    assert A.dim() == 2 and A.stride(1) == 1
    _check(_lib().rd_build_transfer_loss(m, _dptr(A), A.stride(0), _stream(stream)), "rd_build_transfer_loss")


def loss_shift(m: int) -> int:
    """The constant rd_build_transfer_loss adds to every label: 2m."""
    return 2 * m


def minplus_gemm(A, B, C, M: int | None = None, N: int | None = None, K: int | None = None, min_out=None,
                 stream=None) -> None:
    """C[:M, :N] = A[:M, :K] (x) B[:K, :N] on int16 CUDA tensors (row-major, unit column stride)."""
    for t in (A, B, C):
        assert t.dim() == 2 and t.stride(1) == 1
    M = C.shape[0] if M is None else M
    N = C.shape[1] if N is None else N
    K = A.shape[1] if K is None else K
    mo = _dptr(min_out) if min_out is not None else None
    _check(_lib().rd_minplus_gemm(_dptr(A), A.stride(0), _dptr(B), B.stride(0), _dptr(C), C.stride(0), M, N, K,
                                  mo, _stream(stream)), "rd_minplus_gemm")


def minplus_gemm_streamk_work_bytes(M: int, N: int, K: int) -> int:
    out = ctypes.c_size_t()
    _check(_lib().rd_minplus_gemm_streamk_work_bytes(M, N, K, ctypes.byref(out)),
           "rd_minplus_gemm_streamk_work_bytes")
    return out.value


def minplus_gemm_streamk_workspace(M: int, N: int, K: int, device="cuda"):
    """A zero-filled workspace for rd_minplus_gemm_streamk (each call leaves it zero-filled again)."""
    import torch

    return torch.zeros(minplus_gemm_streamk_work_bytes(M, N, K), dtype=torch.uint8, device=device)


def minplus_gemm_streamk(A, B, C, work, M: int | None = None, N: int | None = None, K: int | None = None,
                         min_out=None, stream=None) -> None:
    """rd_minplus_gemm_streamk: C[:M, :N] = A[:M, :K] (x) B[:K, :N], the k-tiles shared evenly by the resident
    CTAs; `work` from minplus_gemm_streamk_workspace."""
    for t in (A, B, C):
        assert t.dim() == 2 and t.stride(1) == 1
    M = C.shape[0] if M is None else M
    N = C.shape[1] if N is None else N
    K = A.shape[1] if K is None else K
    mo = _dptr(min_out) if min_out is not None else None
    _check(_lib().rd_minplus_gemm_streamk(_dptr(A), A.stride(0), _dptr(B), B.stride(0), _dptr(C), C.stride(0), M, N,
                                          K, _dptr(work), work.numel() * work.element_size(), mo, _stream(stream)),
           "rd_minplus_gemm_streamk")


def minplus_gemv(x, B, y, N: int | None = None, K: int | None = None, min_out=None, stream=None) -> None:
    """y[:N] = x[:K] (x) B[:K, :N] (row vector times matrix) on int16 CUDA tensors."""
    N = y.numel() if N is None else N
    K = x.numel() if K is None else K
    mo = _dptr(min_out) if min_out is not None else None
    _check(_lib().rd_minplus_gemv(_dptr(x), _dptr(B), B.stride(0), _dptr(y), N, K, mo, _stream(stream)),
           "rd_minplus_gemv")


class GemmProblem(ctypes.Structure):
    """rd_gemm_problem of include/rd.h."""
    _fields_ = [("A", ctypes.c_void_p), ("lda", ctypes.c_int64), ("B", ctypes.c_void_p), ("ldb", ctypes.c_int64),
                ("C", ctypes.c_void_p), ("ldc", ctypes.c_int64), ("M", ctypes.c_int64), ("N", ctypes.c_int64),
                ("K", ctypes.c_int64), ("min_out", ctypes.c_void_p)]


def minplus_gemm_batched(problems, stream=None) -> None:
    """problems: list of (A, B, C) or (A, B, C, M, N, K, min_out) -- all products in one persistent launch."""
    arr = (GemmProblem * max(1, len(problems)))()
    for i, pr in enumerate(problems):
        A, B, C = pr[:3]
        M = pr[3] if len(pr) > 3 else C.shape[0]
        N = pr[4] if len(pr) > 4 else C.shape[1]
        K = pr[5] if len(pr) > 5 else A.shape[1]
        mo = pr[6] if len(pr) > 6 else None
        arr[i] = GemmProblem(A.data_ptr(), A.stride(0), B.data_ptr(), B.stride(0), C.data_ptr(), C.stride(0), M, N,
                             K, mo.data_ptr() if mo is not None else None)
    _check(_lib().rd_minplus_gemm_batched(arr, len(problems), _stream(stream)), "rd_minplus_gemm_batched")


class PowerRun(ctypes.Structure):
    """rd_power_run of include/rd.h."""
    _fields_ = [("A", ctypes.c_void_p), ("N", ctypes.c_int64), ("lda", ctypes.c_int64),
                ("block_start", ctypes.c_void_p), ("records", ctypes.c_void_p), ("work", ctypes.c_void_p),
                ("work_bytes", ctypes.c_size_t), ("gamma_host", ctypes.c_void_p), ("k", ctypes.c_int32),
                ("p", ctypes.c_int32), ("q", ctypes.c_int64), ("status", ctypes.c_int),
                ("split_info", ctypes.c_void_p), ("split_plan", ctypes.c_void_p), ("split_X", ctypes.c_void_p),
                ("split_ldx", ctypes.c_int64)]


def power_until_periodic_multi(runs, R: int, kmax: int, graph_steps: int = 8, stream=None, wait_ms: int = 1000,
                               stall_run: int = -1) -> list:
    """runs: list of (A, n, plan, work), plan from sparse_plan() (rows per block R) or split_plan().
    All searches advance together; returns one result dict per run.  wait_ms and stall_run: see
    rd_power_until_periodic_multi_bounded (the defaults are rd_power_until_periodic_multi)."""
    arr = (PowerRun * len(runs))()
    gammas = []
    for i, (A, n, plan, work) in enumerate(runs):
        g = np.zeros(kmax + 1, dtype=np.int64)
        gammas.append(g)
        if "info" in plan:  # row-split step
            X = plan["X"]
            arr[i] = PowerRun(A.data_ptr(), n, A.stride(0), None, None, work.data_ptr(),
                              work.numel() * work.element_size(), g.ctypes.data, 0, 0, 0, 0,
                              ctypes.addressof(plan["info"]), plan["plan"].data_ptr(), X.data_ptr(), X.stride(0))
            continue
        assert plan["R"] == R
        arr[i] = PowerRun(A.data_ptr(), n, A.stride(0), plan["block_start"].data_ptr(), plan["records"].data_ptr(),
                          work.data_ptr(), work.numel() * work.element_size(), g.ctypes.data, 0, 0, 0, 0)
    _check(_lib().rd_power_until_periodic_multi_bounded(arr, len(runs), R, kmax, graph_steps, wait_ms, stall_run,
                                                        _stream(stream)), "rd_power_until_periodic_multi")
    out = []
    for i in range(len(runs)):
        st = arr[i].status
        if i == stall_run:
            out.append(dict(status=st, found=False, k=None, p=None, q=None, j=kmax, gamma=gammas[i]))
            continue
        _check(st, f"rd_power_until_periodic_multi run {i}", ok=(RD_OK, RD_NOT_FOUND))
        found = st == RD_OK
        out.append(dict(status=st, found=found, k=arr[i].k if found else None, p=arr[i].p if found else None,
                        q=arr[i].q if found else None, j=arr[i].k + arr[i].p if found else kmax, gamma=gammas[i]))
    return out


class Relation(ctypes.Structure):
    """rd_relation_t: the first repeat A^(k+p) = q (x) A^k of one m and how many gamma values go with it."""
    _fields_ = [("m", ctypes.c_int32), ("found", ctypes.c_int32), ("k", ctypes.c_int32), ("p", ctypes.c_int32),
                ("q", ctypes.c_int64), ("j", ctypes.c_int32), ("reserved", ctypes.c_int32)]


def _relation_dict(rel: Relation, gamma: np.ndarray) -> dict:
    found = bool(rel.found)
    return dict(m=rel.m, found=found, k=rel.k if found else None, p=rel.p if found else None,
                q=rel.q if found else None, j=rel.j, gamma=[int(v) for v in gamma[1: rel.j + 1]])


def _relation_args(rec: dict):
    """(Relation, gamma array of j + 1 int64) from a record dict (gamma lists n = 1..j)."""
    found = bool(rec["found"])
    g = [int(v) for v in rec["gamma"]]
    rel = Relation(m=int(rec["m"]), found=1 if found else 0, k=int(rec["k"]) if found else 0,
                   p=int(rec["p"]) if found else 0, q=int(rec["q"]) if found else 0, j=len(g), reserved=0)
    if int(rec.get("j", len(g))) != len(g):
        raise ValueError(f"record for m = {rec['m']}: j = {rec['j']} but {len(g)} gamma values")
    gamma = np.ascontiguousarray([RD_GAMMA_UNSET] + g, dtype=np.int64)
    return rel, gamma


def _export(call, where: str) -> dict | None:
    rel = Relation()
    st = call(ctypes.byref(rel), None, 0)
    if st == RD_NOT_FOUND and where == "rd_server_export":
        return None
    _check(st, where)
    gamma = np.zeros(rel.j + 1, dtype=np.int64)
    _check(call(ctypes.byref(rel), gamma.ctypes.data, len(gamma)), where)
    return _relation_dict(rel, gamma)


class ServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("answered", ctypes.c_uint64), ("steps", ctypes.c_uint64),
                ("jobs_admitted", ctypes.c_uint64), ("jobs_completed", ctypes.c_uint64),
                ("bytes_in_use", ctypes.c_size_t), ("bytes_peak", ctypes.c_size_t)]


class Server:
    """rd_server_*: gamma_R queries answered with continuous batching of the period searches."""

    def __init__(self, hbm_budget_bytes: int, kmax: int = 256):
        h = ctypes.c_void_p()
        _check(_lib().rd_server_create(hbm_budget_bytes, kmax, ctypes.byref(h)), "rd_server_create")
        self._h = h

    def submit(self, ms, ns) -> np.ndarray:
        ms = np.ascontiguousarray(ms, dtype=np.int32)
        ns = np.ascontiguousarray(ns, dtype=np.int64)
        t = np.zeros(len(ms), dtype=np.uint64)
        _check(_lib().rd_server_submit(self._h, len(ms), ms.ctypes.data, ns.ctypes.data, t.ctypes.data),
               "rd_server_submit")
        return t

    def wait(self, tickets, timeout_s: float = 600.0):
        """(gamma, status, latency_s) arrays for the tickets; raises RdError(RD_ERR_TIMEOUT) on timeout."""
        tickets = np.ascontiguousarray(tickets, dtype=np.uint64)
        g = np.zeros(len(tickets), dtype=np.int64)
        st = np.zeros(len(tickets), dtype=np.int32)
        lat = np.zeros(len(tickets), dtype=np.float64)
        _check(_lib().rd_server_wait(self._h, len(tickets), tickets.ctypes.data, timeout_s, g.ctypes.data,
                                     st.ctypes.data, lat.ctypes.data), "rd_server_wait")
        return g, st, lat

    def export_relation(self, m: int) -> dict | None:
        """rd_server_export: the server's final record for m as a dict, or None while it has none."""
        return _export(lambda r, g, c: _lib().rd_server_export(self._h, m, r, g, c), "rd_server_export")

    def import_relation(self, rec: dict) -> None:
        """rd_server_import: warm start -- queries for rec['m'] are answered from the record."""
        rel, gamma = _relation_args(rec)
        _check(_lib().rd_server_import(self._h, ctypes.byref(rel), gamma.ctypes.data), "rd_server_import")

    def stats(self) -> dict:
        s = ServerStats()
        _check(_lib().rd_server_stats(self._h, ctypes.byref(s)), "rd_server_stats")
        return {f: getattr(s, f) for f, _ in ServerStats._fields_}

    def close(self) -> None:
        if self._h:
            _lib().rd_server_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def minplus_gemm_host_work_bytes(M: int, N: int, K: int) -> int:
    out = ctypes.c_size_t()
    _check(_lib().rd_minplus_gemm_host_work_bytes(M, N, K, ctypes.byref(out)), "rd_minplus_gemm_host_work_bytes")
    return out.value


def minplus_gemm_host(a, b, c, work, min_out=None, stream=None) -> None:
    """rd_minplus_gemm_host: C = A (x) B with A, B, C in host memory (CPU tensors or numpy int16 arrays, pinned
    for asynchronous copies), staged in the device tensor `work`.  Asynchronous on the stream."""
    def host_ptr(x):
        if hasattr(x, "data_ptr"):
            if x.is_cuda:
                raise ValueError("expected a host tensor")
            return ctypes.c_void_p(x.data_ptr()), x.stride(0)
        return ctypes.c_void_p(x.ctypes.data), x.strides[0] // 2

    (pa, lda), (pb, ldb), (pc, ldc) = host_ptr(a), host_ptr(b), host_ptr(c)
    M, K = a.shape
    N = b.shape[1]
    mo = _dptr(min_out) if min_out is not None else None
    _check(_lib().rd_minplus_gemm_host(pa, lda, pb, ldb, pc, ldc, M, N, K, _dptr(work),
                                       work.numel() * work.element_size(), mo, _stream(stream)),
           "rd_minplus_gemm_host")


class AddminPeak(ctypes.Structure):
    _fields_ = [("addmin_per_clk_per_sm", ctypes.c_double), ("addmin_per_s", ctypes.c_double),
                ("sm_mhz", ctypes.c_double), ("ms", ctypes.c_double), ("sm_count", ctypes.c_int32),
                ("ctas_per_sm", ctypes.c_int32), ("lanes_per_clk_per_sm", ctypes.c_int32)]


RD_PEAK_WORK_BYTES = 65536


def measure_addmin_peak(trips: int = 8192, stream=None) -> dict:
    """rd_measure_addmin_peak: the DPX add-min rate of the current device (per SM clock and per second)."""
    import torch

    work = torch.empty(RD_PEAK_WORK_BYTES, dtype=torch.uint8, device="cuda")
    out = AddminPeak()
    _check(_lib().rd_measure_addmin_peak(_dptr(work), RD_PEAK_WORK_BYTES, trips, ctypes.byref(out), _stream(stream)),
           "rd_measure_addmin_peak")
    return {f: getattr(out, f) for f, _ in AddminPeak._fields_}


def power_work_bytes(n: int, ld: int, kmax: int, slots: int) -> int:
    out = ctypes.c_size_t()
    _check(_lib().rd_power_work_bytes(n, ld, kmax, slots, ctypes.byref(out)), "rd_power_work_bytes")
    return out.value


def power_until_periodic(A, n: int, kmax: int, work, stream=None) -> dict:
    """Algorithm 2 on the device.  Returns dict(status, found, k, p, q, j, gamma (np.int64, index 1..j))."""
    gamma = np.zeros(kmax + 1, dtype=np.int64)
    k, p, q = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int64()
    st = _lib().rd_power_until_periodic(_dptr(A), n, A.stride(0), kmax, _dptr(work), work.numel() * work.element_size(),
                                        ctypes.c_void_p(gamma.ctypes.data), ctypes.byref(k), ctypes.byref(p),
                                        ctypes.byref(q), _stream(stream))
    _check(st, "rd_power_until_periodic", ok=(RD_OK, RD_NOT_FOUND))
    found = st == RD_OK
    j = k.value + p.value if found else kmax
    return dict(status=st, found=found, k=k.value if found else None, p=p.value if found else None,
                q=q.value if found else None, j=j, gamma=gamma)


def power_until_periodic_noalloc(A, n: int, kmax: int, stream=None) -> dict:
    """rd_power_until_periodic on the library's static scratch (no work buffer, no allocation)."""
    gamma = np.zeros(kmax + 1, dtype=np.int64)
    k, p, q = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int64()
    st = _lib().rd_power_until_periodic_noalloc(_dptr(A), n, A.stride(0), kmax, ctypes.c_void_p(gamma.ctypes.data),
                                                ctypes.byref(k), ctypes.byref(p), ctypes.byref(q), _stream(stream))
    _check(st, "rd_power_until_periodic_noalloc", ok=(RD_OK, RD_NOT_FOUND))
    found = st == RD_OK
    j = k.value + p.value if found else kmax
    return dict(status=st, found=found, k=k.value if found else None, p=p.value if found else None,
                q=q.value if found else None, j=j, gamma=gamma)


def sparse_count(A, M: int, K: int, R: int, block_start, stream=None) -> int:
    """Block-sparse form, step 1: block_start (int64, ceil(M/R)+1) and the number of entries."""
    ent = ctypes.c_int64()
    _check(_lib().rd_sparse_count(_dptr(A), A.stride(0), M, K, R, _dptr(block_start), ctypes.byref(ent),
                                  _stream(stream)), "rd_sparse_count")
    return ent.value


def sparse_build(A, M: int, K: int, R: int, block_start, records, stream=None) -> None:
    """Block-sparse form, step 2: the entry records (int32 view of uint32)."""
    _check(_lib().rd_sparse_build(_dptr(A), A.stride(0), M, K, R, _dptr(block_start), _dptr(records),
                                  _stream(stream)), "rd_sparse_build")


def sparse_plan(A, M: int, K: int, R: int = 4, stream=None) -> dict:
    """Allocate (torch) and build the block-sparse form of A[:M, :K]."""
    import torch

    nb = (M + R - 1) // R
    start = torch.empty(nb + 1, dtype=torch.int64, device=A.device)
    ent = sparse_count(A, M, K, R, start, stream)
    words = _lib().rd_sparse_record_words(R)
    rec = torch.empty(max(ent, 1) * words, dtype=torch.int32, device=A.device)
    sparse_build(A, M, K, R, start, rec, stream)
    return dict(R=R, M=M, K=K, entries=ent, block_start=start, records=rec)


def sparse_minplus(plan: dict, B, C, N: int | None = None, min_out=None, stream=None) -> None:
    """C[:M, :N] = A (x) B[:K, :N] with A given by sparse_plan()."""
    N = C.shape[1] if N is None else N
    mo = _dptr(min_out) if min_out is not None else None
    _check(_lib().rd_sparse_minplus(plan["R"], plan["M"], _dptr(plan["block_start"]), _dptr(plan["records"]),
                                    _dptr(B), B.stride(0), N, _dptr(C), C.stride(0), mo, _stream(stream)),
           "rd_sparse_minplus")


def sparse_tune(A, n: int, scratch, stream=None):
    """Native autotuner: (best R, {R: ms per product A (x) A}) for the sparse step on A[:n, :n]."""
    best = ctypes.c_int()
    ms = (ctypes.c_float * 4)()
    _check(_lib().rd_sparse_tune(_dptr(A), A.stride(0), n, _dptr(scratch), scratch.numel() * scratch.element_size(),
                                 ctypes.byref(best), ms, _stream(stream)), "rd_sparse_tune")
    return best.value, {R: ms[i] for i, R in enumerate((1, 2, 4, 8)) if ms[i] >= 0}


def sparse_minplus_tma(plan: dict, B, C, err, N: int | None = None, min_out=None, stream=None) -> None:
    """sparse_minplus through the bulk-copy kernel; err is a zeroed device int32 that receives 8 on a timeout."""
    N = C.shape[1] if N is None else N
    mo = _dptr(min_out) if min_out is not None else None
    _check(_lib().rd_sparse_minplus_tma(plan["R"], plan["M"], _dptr(plan["block_start"]), _dptr(plan["records"]),
                                        _dptr(B), B.stride(0), N, _dptr(C), C.stride(0), mo, _dptr(err),
                                        _stream(stream)), "rd_sparse_minplus_tma")


def sparse_minplus_tma_bounded(plan: dict, B, C, err, wait_limit: int, stop_at: int, N: int | None = None,
                               min_out=None, stream=None) -> None:
    """sparse_minplus_tma with an explicit wait limit and producer stop point (the timeout path's test knobs)."""
    N = C.shape[1] if N is None else N
    mo = _dptr(min_out) if min_out is not None else None
    _check(_lib().rd_sparse_minplus_tma_bounded(plan["R"], plan["M"], _dptr(plan["block_start"]),
                                                _dptr(plan["records"]), _dptr(B), B.stride(0), N, _dptr(C),
                                                C.stride(0), mo, _dptr(err), wait_limit, stop_at, _stream(stream)),
           "rd_sparse_minplus_tma_bounded")


def power_until_periodic_sparse(A, n: int, plan: dict, kmax: int, work, stream=None) -> dict:
    """rd_power_until_periodic with the dense x sparse step."""
    gamma = np.zeros(kmax + 1, dtype=np.int64)
    k, p, q = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int64()
    st = _lib().rd_power_until_periodic_sparse(_dptr(A), n, A.stride(0), plan["R"], _dptr(plan["block_start"]),
                                               _dptr(plan["records"]), kmax, _dptr(work),
                                               work.numel() * work.element_size(), ctypes.c_void_p(gamma.ctypes.data),
                                               ctypes.byref(k), ctypes.byref(p), ctypes.byref(q), _stream(stream))
    _check(st, "rd_power_until_periodic_sparse", ok=(RD_OK, RD_NOT_FOUND))
    found = st == RD_OK
    j = k.value + p.value if found else kmax
    return dict(status=st, found=found, k=k.value if found else None, p=p.value if found else None,
                q=q.value if found else None, j=j, gamma=gamma)


class SplitInfo(ctypes.Structure):
    """rd_split_info_t of include/rd.h."""
    _fields_ = [("m", ctypes.c_int32), ("j", ctypes.c_int32), ("N", ctypes.c_int64), ("n_rho", ctypes.c_int32),
                ("n_sigma", ctypes.c_int32), ("n_pi", ctypes.c_int32), ("n_phi", ctypes.c_int32),
                ("list1_entries", ctypes.c_int64), ("list2_entries", ctypes.c_int64), ("x_rows", ctypes.c_int64),
                ("plan_bytes", ctypes.c_uint64), ("w1", ctypes.c_int32), ("w2", ctypes.c_int32),
                ("slots1", ctypes.c_int32), ("slots2", ctypes.c_int32), ("lmax1", ctypes.c_int32),
                ("lmax2", ctypes.c_int32), ("k1", ctypes.c_int32), ("k2", ctypes.c_int32),
                ("chunk_cols", ctypes.c_int32)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


def split_check_flags(reset: bool = True) -> int | None:
    """rd_split_check_flags: the row-split passes' index-check bits of the current device (checked build),
    or None for a library built without checks."""
    v = ctypes.c_uint32()
    st = _lib().rd_split_check_flags(ctypes.byref(v), 1 if reset else 0)
    if st == RD_NOT_FOUND:
        return None
    _check(st, "rd_split_check_flags")
    return v.value


def split_default_j(m: int) -> int:
    """The default split row of the row-split step (0 when m has none)."""
    return _lib().rd_split_default_j(m)


def split_plan_bytes(m: int, j: int) -> int:
    out = ctypes.c_size_t()
    _check(_lib().rd_split_plan_bytes(m, j, ctypes.byref(out)), "rd_split_plan_bytes")
    return out.value


def split_plan(m: int, j: int | None = None, device="cuda", x_ld: int | None = None, chunk_cols: int = 0,
               stream=None) -> dict:
    """Allocate (torch) and build the row-split plan of A(G) for m rows, plus its intermediate X
    (all N columns, or one chunk of chunk_cols columns)."""
    import torch

    j = split_default_j(m) if j is None else j
    plan = torch.empty(split_plan_bytes(m, j), dtype=torch.uint8, device=device)
    info = SplitInfo()
    _check(_lib().rd_split_plan(m, j, _dptr(plan), plan.numel(), ctypes.byref(info), _stream(stream)),
           "rd_split_plan")
    info.chunk_cols = chunk_cols
    ld = (chunk_cols if chunk_cols else padded_dim(info.N)) if x_ld is None else x_ld
    X = torch.empty((info.x_rows, ld), dtype=torch.int16, device=device)
    return dict(info=info, plan=plan, X=X)


def split_minplus(plan: dict, B, C, min_out=None, stream=None) -> None:
    """C[:N, :N] = A(G) (x) B[:N, :N] through the two row-split passes."""
    mo = _dptr(min_out) if min_out is not None else None
    X = plan["X"]
    _check(_lib().rd_split_minplus(ctypes.byref(plan["info"]), _dptr(plan["plan"]), _dptr(B), B.stride(0), _dptr(X),
                                   X.stride(0), _dptr(C), C.stride(0), mo, _stream(stream)), "rd_split_minplus")


def power_until_periodic_split(A, plan: dict, kmax: int, work, stream=None) -> dict:
    """rd_power_until_periodic with the row-split step; A is A(G) for the plan's m."""
    gamma = np.zeros(kmax + 1, dtype=np.int64)
    k, p, q = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int64()
    X = plan["X"]
    st = _lib().rd_power_until_periodic_split(_dptr(A), A.stride(0), ctypes.byref(plan["info"]), _dptr(plan["plan"]),
                                              _dptr(X), X.stride(0), kmax, _dptr(work),
                                              work.numel() * work.element_size(), ctypes.c_void_p(gamma.ctypes.data),
                                              ctypes.byref(k), ctypes.byref(p), ctypes.byref(q), _stream(stream))
    _check(st, "rd_power_until_periodic_split", ok=(RD_OK, RD_NOT_FOUND))
    found = st == RD_OK
    j = k.value + p.value if found else kmax
    return dict(status=st, found=found, k=k.value if found else None, p=p.value if found else None,
                q=q.value if found else None, j=j, gamma=gamma)


# ---------------------------------------------------------------- tuning table and autotuners

RD_TUNE_GEMM_SPLITK, RD_TUNE_SPLIT, RD_TUNE_SPARSE_R = 1, 2, 3
RD_TUNE_MAX = 256
TUNE_MODES = {RD_TUNE_GEMM_SPLITK: "gemm_splitk", RD_TUNE_SPLIT: "split", RD_TUNE_SPARSE_R: "sparse_r"}


class TuneEntry(ctypes.Structure):
    """rd_tune_entry_t of include/rd.h."""
    _fields_ = [("mode", ctypes.c_int32), ("key", ctypes.c_int32), ("aux", ctypes.c_int32),
                ("p", ctypes.c_int32 * 4), ("ms", ctypes.c_float)]

    def as_dict(self) -> dict:
        return dict(mode=TUNE_MODES.get(self.mode, self.mode), key=self.key, aux=self.aux, p=list(self.p),
                    ms=round(float(self.ms), 6))

    @classmethod
    def from_dict(cls, d: dict) -> "TuneEntry":
        names = {v: k for k, v in TUNE_MODES.items()}
        mode = names.get(d["mode"], d["mode"])
        p = list(d["p"]) + [0] * (4 - len(d["p"]))
        return cls(int(mode), int(d["key"]), int(d["aux"]), (ctypes.c_int32 * 4)(*p[:4]), float(d.get("ms", -1.0)))


def tune_bucket(x: int) -> int:
    """ceil(log2(x)): the size class of the tuning table's keys."""
    return _lib().rd_tune_bucket(int(x))


def tune_table() -> list[dict]:
    """The library's tuning table, one dict per entry."""
    n = ctypes.c_int()
    arr = (TuneEntry * RD_TUNE_MAX)()
    _check(_lib().rd_tune_get(arr, RD_TUNE_MAX, ctypes.byref(n)), "rd_tune_get")
    return [arr[i].as_dict() for i in range(n.value)]


def tune_set(entries: list[dict]) -> None:
    """Replace the library's tuning table (an empty list clears it)."""
    arr = (TuneEntry * max(1, len(entries)))(*[TuneEntry.from_dict(e) for e in entries])
    _check(_lib().rd_tune_set(arr, len(entries)), "rd_tune_set")


def tune_lookup(mode: int, key: int, aux: int) -> dict | None:
    out = TuneEntry()
    st = _check(_lib().rd_tune_lookup(mode, key, aux, ctypes.byref(out)), "rd_tune_lookup", ok=(RD_OK, RD_NOT_FOUND))
    return out.as_dict() if st == RD_OK else None


def tune_gemm(A, B, C, M: int | None = None, N: int | None = None, K: int | None = None, reps: int = 3,
              stream=None) -> dict:
    """Native autotuner of the split-K factor of minplus_gemm for an M x N x K product (C is overwritten)."""
    M = C.shape[0] if M is None else M
    N = C.shape[1] if N is None else N
    K = A.shape[1] if K is None else K
    out = TuneEntry()
    _check(_lib().rd_tune_gemm(_dptr(A), A.stride(0), _dptr(B), B.stride(0), _dptr(C), C.stride(0), M, N, K, reps,
                               ctypes.byref(out), _stream(stream)), "rd_tune_gemm")
    return out.as_dict()


def tune_split(plan: dict, B, C, reps: int = 2, stream=None) -> dict:
    """Native autotuner of the row-split passes' launch shape; updates plan["info"] (X and C are overwritten)."""
    out = TuneEntry()
    X = plan["X"]
    _check(_lib().rd_tune_split(ctypes.byref(plan["info"]), _dptr(plan["plan"]), _dptr(B), B.stride(0), _dptr(X),
                                X.stride(0), _dptr(C), C.stride(0), reps, ctypes.byref(out), _stream(stream)),
           "rd_tune_split")
    return out.as_dict()


def power_slot(n: int, ld: int, kmax: int, work_bytes: int, k: int) -> int:
    """Byte offset of the resident normalised power P_k inside the work buffer."""
    out = ctypes.c_size_t()
    _check(_lib().rd_power_slot(n, ld, kmax, work_bytes, k, ctypes.byref(out)), "rd_power_slot")
    return out.value


def gamma_R(m: int, n: int) -> int:
    """gamma_R(P_m box C_n), from the library's per-process cache."""
    out = ctypes.c_int64()
    _check(_lib().rd_gamma_R(m, n, ctypes.byref(out)), "rd_gamma_R")
    return out.value


def gamma_R_clear() -> None:
    """rd_gamma_R_clear: forget every cached m (the next rd_gamma_R of each m searches again)."""
    _check(_lib().rd_gamma_R_clear(), "rd_gamma_R_clear")


def gamma_R_export(m: int) -> dict:
    """rd_gamma_R_export: dict(m, found, k, p, q, j, gamma) with gamma = [gamma(1), ..., gamma(j)];
    runs the period search first when m is not cached."""
    return _export(lambda r, g, c: _lib().rd_gamma_R_export(m, r, g, c), "rd_gamma_R_export")


def gamma_R_import(rec: dict) -> None:
    """rd_gamma_R_import: install a record (as gamma_R_export returns it) as the cache entry of rec['m']."""
    rel, gamma = _relation_args(rec)
    _check(_lib().rd_gamma_R_import(ctypes.byref(rel), gamma.ctypes.data), "rd_gamma_R_import")


# ---------------------------------------------------------------- allocation helpers (torch owns device memory)

def transfer_matrix(m: int, device="cuda", stream=None):
    """Allocate and build A(G); returns (A, N) with A of shape (N, ld)."""
    import torch

    n = state_count(m)
    A = torch.empty((n, padded_dim(n)), dtype=torch.int16, device=device)
    build_transfer(m, A, stream)
    return A, n


def power_workspace(n: int, ld: int, kmax: int, slots: int, device="cuda"):
    import torch

    return torch.empty(power_work_bytes(n, ld, kmax, slots), dtype=torch.uint8, device=device)
