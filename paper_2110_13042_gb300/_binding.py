"""ctypes binding of the C ABI in ``include/ata.h`` (argument marshalling only).

Every function here forwards to the entry point of the same name in
``libata.so``; all arithmetic happens in the library's CUDA kernels.  Tensor
arguments are accepted only to read their device pointer, shape and stride.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))

ATA_F64, ATA_F64_EMU, ATA_F32, ATA_F32_BF16, ATA_F32_FP8 = 0, 1, 2, 4, 5
ATA_TRANS, ATA_PACKED = 1, 2
STATUS = {0: "ATA_OK", 1: "ATA_ERR_INVALID", 2: "ATA_ERR_DTYPE", 3: "ATA_ERR_ALLOC",
          4: "ATA_ERR_CUDA", 5: "ATA_ERR_TIMEOUT", 6: "ATA_ERR_UNSUPPORTED"}
PLAN_FIELDS = ("cutoff", "depth", "slices", "panels", "blocks", "products", "tiles",
               "workspace_bytes", "leaf_madds", "plain_madds", "split_k", "fused_groups",
               "comb_regions")

_lib = None


class AtaError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        super().__init__(f"{what}: {STATUS.get(status, status)} ({status_string(status)})")


def library_path() -> str:
    return os.path.join(HERE, "_build", "libata.so")


def load():
    """Load libata.so (fails loudly if it was not built)."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with "
                           "`python -c \"import __graft_entry__ as g; g.build()\"`")
    L = ctypes.CDLL(path)
    i64, vp, ip = ctypes.c_int64, ctypes.c_void_p, ctypes.c_int
    L.ata_create.argtypes = [ctypes.POINTER(vp), vp]
    L.ata_set_config.argtypes = [vp, vp]
    L.ata_lower.argtypes = [vp, i64, i64, vp, i64, vp, i64, ip, vp]
    L.ata_batched.argtypes = [vp, ip, vp, vp, vp, vp, vp, vp, ip, vp]
    L.ata_batched_dev.argtypes = [vp, ip, vp, vp, vp, vp, vp, vp, ip, vp]
    L.ata_sync.argtypes = [vp, vp]
    L.ata_destroy.argtypes = [vp]
    L.ata_status_string.argtypes = [ip]
    L.ata_status_string.restype = ctypes.c_char_p
    L.ata_plan_info.argtypes = [vp, i64, i64, ip, ctypes.POINTER(i64)]
    L.ata_syrk_ex.argtypes = [vp, ip, i64, i64, ctypes.c_double, vp, i64, ctypes.c_double, vp, i64, ip, vp]
    L.ata_lower_aat.argtypes = [vp, i64, i64, vp, i64, vp, i64, ip, vp]
    L.ata_plan_blocks.argtypes = [vp, i64, i64, ip, ctypes.POINTER(i64), i64, ctypes.POINTER(i64)]
    L.ata_syrk.argtypes = [vp, i64, i64, ctypes.c_double, vp, i64, ctypes.c_double, vp, i64, ip, vp]
    L.ata_lower_noalloc.argtypes = [i64, i64, vp, i64, vp, i64, ip, vp]
    L.ata_lower_noalloc.restype = ip
    L.ata_last_error.argtypes = [vp]
    L.ata_last_error.restype = ctypes.c_char_p
    L.ata_set_timing.argtypes = [vp, ip]
    L.ata_phase_times.argtypes = [vp, ctypes.POINTER(ctypes.c_double)]
    L.ata_tune.argtypes = [vp, i64, i64, vp, i64, vp, i64, ip, vp, ctypes.c_double, ctypes.POINTER(i64)]
    L.ata_tune_clear.argtypes = [vp]
    L.ata_check_wait_timeout.argtypes = [vp, i64, vp]
    for f in ("ata_create", "ata_set_config", "ata_lower", "ata_syrk", "ata_syrk_ex", "ata_lower_aat",
              "ata_batched", "ata_batched_dev", "ata_sync",
              "ata_destroy", "ata_plan_info", "ata_plan_blocks", "ata_version", "ata_set_timing",
              "ata_phase_times", "ata_tune", "ata_tune_clear", "ata_check_wait_timeout"):
        getattr(L, f).restype = ip
    _lib = L
    return L


def status_string(status: int) -> str:
    return load().ata_status_string(int(status)).decode()


def version() -> int:
    return int(load().ata_version())


class Config(ctypes.Structure):
    _fields_ = [("cutoff", ctypes.c_int), ("strassen_depth", ctypes.c_int),
                ("slices", ctypes.c_int), ("strassen_min", ctypes.c_int),
                ("strassen_variant", ctypes.c_int), ("streams", ctypes.c_int), ("split_k", ctypes.c_int),
                ("reserved", ctypes.c_int * 1)]


def _config(cutoff=0, depth=-1, slices=0, strassen_min=0, variant=0, streams=0, split_k=0) -> Config:
    return Config(int(cutoff), int(depth), int(slices), int(strassen_min), int(variant), int(streams),
                  int(split_k), (ctypes.c_int * 1)())


def _check(rc: int, what: str):
    if rc != 0:
        raise AtaError(rc, what)


def plan_info(m: int, n: int, dtype: int, handle: "Handle | None" = None) -> dict:
    out = (ctypes.c_int64 * len(PLAN_FIELDS))()
    _check(load().ata_plan_info(handle._h if handle else None, int(m), int(n), int(dtype), out),
           "ata_plan_info")
    return dict(zip(PLAN_FIELDS, (int(v) for v in out)))


def plan_blocks(m: int, n: int, dtype: int, handle: "Handle | None" = None) -> list:
    """Off-diagonal blocks (r0, p, c0, q, strassen_depth) of the plan, in
    recursion order (host-only planner call, ata_plan_blocks)."""
    L = load()
    count = ctypes.c_int64()
    hh = handle._h if handle else None
    _check(L.ata_plan_blocks(hh, int(m), int(n), int(dtype), None, 0, ctypes.byref(count)), "ata_plan_blocks")
    out = (ctypes.c_int64 * (5 * max(count.value, 1)))()
    _check(L.ata_plan_blocks(hh, int(m), int(n), int(dtype), out, count.value, ctypes.byref(count)),
           "ata_plan_blocks")
    return [tuple(int(v) for v in out[5 * i:5 * i + 5]) for i in range(count.value)]


def lower_noalloc_ptr(m, n, A_ptr, lda, C_ptr, ldc, dtype, stream=None) -> int:
    """ata_lower_noalloc through the C ABI; returns the status code."""
    return int(load().ata_lower_noalloc(int(m), int(n), A_ptr, int(lda), C_ptr, int(ldc), int(dtype),
                                        _stream_ptr(stream)))


def _stream_ptr(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)  # torch.cuda.Stream


def _ld(T) -> int:
    """Leading dimension of a row-major 2-D tensor.  A tensor with a single
    row may report any row stride (torch treats size-1 dimensions as
    contiguous whatever their stride), so its row length stands in."""
    return int(T.stride(0)) if T.shape[0] > 1 else max(int(T.shape[1]), 1)


def _check_rowmajor(*Ts):
    for T in Ts:  # empty tensors may report any strides
        if T.dim() == 2 and T.numel() > 0 and T.shape[1] > 1 and T.stride(1) != 1:
            raise ValueError("matrices must be row-major with unit column stride")


class Handle:
    """Owns an ``ata_handle`` (workspace, plan cache, device status word)."""

    def __init__(self, cutoff=0, depth=-1, slices=0, strassen_min=0, variant=0, streams=0, split_k=0):
        L = load()
        self._h = ctypes.c_void_p()
        cfg = _config(cutoff, depth, slices, strassen_min, variant, streams, split_k)
        _check(L.ata_create(ctypes.byref(self._h), ctypes.byref(cfg)), "ata_create")

    def set_config(self, cutoff=0, depth=-1, slices=0, strassen_min=0, variant=0, streams=0, split_k=0):
        cfg = _config(cutoff, depth, slices, strassen_min, variant, streams, split_k)
        _check(load().ata_set_config(self._h, ctypes.byref(cfg)), "ata_set_config")

    def lower_ptr(self, m, n, A_ptr, lda, C_ptr, ldc, dtype, stream=None) -> int:
        """Raw C-ABI call; returns the status code (no exception)."""
        return int(load().ata_lower(self._h, int(m), int(n), A_ptr, int(lda), C_ptr, int(ldc),
                                    int(dtype), _stream_ptr(stream)))

    def last_error(self) -> str:
        return load().ata_last_error(self._h).decode()

    def lower(self, A, C, dtype, stream=None):
        """low(C) <- low(A^T A) for row-major CUDA tensors A (m x n) and C (n x n)."""
        m, n = A.shape
        _check_rowmajor(A, C)
        rc = self.lower_ptr(m, n, A.data_ptr(), _ld(A), C.data_ptr(), _ld(C), dtype, stream)
        if rc != 0:
            raise AtaError(rc, f"ata_lower [{self.last_error()}]")

    def syrk_ptr(self, m, n, alpha, A_ptr, lda, beta, C_ptr, ldc, dtype, stream=None) -> int:
        """Raw ata_syrk call; returns the status code (no exception)."""
        return int(load().ata_syrk(self._h, int(m), int(n), float(alpha), A_ptr, int(lda), float(beta), C_ptr,
                                   int(ldc), int(dtype), _stream_ptr(stream)))

    def syrk(self, A, C, dtype, alpha=1.0, beta=0.0, stream=None):
        """low(C) <- alpha low(A^T A) + beta low(C) for row-major CUDA tensors."""
        m, n = A.shape
        _check_rowmajor(A, C)
        rc = self.syrk_ptr(m, n, alpha, A.data_ptr(), _ld(A), beta, C.data_ptr(), _ld(C), dtype, stream)
        if rc != 0:
            raise AtaError(rc, f"ata_syrk [{self.last_error()}]")

    def syrk_ex_ptr(self, flags, m, n, alpha, A_ptr, lda, beta, C_ptr, ldc, dtype, stream=None) -> int:
        """Raw ata_syrk_ex call; returns the status code (no exception)."""
        return int(load().ata_syrk_ex(self._h, int(flags), int(m), int(n), float(alpha), A_ptr, int(lda),
                                      float(beta), C_ptr, int(ldc), int(dtype), _stream_ptr(stream)))

    def syrk_ex(self, A, C, dtype, flags=0, alpha=1.0, beta=0.0, stream=None):
        """ata_syrk_ex on a row-major CUDA tensor A (m x n).  C: n x n (m x m
        with ATA_TRANS) row-major, or a 1-D tensor of the packed lower
        triangle with ATA_PACKED."""
        m, n = A.shape
        _check_rowmajor(A, C)
        ldc = _ld(C) if C.dim() == 2 else 0
        rc = self.syrk_ex_ptr(flags, m, n, alpha, A.data_ptr(), _ld(A), beta, C.data_ptr(), ldc, dtype, stream)
        if rc != 0:
            raise AtaError(rc, f"ata_syrk_ex [{self.last_error()}]")

    def lower_aat(self, A, C, dtype, stream=None):
        """low(C) <- low(A A^T) for a row-major CUDA tensor A (m x n), C m x m (ata_lower_aat)."""
        m, n = A.shape
        _check_rowmajor(A, C)
        rc = int(load().ata_lower_aat(self._h, int(m), int(n), A.data_ptr(), _ld(A), C.data_ptr(), _ld(C),
                                      int(dtype), _stream_ptr(stream)))
        if rc != 0:
            raise AtaError(rc, f"ata_lower_aat [{self.last_error()}]")

    def batched_ptr(self, ms, ns, A_ptrs, ldas, C_ptrs, ldcs, dtype, stream=None) -> int:
        count = len(ms)
        I64 = ctypes.c_int64 * count
        VP = ctypes.c_void_p * count
        return int(load().ata_batched(self._h, count, I64(*ms), I64(*ns), VP(*A_ptrs), I64(*ldas),
                                      VP(*C_ptrs), I64(*ldcs), int(dtype), _stream_ptr(stream)))

    def batched_dev_ptr(self, ms, ns, A_table_ptr, ldas, C_table_ptr, ldcs, dtype, stream=None) -> int:
        """ata_batched_dev: A_table_ptr / C_table_ptr are device addresses of
        arrays of len(ms) device pointers (e.g. int64 CUDA tensors)."""
        count = len(ms)
        I64 = ctypes.c_int64 * count
        return int(load().ata_batched_dev(self._h, count, I64(*ms), I64(*ns), A_table_ptr, I64(*ldas), C_table_ptr,
                                          I64(*ldcs), int(dtype), _stream_ptr(stream)))

    def batched_dev_call(self, ms, ns, A_table_ptr, ldas, C_table_ptr, ldcs, dtype, stream=None):
        """A zero-argument callable that runs ata_batched_dev with these
        arguments, marshalled once (for calls repeated on the same shapes and
        pointer tables; the tables' contents may change between calls)."""
        count = len(ms)
        I64 = ctypes.c_int64 * count
        args = (self._h, count, I64(*ms), I64(*ns), ctypes.c_void_p(A_table_ptr), I64(*ldas),
                ctypes.c_void_p(C_table_ptr), I64(*ldcs), int(dtype), _stream_ptr(stream))
        fn = load().ata_batched_dev

        def call():
            rc = int(fn(*args))
            if rc != 0:
                raise AtaError(rc, f"ata_batched_dev [{self.last_error()}]")
        return call

    def batched(self, As, Cs, dtype, stream=None):
        """low(C_i) <- low(A_i^T A_i) for lists of row-major CUDA tensors in one
        persistent launch (ata_batched)."""
        if len(As) != len(Cs):
            raise ValueError("As and Cs must have the same length")
        for A, C in zip(As, Cs):
            _check_rowmajor(A, C)
        ms = [int(A.shape[0]) for A in As]
        ns = [int(A.shape[1]) for A in As]
        ldas = [max(_ld(A) if A.shape[0] else 1, n, 1) for A, n in zip(As, ns)]
        ldcs = [max(_ld(C) if C.shape[0] else 1, n, 1) for C, n in zip(Cs, ns)]
        rc = self.batched_ptr(ms, ns, [A.data_ptr() for A in As], ldas, [C.data_ptr() for C in Cs], ldcs,
                              dtype, stream)
        if rc != 0:
            raise AtaError(rc, f"ata_batched [{self.last_error()}]")

    def tune(self, A, C, dtype, stream=None, budget_ms: float = 3000.0) -> dict:
        """ata_tune on row-major CUDA tensors A (m x n) and C (n x n): time the
        candidate plans, keep the fastest for this shape, leave low(A^T A) in C."""
        m, n = A.shape
        out = (ctypes.c_int64 * 4)()
        _check_rowmajor(A, C)
        rc = int(load().ata_tune(self._h, int(m), int(n), A.data_ptr(), _ld(A), C.data_ptr(), _ld(C),
                                 int(dtype), _stream_ptr(stream), float(budget_ms), out))
        if rc != 0:
            raise AtaError(rc, f"ata_tune [{self.last_error()}]")
        return {"cutoff": out[0], "depth": out[1], "strassen_min": out[2], "candidates": out[3]}

    def tune_clear(self):
        _check(load().ata_tune_clear(self._h), "ata_tune_clear")

    def set_timing(self, enable: bool = True):
        _check(load().ata_set_timing(self._h, 1 if enable else 0), "ata_set_timing")

    def phase_times(self) -> list:
        """[colmax, prep, leaf, combine] device milliseconds of the last call."""
        out = (ctypes.c_double * 4)()
        _check(load().ata_phase_times(self._h, out), "ata_phase_times")
        return [float(v) for v in out]

    def check_wait_timeout(self, budget_ns: int, stream=None) -> int:
        """ata_check_wait_timeout: a bounded device wait on a barrier nothing
        completes; returns the launch status (the timeout itself is reported
        by the next sync())."""
        return int(load().ata_check_wait_timeout(self._h, int(budget_ns), _stream_ptr(stream)))

    def sync(self, stream=None) -> int:
        return int(load().ata_sync(self._h, _stream_ptr(stream)))

    def close(self):
        if self._h:
            load().ata_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
