"""GB300-native dose-deposition SpMV (arXiv 2103.09683), Python binding.

Argument marshalling over the C ABI of libdose.so (include/dose.h): every step
of the dose calculation runs in the library's CUDA kernels.  PyTorch provides
device memory, streams, CUDA graphs and autograd plumbing only.  There is no
CPU fallback: if the library is missing, loading raises.

    import paper_2103_09683_gb300 as dose
    A = dose.DoseMatrix.from_csr(row_ptr, col, values_f64=val, ncols=nc, fmt="u16")
    d = A.spmv(x)                      # d = A x          (Sec. II-A)
    g = A.adjoint(r)                   # g = A^T r
    f, g = A.fwd_adj_quadratic(x, p, w)   # one pass: d, f, gradient
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import _build

__all__ = ["build", "load", "DoseMatrix", "DoseError", "FORMATS", "spmv_batched", "adjoint_noalloc", "dose_spmv",
           "QuadraticDoseObjective", "pg_solve", "PGSolver", "encode_host", "library_path", "selftest_bounded_wait",
           "ScenarioSet"]

FORMATS = {"u16": 0, "bf16": 1, "fp8": 2, "f16": 3, "f32": 4}
_NO_SCALES = ("bf16", "f16", "f32")
_VAL_NP = {"fp8": np.uint8, "f32": np.uint32}      # stored value dtype (default uint16)
CREATE_COMPENSATED = 0x1
CREATE_U16_INDEX = 0x2
CREATE_SELL = 0x4
SPMV_F64_NATIVE = 0x1
ROBUST_MODES = {"expected": 0, "worst": 1}
_STATUS = {0: "DOSE_OK", 1: "DOSE_ERR_INVALID_ARG", 2: "DOSE_ERR_OOM", 3: "DOSE_ERR_CUDA",
           4: "DOSE_ERR_UNSUPPORTED", 5: "DOSE_ERR_TIMEOUT", 6: "DOSE_ERR_IO", 7: "DOSE_ERR_BOUNDS"}


class DoseError(RuntimeError):
    """A libdose call returned an error status."""

    def __init__(self, status: int, message: str):
        super().__init__(f"{_STATUS.get(status, status)}: {message}")
        self.status = status


class _Desc(ctypes.Structure):
    _fields_ = [("nrows", ctypes.c_uint32), ("ncols", ctypes.c_uint32), ("nnz", ctypes.c_uint64),
                ("row_ptr", ctypes.c_void_p), ("col_idx", ctypes.c_void_p), ("fmt", ctypes.c_int),
                ("values", ctypes.c_void_p), ("scales", ctypes.c_void_p),
                ("values_f64", ctypes.c_void_p), ("on_device", ctypes.c_int)]


class Tuning(ctypes.Structure):
    """Schedule knobs (0 = default); see dose_tuning in include/dose.h."""
    _fields_ = [("tile_nnz", ctypes.c_uint32), ("tile_rows", ctypes.c_uint32),
                ("coop_nnz", ctypes.c_uint32), ("lane_target", ctypes.c_uint32),
                ("stages", ctypes.c_uint32), ("consumer_warps", ctypes.c_uint32),
                ("l2_prefetch", ctypes.c_uint32),
                ("adj_tile_nnz", ctypes.c_uint32), ("adj_tile_rows", ctypes.c_uint32),
                ("adj_stages", ctypes.c_uint32), ("adj_forward_warps", ctypes.c_uint32),
                ("adj_scatter_warps", ctypes.c_uint32), ("adj_l2_prefetch", ctypes.c_uint32),
                ("row_order", ctypes.c_uint32), ("adj_row_order", ctypes.c_uint32),
                ("sell_sigma", ctypes.c_uint32),
                ("adj_layout", ctypes.c_uint32), ("rg_tile_union", ctypes.c_uint32),
                ("rg_tile_rows", ctypes.c_uint32), ("rg_stages", ctypes.c_uint32), ("rg_warps", ctypes.c_uint32),
                ("rg_l2_prefetch", ctypes.c_uint32), ("fwd_layout", ctypes.c_uint32)]

    def as_dict(self):
        return {k: int(getattr(self, k)) for k, _ in self._fields_}


class _Info(ctypes.Structure):
    _fields_ = [("nrows", ctypes.c_uint32), ("ncols", ctypes.c_uint32), ("nnz", ctypes.c_uint64),
                ("fmt", ctypes.c_uint32), ("flags", ctypes.c_uint32),
                ("n_stages", ctypes.c_uint32), ("n_coop_rows", ctypes.c_uint32),
                ("lanes_hist", ctypes.c_uint32 * 6), ("grid", ctypes.c_uint32),
                ("block", ctypes.c_uint32), ("adj_n_stages", ctypes.c_uint32),
                ("adj_block_fused", ctypes.c_uint32), ("adj_block_adjoint", ctypes.c_uint32),
                ("max_row_len", ctypes.c_uint32), ("adj_window", ctypes.c_uint32),
                ("fwd_window", ctypes.c_uint32), ("device_bytes", ctypes.c_uint64), ("spmv_bytes", ctypes.c_uint64),
                ("adjoint_bytes", ctypes.c_uint64), ("fused_bytes", ctypes.c_uint64), ("spmv_f64_bytes", ctypes.c_uint64),
                ("sell_entries", ctypes.c_uint64),
                ("scale", ctypes.c_float), ("tuning", Tuning),
                ("adj_layout_fused", ctypes.c_uint32), ("adj_layout_adjoint", ctypes.c_uint32),
                ("rg_groups", ctypes.c_uint64), ("rg_union_entries", ctypes.c_uint64),
                ("rg_window", ctypes.c_uint32), ("rg_warps_fused", ctypes.c_uint32),
                ("rg_index_bytes", ctypes.c_uint32), ("rg_pad", ctypes.c_uint32), ("fingerprint", ctypes.c_uint64),
                ("spmv_layout", ctypes.c_uint32), ("pad2", ctypes.c_uint32), ("rg_spmv_bytes", ctypes.c_uint64)]


_lib = None
_lock = threading.Lock()
_P = ctypes.c_void_p
EXPORTS = {
    "dose_create_matrix": (ctypes.c_int, [_P, ctypes.c_uint, _P, _P, _P]),
    "dose_spmv": (ctypes.c_int, [_P, _P, _P, _P]),
    "dose_spmv_f64": (ctypes.c_int, [_P, _P, _P, ctypes.c_uint, _P]),
    "dose_spmv_batched": (ctypes.c_int, [_P, ctypes.c_int, _P, _P, ctypes.c_int, _P]),
    "dose_spmv_batched_plan": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, _P, _P]),
    "dose_adjoint": (ctypes.c_int, [_P, _P, _P, _P]),
    "dose_fwd_adj_quadratic": (ctypes.c_int, [_P, _P, _P, _P, _P, _P, _P, _P]),
    "dose_pg_step": (ctypes.c_int, [_P, _P, _P, _P, ctypes.c_float, _P, _P, _P]),
    "dose_destroy": (ctypes.c_int, [_P]),
    "dose_create_multibeam": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_uint, _P, _P, _P]),
    "dose_create_scenarios": (ctypes.c_int, [_P, ctypes.c_int, _P, _P]),
    "dose_destroy_scenarios": (ctypes.c_int, [_P]),
    "dose_robust_quadratic": (ctypes.c_int, [_P, ctypes.c_int, _P, _P, _P, _P, _P, _P, _P]),
    "dose_robust_pg_step": (ctypes.c_int, [_P, ctypes.c_int, _P, _P, _P, ctypes.c_float, _P, _P, _P]),
    "dose_matrix_info": (ctypes.c_int, [_P, _P]),
    "dose_set_tuning": (ctypes.c_int, [_P, _P]),
    "dose_autotune": (ctypes.c_int, [_P, _P, _P, _P]),
    "dose_autotune_cached": (ctypes.c_int, [_P, _P, ctypes.c_int, ctypes.c_uint, ctypes.c_char_p, _P, _P, _P]),
    "dose_fingerprint_host": (ctypes.c_int, [_P, ctypes.c_uint, _P]),
    "dose_autotune_cache_lookup": (ctypes.c_int, [ctypes.c_char_p, ctypes.c_char_p, ctypes.c_uint64, ctypes.c_uint,
                                                  _P, _P, _P]),
    "dose_autotune_cache_store": (ctypes.c_int, [ctypes.c_char_p, ctypes.c_char_p, ctypes.c_uint64, ctypes.c_uint,
                                                 _P, _P]),
    "dose_gpu_name": (ctypes.c_char_p, [ctypes.c_int, ctypes.c_char_p, ctypes.c_int]),
    "dose_encode_host": (ctypes.c_int, [ctypes.c_int, ctypes.c_uint32, _P, ctypes.c_uint64, _P, _P, _P]),
    "dose_device_status": (ctypes.c_int, [_P, _P]),
    "dose_adjoint_noalloc": (ctypes.c_int, [ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint64, _P, _P, ctypes.c_int,
                                            _P, _P, ctypes.c_float, _P, _P, _P]),
    "dose_selftest_bounded_wait": (ctypes.c_int, [ctypes.c_uint32, _P]),
    "dose_last_error": (ctypes.c_char_p, []),
    "dose_version": (ctypes.c_char_p, []),
}


TUNE_FORWARD, TUNE_FUSED, TUNE_BATCHED = 1, 2, 4


class _Report(ctypes.Structure):
    _fields_ = [("source", ctypes.c_int32), ("purposes", ctypes.c_uint32), ("fingerprint", ctypes.c_uint64),
                ("ms", ctypes.c_double * 3)]


def fingerprint_host(row_ptr, col, *, ncols: int, fmt: str = "u16", flags: int = 0) -> int:
    """dose_fingerprint_host: the autotune cache key dose_create_matrix gives
    this structure (host arrays; no GPU)."""
    rp = np.ascontiguousarray(row_ptr, dtype=np.uint32)
    ci = np.ascontiguousarray(col, dtype=np.uint32)
    d = _Desc(nrows=len(rp) - 1, ncols=int(ncols), nnz=len(ci), row_ptr=rp.ctypes.data, col_idx=ci.ctypes.data,
              fmt=FORMATS[fmt], on_device=0)
    out = ctypes.c_uint64()
    _check(load().dose_fingerprint_host(ctypes.byref(d), int(flags), ctypes.byref(out)))
    return out.value


def autotune_cache_lookup(path, gpu: str, fingerprint: int, purposes: int):
    """(tuning dict, [ms x3]) of a cache entry, or None (host only)."""
    t, ms, found = Tuning(), (ctypes.c_double * 3)(), ctypes.c_int()
    _check(load().dose_autotune_cache_lookup(os.fsencode(path), gpu.encode(), int(fingerprint), int(purposes),
                                             ctypes.byref(t), ms, ctypes.byref(found)))
    return (t.as_dict(), list(ms)) if found.value else None


def autotune_cache_store(path, gpu: str, fingerprint: int, purposes: int, tuning: dict, ms=(0.0, 0.0, 0.0)):
    """Add or replace a cache entry (host only)."""
    t = Tuning(**{k: int(v) for k, v in tuning.items()})
    m = (ctypes.c_double * 3)(*ms)
    _check(load().dose_autotune_cache_store(os.fsencode(path), gpu.encode(), int(fingerprint), int(purposes),
                                            ctypes.byref(t), m))


def gpu_name(device: int = 0) -> str:
    """The GPU name the autotune cache keys on."""
    buf = ctypes.create_string_buffer(256)
    return load().dose_gpu_name(int(device), buf, 256).decode()


def build(force: bool = False, debug: bool | None = None) -> str:
    """Compile libdose.so for sm_103a (nvcc) and return its path; debug (default:
    DOSE_DEBUG_CHECKS in the environment) builds libdose_debug.so instead."""
    return _build.build(force=force, debug=debug_checks() if debug is None else debug)


def library_path() -> str:
    return _build.LIB


def debug_checks() -> bool:
    """DOSE_DEBUG_CHECKS=1 in the environment selects the debug-checked library
    (kernels test their indices and record DOSE_ERR_BOUNDS instead of an
    out-of-bounds access)."""
    return os.environ.get("DOSE_DEBUG_CHECKS", "") not in ("", "0")


def load():
    """Load libdose.so (built by build()), or libdose_debug.so under
    DOSE_DEBUG_CHECKS=1; raise if it is missing."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.LIB_DEBUG if debug_checks() else _build.LIB
            if not os.path.exists(path):
                raise RuntimeError(f"{os.path.basename(path)} is not built: call paper_2103_09683_gb300.build() "
                                   "first (there is no CPU fallback)")
            lib = ctypes.CDLL(path)
            for name, (res, args) in EXPORTS.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def _val_torch(fmt):
    """torch dtype carrying the stored values' bits."""
    torch = _torch()
    return {"fp8": torch.uint8, "f32": torch.int32}.get(fmt, torch.int16)


def _check(status: int):
    if status != 0:
        msg = load().dose_last_error().decode(errors="replace")
        raise DoseError(status, msg)


def _torch():
    import torch
    return torch


def _stream_handle(stream):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _dptr(t, dtype, n=None, what="tensor"):
    """Device pointer of a contiguous CUDA tensor of the given dtype (and length)."""
    torch = _torch()
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{what} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{what} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{what} must be contiguous")
    if n is not None and t.numel() != n:
        raise ValueError(f"{what} has {t.numel()} elements, expected {n}")
    return ctypes.c_void_p(t.data_ptr()) if t.numel() else ctypes.c_void_p(0)


def selftest_bounded_wait(limit_us: int = 20000, stream=None) -> int:
    """Run the device self-test of the bounded waits; returns the status code
    (5 = DOSE_ERR_TIMEOUT, the expected result)."""
    return int(load().dose_selftest_bounded_wait(ctypes.c_uint32(limit_us), _stream_handle(stream)))


def encode_host(fmt: str, row_ptr: np.ndarray, values_f64: np.ndarray):
    """The library's own encoder (host code, no GPU): returns (codes, scales)."""
    lib = load()
    rp = np.ascontiguousarray(row_ptr, dtype=np.uint32)
    v = np.ascontiguousarray(values_f64, dtype=np.float64)
    nrows = rp.size - 1
    f = FORMATS[fmt]
    codes = np.empty(v.size, dtype=_VAL_NP.get(fmt, np.uint16))
    scales = np.empty(nrows if fmt == "fp8" else 1, dtype=np.float32)
    _check(lib.dose_encode_host(f, nrows, rp.ctypes.data, v.size, v.ctypes.data if v.size else None,
                                codes.ctypes.data if codes.size else None, scales.ctypes.data))
    return codes, (None if fmt in _NO_SCALES else scales)


class DoseMatrix:
    """A dose-deposition matrix resident on the GPU (library-owned handle)."""

    def __init__(self, handle, nrows, ncols, nnz, fmt):
        self._h = ctypes.c_void_p(handle)
        self.nrows, self.ncols, self.nnz, self.fmt = nrows, ncols, nnz, fmt

    # ---- construction
    @classmethod
    def from_csr(cls, row_ptr, col, *, ncols: int, fmt: str = "u16", values=None, scales=None,
                 values_f64=None, compensated: bool = False, index16: bool = False, sell: bool = False,
                 tuning: dict | None = None, stream=None):
        """Create from host (numpy) or device (torch CUDA) CSR arrays.

        Pass either encoded `values` (+ `scales`) in the stored format, or
        `values_f64` (host) to let the library encode.  `compensated`: Dot2
        accumulation on rows longer than 128 entries; `index16`: the dose SpMV
        reads 16-bit column indices (ncols <= 65536); `sell`: dose_spmv runs on a
        SELL-32-sigma copy (tuning sell_sigma).
        """
        torch = _torch()
        lib = load()
        on_dev = isinstance(row_ptr, torch.Tensor) and row_ptr.is_cuda
        keep = []

        def host(a, dt):
            a = np.ascontiguousarray(a, dtype=dt)
            keep.append(a)
            return a.ctypes.data if a.size else None

        def dev(a, dt, what):
            p = _dptr(a, dt, what=what)
            keep.append(a)
            return p.value

        nrows = int(row_ptr.shape[0]) - 1
        nnz = int(col.shape[0])
        d = _Desc()
        d.nrows, d.ncols, d.nnz, d.fmt = nrows, int(ncols), nnz, FORMATS[fmt]
        d.on_device = 1 if on_dev else 0
        vdt_np = _VAL_NP.get(fmt, np.uint16)
        if on_dev:
            d.row_ptr = dev(row_ptr, torch.int32, "row_ptr") if row_ptr.dtype == torch.int32 else \
                dev(row_ptr.view(torch.int32), torch.int32, "row_ptr")
            d.col_idx = dev(col if col.dtype == torch.int32 else col.view(torch.int32), torch.int32, "col")
            if values is None:
                raise ValueError("device CSR needs encoded values")
            vt = _val_torch(fmt)
            d.values = dev(values if values.dtype == vt else values.view(vt), vt, "values")
            if fmt not in _NO_SCALES:
                d.scales = dev(scales, torch.float32, "scales")
        else:
            d.row_ptr = host(row_ptr, np.uint32)
            d.col_idx = host(col, np.uint32)
            if values is not None:
                d.values = host(values, vdt_np)
                if fmt not in _NO_SCALES:
                    d.scales = host(np.asarray(scales, dtype=np.float32).reshape(-1), np.float32)
            elif values_f64 is not None:
                d.values_f64 = host(values_f64, np.float64)
            else:
                raise ValueError("give values (+scales) or values_f64")
        t = None
        if tuning:
            t = Tuning(**{k: int(v) for k, v in tuning.items()})
        out = ctypes.c_void_p()
        stream_h = _stream_handle(stream) if torch.cuda.is_available() else ctypes.c_void_p(0)
        flags = ((CREATE_COMPENSATED if compensated else 0) | (CREATE_U16_INDEX if index16 else 0) |
                 (CREATE_SELL if sell else 0))
        _check(lib.dose_create_matrix(ctypes.byref(d), flags,
                                      ctypes.byref(t) if t is not None else None, stream_h,
                                      ctypes.byref(out)))
        return cls(out.value, nrows, int(ncols), nnz, fmt)

    @classmethod
    def from_multibeam(cls, beams, *, fmt: str = "u16", compensated: bool = False, index16: bool = False,
                       tuning: dict | None = None, stream=None):
        """One handle for a plan of several beams on one voxel grid
        (dose_create_multibeam): columns are the beams' spots in beam order, so
        spmv([x_1; ...; x_B]) is the total dose sum_b A_b x_b.  beams: host
        (numpy) tuples (row_ptr, col, ncols, values_f64) or, for BF16/F16/F32
        (U16 with one scale), (row_ptr, col, ncols, values, scales)."""
        torch = _torch()
        lib = load()
        keep = []

        def host(a, dt):
            a = np.ascontiguousarray(a, dtype=dt)
            keep.append(a)
            return a.ctypes.data if a.size else None

        descs = (_Desc * len(beams))()
        nrows = None
        for d, bm in zip(descs, beams):
            rp, col, nc = bm[0], bm[1], int(bm[2])
            d.nrows, d.ncols, d.nnz, d.fmt = len(rp) - 1, nc, len(col), FORMATS[fmt]
            nrows = d.nrows
            d.row_ptr, d.col_idx = host(rp, np.uint32), host(col, np.uint32)
            if len(bm) == 4:
                d.values_f64 = host(bm[3], np.float64)
            else:
                d.values = host(bm[3], _VAL_NP.get(fmt, np.uint16))
                if fmt not in _NO_SCALES:
                    d.scales = host(np.asarray(bm[4], dtype=np.float32).reshape(-1), np.float32)
            d.on_device = 0
        t = Tuning(**{k: int(v) for k, v in tuning.items()}) if tuning else None
        out = ctypes.c_void_p()
        stream_h = _stream_handle(stream) if torch.cuda.is_available() else ctypes.c_void_p(0)
        flags = (CREATE_COMPENSATED if compensated else 0) | (CREATE_U16_INDEX if index16 else 0)
        _check(lib.dose_create_multibeam(descs, len(beams), flags, ctypes.byref(t) if t is not None else None,
                                         stream_h, ctypes.byref(out)))
        return cls(out.value, nrows, sum(int(b[2]) for b in beams), sum(len(b[1]) for b in beams), fmt)

    def close(self):
        if self._h and self._h.value:
            load().dose_destroy(self._h)
            self._h = ctypes.c_void_p(0)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def handle(self):
        return self._h

    # ---- compute (asynchronous on the current or given stream)
    def spmv(self, x, d=None, stream=None):
        """d = A x.  x: CUDA float32 [ncols]; d (optional): CUDA float32 [nrows]."""
        torch = _torch()
        if d is None:
            d = torch.empty(self.nrows, dtype=torch.float32, device=x.device)
        _check(load().dose_spmv(self._h, _dptr(x, torch.float32, self.ncols, "x"),
                                _dptr(d, torch.float32, self.nrows, "d"), _stream_handle(stream)))
        return d

    def spmv_f64(self, x, d=None, native: bool = False, stream=None):
        """d = A x with FP64 vectors (the paper's Half/double interface).
        x: CUDA float64 [ncols]; d (optional): CUDA float64 [nrows].  `native`:
        FP64 FMA accumulation instead of double-float pairs."""
        torch = _torch()
        if d is None:
            d = torch.empty(self.nrows, dtype=torch.float64, device=x.device)
        _check(load().dose_spmv_f64(self._h, _dptr(x, torch.float64, self.ncols, "x"),
                                    _dptr(d, torch.float64, self.nrows, "d"),
                                    SPMV_F64_NATIVE if native else 0, _stream_handle(stream)))
        return d

    def adjoint(self, r, g=None, stream=None):
        """g = A^T r.  r: CUDA float32 [nrows]."""
        torch = _torch()
        if g is None:
            g = torch.empty(self.ncols, dtype=torch.float32, device=r.device)
        _check(load().dose_adjoint(self._h, _dptr(r, torch.float32, self.nrows, "r"),
                                   _dptr(g, torch.float32, self.ncols, "g"), _stream_handle(stream)))
        return g

    def fwd_adj_quadratic(self, x, p, w, d=None, f=None, g=None, stream=None, want_d=False):
        """One pass: f = sum w (Ax - p)^2 (FP64 device scalar) and g = grad f."""
        torch = _torch()
        dev = x.device
        if f is None:
            f = torch.empty(1, dtype=torch.float64, device=dev)
        if g is None:
            g = torch.empty(self.ncols, dtype=torch.float32, device=dev)
        if d is None and want_d:
            d = torch.empty(self.nrows, dtype=torch.float32, device=dev)
        dptr = _dptr(d, torch.float32, self.nrows, "d") if d is not None else None
        _check(load().dose_fwd_adj_quadratic(
            self._h, _dptr(x, torch.float32, self.ncols, "x"), _dptr(p, torch.float32, self.nrows, "p"),
            _dptr(w, torch.float32, self.nrows, "w"), dptr, _dptr(f, torch.float64, 1, "f"),
            _dptr(g, torch.float32, self.ncols, "g"), _stream_handle(stream)))
        return (f, g, d) if want_d else (f, g)

    def pg_step(self, x, p, w, eta: float, f=None, g=None, stream=None):
        """x <- max(0, x - eta grad f(x)) in place; returns f(x) before the step."""
        torch = _torch()
        if f is None:
            f = torch.empty(1, dtype=torch.float64, device=x.device)
        gptr = _dptr(g, torch.float32, self.ncols, "g") if g is not None else None
        _check(load().dose_pg_step(self._h, _dptr(x, torch.float32, self.ncols, "x"),
                                   _dptr(p, torch.float32, self.nrows, "p"),
                                   _dptr(w, torch.float32, self.nrows, "w"), ctypes.c_float(eta),
                                   _dptr(f, torch.float64, 1, "f"), gptr, _stream_handle(stream)))
        return f

    # ---- schedule
    def info(self) -> dict:
        inf = _Info()
        _check(load().dose_matrix_info(self._h, ctypes.byref(inf)))
        out = {k: getattr(inf, k) for k, _ in _Info._fields_ if k not in ("lanes_hist", "tuning")}
        out["lanes_hist"] = list(inf.lanes_hist)
        out["tuning"] = inf.tuning.as_dict()
        return out

    def set_tuning(self, **knobs):
        t = Tuning(**{k: int(v) for k, v in knobs.items()})
        _check(load().dose_set_tuning(self._h, ctypes.byref(t)))

    def autotune(self, x=None, stream=None, *, mode=None, purposes=("forward", "fused"), cache=None) -> dict:
        """Choose the schedule knobs by timing candidates on this GPU.  mode=None:
        dose_autotune (sweep, no cache); "off" | "cached" | "full" | "env":
        dose_autotune_cached with the JSON cache at `cache` (None = the library's
        default path).  Returns the knobs in effect; with a mode, also
        "source" ("off", "cache" or "sweep") and the sweep's times in ms."""
        torch = _torch()
        t = Tuning()
        xp = None if x is None else _dptr(x, torch.float32, self.ncols, "x")
        if mode is None:
            _check(load().dose_autotune(self._h, xp, _stream_handle(stream), ctypes.byref(t)))
            return t.as_dict()
        modes = {"env": -1, "off": 0, "cached": 1, "full": 2}
        bits = {"forward": TUNE_FORWARD, "fused": TUNE_FUSED, "batched": TUNE_BATCHED}
        rep = _Report()
        _check(load().dose_autotune_cached(self._h, xp, modes[mode], sum(bits[p] for p in purposes),
                                           None if cache is None else os.fsencode(cache), _stream_handle(stream),
                                           ctypes.byref(t), ctypes.byref(rep)))
        out = t.as_dict()
        out.update(source=("off", "cache", "sweep")[rep.source], fingerprint=rep.fingerprint,
                   ms_forward=rep.ms[0], ms_fused=rep.ms[1], ms_batched=rep.ms[2])
        return out

    def device_status(self, stream=None):
        """Synchronise and raise DoseError if a kernel recorded a failure."""
        _check(load().dose_device_status(self._h, _stream_handle(stream)))


def adjoint_noalloc(row_ptr, col, values, r, *, ncols: int, fmt: str = "u16", scale: float = 1.0,
                    row_scales=None, g=None, stream=None):
    """g = A^T r from caller-held device CSR arrays, allocating no device memory
    in the library (dose_adjoint_noalloc).  All arrays are CUDA tensors: row_ptr
    and col int32 (bit patterns of uint32), values int16 (u16/bf16/f16 codes), int32 (f32 bits) or
    uint8 (fp8), r float32; g (optional) float32 [ncols]."""
    torch = _torch()
    nrows = int(row_ptr.numel()) - 1
    nnz = int(col.numel())
    if g is None:
        g = torch.empty(ncols, dtype=torch.float32, device=r.device)
    vt = _val_torch(fmt)
    rs = _dptr(row_scales, torch.float32, nrows, "row_scales") if fmt == "fp8" else None
    _check(load().dose_adjoint_noalloc(
        nrows, int(ncols), nnz, _dptr(row_ptr, torch.int32, nrows + 1, "row_ptr"), _dptr(col, torch.int32, nnz, "col"),
        FORMATS[fmt], _dptr(values, vt, nnz, "values"), rs, ctypes.c_float(scale),
        _dptr(r, torch.float32, nrows, "r"), _dptr(g, torch.float32, int(ncols), "g"), _stream_handle(stream)))
    return g


def spmv_batched(mats, Xs, Ds=None, stream=None):
    """D_m = A_m X_m for all m in one launch.  X_m: CUDA float32 [ncols_m, nvec]."""
    torch = _torch()
    n = len(mats)
    if n == 0:
        return []
    nvec = int(Xs[0].shape[1]) if Xs[0].dim() == 2 else 1
    if Ds is None:
        Ds = [torch.empty((A.nrows, nvec), dtype=torch.float32, device=Xs[0].device) for A in mats]
    hs = (ctypes.c_void_p * n)(*[A.handle.value for A in mats])
    xp = (ctypes.c_void_p * n)(*[_dptr(X, torch.float32, A.ncols * nvec, "X").value
                                 for A, X in zip(mats, Xs)])
    dp = (ctypes.c_void_p * n)(*[_dptr(D, torch.float32, A.nrows * nvec, "D").value
                                 for A, D in zip(mats, Ds)])
    _check(load().dose_spmv_batched(hs, n, xp, dp, nvec, _stream_handle(stream)))
    return Ds


def spmv_batched_plan(mats, nvec):
    """(layout, launches) of dose_spmv_batched for these matrices: layout 2 = row
    groups, 1 = CSR; launches = kernels per call."""
    n = len(mats)
    hs = (ctypes.c_void_p * max(n, 1))(*[A.handle.value for A in mats])
    lay, nl = ctypes.c_int(), ctypes.c_int()
    _check(load().dose_spmv_batched_plan(hs, n, int(nvec), ctypes.byref(lay), ctypes.byref(nl)))
    return lay.value, nl.value


class ScenarioSet:
    """Matrices of one shape under several uncertainty scenarios, with their
    probabilities (dose_create_scenarios); robust objective and PG step."""

    def __init__(self, mats, prob=None):
        lib = load()
        self.mats = list(mats)   # the handles must outlive the set
        self.nrows, self.ncols = self.mats[0].nrows, self.mats[0].ncols
        n = len(self.mats)
        hs = (ctypes.c_void_p * n)(*[A.handle.value for A in self.mats])
        pr = None if prob is None else np.ascontiguousarray(prob, dtype=np.float64)
        out = ctypes.c_void_p()
        _check(lib.dose_create_scenarios(hs, n, pr.ctypes.data if pr is not None else None, ctypes.byref(out)))
        self._h = out

    def robust_quadratic(self, x, p, w, mode: str = "expected", f=None, g=None, f_scen=None, stream=None):
        """(F, g[, f_s]) of the robust quadratic objective (device tensors)."""
        torch = _torch()
        dev = x.device
        f = torch.empty(1, dtype=torch.float64, device=dev) if f is None else f
        g = torch.empty(self.ncols, dtype=torch.float32, device=dev) if g is None else g
        _check(load().dose_robust_quadratic(
            self._h, ROBUST_MODES[mode], _dptr(x, torch.float32, self.ncols, "x"),
            _dptr(p, torch.float32, self.nrows, "p"), _dptr(w, torch.float32, self.nrows, "w"),
            _dptr(f, torch.float64, 1, "f"),
            _dptr(f_scen, torch.float64, len(self.mats), "f_scen") if f_scen is not None else None,
            _dptr(g, torch.float32, self.ncols, "g"), _stream_handle(stream)))
        return (f, g, f_scen) if f_scen is not None else (f, g)

    def pg_step(self, x, p, w, eta: float, mode: str = "expected", f=None, g=None, stream=None):
        """F at x, then x <- max(0, x - eta g) in place; returns F (device double)."""
        torch = _torch()
        f = torch.empty(1, dtype=torch.float64, device=x.device) if f is None else f
        _check(load().dose_robust_pg_step(
            self._h, ROBUST_MODES[mode], _dptr(x, torch.float32, self.ncols, "x"),
            _dptr(p, torch.float32, self.nrows, "p"), _dptr(w, torch.float32, self.nrows, "w"),
            ctypes.c_float(eta), _dptr(f, torch.float64, 1, "f"),
            _dptr(g, torch.float32, self.ncols, "g") if g is not None else None, _stream_handle(stream)))
        return f

    def close(self):
        if self._h and self._h.value:
            load().dose_destroy_scenarios(self._h)
            self._h = ctypes.c_void_p(0)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------------ autograd

def _autograd():
    torch = _torch()

    class _DoseSpMV(torch.autograd.Function):
        """d = A x with backward g = A^T grad_d (the hand-written adjoint kernel)."""

        @staticmethod
        def forward(ctx, x, A):
            ctx.A = A
            return A.spmv(x.contiguous())

        @staticmethod
        def backward(ctx, grad_d):
            return ctx.A.adjoint(grad_d.contiguous().float()), None

    class _Quadratic(torch.autograd.Function):
        """f(x) = sum w (A x - p)^2 in one fused pass; backward scales the saved gradient."""

        @staticmethod
        def forward(ctx, x, A, p, w):
            f, g = A.fwd_adj_quadratic(x.contiguous(), p, w)
            ctx.save_for_backward(g)
            return f.reshape(())

        @staticmethod
        def backward(ctx, grad_f):
            (g,) = ctx.saved_tensors
            return (grad_f.to(g.dtype) * g), None, None, None

    return _DoseSpMV, _Quadratic


_AG = None


def dose_spmv(A: DoseMatrix, x):
    """Differentiable d = A x (torch.autograd): backward runs dose_adjoint."""
    global _AG
    if _AG is None:
        _AG = _autograd()
    return _AG[0].apply(x, A)


def QuadraticDoseObjective(A: DoseMatrix, x, p, w):
    """Differentiable f = sum_i w_i (d_i - p_i)^2 (FP64 scalar), d = A x."""
    global _AG
    if _AG is None:
        _AG = _autograd()
    return _AG[1].apply(x, A, p, w)


class PGSolver:
    """Projected-gradient iterations x <- max(0, x - eta grad f) captured once in a
    CUDA graph (torch.cuda.CUDAGraph) and replayed: `iters` dose_pg_step calls per
    replay, f of every step written to a device buffer."""

    def __init__(self, A: DoseMatrix, x, p, w, eta: float, iters: int, use_graph: bool = True):
        torch = _torch()
        self.A, self.x, self.p, self.w, self.eta, self.iters = A, x, p, w, float(eta), int(iters)
        self.f_hist = torch.zeros(self.iters, dtype=torch.float64, device=x.device)
        self.steps_done = 0
        self.graph = None
        if use_graph:
            s = torch.cuda.Stream()
            s.wait_stream(torch.cuda.current_stream())
            self.graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(self.graph, stream=s):
                self._enqueue(s)
            torch.cuda.current_stream().wait_stream(s)

    def _enqueue(self, stream):
        for k in range(self.iters):
            self.A.pg_step(self.x, self.p, self.w, self.eta, f=self.f_hist[k:k + 1], stream=stream)

    def run(self):
        """Run `iters` steps (one graph launch when captured); returns f_hist."""
        if self.graph is not None:
            self.graph.replay()
        else:
            self._enqueue(None)
        self.steps_done += self.iters
        return self.f_hist

    def checkpoint(self, path: str):
        """Save the optimiser state (x, steps done, eta, the last run's f) to an .npz."""
        save_pg_state(path, self.x, self.steps_done, self.eta, self.f_hist)

    def resume(self, path: str):
        """Load a checkpoint into this solver: x is overwritten in place (the
        captured graph keeps pointing at it); returns the steps done."""
        self.steps_done, _ = load_pg_state(path, self.x, self.eta)
        return self.steps_done


def save_pg_state(path: str, x, steps_done: int, eta: float, f_hist=None):
    """Projected-gradient state as an .npz: x (float32), the number of steps
    done, the step size and the f values of the last run (float64)."""
    xs = x.detach().to("cpu").numpy().astype(np.float32, copy=True)
    fh = (f_hist.detach().to("cpu").numpy().astype(np.float64, copy=True) if f_hist is not None
          else np.zeros(0, dtype=np.float64))
    np.savez(path, x=xs, steps_done=np.int64(steps_done), eta=np.float64(eta), f_hist=fh)


def load_pg_state(path: str, x, eta: float | None = None):
    """Copy a saved x into the tensor x (same length, in place) and return
    (steps done, f history).  With eta given, the saved step size must match."""
    with np.load(path) as z:
        xs, steps, eta0, fh = z["x"], int(z["steps_done"]), float(z["eta"]), z["f_hist"]
    if xs.size != x.numel():
        raise ValueError(f"checkpoint has {xs.size} spot weights, x has {x.numel()}")
    if eta is not None and float(eta) != eta0:
        raise ValueError(f"checkpoint was taken with eta = {eta0}, not {eta}")
    torch = _torch()
    x.copy_(torch.from_numpy(xs).to(x.device, x.dtype).reshape(x.shape))
    return steps, fh


def pg_solve(A: DoseMatrix, x, p, w, eta: float, iters: int = 100, use_graph: bool = True):
    """Run `iters` projected-gradient steps on x (in place); returns f per step."""
    return PGSolver(A, x, p, w, eta, iters, use_graph).run()
