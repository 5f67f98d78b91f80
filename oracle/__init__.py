"""FP64 CPU oracle of the dose calculation -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The CUDA library (paper_2103_09683_gb300)
never imports it, and the two share no code: the oracle decodes, encodes and
multiplies with its own plain C loops (dose_oracle.c), in FP64.

Paper passages followed:
  * d = A x with A the dose-deposition matrix, rows = voxels, columns = spots
    (Sec. II-A); A is fixed during optimisation, only x changes.
  * One output per row equal to the row's dot product over its CSR entries
    (Sec. III, Listing 1); CSR layout with value, column-index and row-start
    arrays (Sec. II-C).
  * Memory-traffic model 6*nnz + 12*nr + 8*nc bytes and 2*nnz flops for the
    half-value / double-vector kernel, giving OI 0.332 for liver beam 1 (Sec. V).
  * 16-bit stored values with FP32/FP64 vectors (Sec. II-D); IEEE half values
    with double vectors and double accumulation, the paper's own kernel (Sec. IV).
The objective, its gradient and the projected-gradient step are the quadratic
dose objective of the optimisation the paper motivates (Sec. I, Sec. II-A).

Every function here is pinned by the ``-m "not gpu"`` tests against brute force,
closed forms or values the paper prints.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_SRC = os.path.join(_HERE, "dose_oracle.c")
_lock = threading.Lock()
_lib = None

U16_SCALE, BF16, FP8E4M3_ROWSCALE, F16, F32 = 0, 1, 2, 3, 4
FORMAT_NAMES = {U16_SCALE: "u16", BF16: "bf16", FP8E4M3_ROWSCALE: "fp8", F16: "f16", F32: "f32"}


def build(force: bool = False) -> str:
    """Compile dose_oracle.c (plain C, -O2, no fast-math, no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
                               _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _SO)
    return _SO


_P = ctypes.c_void_p
_U32, _U64, _F64, _F32, _U8, _U16 = (ctypes.c_uint32, ctypes.c_uint64, ctypes.c_double,
                                     ctypes.c_float, ctypes.c_uint8, ctypes.c_uint16)


def _load():
    global _lib
    with _lock:
        if _lib is None:
            # DOSE_ORACLE_SO lets the mutation tests load a deliberately broken
            # copy of the oracle and check that the pins reject it.
            lib = ctypes.CDLL(os.environ.get("DOSE_ORACLE_SO") or build())
            sig = {
                "oracle_fp8_e4m3_value": (_F64, [_U8]),
                "oracle_bf16_value": (_F64, [_U16]),
                "oracle_fp8_e4m3_nearest": (_U8, [_F64]),
                "oracle_bf16_round": (_U16, [_F64]),
                "oracle_f16_value": (_F64, [_U16]),
                "oracle_f16_round": (_U16, [_F64]),
                "oracle_encode_f16": (ctypes.c_int, [_U64, _P, _P]),
                "oracle_encode_f32": (ctypes.c_int, [_U64, _P, _P]),
                "oracle_decode_f32": (None, [_U64, _P, _P]),
                "oracle_decode_f16": (None, [_U64, _P, _P]),
                "oracle_encode_u16": (ctypes.c_int, [_U64, _P, _P, _P]),
                "oracle_encode_bf16": (ctypes.c_int, [_U64, _P, _P]),
                "oracle_encode_fp8_rowscale": (ctypes.c_int, [_U32, _P, _P, _P, _P]),
                "oracle_decode_u16": (None, [_U64, _P, _F32, _P]),
                "oracle_decode_bf16": (None, [_U64, _P, _P]),
                "oracle_decode_fp8_rowscale": (None, [_U32, _P, _P, _P, _P]),
                "oracle_spmv": (None, [_U32, _P, _P, _P, _P, _P]),
                "oracle_spmv_rows": (None, [_U64, _P, _P, _P, _P, _P, _P]),
                "oracle_spmm": (None, [_U32, _U32, _P, _P, _P, _P, _P]),
                "oracle_spmv_t": (None, [_U32, _U32, _P, _P, _P, _P, _P]),
                "oracle_abs_spmv_t": (None, [_U32, _U32, _P, _P, _P, _P, _P]),
                "oracle_objective": (_F64, [_U32, _P, _P, _P, _P]),
                "oracle_fgrad": (_F64, [_U32, _U32, _P, _P, _P, _P, _P, _P, _P, _P]),
                "oracle_pg": (ctypes.c_int, [_U32, _U32, _P, _P, _P, _P, _P, _F64, _U32, _P, _P]),
                "oracle_norm2_sq": (_F64, [_U32, _U32, _P, _P, _P, _U32]),
                "oracle_robust_combine": (_F64, [_U32, _U32, ctypes.c_int, _P, _P, _P, _P, _P]),
            }
            for name, (res, args) in sig.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def _c(a, dtype):
    """Contiguous array of the given dtype (copy only when needed)."""
    return np.ascontiguousarray(a, dtype=dtype)


def _ptr(a):
    return a.ctypes.data if a.size else None


# ------------------------------------------------------------------ formats

def fp8_e4m3_value(code: int) -> float:
    return _load().oracle_fp8_e4m3_value(int(code))


def bf16_value(bits: int) -> float:
    return _load().oracle_bf16_value(int(bits))


def fp8_e4m3_nearest(t: float) -> int:
    return int(_load().oracle_fp8_e4m3_nearest(float(t)))


def bf16_round(v: float) -> int:
    return int(_load().oracle_bf16_round(float(v)))


def f16_value(bits: int) -> float:
    return _load().oracle_f16_value(int(bits))


def f16_round(v: float) -> int:
    return int(_load().oracle_f16_round(float(v)))


class Encoded:
    """A CSR matrix in one stored format, plus its FP64 decoded values."""

    def __init__(self, fmt, nrows, ncols, row_ptr, col, values, scales, decoded):
        self.fmt, self.nrows, self.ncols = fmt, nrows, ncols
        self.row_ptr, self.col = row_ptr, col
        self.values = values      # uint16 (u16 codes, bf16 or f16 bits), uint8 (e4m3 codes), uint32 (f32 bits)
        self.scales = scales      # float32[1] (u16), float32[nrows] (fp8) or None (bf16, f16, f32)
        self.decoded = decoded    # float64[nnz], exact value of each stored entry

    @property
    def nnz(self):
        return int(self.col.size)


def encode(csr, fmt: int) -> Encoded:
    """Encode a dosegen.CSR's FP64 values into a stored format (the readings above)."""
    lib = _load()
    rp = _c(csr.row_ptr, np.uint32)
    col = _c(csr.col, np.uint32)
    v = _c(csr.val, np.float64)
    nnz = v.size
    dec = np.empty(nnz, dtype=np.float64)
    if fmt == U16_SCALE:
        q = np.empty(nnz, dtype=np.uint16)
        s = np.zeros(1, dtype=np.float32)
        if lib.oracle_encode_u16(nnz, _ptr(v), s.ctypes.data, _ptr(q)) != 0:
            raise ValueError("u16 encoding needs non-negative values")
        lib.oracle_decode_u16(nnz, _ptr(q), float(s[0]), _ptr(dec))
        return Encoded(fmt, csr.nrows, csr.ncols, rp, col, q, s, dec)
    if fmt == BF16:
        q = np.empty(nnz, dtype=np.uint16)
        lib.oracle_encode_bf16(nnz, _ptr(v), _ptr(q))
        lib.oracle_decode_bf16(nnz, _ptr(q), _ptr(dec))
        return Encoded(fmt, csr.nrows, csr.ncols, rp, col, q, None, dec)
    if fmt == F16:
        q = np.empty(nnz, dtype=np.uint16)
        lib.oracle_encode_f16(nnz, _ptr(v), _ptr(q))
        lib.oracle_decode_f16(nnz, _ptr(q), _ptr(dec))
        return Encoded(fmt, csr.nrows, csr.ncols, rp, col, q, None, dec)
    if fmt == F32:
        q = np.empty(nnz, dtype=np.uint32)
        lib.oracle_encode_f32(nnz, _ptr(v), _ptr(q))
        lib.oracle_decode_f32(nnz, _ptr(q), _ptr(dec))
        return Encoded(fmt, csr.nrows, csr.ncols, rp, col, q, None, dec)
    if fmt == FP8E4M3_ROWSCALE:
        q = np.empty(nnz, dtype=np.uint8)
        s = np.empty(csr.nrows, dtype=np.float32)
        if lib.oracle_encode_fp8_rowscale(csr.nrows, _ptr(rp), _ptr(v), _ptr(s), _ptr(q)) != 0:
            raise ValueError("fp8 encoding needs non-negative values")
        lib.oracle_decode_fp8_rowscale(csr.nrows, _ptr(rp), _ptr(q), _ptr(s), _ptr(dec))
        return Encoded(fmt, csr.nrows, csr.ncols, rp, col, q, s, dec)
    raise ValueError(f"unknown format {fmt}")


def decode(fmt, nrows, row_ptr, values, scales) -> np.ndarray:
    """FP64 value of every stored entry."""
    lib = _load()
    rp = _c(row_ptr, np.uint32)
    nnz = int(np.asarray(values).size)
    dec = np.empty(nnz, dtype=np.float64)
    if fmt == U16_SCALE:
        q = _c(values, np.uint16)
        lib.oracle_decode_u16(nnz, _ptr(q), float(np.asarray(scales).reshape(-1)[0]), _ptr(dec))
    elif fmt == BF16:
        q = _c(values, np.uint16)
        lib.oracle_decode_bf16(nnz, _ptr(q), _ptr(dec))
    elif fmt == F16:
        q = _c(values, np.uint16)
        lib.oracle_decode_f16(nnz, _ptr(q), _ptr(dec))
    elif fmt == F32:
        q = _c(values, np.uint32)
        lib.oracle_decode_f32(nnz, _ptr(q), _ptr(dec))
    elif fmt == FP8E4M3_ROWSCALE:
        q = _c(values, np.uint8)
        s = _c(scales, np.float32)
        lib.oracle_decode_fp8_rowscale(nrows, _ptr(rp), _ptr(q), _ptr(s), _ptr(dec))
    else:
        raise ValueError(f"unknown format {fmt}")
    return dec


# ----------------------------------------------------------------- products

def spmv(nrows, row_ptr, col, a, x) -> np.ndarray:
    """d = A x in FP64 (Listing 1's row dot products; empty rows give 0)."""
    lib = _load()
    rp, cl, av, xv = _c(row_ptr, np.uint32), _c(col, np.uint32), _c(a, np.float64), _c(x, np.float64)
    d = np.empty(nrows, dtype=np.float64)
    lib.oracle_spmv(nrows, _ptr(rp), _ptr(cl), _ptr(av), _ptr(xv), _ptr(d))
    return d


def spmv_rows(rows, row_ptr, col, a, x) -> np.ndarray:
    """Selected entries d[rows] of d = A x in FP64."""
    lib = _load()
    sel = _c(rows, np.uint32)
    rp, cl, av, xv = _c(row_ptr, np.uint32), _c(col, np.uint32), _c(a, np.float64), _c(x, np.float64)
    d = np.empty(sel.size, dtype=np.float64)
    lib.oracle_spmv_rows(sel.size, _ptr(sel), _ptr(rp), _ptr(cl), _ptr(av), _ptr(xv), _ptr(d))
    return d


def spmm(nrows, row_ptr, col, a, X) -> np.ndarray:
    """D = A X in FP64 for X of shape (ncols, nvec)."""
    lib = _load()
    X = _c(X, np.float64)
    nvec = X.shape[1]
    rp, cl, av = _c(row_ptr, np.uint32), _c(col, np.uint32), _c(a, np.float64)
    D = np.empty((nrows, nvec), dtype=np.float64)
    lib.oracle_spmm(nrows, nvec, _ptr(rp), _ptr(cl), _ptr(av), _ptr(X), _ptr(D))
    return D


def spmv_t(nrows, ncols, row_ptr, col, a, r) -> np.ndarray:
    """g = A^T r in FP64, scattering rows in order."""
    lib = _load()
    rp, cl, av, rv = _c(row_ptr, np.uint32), _c(col, np.uint32), _c(a, np.float64), _c(r, np.float64)
    g = np.empty(ncols, dtype=np.float64)
    lib.oracle_spmv_t(nrows, ncols, _ptr(rp), _ptr(cl), _ptr(av), _ptr(rv), _ptr(g))
    return g


def abs_spmv_t(nrows, ncols, row_ptr, col, a, r) -> np.ndarray:
    """|A|^T |r| in FP64 (error scale for the adjoint)."""
    lib = _load()
    rp, cl, av, rv = _c(row_ptr, np.uint32), _c(col, np.uint32), _c(a, np.float64), _c(r, np.float64)
    g = np.empty(ncols, dtype=np.float64)
    lib.oracle_abs_spmv_t(nrows, ncols, _ptr(rp), _ptr(cl), _ptr(av), _ptr(rv), _ptr(g))
    return g


def objective(d, p, w):
    """(f, r): f = sum w (d-p)^2 and r = 2 w (d-p), in FP64."""
    lib = _load()
    dv, pv, wv = _c(d, np.float64), _c(p, np.float64), _c(w, np.float64)
    r = np.empty(dv.size, dtype=np.float64)
    f = lib.oracle_objective(dv.size, _ptr(dv), _ptr(pv), _ptr(wv), _ptr(r))
    return f, r


def fgrad(nrows, ncols, row_ptr, col, a, x, p, w):
    """(f(x), grad f(x)) of the quadratic dose objective in FP64."""
    lib = _load()
    rp, cl, av = _c(row_ptr, np.uint32), _c(col, np.uint32), _c(a, np.float64)
    xv, pv, wv = _c(x, np.float64), _c(p, np.float64), _c(w, np.float64)
    g = np.empty(ncols, dtype=np.float64)
    work = np.empty(2 * nrows, dtype=np.float64)
    f = lib.oracle_fgrad(nrows, ncols, _ptr(rp), _ptr(cl), _ptr(av), _ptr(xv), _ptr(pv), _ptr(wv),
                         _ptr(g), _ptr(work))
    return f, g


def multibeam_spmv(beams, xs) -> np.ndarray:
    """Total dose of a plan, d = sum_b A_b x_b over its beams on one voxel grid
    (Sec. I: the doses of multiple beams): each beam's FP64 product (spmv),
    added in beam order.  beams: list of (nrows, row_ptr, col, a)."""
    d = None
    for (nrows, rp, col, a), x in zip(beams, xs):
        db = spmv(nrows, rp, col, a, x)
        d = db if d is None else d + db
    return d


EXPECTED, WORST_CASE = 0, 1


def robust_quadratic(scenarios, x, p, w, mode, prob=None):
    """Robust quadratic dose objective over scenarios (Sec. I: uncertainty
    realisations), each scenario a matrix (nrows, ncols, row_ptr, col, a) of the
    same shape: f_s, g_s of every scenario (fgrad), combined by
    oracle_robust_combine (expected value with probabilities `prob`, default
    uniform; or worst case).  Returns (F, G, f_s, s*)."""
    lib = _load()
    S = len(scenarios)
    ncols = scenarios[0][1]
    fs = np.empty(S, dtype=np.float64)
    gs = np.empty((S, ncols), dtype=np.float64)
    for s, (nr, nc, rp, col, a) in enumerate(scenarios):
        fs[s], gs[s] = fgrad(nr, nc, rp, col, a, x, p, w)
    pr = _c(np.full(S, 1.0 / S) if prob is None else prob, np.float64)
    G = np.empty(ncols, dtype=np.float64)
    arg = ctypes.c_int32(0)
    F = lib.oracle_robust_combine(S, ncols, int(mode), _ptr(pr), _ptr(fs), gs.ctypes.data, _ptr(G),
                                  ctypes.addressof(arg))
    return F, G, fs, int(arg.value)


def pg(nrows, ncols, row_ptr, col, a, x0, p, w, eta, iters):
    """Projected gradient x <- max(0, x - eta grad f): returns (x_final, f_hist[iters])."""
    lib = _load()
    rp, cl, av = _c(row_ptr, np.uint32), _c(col, np.uint32), _c(a, np.float64)
    x = np.array(x0, dtype=np.float64, copy=True)
    pv, wv = _c(p, np.float64), _c(w, np.float64)
    fh = np.empty(iters, dtype=np.float64)
    if lib.oracle_pg(nrows, ncols, _ptr(rp), _ptr(cl), _ptr(av), _ptr(pv), _ptr(wv), float(eta),
                     iters, _ptr(x), _ptr(fh)) != 0:
        raise MemoryError("oracle_pg")
    return x, fh


def norm2_sq(nrows, ncols, row_ptr, col, a, iters=50) -> float:
    """lambda_max(A^T A) by power iteration from the all-ones vector."""
    lib = _load()
    rp, cl, av = _c(row_ptr, np.uint32), _c(col, np.uint32), _c(a, np.float64)
    return float(lib.oracle_norm2_sq(nrows, ncols, _ptr(rp), _ptr(cl), _ptr(av), iters))


def pg_step_size(nrows, ncols, row_ptr, col, a, w, iters=50) -> float:
    """eta = 1 / (2 max(w) ||A||_2^2), the projected-gradient step."""
    return 1.0 / (2.0 * float(np.max(w)) * norm2_sq(nrows, ncols, row_ptr, col, a, iters))


# ------------------------------------------------------------- byte model

def paper_traffic_bytes(nnz, nr, nc):
    """Sec. V model of the half-value / double-vector CSR SpMV: 6 nnz + 12 nr + 8 nc.

    Per entry a 2-byte value and a 4-byte column index; per row one 4-byte row
    pointer and one 8-byte output; per column one 8-byte input (infinite cache).
    """
    return 6 * nnz + 12 * nr + 8 * nc


def paper_operational_intensity(nnz, nr, nc):
    """2 nnz flops over the Sec. V byte model."""
    return 2.0 * nnz / paper_traffic_bytes(nnz, nr, nc)


def csr_storage_bytes(nnz, nr, value_bytes=2, index_bytes=4, ptr_bytes=4):
    """Storage of a CSR matrix: values + column indices + (nr+1) row pointers."""
    return (value_bytes + index_bytes) * nnz + ptr_bytes * (nr + 1)
