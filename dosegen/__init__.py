"""Seeded synthetic inputs for the dose SpMV: pencil-beam matrices, spot weights,
objective targets, and small random CSR matrices for edge-case tests.

This package is shared by the oracle-based tests, the CUDA path's tests and the
benchmark.  It holds input generation only -- none of the dose calculation's
arithmetic (no value encoding, no products, no reductions of the method).

The pencil-beam model stands in for the clinical Monte Carlo matrices of the
paper (Sec. II-A; Table I; Fig. 2): rows are voxels, columns are spots, about
70-90 % of rows are empty and non-empty rows hold tens to hundreds of entries.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass, replace

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libpencilbeam.so")
_SRC = os.path.join(_HERE, "pencilbeam.c")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the generator's C source into a shared library (gcc, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
                               "-ffp-contract=off", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _SO)
    return _SO


class _Params(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
                ("sx", ctypes.c_int32), ("sy", ctypes.c_int32),
                ("dx", ctypes.c_double), ("dy", ctypes.c_double),
                ("sigma", ctypes.c_double), ("tau", ctypes.c_double),
                ("shift_x", ctypes.c_double), ("shift_y", ctypes.c_double),
                ("seed", ctypes.c_uint64)]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.pb_count.restype = ctypes.c_int64
            lib.pb_count.argtypes = [ctypes.POINTER(_Params), ctypes.c_void_p]
            lib.pb_fill.restype = ctypes.c_int
            lib.pb_fill.argtypes = [ctypes.POINTER(_Params), ctypes.c_void_p, ctypes.c_void_p,
                                    ctypes.c_void_p]
            lib.pb_uniform_f32.restype = None
            lib.pb_uniform_f32.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_void_p]
            lib.pb_uniform_f64.restype = None
            lib.pb_uniform_f64.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_void_p]
            lib.pb_splitmix64_at.restype = ctypes.c_uint64
            lib.pb_splitmix64_at.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
            _lib = lib
    return _lib


@dataclass(frozen=True)
class Beam:
    """One pencil-beam dose-deposition matrix: grid, spot lattice, model knobs."""
    grid: tuple          # (nx, ny, nz) voxels
    lattice: tuple       # (sx, sy) spots; column j = b*sx + a
    spacing: tuple       # (dx, dy) spot spacing in voxels
    sigma: float         # lateral Gaussian sigma in voxels
    tau: float           # truncation threshold (fraction of the spot maximum)
    seed: int            # beam seed: Bragg depths of the spots
    shift: tuple = (0.0, 0.0)   # setup-shift scenario (lateral shift of spot centres)

    @property
    def nrows(self) -> int:
        return self.grid[0] * self.grid[1] * self.grid[2]

    @property
    def ncols(self) -> int:
        return self.lattice[0] * self.lattice[1]

    def _params(self) -> _Params:
        return _Params(self.grid[0], self.grid[1], self.grid[2], self.lattice[0], self.lattice[1],
                       float(self.spacing[0]), float(self.spacing[1]), float(self.sigma),
                       float(self.tau), float(self.shift[0]), float(self.shift[1]),
                       int(self.seed) & 0xFFFFFFFFFFFFFFFF)


@dataclass
class CSR:
    """A CSR matrix with FP64 values (row_ptr/col uint32, as the library stores them)."""
    nrows: int
    ncols: int
    row_ptr: np.ndarray   # uint32[nrows+1]
    col: np.ndarray       # uint32[nnz]
    val: np.ndarray       # float64[nnz]

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1]) if self.nrows else 0

    def row_lengths(self) -> np.ndarray:
        return np.diff(self.row_ptr.astype(np.int64))


SEED0 = 20210317

# Truncation thresholds below were found once by log-space bisection on the
# nnz count (count_nnz) so that each matrix lands within 5 % of its nnz target.
TINY = Beam(grid=(32, 32, 20), lattice=(25, 20), spacing=(32 / 25, 32 / 20), sigma=3.0,
            tau=0.2423, seed=SEED0 + 0)
CLINICAL = Beam(grid=(256, 256, 160), lattice=(80, 50), spacing=(1.25, 1.25), sigma=4.0,
                tau=0.009134, seed=SEED0 + 1)

# Shaped like liver beam 1 of Table I (2.97e6 rows, 6.80e4 columns, 1.48e9
# entries, ~70 % empty rows, Fig. 2): 150x150x132 voxels, 272x250 spots a
# quarter voxel apart (dense enough that the central voxels see thousands of
# spots, as the energy layers of a real beam do).
LIVER1_SHAPED = Beam(grid=(150, 150, 132), lattice=(272, 250), spacing=(0.25, 0.25), sigma=4.0,
                     tau=0.028798, seed=SEED0 + 9)

NNZ_TARGETS = {"tiny": 2.0e5, "clinical": 1.5e8, "liver1": 1.48e9}

_SCENARIO_SHIFTS = [(sx, sy) for sy in (-3.0, 0.0, 3.0) for sx in (-3.0, 0.0, 3.0)]


def batched_beams() -> list:
    """Three beams x nine lateral setup shifts {-3,0,+3}^2 voxels = 27 matrices.

    Beam grids and spot counts: 160x160x80 / 1000 spots (40x25), 200x200x120 / 2500
    (50x50), 256x256x120 / 4000 (80x50); sigma, spacing and tau as the clinical beam.
    """
    shapes = [((160, 160, 80), (40, 25)), ((200, 200, 120), (50, 50)), ((256, 256, 120), (80, 50))]
    out = []
    for b, (grid, lat) in enumerate(shapes):
        base = replace(CLINICAL, grid=grid, lattice=lat, seed=SEED0 + 3 + 100 * (b + 1))
        for sh in _SCENARIO_SHIFTS:
            out.append(replace(base, shift=sh))
    return out


def count_nnz(beam: Beam, row_lengths: bool = False):
    """Total nnz of a beam (and the row-length array when asked)."""
    lib = _load()
    p = beam._params()
    if row_lengths:
        rl = np.empty(beam.nrows, dtype=np.uint32)
        n = lib.pb_count(ctypes.byref(p), rl.ctypes.data)
    else:
        rl = None
        n = lib.pb_count(ctypes.byref(p), None)
    if n < 0:
        raise RuntimeError("pencil-beam generator: bad parameters or out of memory")
    return (int(n), rl) if row_lengths else int(n)


def generate(beam: Beam) -> CSR:
    """Generate the beam's CSR matrix (FP64 values, ascending columns per row)."""
    lib = _load()
    nnz, rl = count_nnz(beam, row_lengths=True)
    if nnz >= 2**32:
        raise ValueError("matrix too large for uint32 row pointers")
    row_ptr = np.zeros(beam.nrows + 1, dtype=np.uint32)
    np.cumsum(rl, out=row_ptr[1:], dtype=np.uint32)
    del rl
    col = np.empty(nnz, dtype=np.uint32)
    val = np.empty(nnz, dtype=np.float64)
    p = beam._params()
    if lib.pb_fill(ctypes.byref(p), row_ptr.ctypes.data, col.ctypes.data, val.ctypes.data) != 0:
        raise RuntimeError("pencil-beam generator: fill failed")
    return CSR(beam.nrows, beam.ncols, row_ptr, col, val)


def generate_along(beam: Beam, axis: str) -> CSR:
    """The beam entering the patient grid `beam.grid` = (nx, ny, nz) along +z
    (the generator's own direction), +x or +y.  The matrix is generated on the
    permuted grid whose depth axis is the entry axis, then its rows are put in
    patient voxel order (row (z*ny + y)*nx + x); the lattice lies in the plane
    across the entry axis, with the generator's lateral axes in cyclic order."""
    nx, ny, nz = beam.grid
    if axis == "z":
        return generate(beam)
    if axis == "x":      # generator (gx, gy, gz) = patient (y, z, x)
        g = replace(beam, grid=(ny, nz, nx))
    elif axis == "y":    # generator (gx, gy, gz) = patient (z, x, y)
        g = replace(beam, grid=(nz, nx, ny))
    else:
        raise ValueError("axis must be 'x', 'y' or 'z'")
    csr = generate(g)
    gnx, gny, gnz = g.grid
    gz, gy, gx = np.meshgrid(np.arange(gnz), np.arange(gny), np.arange(gnx), indexing="ij")
    if axis == "x":
        x, y, z = gz, gx, gy
    else:
        x, y, z = gy, gz, gx
    patient_row = ((z * ny + y) * nx + x).reshape(-1)          # generator row -> patient row
    src = np.empty(csr.nrows, dtype=np.int64)
    src[patient_row] = np.arange(csr.nrows)                    # patient row -> generator row
    rp = csr.row_ptr.astype(np.int64)
    lens = (rp[1:] - rp[:-1])[src]
    row_ptr = np.zeros(csr.nrows + 1, dtype=np.int64)
    np.cumsum(lens, out=row_ptr[1:])
    take = np.repeat(rp[src] - row_ptr[:-1], lens) + np.arange(int(row_ptr[-1]))
    return CSR(csr.nrows, csr.ncols, row_ptr.astype(np.uint32), csr.col[take], csr.val[take])


# A three-beam plan on one patient grid (entry along +z, +x, +y), each beam under
# the nine lateral setup shifts: scenario s holds the three beams under shift s.
ROBUST_GRID = (160, 160, 100)
ROBUST_AXES = ("z", "x", "y")


def robust_plan(grid=ROBUST_GRID, lattice=(40, 25), base: Beam = None) -> list:
    """Scenarios x beams: out[s][b] = (Beam, axis) for the 9 setup shifts and the
    three entry axes.  Beam b's lattice spans its lateral plane with the
    clinical beam's spacing, sigma and tau unless `base` gives others."""
    base = base or CLINICAL
    out = []
    for sh in _SCENARIO_SHIFTS:
        row = []
        for b, axis in enumerate(ROBUST_AXES):
            beam = replace(base, grid=tuple(grid), lattice=tuple(lattice), seed=SEED0 + 7 + 100 * (b + 1),
                           shift=sh)
            row.append((beam, axis))
        out.append(row)
    return out


def spot_weights(n: int, seed: int, nvec: int = 1) -> np.ndarray:
    """Seeded FP32 spot weights uniform in [0,1): shape (n,) or (n, nvec) row-major."""
    lib = _load()
    out = np.empty(n * nvec, dtype=np.float32)
    lib.pb_uniform_f32(int(seed) & 0xFFFFFFFFFFFFFFFF, n * nvec, out.ctypes.data)
    return out if nvec == 1 else out.reshape(n, nvec)


def spot_weights_f64(n: int, seed: int) -> np.ndarray:
    """Seeded FP64 spot weights uniform in [0,1) with all 53 bits random: shape (n,)."""
    lib = _load()
    out = np.empty(n, dtype=np.float64)
    lib.pb_uniform_f64(int(seed) & 0xFFFFFFFFFFFFFFFF, n, out.ctypes.data)
    return out


def weight_seed(beam: Beam, k: int = 0) -> int:
    """Seed of the k-th spot-weight vector of a beam."""
    return (beam.seed * 7919 + 0x5EED + k) & 0xFFFFFFFFFFFFFFFF


def ellipsoid_target(beam: Beam, semi_axes=(8.0, 8.0, 4.0), depth_frac: float = 0.6,
                     dose: float = 60.0, w_in: float = 10.0, w_out: float = 1.0):
    """Prescription p and voxel weights w of a quadratic dose objective.

    Target = ellipsoid centred laterally on the grid at depth depth_frac*nz with the
    given semi-axes (voxels), tested at voxel centres; p = dose inside, 0 outside;
    w = w_in inside, w_out outside.  Returns float32 arrays (p, w) of length nrows.
    """
    nx, ny, nz = beam.grid
    iz, iy, ix = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    ex = (ix + 0.5 - nx / 2) / semi_axes[0]
    ey = (iy + 0.5 - ny / 2) / semi_axes[1]
    ez = (iz + 0.5 - depth_frac * nz) / semi_axes[2]
    inside = (ex * ex + ey * ey + ez * ez <= 1.0).reshape(-1)
    p = np.where(inside, dose, 0.0).astype(np.float32)
    w = np.where(inside, w_in, w_out).astype(np.float32)
    return p, w


def random_csr(nrows: int, ncols: int, seed: int, density: float = 0.1, empty_frac: float = 0.3,
               lengths=None, vmin: float = 1e-3, vmax: float = 1.0) -> CSR:
    """Small seeded random CSR: unique ascending columns, positive FP64 values.

    `lengths` (optional) fixes every row length exactly; otherwise rows are empty
    with probability empty_frac and binomial(ncols, density) long otherwise.
    """
    rng = np.random.default_rng(seed)
    if lengths is None:
        lens = rng.binomial(ncols, density, size=nrows)
        lens[rng.random(nrows) < empty_frac] = 0
    else:
        lens = np.asarray(lengths, dtype=np.int64)
        assert lens.shape == (nrows,) and lens.max(initial=0) <= ncols
    row_ptr = np.zeros(nrows + 1, dtype=np.uint32)
    np.cumsum(lens, out=row_ptr[1:])
    cols = [np.sort(rng.choice(ncols, size=int(n), replace=False)) for n in lens]
    col = (np.concatenate(cols) if nrows else np.zeros(0)).astype(np.uint32)
    val = rng.uniform(vmin, vmax, size=col.size)
    return CSR(nrows, ncols, row_ptr, col, val)
