"""Seeded synthetic Oseen workloads and their algebraic partition (inputs only).

The paper's experiments use IFISS Q2-Q1 leaky-cavity matrices, which are not
available; MAC finite-volume Oseen systems with the same structure
(C = [D E^T; -E 0], Section 1) stand in for them.  This module holds no
arithmetic of the preconditioner: it writes the matrix, the right-hand side and
the vertex-separator partition that both the CUDA library and the CPU oracle
read.  The C source is ``ddgen.c`` next to this file.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ddgen.c")
_LIB_PATH = os.path.join(_HERE, "_ddgen.so")
_lib = None

WIND_NONE, WIND_POLY, WIND_FOURIER = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile ddgen.c into _ddgen.so next to it (plain gcc, portable flags)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        i32p = ctypes.POINTER(ctypes.c_int32)
        f64p = ctypes.POINTER(ctypes.c_double)
        lib.ddg_mac_size.restype = ctypes.c_int64
        lib.ddg_mac_size.argtypes = [ctypes.c_int]
        lib.ddg_mac_nnz_bound.restype = ctypes.c_int64
        lib.ddg_mac_nnz_bound.argtypes = [ctypes.c_int]
        lib.ddg_mac_assemble.restype = ctypes.c_int64
        lib.ddg_mac_assemble.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                         ctypes.c_uint64, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                         i32p, i32p, f64p, f64p]
        lib.ddg_partition.restype = ctypes.c_int
        lib.ddg_partition.argtypes = [ctypes.c_int32, i32p, i32p, f64p, ctypes.c_int32, ctypes.c_int32, i32p, i32p,
                                      ctypes.POINTER(ctypes.c_int64)]
        lib.ddg_aggregates.restype = ctypes.c_int32
        lib.ddg_aggregates.argtypes = [ctypes.c_int32, i32p, i32p, f64p, i32p, i32p, ctypes.c_int32, i32p]
        lib.ddg_uniform.restype = None
        lib.ddg_uniform.argtypes = [ctypes.c_uint64, ctypes.c_int64, ctypes.c_double, ctypes.c_double, f64p]
        lib.ddg_raw.restype = None
        lib.ddg_raw.argtypes = [ctypes.c_uint64, ctypes.c_int64, ctypes.POINTER(ctypes.c_uint64)]
        lib.ddg_spacing.restype = None
        lib.ddg_spacing.argtypes = [ctypes.c_int, ctypes.c_double, f64p]
        lib.ddg_wind_info.restype = ctypes.c_int
        lib.ddg_wind_info.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_int, ctypes.c_uint64,
                                      f64p, i32p, i32p, f64p]
        lib.ddg_mac_layout.restype = None
        lib.ddg_mac_layout.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_int8), i32p]
        _lib = lib
    return _lib


def _p(a, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


@dataclass
class CSR:
    """Square CSR matrix with int32 indices and float64 values (host)."""
    n: int
    rowptr: np.ndarray
    col: np.ndarray
    val: np.ndarray

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])

    def to_dense(self) -> np.ndarray:
        a = np.zeros((self.n, self.n))
        for i in range(self.n):
            s, e = self.rowptr[i], self.rowptr[i + 1]
            a[i, self.col[s:e]] += self.val[s:e]
        return a

    def to_scipy(self):
        import scipy.sparse as sp
        return sp.csr_matrix((self.val, self.col, self.rowptr), shape=(self.n, self.n))


def uniform(seed: int, n: int, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    """n uniform draws in [lo, hi) from xoshiro256** seeded by SplitMix64(seed)."""
    out = np.empty(n, dtype=np.float64)
    _load().ddg_uniform(ctypes.c_uint64(seed), n, lo, hi, _p(out, ctypes.c_double))
    return out


def raw_stream(seed: int, n: int) -> np.ndarray:
    out = np.empty(n, dtype=np.uint64)
    _load().ddg_raw(ctypes.c_uint64(seed), n, _p(out, ctypes.c_uint64))
    return out


def spacing(n: int, r: float) -> np.ndarray:
    """Cell widths of the symmetric geometric grid (h_k ~ r^k from each wall)."""
    h = np.empty(n)
    _load().ddg_spacing(n, r, _p(h, ctypes.c_double))
    return h


def mac_layout(n: int):
    """(kind, cell) per unknown: kind 0 pressure, 1 u-face, 2 v-face; cell = j*n+i."""
    N = 3 * n * n - 2 * n
    kind = np.empty(N, dtype=np.int8)
    cell = np.empty(N, dtype=np.int32)
    _load().ddg_mac_layout(n, _p(kind, ctypes.c_int8), _p(cell, ctypes.c_int32))
    return kind, cell


def wind_info(n: int, stretch: float, wind: int, seed: int):
    amp = ctypes.c_double()
    mk = np.zeros(8, np.int32)
    nk = np.zeros(8, np.int32)
    ak = np.zeros(8)
    _load().ddg_wind_info(n, stretch, wind, ctypes.c_uint64(seed), ctypes.byref(amp),
                          _p(mk, ctypes.c_int32), _p(nk, ctypes.c_int32), _p(ak, ctypes.c_double))
    return amp.value, mk, nk, ak


def mac_system(n: int, nu: float, stretch: float = 1.0, wind: int = WIND_POLY, wind_seed: int = 0,
               lid: float = 1.0, pin: bool = True, scale: bool = True):
    """Assemble the MAC Oseen saddle-point matrix; returns (CSR, wall right-hand side)."""
    lib = _load()
    N = int(lib.ddg_mac_size(n))
    bound = int(lib.ddg_mac_nnz_bound(n))
    rowptr = np.zeros(N + 1, np.int32)
    col = np.zeros(bound, np.int32)
    val = np.zeros(bound, np.float64)
    rhs = np.zeros(N, np.float64)
    nnz = lib.ddg_mac_assemble(n, nu, stretch, wind, ctypes.c_uint64(wind_seed), lid, int(pin), int(scale),
                               _p(rowptr, ctypes.c_int32), _p(col, ctypes.c_int32),
                               _p(val, ctypes.c_double), _p(rhs, ctypes.c_double))
    if nnz < 0:
        raise MemoryError("ddg_mac_assemble failed")
    return CSR(N, rowptr, col[:nnz].copy(), val[:nnz].copy()), rhs


IFACE_ASCENDING, IFACE_RCM = 0, 1


def partition(A: CSR, m: int, iface_order: int = IFACE_ASCENDING):
    """Vertex-separator partition into m interiors + interface; returns (part, perm, moved)."""
    part = np.zeros(A.n, np.int32)
    perm = np.zeros(A.n, np.int32)
    stats = (ctypes.c_int64 * 2)()
    rc = _load().ddg_partition(A.n, _p(A.rowptr, ctypes.c_int32), _p(A.col, ctypes.c_int32),
                               _p(A.val, ctypes.c_double), m, iface_order, _p(part, ctypes.c_int32),
                               _p(perm, ctypes.c_int32), stats)
    if rc != 0:
        raise ValueError(f"ddg_partition failed (n={A.n}, m={m})")
    return part, perm, (int(stats[0]), int(stats[1]))


def aggregates(A: CSR, part: np.ndarray, perm: np.ndarray, sz: int) -> np.ndarray:
    """Offsets of consecutive interface aggregates of nominal size sz (see ddgen.c)."""
    nG = int((part < 0).sum())
    off = np.zeros(nG + 2, np.int32)
    na = _load().ddg_aggregates(A.n, _p(A.rowptr, ctypes.c_int32), _p(A.col, ctypes.c_int32),
                                _p(A.val, ctypes.c_double), _p(np.ascontiguousarray(part, np.int32), ctypes.c_int32),
                                _p(np.ascontiguousarray(perm, np.int32), ctypes.c_int32), sz,
                                _p(off, ctypes.c_int32))
    if na < 0:
        raise ValueError("ddg_aggregates failed")
    return off[:na + 1].copy()


@dataclass
class Workload:
    """One synthetic system: matrix, right-hand side and partition."""
    name: str
    grid: int
    nu: float
    stretch: float
    m: int
    A: CSR
    b: np.ndarray
    part: np.ndarray
    perm: np.ndarray
    meta: dict = field(default_factory=dict)
    sz: int = 64
    agg: np.ndarray = None

    @property
    def n_interface(self) -> int:
        return int((self.part < 0).sum())


def make_workload(name: str, grid: int, nu: float, stretch: float, wind: int, wind_seed: int, m: int,
                  rhs_seed: int = 0, sz: int = 64) -> Workload:
    A, _ = mac_system(grid, nu, stretch, wind, wind_seed)
    part, perm, moved = partition(A, m)
    b = uniform(rhs_seed, A.n, -1.0, 1.0)
    agg = aggregates(A, part, perm, sz)
    return Workload(name, grid, nu, stretch, m, A, b, part, perm,
                    dict(wind=wind, wind_seed=wind_seed, rhs_seed=rhs_seed, repaired=moved), sz, agg)


def cavity32() -> Workload:
    """32x32 uniform MAC Oseen, nu=0.01, wind (2y(1-x^2), -2x(1-y^2)), 4 subdomains."""
    return make_workload("oseen_mac_32x32_uniform_nu1e-2_m4", 32, 1e-2, 1.0, WIND_POLY, 0, 4)


def fourier256() -> Workload:
    """256x256 uniform MAC Oseen, nu=1e-3, seeded 8-mode Fourier wind, 64 subdomains."""
    return make_workload("oseen_mac_256x256_uniform_nu1e-3_m64", 256, 1e-3, 1.0, WIND_FOURIER, 2000, 64)


def stretched512() -> Workload:
    """512x512 MAC Oseen stretched toward the walls (ratio 1.02), nu=1e-3, 256 subdomains."""
    return make_workload("oseen_mac_512x512_stretch1.02_nu1e-3_m256", 512, 1e-3, 1.02, WIND_FOURIER, 3000, 256)


def batch64_specs(count: int = 64, seed: int = 4000):
    """Sizes, viscosities and subdomain counts of the 64-system batch (seeded)."""
    u = uniform(seed, 3 * count, 0.0, 1.0).reshape(count, 3)
    sides = [64, 96, 128, 192, 256]
    ms = [16, 32, 64]
    out = []
    for i in range(count):
        side = sides[min(int(u[i, 0] * 5), 4)]
        nu = 10.0 ** (-3.0 + u[i, 1])
        m = ms[min(int(u[i, 2] * 3), 2)]
        out.append(dict(grid=side, nu=nu, m=m, wind_seed=4000 + i))
    return out


def batch_workloads(specs, sz: int = 64, rhs_seed: int = 0):
    """One uniform-grid Fourier-wind Oseen workload per spec (grid, nu, m, wind_seed)."""
    return [make_workload(f"oseen_mac_{s['grid']}x{s['grid']}_nu{s['nu']:.2e}_m{s['m']}", s["grid"], s["nu"], 1.0,
                          WIND_FOURIER, s["wind_seed"], s["m"], rhs_seed=rhs_seed, sz=sz) for s in specs]


def batch64(sz: int = 2048):
    """The 64-system batch: sides in {64,...,256}, nu log-uniform in [1e-3, 1e-2], 16-64 subdomains each."""
    return batch_workloads(batch64_specs(), sz=sz)


def batch_small(count: int = 48, seed: int = 4100):
    """A small batch with many tiny subdomains: 16x16-32x32 grids split into 16-64 subdomains each."""
    u = uniform(seed, 2 * count, 0.0, 1.0).reshape(count, 2)
    out = []
    for i in range(count):
        grid = [16, 24, 32][min(int(u[i, 0] * 3), 2)]
        m = [16, 32, 64][min(int(u[i, 1] * 3), 2)] if i else 64
        out.append(dict(grid=grid, nu=10.0 ** (-3.0 + u[i, 1]), m=m, wind_seed=seed + i))
    return batch_workloads(out, sz=64)


def stretched1024() -> Workload:
    """1024x1024 MAC Oseen with wall stretching of max aspect 100, nu=1e-3, 1024 subdomains."""
    r = 100.0 ** (1.0 / 511.0)
    return make_workload("oseen_mac_1024x1024_aspect100_nu1e-3_m1024", 1024, 1e-3, r, WIND_FOURIER, 5000, 1024)


def learned64(seed: int) -> Workload:
    """One problem of the learned correction's family: 64x64 MAC Oseen with nu
    log-uniform in [1e-3, 1e-2] and wall stretching ratio uniform in [1, 1.03]
    (both drawn from the seed's stream), the seeded 8-mode Fourier wind, 4
    subdomains, aggregates of nominal size 64.  The training set uses seeds
    5000-6999; seeds 9000 and up are held out."""
    u = uniform(seed, 2, 0.0, 1.0)
    nu = log_uniform(1e-3, 1e-2, float(u[0]))
    return make_workload(f"oseen_mac_64x64_learned_seed{seed}", 64, nu, 1.0 + 0.03 * float(u[1]), WIND_FOURIER,
                         seed, 4, sz=64)


def max_aspect(n: int, r: float) -> float:
    h = spacing(n, r)
    return float(h.max() / h.min())


def log_uniform(lo: float, hi: float, u: float) -> float:
    return math.exp(math.log(lo) + (math.log(hi) - math.log(lo)) * u)
