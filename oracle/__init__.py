"""CPU oracle (plain FP64 C) for the algebraic-DD preconditioned GMRES solve.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this package; the library's
product path never does.  The C source ``dd_oracle.c`` follows the paper step
by step (Algorithm 1 for the setup, Algorithm 2 for the apply, Section 5 for
restarted GMRES); see its header for the readings taken where the paper is
ambiguous.  Every function here is pinned by ``tests/test_oracle_*.py``
against the mathematics (brute-force dense constructions, the spectral
theorem, library special cases); none of its outputs comes from the CUDA path.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dd_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_dd_oracle.so")
_lib = None

EXACT, MSCE_INF, MSCN, MSCNR, LUM, IDENTITY = 0, 1, 2, 3, 4, -1
OMSCN, OMSCNR, OLUM, MSCE = 6, 7, 8, 9
STATUS = {0: "ok", 1: "invalid_arg", 2: "invalid_partition", 3: "singular_block", 4: "singular_schur",
          5: "not_converged", 6: "nonfinite", 8: "oom"}


def build(force: bool = False) -> str:
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _p(a, ct):
    return None if a is None else a.ctypes.data_as(ctypes.POINTER(ct))


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        i32p, f64p, i64p = (ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_double),
                            ctypes.POINTER(ctypes.c_int64))
        vp = ctypes.c_void_p
        lib.orc_setup.restype = ctypes.c_int
        lib.orc_setup.argtypes = [ctypes.c_int32, i32p, i32p, f64p, ctypes.c_int32, i32p, i32p, ctypes.c_int32,
                                  i32p, ctypes.c_int32, ctypes.c_int32, ctypes.c_double, ctypes.POINTER(vp)]
        lib.orc_setup2.restype = ctypes.c_int
        lib.orc_setup2.argtypes = [ctypes.c_int32, i32p, i32p, f64p, ctypes.c_int32, i32p, i32p, ctypes.c_int32,
                                   i32p, ctypes.c_int32, ctypes.c_int32, ctypes.c_double, i32p, ctypes.c_int32,
                                   ctypes.c_int32, ctypes.POINTER(vp)]
        lib.orc_setup3.restype = ctypes.c_int
        lib.orc_setup3.argtypes = [ctypes.c_int32, i32p, i32p, f64p, ctypes.c_int32, i32p, i32p, ctypes.c_int32,
                                   i32p, ctypes.c_int32, ctypes.c_int32, ctypes.c_double, i32p, ctypes.c_int32,
                                   ctypes.c_int32, ctypes.c_double, ctypes.POINTER(vp)]
        lib.orc_band_ilu_dense.restype = ctypes.c_int
        lib.orc_band_ilu_dense.argtypes = [ctypes.c_int32, f64p, ctypes.c_int32, ctypes.c_int32, ctypes.c_double,
                                           ctypes.c_double, i32p, f64p]
        lib.orc_block_size.restype = ctypes.c_int32
        lib.orc_block_size.argtypes = [vp, ctypes.c_int32]
        lib.orc_overlaps.argtypes = [vp, i32p]
        lib.orc_schur_dense.restype = ctypes.c_int
        lib.orc_schur_dense.argtypes = [vp, f64p]
        lib.orc_free.argtypes = [vp]
        lib.orc_apply.restype = ctypes.c_int
        lib.orc_apply.argtypes = [vp, f64p, f64p]
        lib.orc_fgmres.restype = ctypes.c_int
        lib.orc_fgmres.argtypes = [vp, f64p, f64p, ctypes.c_double, ctypes.c_int32, ctypes.c_int32, i32p, i32p,
                                   f64p, f64p, ctypes.c_int32]
        lib.orc_sizes.argtypes = [vp, i64p]
        lib.orc_agg_offsets.argtypes = [vp, i32p]
        lib.orc_perm.argtypes = [vp, i32p]
        lib.orc_interior_offsets.argtypes = [vp, i32p]
        lib.orc_bandwidths.argtypes = [vp, i32p]
        lib.orc_schur_block.restype = ctypes.c_int
        lib.orc_schur_block.argtypes = [vp, ctypes.c_int32, f64p]
        lib.orc_replace_block.restype = ctypes.c_int
        lib.orc_replace_block.argtypes = [vp, ctypes.c_int32, f64p, ctypes.c_double]
        lib.orc_bad_block.restype = ctypes.c_int32
        lib.orc_bad_block.argtypes = [vp]
        lib.orc_dense_lu.restype = ctypes.c_int
        lib.orc_dense_lu.argtypes = [ctypes.c_int32, f64p, i32p, ctypes.c_double]
        lib.orc_dense_lu_solve.argtypes = [ctypes.c_int32, f64p, i32p, f64p]
        lib.orc_band_lu_dense.restype = ctypes.c_int
        lib.orc_band_lu_dense.argtypes = [ctypes.c_int32, f64p, ctypes.c_int32, ctypes.c_int32, ctypes.c_double,
                                          i32p, f64p]
        lib.orc_spmv.argtypes = [ctypes.c_int32, i32p, i32p, f64p, f64p, f64p]
        lib.orc_num_threads.restype = ctypes.c_int
        lib.orc_set_threads.argtypes = [ctypes.c_int]
        _lib = lib
    return _lib


class OracleError(RuntimeError):
    def __init__(self, status, bad_block=-1):
        super().__init__(f"oracle status {status} ({STATUS.get(status, '?')}), bad_block={bad_block}")
        self.status = status
        self.bad_block = bad_block


def num_threads() -> int:
    return int(_load().orc_num_threads())


def set_threads(t: int) -> None:
    _load().orc_set_threads(int(t))


def dense_lu(a: np.ndarray, pivtol: float = 1e-14):
    """P a = L U with partial pivoting (first max); returns (lu, piv, status)."""
    n = a.shape[0]
    lu = np.ascontiguousarray(a, dtype=np.float64).copy()
    piv = np.zeros(n, np.int32)
    rc = _load().orc_dense_lu(n, _p(lu, ctypes.c_double), _p(piv, ctypes.c_int32), pivtol)
    return lu, piv, int(rc)


def dense_lu_solve(lu, piv, b):
    x = np.ascontiguousarray(b, dtype=np.float64).copy()
    _load().orc_dense_lu_solve(lu.shape[0], _p(lu, ctypes.c_double), _p(piv, ctypes.c_int32),
                               _p(x, ctypes.c_double))
    return x


def band_lu_solve(a: np.ndarray, kl: int, ku: int, b: np.ndarray, pivtol: float = 1e-14):
    """Band LU of the dense matrix a (bandwidths kl, ku); returns (x, piv, status)."""
    n = a.shape[0]
    a = np.ascontiguousarray(a, dtype=np.float64)
    x = np.ascontiguousarray(b, dtype=np.float64).copy()
    piv = np.zeros(n, np.int32)
    rc = _load().orc_band_lu_dense(n, _p(a, ctypes.c_double), kl, ku, pivtol, _p(piv, ctypes.c_int32),
                                   _p(x, ctypes.c_double))
    return x, piv, int(rc)


def band_ilu_solve(a: np.ndarray, kl: int, ku: int, b: np.ndarray, tau: float, pivtol: float = 1e-14):
    """Incomplete band LU (drop tolerance tau) of the dense matrix a; returns (x, piv, status)."""
    n = a.shape[0]
    a = np.ascontiguousarray(a, dtype=np.float64)
    x = np.ascontiguousarray(b, dtype=np.float64).copy()
    piv = np.zeros(n, np.int32)
    rc = _load().orc_band_ilu_dense(n, _p(a, ctypes.c_double), kl, ku, pivtol, float(tau),
                                    _p(piv, ctypes.c_int32), _p(x, ctypes.c_double))
    return x, piv, int(rc)


def spmv(A, x):
    y = np.zeros(A.n)
    x = np.ascontiguousarray(x, dtype=np.float64)
    _load().orc_spmv(A.n, _p(A.rowptr, ctypes.c_int32), _p(A.col, ctypes.c_int32), _p(A.val, ctypes.c_double),
                     _p(x, ctypes.c_double), _p(y, ctypes.c_double))
    return y


class OracleDD:
    """The preconditioner B of the paper for one kind, built on the CPU."""

    def __init__(self, A, part, m, kind, perm=None, sz=64, agg_offsets=None, pivtol=1e-14, raise_on_error=True,
                 overlap=0, overlaps=None, radius=0, ilu_tol=0.0):
        """overlap / overlaps: the overlap widths of OMSCN, OMSCNR and OLUM (one
        width for all aggregates, capped by the next aggregate's size, or one
        per aggregate); radius: the path-length radius of MSCE; ilu_tol: the
        drop tolerance of the incomplete LU of the interior blocks (0: exact)."""
        lib = _load()
        self._lib = lib
        self.A = A
        self._keep = [np.ascontiguousarray(A.rowptr, np.int32), np.ascontiguousarray(A.col, np.int32),
                      np.ascontiguousarray(A.val, np.float64), np.ascontiguousarray(part, np.int32)]
        perm_a = None if perm is None else np.ascontiguousarray(perm, np.int32)
        agg_a = None if agg_offsets is None else np.ascontiguousarray(agg_offsets, np.int32)
        nagg = 0 if agg_a is None else len(agg_a) - 1
        ovl_a = None if overlaps is None else np.ascontiguousarray(overlaps, np.int32)
        h = ctypes.c_void_p()
        rc = lib.orc_setup3(A.n, _p(self._keep[0], ctypes.c_int32), _p(self._keep[1], ctypes.c_int32),
                            _p(self._keep[2], ctypes.c_double), m, _p(self._keep[3], ctypes.c_int32),
                            _p(perm_a, ctypes.c_int32), nagg, _p(agg_a, ctypes.c_int32), sz, kind, pivtol,
                            _p(ovl_a, ctypes.c_int32), int(overlap), int(radius), float(ilu_tol),
                            ctypes.byref(h))
        self._h = h
        self.status = int(rc)
        self.bad_block = int(lib.orc_bad_block(h)) if h.value else -1
        if rc != 0 and raise_on_error:
            self.close()
            raise OracleError(rc, self.bad_block)
        if h.value:
            s = np.zeros(6, np.int64)
            lib.orc_sizes(h, _p(s, ctypes.c_int64))
            self.n, self.m, self.nI, self.nG, self.nagg, self.kind = (int(v) for v in s)

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.orc_free(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def agg_offsets(self):
        o = np.zeros(self.nagg + 1, np.int32)
        self._lib.orc_agg_offsets(self._h, _p(o, ctypes.c_int32))
        return o

    def perm(self):
        o = np.zeros(self.n, np.int32)
        self._lib.orc_perm(self._h, _p(o, ctypes.c_int32))
        return o

    def interior_offsets(self):
        o = np.zeros(self.m + 1, np.int32)
        self._lib.orc_interior_offsets(self._h, _p(o, ctypes.c_int32))
        return o

    def bandwidths(self):
        o = np.zeros(2 * self.m, np.int32)
        self._lib.orc_bandwidths(self._h, _p(o, ctypes.c_int32))
        return o.reshape(self.m, 2)

    def overlaps(self):
        o = np.zeros(self.nagg, np.int32)
        self._lib.orc_overlaps(self._h, _p(o, ctypes.c_int32))
        return o

    def schur_dense(self):
        """The whole S_hat (n_G x n_G), blocks placed as the apply uses them."""
        o = np.zeros((self.nG, self.nG))
        if self._lib.orc_schur_dense(self._h, _p(o, ctypes.c_double)) != 0:
            raise OracleError(1)
        return o

    def schur_block(self, i):
        p = int(self._lib.orc_block_size(self._h, int(i)))
        if p < 0:
            raise IndexError(i)
        o = np.zeros((p, p))
        if self._lib.orc_schur_block(self._h, i, _p(o, ctypes.c_double)) != 0:
            raise IndexError(i)
        return o

    def replace_block(self, i, blk, pivtol=1e-14):
        """Use blk as S_hat block i if its LU passes the pivot test; returns whether it did."""
        blk = np.ascontiguousarray(blk, np.float64)
        rc = self._lib.orc_replace_block(self._h, int(i), _p(blk, ctypes.c_double), float(pivtol))
        if rc not in (0, 4):
            raise OracleError(rc)
        return rc == 0

    def apply(self, y):
        y = np.ascontiguousarray(y, np.float64)
        x = np.zeros(self.n)
        rc = self._lib.orc_apply(self._h, _p(y, ctypes.c_double), _p(x, ctypes.c_double))
        if rc != 0:
            raise OracleError(rc)
        return x

    def fgmres(self, b, tol=1e-8, restart=50, maxit=3000, hist_cap=4096):
        b = np.ascontiguousarray(b, np.float64)
        x = np.zeros(self.n)
        it = ctypes.c_int32()
        rs = ctypes.c_int32()
        rel = ctypes.c_double()
        hist = np.zeros(hist_cap)
        rc = self._lib.orc_fgmres(self._h, _p(b, ctypes.c_double), _p(x, ctypes.c_double), tol, restart, maxit,
                                  ctypes.byref(it), ctypes.byref(rs), ctypes.byref(rel),
                                  _p(hist, ctypes.c_double), hist_cap)
        return dict(x=x, status=int(rc), iters=int(it.value), restarts=int(rs.value), relres=float(rel.value),
                    history=hist[:min(int(it.value), hist_cap)].copy())
