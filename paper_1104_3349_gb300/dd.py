"""ctypes binding of libdd (include/dd.h): argument marshalling only.

Every step of the setup, the apply and the GMRES solve runs in the library's
CUDA kernels; PyTorch supplies device memory and streams.  There is no CPU
fallback: without the compiled library every entry point raises.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from concurrent.futures import ThreadPoolExecutor

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
_ROOT = os.path.dirname(_PKG)
_CSRC = os.path.join(_PKG, "csrc")
_INCLUDE = os.path.join(_ROOT, "include")
_BUILD = os.path.join(_ROOT, "_build")
LIB_PATH = os.path.join(_PKG, "libdd.so")
# the checked build (-DDD_CHECKED): device index, size and alignment checks
# that record DD_ERR_CHECK instead of faulting; selected with DD_CHECKED=1
LIB_CHECKED_PATH = os.path.join(_PKG, "libdd_checked.so")
SOURCES = ["dd_api.cu", "k_band.cu", "k_dense.cu", "k_krylov.cu", "k_mlp.cu"]
NVCC_FLAGS = ["-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-lineinfo", "-std=c++17",
              "-Xcompiler", "-fPIC", "-I" + _INCLUDE]

DD_EXACT, DD_MSCE_INF, DD_MSCN, DD_MSCNR, DD_LUM = 0, 1, 2, 3, 4
DD_FP64, DD_FP32, DD_FP32_TF32 = 0, 1, 2
STATUS_NAMES = {0: "DD_OK", 1: "DD_ERR_INVALID_ARG", 2: "DD_ERR_INVALID_PARTITION",
                3: "DD_ERR_SINGULAR_BLOCK", 4: "DD_ERR_SINGULAR_SCHUR", 5: "DD_ERR_NOT_CONVERGED",
                6: "DD_ERR_NONFINITE", 7: "DD_ERR_TIMEOUT", 8: "DD_ERR_OOM", 9: "DD_ERR_CUDA",
                10: "DD_ERR_CHECK"}
DD_LEARNED = 5
DD_OMSCN, DD_OMSCNR, DD_OLUM, DD_MSCE = 6, 7, 8, 9
KINDS = {"exact": DD_EXACT, "msce_inf": DD_MSCE_INF, "mscn": DD_MSCN, "mscnr": DD_MSCNR, "lum": DD_LUM,
         "learned": DD_LEARNED, "omscn": DD_OMSCN, "omscnr": DD_OMSCNR, "olum": DD_OLUM, "msce": DD_MSCE}
MLP_IN, MLP_HIDDEN = 14, 64
MLP_NPARAM = MLP_HIDDEN * MLP_IN + 2 * MLP_HIDDEN + 1


def _nvcc():
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def build(force: bool = False, verbose: bool = False, checked: bool = False, both: bool = False) -> str:
    """Compile the CUDA sources for sm_103a (in parallel) and link libdd.so
    in-tree (checked: libdd_checked.so with -DDD_CHECKED; both: the two
    libraries, compiled side by side).  Returns the path of the library
    asked for (the plain one with both)."""
    variants = [False, True] if both else [checked]
    srcs = [os.path.join(_CSRC, s) for s in SOURCES]
    deps = srcs + [os.path.join(_CSRC, "dd_internal.h"), os.path.join(_INCLUDE, "dd.h")]
    todo = []
    for chk in variants:
        path = LIB_CHECKED_PATH if chk else LIB_PATH
        if force or not os.path.exists(path) or any(os.path.getmtime(d) > os.path.getmtime(path) for d in deps):
            todo.append(chk)
    nvcc = _nvcc()

    def compile_one(job):
        src, chk = job
        bdir = os.path.join(_BUILD, "checked" if chk else "plain")
        os.makedirs(bdir, exist_ok=True)
        obj = os.path.join(bdir, os.path.basename(src) + ".o")
        cmd = [nvcc, *NVCC_FLAGS, *(["-DDD_CHECKED"] if chk else []), "-c", src, "-o", obj]
        if verbose:
            print(" ".join(cmd))
        subprocess.check_call(cmd)
        return obj

    if todo:
        jobs = [(src, chk) for chk in todo for src in srcs]
        with ThreadPoolExecutor(max_workers=len(jobs)) as ex:
            objs = list(ex.map(compile_one, jobs))
        for chk in todo:
            path = LIB_CHECKED_PATH if chk else LIB_PATH
            mine = [o for (src, c), o in zip(jobs, objs) if c == chk]
            tmp = path + f".{os.getpid()}.tmp"
            subprocess.check_call([nvcc, "-shared", "-o", tmp, *mine, "-lcudart"])
            os.replace(tmp, path)
    return LIB_CHECKED_PATH if (checked and not both) else LIB_PATH


class dd_csr(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("nnz", ctypes.c_int64), ("rowptr", ctypes.c_void_p),
                ("col", ctypes.c_void_p), ("val", ctypes.c_void_p)]


class dd_partition(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int32), ("part", ctypes.c_void_p), ("perm", ctypes.c_void_p),
                ("sz", ctypes.c_int32), ("agg_offsets", ctypes.c_void_p), ("n_agg", ctypes.c_int32)]


class dd_opts(ctypes.Structure):
    _fields_ = [("prec", ctypes.c_int32), ("pivot_tol", ctypes.c_double), ("use_graph", ctypes.c_int32),
                ("max_restart", ctypes.c_int32), ("autotune", ctypes.c_int32), ("krylov_ctas_per_sm", ctypes.c_int32),
                ("time_kernels", ctypes.c_int32), ("sweep_cluster", ctypes.c_int32),
                ("mlp_weights", ctypes.c_char_p), ("overlap", ctypes.c_int32), ("radius", ctypes.c_int32),
                ("krylov_threads", ctypes.c_int32), ("sweep_prefetch", ctypes.c_int32),
                ("pad_opts", ctypes.c_int32), ("ilu_tol", ctypes.c_double)]


class dd_info(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int32), ("restarts", ctypes.c_int32), ("bad_block", ctypes.c_int32),
                ("status", ctypes.c_int32), ("relres_true", ctypes.c_double), ("setup_ms", ctypes.c_double),
                ("solve_ms", ctypes.c_double), ("history", ctypes.c_void_p), ("history_cap", ctypes.c_int32),
                ("pad2", ctypes.c_int32)]


class dd_stats(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("n_interior", ctypes.c_int64), ("n_interface", ctypes.c_int64),
                ("nnz", ctypes.c_int64), ("m", ctypes.c_int32), ("n_agg", ctypes.c_int32),
                ("max_agg", ctypes.c_int32), ("kl_max", ctypes.c_int32), ("ku_max", ctypes.c_int32),
                ("tile", ctypes.c_int32), ("factor_bytes", ctypes.c_int64), ("factor_nonzeros", ctypes.c_int64),
                ("schur_bytes", ctypes.c_int64), ("coupling_nnz", ctypes.c_int64), ("setup_ms", ctypes.c_double),
                ("launches", ctypes.c_int64), ("stage_bytes", ctypes.c_int32), ("sweep_grid", ctypes.c_int32),
                ("sweep_slots", ctypes.c_int32), ("tuned", ctypes.c_int32), ("tuned_us", ctypes.c_double),
                ("batch", ctypes.c_int32), ("graphs", ctypes.c_int32), ("learned_entries", ctypes.c_int64),
                ("learned_fallback", ctypes.c_int32), ("sweep_prefetch", ctypes.c_int32),
                ("krylov_steps", ctypes.c_int64), ("cgs2_ms", ctypes.c_double), ("cgs2_fma", ctypes.c_double),
                ("spmv_ms", ctypes.c_double), ("sweep_cluster", ctypes.c_int32), ("msce_nodes_max", ctypes.c_int32)]


EXPORTS = ["dd_setup", "dd_setup_batched", "dd_apply", "dd_apply_part", "dd_apply_noalloc", "gmres_solve",
           "dd_check_status", "dd_set_wait_limit", "dd_fp64_peak",
           "gmres_solve_batched", "dd_spmv", "dd_get_stats", "dd_get_bad_block", "dd_destroy", "dd_last_error",
           "dd_learned_entries", "dd_mlp_create", "dd_mlp_set_data", "dd_mlp_loss_grad", "dd_mlp_adam_step",
           "dd_mlp_predict", "dd_mlp_get", "dd_mlp_set_adam", "dd_mlp_destroy"]
NOALLOC_MAX_ELEMS = 1 << 20

_lib = None


def load(path: str = None):
    """Load libdd.so (libdd_checked.so when DD_CHECKED=1 in the environment);
    raises if it has not been built (no fallback path exists)."""
    global _lib
    if _lib is not None:
        return _lib
    if path is None:
        path = LIB_CHECKED_PATH if os.environ.get("DD_CHECKED") == "1" else LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError(f"libdd.so not built ({path}); run __graft_entry__.build()")
    lib = ctypes.CDLL(path)
    vp = ctypes.c_void_p
    lib.dd_setup.restype = ctypes.c_int
    lib.dd_setup.argtypes = [ctypes.POINTER(dd_csr), ctypes.POINTER(dd_partition), ctypes.c_int,
                             ctypes.POINTER(dd_opts), vp, ctypes.POINTER(vp)]
    lib.dd_setup_batched.restype = ctypes.c_int
    lib.dd_setup_batched.argtypes = [ctypes.c_int32, ctypes.POINTER(dd_csr), ctypes.POINTER(dd_partition),
                                     ctypes.c_int, ctypes.POINTER(dd_opts), vp, ctypes.POINTER(vp)]
    lib.gmres_solve_batched.restype = ctypes.c_int
    lib.gmres_solve_batched.argtypes = [vp, ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.c_double,
                                        ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(dd_info), vp]
    lib.dd_apply.restype = ctypes.c_int
    lib.dd_apply.argtypes = [vp, vp, vp, vp]
    lib.gmres_solve.restype = ctypes.c_int
    lib.gmres_solve.argtypes = [vp, vp, vp, ctypes.c_double, ctypes.c_int32, ctypes.c_int32,
                                ctypes.POINTER(dd_info), vp]
    lib.dd_apply_noalloc.restype = ctypes.c_int
    lib.dd_apply_noalloc.argtypes = [vp, vp, vp, vp]
    lib.dd_apply_part.restype = ctypes.c_int
    lib.dd_apply_part.argtypes = [vp, ctypes.c_int32, vp, vp, vp]
    lib.dd_check_status.restype = ctypes.c_int
    lib.dd_check_status.argtypes = [vp, vp]
    lib.dd_fp64_peak.restype = ctypes.c_int
    lib.dd_fp64_peak.argtypes = [ctypes.POINTER(ctypes.c_double), vp]
    lib.dd_set_wait_limit.restype = ctypes.c_int
    lib.dd_set_wait_limit.argtypes = [vp, ctypes.c_uint32]
    lib.dd_spmv.restype = ctypes.c_int
    lib.dd_spmv.argtypes = [vp, vp, vp, vp]
    lib.dd_get_stats.restype = ctypes.c_int
    lib.dd_get_stats.argtypes = [vp, ctypes.POINTER(dd_stats)]
    lib.dd_get_bad_block.restype = ctypes.c_int32
    lib.dd_get_bad_block.argtypes = [vp]
    lib.dd_destroy.restype = ctypes.c_int
    lib.dd_destroy.argtypes = [vp]
    lib.dd_last_error.restype = ctypes.c_char_p
    lib.dd_last_error.argtypes = [vp]
    i64, f32p = ctypes.c_int64, ctypes.POINTER(ctypes.c_float)
    lib.dd_learned_entries.restype = ctypes.c_int
    lib.dd_learned_entries.argtypes = [vp, vp, vp, vp, i64, ctypes.POINTER(i64)]
    lib.dd_mlp_create.restype = ctypes.c_int
    lib.dd_mlp_create.argtypes = [vp, ctypes.POINTER(vp)]
    lib.dd_mlp_set_data.restype = ctypes.c_int
    lib.dd_mlp_set_data.argtypes = [vp, vp, vp, i64, vp]
    lib.dd_mlp_loss_grad.restype = ctypes.c_int
    lib.dd_mlp_loss_grad.argtypes = [vp, i64, i64, ctypes.POINTER(ctypes.c_double), vp, vp]
    lib.dd_mlp_adam_step.restype = ctypes.c_int
    lib.dd_mlp_adam_step.argtypes = [vp, i64, i64, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float, vp]
    lib.dd_mlp_predict.restype = ctypes.c_int
    lib.dd_mlp_predict.argtypes = [vp, i64, i64, vp, vp]
    lib.dd_mlp_get.restype = ctypes.c_int
    lib.dd_mlp_get.argtypes = [vp, vp, vp, vp, ctypes.POINTER(i64)]
    lib.dd_mlp_set_adam.restype = ctypes.c_int
    lib.dd_mlp_set_adam.argtypes = [vp, vp, vp, i64]
    lib.dd_mlp_destroy.restype = ctypes.c_int
    lib.dd_mlp_destroy.argtypes = [vp]
    _lib = lib
    return lib


class DDError(RuntimeError):
    def __init__(self, status: int, msg: str, bad_block: int = -1):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status
        self.bad_block = bad_block


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def _stream_handle(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _dev_ptr(t, n):
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise TypeError("expected a contiguous float64 CUDA tensor")
    if t.numel() != n:
        raise ValueError(f"expected {n} elements, got {t.numel()}")
    return ctypes.c_void_p(t.data_ptr())


class DD:
    """One preconditioner B built by dd_setup; owns the library handle."""

    def __init__(self, A, part, m, kind="msce_inf", perm=None, sz=64, agg_offsets=None, prec=DD_FP64,
                 pivot_tol=0.0, max_restart=50, stream=None, raise_on_error=True, use_graph=False,
                 autotune=False, mlp_weights=None, krylov_ctas_per_sm=0, time_kernels=False, sweep_cluster=0,
                 overlap=0, radius=0, krylov_threads=0, sweep_prefetch=0, ilu_tol=0.0):
        lib = load()
        self._lib = lib
        self.n = int(A.n)
        self._arrs = [np.ascontiguousarray(A.rowptr, np.int32), np.ascontiguousarray(A.col, np.int32),
                      np.ascontiguousarray(A.val, np.float64), np.ascontiguousarray(part, np.int32),
                      None if perm is None else np.ascontiguousarray(perm, np.int32),
                      None if agg_offsets is None else np.ascontiguousarray(agg_offsets, np.int32)]
        rp, col, val, pa, pe, ag = self._arrs
        csr = dd_csr(self.n, int(rp[-1]), _ptr(rp), _ptr(col), _ptr(val))
        pt = dd_partition(int(m), _ptr(pa), _ptr(pe), int(sz), _ptr(ag), 0 if ag is None else len(ag) - 1)
        o = dd_opts(int(prec), float(pivot_tol), int(bool(use_graph)), int(max_restart), int(bool(autotune)),
                    int(krylov_ctas_per_sm))
        o.time_kernels = int(bool(time_kernels))
        o.sweep_cluster = int(sweep_cluster)
        o.overlap = int(overlap)
        o.radius = int(radius)
        o.krylov_threads = int(krylov_threads)
        o.sweep_prefetch = int(sweep_prefetch)
        o.ilu_tol = float(ilu_tol)
        self._wpath = None if mlp_weights is None else os.fsencode(mlp_weights)
        o.mlp_weights = self._wpath
        k = KINDS[kind] if isinstance(kind, str) else int(kind)
        h = ctypes.c_void_p()
        rc = lib.dd_setup(ctypes.byref(csr), ctypes.byref(pt), k, ctypes.byref(o), _stream_handle(stream),
                          ctypes.byref(h))
        self._h = h
        self.status = int(rc)
        self.prec = int(prec)
        self.bad_block = int(lib.dd_get_bad_block(h)) if h.value else -1
        if rc != 0:
            msg = lib.dd_last_error(h if h.value else None).decode()
            if raise_on_error:
                self.close()
                raise DDError(rc, msg, self.bad_block)
            self.error = msg

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.dd_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc):
        if rc != 0:
            raise DDError(rc, self._lib.dd_last_error(self._h).decode())

    def apply(self, y, x, stream=None):
        """x = B^-1 y (device tensors, float64, original numbering)."""
        self._check(self._lib.dd_apply(self._h, _dev_ptr(y, self.n), _dev_ptr(x, self.n), _stream_handle(stream)))

    def apply_noalloc(self, y, x, stream=None):
        """x = B^-1 y with the library's fixed device scratch instead of handle buffers."""
        self._check(self._lib.dd_apply_noalloc(self._h, _dev_ptr(y, self.n), _dev_ptr(x, self.n),
                                               _stream_handle(stream)))

    def apply_part(self, part, y, x, stream=None):
        """One of the apply's three kernels (0: interior solve, 1: interface, 2: back-substitution)."""
        self._check(self._lib.dd_apply_part(self._h, int(part), _dev_ptr(y, self.n), _dev_ptr(x, self.n),
                                            _stream_handle(stream)))

    def check_status(self, stream=None):
        """Synchronise the stream and return (and clear) the handle's device status word."""
        return int(self._lib.dd_check_status(self._h, _stream_handle(stream)))

    def set_wait_limit(self, first_wait_polls):
        """Test hook: polls of the first bounded wait of every sweep CTA (0: give up at once)."""
        self._check(self._lib.dd_set_wait_limit(self._h, int(first_wait_polls) & 0xFFFFFFFF))

    def spmv(self, x, y, stream=None):
        self._check(self._lib.dd_spmv(self._h, _dev_ptr(x, self.n), _dev_ptr(y, self.n), _stream_handle(stream)))

    def gmres(self, b, x, tol=1e-8, restart=50, maxit=3000, history_cap=4096, stream=None):
        """Right-preconditioned restarted FGMRES; returns a dict (status, iters, ...)."""
        hist = np.zeros(history_cap)
        info = dd_info()
        info.history = hist.ctypes.data_as(ctypes.c_void_p).value
        info.history_cap = history_cap
        rc = self._lib.gmres_solve(self._h, _dev_ptr(b, self.n), _dev_ptr(x, self.n), float(tol), int(restart),
                                   int(maxit), ctypes.byref(info), _stream_handle(stream))
        if rc not in (0, 5, 6):
            self._check(rc)
        return dict(status=int(rc), iters=int(info.iters), restarts=int(info.restarts),
                    relres=float(info.relres_true), solve_ms=float(info.solve_ms), setup_ms=float(info.setup_ms),
                    history=hist[:min(info.iters, history_cap)].copy())

    def stats(self):
        s = dd_stats()
        self._check(self._lib.dd_get_stats(self._h, ctypes.byref(s)))
        return {f: getattr(s, f) for f, _ in dd_stats._fields_}

    def learned_entries(self):
        """(entries [n x 3] aggregate/row/col, raw features [n x 14] FP64, Delta [n]) of a DD_LEARNED handle."""
        cnt = ctypes.c_int64()
        self._check(self._lib.dd_learned_entries(self._h, None, None, None, 0, ctypes.byref(cnt)))
        n = cnt.value
        ents = np.zeros((n, 3), np.int32)
        feats = np.zeros((n, MLP_IN), np.float64)
        delta = np.zeros(n, np.float32)
        self._check(self._lib.dd_learned_entries(self._h, _ptr(ents), _ptr(feats), _ptr(delta), n, ctypes.byref(cnt)))
        return ents, feats, delta


def fp64_peak(stream=None) -> float:
    """FP64 fused multiply-adds per second / 1e9 of the current device (dd_fp64_peak)."""
    lib = load()
    v = ctypes.c_double()
    rc = lib.dd_fp64_peak(ctypes.byref(v), _stream_handle(stream))
    if rc != 0:
        raise DDError(rc, "dd_fp64_peak")
    return float(v.value)


class DDBatch:
    """A batch of independent systems behind one handle (dd_setup_batched)."""

    def __init__(self, systems, kind="msce_inf", prec=DD_FP64, pivot_tol=0.0, max_restart=50, stream=None,
                 use_graph=False, autotune=False, mlp_weights=None, krylov_ctas_per_sm=0, sweep_cluster=0,
                 sweep_prefetch=0, ilu_tol=0.0):
        """systems: list of (A, part, m, perm, agg_offsets) with A a CSR (perm, agg_offsets may be None)."""
        lib = load()
        self._lib = lib
        self.count = len(systems)
        self.sizes = [int(sy[0].n) for sy in systems]
        self._arrs = []
        csrs = (dd_csr * self.count)()
        pts = (dd_partition * self.count)()
        for q, (A, part, m, perm, agg) in enumerate(systems):
            arrs = [np.ascontiguousarray(A.rowptr, np.int32), np.ascontiguousarray(A.col, np.int32),
                    np.ascontiguousarray(A.val, np.float64), np.ascontiguousarray(part, np.int32),
                    None if perm is None else np.ascontiguousarray(perm, np.int32),
                    None if agg is None else np.ascontiguousarray(agg, np.int32)]
            self._arrs.append(arrs)
            rp, col, val, pa, pe, ag = arrs
            csrs[q] = dd_csr(int(A.n), int(rp[-1]), _ptr(rp), _ptr(col), _ptr(val))
            pts[q] = dd_partition(int(m), _ptr(pa), _ptr(pe), 64, _ptr(ag), 0 if ag is None else len(ag) - 1)
        o = dd_opts(int(prec), float(pivot_tol), int(bool(use_graph)), int(max_restart), int(bool(autotune)),
                    int(krylov_ctas_per_sm))
        o.sweep_cluster = int(sweep_cluster)
        o.sweep_prefetch = int(sweep_prefetch)
        o.ilu_tol = float(ilu_tol)
        self._wpath = None if mlp_weights is None else os.fsencode(mlp_weights)
        o.mlp_weights = self._wpath
        k = KINDS[kind] if isinstance(kind, str) else int(kind)
        h = ctypes.c_void_p()
        rc = lib.dd_setup_batched(self.count, csrs, pts, k, ctypes.byref(o), _stream_handle(stream), ctypes.byref(h))
        self._h = h
        self.n = sum(self.sizes)
        if rc != 0:
            msg = lib.dd_last_error(h if h.value else None).decode()
            bad = int(lib.dd_get_bad_block(h)) if h.value else -1
            self.close()
            raise DDError(rc, msg, bad)

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.dd_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def apply(self, y, x, stream=None):
        """x = B^-1 y on the concatenated vector (every system's block)."""
        rc = self._lib.dd_apply(self._h, _dev_ptr(y, self.n), _dev_ptr(x, self.n), _stream_handle(stream))
        if rc != 0:
            raise DDError(rc, self._lib.dd_last_error(self._h).decode())

    def gmres(self, bs, xs, tol=1e-8, restart=30, maxit=3000, history_cap=4096, stream=None):
        """Independent FGMRES solves; bs, xs: lists of device tensors. Returns (status, [per-system dicts])."""
        if len(bs) != self.count or len(xs) != self.count:
            raise ValueError("one right-hand side and one solution per system")
        bp = (ctypes.c_void_p * self.count)(*[_dev_ptr(b, n).value for b, n in zip(bs, self.sizes)])
        xp = (ctypes.c_void_p * self.count)(*[_dev_ptr(x, n).value for x, n in zip(xs, self.sizes)])
        infos = (dd_info * self.count)()
        hists = [np.zeros(history_cap) for _ in range(self.count)]
        for q in range(self.count):
            infos[q].history = hists[q].ctypes.data_as(ctypes.c_void_p).value
            infos[q].history_cap = history_cap
        rc = self._lib.gmres_solve_batched(self._h, bp, xp, float(tol), int(restart), int(maxit), infos,
                                           _stream_handle(stream))
        if rc not in (0, 5, 6):
            raise DDError(rc, self._lib.dd_last_error(self._h).decode())
        out = [dict(status=int(i.status), iters=int(i.iters), restarts=int(i.restarts), relres=float(i.relres_true),
                    solve_ms=float(i.solve_ms), setup_ms=float(i.setup_ms),
                    history=h[:min(i.iters, history_cap)].copy()) for i, h in zip(infos, hists)]
        return int(rc), out

    def stats(self):
        s = dd_stats()
        rc = self._lib.dd_get_stats(self._h, ctypes.byref(s))
        if rc != 0:
            raise DDError(rc, "dd_get_stats")
        return {f: getattr(s, f) for f, _ in dd_stats._fields_}


class MLP:
    """Training handle of the learned Schur correction's network (dd_mlp_*)."""

    def __init__(self, params):
        lib = load()
        self._lib = lib
        p = np.ascontiguousarray(params, np.float32)
        if p.shape != (MLP_NPARAM,):
            raise ValueError(f"expected {MLP_NPARAM} parameters")
        h = ctypes.c_void_p()
        rc = lib.dd_mlp_create(_ptr(p), ctypes.byref(h))
        if rc != 0:
            raise DDError(rc, "dd_mlp_create")
        self._h = h
        self.n = 0

    def _check(self, rc, what):
        if rc != 0:
            raise DDError(rc, what)

    def set_data(self, X, y, stream=None):
        X = np.ascontiguousarray(X, np.float32)
        y = np.ascontiguousarray(y, np.float32)
        if X.ndim != 2 or X.shape[1] != MLP_IN or len(y) != len(X):
            raise ValueError("X must be n x 14 and y n long")
        self._check(self._lib.dd_mlp_set_data(self._h, _ptr(X), _ptr(y), len(y), _stream_handle(stream)), "set_data")
        self.n = len(y)

    def loss_grad(self, lo=0, hi=None, stream=None):
        hi = self.n if hi is None else hi
        loss = ctypes.c_double()
        g = np.zeros(MLP_NPARAM, np.float32)
        self._check(self._lib.dd_mlp_loss_grad(self._h, lo, hi, ctypes.byref(loss), _ptr(g), _stream_handle(stream)),
                    "loss_grad")
        return loss.value, g

    def adam_step(self, lo, hi, lr, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
        self._check(self._lib.dd_mlp_adam_step(self._h, lo, hi, lr, beta1, beta2, eps, _stream_handle(stream)),
                    "adam_step")

    def predict(self, lo=0, hi=None, stream=None):
        hi = self.n if hi is None else hi
        out = np.zeros(hi - lo, np.float32)
        self._check(self._lib.dd_mlp_predict(self._h, lo, hi, _ptr(out), _stream_handle(stream)), "predict")
        return out

    def get(self):
        p, m, v = (np.zeros(MLP_NPARAM, np.float32) for _ in range(3))
        st = ctypes.c_int64()
        self._check(self._lib.dd_mlp_get(self._h, _ptr(p), _ptr(m), _ptr(v), ctypes.byref(st)), "get")
        return p, m, v, st.value

    def set_adam(self, m, v, step):
        m = np.ascontiguousarray(m, np.float32)
        v = np.ascontiguousarray(v, np.float32)
        self._check(self._lib.dd_mlp_set_adam(self._h, _ptr(m), _ptr(v), int(step)), "set_adam")

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.dd_mlp_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
