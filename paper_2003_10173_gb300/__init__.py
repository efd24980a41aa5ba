"""Python binding of the GB300 H^2 Hessian library (libh2hess.so, C ABI in include/h2.h).

The binding only marshals arguments: every step of construction and application
runs in the library's CUDA kernels.  Device buffers are passed as torch tensors
(or raw integer device pointers); torch is used for device memory and streams.
If the shared library is missing, importing the binding's entry points raises:
there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libh2hess.so")

H2_OK = 0
H2_ERR_INVALID_ARG = -1
H2_ERR_CUDA = -2
H2_ERR_OP_FAILED = -3
H2_ERR_NAN = -4
H2_ERR_OOM = -5
H2_ERR_DEVICE_CHECK = -6
H2_WARN_TOL_NOT_MET = 1

H2_ADM_WEAK = 0
H2_ADM_STRONG = 1

H2_FP64 = 0
H2_FP32 = 1
H2_TF32 = 2
H2_BF16 = 3
H2_TF32X3 = 4
H2_FP32C = 5
H2_SAMPLING_WEAK = 0
H2_SAMPLING_COLORED = 1

H2_MAX_LEVELS = 32

OP_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p,
                         ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p)


class BuildOpts(ctypes.Structure):
    _fields_ = [
        ("kmax", ctypes.c_int), ("q0", ctypes.c_int), ("b_inc", ctypes.c_int), ("q_max", ctypes.c_int),
        ("adaptive", ctypes.c_int), ("seed", ctypes.c_uint64), ("norm_est", ctypes.c_double),
        ("norm_maxit", ctypes.c_int), ("norm_rtol", ctypes.c_double), ("keep_fp32", ctypes.c_int),
        ("keep_bf16", ctypes.c_int), ("stream", ctypes.c_void_p),
        ("q_level", ctypes.c_void_p), ("q_level_stride", ctypes.c_int), ("q_test", ctypes.c_int),
        ("global_rank", ctypes.c_int), ("sampling", ctypes.c_int), ("batch_workers", ctypes.c_int),
        ("certified", ctypes.c_int),
    ]


H2_MAX_INVERT_ITERS = 64


class InvertOpts(ctypes.Structure):
    _fields_ = [
        ("order", ctypes.c_int), ("eps", ctypes.c_double), ("eps_loose", ctypes.c_double),
        ("theta", ctypes.c_double), ("max_iter", ctypes.c_int), ("shift", ctypes.c_double),
        ("res_maxit", ctypes.c_int), ("res_rtol", ctypes.c_double), ("seed", ctypes.c_uint64),
        ("x0", ctypes.c_void_p), ("unroll", ctypes.c_int),
    ]


class InvertStats(ctypes.Structure):
    _fields_ = [
        ("iterations", ctypes.c_int), ("converged", ctypes.c_int), ("norm_A", ctypes.c_double),
        ("alpha", ctypes.c_double), ("err", ctypes.c_double * (H2_MAX_INVERT_ITERS + 1)),
        ("eps_k", ctypes.c_double * H2_MAX_INVERT_ITERS), ("samples", ctypes.c_int64 * H2_MAX_INVERT_ITERS),
        ("t_build", ctypes.c_double * H2_MAX_INVERT_ITERS), ("final_err", ctypes.c_double),
        ("t_total", ctypes.c_double),
    ]

    def as_dict(self) -> dict:
        k = self.iterations
        return {"iterations": k, "converged": bool(self.converged), "norm_A": self.norm_A, "alpha": self.alpha,
                "err": [float(x) for x in self.err[:k + 1]], "eps_k": [float(x) for x in self.eps_k[:k]],
                "samples": [int(x) for x in self.samples[:k]], "t_build": [float(x) for x in self.t_build[:k]],
                "final_err": self.final_err, "t_total": self.t_total}


class Stats(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int64), ("levels", ctypes.c_int), ("leaf_max", ctypes.c_int),
        ("samples", ctypes.c_int64), ("norm_products", ctypes.c_int64),
        ("range_probes", ctypes.c_int * H2_MAX_LEVELS), ("proj_probes", ctypes.c_int * H2_MAX_LEVELS),
        ("max_rank", ctypes.c_int * H2_MAX_LEVELS),
        ("far_lower", ctypes.c_int64), ("near_lower", ctypes.c_int64),
        ("entries_D", ctypes.c_int64), ("entries_S", ctypes.c_int64), ("entries_U", ctypes.c_int64),
        ("entries_E", ctypes.c_int64),
        ("norm_est", ctypes.c_double), ("tau_basis", ctypes.c_double), ("tau_test", ctypes.c_double),
        ("tol_met", ctypes.c_int),
        ("t_total", ctypes.c_double), ("t_norm", ctypes.c_double), ("t_op", ctypes.c_double),
        ("t_peel", ctypes.c_double), ("t_assemble", ctypes.c_double),
        ("op_calls", ctypes.c_int64),
        ("range_calls", ctypes.c_int * H2_MAX_LEVELS), ("range_need", ctypes.c_int * H2_MAX_LEVELS),
        ("range_passed", ctypes.c_int * H2_MAX_LEVELS),
    ]

    def as_dict(self) -> dict:
        L = self.levels
        d = {f: getattr(self, f) for f, _ in self._fields_}
        for k in ("range_probes", "proj_probes", "max_rank", "range_calls", "range_need", "range_passed"):
            d[k] = [int(x) for x in getattr(self, k)[: L + 1]]
        return d


_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_I = ctypes.c_int
_D = ctypes.c_double
_SIGS = {
    "h2_build_opts_default": (_I, [ctypes.POINTER(BuildOpts)]),
    "h2_tree_create": (_I, [_P, _I64, _I, _I, _I, _D, ctypes.POINTER(_P)]),
    "h2_tree_free": (None, [_P]),
    "h2_tree_info": (_I, [_P, _P, _P, _P, _P]),
    "h2_tree_perm": (_I, [_P, _P]),
    "h2_tree_boxes": (_I, [_P, _I, _P, _P]),
    "h2_tree_far": (_I, [_P, _I, _P, _P]),
    "h2_tree_near": (_I, [_P, _P, _P]),
    "h2_build": (_I, [_P, _P, _P, _D, ctypes.POINTER(BuildOpts), ctypes.POINTER(_P)]),
    "h2_import": (_I, [_P, _P, _P, _P, _P, _P, _I, _I, ctypes.POINTER(_P)]),
    "h2_factor_sizes": (_I, [_P, _P, _P, _P, _P, _P]),
    "h2_export": (_I, [_P, _P, _P, _P, _P, _P]),
    "h2_matvec": (_I, [_P, _P, _I64, _P, _I64, _I64, _I, _P]),
    "h2_build_batched": (_I, [_I, _P, _P, _P, _D, ctypes.POINTER(BuildOpts), _P]),
    "h2_batch_create": (_I, [_I, _P, ctypes.POINTER(_P)]),
    "h2_batch_matvec": (_I, [_P, _P, _P, _P, _P, _I64, _I, _P]),
    "h2_batch_tuned": (_I, [_P, _I64, _I, _P]),
    "h2_batch_free": (None, [_P]),
    "h2_matvec_batched": (_I, [_I, _P, _P, _P, _P, _P, _I64, _I, _P]),
    "h2_rankmodel_save": (_I, [_P, ctypes.c_char_p]),
    "h2_rankmodel_load": (_I, [ctypes.c_char_p, ctypes.POINTER(_P)]),
    "h2_matvec_noalloc": (_I, [_P, _P, _I64, _P, _I64, _I64, _I, _P]),
    "h2_matvec_host": (_I, [_P, _P, _I64, _P, _I64, _I64, _I, _P]),
    "h2_rankmodel_targets": (_I, [_P, _P, _P, _P]),
    "h2_get_stats": (_I, [_P, ctypes.POINTER(Stats)]),
    "h2_profile": (_I, [_P, _I]),
    "h2_device_status": (_I, [_P]),
    "h2_profile_read": (_I, [_P, _P, _P]),
    "h2_gemm_profile": (_I, [_I]),
    "h2_gemm_profile_read": (_I, [_P, _P, _P, _P]),
    "h2_stack_profile_read": (_I, [_I, _P, _P, _P]),
    "h2_free": (None, [_P]),
    "h2_colored_plan": (_I, [_P, _I, _P]),
    "h2_lowrank_update": (_I, [_P, _P, _I64, _I, _P, _D, ctypes.POINTER(BuildOpts), ctypes.POINTER(_P)]),
    "h2_invert_opts_default": (_I, [ctypes.POINTER(InvertOpts)]),
    "h2_invert": (_I, [_P, ctypes.POINTER(InvertOpts), ctypes.POINTER(BuildOpts), ctypes.POINTER(_P),
                       ctypes.POINTER(InvertStats)]),
    "h2_rankmodel_create": (_I, [ctypes.c_uint64, _I, ctypes.POINTER(_P)]),
    "h2_rankmodel_free": (None, [_P]),
    "h2_rankmodel_get": (_I, [_P, _P, _P, _P, _P]),
    "h2_rankmodel_set": (_I, [_P, _P, _P, _P, _I64]),
    "h2_rankmodel_features": (_I, [_P, _D, _D, _D, _P]),
    "h2_rankmodel_loss_grad": (_I, [_P, _P, _P, _I64, _P, _P]),
    "h2_rankmodel_train": (_I, [_P, _P, _P, _I64, _P, _I, _I, ctypes.c_float, _P, _P]),
    "h2_rankmodel_predict": (_I, [_P, _P, _I64, _P, _P]),
    "h2_rankmodel_q_levels": (_I, [_P, _P, _D, _D, _D, _I, _I, _P, _P]),
    "h2_heat2d_create": (_I, [_I, _D, _D, _D, _P, ctypes.POINTER(_P)]),
    "h2_heat2d_apply": (_I, [_P, _I64, _I64, _P, _I64, _P, _I64, _P]),
    "h2_heat2d_destroy": (None, [_P]),
    "h2_dense_op_create": (_I, [_P, _I64, _I64, ctypes.POINTER(_P)]),
    "h2_dense_op_apply": (_I, [_P, _I64, _I64, _P, _I64, _P, _I64, _P]),
    "h2_dense_op_destroy": (None, [_P]),
    "h2_lowrank_op_create": (_I, [_P, _I64, _I64, _I64, ctypes.c_double, ctypes.POINTER(_P)]),
    "h2_lowrank_op_apply": (_I, [_P, _I64, _I64, _P, _I64, _P, _I64, _P]),
    "h2_lowrank_op_destroy": (None, [_P]),
    "h2_error_string": (ctypes.c_char_p, [_I]),
    "h2_last_error": (ctypes.c_char_p, []),
    "h2_launch_count": (_I64, []),
    "h2_device_bytes": (_I64, []),
    "h2_set_device_limit": (_I, [_I64]),
    "h2_version": (ctypes.c_char_p, []),
}

_lib = None


class H2Error(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{msg} (status {status})")
        self.status = status


def lib():
    """Load libh2hess.so (raises if it has not been built: there is no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: run paper_2003_10173_gb300.build_lib.build()")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def exported_symbols():
    return list(_SIGS)


def _check(status: int, allow_warn: bool = False) -> int:
    if status < 0 or (status > 0 and not allow_warn):
        L = lib()
        raise H2Error(status, f"{L.h2_error_string(status).decode()}: {L.h2_last_error().decode()}")
    return status


def _ptr(x) -> int:
    """Device or host address of a torch tensor / numpy array / int."""
    if x is None:
        return 0
    if isinstance(x, int):
        return x
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    return x.data_ptr()


def _stream_ptr(stream) -> int:
    if stream is None:
        return 0
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def default_opts(**kw) -> BuildOpts:
    o = BuildOpts()
    _check(lib().h2_build_opts_default(ctypes.byref(o)))
    for k, v in kw.items():
        if k == "stream":
            v = _stream_ptr(v)
        if k == "q_level":
            if v is None:
                v = 0
            else:
                arr = np.ascontiguousarray(v, dtype=np.int32)
                o._q_level_keep = arr          # the library reads it during the build call
                v = arr.ctypes.data
        setattr(o, k, v)
    return o


class Tree:
    """KD cluster tree + block partition (host data)."""

    def __init__(self, coords: np.ndarray, leaf: int, adm: int = H2_ADM_STRONG, eta: float = 0.7):
        coords = np.ascontiguousarray(coords, dtype=np.float64)
        if coords.ndim != 2:
            raise ValueError("coords must be (n, dim)")
        h = ctypes.c_void_p()
        _check(lib().h2_tree_create(coords.ctypes.data, coords.shape[0], coords.shape[1], leaf, adm, eta,
                                    ctypes.byref(h)))
        self._h = h
        lv, n, nf, nn = _I(), _I64(), _I64(), _I64()
        _check(lib().h2_tree_info(h, ctypes.byref(lv), ctypes.byref(n), ctypes.byref(nf), ctypes.byref(nn)))
        self.L, self.N, self.n_far, self.n_near = lv.value, n.value, nf.value, nn.value

    @property
    def handle(self):
        return self._h

    def perm(self) -> np.ndarray:
        out = np.empty(self.N, dtype=np.int64)
        _check(lib().h2_tree_perm(self._h, out.ctypes.data))
        return out

    def boxes(self, level: int):
        st = np.empty(1 << level, dtype=np.int64)
        sz = np.empty(1 << level, dtype=np.int64)
        _check(lib().h2_tree_boxes(self._h, level, st.ctypes.data, sz.ctypes.data))
        return st, sz

    def far(self, level: int) -> np.ndarray:
        c = _I64()
        _check(lib().h2_tree_far(self._h, level, ctypes.byref(c), None))
        out = np.empty((c.value, 2), dtype=np.int32)
        _check(lib().h2_tree_far(self._h, level, ctypes.byref(c), out.ctypes.data))
        return out

    def colored_plan(self, q: int) -> dict:
        """h2_colored_plan: per level the colours of the range pass, the probe slots of the projection
        pass and the lower far pairs of coloured sampling with q probes per block, and the leaf colours."""
        out = np.zeros(3 * (self.L + 1) + 1, dtype=np.int32)
        _check(lib().h2_colored_plan(self._h, q, out.ctypes.data))
        lv = out[:-1].reshape(self.L + 1, 3)
        return {"colors": lv[:, 0].tolist(), "slots": lv[:, 1].tolist(), "pairs": lv[:, 2].tolist(),
                "leaf_colors": int(out[-1])}

    def near(self) -> np.ndarray:
        c = _I64()
        _check(lib().h2_tree_near(self._h, ctypes.byref(c), None))
        out = np.empty((c.value, 2), dtype=np.int32)
        _check(lib().h2_tree_near(self._h, ctypes.byref(c), out.ctypes.data))
        return out

    def close(self):
        if self._h:
            lib().h2_tree_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class HeatOperator:
    """The library's heat-equation misfit Hessian H = F diag(mask) F / sigma^2 (device state)."""

    def __init__(self, n: int, kappa: float, T: float, sigma: float, mask: np.ndarray):
        mask = np.ascontiguousarray(mask, dtype=np.float64)
        if mask.size != n * n:
            raise ValueError("mask must have n*n entries")
        h = ctypes.c_void_p()
        _check(lib().h2_heat2d_create(n, kappa, T, sigma, mask.ctypes.data, ctypes.byref(h)))
        self.ctx = h
        self.N = n * n
        self.fn = ctypes.cast(lib().h2_heat2d_apply, ctypes.c_void_p)
        self._mask = mask

    def apply(self, X, Y, nrhs: int, stream=None, ldx: int | None = None, ldy: int | None = None):
        _check(lib().h2_heat2d_apply(self.ctx, self.N, nrhs, _ptr(X), ldx or self.N, _ptr(Y), ldy or self.N,
                                     _stream_ptr(stream)))

    def close(self):
        if self.ctx:
            lib().h2_heat2d_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class LowRankOperator:
    """Y = scale Z (Z^T X) with a caller-owned FP64 device matrix Z (n x r, column-major: a torch
    tensor of shape (r, n); kept alive by this object)."""

    def __init__(self, Zt, scale: float = 1.0):
        self.Z = Zt
        r, n = Zt.shape
        h = ctypes.c_void_p()
        _check(lib().h2_lowrank_op_create(_ptr(Zt), n, r, n, float(scale), ctypes.byref(h)))
        self.ctx = h
        self.N = n
        self.fn = ctypes.cast(lib().h2_lowrank_op_apply, ctypes.c_void_p)

    def apply(self, X, Y, nrhs: int, stream=None, ldx: int | None = None, ldy: int | None = None):
        _check(lib().h2_lowrank_op_apply(self.ctx, self.N, nrhs, _ptr(X), ldx or self.N, _ptr(Y), ldy or self.N,
                                         _stream_ptr(stream)))

    def close(self):
        if self.ctx:
            lib().h2_lowrank_op_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class DenseOperator:
    """Y = A X with a caller-owned dense FP64 device matrix (kept alive by this object)."""

    def __init__(self, A):
        self.A = A
        n = A.shape[0]
        h = ctypes.c_void_p()
        _check(lib().h2_dense_op_create(_ptr(A), n, n, ctypes.byref(h)))
        self.ctx = h
        self.N = n
        self.fn = ctypes.cast(lib().h2_dense_op_apply, ctypes.c_void_p)

    def close(self):
        if self.ctx:
            lib().h2_dense_op_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class PyOperator:
    """Wraps a Python callable f(X_ptr, ldx, Y_ptr, ldy, nrhs, stream_ptr) -> int as an h2_op_fn."""

    def __init__(self, N: int, fn):
        self.N = N

        def tramp(ctx, n, nrhs, X, ldx, Y, ldy, stream):
            try:
                return int(fn(X, ldx, Y, ldy, nrhs, stream) or 0)
            except Exception:
                return 99

        self._cb = OP_FN(tramp)
        self.fn = ctypes.cast(self._cb, ctypes.c_void_p)
        self.ctx = None


class H2:
    """A built H^2 approximation (device factors owned by the library)."""

    def __init__(self, handle, status: int = 0):
        self._h = handle
        self.status = status

    @classmethod
    def build(cls, op, tree: Tree, tol: float, opts: BuildOpts | None = None) -> "H2":
        h = ctypes.c_void_p()
        st = lib().h2_build(op.fn, op.ctx, tree.handle, tol, ctypes.byref(opts) if opts is not None else None,
                            ctypes.byref(h))
        _check(st, allow_warn=True)
        return cls(h, st)

    @classmethod
    def from_factors(cls, tree: Tree, ranks, U, E, S, D, keep_fp32=False, keep_bf16=False) -> "H2":
        arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in (U, E, S, D)]
        rk = np.ascontiguousarray(ranks, dtype=np.int32)
        h = ctypes.c_void_p()
        _check(lib().h2_import(tree.handle, rk.ctypes.data, *[a.ctypes.data if a.size else None for a in arrs],
                               int(keep_fp32), int(keep_bf16), ctypes.byref(h)))
        return cls(h)

    def factor_sizes(self):
        v = [_I64() for _ in range(5)]
        _check(lib().h2_factor_sizes(self._h, *[ctypes.byref(x) for x in v]))
        return [x.value for x in v]

    def export(self):
        nr, nu, ne, ns, nd = self.factor_sizes()
        rk = np.empty(nr, dtype=np.int32)
        out = [np.empty(max(n, 1)) for n in (nu, ne, ns, nd)]
        _check(lib().h2_export(self._h, rk.ctypes.data, *[a.ctypes.data for a in out]))
        return (rk,) + tuple(a[:n] for a, n in zip(out, (nu, ne, ns, nd)))

    def matvec(self, X, Y, nrhs: int, mode: int = H2_FP64, stream=None, ldx: int | None = None,
               ldy: int | None = None):
        n = self.stats()["n"]
        _check(lib().h2_matvec(self._h, _ptr(X), ldx or n, _ptr(Y), ldy or n, nrhs, mode, _stream_ptr(stream)))

    def matvec_host(self, X, Y, nrhs: int, mode: int = H2_FP64, stream=None, ldx: int | None = None,
                    ldy: int | None = None):
        """h2_matvec_host: X and Y in host memory (CPU tensors or arrays; pinned for full-speed copies);
        returns when Y is complete."""
        n = self.stats()["n"]
        _check(lib().h2_matvec_host(self._h, _ptr(X), ldx or n, _ptr(Y), ldy or n, nrhs, mode, _stream_ptr(stream)))

    def matvec_noalloc(self, X, Y, nrhs: int, mode: int = H2_FP64, stream=None, ldx: int | None = None,
                       ldy: int | None = None):
        """h2_matvec with the library's fixed 32 MiB device scratch instead of an allocated workspace."""
        n = self.stats()["n"]
        _check(lib().h2_matvec_noalloc(self._h, _ptr(X), ldx or n, _ptr(Y), ldy or n, nrhs, mode,
                                       _stream_ptr(stream)))

    def lowrank_update(self, B, r: int, tol: float, M=None, opts: BuildOpts | None = None, ldb: int | None = None):
        """h2_lowrank_update: a new H2 for A + B M B^T, recompressed to tol.  B is a device tensor
        (n x r in original order, column-major: a (r, n) row-major tensor or any pointer with ldb);
        M a host r x r array (None: identity)."""
        n = self.stats()["n"]
        Mh = None if M is None else np.asfortranarray(np.asarray(M, dtype=np.float64).reshape(r, r))
        h = ctypes.c_void_p()
        st = lib().h2_lowrank_update(self._h, _ptr(B) if r else None, ldb or n, r,
                                     Mh.ctypes.data if Mh is not None else None, tol,
                                     ctypes.byref(opts) if opts is not None else None, ctypes.byref(h))
        _check(st, allow_warn=True)
        return H2(h, st)

    STAGES = ("leaf_up", "up", "couple", "down", "leaf_near", "near")

    def profile(self, enable: bool = True):
        _check(lib().h2_profile(self._h, int(enable)))

    def profile_read(self) -> dict:
        ms = np.zeros(6)
        n = np.zeros(6, dtype=np.int64)
        _check(lib().h2_profile_read(self._h, ms.ctypes.data, n.ctypes.data))
        return {k: (float(ms[i]), int(n[i])) for i, k in enumerate(self.STAGES)}

    def device_status(self) -> int:
        return int(lib().h2_device_status(self._h))

    def stats(self) -> dict:
        s = Stats()
        _check(lib().h2_get_stats(self._h, ctypes.byref(s)))
        return s.as_dict()

    def close(self):
        if self._h:
            lib().h2_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def invert(A: "H2", shift: float = 0.0, order: int = 2, eps: float = 1e-6, eps_loose: float | None = None,
           theta: float = 0.1, max_iter: int = 50, build_opts: BuildOpts | None = None, **kw):
    """Hierarchical hyperpower (order 2: Newton-Schulz) inverse of A + shift I; returns (H2, stats)."""
    o = InvertOpts()
    _check(lib().h2_invert_opts_default(ctypes.byref(o)))
    o.order, o.eps, o.theta, o.max_iter, o.shift = order, eps, theta, max_iter, shift
    o.eps_loose = eps if eps_loose is None else eps_loose
    for k, v in kw.items():
        if k == "x0" and isinstance(v, H2):
            v = v._h.value
        setattr(o, k, v)
    st = InvertStats()
    h = ctypes.c_void_p()
    status = lib().h2_invert(A._h, ctypes.byref(o), ctypes.byref(build_opts) if build_opts is not None else None,
                             ctypes.byref(h), ctypes.byref(st))
    _check(status, allow_warn=True)
    return H2(h, status), st.as_dict()


def gemm_profile(enable: bool = True):
    _check(lib().h2_gemm_profile(int(enable)))


def gemm_profile_read():
    """(milliseconds, algorithmic flops, launches, algorithmic bytes) of the GEMM launches since the last read."""
    ms, fl, n, by = _D(), _D(), _I64(), _D()
    _check(lib().h2_gemm_profile_read(ctypes.byref(ms), ctypes.byref(fl), ctypes.byref(n), ctypes.byref(by)))
    return ms.value, fl.value, n.value, by.value


def stack_profile_read(which: int):
    """(milliseconds, algorithmic QR flops, launches) of the stacked QR (0) or truncated-SVD (1) launches
    since the last read (recorded while gemm_profile is on)."""
    ms, fl, n = _D(), _D(), _I64()
    _check(lib().h2_stack_profile_read(which, ctypes.byref(ms), ctypes.byref(fl), ctypes.byref(n)))
    return ms.value, fl.value, n.value


def build_batched(ops, trees, tol: float, opts: BuildOpts | None = None):
    """Construct several H^2 matrices in one call (concurrent workers); returns a list of H2."""
    n = len(ops)
    fns = (ctypes.c_void_p * n)(*[o.fn.value if hasattr(o.fn, "value") else o.fn for o in ops])
    ctxs = (ctypes.c_void_p * n)(*[o.ctx.value if isinstance(o.ctx, ctypes.c_void_p) else o.ctx for o in ops])
    trs = (ctypes.c_void_p * n)(*[t.handle.value for t in trees])
    outs = (ctypes.c_void_p * n)()
    st = lib().h2_build_batched(n, fns, ctxs, trs, tol, ctypes.byref(opts) if opts is not None else None, outs)
    _check(st, allow_warn=True)
    return [H2(ctypes.c_void_p(outs[i]), st) for i in range(n)]


def matvec_batched(handles, Xs, Ys, nrhs: int, mode: int = H2_FP64, stream=None):
    """One-shot batched application of several handles (h2_matvec_batched)."""
    n = len(handles)
    hp = (ctypes.c_void_p * n)(*[h._h.value for h in handles])
    xp = (ctypes.c_void_p * n)(*[_ptr(x) for x in Xs])
    yp = (ctypes.c_void_p * n)(*[_ptr(y) for y in Ys])
    lx = (ctypes.c_int64 * n)(*[h.stats()["n"] for h in handles])
    _check(lib().h2_matvec_batched(n, hp, xp, lx, yp, lx, nrhs, mode, _stream_ptr(stream)))


class Batch:
    """Merged, autotuned and graph-captured matvec over several handles (which must stay alive)."""

    def __init__(self, handles):
        self.handles = list(handles)
        n = len(self.handles)
        arr = (ctypes.c_void_p * n)(*[h._h.value for h in self.handles])
        b = ctypes.c_void_p()
        _check(lib().h2_batch_create(n, arr, ctypes.byref(b)))
        self._b = b

    def matvec(self, Xs, Ys, nrhs: int, mode: int = H2_FP64, stream=None):
        n = len(self.handles)
        xp = (ctypes.c_void_p * n)(*[_ptr(x) for x in Xs])
        yp = (ctypes.c_void_p * n)(*[_ptr(y) for y in Ys])
        lx = (ctypes.c_int64 * n)(*[h.stats()["n"] for h in self.handles])
        _check(lib().h2_batch_matvec(self._b, xp, lx, yp, lx, nrhs, mode, _stream_ptr(stream)))

    def tuned(self, nrhs: int, mode: int) -> int:
        v = _I()
        _check(lib().h2_batch_tuned(self._b, nrhs, mode, ctypes.byref(v)))
        return v.value

    def close(self):
        if self._b:
            lib().h2_batch_free(self._b)
            self._b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


RM_FEATURES = 8
RM_WIDTH = 64
RM_NPARAM = 64 * 8 + 64 + 64 * 64 + 64 + 64 + 1


def rank_features(tree: Tree, kappa_T: float, density: float, tol: float) -> np.ndarray:
    """Per-level features of the rank model ((L+1) x 8, host FP64), computed by the library."""
    out = np.empty((tree.L + 1, RM_FEATURES))
    _check(lib().h2_rankmodel_features(tree.handle, kappa_T, density, tol, out.ctypes.data))
    return out


class RankModel:
    """Learned per-level probe counts (MLP with hand-written forward/backward/Adam kernels)."""

    def __init__(self, seed: int = 0, bf16: bool = True):
        h = ctypes.c_void_p()
        _check(lib().h2_rankmodel_create(seed, int(bf16), ctypes.byref(h)))
        self._m = h
        self.bf16 = bool(bf16)

    def get(self):
        p, m, v = (np.empty(RM_NPARAM, dtype=np.float32) for _ in range(3))
        st = _I64()
        _check(lib().h2_rankmodel_get(self._m, p.ctypes.data, m.ctypes.data, v.ctypes.data, ctypes.byref(st)))
        return p, m, v, st.value

    def set(self, params=None, adam_m=None, adam_v=None, step: int = -1):
        arrs = [None if a is None else np.ascontiguousarray(a, dtype=np.float32) for a in (params, adam_m, adam_v)]
        for a in arrs:
            if a is not None and a.size != RM_NPARAM:
                raise ValueError("parameter arrays need RM_NPARAM entries")
        _check(lib().h2_rankmodel_set(self._m, *[a.ctypes.data if a is not None else None for a in arrs], step))

    def loss_grad(self, X, t):
        """Loss and gradient over all rows of X (device float32 n x 8) and t (device float32 n)."""
        loss = ctypes.c_float()
        g = np.empty(RM_NPARAM, dtype=np.float32)
        _check(lib().h2_rankmodel_loss_grad(self._m, _ptr(X), _ptr(t), X.shape[0], ctypes.byref(loss), g.ctypes.data))
        return float(loss.value), g

    def train(self, X, t, steps: int, batch: int, lr: float, idx=None, loss_out=None, stream=None):
        _check(lib().h2_rankmodel_train(self._m, _ptr(X), _ptr(t), X.shape[0], _ptr(idx), steps, batch, lr,
                                        _ptr(loss_out), _stream_ptr(stream)))

    def predict(self, X, y, stream=None):
        _check(lib().h2_rankmodel_predict(self._m, _ptr(X), X.shape[0], _ptr(y), _stream_ptr(stream)))

    def q_levels(self, tree: Tree, kappa_T: float, density: float, tol: float, pad: int = 8, q_max: int = 256):
        """Start counts per level for BuildOpts.q_level and the raw predictions."""
        q = np.empty(tree.L + 1, dtype=np.int32)
        y = np.empty(tree.L + 1, dtype=np.float32)
        _check(lib().h2_rankmodel_q_levels(self._m, tree.handle, kappa_T, density, tol, pad, q_max, q.ctypes.data,
                                           y.ctypes.data))
        return q, y

    def save(self, path: str):
        _check(lib().h2_rankmodel_save(self._m, os.fsencode(path)))

    @classmethod
    def load(cls, path: str) -> "RankModel":
        h = ctypes.c_void_p()
        _check(lib().h2_rankmodel_load(os.fsencode(path), ctypes.byref(h)))
        m = cls.__new__(cls)
        m._m = h
        return m

    def close(self):
        if self._m:
            lib().h2_rankmodel_free(self._m)
            self._m = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def rank_targets(G: "H2"):
    """(levels, log2(1 + need)) of the sampled levels of a construction (h2_rankmodel_targets)."""
    lv = (ctypes.c_int32 * H2_MAX_LEVELS)()
    tg = (ctypes.c_float * H2_MAX_LEVELS)()
    n = ctypes.c_int()
    _check(lib().h2_rankmodel_targets(G._h, lv, tg, ctypes.byref(n)))
    return [int(lv[i]) for i in range(n.value)], [float(tg[i]) for i in range(n.value)]


def launch_count() -> int:
    return int(lib().h2_launch_count())


def device_bytes() -> int:
    """Device bytes the library currently holds."""
    return int(lib().h2_device_bytes())


def set_device_limit(nbytes: int) -> None:
    """Cap the library's device bytes (<= 0 removes the cap); allocations above it fail with OOM."""
    _check(lib().h2_set_device_limit(int(nbytes)))


def version() -> str:
    return lib().h2_version().decode()
