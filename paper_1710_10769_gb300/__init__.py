"""Python binding of the GB300 HP-CONCORD library (``libhpconcord.so``).

Argument marshalling only: every step of the solver runs in the library's CUDA
kernels behind the C ABI of ``include/hpconcord.h``.  Functions keep the C
names without the ``hpc_`` prefix.  Device arrays are torch CUDA tensors (used
for device memory and streams); host arrays are numpy arrays.  There is no CPU
fallback: if the library cannot be loaded, every call raises.
"""
from __future__ import annotations

import ctypes as C
import dataclasses
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB = None

OK, NOT_CONVERGED = 0, 1
ERR_ARG, ERR_OOM, ERR_CAPACITY, ERR_NONPOS_DIAG, ERR_NAN, ERR_LS_FAIL, ERR_CUDA, ERR_NOT_IMPLEMENTED, \
    ERR_DEVICE_TIMEOUT = -1, -2, -3, -4, -5, -6, -7, -8, -9
COV, OBS, AUTO = 0, 1, 2
F32, F64, BF16 = 0, 1, 2
PREC_AUTO, PREC_FP64, PREC_FP32, PREC_BF16X3, PREC_TF32 = -1, 0, 1, 2, 3


class Options(C.Structure):
    _fields_ = [("eps", C.c_double), ("max_iter", C.c_int64), ("max_halvings", C.c_int32),
                ("precision", C.c_int32), ("value_dtype", C.c_int32), ("ls_window", C.c_int32),
                ("capacity", C.c_int64), ("max_capacity", C.c_int64), ("x_on_host", C.c_int32),
                ("timing", C.c_int32), ("device_loop", C.c_int32), ("reserved_", C.c_int32)]


class Stats(C.Structure):
    _fields_ = [("iterations", C.c_int64), ("ls_trials", C.c_int64), ("nnz", C.c_int64),
                ("status", C.c_int32), ("accepted_halvings", C.c_int32), ("f", C.c_double),
                ("F", C.c_double), ("rel_change", C.c_double), ("ms_total", C.c_double),
                ("ms_gram", C.c_double), ("ms_grad_pass", C.c_double), ("grad_pass_launches", C.c_int64),
                ("kernel_launches", C.c_int64), ("capacity_regrows", C.c_int64), ("candidates", C.c_int64),
                ("ms_gram_kernel", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Info(C.Structure):
    _fields_ = [("n", C.c_int64), ("p", C.c_int64), ("ld", C.c_int64), ("variant", C.c_int32),
                ("precision", C.c_int32), ("value_dtype", C.c_int32), ("pad_", C.c_int32),
                ("capacity", C.c_int64), ("device_bytes", C.c_int64), ("lambda1", C.c_double),
                ("lambda2", C.c_double)]


PRECISION_NAMES = {PREC_FP64: "fp64", PREC_FP32: "fp32", PREC_BF16X3: "bf16x3", PREC_TF32: "tf32"}


class PathPoint(C.Structure):
    _fields_ = [("lambda1", C.c_double), ("iterations", C.c_int64), ("ls_trials", C.c_int64), ("nnz", C.c_int64),
                ("status", C.c_int32), ("pad_", C.c_int32), ("f", C.c_double), ("F", C.c_double),
                ("rel_change", C.c_double), ("ms", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "pad_"}


class HypergradInfo(C.Structure):
    _fields_ = [("cg_iterations", C.c_int64), ("rel_residual", C.c_double), ("support", C.c_int64),
                ("converged", C.c_int32), ("pad_", C.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "pad_"}


class Tuning(C.Structure):
    _fields_ = [("gram_band", C.c_int32), ("ls_window", C.c_int32), ("ls_blocks_per_sm", C.c_int32),
                ("rows_ctas_per_sm", C.c_int32), ("gram_maxima", C.c_int32), ("screen_bounds", C.c_int32),
                ("gram_schedule", C.c_int32), ("gram_chunk", C.c_int32),
                ("gram_lead", C.c_int32), ("fused_tail", C.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


TUNE_MAX_TRIALS = 48
TUNE_KNOBS = ("gram_band", "ls_window", "ls_blocks_per_sm", "rows_ctas_per_sm", "gram_maxima", "gram_schedule")


class TuneTrial(C.Structure):
    _fields_ = [("knob", C.c_int32), ("value", C.c_int32), ("ms", C.c_double)]


class TuneReport(C.Structure):
    _fields_ = [("ntrials", C.c_int32), ("pad_", C.c_int32), ("trials", TuneTrial * TUNE_MAX_TRIALS)]

    def as_list(self):
        return [{"knob": TUNE_KNOBS[t.knob], "value": t.value, "ms": t.ms} for t in self.trials[: self.ntrials]]


class HpcError(RuntimeError):
    def __init__(self, status, where):
        lib = load()
        msg = lib.hpc_status_string(status).decode()
        extra = lib.hpc_last_error().decode()
        super().__init__(f"{where}: {msg} ({status}){' - ' + extra if extra else ''}")
        self.status = status


_P = C.c_void_p
_SIGS = {
    "hpc_default_options": (None, [C.POINTER(Options)]),
    "hpc_status_string": (C.c_char_p, [C.c_int]),
    "hpc_last_error": (C.c_char_p, []),
    "hpc_create": (C.c_int, [C.POINTER(_P), _P, C.c_int, C.c_int64, C.c_int64, C.c_double, C.c_double, C.c_int,
                             C.POINTER(Options), _P]),
    "hpc_load_x": (C.c_int, [_P, _P, C.c_int, C.c_int]),
    "hpc_prefetch_x": (C.c_int, [_P, _P, C.c_int, C.c_int]),
    "hpc_solve": (C.c_int, [_P, C.POINTER(Stats)]),
    "hpc_iterate": (C.c_int, [_P, C.c_int64, C.POINTER(Stats)]),
    "hpc_get_omega": (C.c_int, [_P, C.POINTER(C.c_int64), _P, _P, _P, C.c_int, C.c_int]),
    "hpc_set_omega": (C.c_int, [_P, C.c_int64, _P, _P, _P, C.c_int, C.c_int]),
    "hpc_set_lambda": (C.c_int, [_P, C.c_double, C.c_double]),
    "hpc_solve_batch": (C.c_int, [C.POINTER(_P), C.c_int, C.c_int, C.POINTER(Stats)]),
    "hpc_solve_path": (C.c_int, [_P, _P, C.c_int64, C.c_double, _P, _P, _P, _P, C.POINTER(C.c_int64)]),
    "hpc_get_s_entries": (C.c_int, [_P, C.c_int64, _P, _P, _P]),
    "hpc_get_candidates": (C.c_int, [_P, C.POINTER(C.c_int64), _P, _P, _P, _P]),
    "hpc_get_info": (C.c_int, [_P, C.POINTER(Info)]),
    "hpc_smooth_value": (C.c_int, [_P, C.POINTER(C.c_double)]),
    "hpc_backward": (C.c_int, [_P, _P, C.c_int, C.c_double, _P, C.c_int64, _P]),
    "hpc_backward_support": (C.c_int, [_P, _P, C.c_int, C.c_double, _P, _P]),
    "hpc_heldout_loss": (C.c_int, [_P, _P, C.c_int, C.c_int64, C.POINTER(C.c_double)]),
    "hpc_choose_variant": (C.c_int, [C.c_int64, C.c_int64, C.c_double, C.c_double, C.c_double, C.c_double,
                                     C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "hpc_hypergrad": (C.c_int, [_P, _P, C.c_int, C.c_int64, C.c_double, C.c_int64, C.POINTER(C.c_double),
                                C.POINTER(C.c_double), C.POINTER(HypergradInfo)]),
    "hpc_destroy": (C.c_int, [_P]),
    "hpc_gram": (C.c_int, [_P, C.c_int, C.c_int64, C.c_int64, _P, C.c_int, C.c_int64, C.c_int, _P]),
    "hpc_gram_noalloc": (C.c_int, [_P, C.c_int, C.c_int64, C.c_int64, _P, C.c_int64, C.c_int, _P]),
    "hpc_get_tuning": (C.c_int, [_P, _P]),
    "hpc_get_block_maxima": (C.c_int, [_P, C.POINTER(C.c_int64), _P]),
    "hpc_set_tuning": (C.c_int, [_P, _P]),
    "hpc_autotune": (C.c_int, [_P, _P, C.c_int, C.c_int, C.c_int64, _P, _P]),
}

EXPORTED = tuple(_SIGS)


def library_path() -> str:
    return os.path.join(_HERE, "libhpconcord.so")


def load(build_if_missing: bool = True):
    """Load libhpconcord.so (building it first if absent); raise if that fails."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = library_path()
    if not os.path.exists(path) and build_if_missing:
        from . import _build

        _build.build()
    lib = C.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _LIB = lib
    return lib


def _check(status, where, allow=(OK,)):
    if status not in allow:
        raise HpcError(status, where)
    return status


def default_options(**kw) -> Options:
    o = Options()
    load().hpc_default_options(C.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def _dtype_code(t) -> int:
    import torch

    if isinstance(t, np.ndarray):
        return {np.dtype(np.float32): F32, np.dtype(np.float64): F64}[t.dtype]
    return {torch.float32: F32, torch.float64: F64, torch.bfloat16: BF16}[t.dtype]


def _matrix(X, rows, cols, what, cuda=None, dtypes=None):
    """Check a row-major matrix argument before its pointer crosses the C ABI, which
    cannot see shapes: a 2-D torch tensor (or numpy array, on the host) of shape (rows,
    cols) (None: any), contiguous, of a supported dtype, on the device when cuda is
    True and on the host when False.  Raises TypeError / ValueError; returns X."""
    import torch

    if isinstance(X, np.ndarray):
        if cuda:
            raise ValueError(f"{what}: a CUDA tensor is required, got a numpy array")
        ok = {np.dtype(np.float32), np.dtype(np.float64)}
        if X.dtype not in ok:
            raise TypeError(f"{what}: dtype {X.dtype} is not float32 or float64")
    elif isinstance(X, torch.Tensor):
        if cuda is not None and X.is_cuda != cuda:
            raise ValueError(f"{what}: must be on the {'GPU' if cuda else 'host'}, got {X.device}")
        if not X.is_contiguous():
            raise ValueError(f"{what}: must be contiguous (row-major)")
        ok = dtypes or (torch.float32, torch.float64, torch.bfloat16)
        if X.dtype not in ok:
            raise TypeError(f"{what}: dtype {X.dtype} is not one of {ok}")
    else:
        raise TypeError(f"{what}: expected a torch tensor or numpy array, got {type(X).__name__}")
    if X.ndim != 2:
        raise ValueError(f"{what}: expected a 2-D matrix, got shape {tuple(X.shape)}")
    if (rows is not None and X.shape[0] != rows) or (cols is not None and X.shape[1] != cols):
        raise ValueError(f"{what}: expected shape ({rows if rows is not None else 'any'}, "
                         f"{cols if cols is not None else 'any'}), got {tuple(X.shape)}")
    return X


def _stream_ptr(stream):
    import torch

    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


@dataclasses.dataclass
class Csr:
    row_ptr: np.ndarray
    col: np.ndarray
    val: np.ndarray

    def to_scipy(self, p):
        import scipy.sparse as sp

        return sp.csr_matrix((self.val, self.col, self.row_ptr), shape=(p, p))


class Solver:
    """A solver handle (``hpc_create`` ... ``hpc_destroy``)."""

    def __init__(self, X, lambda1, lambda2, variant=COV, stream=None, n=None, p=None, xdtype=None, **options):
        lib = load()
        self._lib = lib
        self.options = default_options(**options)
        if isinstance(X, np.ndarray):
            self.options.x_on_host = 1
            X = np.ascontiguousarray(X)
            ptr = X.ctypes.data_as(C.c_void_p)
            n, p = X.shape
            xdt = _dtype_code(X)
        elif X is not None and not X.is_cuda:
            _matrix(X, None, None, "X", cuda=False)
            self.options.x_on_host = 1
            ptr = C.c_void_p(X.data_ptr())
            n, p = X.shape
            xdt = _dtype_code(X)
        elif X is None:
            ptr = None
            xdt = F32 if xdtype is None else xdtype
        else:
            _matrix(X, None, None, "X", cuda=True)
            ptr = C.c_void_p(X.data_ptr())
            n, p = X.shape
            xdt = _dtype_code(X)
        self.n, self.p = int(n), int(p)
        self._stream = _stream_ptr(stream)
        h = C.c_void_p()
        st = lib.hpc_create(C.byref(h), ptr, xdt, self.n, self.p, float(lambda1), float(lambda2), variant,
                            C.byref(self.options), self._stream)
        _check(st, "hpc_create")
        self._h = h
        self.stats = Stats()

    def close(self):
        if getattr(self, "_h", None):
            self._lib.hpc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def load_x(self, X):
        if isinstance(X, np.ndarray):
            X = _matrix(np.ascontiguousarray(X), self.n, self.p, "X")
            st = self._lib.hpc_load_x(self._h, X.ctypes.data_as(C.c_void_p), _dtype_code(X), 1)
        elif not _matrix(X, self.n, self.p, "X").is_cuda:
            st = self._lib.hpc_load_x(self._h, C.c_void_p(X.data_ptr()), _dtype_code(X), 1)
        else:
            st = self._lib.hpc_load_x(self._h, C.c_void_p(X.data_ptr()), _dtype_code(X), 0)
        return _check(st, "hpc_load_x")

    def prefetch_x(self, X):
        """hpc_prefetch_x: stage the next data set on a second stream (a copy-engine
        transfer now, its Gram panels after the next load's Gram).  Pipeline:
        prefetch_x(X_next); load_x(X_cur); solve() -- with distinct buffers."""
        if isinstance(X, np.ndarray):
            X = _matrix(np.ascontiguousarray(X), self.n, self.p, "X")
            st = self._lib.hpc_prefetch_x(self._h, X.ctypes.data_as(C.c_void_p), _dtype_code(X), 1)
        else:
            _matrix(X, self.n, self.p, "X")
            st = self._lib.hpc_prefetch_x(self._h, C.c_void_p(X.data_ptr()), _dtype_code(X), 0 if X.is_cuda else 1)
        return _check(st, "hpc_prefetch_x")

    def solve(self, allow_not_converged=True) -> Stats:
        st = self._lib.hpc_solve(self._h, C.byref(self.stats))
        _check(st, "hpc_solve", (OK, NOT_CONVERGED) if allow_not_converged else (OK,))
        return self.stats

    def iterate(self, k) -> Stats:
        st = self._lib.hpc_iterate(self._h, int(k), C.byref(self.stats))
        _check(st, "hpc_iterate")
        return self.stats

    def block_maxima(self) -> np.ndarray:
        """hpc_get_block_maxima: the bound screening's max |S_ij| per (row, column block)
        as float32 (decoded from the BF16 bit patterns), shape (p, nb)."""
        c = C.c_int64(0)
        _check(self._lib.hpc_get_block_maxima(self._h, C.byref(c), None), "hpc_get_block_maxima")
        out = np.empty(c.value, np.uint16)
        _check(self._lib.hpc_get_block_maxima(self._h, C.byref(c), out.ctypes.data_as(C.c_void_p)),
               "hpc_get_block_maxima")
        return (out.astype(np.uint32) << 16).view(np.float32).reshape(self.p, -1)

    def get_tuning(self) -> dict:
        t = Tuning()
        _check(self._lib.hpc_get_tuning(self._h, C.byref(t)), "hpc_get_tuning")
        return t.as_dict()

    def set_tuning(self, **kw):
        t = Tuning()
        _check(self._lib.hpc_get_tuning(self._h, C.byref(t)), "hpc_get_tuning")
        for k, v in kw.items():
            setattr(t, k, int(v))
        _check(self._lib.hpc_set_tuning(self._h, C.byref(t)), "hpc_set_tuning")

    def autotune(self, X=None, iters=5):
        """hpc_autotune: time the launch-shape candidates on this problem and keep the
        fastest.  With X the Gram's band is tuned too (the data is reloaded and the
        iterate returns to the identity, as in load_x).  Returns (tuning, trials)."""
        t = Tuning()
        rep = TuneReport()
        if X is None:
            ptr, xdt, host = None, F32, 0
        elif isinstance(X, np.ndarray):
            X = _matrix(np.ascontiguousarray(X), self.n, self.p, "X")
            ptr, xdt, host = X.ctypes.data_as(C.c_void_p), _dtype_code(X), 1
        else:
            _matrix(X, self.n, self.p, "X")
            ptr, xdt, host = C.c_void_p(X.data_ptr()), _dtype_code(X), 0 if X.is_cuda else 1
        _check(self._lib.hpc_autotune(self._h, ptr, xdt, host, int(iters), C.byref(t), C.byref(rep)), "hpc_autotune")
        return t.as_dict(), rep.as_list()

    def info(self) -> Info:
        inf = Info()
        _check(self._lib.hpc_get_info(self._h, C.byref(inf)), "hpc_get_info")
        return inf

    def precision_used(self) -> int:
        return self.info().precision

    def precision_name(self) -> str:
        return PRECISION_NAMES[self.precision_used()]

    def nnz(self) -> int:
        m = C.c_int64(0)
        _check(self._lib.hpc_get_omega(self._h, C.byref(m), None, None, None, F64, 0), "hpc_get_omega")
        return m.value

    def get_omega(self, dtype=np.float64) -> Csr:
        m = C.c_int64(self.nnz())
        rp = np.empty(self.p + 1, np.int64)
        ci = np.empty(max(m.value, 1), np.int32)
        v = np.empty(max(m.value, 1), dtype)
        code = F64 if np.dtype(dtype) == np.float64 else F32
        _check(self._lib.hpc_get_omega(self._h, C.byref(m), rp.ctypes.data_as(C.c_void_p),
                                       ci.ctypes.data_as(C.c_void_p), v.ctypes.data_as(C.c_void_p), code, 0),
               "hpc_get_omega")
        return Csr(rp, ci[: m.value], v[: m.value])

    def get_omega_device(self, row_ptr, col, val):
        m = C.c_int64(col.numel())
        code = F64 if str(val.dtype) == "torch.float64" else F32
        _check(self._lib.hpc_get_omega(self._h, C.byref(m), C.c_void_p(row_ptr.data_ptr()),
                                       C.c_void_p(col.data_ptr()), C.c_void_p(val.data_ptr()), code, 1),
               "hpc_get_omega")
        return m.value

    def omega_dense(self) -> np.ndarray:
        return self.get_omega().to_scipy(self.p).toarray()

    def set_omega(self, csr: Csr):
        rp = np.ascontiguousarray(csr.row_ptr, dtype=np.int64)
        ci = np.ascontiguousarray(csr.col, dtype=np.int32)
        v = np.ascontiguousarray(csr.val, dtype=np.float64)
        return _check(self._lib.hpc_set_omega(self._h, int(ci.size), rp.ctypes.data_as(C.c_void_p),
                                              ci.ctypes.data_as(C.c_void_p), v.ctypes.data_as(C.c_void_p), F64, 0),
                      "hpc_set_omega")

    def set_lambda(self, lambda1, lambda2):
        return _check(self._lib.hpc_set_lambda(self._h, float(lambda1), float(lambda2)), "hpc_set_lambda")

    def solve_path(self, lambda1s, lambda2, return_estimates=True, capacity=None):
        """Warm-started path over lambda1s (``hpc_solve_path``): (points, [Csr per point])."""
        lam = np.ascontiguousarray(lambda1s, dtype=np.float64)
        k = lam.size
        pts = (PathPoint * max(k, 1))()
        if not return_estimates:
            st = self._lib.hpc_solve_path(self._h, lam.ctypes.data_as(C.c_void_p), k, float(lambda2), pts,
                                          None, None, None, None)
            _check(st, "hpc_solve_path", (OK, NOT_CONVERGED))
            return [pts[t].as_dict() for t in range(k)], None
        cap = capacity or max(64 * self.p * k, 1024)
        while True:
            rp = np.empty(k * (self.p + 1), np.int64)
            ci = np.empty(cap, np.int32)
            v = np.empty(cap, np.float32)
            c = C.c_int64(cap)
            st = self._lib.hpc_solve_path(self._h, lam.ctypes.data_as(C.c_void_p), k, float(lambda2), pts,
                                          rp.ctypes.data_as(C.c_void_p), ci.ctypes.data_as(C.c_void_p),
                                          v.ctypes.data_as(C.c_void_p), C.byref(c))
            if st == ERR_CAPACITY and c.value > cap:
                raise HpcError(st, "hpc_solve_path (output capacity %d < %d)" % (cap, c.value))
            _check(st, "hpc_solve_path", (OK, NOT_CONVERGED))
            break
        out, off = [], 0
        for t in range(k):
            r = rp[t * (self.p + 1):(t + 1) * (self.p + 1)]
            m = int(r[-1])
            out.append(Csr(r.copy(), ci[off:off + m].copy(), v[off:off + m].astype(np.float64)))
            off += m
        return [pts[t].as_dict() for t in range(k)], out

    # ------------------------------------------------------------ differentiation
    def smooth_value(self) -> float:
        """f(Omega) at the current estimate (``hpc_smooth_value``)."""
        f = C.c_double(0.0)
        _check(self._lib.hpc_smooth_value(self._h, C.byref(f)), "hpc_smooth_value")
        return f.value

    def backward(self, X, grad_loss=1.0, domega=True, dx=True):
        """(dL/dOmega dense (p, p), dL/dX (n, p)) times grad_loss at the current estimate
        (``hpc_backward``); X is the device data the solver was loaded with."""
        import torch

        _matrix(X, self.n, self.p, "X", cuda=True)
        dt = torch.float64 if self.info().value_dtype == F64 else torch.float32
        dO = torch.empty((self.p, self.p), dtype=dt, device=X.device) if domega else None
        dX = torch.empty((self.n, self.p), dtype=dt, device=X.device) if dx else None
        st = self._lib.hpc_backward(self._h, C.c_void_p(X.data_ptr()), _dtype_code(X), float(grad_loss),
                                    C.c_void_p(dO.data_ptr()) if dO is not None else None,
                                    dO.stride(0) if dO is not None else self.p,
                                    C.c_void_p(dX.data_ptr()) if dX is not None else None)
        _check(st, "hpc_backward")
        return dO, dX

    def backward_support(self, X=None, grad_loss=1.0, dx=False):
        """(dL/dOmega at the estimate's entries in CSR order as an FP64 (nnz,) device tensor,
        dL/dX (n, p) or None) times grad_loss (``hpc_backward_support``)."""
        import torch

        dev = X.device if X is not None else torch.device("cuda")
        if X is not None:
            _matrix(X, self.n, self.p, "X", cuda=True)
        elif dx:
            raise ValueError("dx needs X")
        m = self.nnz()
        dv = torch.empty(max(m, 1), dtype=torch.float64, device=dev)
        dX = None
        if dx:
            dt = torch.float64 if self.info().value_dtype == F64 else torch.float32
            dX = torch.empty((self.n, self.p), dtype=dt, device=dev)
        st = self._lib.hpc_backward_support(self._h, C.c_void_p(X.data_ptr()) if X is not None else None,
                                            _dtype_code(X) if X is not None else F32, float(grad_loss),
                                            C.c_void_p(dv.data_ptr()),
                                            C.c_void_p(dX.data_ptr()) if dX is not None else None)
        _check(st, "hpc_backward_support")
        return dv[:m], dX

    def set_omega_device(self, row_ptr, col, val):
        """hpc_set_omega from device tensors: row_ptr (p+1,) int64, col (nnz,) int32, val (nnz,)
        float32 or float64; a symmetric pattern with every diagonal entry present and positive."""
        code = F64 if str(val.dtype) == "torch.float64" else F32
        return _check(self._lib.hpc_set_omega(self._h, int(col.numel()), C.c_void_p(row_ptr.data_ptr()),
                                              C.c_void_p(col.data_ptr()), C.c_void_p(val.data_ptr()), code, 1),
                      "hpc_set_omega")

    def heldout_loss(self, Xval) -> float:
        """L_val = -sum log w_ii + tr(Omega S_val Omega)/2 at the current estimate (``hpc_heldout_loss``)."""
        _matrix(Xval, None, self.p, "Xval", cuda=True)
        out = C.c_double(0.0)
        _check(self._lib.hpc_heldout_loss(self._h, C.c_void_p(Xval.data_ptr()), _dtype_code(Xval), Xval.shape[0],
                                          C.byref(out)), "hpc_heldout_loss")
        return out.value

    def hypergrad(self, Xval, tol=1e-8, max_iter=20000):
        """(dL_val/dlambda1, dL_val/dlambda2, info) at the current estimate (``hpc_hypergrad``)."""
        _matrix(Xval, None, self.p, "Xval", cuda=True)
        d1, d2 = C.c_double(0.0), C.c_double(0.0)
        inf = HypergradInfo()
        st = self._lib.hpc_hypergrad(self._h, C.c_void_p(Xval.data_ptr()), _dtype_code(Xval), Xval.shape[0],
                                     float(tol), int(max_iter), C.byref(d1), C.byref(d2), C.byref(inf))
        _check(st, "hpc_hypergrad", (OK, NOT_CONVERGED))
        return d1.value, d2.value, inf.as_dict()

    def omega_values(self, device="cuda", dtype=None):
        """The estimate's CSR (row_ptr, col, val) as device tensors (``hpc_get_omega`` on device)."""
        import torch

        m = self.nnz()
        dt = dtype or (torch.float64 if self.info().value_dtype == F64 else torch.float32)
        rp = torch.empty(self.p + 1, dtype=torch.int64, device=device)
        ci = torch.empty(max(m, 1), dtype=torch.int32, device=device)
        v = torch.empty(max(m, 1), dtype=dt, device=device)
        self.get_omega_device(rp, ci, v)
        return rp, ci[:m], v[:m]

    def s_entries(self, rows, cols) -> np.ndarray:
        rows = np.ascontiguousarray(rows, dtype=np.int64)
        cols = np.ascontiguousarray(cols, dtype=np.int64)
        out = np.empty(rows.size, np.float64)
        _check(self._lib.hpc_get_s_entries(self._h, rows.size, rows.ctypes.data_as(C.c_void_p),
                                           cols.ctypes.data_as(C.c_void_p), out.ctypes.data_as(C.c_void_p)),
               "hpc_get_s_entries")
        return out

    def candidates(self):
        m = C.c_int64(0)
        _check(self._lib.hpc_get_candidates(self._h, C.byref(m), None, None, None, None), "hpc_get_candidates")
        k = m.value
        r = np.empty(max(k, 1), np.int64)
        c = np.empty(max(k, 1), np.int64)
        o = np.empty(max(k, 1), np.float64)
        g = np.empty(max(k, 1), np.float64)
        _check(self._lib.hpc_get_candidates(self._h, C.byref(m), r.ctypes.data_as(C.c_void_p),
                                            c.ctypes.data_as(C.c_void_p), o.ctypes.data_as(C.c_void_p),
                                            g.ctypes.data_as(C.c_void_p)), "hpc_get_candidates")
        return r[:k], c[:k], o[:k], g[:k]


def _check_s(S, p, dtypes):
    """S for hpc_gram*: a CUDA (p, lds) tensor with lds >= p and unit column stride."""
    import torch

    if not isinstance(S, torch.Tensor) or not S.is_cuda or S.dim() != 2:
        raise ValueError("S: expected a 2-D CUDA tensor")
    if S.dtype not in dtypes:
        raise TypeError(f"S: dtype {S.dtype} is not one of {dtypes}")
    if S.shape[0] != p or S.shape[1] < p or S.stride(1) != 1 or S.stride(0) < p:
        raise ValueError(f"S: expected ({p}, >= {p}) rows of unit stride, got shape {tuple(S.shape)} "
                         f"strides {S.stride()}")


def gram(X, S, precision=PREC_AUTO, stream=None):
    """S = X^T X / n on the device (``hpc_gram``); S is a (p, lds) tensor, lds >= p."""
    import torch

    n, p = _matrix(X, None, None, "X", cuda=True).shape
    _check_s(S, p, (torch.float32, torch.float64))
    st = load().hpc_gram(C.c_void_p(X.data_ptr()), _dtype_code(X), n, p, C.c_void_p(S.data_ptr()),
                         _dtype_code(S), S.stride(0), precision, _stream_ptr(stream))
    return _check(st, "hpc_gram")


GRAM_NOALLOC_SCRATCH_BYTES = 64 << 20


def gram_noalloc(X, S, precision=PREC_AUTO, stream=None):
    """S = X^T X / n through ``hpc_gram_noalloc``: the tensor-core Gram with its scratch in a
    static device array, for callers that must not allocate device memory; S is a float32
    (p, lds) tensor."""
    import torch

    n, p = _matrix(X, None, None, "X", cuda=True).shape
    _check_s(S, p, (torch.float32,))
    st = load().hpc_gram_noalloc(C.c_void_p(X.data_ptr()), _dtype_code(X), n, p, C.c_void_p(S.data_ptr()),
                                 S.stride(0), precision, _stream_ptr(stream))
    return _check(st, "hpc_gram_noalloc")


def _make_smooth_loss():
    import torch

    class ConcordSmoothLoss(torch.autograd.Function):
        """L(Omega, X) = -sum log w_ii + tr(Omega S Omega)/2 + lambda2/2 ||Omega||_F^2, S = X^T X / n,
        evaluated at the Omega it is given, with the library's adjoint as backward.

        Inputs: X (n, p), the device data the solver was loaded with; omega, either
        - the values (nnz,) of a matrix with the solver's current CSR pattern
          (Solver.omega_values() gives the estimate's), or
        - a dense symmetric (p, p) tensor with a positive diagonal;
        and the solver.  forward loads omega into the solver as its iterate (hpc_set_omega:
        it replaces the solver's estimate) and returns f there (hpc_smooth_value); backward
        returns dL/dX (hpc_backward) and dL/dOmega at the same omega: dense from
        hpc_backward for the dense form, on the pattern from hpc_backward_support (no p x p
        buffer) for the values form."""

        @staticmethod
        def forward(ctx, X, omega, solver):
            p = solver.p
            dev = X.device
            if tuple(omega.shape) == (p, p):
                if not torch.equal(omega, omega.t()):
                    raise ValueError("omega: the smooth loss is defined here for symmetric matrices")
                nz = omega != 0
                nz.fill_diagonal_(True)
                rows, cols = nz.nonzero(as_tuple=True)               # row-major: columns ascending
                counts = torch.bincount(rows, minlength=p)
                rp = torch.zeros(p + 1, dtype=torch.int64, device=dev)
                rp[1:] = torch.cumsum(counts, 0)
                vals = omega[rows, cols].to(torch.float64)
                solver.set_omega_device(rp, cols.to(torch.int32).contiguous(), vals.contiguous())
                ctx.form = "dense"
            else:
                rp, ci, cur = solver.omega_values(device=dev)
                if omega.dim() != 1 or omega.numel() != ci.numel():
                    raise ValueError(f"omega: expected ({p}, {p}) or the ({ci.numel()},) values of the solver's "
                                     f"pattern, got {tuple(omega.shape)}")
                solver.set_omega_device(rp, ci, omega.detach().to(cur.dtype).contiguous())
                ctx.form = "values"
            ctx.solver = solver
            ctx.save_for_backward(X)
            ctx.omega_dtype = omega.dtype
            return torch.tensor(solver.smooth_value(), dtype=torch.float64, device=dev)

        @staticmethod
        def backward(ctx, gL):
            (X,) = ctx.saved_tensors
            s = ctx.solver
            want_o, want_x = ctx.needs_input_grad[1], ctx.needs_input_grad[0]
            g_om, dX = None, None
            if ctx.form == "dense":
                dO, dX = s.backward(X, float(gL), domega=want_o, dx=want_x)
                if want_o:
                    g_om = dO.to(ctx.omega_dtype)
            else:
                dv, dX = s.backward_support(X, float(gL), dx=want_x)
                if want_o:
                    g_om = dv.to(ctx.omega_dtype)
            if want_x:
                dX = dX.to(X.dtype)
            return dX, g_om, None

    return ConcordSmoothLoss


_SMOOTH_LOSS = None


def concord_smooth_loss(X, omega, solver):
    """Autograd entry point of the smooth CONCORD loss (see ConcordSmoothLoss)."""
    global _SMOOTH_LOSS
    if _SMOOTH_LOSS is None:
        _SMOOTH_LOSS = _make_smooth_loss()
    return _SMOOTH_LOSS.apply(X, omega, solver)


def choose_variant(n, p, s=0.0, t=0.0, d=0.0, gamma_ratio=0.0):
    """Lemma 3.1's choice (``hpc_choose_variant``): (COV or OBS, modelled Cov cost, modelled Obs cost)."""
    lib = load()
    cc, co = C.c_double(0.0), C.c_double(0.0)
    v = lib.hpc_choose_variant(int(n), int(p), float(s), float(t), float(d), float(gamma_ratio), C.byref(cc),
                               C.byref(co))
    if v < 0:
        raise HpcError(v, "hpc_choose_variant")
    return v, cc.value, co.value


def solve_batch(solvers, threads=0):
    """Solve independent problems concurrently (``hpc_solve_batch``); each Solver should have
    been created on its own CUDA stream.  Returns the list of per-problem stats dicts."""
    lib = load()
    k = len(solvers)
    hs = (C.c_void_p * max(k, 1))(*[s._h for s in solvers])
    st = (Stats * max(k, 1))()
    _check(lib.hpc_solve_batch(hs, k, int(threads), st), "hpc_solve_batch", (OK, NOT_CONVERGED))
    return [st[t].as_dict() for t in range(k)]
