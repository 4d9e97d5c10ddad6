"""Thin ctypes binding over the C ABI in include/nufft_gb300.h.

Argument marshalling only: every step of the transform runs in the CUDA
library.  Arrays are torch CUDA tensors (PyTorch provides device memory and the
stream); the functions take their raw device pointers.  If the compiled
library is missing this module raises instead of falling back to anything.
"""
from __future__ import annotations

import ctypes
import os
import threading

from .build import LIB

NUFFT_OK = 0
NUFFT_ERR_ARG = -1
NUFFT_ERR_EPS = -2
NUFFT_ERR_SIZE = -3
NUFFT_ERR_ALLOC = -4
NUFFT_ERR_CUDA = -5
NUFFT_ERR_CUFFT = -6
NUFFT_ERR_NOPTS = -7
NUFFT_ERR_CHECK = -8
FAIL_ALLOC, FAIL_CUFFT = 1, 2
NUFFT_ERR_METHOD = -9

METHOD_AUTO, METHOD_GM, METHOD_GM_SORT, METHOD_SM = 0, 1, 2, 3
METHODS = {"auto": 0, "gm": 1, "gmsort": 2, "sm": 3}

# symbols declared in include/nufft_gb300.h
EXPORTS = (
    "nufft_default_opts", "nufft_makeplan", "nufft_setpts", "nufft_execute", "nufft_destroy",
    "nufft_strerror", "nufft_spread", "nufft_interp", "nufft_fft", "nufft_deconvolve",
    "nufft_precorrect", "nufft_get_params", "nufft_get_finegrid", "nufft_get_sort",
    "nufft_spread_add", "nufft_get_launch_count", "nufft_binsort_noalloc",
    "nufft_batch_create", "nufft_batch_execute", "nufft_batch_capture", "nufft_batch_launch",
    "nufft_batch_destroy", "nufft_autotune", "nufft_tune_cache_save", "nufft_tune_cache_load",
    "nufft_tune_cache_clear", "nufft_get_tiles", "nufft_picker_create", "nufft_picker_destroy",
    "nufft_picker_set_params", "nufft_picker_get_params", "nufft_picker_save",
    "nufft_picker_load", "nufft_picker_predict", "nufft_picker_grad", "nufft_picker_step",
    "nufft_picker_train", "nufft_picker_loss", "nufft_picker_install", "nufft_picker_features",
    "nufft_point_skew", "nufft_fma_peak", "nufft_execute_host", "nufft_get_status",
    "nufft_debug_fail", "nufft_setpts3", "nufft_pick",
)

PICKER_NFEAT = 12
PICKER_NPARAM = 5057


class NufftError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        super().__init__("%s failed: %s (%d)" % (where, strerror(code), code))


class TuneTrial(ctypes.Structure):
    _fields_ = [
        ("method", ctypes.c_int),
        ("bin", ctypes.c_int * 3),
        ("msub", ctypes.c_int),
        ("threads", ctypes.c_int),
        ("exec_ms", ctypes.c_double),
        ("setpts_ms", ctypes.c_double),
    ]


class Opts(ctypes.Structure):
    _fields_ = [
        ("method", ctypes.c_int),
        ("bin", ctypes.c_int * 3),
        ("msub", ctypes.c_int),
        ("upsampfac", ctypes.c_double),
        ("stream", ctypes.c_void_p),
        ("threads", ctypes.c_int),
        ("ctas_per_sm", ctypes.c_int),
        ("use_picker", ctypes.c_int),
        ("unordered_bins", ctypes.c_int),
        ("debug_checks", ctypes.c_int),
    ]


_lib = None
_lock = threading.Lock()


def library_path() -> str:
    return LIB


def load():
    """Load libnufft_gb300.so; raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB):
            raise ImportError("libnufft_gb300.so is not built (run __graft_entry__.build() "
                              "or python -m paper_2102_08463_gb300.build): %s" % LIB)
        lib = ctypes.CDLL(LIB)
        P = ctypes.c_void_p
        I = ctypes.c_int
        I64 = ctypes.c_int64
        lib.nufft_default_opts.argtypes = [ctypes.POINTER(Opts)]
        lib.nufft_default_opts.restype = None
        lib.nufft_makeplan.argtypes = [I, I, ctypes.POINTER(I64), I, I, ctypes.c_double, I,
                                       ctypes.POINTER(Opts), ctypes.POINTER(P)]
        lib.nufft_setpts.argtypes = [P, I64, P, P, P]
        lib.nufft_setpts3.argtypes = [P, I64, P, P, P, I64, P, P, P]
        lib.nufft_execute.argtypes = [P, P, P]
        lib.nufft_destroy.argtypes = [P]
        lib.nufft_strerror.argtypes = [I]
        lib.nufft_strerror.restype = ctypes.c_char_p
        lib.nufft_spread.argtypes = [P, P]
        lib.nufft_interp.argtypes = [P, P]
        lib.nufft_fft.argtypes = [P]
        lib.nufft_deconvolve.argtypes = [P, P]
        lib.nufft_precorrect.argtypes = [P, P]
        lib.nufft_get_params.argtypes = [P, ctypes.POINTER(I), ctypes.POINTER(ctypes.c_double),
                                         ctypes.POINTER(I64), ctypes.POINTER(I),
                                         ctypes.POINTER(I64), ctypes.POINTER(I),
                                         ctypes.POINTER(I)]
        lib.nufft_get_finegrid.argtypes = [P, ctypes.POINTER(P), ctypes.POINTER(ctypes.c_size_t)]
        lib.nufft_get_sort.argtypes = [P, P, P, P]
        lib.nufft_spread_add.argtypes = [P, P]
        lib.nufft_get_launch_count.argtypes = []
        lib.nufft_autotune.argtypes = [I, I, ctypes.POINTER(I64), I, I, ctypes.c_double, I,
                                       ctypes.POINTER(Opts), I64, P, P, P, P, P, I,
                                       ctypes.POINTER(Opts), ctypes.POINTER(ctypes.c_double),
                                       ctypes.POINTER(TuneTrial), I, ctypes.POINTER(I)]
        lib.nufft_tune_cache_save.argtypes = [ctypes.c_char_p]
        lib.nufft_tune_cache_load.argtypes = [ctypes.c_char_p]
        lib.nufft_tune_cache_clear.argtypes = []
        lib.nufft_batch_create.argtypes = [ctypes.POINTER(P), I, P, ctypes.POINTER(P)]
        lib.nufft_batch_execute.argtypes = [P, ctypes.POINTER(P), ctypes.POINTER(P)]
        lib.nufft_batch_capture.argtypes = [P, ctypes.POINTER(P), ctypes.POINTER(P)]
        lib.nufft_batch_launch.argtypes = [P]
        lib.nufft_batch_destroy.argtypes = [P]
        lib.nufft_binsort_noalloc.argtypes = [I, I, I64, P, P, P, ctypes.POINTER(I64),
                                              ctypes.POINTER(I), P, P, P]
        F = ctypes.c_float
        FP = ctypes.POINTER(ctypes.c_float)
        lib.nufft_get_tiles.argtypes = [P, ctypes.POINTER(Opts)]
        lib.nufft_picker_create.argtypes = [ctypes.c_uint64, ctypes.POINTER(P)]
        lib.nufft_picker_destroy.argtypes = [P]
        lib.nufft_picker_set_params.argtypes = [P, FP]
        lib.nufft_picker_get_params.argtypes = [P, FP]
        lib.nufft_picker_save.argtypes = [P, ctypes.c_char_p]
        lib.nufft_picker_load.argtypes = [P, ctypes.c_char_p]
        lib.nufft_picker_predict.argtypes = [P, I64, P, P, P]
        lib.nufft_picker_grad.argtypes = [P, I64, P, P, P, P, P]
        lib.nufft_picker_step.argtypes = [P, I64, P, P, F, P, P]
        lib.nufft_picker_train.argtypes = [P, I64, P, P, I, I, F, ctypes.c_uint64, FP, P]
        lib.nufft_picker_loss.argtypes = [P, I64, P, P, P, P]
        lib.nufft_picker_install.argtypes = [P]
        lib.nufft_picker_features.argtypes = [I, I, ctypes.POINTER(I64), ctypes.c_double, I,
                                              ctypes.c_double, I64, ctypes.c_double,
                                              ctypes.POINTER(Opts), FP]
        lib.nufft_point_skew.argtypes = [I, I, I64, P, P, P, ctypes.POINTER(ctypes.c_double), P]
        lib.nufft_pick.argtypes = [I, I, ctypes.POINTER(I64), ctypes.c_double, I, I64, P, P, P, P,
                                   ctypes.POINTER(Opts)]
        lib.nufft_fma_peak.argtypes = [I, ctypes.POINTER(ctypes.c_double), P]
        lib.nufft_execute_host.argtypes = [P, I64, P, P, P, P, P]
        lib.nufft_get_status.argtypes = [P]
        lib.nufft_debug_fail.argtypes = [I, I]
        for name in EXPORTS:
            if name not in ("nufft_default_opts", "nufft_strerror", "nufft_get_launch_count"):
                getattr(lib, name).restype = I
        lib.nufft_get_launch_count.restype = ctypes.c_uint64
        _lib = lib
        return lib


def strerror(code: int) -> str:
    try:
        return load().nufft_strerror(int(code)).decode()
    except ImportError:
        return "error %d" % code


def default_opts() -> Opts:
    o = Opts()
    load().nufft_default_opts(ctypes.byref(o))
    return o


def _check(rc, where):
    if rc != NUFFT_OK:
        raise NufftError(rc, where)


def _dptr(t, dtype=None, what="array"):
    """Raw device pointer of a contiguous CUDA tensor (None passes NULL)."""
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("%s must be a CUDA tensor" % what)
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % what)
    if dtype is not None and t.dtype != dtype:
        raise TypeError("%s has dtype %s, expected %s" % (what, t.dtype, dtype))
    return ctypes.c_void_p(t.data_ptr())


def _hptr(t, dtype=None, what="array"):
    """Raw pointer of a contiguous host (CPU) tensor (None passes NULL)."""
    if t is None:
        return None
    if t.is_cuda:
        raise ValueError("%s must be a host tensor" % what)
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % what)
    if dtype is not None and t.dtype != dtype:
        raise TypeError("%s must be %s, got %s" % (what, dtype, t.dtype))
    return ctypes.c_void_p(t.data_ptr())


def makeplan(type_, dim, nmodes, iflag=+1, ntransf=1, eps=1e-6, prec=-1, opts=None):
    """nufft_makeplan; returns the opaque handle (int)."""
    lib = load()
    arr = (ctypes.c_int64 * 3)(*([int(v) for v in nmodes] + [1] * (3 - len(nmodes))))
    h = ctypes.c_void_p()
    rc = lib.nufft_makeplan(int(type_), int(dim), arr, int(iflag), int(ntransf), float(eps),
                            int(prec), ctypes.byref(opts) if opts is not None else None,
                            ctypes.byref(h))
    _check(rc, "nufft_makeplan")
    return h.value


def setpts(h, M, x, y, z=None):
    _check(load().nufft_setpts(ctypes.c_void_p(h), int(M), x, y, z), "nufft_setpts")


def setpts3(h, M, x, y, z, K, s, t, u):
    _check(load().nufft_setpts3(ctypes.c_void_p(h), int(M), x, y, z, int(K), s, t, u),
           "nufft_setpts3")


def execute(h, c, f):
    _check(load().nufft_execute(ctypes.c_void_p(h), c, f), "nufft_execute")


def destroy(h):
    if h:
        _check(load().nufft_destroy(ctypes.c_void_p(h)), "nufft_destroy")


def spread(h, c):
    _check(load().nufft_spread(ctypes.c_void_p(h), c), "nufft_spread")


def spread_add(h, c):
    _check(load().nufft_spread_add(ctypes.c_void_p(h), c), "nufft_spread_add")


def binsort_noalloc(dim, prec, M, x, y, z, nf, bins, perm, bincount, stream=None):
    """nufft_binsort_noalloc: stable bin-sort into caller buffers, no allocation."""
    nfa = (ctypes.c_int64 * 3)(*([int(v) for v in nf] + [1] * (3 - len(nf))))
    ba = (ctypes.c_int * 3)(*([int(v) for v in bins] + [1] * (3 - len(bins))))
    _check(load().nufft_binsort_noalloc(int(dim), int(prec), int(M), x, y, z, nfa, ba, perm,
                                        bincount, stream), "nufft_binsort_noalloc")


def autotune(type_, N, eps, M, x, y, z, c, f, iflag=+1, ntransf=1, prec=-1, reps=3,
             base=None, stream=None, max_trials=256):
    """nufft_autotune on torch tensors; returns (best Opts, best_ms, list of trial dicts)."""
    import torch
    lib = load()
    o = base if base is not None else default_opts()
    if stream is None:
        stream = torch.cuda.current_stream()
    o.stream = ctypes.c_void_p(stream.cuda_stream)
    arr = (ctypes.c_int64 * 3)(*([int(v) for v in N] + [1] * (3 - len(N))))
    best = Opts()
    ms = ctypes.c_double()
    trials = (TuneTrial * max_trials)()
    nt = ctypes.c_int()
    _check(lib.nufft_autotune(int(type_), len(N), arr, int(iflag), int(ntransf), float(eps),
                              int(prec), ctypes.byref(o), int(M), _dptr(x), _dptr(y), _dptr(z),
                              _dptr(c), _dptr(f), int(reps), ctypes.byref(best), ctypes.byref(ms),
                              trials, max_trials, ctypes.byref(nt)), "nufft_autotune")
    out = [dict(method=t.method, bin=tuple(t.bin), msub=t.msub, threads=t.threads,
                exec_ms=t.exec_ms, setpts_ms=t.setpts_ms) for t in trials[: nt.value]]
    return best, ms.value, out


def tune_cache_save(path):
    _check(load().nufft_tune_cache_save(str(path).encode()), "nufft_tune_cache_save")


def tune_cache_load(path):
    _check(load().nufft_tune_cache_load(str(path).encode()), "nufft_tune_cache_load")


def tune_cache_clear():
    _check(load().nufft_tune_cache_clear(), "nufft_tune_cache_clear")


class Batch:
    """Batched execution of several Plan objects (nufft_batch_*).

    Batch(plans, stream=None): plans must have their points set.  execute(cs, fs)
    runs all transforms (cs[k], fs[k] as Plan.execute would take / fill);
    capture(cs, fs) records a CUDA graph that launch() replays.
    """

    def __init__(self, plans, stream=None):
        import torch
        self.plans = list(plans)
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        arr = (ctypes.c_void_p * len(self.plans))(*[p.handle for p in self.plans])
        h = ctypes.c_void_p()
        _check(load().nufft_batch_create(arr, len(self.plans), ctypes.c_void_p(stream.cuda_stream),
                                         ctypes.byref(h)), "nufft_batch_create")
        self.handle = h.value

    def _ptrs(self, cs, fs):
        n = len(self.plans)
        c = (ctypes.c_void_p * n)(*[ctypes.c_void_p(x.data_ptr()) if x is not None else None
                                    for x in cs])
        f = (ctypes.c_void_p * n)(*[ctypes.c_void_p(x.data_ptr()) for x in fs])
        self._keep = (cs, fs)
        return c, f

    def execute(self, cs, fs):
        c, f = self._ptrs(cs, fs)
        _check(load().nufft_batch_execute(ctypes.c_void_p(self.handle), c, f), "nufft_batch_execute")

    def capture(self, cs, fs):
        c, f = self._ptrs(cs, fs)
        _check(load().nufft_batch_capture(ctypes.c_void_p(self.handle), c, f), "nufft_batch_capture")

    def launch(self):
        _check(load().nufft_batch_launch(ctypes.c_void_p(self.handle)), "nufft_batch_launch")

    def close(self):
        if self.handle:
            load().nufft_batch_destroy(ctypes.c_void_p(self.handle))
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def get_tiles(h):
    """The plan's current method, bins, M_sub and threads."""
    o = Opts()
    _check(load().nufft_get_tiles(ctypes.c_void_p(h), ctypes.byref(o)), "nufft_get_tiles")
    return dict(method=o.method, bin=tuple(o.bin), msub=o.msub, threads=o.threads)


def picker_features(type_, N, eps, M, skew, method, bins=None, msub=0, threads=0, prec=-1,
                    upsampfac=2.0):
    """nufft_picker_features: the 12 cost-model features of a problem and a tiling."""
    o = default_opts()
    o.method = METHODS[method] if isinstance(method, str) else int(method)
    for i, b in enumerate(bins or ()):
        o.bin[i] = int(b)
    o.msub = int(msub)
    o.threads = int(threads)
    arr = (ctypes.c_int64 * 3)(*([int(v) for v in N] + [1] * (3 - len(N))))
    out = (ctypes.c_float * PICKER_NFEAT)()
    _check(load().nufft_picker_features(int(type_), len(N), arr, float(eps), int(prec),
                                        float(upsampfac), int(M), float(skew), ctypes.byref(o),
                                        out), "nufft_picker_features")
    return list(out)


def point_skew(x, y, z=None, stream=None):
    """nufft_point_skew on torch tensors (float32 or float64); synchronizes."""
    import torch
    dim = 2 if z is None else 3
    prec = 0 if x.dtype == torch.float32 else 1
    if stream is None:
        stream = torch.cuda.current_stream()
    s = ctypes.c_double()
    _check(load().nufft_point_skew(dim, prec, int(x.shape[0]), _dptr(x), _dptr(y), _dptr(z),
                                   ctypes.byref(s), ctypes.c_void_p(stream.cuda_stream)),
           "nufft_point_skew")
    return s.value


def pick(type_, N, eps, x, y=None, z=None, stream=None):
    """nufft_pick on torch tensors: the upsampling factor and tiles the installed
    picker predicts fastest for these points, as Plan keyword arguments
    (upsampfac, prec, method, bins, msub, threads); prec is the points' own."""
    import torch
    dim = len(N)
    prec = 0 if x.dtype == torch.float32 else 1
    if stream is None:
        stream = torch.cuda.current_stream()
    o = default_opts()
    arr = (ctypes.c_int64 * 3)(*([int(v) for v in N] + [1] * (3 - dim)))
    _check(load().nufft_pick(int(type_), dim, arr, float(eps), prec, int(x.shape[0]), _dptr(x),
                             _dptr(y), _dptr(z), ctypes.c_void_p(stream.cuda_stream),
                             ctypes.byref(o)), "nufft_pick")
    inv = {v: k for k, v in METHODS.items()}
    return dict(upsampfac=o.upsampfac, prec=prec, method=inv.get(o.method, o.method),
                bins=tuple(o.bin[:dim]) if o.bin[0] > 0 else None, msub=o.msub, threads=o.threads)


class Picker:
    """The learned tile picker (nufft_picker_*): a 12-64-64-1 ReLU perceptron
    predicting log2 of execute milliseconds; tensors are float32 CUDA tensors."""

    def __init__(self, seed=0, params=None, path=None):
        import torch
        self._torch = torch
        h = ctypes.c_void_p()
        _check(load().nufft_picker_create(ctypes.c_uint64(int(seed) & (2 ** 64 - 1)),
                                          ctypes.byref(h)), "nufft_picker_create")
        self.handle = h.value
        if params is not None:
            self.set_params(params)
        if path is not None:
            self.load(path)

    def _st(self, stream):
        s = stream if stream is not None else self._torch.cuda.current_stream()
        return ctypes.c_void_p(s.cuda_stream)

    def set_params(self, params):
        import numpy as np
        a = np.ascontiguousarray(params, dtype=np.float32).reshape(-1)
        if a.size != PICKER_NPARAM:
            raise ValueError("expected %d parameters" % PICKER_NPARAM)
        _check(load().nufft_picker_set_params(ctypes.c_void_p(self.handle),
                                              a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))),
               "nufft_picker_set_params")

    def get_params(self):
        import numpy as np
        a = np.empty(PICKER_NPARAM, dtype=np.float32)
        _check(load().nufft_picker_get_params(ctypes.c_void_p(self.handle),
                                              a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))),
               "nufft_picker_get_params")
        return a

    def save(self, path):
        _check(load().nufft_picker_save(ctypes.c_void_p(self.handle), str(path).encode()),
               "nufft_picker_save")

    def load(self, path):
        _check(load().nufft_picker_load(ctypes.c_void_p(self.handle), str(path).encode()),
               "nufft_picker_load")

    def predict(self, X, stream=None):
        y = self._torch.empty(X.shape[0], dtype=self._torch.float32, device=X.device)
        _check(load().nufft_picker_predict(ctypes.c_void_p(self.handle), int(X.shape[0]),
                                           _dptr(X, self._torch.float32, "X"), _dptr(y),
                                           self._st(stream)), "nufft_picker_predict")
        return y

    def grad(self, X, T, stream=None):
        torch = self._torch
        g = torch.empty(PICKER_NPARAM, dtype=torch.float32, device=X.device)
        L = torch.empty(1, dtype=torch.float32, device=X.device)
        _check(load().nufft_picker_grad(ctypes.c_void_p(self.handle), int(X.shape[0]),
                                        _dptr(X, torch.float32, "X"), _dptr(T, torch.float32, "T"),
                                        _dptr(g), _dptr(L), self._st(stream)), "nufft_picker_grad")
        return g, L

    def step(self, X, T, lr, stream=None):
        torch = self._torch
        L = torch.empty(1, dtype=torch.float32, device=X.device)
        _check(load().nufft_picker_step(ctypes.c_void_p(self.handle), int(X.shape[0]),
                                        _dptr(X, torch.float32, "X"), _dptr(T, torch.float32, "T"),
                                        float(lr), _dptr(L), self._st(stream)), "nufft_picker_step")
        return L

    def train(self, X, T, epochs, batch=256, lr=1e-3, seed=0, stream=None):
        torch = self._torch
        out = ctypes.c_float()
        _check(load().nufft_picker_train(ctypes.c_void_p(self.handle), int(X.shape[0]),
                                         _dptr(X, torch.float32, "X"),
                                         _dptr(T, torch.float32, "T"), int(epochs), int(batch),
                                         float(lr), ctypes.c_uint64(int(seed) & (2 ** 64 - 1)),
                                         ctypes.byref(out), self._st(stream)), "nufft_picker_train")
        return out.value

    def loss(self, X, T, stream=None):
        torch = self._torch
        L = torch.empty(1, dtype=torch.float32, device=X.device)
        _check(load().nufft_picker_loss(ctypes.c_void_p(self.handle), int(X.shape[0]),
                                        _dptr(X, torch.float32, "X"), _dptr(T, torch.float32, "T"),
                                        _dptr(L), self._st(stream)), "nufft_picker_loss")
        return L

    def install(self):
        _check(load().nufft_picker_install(ctypes.c_void_p(self.handle)), "nufft_picker_install")

    @staticmethod
    def uninstall():
        _check(load().nufft_picker_install(None), "nufft_picker_install")

    def close(self):
        if self.handle:
            load().nufft_picker_destroy(ctypes.c_void_p(self.handle))
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def get_launch_count() -> int:
    return int(load().nufft_get_launch_count())


def get_status(h):
    """nufft_get_status: raises NufftError(NUFFT_ERR_CHECK) if a device-side check failed."""
    _check(load().nufft_get_status(h), "nufft_get_status")


def debug_fail(kind, after):
    """nufft_debug_fail: arm (after >= 0) or disarm a host-side injected failure;
    returns the number of allocations / cuFFT plans made since the last call."""
    rc = load().nufft_debug_fail(int(kind), int(after))
    if rc < 0:
        raise NufftError(rc, "nufft_debug_fail")
    return rc


def fma_peak(prec=0, stream=None) -> float:
    """Measured FMA throughput of the current device in TFLOP/s (prec 0 float, 1 double)."""
    v = ctypes.c_double(0.0)
    _check(load().nufft_fma_peak(int(prec), ctypes.byref(v), stream), "nufft_fma_peak")
    return float(v.value)


def interp(h, c):
    _check(load().nufft_interp(ctypes.c_void_p(h), c), "nufft_interp")


def fft(h):
    _check(load().nufft_fft(ctypes.c_void_p(h)), "nufft_fft")


def deconvolve(h, f):
    _check(load().nufft_deconvolve(ctypes.c_void_p(h), f), "nufft_deconvolve")


def precorrect(h, f):
    _check(load().nufft_precorrect(ctypes.c_void_p(h), f), "nufft_precorrect")


def get_params(h):
    w = ctypes.c_int()
    beta = ctypes.c_double()
    nf = (ctypes.c_int64 * 3)()
    bins = (ctypes.c_int * 3)()
    nbins = ctypes.c_int64()
    prec = ctypes.c_int()
    method = ctypes.c_int()
    _check(load().nufft_get_params(ctypes.c_void_p(h), ctypes.byref(w), ctypes.byref(beta), nf,
                                   bins, ctypes.byref(nbins), ctypes.byref(prec),
                                   ctypes.byref(method)), "nufft_get_params")
    return dict(w=w.value, beta=beta.value, nf=tuple(nf), bins=tuple(bins), nbins=nbins.value,
                prec=prec.value, method=method.value)


def get_finegrid(h):
    p = ctypes.c_void_p()
    n = ctypes.c_size_t()
    _check(load().nufft_get_finegrid(ctypes.c_void_p(h), ctypes.byref(p), ctypes.byref(n)),
           "nufft_get_finegrid")
    return p.value, n.value


def get_sort(h, t=None, bincounts=None, nsub=None):
    _check(load().nufft_get_sort(ctypes.c_void_p(h), t, bincounts, nsub), "nufft_get_sort")


# ---------------------------------------------------------------------------
# Convenience object over the handle, on torch tensors.
# ---------------------------------------------------------------------------
class Plan:
    """A plan bound to torch's current CUDA stream (or an explicit one).

    Plan(type, N, eps, iflag=+1, ntransf=1, prec=-1, method="auto", ...)
    N is (N1,), (N1, N2) or (N1, N2, N3).  Arrays: x, y, z real tensors of the plan
    precision; c complex (ntransf, M) / (M,); f complex ([ntransf,] N3, N2, N1).
    """

    def __init__(self, type_, N, eps, iflag=+1, ntransf=1, prec=-1, method="auto",
                 bins=None, msub=0, upsampfac=2.0, stream=None, threads=0, ctas_per_sm=0,
                 use_picker=False, unordered_bins=False, debug_checks=False):
        import torch
        self._torch = torch
        self.type = int(type_)
        self.N = tuple(int(v) for v in N)
        self.dim = len(self.N)
        self.ntransf = int(ntransf)
        o = default_opts()
        o.method = METHODS[method] if isinstance(method, str) else int(method)
        if bins:
            for i, b in enumerate(bins):
                o.bin[i] = int(b)
        o.msub = int(msub)
        o.upsampfac = float(upsampfac)
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        o.stream = ctypes.c_void_p(stream.cuda_stream)
        o.threads = int(threads)
        o.ctas_per_sm = int(ctas_per_sm)
        o.use_picker = 1 if use_picker else 0
        o.unordered_bins = 1 if unordered_bins else 0
        o.debug_checks = 1 if debug_checks else 0
        self.handle = None
        self.handle = makeplan(self.type, self.dim, self.N, iflag, ntransf, eps, prec, o)
        self.params = get_params(self.handle)
        self.real_dtype = torch.float32 if self.params["prec"] == 0 else torch.float64
        self.complex_dtype = torch.complex64 if self.params["prec"] == 0 else torch.complex128
        self.M = 0
        self._pts = None

    def setpts(self, x, y=None, z=None):
        M = x.shape[0]
        rd = self.real_dtype
        setpts(self.handle, M, _dptr(x, rd, "x"), _dptr(y, rd, "y") if self.dim >= 2 else None,
               _dptr(z, rd, "z") if self.dim == 3 else None)
        self.M = M
        self._pts = (x, y, z)   # keep alive until the stream has consumed them

    def execute(self, c=None, f=None):
        """Type 1: c -> new f (or into f).  Type 2: f -> new c (or into c)."""
        torch = self._torch
        cd = self.complex_dtype
        shp_f = tuple(reversed(self.N))
        shp_c = (self.M,)
        if self.ntransf > 1:
            shp_f = (self.ntransf,) + shp_f
            shp_c = (self.ntransf,) + shp_c
        dev = torch.device("cuda", torch.cuda.current_device())
        if self.type == 1:
            if f is None:
                f = torch.empty(shp_f, dtype=cd, device=dev)
            execute(self.handle, _dptr(c, cd, "c"), _dptr(f, cd, "f"))
            return f
        if c is None:
            c = torch.empty(shp_c, dtype=cd, device=dev)
        execute(self.handle, _dptr(c, cd, "c"), _dptr(f, cd, "f"))
        return c

    def execute_host(self, x, y=None, z=None, c=None, f=None, sync=True):
        """nufft_execute_host on host (CPU) tensors: set the points and execute with
        the copies inside the call.  Type 1 reads c and returns f (new, or into f);
        type 2 reads f and returns c.  Pinned tensors let the copies overlap the
        kernels.  With sync=True the plan's stream is synchronised before returning."""
        torch = self._torch
        rd, cd = self.real_dtype, self.complex_dtype
        M = x.shape[0]
        shp_f = tuple(reversed(self.N))
        shp_c = (M,)
        if self.ntransf > 1:
            shp_f = (self.ntransf,) + shp_f
            shp_c = (self.ntransf,) + shp_c
        pin = bool(x.is_pinned())
        if self.type == 1:
            if f is None:
                f = torch.empty(shp_f, dtype=cd, pin_memory=pin)
        elif c is None:
            c = torch.empty(shp_c, dtype=cd, pin_memory=pin)
        args = [_hptr(x, rd, "x"), _hptr(y, rd, "y") if self.dim >= 2 else None,
                _hptr(z, rd, "z") if self.dim == 3 else None,
                _hptr(c, cd, "c"), _hptr(f, cd, "f")]
        _check(load().nufft_execute_host(self.handle, M, *args), "nufft_execute_host")
        self.M = M
        self._pts = (x, y, z, c, f)   # keep alive until the stream has consumed them
        if sync:
            self.stream.synchronize()
        return f if self.type == 1 else c

    def finegrid(self):
        """Copy of the plan's fine grid as a complex tensor ([ntransf,] n3, n2, n1).

        Synchronises the plan's stream first (a test and diagnostics helper).
        """
        torch = self._torch
        ptr, nbytes = get_finegrid(self.handle)
        nf = self.params["nf"][: self.dim]
        shape = tuple(reversed(nf))
        if self.ntransf > 1:
            shape = (self.ntransf,) + shape
        self.stream.synchronize()
        view = _DeviceView(ptr, shape, "<c8" if self.params["prec"] == 0 else "<c16")
        return torch.as_tensor(view, device="cuda").clone()

    def tiles(self):
        return get_tiles(self.handle)

    def sort(self):
        torch = self._torch
        t = torch.empty(max(self.M, 1), dtype=torch.int32, device="cuda")
        bc = torch.empty(self.params["nbins"], dtype=torch.int32, device="cuda")
        ns = torch.empty(1, dtype=torch.int32, device="cuda")
        get_sort(self.handle, _dptr(t), _dptr(bc), _dptr(ns))
        return t[: self.M], bc, int(ns.item())

    def close(self):
        if self.handle:
            destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class _DeviceView:
    """Minimal __cuda_array_interface__ exporter for a library-owned buffer."""

    def __init__(self, ptr, shape, typestr):
        self.__cuda_array_interface__ = {
            "shape": tuple(int(v) for v in shape),
            "typestr": typestr,
            "data": (int(ptr), False),
            "version": 3,
            "strides": None,
        }


class Plan3:
    """Type 3 plan (nonuniform points to nonuniform frequencies):
    f_k = sum_j c_j exp(i iflag s_k . x_j).

    Plan3(dim, eps, iflag=+1, ntransf=1, prec=-1, stream=None); setpts(xs, ss) with
    xs / ss lists of dim real device tensors (M points, K frequencies);
    execute(c) -> f of shape ([ntransf,] K).
    """

    def __init__(self, dim, eps, iflag=+1, ntransf=1, prec=-1, stream=None, debug_checks=False):
        import torch
        self._torch = torch
        self.dim = int(dim)
        self.ntransf = int(ntransf)
        o = default_opts()
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        o.stream = ctypes.c_void_p(stream.cuda_stream)
        o.debug_checks = 1 if debug_checks else 0
        self.handle = None
        self.handle = makeplan(3, self.dim, [1] * self.dim, iflag, ntransf, eps, prec, o)
        self.params = get_params(self.handle)
        self.real_dtype = torch.float32 if self.params["prec"] == 0 else torch.float64
        self.complex_dtype = torch.complex64 if self.params["prec"] == 0 else torch.complex128
        self.M = self.K = 0
        self._keep = None

    def setpts(self, xs, ss):
        rd = self.real_dtype
        if len(xs) != self.dim or len(ss) != self.dim:
            raise ValueError("need %d coordinate arrays for points and for frequencies" % self.dim)
        M, K = xs[0].shape[0], ss[0].shape[0]
        xp = [_dptr(a, rd, "x") for a in xs] + [None] * (3 - self.dim)
        sp = [_dptr(a, rd, "s") for a in ss] + [None] * (3 - self.dim)
        setpts3(self.handle, M, xp[0], xp[1], xp[2], K, sp[0], sp[1], sp[2])
        self.M, self.K = M, K
        self._keep = (xs, ss)
        self.params = get_params(self.handle)   # the spreading grid sizes (nf)

    def execute(self, c, f=None):
        torch = self._torch
        shp = (self.K,) if self.ntransf == 1 else (self.ntransf, self.K)
        if f is None:
            f = torch.empty(shp, dtype=self.complex_dtype, device="cuda")
        cd = self.complex_dtype
        execute(self.handle, _dptr(c, cd, "c"), _dptr(f, cd, "f"))
        return f

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
        return False

    def close(self):
        if self.handle:
            destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
