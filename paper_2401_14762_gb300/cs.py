"""ctypes binding of libcs_hsi.so with the C ABI's call names (include/cs_hsi.h).

Argument marshalling only: arrays are torch tensors (CUDA or CPU) or numpy arrays,
passed to the library as raw pointers; every step of the recovery runs in the
library's CUDA kernels.  There is no CPU fallback: if the library is not built, or
there is no GB300, the calls raise.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libcs_hsi.so")

CS_OK, CS_ERR_ARG, CS_ERR_SHAPE, CS_ERR_CUDA, CS_ERR_OOM = 0, 1, 2, 3, 4
CS_ERR_NOT_SPD, CS_ERR_TIMEOUT, CS_ERR_NONFINITE, CS_ERR_NO_DEVICE = 5, 6, 7, 8
CS_FP32, CS_BF16, CS_FP8_E4M3 = 0, 1, 2

EXPORTED = ["cs_opts_default", "cs_create", "cs_destroy", "cs_get_lipschitz", "cs_get_dictionary",
            "cs_measure", "cs_recover_fista", "cs_recover_admm", "cs_recover_gomp",
            "cs_recover_biht", "cs_recover_cosamp", "cs_get_work", "cs_get_last_precision",
            "cs_autotune", "cs_set_tuning",
            "cs_recover_gomp_noalloc",
            "cs_recover_batch", "cs_recover_stream", "cs_sparsify", "cs_create_complex",
            "cs_sync", "cs_last_error"]
CS_ALGO_FISTA, CS_ALGO_ADMM, CS_ALGO_GOMP, CS_ALGO_BIHT, CS_ALGO_COSAMP = 0, 1, 2, 3, 4


class CsError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"cs status {status}: {msg}")
        self.status = status


class cs_batch_item(ctypes.Structure):
    _fields_ = [("ctx", ctypes.c_void_p), ("Y", ctypes.c_void_p), ("X", ctypes.c_void_p),
                ("P", ctypes.c_int64), ("kappa_per_pixel", ctypes.c_void_p),
                ("iters_out", ctypes.c_void_p), ("converged_out", ctypes.c_void_p)]


class cs_algo_params(ctypes.Structure):
    _fields_ = [("lambda_", ctypes.c_double), ("rho", ctypes.c_double), ("iters", ctypes.c_int),
                ("kappa", ctypes.c_int), ("G", ctypes.c_int)]


class cs_tuning(ctypes.Structure):
    _fields_ = [("factor_rows", ctypes.c_int), ("warps_per_cta", ctypes.c_int),
                ("ms", ctypes.c_double), ("ms_default", ctypes.c_double),
                ("tuned", ctypes.c_int)]


class cs_opts(ctypes.Structure):
    _fields_ = [("eps", ctypes.c_double), ("max_iters", ctypes.c_int), ("prec", ctypes.c_int),
                ("mu", ctypes.c_double), ("iters_out", ctypes.c_void_p),
                ("converged_out", ctypes.c_void_p), ("kappa_per_pixel", ctypes.c_void_p),
                ("cycle_skip", ctypes.c_int)]


_lib = None


def load_library(path: str = LIB_PATH):
    """Loads libcs_hsi.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with "
                           "`python -m paper_2401_14762_gb300.build` (needs nvcc)")
    lib = ctypes.CDLL(path)
    vp, i32, i64, dbl = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
    op = ctypes.POINTER(cs_opts)
    lib.cs_opts_default.argtypes = [op]
    lib.cs_opts_default.restype = None
    lib.cs_create.argtypes = [ctypes.POINTER(vp), i32, i32, vp, vp, vp, dbl, vp]
    lib.cs_destroy.argtypes = [vp]
    lib.cs_create_complex.argtypes = [ctypes.POINTER(vp), i32, i32, vp, dbl, vp]
    lib.cs_destroy.restype = None
    lib.cs_get_lipschitz.argtypes = [vp, ctypes.POINTER(dbl)]
    lib.cs_get_dictionary.argtypes = [vp, vp]
    lib.cs_measure.argtypes = [vp, vp, vp, vp, i64]
    lib.cs_recover_fista.argtypes = [vp, vp, vp, i64, dbl, i32, op]
    lib.cs_recover_admm.argtypes = [vp, vp, vp, i64, dbl, dbl, i32, op]
    lib.cs_recover_gomp.argtypes = [vp, vp, vp, i64, i32, i32, op]
    lib.cs_recover_biht.argtypes = [vp, vp, vp, i64, i32, op]
    lib.cs_recover_cosamp.argtypes = [vp, vp, vp, i64, i32, op]
    lib.cs_get_work.argtypes = [vp, ctypes.POINTER(dbl)]
    lib.cs_get_last_precision.argtypes = [vp, ctypes.POINTER(i32)]
    lib.cs_autotune.argtypes = [vp, i32, ctypes.POINTER(cs_algo_params), vp, i64,
                                ctypes.POINTER(cs_opts), ctypes.POINTER(cs_tuning)]
    lib.cs_set_tuning.argtypes = [vp, i32, ctypes.POINTER(cs_algo_params),
                                  ctypes.POINTER(cs_tuning)]
    lib.cs_recover_gomp_noalloc.argtypes = [vp, i32, i32, vp, vp, i64, i32, i32, op, vp]
    lib.cs_recover_batch.argtypes = [ctypes.POINTER(cs_batch_item), i32, i32,
                                     ctypes.POINTER(cs_algo_params), op]
    lib.cs_sparsify.argtypes = [vp, vp, vp, i64, dbl, i32, vp, vp]
    lib.cs_recover_stream.argtypes = [vp, i32, ctypes.POINTER(cs_algo_params), vp, vp, i64,
                                      i64, op]
    lib.cs_sync.argtypes = [vp]
    lib.cs_last_error.argtypes = []
    lib.cs_last_error.restype = ctypes.c_char_p
    for name in EXPORTED:
        if name not in ("cs_opts_default", "cs_destroy", "cs_last_error"):
            getattr(lib, name).restype = i32
    _lib = lib
    return lib


def _check(status: int):
    if status != CS_OK:
        raise CsError(status, load_library().cs_last_error().decode())


def _ptr(a, dtype=None):
    """Raw pointer of a contiguous torch tensor or numpy array (None -> NULL)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if dtype is not None and a.dtype != dtype:
            raise TypeError(f"expected {dtype}, got {a.dtype}")
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data
    import torch
    if isinstance(a, torch.Tensor):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        if dtype is not None and a.dtype != {np.float32: torch.float32, np.float64: torch.float64,
                                            np.int32: torch.int32, np.uint8: torch.uint8,
                                            np.int16: torch.int16, np.int64: torch.int64}[dtype]:
            raise TypeError(f"expected {dtype}, got {a.dtype}")
        return a.data_ptr()
    raise TypeError(f"unsupported array type {type(a)}")


def _default_stream():
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
    except Exception:
        pass
    return None


class Context:
    """Owns a cs_ctx handle (released by cs_destroy / close())."""

    def __init__(self, handle, M, N):
        self.handle, self.M, self.N = handle, M, N

    def close(self):
        if self.handle:
            load_library().cs_destroy(self.handle)
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


def cs_opts_default() -> cs_opts:
    o = cs_opts()
    load_library().cs_opts_default(ctypes.byref(o))
    return o


def make_opts(eps=1e-8, max_iters=100, prec=CS_FP32, mu=0.1, iters_out=None,
              converged_out=None, kappa_per_pixel=None, cycle_skip=True) -> cs_opts:
    o = cs_opts_default()
    o.eps, o.max_iters, o.prec, o.mu = float(eps), int(max_iters), int(prec), float(mu)
    o.cycle_skip = 1 if cycle_skip else 0
    o.iters_out = _ptr(iters_out, np.int32)
    o.converged_out = _ptr(converged_out, np.uint8)
    o.kappa_per_pixel = _ptr(kappa_per_pixel, np.int16)
    return o


def cs_create(M, N, A=None, Phi=None, Psi=None, admm_rho=0.0, stream=None) -> Context:
    """Builds the FP64 dictionary A = Phi Psi (or takes A), its Gram matrix, the Lipschitz
    constant and optionally the ADMM factor on the device (Eq. 1, Section II-A)."""
    lib = load_library()
    keep = []

    def host64(a):
        if a is None:
            return None
        a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
        keep.append(a)
        return a.ctypes.data

    h = ctypes.c_void_p()
    st = lib.cs_create(ctypes.byref(h), int(M), int(N), host64(A), host64(Phi), host64(Psi),
                       float(admm_rho), stream if stream is not None else _default_stream())
    _check(st)
    return Context(h.value, int(M), int(N))


def cs_create_complex(M, N, A, admm_rho=0.0, stream=None) -> Context:
    """Context for the complex M x N dictionary A (the paper's DFT / partial-Fourier
    setup, Section II).  Y and X on it are complex64 arrays (P x M, P x N) passed as
    float32 (re, im) pairs; FISTA and ADMM threshold the moduli."""
    lib = load_library()
    A = np.ascontiguousarray(np.asarray(A, dtype=np.complex128))
    h = ctypes.c_void_p()
    st = lib.cs_create_complex(ctypes.byref(h), int(M), int(N), A.ctypes.data, float(admm_rho),
                               stream if stream is not None else _default_stream())
    _check(st)
    return Context(h.value, 2 * int(M), 2 * int(N))


def cs_destroy(ctx: Context):
    ctx.close()


def cs_get_lipschitz(ctx: Context) -> float:
    L = ctypes.c_double()
    _check(load_library().cs_get_lipschitz(ctx.handle, ctypes.byref(L)))
    return L.value


def cs_get_dictionary(ctx: Context) -> np.ndarray:
    A = np.empty((ctx.M, ctx.N))
    _check(load_library().cs_get_dictionary(ctx.handle, A.ctypes.data))
    return A


def _rows(a):
    return int(a.shape[0])


def cs_measure(ctx: Context, X, Y, E=None, P=None):
    """Y = X A^T (+ E) (Eq. 1)."""
    P = _rows(X) if P is None else P
    _check(load_library().cs_measure(ctx.handle, _ptr(X, np.float32), _ptr(Y, np.float32),
                                     _ptr(E, np.float32), int(P)))
    return Y


def cs_sparsify(ctx: Context, F, X, T, ddof=1, kappa_out=None, recomputed_out=None, P=None):
    """Sparsification of Section II: X = Psi^T F per pixel with x_i zeroed where
    |x_i| - mean|x| < T std|x|.  F, X (P x N float32), kappa_out (P int16) and
    recomputed_out (1 int64: pixels decided in FP64) are device tensors."""
    P = _rows(F) if P is None else P
    _check(load_library().cs_sparsify(ctx.handle, _ptr(F, np.float32), _ptr(X, np.float32),
                                      int(P), float(T), int(ddof), _ptr(kappa_out, np.int16),
                                      _ptr(recomputed_out, np.int64)))
    return X


def cs_recover_fista(ctx: Context, Y, X, lam, iters, opts: cs_opts | None = None, P=None):
    P = _rows(Y) if P is None else P
    _check(load_library().cs_recover_fista(ctx.handle, _ptr(Y, np.float32), _ptr(X, np.float32),
                                           int(P), float(lam), int(iters),
                                           ctypes.byref(opts) if opts else None))
    return X


def cs_recover_admm(ctx: Context, Y, X, rho, lam, iters, opts: cs_opts | None = None, P=None):
    P = _rows(Y) if P is None else P
    _check(load_library().cs_recover_admm(ctx.handle, _ptr(Y, np.float32), _ptr(X, np.float32),
                                          int(P), float(rho), float(lam), int(iters),
                                          ctypes.byref(opts) if opts else None))
    return X


def cs_recover_gomp(ctx: Context, Y, X, kappa, G, opts: cs_opts | None = None, P=None):
    P = _rows(Y) if P is None else P
    _check(load_library().cs_recover_gomp(ctx.handle, _ptr(Y, np.float32), _ptr(X, np.float32),
                                          int(P), int(kappa), int(G),
                                          ctypes.byref(opts) if opts else None))
    return X


def cs_recover_batch(items, algo, lam=0.0, rho=1.0, iters=0, kappa=0, G=0,
                     opts: cs_opts | None = None):
    """Recovers several cubes with one algorithm (one launch for the greedy methods).
    items: sequence of dicts with keys ctx, Y, X and optionally kappa_per_pixel, iters_out,
    converged_out (device tensors).  Runs on items[0]'s context stream."""
    arr = (cs_batch_item * len(items))()
    for i, it in enumerate(items):
        arr[i].ctx = it["ctx"].handle
        arr[i].Y = _ptr(it["Y"], np.float32)
        arr[i].X = _ptr(it["X"], np.float32)
        arr[i].P = int(it.get("P", _rows(it["Y"])))
        arr[i].kappa_per_pixel = _ptr(it.get("kappa_per_pixel"), np.int16)
        arr[i].iters_out = _ptr(it.get("iters_out"), np.int32)
        arr[i].converged_out = _ptr(it.get("converged_out"), np.uint8)
    prm = cs_algo_params(float(lam), float(rho), int(iters), int(kappa), int(G))
    _check(load_library().cs_recover_batch(arr, len(items), int(algo), ctypes.byref(prm),
                                           ctypes.byref(opts) if opts else None))


def cs_recover_stream(ctx: Context, algo, Y, X, chunk_pixels, lam=0.0, rho=1.0, iters=0,
                      kappa=0, G=0, opts: cs_opts | None = None, P=None):
    """Pushbroom recovery of a cube in host memory (numpy arrays or CPU tensors, pinned for
    overlap), chunk_pixels pixels at a time, double-buffered through the device."""
    P = _rows(Y) if P is None else P
    prm = cs_algo_params(float(lam), float(rho), int(iters), int(kappa), int(G))
    _check(load_library().cs_recover_stream(ctx.handle, int(algo), ctypes.byref(prm),
                                            _ptr(Y, np.float32), _ptr(X, np.float32), int(P),
                                            int(chunk_pixels),
                                            ctypes.byref(opts) if opts else None))
    return X


def cs_recover_biht(ctx: Context, Y, X, kappa, opts: cs_opts | None = None, P=None):
    P = _rows(Y) if P is None else P
    _check(load_library().cs_recover_biht(ctx.handle, _ptr(Y, np.float32), _ptr(X, np.float32),
                                          int(P), int(kappa),
                                          ctypes.byref(opts) if opts else None))
    return X


def cs_recover_cosamp(ctx: Context, Y, X, kappa, opts: cs_opts | None = None, P=None):
    P = _rows(Y) if P is None else P
    _check(load_library().cs_recover_cosamp(ctx.handle, _ptr(Y, np.float32), _ptr(X, np.float32),
                                            int(P), int(kappa),
                                            ctypes.byref(opts) if opts else None))
    return X


def cs_autotune(ctx: Context, algo: int, Y, kappa: int, G: int = 0,
                opts: cs_opts | None = None, cache: str | None = None, P=None) -> dict:
    """Chooses the greedy kernel's launch configuration for (algo, kappa, G) on this
    context by timing the candidates on the sample Y (device, P x M); later calls with
    the same parameters use it.  With `cache` (a JSON file path) a configuration chosen
    before for the same device, algorithm, M x N, kappa and G is installed instead of
    measured, and a new choice is added to the file."""
    import json
    lib = load_library()
    prm = cs_algo_params(0.0, 0.0, 0, int(kappa), int(G))
    key = None
    if cache:
        try:
            import torch
            dev = torch.cuda.get_device_name()
        except Exception:
            dev = "cuda"
        key = f"{dev}|algo{algo}|{ctx.M}x{ctx.N}|kappa{kappa}|G{G}"
        try:
            with open(cache) as f:
                rec = json.load(f).get(key)
        except (OSError, ValueError):
            rec = None
        if rec:
            t = cs_tuning(rec["factor_rows"], rec["warps_per_cta"], rec["ms"],
                          rec["ms_default"], rec["tuned"])
            _check(lib.cs_set_tuning(ctx.handle, int(algo), ctypes.byref(prm), ctypes.byref(t)))
            return dict(rec, cached=True)
    n = int(P if P is not None else Y.shape[0])
    t = cs_tuning()
    o = opts if opts is not None else cs_opts_default()
    _check(lib.cs_autotune(ctx.handle, int(algo), ctypes.byref(prm), _ptr(Y, np.float32), n,
                           ctypes.byref(o), ctypes.byref(t)))
    rec = {"factor_rows": t.factor_rows, "warps_per_cta": t.warps_per_cta, "ms": t.ms,
           "ms_default": t.ms_default, "tuned": t.tuned, "sample_pixels": n}
    if cache:
        try:
            with open(cache) as f:
                allrec = json.load(f)
        except (OSError, ValueError):
            allrec = {}
        allrec[key] = rec
        with open(cache, "w") as f:
            json.dump(allrec, f, indent=1, sort_keys=True)
    return dict(rec, cached=False)


def cs_get_last_precision(ctx: Context) -> str:
    """The arithmetic of the last recovery call's products: "bf16" (split-BF16 tensor
    cores) or "fp32"."""
    v = ctypes.c_int32(0)
    _check(load_library().cs_get_last_precision(ctx.handle, ctypes.byref(v)))
    return {CS_FP32: "fp32", CS_BF16: "bf16"}.get(v.value, str(v.value))


def cs_get_work(ctx: Context) -> float:
    """Algorithmic flops of the last greedy call on this context."""
    f = ctypes.c_double()
    _check(load_library().cs_get_work(ctx.handle, ctypes.byref(f)))
    return f.value


def cs_recover_gomp_noalloc(A_dev, M, N, Y, X, kappa, G, opts: cs_opts | None = None, P=None,
                            stream=None):
    """gOMP without a context or any device allocation (for callers that cannot allocate);
    A_dev, Y and X are device arrays the caller owns."""
    P = _rows(Y) if P is None else P
    _check(load_library().cs_recover_gomp_noalloc(
        _ptr(A_dev, np.float64), int(M), int(N), _ptr(Y, np.float32), _ptr(X, np.float32),
        int(P), int(kappa), int(G), ctypes.byref(opts) if opts else None,
        stream if stream is not None else _default_stream()))
    return X


def cs_sync(ctx: Context):
    _check(load_library().cs_sync(ctx.handle))


def cs_last_error() -> str:
    return load_library().cs_last_error().decode()
