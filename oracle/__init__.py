"""FP64 CPU oracle for per-pixel sparse recovery of a compressed hyperspectral cube.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The GPU library never imports it and shares no code with it.

The arithmetic lives in ``cs_oracle.c`` (plain C, double precision, one pixel
at a time, following Algorithms 1-5 of the paper step by step).  This module
only compiles that file, marshals numpy arrays through ctypes and adds the two
evaluation metrics of Section III (PSNR and relative L2).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cs_oracle.c")
_LIB = os.path.join(_HERE, "libcs_oracle.so")
_lock = threading.Lock()
_lib = None

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int32)


def build(force: bool = False) -> str:
    """Compile cs_oracle.c into an in-tree shared library (gcc, -O2, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def use_library(path: str | None):
    """Point the wrapper at another build of cs_oracle.c (None restores the default).

    Used only by the test that plants mistakes in copies of the oracle and checks
    that the pins catch them."""
    global _lib
    with _lock:
        _lib = None
    if path is not None:
        _configure(ctypes.CDLL(path))


def _load():
    with _lock:
        lib = _lib
    return lib if lib is not None else _configure(ctypes.CDLL(build()))


def _configure(lib):
    global _lib
    with _lock:
        i32, i64, dbl = ctypes.c_int, ctypes.c_int64, ctypes.c_double
        lib.or_dct2_psi.argtypes = [i32, _dp]
        lib.or_dictionary.argtypes = [i32, i32, _dp, _dp, _dp]
        lib.or_measure.argtypes = [i32, i32, _dp, i64, _dp, _dp, _dp]
        lib.or_lipschitz.argtypes = [i32, i32, _dp]
        lib.or_lipschitz.restype = dbl
        lib.or_support_lstsq.argtypes = [i32, i32, _dp, _ip, i32, _dp, _dp]
        lib.or_argmax_k.argtypes = [i32, _dp, i32, _ip]
        lib.or_argmax_k.restype = dbl
        lib.or_fista.argtypes = [i32, i32, _dp, i64, _dp, _dp, dbl, dbl, dbl, i32, _ip, i32]
        lib.or_admm.argtypes = [i32, i32, _dp, i64, _dp, _dp, dbl, dbl, dbl, i32, _ip, i32]
        lib.or_gomp.argtypes = [i32, i32, _dp, i64, _dp, _dp, i32, i32, dbl, i32, _ip, _dp,
                                i32]
        lib.or_biht.argtypes = [i32, i32, _dp, i64, _dp, _dp, i32, dbl, dbl, i32, _ip, _dp,
                                i32]
        lib.or_cosamp.argtypes = [i32, i32, _dp, i64, _dp, _dp, i32, dbl, i32, _ip, _dp, i32]
        lib.or_sparsify.argtypes = [i32, _dp, i64, _dp, dbl, i32, _dp, _ip]
        lib.or_dft_psi.argtypes = [i32, _dp]
        lib.or_partial_fourier.argtypes = [i32, i32, _ip, _dp]
        lib.or_cfista.argtypes = [i32, i32, _dp, i64, _dp, _dp, dbl, dbl, dbl, i32, _ip, i32]
        lib.or_cgomp.argtypes = [i32, i32, _dp, i64, _dp, _dp, i32, i32, dbl, i32, _ip, i32]
        lib.or_ccosamp.argtypes = [i32, i32, _dp, i64, _dp, _dp, i32, dbl, i32, _ip, i32]
        lib.or_cadmm.argtypes = [i32, i32, _dp, i64, _dp, _dp, dbl, dbl, dbl, i32, _ip, i32]
        lib.or_cbiht.argtypes = [i32, i32, _dp, i64, _dp, _dp, i32, dbl, dbl, i32, _ip, i32]
        lib.or_max_threads.restype = i32
        _lib = lib
    return _lib


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(_dp)


def _iptr(a):
    return None if a is None else a.ctypes.data_as(_ip)


def max_threads() -> int:
    return int(_load().or_max_threads())


# --------------------------------------------------------------------------
# Eq. 1: transform, dictionary, measurement, Lipschitz constant
# --------------------------------------------------------------------------
def dct2_psi(N: int) -> np.ndarray:
    """Orthonormal DCT-II synthesis matrix Psi (N x N); column k is atom k."""
    out = np.empty((N, N))
    _load().or_dct2_psi(N, _ptr(out))
    return out


def dictionary(Phi: np.ndarray, Psi: np.ndarray | None = None) -> np.ndarray:
    """A = Phi Psi (Eq. 1).  Psi defaults to the orthonormal DCT-II."""
    Phi = _f64(Phi)
    M, N = Phi.shape
    Psi = dct2_psi(N) if Psi is None else _f64(Psi)
    A = np.empty((M, N))
    _load().or_dictionary(M, N, _ptr(Phi), _ptr(Psi), _ptr(A))
    return A


def measure(A: np.ndarray, X: np.ndarray, E: np.ndarray | None = None) -> np.ndarray:
    """Y[p] = A X[p] (+ E[p]) for every pixel (Eq. 1)."""
    A, X = _f64(A), _f64(X)
    M, N = A.shape
    P = X.shape[0]
    Y = np.empty((P, M))
    Eh = None if E is None else _f64(E)
    _load().or_measure(M, N, _ptr(A), P, _ptr(X), None if Eh is None else _ptr(Eh), _ptr(Y))
    return Y


def lipschitz(A: np.ndarray) -> float:
    """L = lambda_max(A^T A) (Section II-A), by Jacobi eigen-iteration on A A^T."""
    A = _f64(A)
    return float(_load().or_lipschitz(A.shape[0], A.shape[1], _ptr(A)))


def support_lstsq(A: np.ndarray, c, y: np.ndarray) -> np.ndarray:
    """s = A(:, c)^+ y, the minimum-norm least-squares solution."""
    A, y = _f64(A), _f64(y)
    c = np.ascontiguousarray(c, dtype=np.int32)
    s = np.zeros(len(c))
    rc = _load().or_support_lstsq(A.shape[0], A.shape[1], _ptr(A), _iptr(c), len(c), _ptr(y),
                                  _ptr(s))
    if rc:
        raise ValueError(f"or_support_lstsq failed ({rc})")
    return s


def argmax_k(v: np.ndarray, k: int):
    """argmax_k(|v|): the k indices of largest magnitude, ties to the lower index.

    Returns (indices, relative gap between the k-th and (k+1)-th magnitude)."""
    v = _f64(v)
    out = np.zeros(k, dtype=np.int32)
    gap = _load().or_argmax_k(len(v), _ptr(v), k, _iptr(out))
    return out, float(gap)


# --------------------------------------------------------------------------
# Algorithms 1-5
# --------------------------------------------------------------------------
def _prep(A, Y):
    A, Y = _f64(A), _f64(Y)
    M, N = A.shape
    if Y.ndim != 2 or Y.shape[1] != M:
        raise ValueError("Y must be P x M")
    return A, Y, M, N, Y.shape[0]


def fista(A, Y, L, lam, eps=0.0, max_iters=500, threads=0):
    """Algorithm 1.  Returns (X [P x N], iterations [P])."""
    A, Y, M, N, P = _prep(A, Y)
    X = np.zeros((P, N))
    it = np.zeros(P, dtype=np.int32)
    rc = _load().or_fista(M, N, _ptr(A), P, _ptr(Y), _ptr(X), float(L), float(lam), float(eps),
                          int(max_iters), _iptr(it), int(threads))
    if rc:
        raise ValueError(f"or_fista failed ({rc})")
    return X, it


def admm(A, Y, rho, lam, eps=0.0, max_iters=500, threads=0):
    """Algorithm 2 (soft threshold lambda/rho).  Returns (X, iterations)."""
    A, Y, M, N, P = _prep(A, Y)
    X = np.zeros((P, N))
    it = np.zeros(P, dtype=np.int32)
    rc = _load().or_admm(M, N, _ptr(A), P, _ptr(Y), _ptr(X), float(rho), float(lam), float(eps),
                         int(max_iters), _iptr(it), int(threads))
    if rc:
        raise ValueError(f"or_admm failed ({rc})")
    return X, it


def gomp(A, Y, kappa, G, eps=1e-8, max_iters=1 << 30, threads=0):
    """Algorithm 3.  Returns (X, iterations, selection margin per pixel)."""
    A, Y, M, N, P = _prep(A, Y)
    X = np.zeros((P, N))
    it = np.zeros(P, dtype=np.int32)
    mg = np.zeros(P)
    rc = _load().or_gomp(M, N, _ptr(A), P, _ptr(Y), _ptr(X), int(kappa), int(G), float(eps),
                         int(min(max_iters, 2**31 - 1)), _iptr(it), _ptr(mg), int(threads))
    if rc:
        raise ValueError(f"or_gomp failed ({rc})")
    return X, it, mg


def biht(A, Y, kappa, mu=0.1, eps=1e-8, max_iters=100, threads=0):
    """Algorithm 4.  Returns (X, iterations, selection margin per pixel)."""
    A, Y, M, N, P = _prep(A, Y)
    X = np.zeros((P, N))
    it = np.zeros(P, dtype=np.int32)
    mg = np.zeros(P)
    rc = _load().or_biht(M, N, _ptr(A), P, _ptr(Y), _ptr(X), int(kappa), float(mu), float(eps),
                         int(max_iters), _iptr(it), _ptr(mg), int(threads))
    if rc:
        raise ValueError(f"or_biht failed ({rc})")
    return X, it, mg


def cosamp(A, Y, kappa, eps=1e-8, max_iters=100, threads=0):
    """Algorithm 5.  Returns (X, iterations, selection margin per pixel)."""
    A, Y, M, N, P = _prep(A, Y)
    X = np.zeros((P, N))
    it = np.zeros(P, dtype=np.int32)
    mg = np.zeros(P)
    rc = _load().or_cosamp(M, N, _ptr(A), P, _ptr(Y), _ptr(X), int(kappa), float(eps),
                           int(max_iters), _iptr(it), _ptr(mg), int(threads))
    if rc:
        raise ValueError(f"or_cosamp failed ({rc})")
    return X, it, mg


# --------------------------------------------------------------------------
# Section II: sparsification pre-processing
# --------------------------------------------------------------------------
def sparsify(F, T, ddof=1, Psi=None):
    """Sparsification of Section II on every pixel (row) of F (P x N spectra).

    x = Psi^T f; x_i is zeroed where |x_i| - mean|x| < T std|x| (std normalised by
    N - ddof).  Psi defaults to the orthonormal DCT-II.  Returns (X, kappa), kappa the
    number of nonzero kept coefficients per pixel."""
    F = _f64(F)
    P, N = F.shape
    Psi = dct2_psi(N) if Psi is None else _f64(Psi)
    X = np.zeros((P, N))
    kappa = np.zeros(P, dtype=np.int32)
    rc = _load().or_sparsify(N, _ptr(Psi), P, _ptr(F), float(T), int(ddof), _ptr(X),
                             _iptr(kappa))
    if rc:
        raise ValueError(f"or_sparsify failed ({rc})")
    return X, kappa


# --------------------------------------------------------------------------
# Section II with the paper's complex transform: unitary DFT Psi, Phi keeping M rows
# (partial Fourier).  Complex arrays are numpy complex128 (interleaved doubles).
# --------------------------------------------------------------------------
def _c128(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.complex128)


def dft_psi(N: int) -> np.ndarray:
    """Unitary DFT synthesis matrix: Psi[n][k] = exp(-2 pi i n k / N) / sqrt(N)."""
    out = np.empty((N, N), dtype=np.complex128)
    _load().or_dft_psi(N, _ptr(out))
    return out


def partial_fourier(M: int, N: int, rows) -> np.ndarray:
    """A = Phi Psi with Phi keeping the spectral samples `rows` (M distinct indices)."""
    rows = np.ascontiguousarray(rows, dtype=np.int32)
    A = np.empty((M, N), dtype=np.complex128)
    rc = _load().or_partial_fourier(M, N, _iptr(rows), _ptr(A))
    if rc:
        raise ValueError(f"or_partial_fourier failed ({rc})")
    return A


def _cprep(A, Y):
    A, Y = _c128(A), _c128(np.atleast_2d(Y))
    return A, Y, A.shape[0], A.shape[1], Y.shape[0]


def cfista(A, Y, L, lam, eps=0.0, max_iters=500, threads=0):
    """Algorithm 1 on complex data (modulus soft threshold).  Returns (X, iterations)."""
    A, Y, M, N, P = _cprep(A, Y)
    X = np.zeros((P, N), dtype=np.complex128)
    it = np.zeros(P, dtype=np.int32)
    rc = _load().or_cfista(M, N, _ptr(A), P, _ptr(Y), _ptr(X), float(L), float(lam), float(eps),
                           int(max_iters), _iptr(it), int(threads))
    if rc:
        raise ValueError(f"or_cfista failed ({rc})")
    return X, it


def cadmm(A, Y, rho, lam, eps=0.0, max_iters=500, threads=0):
    """Algorithm 2 on complex data (threshold lambda / rho).  Returns (X, iterations)."""
    A, Y, M, N, P = _cprep(A, Y)
    X = np.zeros((P, N), dtype=np.complex128)
    it = np.zeros(P, dtype=np.int32)
    rc = _load().or_cadmm(M, N, _ptr(A), P, _ptr(Y), _ptr(X), float(rho), float(lam), float(eps),
                          int(max_iters), _iptr(it), int(threads))
    if rc:
        raise ValueError(f"or_cadmm failed ({rc})")
    return X, it


def cbiht(A, Y, kappa, mu=0.1, eps=1e-8, max_iters=100, threads=0):
    """Algorithm 4 on complex data.  Returns (X, iterations)."""
    A, Y, M, N, P = _cprep(A, Y)
    X = np.zeros((P, N), dtype=np.complex128)
    it = np.zeros(P, dtype=np.int32)
    rc = _load().or_cbiht(M, N, _ptr(A), P, _ptr(Y), _ptr(X), int(kappa), float(mu), float(eps),
                          int(max_iters), _iptr(it), int(threads))
    if rc:
        raise ValueError(f"or_cbiht failed ({rc})")
    return X, it


def cgomp(A, Y, kappa, G, eps=1e-8, max_iters=1 << 30, threads=0):
    """Algorithm 3 on complex data.  Returns (X, iterations)."""
    A, Y, M, N, P = _cprep(A, Y)
    X = np.zeros((P, N), dtype=np.complex128)
    it = np.zeros(P, dtype=np.int32)
    rc = _load().or_cgomp(M, N, _ptr(A), P, _ptr(Y), _ptr(X), int(kappa), int(G), float(eps),
                          int(max_iters), _iptr(it), int(threads))
    if rc:
        raise ValueError(f"or_cgomp failed ({rc})")
    return X, it


def ccosamp(A, Y, kappa, eps=1e-8, max_iters=100, threads=0):
    """Algorithm 5 on complex data.  Returns (X, iterations)."""
    A, Y, M, N, P = _cprep(A, Y)
    X = np.zeros((P, N), dtype=np.complex128)
    it = np.zeros(P, dtype=np.int32)
    rc = _load().or_ccosamp(M, N, _ptr(A), P, _ptr(Y), _ptr(X), int(kappa), float(eps),
                            int(max_iters), _iptr(it), int(threads))
    if rc:
        raise ValueError(f"or_ccosamp failed ({rc})")
    return X, it


# --------------------------------------------------------------------------
# Section III metrics
# --------------------------------------------------------------------------
def rel_l2(X, X_ref) -> float:
    """||X - X_ref||_F / ||X_ref||_F over the whole cube."""
    X, X_ref = _f64(X), _f64(X_ref)
    den = np.linalg.norm(X_ref)
    return float(np.linalg.norm(X - X_ref) / (den if den > 0 else 1.0))


def psnr(X, X_ref, Psi=None) -> float:
    """PSNR = 10 log10(peak^2 / MSE) in the band domain f = Psi x, peak = max |f_ref|.

    The paper uses PSNR between recovered and reference cubes (Section III) without
    printing its formula; this is the usual definition with the reference's peak."""
    X, X_ref = _f64(X), _f64(X_ref)
    N = X.shape[1]
    Psi = dct2_psi(N) if Psi is None else _f64(Psi)
    F, F_ref = X @ Psi.T, X_ref @ Psi.T
    mse = float(np.mean((F - F_ref) ** 2))
    peak = float(np.max(np.abs(F_ref)))
    if mse == 0.0:
        return float("inf")
    return 10.0 * np.log10(peak * peak / mse)
