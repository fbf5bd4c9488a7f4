"""CPU oracle for the NDFT / NFFT / nonlinear CAF (arXiv 1402.0532).

TEST INFRASTRUCTURE ONLY: the test-suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers.  The product path (the
CUDA library and its Python binding) never imports this package.

The arithmetic lives in ``ndft_oracle.c`` (plain C, double precision, the
operator evaluated literally by its sign cases, Eq. 1-2 and Eq. 6).  This
module only compiles it with gcc and marshals numpy arrays through ctypes.

Every function states the passage of the paper it follows:

=====================  ====================================================
``otimes``             Eq. 1-2, real a (x) b = sgn(a b)(|a| + |b|)
``cotimes``            Eq. 6, complex extension
``vecprod``            Eq. 3, <x (.) y> = sum x_i (x) y_i
``twiddle``            W = exp(-j 2 pi / N), defined under Eq. 8
``ndft``               Eq. 8 (Sec. 2), X = F (.) x
``nfft``/``nfft_f32``  Sec. 3, radix-2 DIT (or DIF) with (x) in every butterfly
``dft``                the linear DFT (numpy FFT), for Eq. 12b
``lagprod``            Eq. 12a inner factor s_surv[i] (x) conj(s_ref[i-l])
``caf``                Eq. 12a, the nonlinear ambiguity surface
``caf_nfft``           Eq. 12a with the NFFT over samples (Sec. 5)
``caf_12b``            Eq. 12b, (x) lag product then the linear DFT
``*_q14``              the same in Q1.14 integers, sums modulo 2^32
``caf_adjoint``        derivative of Eq. 1-2 chained through Eq. 6, 12a (s_surv)
``caf_adjoint_ref``    the same with respect to s_ref
=====================  ====================================================
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ndft_oracle.c")
_LIB_PATH = os.path.join(_HERE, "libndft_oracle.so")
_lock = threading.Lock()
_lib = None

F_NO_CONJ_REF = 0x1
F_CIRCULAR_LAG = 0x2


def build(force: bool = False) -> str:
    """Compile ndft_oracle.c with gcc (no fast-math, no FP contraction)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
               "-shared", "-fPIC", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            d, i64, i32, u32 = ctypes.c_double, ctypes.c_int64, ctypes.c_int, ctypes.c_uint32
            P = ctypes.c_void_p
            lib.oracle_otimes.restype = d
            lib.oracle_otimes.argtypes = [d, d]
            lib.oracle_cotimes.argtypes = [P, P, P]
            lib.oracle_vecprod.restype = d
            lib.oracle_vecprod.argtypes = [P, P, i64]
            lib.oracle_twiddle.argtypes = [i64, i64, P]
            lib.oracle_twiddle_q14.argtypes = [i64, i64, P]
            lib.oracle_twiddle_table_f32.argtypes = [i64, P]
            lib.oracle_twiddle_table_q14.argtypes = [i64, P]
            lib.oracle_ndft.argtypes = [P, i64, i64, i64, i64, P]
            lib.oracle_nfft.argtypes = [P, i64, i64, P]
            lib.oracle_nfft_f32.argtypes = [P, i64, i64, P]
            lib.oracle_nfft_dif.argtypes = [P, i64, i64, P]
            lib.oracle_nfft_dif_f32.argtypes = [P, i64, i64, P]
            lib.oracle_nfft_bound.argtypes = [P, i64, i64, i32, P, P, P]
            lib.oracle_lagprod.argtypes = [P, P, i64, i64, u32, P]
            lib.oracle_lagprod_f32.argtypes = [P, P, i64, i64, u32, P]
            lib.oracle_caf.argtypes = [P, P, i64, i64, i64, i64, i64, u32, i32, P]
            lib.oracle_caf_cells.argtypes = [P, P, i64, P, P, i64, u32, i32, P]
            lib.oracle_ndft_q14.argtypes = [P, i64, i64, i64, i64, P, P]
            lib.oracle_caf_q14.argtypes = [P, P, i64, i64, i64, i64, i64, u32, P, P]
            lib.oracle_caf_adjoint.argtypes = [P, P, i64, i64, i64, i64, i64, u32, P, P]
            lib.oracle_caf_adjoint_ref.argtypes = [P, P, i64, i64, i64, i64, i64, u32, P, P]
            lib.oracle_caf_adjoint_at.argtypes = [P, P, i64, i64, i64, i64, i64, u32, P, i32, P, i64, P]
            lib.oracle_num_threads.restype = i32
            for name in ("oracle_ndft", "oracle_nfft", "oracle_nfft_f32", "oracle_nfft_dif",
                         "oracle_nfft_dif_f32", "oracle_nfft_bound", "oracle_lagprod",
                         "oracle_lagprod_f32", "oracle_caf", "oracle_caf_cells", "oracle_ndft_q14",
                         "oracle_caf_q14", "oracle_caf_adjoint", "oracle_caf_adjoint_ref",
                         "oracle_caf_adjoint_at"):
                getattr(lib, name).restype = i32
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _c128(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.complex128)


def _check(rc: int, what: str):
    if rc != 0:
        raise RuntimeError(f"oracle {what} failed with code {rc}")


def num_threads() -> int:
    return int(_load().oracle_num_threads())


# --- Eq. 1-3, Eq. 6 ---------------------------------------------------------
def otimes(a: float, b: float) -> float:
    """Eq. 1-2: a (x) b = sgn(a b)(|a| + |b|), 0 when a or b is 0."""
    return float(_load().oracle_otimes(float(a), float(b)))


def cotimes(a: complex, b: complex) -> complex:
    """Eq. 6: a_r(x)b_r - a_i(x)b_i + j(a_i(x)b_r + b_i(x)a_r)."""
    A = _c128([a])
    B = _c128([b])
    out = np.zeros(1, np.complex128)
    _load().oracle_cotimes(_ptr(A), _ptr(B), _ptr(out))
    return complex(out[0])


def vecprod(x, y) -> float:
    """Eq. 3: <x (.) y> = sum_i x_i (x) y_i."""
    x = np.ascontiguousarray(x, np.float64)
    y = np.ascontiguousarray(y, np.float64)
    assert x.shape == y.shape and x.ndim == 1
    return float(_load().oracle_vecprod(_ptr(x), _ptr(y), x.size))


# --- twiddles ----------------------------------------------------------------
def twiddle(N: int, m: int) -> complex:
    """W^m = exp(-j 2 pi m / N) with exact values on the axes."""
    out = np.zeros(1, np.complex128)
    _load().oracle_twiddle(N, m, _ptr(out))
    return complex(out[0])


def twiddle_q14(N: int, m: int) -> tuple[int, int]:
    out = np.zeros(2, np.int32)
    _load().oracle_twiddle_q14(N, m, _ptr(out))
    return int(out[0]), int(out[1])


def twiddle_table_f32(N: int) -> np.ndarray:
    out = np.zeros(N, np.complex64)
    _load().oracle_twiddle_table_f32(N, _ptr(out))
    return out


def twiddle_table_q14(N: int) -> np.ndarray:
    out = np.zeros((N, 2), np.int16)
    _load().oracle_twiddle_table_q14(N, _ptr(out))
    return out


# --- Eq. 8 / Sec. 3 -------------------------------------------------------------
def ndft(x, p0: int = 0, nbins: int | None = None) -> np.ndarray:
    """Eq. 8: X[b, k] = sum_n W^(((p0+k) n) mod N) (x) x[b, n]; x is [batch, N]."""
    x = _c128(x)
    if x.ndim == 1:
        return ndft(x[None], p0, nbins)[0]
    B, N = x.shape
    nb = N if nbins is None else nbins
    X = np.zeros((B, nb), np.complex128)
    _check(_load().oracle_ndft(_ptr(x), B, N, p0, nb, _ptr(X)), "ndft")
    return X


def nfft(x, dif: bool = False) -> np.ndarray:
    """Sec. 3: the (x)-butterfly radix-2 NFFT in double precision, by
    decimation in time (the recursion Sec. 3 writes out) or, dif=True, by
    decimation in frequency (the other FFT order Sec. 3 names)."""
    x = _c128(x)
    if x.ndim == 1:
        return nfft(x[None], dif)[0]
    B, N = x.shape
    X = np.zeros((B, N), np.complex128)
    fn = _load().oracle_nfft_dif if dif else _load().oracle_nfft
    _check(fn(_ptr(x), B, N, _ptr(X)), "nfft")
    return X


def nfft_f32(x, dif: bool = False) -> np.ndarray:
    """Sec. 3 recursion evaluated in fp32 (one rounding per operation)."""
    x = np.ascontiguousarray(x, np.complex64)
    if x.ndim == 1:
        return nfft_f32(x[None], dif)[0]
    B, N = x.shape
    X = np.zeros((B, N), np.complex64)
    fn = _load().oracle_nfft_dif_f32 if dif else _load().oracle_nfft_f32
    _check(fn(_ptr(x), B, N, _ptr(X)), "nfft_f32")
    return X


def nfft_bound(x, dif: bool = False):
    """Sec. 3 recursion in fp64 with a running error bound for an fp32
    evaluation of the same recursion: returns (X, bound, stable).  X equals
    ``nfft(x, dif)``; bound[b, k] holds the bounds of the Re and Im parts as
    the real and imaginary parts of one complex number; stable[b] is True when
    every data operand of every (x) of vector b keeps its fp64 sign in fp32,
    in which case |Re/Im (X32 - X)| <= Re/Im bound.  x must be representable
    in fp32 (complex64 values)."""
    x = np.ascontiguousarray(x, np.complex64).astype(np.complex128)
    if x.ndim == 1:
        X, b, s = nfft_bound(x[None], dif)
        return X[0], b[0], s[0]
    B, N = x.shape
    X = np.zeros((B, N), np.complex128)
    bound = np.zeros((B, N), np.complex128)
    stable = np.zeros(B, np.int32)
    _check(_load().oracle_nfft_bound(_ptr(x), B, N, 1 if dif else 0, _ptr(X), _ptr(bound), _ptr(stable)),
           "nfft_bound")
    return X, bound, stable.astype(bool)


def within_bound(got, want, bound) -> np.ndarray:
    """Elementwise |Re/Im (got - want)| <= Re/Im bound."""
    d = np.asarray(got, np.complex128) - want
    return (np.abs(d.real) <= bound.real) & (np.abs(d.imag) <= bound.imag)


def dft(x, p0: int = 0, nbins: int | None = None) -> np.ndarray:
    """The ordinary DFT (the linear transform Eq. 8 approximates) at bins
    p0 .. p0 + nbins - 1 mod N, in double precision via numpy's FFT."""
    x = _c128(x)
    N = x.shape[-1]
    nb = N if nbins is None else nbins
    return np.fft.fft(x, axis=-1)[..., (p0 + np.arange(nb)) % N]


# --- Eq. 12a ---------------------------------------------------------------------
def lagprod(s_surv, s_ref, lag: int, flags: int = 0) -> np.ndarray:
    ss, sr = _c128(s_surv), _c128(s_ref)
    z = np.zeros(ss.size, np.complex128)
    _check(_load().oracle_lagprod(_ptr(ss), _ptr(sr), ss.size, lag, flags, _ptr(z)), "lagprod")
    return z


def lagprod_f32(s_surv, s_ref, lag: int, flags: int = 0) -> np.ndarray:
    ss = np.ascontiguousarray(s_surv, np.complex64)
    sr = np.ascontiguousarray(s_ref, np.complex64)
    z = np.zeros(ss.size, np.complex64)
    _check(_load().oracle_lagprod_f32(_ptr(ss), _ptr(sr), ss.size, lag, flags, _ptr(z)), "lagprod_f32")
    return z


def caf(s_surv, s_ref, lag0: int, nlags: int, p0: int, nbins: int, flags: int = 0,
        z32: bool = False) -> np.ndarray:
    """Eq. 12a surface A[l, p], shape [nlags, nbins].  z32: lag product in fp32."""
    ss, sr = _c128(s_surv), _c128(s_ref)
    A = np.zeros((nlags, nbins), np.complex128)
    _check(_load().oracle_caf(_ptr(ss), _ptr(sr), ss.size, lag0, nlags, p0, nbins, flags, int(z32),
                              _ptr(A)), "caf")
    return A


def caf_nfft(s_surv, s_ref, lag0: int, nlags: int, p0: int, nbins: int, flags: int = 0,
             f32: bool = False, dif: bool = False) -> np.ndarray:
    """Eq. 12a with the sum over samples taken by the Sec. 3 NFFT (the form the
    paper simulates in Sec. 5): row a is the NFFT of the lag product for lag
    lag0 + a, read at bins p0 .. p0 + nbins - 1 (mod N).  f32: lag product and
    NFFT in fp32, one rounding per operation; else fp64.  dif: the
    decimation-in-frequency NFFT.  Shape [nlags, nbins]."""
    N = len(s_surv)
    lp = lagprod_f32 if f32 else lagprod
    Z = np.stack([lp(s_surv, s_ref, lag0 + a, flags) for a in range(nlags)])
    X = nfft_f32(Z, dif) if f32 else nfft(Z, dif)
    return X[:, (p0 + np.arange(nbins)) % N]


def caf_12b(s_surv, s_ref, lag0: int, nlags: int, p0: int, nbins: int, flags: int = 0,
            z32: bool = False) -> np.ndarray:
    """Eq. 12b: the lag product formed with (x) (as in Eq. 12a, s_ref
    conjugated), then the ordinary DFT over samples, at bins p0 .. p0 + nbins - 1
    (mod N); double precision (z32: lag product in fp32).  Shape [nlags, nbins]."""
    lp = lagprod_f32 if z32 else lagprod
    Z = np.stack([lp(s_surv, s_ref, lag0 + a, flags).astype(np.complex128) for a in range(nlags)])
    return dft(Z, p0, nbins)


def caf_cells(s_surv, s_ref, lags, bins, flags: int = 0, z32: bool = False) -> np.ndarray:
    """Eq. 12a at the listed (lag, bin) cells only."""
    ss, sr = _c128(s_surv), _c128(s_ref)
    L = np.ascontiguousarray(lags, np.int64)
    P = np.ascontiguousarray(bins, np.int64)
    assert L.shape == P.shape
    A = np.zeros(L.size, np.complex128)
    _check(_load().oracle_caf_cells(_ptr(ss), _ptr(sr), ss.size, _ptr(L), _ptr(P), L.size, flags,
                                    int(z32), _ptr(A)), "caf_cells")
    return A


# --- Q1.14 --------------------------------------------------------------------------
def ndft_q14(x, p0: int = 0, nbins: int | None = None):
    """x: int16 [batch, N, 2] -> (int32 [batch, nbins, 2] modulo 2^32, #cells that wrapped)."""
    x = np.ascontiguousarray(x, np.int16)
    B, N, _ = x.shape
    nb = N if nbins is None else nbins
    X = np.zeros((B, nb, 2), np.int32)
    novf = np.zeros(1, np.int64)
    _check(_load().oracle_ndft_q14(_ptr(x), B, N, p0, nb, _ptr(X), _ptr(novf)), "ndft_q14")
    return X, int(novf[0])


def caf_q14(s_surv, s_ref, lag0: int, nlags: int, p0: int, nbins: int, flags: int = 0):
    """Eq. 12a in Q1.14: int16 [N, 2] inputs -> (int32 [nlags, nbins, 2], #cells that wrapped)."""
    ss = np.ascontiguousarray(s_surv, np.int16)
    sr = np.ascontiguousarray(s_ref, np.int16)
    N = ss.shape[0]
    A = np.zeros((nlags, nbins, 2), np.int32)
    novf = np.zeros(1, np.int64)
    _check(_load().oracle_caf_q14(_ptr(ss), _ptr(sr), N, lag0, nlags, p0, nbins, flags, _ptr(A),
                                  _ptr(novf)), "caf_q14")
    return A, int(novf[0])


# --- adjoint -------------------------------------------------------------------------
def caf_adjoint(s_surv, s_ref, lag0: int, nlags: int, p0: int, nbins: int, dA, flags: int = 0):
    """dL/ds_surv (as dRe + j dIm) given dA = dL/dRe A + j dL/dIm A, shape [nlags, nbins]."""
    ss, sr = _c128(s_surv), _c128(s_ref)
    g = _c128(dA)
    assert g.shape == (nlags, nbins)
    ds = np.zeros(ss.size, np.complex128)
    _check(_load().oracle_caf_adjoint(_ptr(ss), _ptr(sr), ss.size, lag0, nlags, p0, nbins, flags,
                                      _ptr(g), _ptr(ds)), "caf_adjoint")
    return ds


def caf_adjoint_ref(s_surv, s_ref, lag0: int, nlags: int, p0: int, nbins: int, dA, flags: int = 0):
    """dL/ds_ref (as dRe + j dIm) given dA = dL/dRe A + j dL/dIm A, shape [nlags, nbins]:
    the chain rule of Eq. 1-2 with d(a (x) b)/db = sgn(a), through Eq. 6 and Eq. 12a."""
    ss, sr = _c128(s_surv), _c128(s_ref)
    g = _c128(dA)
    assert g.shape == (nlags, nbins)
    ds = np.zeros(sr.size, np.complex128)
    _check(_load().oracle_caf_adjoint_ref(_ptr(ss), _ptr(sr), ss.size, lag0, nlags, p0, nbins, flags,
                                          _ptr(g), _ptr(ds)), "caf_adjoint_ref")
    return ds


def caf_adjoint_at(s_surv, s_ref, lag0: int, nlags: int, p0: int, nbins: int, dA, which: str, idx,
                   flags: int = 0):
    """caf_adjoint (which="surv") or caf_adjoint_ref (which="ref") at the listed indices only."""
    ss, sr = _c128(s_surv), _c128(s_ref)
    g = _c128(dA)
    assert g.shape == (nlags, nbins)
    ix = np.ascontiguousarray(idx, dtype=np.int64)
    out = np.zeros(ix.size, np.complex128)
    _check(_load().oracle_caf_adjoint_at(_ptr(ss), _ptr(sr), ss.size, lag0, nlags, p0, nbins, flags, _ptr(g),
                                         {"surv": 0, "ref": 1}[which], _ptr(ix), ix.size, _ptr(out)),
           "caf_adjoint_at")
    return out


def masked_abs_loss_grad(A: np.ndarray, mask: np.ndarray):
    """L = sum over the mask of |A|; returns (L, dL/dRe A + j dL/dIm A) = (L, A/|A| on the mask)."""
    A = _c128(A)
    mag = np.abs(A)
    L = float(np.sum(mag[mask]))
    g = np.zeros_like(A)
    nz = mask & (mag > 0)
    g[nz] = A[nz] / mag[nz]
    return L, g
