"""Pure-Python literal evaluation of the paper's definitions for tiny inputs.

Written independently of ``oracle/ndft_oracle.c`` so the two can pin each
other: plain Python floats / ints, one scalar at a time, no numpy arithmetic.

* real (x): Eq. 1-2          * complex (x): Eq. 6
* NDFT: Eq. 8                * NFFT: Sec. 3 (recursive DIT, (x) at every twiddle)
* CAF: Eq. 12a with s_ref conjugated and zero outside [0, N)
"""
from __future__ import annotations

import math


def sgn(v):
    return 1 if v > 0 else (-1 if v < 0 else 0)


def ox(a, b):
    """Eq. 1-2 (works for floats and for Python ints)."""
    s = sgn(a) * sgn(b)
    if s == 0:
        return 0 if isinstance(a, int) and isinstance(b, int) else 0.0
    return s * (abs(a) + abs(b))


def cox(a, b):
    """Eq. 6 on (re, im) tuples."""
    ar, ai = a
    br, bi = b
    return (ox(ar, br) - ox(ai, bi), ox(ai, br) + ox(bi, ar))


def twiddle(N, m):
    """exp(-j 2 pi m / N), quadrant reduced in integers so the axis values are exact."""
    m %= N
    q, r = divmod(4 * m, N)
    a = (math.pi / 2) * (r / N)
    c, s = math.cos(a), math.sin(a)
    ct, st = [(c, s), (-s, c), (-c, -s), (s, -c)][q]
    return (ct + 0.0, -st + 0.0)


def ndft(x, p0=0, nbins=None):
    N = len(x)
    nb = N if nbins is None else nbins
    out = []
    for k in range(nb):
        p = (p0 + k) % N
        re = im = 0.0
        for n in range(N):
            cr, ci = cox(twiddle(N, p * n), x[n])
            re += cr
            im += ci
        out.append((re, im))
    return out


def nfft(x):
    N = len(x)
    if N == 1:
        return [x[0]]
    E = nfft(x[0::2])
    O = nfft(x[1::2])
    h = N // 2
    out = [None] * N
    for k in range(h):
        tr, ti = cox(twiddle(N, k), O[k])
        out[k] = (E[k][0] + tr, E[k][1] + ti)
        out[k + h] = (E[k][0] - tr, E[k][1] - ti)
    return out


def nfft_dif(x):
    N = len(x)
    if N == 1:
        return [x[0]]
    h = N // 2
    Y = [(x[m][0] + x[m + h][0], x[m][1] + x[m + h][1]) for m in range(h)]
    Z = [cox(twiddle(N, m), (x[m][0] - x[m + h][0], x[m][1] - x[m + h][1])) for m in range(h)]
    YY, ZZ = nfft_dif(Y), nfft_dif(Z)
    out = [None] * N
    for k in range(h):
        out[2 * k] = YY[k]
        out[2 * k + 1] = ZZ[k]
    return out


def dft(x):
    import cmath
    N = len(x)
    return [sum(complex(*x[n]) * cmath.exp(-2j * cmath.pi * k * n / N) for n in range(N)) for k in range(N)]


def lagprod(s_surv, s_ref, lag):
    N = len(s_surv)
    z = []
    for i in range(N):
        j = i - lag
        c = (s_ref[j][0], -s_ref[j][1]) if 0 <= j < N else (0.0, 0.0)
        z.append(cox(s_surv[i], c))
    return z


def caf(s_surv, s_ref, lag0, nlags, p0, nbins):
    N = len(s_surv)
    A = []
    for a in range(nlags):
        z = lagprod(s_surv, s_ref, lag0 + a)
        row = []
        for k in range(nbins):
            p = (p0 + k) % N
            re = im = 0.0
            for i in range(N):
                cr, ci = cox(z[i], twiddle(N, i * p))
                re += cr
                im += ci
            row.append((re, im))
        A.append(row)
    return A


def as_pairs(arr):
    return [(float(v.real), float(v.imag)) for v in arr]
