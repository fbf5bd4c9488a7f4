"""Pins for the CPU oracle: values and properties fixed by the paper or by the
mathematics, none of them obtained by re-running the oracle's own formulas.

Each test names the passage it pins.  A plausible slip in the oracle (a
dropped term of Eq. 6, a wrong sign, a transposed twiddle index, a missing
conjugate, a wrong recursion split) fails at least one of them.
"""
import json
import math
import os

import numpy as np
import pytest

import literal
from paper_1402_0532_gb300 import scenes

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _hand():
    with open(os.path.join(GOLDEN, "hand_cases.json")) as f:
        return json.load(f)


def _c(pairs):
    return np.array([complex(a, b) for a, b in pairs])


def _tw(N):
    """Twiddle matrix built independently with numpy's fft of unit impulses:
    column n of the DFT matrix is fft(e_n); axis values are snapped exactly."""
    F = np.fft.fft(np.eye(N), axis=0)  # F[k, n] = exp(-j 2 pi k n / N)
    k = np.arange(N)[:, None]
    n = np.arange(N)[None, :]
    m = (k * n) % N
    re = np.where((4 * m == N) | (4 * m == 3 * N), 0.0, F.real)
    im = np.where((m == 0) | (2 * m == N), 0.0, F.imag)
    return re + 1j * im


def _sig(v):
    return np.sign(v.real) + 1j * np.sign(v.imag)


# --------------------------------------------------------------------------
# Eq. 1-2: the sign cases, including zeros and negative zero.
# --------------------------------------------------------------------------
@pytest.mark.parametrize("a,b,want", [
    (2.0, 3.0, 5.0), (-2.0, 3.0, -5.0), (2.0, -3.0, -5.0), (-2.0, -3.0, 5.0),
    (0.0, 3.0, 0.0), (3.0, 0.0, 0.0), (0.0, 0.0, 0.0), (-0.0, 3.0, 0.0), (3.0, -0.0, 0.0),
    (-0.0, -7.5, 0.0), (1.5, -0.25, -1.75), (-1e-300, 1e300, -1e300),
])
def test_sign_cases_eq2(oracle, a, b, want):
    got = oracle.otimes(a, b)
    assert got == want
    if want == 0.0:
        assert math.copysign(1.0, got) == 1.0, "the 'otherwise' case returns +0"
    assert oracle.otimes(b, a) == got  # commutative
    assert literal.ox(a, b) == want


def test_real_identity_bit_exact(oracle):
    """a (x) b = sgn(b) a + sgn(a) b exactly (both addends are exact in IEEE)."""
    rng = np.random.default_rng(10)
    v = rng.standard_normal(4000) * 10.0 ** rng.integers(-3, 4, 4000)
    v[::17] = 0.0
    for a, b in zip(v[:2000], v[2000:]):
        want = np.sign(b) * a + np.sign(a) * b
        assert oracle.otimes(a, b) == want


# --------------------------------------------------------------------------
# Eq. 3 and Eq. 5: <x (.) x> = 2 ||x||_1.
# --------------------------------------------------------------------------
def test_l1_norm_eq5(oracle):
    rng = np.random.default_rng(11)
    x = rng.integers(-50, 51, 1000).astype(np.float64)  # integer-valued: sums exact
    assert oracle.vecprod(x, x) == 2.0 * np.abs(x).sum()
    y = rng.standard_normal(100000)
    l1 = math.fsum(np.abs(y))
    assert abs(oracle.vecprod(y, y) - 2.0 * l1) <= 1e-12 * l1


def test_vecprod_eq3_small(oracle):
    x = np.array([1.0, -2.0, 0.0, 3.0])
    y = np.array([4.0, 5.0, -6.0, -0.5])
    # 1(x)4 = 5, -2(x)5 = -7, 0(x)-6 = 0, 3(x)-0.5 = -3.5
    assert oracle.vecprod(x, y) == 5.0 - 7.0 + 0.0 - 3.5


# --------------------------------------------------------------------------
# Eq. 6: the complex operator.
# --------------------------------------------------------------------------
def test_complex_operator_eq6_terms(oracle):
    # a = 1+2j, b = 3-4j: 1(x)3 - 2(x)(-4) + j(2(x)3 + (-4)(x)1) = 4 + 6 + j(5 - 5)
    assert oracle.cotimes(1 + 2j, 3 - 4j) == complex(10.0, 0.0)
    # a = -1+0.5j, b = 2+2j: (-1)(x)2 - 0.5(x)2 + j(0.5(x)2 + 2(x)(-1)) = -3 - 2.5 + j(2.5 - 3)
    assert oracle.cotimes(-1 + 0.5j, 2 + 2j) == complex(-5.5, -0.5)
    assert oracle.cotimes(0j, 2 + 2j) == 0j


def test_complex_identity_and_symmetries(oracle):
    rng = np.random.default_rng(12)
    a = rng.standard_normal(500) + 1j * rng.standard_normal(500)
    b = rng.standard_normal(500) + 1j * rng.standard_normal(500)
    a[::7] = a[::7].real  # exact zero imaginary parts
    b[::11] = 1j * b[::11].imag
    for u, v in zip(a, b):
        got = oracle.cotimes(u, v)
        want = _sig(u) * v + u * _sig(v)  # sigma(a) b + a sigma(b)
        assert abs(got - want) <= 4e-16 * (abs(u) + abs(v)) * 4
        assert oracle.cotimes(v, u) == got  # commutative
        assert oracle.cotimes(-u, v) == -got  # odd
        assert oracle.cotimes(np.conj(u), np.conj(v)) == np.conj(got)
        # a (x) conj(a) = 2(|a_r| + |a_i|) + 0j exactly (complex analogue of Eq. 5)
        assert oracle.cotimes(u, np.conj(u)) == complex(2 * (abs(u.real) + abs(u.imag)), 0.0)
        assert oracle.cotimes(u, v) == complex(*literal.cox((u.real, u.imag), (v.real, v.imag)))


# --------------------------------------------------------------------------
# Twiddles: W^m with exact axis values.
# --------------------------------------------------------------------------
@pytest.mark.parametrize("N", [1, 2, 3, 4, 6, 7, 8, 12, 64, 1000, 1024, 65536])
def test_twiddles(oracle, N):
    ms = np.unique(np.concatenate([np.arange(min(N, 64)), np.arange(N - min(N, 64), N),
                                   np.array([N // 4, N // 2, 3 * N // 4]) % N]))
    for m in ms:
        w = oracle.twiddle(N, int(m))
        ang = -2.0 * np.pi * m / N
        assert abs(w - complex(np.cos(ang), np.sin(ang))) < 1e-15 * max(1, m)
        if (4 * m) % N == 0:
            # on an axis: both components in {0, +-1}, exactly, zeros positive
            assert w.real in (0.0, 1.0, -1.0) and w.imag in (0.0, 1.0, -1.0)
            for v in (w.real, w.imag):
                assert v != 0 or math.copysign(1.0, v) == 1.0
        assert w == complex(*literal.twiddle(N, int(m)))
        if N % 2 == 0:
            assert oracle.twiddle(N, int(m) + N // 2) == -w or w == 0
    assert oracle.twiddle(4, 1) == complex(0.0, -1.0)
    assert oracle.twiddle(8, 2) == complex(0.0, -1.0)


def test_twiddle_q14(oracle):
    assert oracle.twiddle_q14(4, 0) == (16384, 0)
    assert oracle.twiddle_q14(4, 1) == (0, -16384)
    assert oracle.twiddle_q14(8, 1) == (11585, -11585)  # round(2^14 / sqrt 2) = 11585
    assert oracle.twiddle_q14(6, 1) == (8192, -14189)   # 2^14 (1/2, -sqrt(3)/2)


# --------------------------------------------------------------------------
# Eq. 8: NDFT worked examples, closed forms and invariants.
# --------------------------------------------------------------------------
def test_hand_cases_ndft_nfft(oracle):
    h = _hand()
    for case in h["cases"]:
        x = _c(case["x"])
        nd = oracle.ndft(x)
        nf = oracle.nfft(x)
        np.testing.assert_array_equal(nd, _c(case["ndft"]))
        np.testing.assert_array_equal(nf, _c(case["nfft"]))
        np.testing.assert_array_equal(oracle.nfft_f32(x.astype(np.complex64)), _c(case["nfft"]))
        assert not np.array_equal(nd, nf)  # Sec. 3: NFFT != NDFT
    d = h["ndft_of_delta"]
    x = np.zeros(d["N"], complex)
    x[0] = 1
    np.testing.assert_array_equal(oracle.ndft(x), np.full(d["N"], complex(*d["value"])))
    d = h["nfft_of_delta"]
    np.testing.assert_array_equal(oracle.nfft(x), np.full(d["N"], complex(*d["value"])))


def test_tone_peak_fig1_eq9(oracle):
    """Eq. 9 / Fig. 1: N = 64, k0 = 7, the NDFT of exp(j 2 pi 7 n / 64) peaks at k = 7.
    At the peak every term is conj(x) (x) x = 2(|cos| + |sin|), so
    X[7] = 4 sum_m |cos(2 pi m / 64)| = 8 cot(pi / 64)."""
    x = scenes.exact_tone(64, 7)
    X = oracle.ndft(x)
    mag = np.abs(X)
    assert int(np.argmax(mag)) == 7
    assert abs(X[7].real - 8.0 / math.tan(math.pi / 64)) < 1e-12 * 163
    assert abs(X[7].imag) < 1e-12
    assert abs(X[7].real - 162.8437409998975) < 1e-9
    others = np.delete(mag, 7)
    assert others.max() < 0.2 * mag[7]  # "slightly scattered" but clearly peaked


@pytest.mark.parametrize("N,k0", [(8, 3), (12, 5), (16, 1), (32, 9), (128, 45), (1024, 333)])
def test_tone_closed_form_and_eq9(oracle, N, k0):
    X = oracle.ndft(scenes.exact_tone(N, k0))
    assert abs(X[k0] - 8.0 / math.tan(math.pi / N)) < 1e-11 * N
    assert np.all(np.abs(X) <= np.abs(X[k0]) + 1e-9)  # Eq. 9


def test_identity_decomposition(oracle):
    """X = S x + F sigma(x), S = sigma(F): F sigma(x) is a plain DFT of a ternary
    sequence (numpy FFT); S x is a dense product with the sign matrix."""
    rng = np.random.default_rng(13)
    for N in (3, 5, 8, 12, 16, 48):
        x = scenes.cn(rng, (4, N))
        x[:, ::5] = x[:, ::5].real  # some exact zeros in the imaginary part
        F = _tw(N)
        S = _sig(F)
        want = x @ S.T + np.fft.fft(_sig(x), axis=1)
        got = oracle.ndft(x)
        np.testing.assert_allclose(got, want, rtol=0, atol=1e-12 * N)


def test_conjugate_pairing_identity(oracle):
    """Bins +c and -c from one pair of real contractions (Eq. 8 with
    W^(-ci) = conj W^(ci) and the odd sign cases of Eq. 2): with F = W^(ci),
    U = sgn(Re F) v + Re F sigma(v) and V = sgn(Im F) v + Im F sigma(v)
    (real matrices times the complex v), X[+c] = U + jV and X[-c] = U - jV;
    the tensor-core form computes exactly these four real products."""
    rng = np.random.default_rng(16)
    for N in (7, 16, 45, 64):
        v = scenes.cn(rng, (3, N))
        v[:, ::4] = v[:, ::4].real  # exact zeros in the imaginary part
        F = _tw(N)
        sv = _sig(v)
        X = oracle.ndft(v)
        for c in range(1, N // 2 + 1):
            Fr, Fi = F[c].real, F[c].imag
            U = v @ np.sign(Fr) + sv @ Fr
            V = v @ np.sign(Fi) + sv @ Fi
            np.testing.assert_allclose(X[:, c], U + 1j * V, rtol=0, atol=1e-11 * N)
            np.testing.assert_allclose(X[:, (N - c) % N], U - 1j * V, rtol=0, atol=1e-11 * N)


def test_ndft_invariants(oracle):
    rng = np.random.default_rng(14)
    N = 40
    x = scenes.cn(rng, (3, N))
    X = oracle.ndft(x)
    S = _sig(_tw(N))
    # (ii) scaling by c > 0 changes only the S x part
    c = 3.5
    np.testing.assert_allclose(oracle.ndft(c * x) - X, (c - 1) * x @ S.T, atol=1e-11)
    # (iii) odd
    np.testing.assert_array_equal(oracle.ndft(-x), -X)
    # (iv) conjugation flips the bin
    Xc = oracle.ndft(np.conj(x))
    np.testing.assert_allclose(Xc, np.conj(X[:, (-np.arange(N)) % N]), atol=1e-12)
    # (v) bin 0: W^0 = 1, so each term is (x_r + sgn x_r) + j (x_i + sgn x_i)
    want0 = (x.real + np.sign(x.real)).sum(1) + 1j * (x.imag + np.sign(x.imag)).sum(1)
    np.testing.assert_allclose(X[:, 0], want0, atol=1e-12)
    # bins p0..p0+nbins-1 with a negative start are the same columns
    np.testing.assert_array_equal(oracle.ndft(x, p0=-5, nbins=11), X[:, (np.arange(-5, 6)) % N])


def test_ndft_brute_force_literal(oracle):
    rng = np.random.default_rng(15)
    for N in (1, 2, 3, 4, 5, 7, 8, 16):
        x = scenes.cn(rng, (N,))
        if N > 2:
            x[1] = 0.0
            x[2] = 1j * x[2].imag
        got = oracle.ndft(x)
        want = _c(literal.ndft(literal.as_pairs(x)))
        np.testing.assert_allclose(got, want, rtol=0, atol=1e-13)


# --------------------------------------------------------------------------
# Sec. 3: the NFFT.
# --------------------------------------------------------------------------
def test_nfft_brute_force_literal(oracle):
    rng = np.random.default_rng(16)
    for N in (1, 2, 4, 8, 16):
        x = scenes.cn(rng, (N,))
        got = oracle.nfft(x)
        want = _c(literal.nfft(literal.as_pairs(x)))
        np.testing.assert_allclose(got, want, rtol=0, atol=1e-13)


def test_nfft_sparse_input_structure(oracle):
    """Sec. 3 recursion on an input that is nonzero only at n = 0 and n = N/2:
    every odd half is all-zero, W (x) 0 = 0 (Eq. 2), so each stage copies E and
    the output is the 2-point NFFT of (x[0], x[N/2]) repeated."""
    N = 16
    x = np.zeros(N, complex)
    x[0] = 2 + 1j
    x[N // 2] = -1 + 3j
    X = oracle.nfft(x)
    # 2-point NFFT of (x0, x_{N/2}) at the first stage, then copied by zero odd halves
    t = oracle.cotimes(1 + 0j, x[N // 2])
    want = np.array([x[0] + t if k % 2 == 0 else x[0] - t for k in range(N)])
    np.testing.assert_array_equal(X, want)


def test_nfft_tone_fig2(oracle):
    """Fig. 2: the NFFT of the N = 64, k0 = 7 tone also peaks at k = 7."""
    X = oracle.nfft(scenes.exact_tone(64, 7))
    assert int(np.argmax(np.abs(X))) == 7
    assert not np.allclose(X, oracle.ndft(scenes.exact_tone(64, 7)))


def test_nfft_f32_matches_f64_when_exact(oracle):
    rng = np.random.default_rng(17)
    for N in (2, 4):
        x = (rng.integers(-20, 21, N) + 1j * rng.integers(-20, 21, N)).astype(np.complex64)
        np.testing.assert_array_equal(oracle.nfft_f32(x), oracle.nfft(x.astype(complex)))
    x = scenes.cn(rng, (8, 256)).astype(np.complex64)
    a = oracle.nfft_f32(x)
    b = oracle.nfft(x.astype(complex))
    assert np.max(np.abs(a - b)) < 1e-4 * np.max(np.abs(b))


# --------------------------------------------------------------------------
# Eq. 12a: lag product and CAF.
# --------------------------------------------------------------------------
def test_lagprod_and_caf_literal(oracle):
    rng = np.random.default_rng(18)
    N = 12
    ss = scenes.cn(rng, (N,))
    sr = scenes.cn(rng, (N,))
    ss[3] = 0
    for lag in (-2, 0, 1, 5, 11, 13):
        np.testing.assert_allclose(oracle.lagprod(ss, sr, lag), _c(literal.lagprod(
            literal.as_pairs(ss), literal.as_pairs(sr), lag)), atol=1e-14)
    A = oracle.caf(ss, sr, -1, 5, -4, 9)
    L = _c([v for row in literal.caf(literal.as_pairs(ss), literal.as_pairs(sr), -1, 5, -4, 9)
            for v in row]).reshape(5, 9)
    np.testing.assert_allclose(A, L, atol=1e-12)
    # the CAF row of lag l is the NDFT of the lag product (left-associative reading)
    for a in range(5):
        np.testing.assert_array_equal(A[a], oracle.ndft(oracle.lagprod(ss, sr, a - 1), p0=-4, nbins=9))
    cells = oracle.caf_cells(ss, sr, [0, 2, 3], [3, -4, 4])
    np.testing.assert_array_equal(cells, [A[1, 7], A[3, 0], A[4, 8]])


def test_caf_autoambiguity_invariant(oracle):
    """s_surv = s_ref with no zero components: z_0 = s (x) conj(s) = 2(|s_r| + |s_i|)
    and A[0, 0] = sum (z_0 (x) 1) = 2 ||s||_1 + N."""
    rng = np.random.default_rng(19)
    N = 300
    s = scenes.cn(rng, (N,))
    A = oracle.caf(s, s, 0, 3, 0, 2)
    l1 = np.sum(np.abs(s.real) + np.abs(s.imag))
    assert abs(A[0, 0] - (2 * l1 + N)) < 1e-10 * N


def test_caf_boundary_zero_and_conjugate(oracle):
    """Lags beyond the signal give z = 0 and A = 0 exactly; with the conjugate the
    zero-lag auto-ambiguity is real at bin 0, without it (ablation flag) it is not."""
    rng = np.random.default_rng(20)
    N = 32
    s = scenes.cn(rng, (N,))
    A = oracle.caf(s, s, N, 2, 0, 4)
    assert np.all(A == 0)
    A0 = oracle.caf(s, s, 0, 1, 0, 1)[0, 0]
    assert A0.imag == 0.0
    Anc = oracle.caf(s, s, 0, 1, 0, 1, flags=oracle.F_NO_CONJ_REF)[0, 0]
    assert Anc.imag != 0.0
    # circular lag: lag N is lag 0
    np.testing.assert_array_equal(oracle.caf(s, s, N, 1, 0, 4, flags=oracle.F_CIRCULAR_LAG),
                                  oracle.caf(s, s, 0, 1, 0, 4))


def test_caf_nfft_literal_and_structure(oracle):
    """Eq. 12a through the Sec. 3 NFFT: each row is the literal recursion applied
    to the literal lag product, read at bins p0 .. p0 + nbins - 1 mod N; with
    s_ref = delta at 0 the zero-lag product is the single impulse
    s_surv[0] (x) 1 at n = 0, whose NFFT is that value at every bin (each odd
    half is zero, W (x) 0 = 0); lags beyond the signal give 0."""
    rng = np.random.default_rng(22)
    for N in (1, 2, 8, 16):
        ss = scenes.cn(rng, (N,))
        sr = scenes.cn(rng, (N,))
        if N > 2:
            ss[2] = 0
        for lag0, nlags, p0, nb in ((0, 3, 0, N), (-2, 4, -N // 2, max(1, N // 2)), (1, 2, 3, 1)):
            got = oracle.caf_nfft(ss, sr, lag0, nlags, p0, nb)
            for a in range(nlags):
                z = literal.lagprod(literal.as_pairs(ss), literal.as_pairs(sr), lag0 + a)
                row = _c(literal.nfft(z))
                want = row[(p0 + np.arange(nb)) % N]
                np.testing.assert_allclose(got[a], want, rtol=0, atol=1e-12)
    N = 64
    ss = scenes.cn(rng, (N,))
    delta = np.zeros(N, complex)
    delta[0] = 1.0
    A = oracle.caf_nfft(ss, delta, 0, 1, 0, N)
    v = complex(np.sign(ss[0].real) * (abs(ss[0].real) + 1), np.sign(ss[0].imag) * (abs(ss[0].imag) + 1))
    np.testing.assert_array_equal(A[0], np.full(N, v))
    assert np.all(oracle.caf_nfft(ss, ss, N, 2, 0, 8) == 0)
    # bin 0 meets only W^0 = 1 at every stage: with small-integer inputs every
    # intermediate is an exact integer, so the fp32 evaluation equals the fp64 one
    si = (rng.integers(-8, 9, 16) + 1j * rng.integers(-8, 9, 16)).astype(np.complex64)
    sr = si[::-1].copy()
    np.testing.assert_array_equal(oracle.caf_nfft(si, sr, -3, 6, 0, 1, f32=True),
                                  oracle.caf_nfft(si, sr, -3, 6, 0, 1).astype(np.complex64))


def test_nfft_dif_literal_and_impulse(oracle):
    """Decimation in frequency (the other FFT order Sec. 3 names): against the
    literal recursion for N <= 16; for an impulse v at n = 0 every difference
    is v or 0 and W (x) 0 = 0, so bin k is f applied popcount(k) times to v,
    f(u) = 1 (x) u (Eq. 6 with W^0 = 1); and DIF differs from DIT."""
    rng = np.random.default_rng(23)
    for N in (1, 2, 4, 8, 16):
        x = scenes.cn(rng, (N,))
        if N > 2:
            x[1] = 0
        got = oracle.nfft(x, dif=True)
        want = _c(literal.nfft_dif(literal.as_pairs(x)))
        np.testing.assert_allclose(got, want, rtol=0, atol=1e-13)
    N = 32
    v = complex(-1.25, 0.5)
    x = np.zeros(N, complex)
    x[0] = v
    X = oracle.nfft(x, dif=True)

    def f(u):
        return complex(np.sign(u.real) * (abs(u.real) + 1), np.sign(u.imag) * (abs(u.imag) + 1))
    for k in range(N):
        u = v
        for _ in range(bin(k).count("1")):
            u = f(u)
        assert X[k] == u
    y = scenes.cn(rng, (64,))
    assert not np.allclose(oracle.nfft(y, dif=True), oracle.nfft(y))
    # fp32 evaluation equals fp64 when every intermediate is an exact small integer
    # (N = 2: the only twiddle is W^0 = 1)
    xi = (rng.integers(-9, 10, (5, 2)) + 1j * rng.integers(-9, 10, (5, 2))).astype(np.complex64)
    np.testing.assert_array_equal(oracle.nfft_f32(xi, dif=True), oracle.nfft(xi, dif=True).astype(np.complex64))


def test_nfft_f32_both_orders_exact_at_n4(oracle):
    """N = 4: the twiddles are W^0 = 1 and W^1 = -j, so with small-integer data
    every intermediate of either order is an exact small integer and the fp32
    evaluation must equal the fp64 one bit for bit.  This reaches the DIF
    difference branch through a non-trivial twiddle and the even/odd output
    interleave, which N = 2 cannot."""
    rng = np.random.default_rng(29)
    x = (rng.integers(-20, 21, (64, 4)) + 1j * rng.integers(-20, 21, (64, 4))).astype(np.complex64)
    x[0] = 0
    x[1, 1::2] = 0
    for dif in (False, True):
        np.testing.assert_array_equal(oracle.nfft_f32(x, dif=dif),
                                      oracle.nfft(x.astype(complex), dif=dif).astype(np.complex64))
    # the two orders are different transforms already at N = 4
    assert not np.array_equal(oracle.nfft(x[2:], dif=True), oracle.nfft(x[2:]))


@pytest.mark.parametrize("N", [8, 256, 1024])
@pytest.mark.parametrize("dif", [False, True])
def test_nfft_f32_within_running_error_bound(oracle, N, dif):
    """The fp32 recursion (either order) against the fp64 one, which the
    literal recursion pins for N <= 16.  (x) jumps at zero, so fp32 can only
    track fp64 while every data operand keeps its sign; the oracle's running
    error analysis marks those vectors (stable) and bounds |X32 - X64| per
    component.  A wrong twiddle index, a swapped difference or a wrong output
    interleave in either recursion moves bins by O(1) and fails the bound."""
    rng = np.random.default_rng(31 + N)
    x = scenes.cn(rng, (200, N)).astype(np.complex64)
    X, bound, stable = oracle.nfft_bound(x, dif=dif)
    np.testing.assert_array_equal(X, oracle.nfft(x.astype(complex), dif=dif))  # same fp64 values
    assert stable.mean() >= 0.9
    X32 = oracle.nfft_f32(x, dif=dif)
    assert oracle.within_bound(X32[stable], X[stable], bound[stable]).all()
    rel = np.abs(X32 - X).max(axis=1) / np.abs(X).max(axis=1)
    assert rel[stable].max() < 1e-5
    # the bound is tight enough to mean something: well under 1e-3 of max|X|
    assert np.median(np.maximum(bound.real, bound.imag).max(axis=1) / np.abs(X).max(axis=1)) < 1e-4


def test_caf_12b_literal_and_parseval(oracle):
    """Eq. 12b: the literal DFT sum of the literal (x) lag product; Parseval
    (sum_p |A[l,p]|^2 = N sum_i |z_l[i]|^2 over all N bins) on a larger case; and
    with s_ref = delta at 0 the zero-lag product is one impulse at n = 0, whose
    DFT is flat."""
    rng = np.random.default_rng(24)
    N = 12
    ss = scenes.cn(rng, (N,))
    sr = scenes.cn(rng, (N,))
    got = oracle.caf_12b(ss, sr, -2, 5, -3, 7)
    for a in range(5):
        z = literal.lagprod(literal.as_pairs(ss), literal.as_pairs(sr), a - 2)
        row = np.array(literal.dft(z))
        np.testing.assert_allclose(got[a], row[(-3 + np.arange(7)) % N], rtol=0, atol=1e-12)
    N = 256
    ss = scenes.cn(rng, (N,))
    sr = scenes.cn(rng, (N,))
    A = oracle.caf_12b(ss, sr, 0, 4, 0, N)
    for a in range(4):
        z = oracle.lagprod(ss, sr, a)
        assert abs(np.sum(np.abs(A[a]) ** 2) - N * np.sum(np.abs(z) ** 2)) < 1e-9 * N * np.sum(np.abs(z) ** 2)
    delta = np.zeros(N, complex)
    delta[0] = 1
    A0 = oracle.caf_12b(ss, delta, 0, 1, 0, N)[0]
    v = oracle.cotimes(ss[0], 1 + 0j)
    np.testing.assert_allclose(A0, np.full(N, v), rtol=0, atol=1e-12)


def test_caf_z32_gate(oracle):
    """Forming the lag product in fp32 changes A by no more than fp32 rounding."""
    sc = scenes.radar_scene(N=2048, nlags=8, nbins=16, seed=21)
    a = oracle.caf(sc.s_surv, sc.s_ref, 0, 8, -8, 16)
    b = oracle.caf(sc.s_surv, sc.s_ref, 0, 8, -8, 16, z32=True)
    assert np.max(np.abs(a - b)) < 1e-4 * np.max(np.abs(a))


# --------------------------------------------------------------------------
# Q1.14 integers.
# --------------------------------------------------------------------------
def test_q14_exact_small(oracle):
    """For N <= 4 every twiddle is exact, so Q1.14 = 2^14 x the real transform."""
    rng = np.random.default_rng(22)
    for N in (2, 4):
        x = (rng.integers(-3000, 3001, N) + 1j * rng.integers(-3000, 3001, N)) / 16384.0
        q = scenes.quantize_q14(x)
        Xq, novf = oracle.ndft_q14(q[None])
        X = oracle.ndft(x) * 16384
        assert novf == 0
        np.testing.assert_array_equal(Xq[0, :, 0], X.real.astype(np.int64))
        np.testing.assert_array_equal(Xq[0, :, 1], X.imag.astype(np.int64))


def test_q14_within_twiddle_rounding(oracle):
    """Larger N: each real (x) moves by at most the Q1.14 twiddle rounding (2^-15)."""
    rng = np.random.default_rng(23)
    N = 96
    x = scenes.cn(rng, (2, N)) * 0.5
    q = scenes.quantize_q14(x)
    xd = (q[..., 0] + 1j * q[..., 1]) / 16384.0
    Xq, novf = oracle.ndft_q14(q)
    X = oracle.ndft(xd)
    err = np.abs(Xq[..., 0] / 16384.0 - X.real) + np.abs(Xq[..., 1] / 16384.0 - X.imag)
    assert novf == 0
    assert err.max() <= 4 * N * 2.0 ** -15


def test_q14_wraps_modulo_2_32(oracle):
    """Saturated inputs overflow int32; the result is the exact sum modulo 2^32,
    checked against Python big integers cell by cell."""
    N = 16384
    ss = np.full((N, 2), 32767, np.int16)
    sr = np.full((N, 2), -32768, np.int16)
    A, novf = oracle.caf_q14(ss, sr, 0, 2, 0, 2)
    assert novf > 0
    tw = {p: [oracle.twiddle_q14(N, i * p) for i in range(N)] for p in (0, 1)}

    def exact(l, p):
        re = im = 0
        for i in range(N):
            j = i - l
            c = (int(sr[j, 0]), -int(sr[j, 1])) if 0 <= j < N else (0, 0)
            z = literal.cox((int(ss[i, 0]), int(ss[i, 1])), c)
            t = literal.cox(z, tw[p][i])
            re += t[0]
            im += t[1]
        return re, im

    for l in (0, 1):
        for p in (0, 1):
            re, im = exact(l, p)
            wrap = lambda v: ((v + 2 ** 31) % 2 ** 32) - 2 ** 31
            assert (int(A[l, p, 0]), int(A[l, p, 1])) == (wrap(re), wrap(im))
    assert abs(exact(0, 0)[0]) >= 2 ** 31  # it really overflowed


# --------------------------------------------------------------------------
# Adjoint: central finite differences of the FP64 forward.
# --------------------------------------------------------------------------
def test_adjoint_finite_differences(oracle):
    rng = np.random.default_rng(24)
    N, lag0, nlags, p0, nbins = 48, 0, 6, -4, 8
    ss = scenes.cn(rng, (N,))
    sr = scenes.cn(rng, (N,))
    A = oracle.caf(ss, sr, lag0, nlags, p0, nbins)
    mask = np.zeros(A.shape, bool)
    mask[1:5, 2:7] = True
    L, gA = oracle.masked_abs_loss_grad(A, mask)
    ds = oracle.caf_adjoint(ss, sr, lag0, nlags, p0, nbins, gA)
    # step below the distance of every touched quantity to a zero crossing
    zs = np.stack([oracle.lagprod(ss, sr, l) for l in range(lag0, lag0 + nlags)])
    checked = 0
    for i in range(N):
        margin = min(abs(ss[i].real), abs(ss[i].imag), np.min(np.abs(zs[:, i].real[zs[:, i] != 0])),
                     np.min(np.abs(zs[:, i].imag[zs[:, i] != 0])))
        h = min(0.25 * margin, 1e-4)
        if h < 1e-7:
            continue
        for comp, unit in ((0, 1.0), (1, 1j)):
            sp, sm = ss.copy(), ss.copy()
            sp[i] += h * unit
            sm[i] -= h * unit
            Lp = np.sum(np.abs(oracle.caf(sp, sr, lag0, nlags, p0, nbins))[mask])
            Lm = np.sum(np.abs(oracle.caf(sm, sr, lag0, nlags, p0, nbins))[mask])
            fd = (Lp - Lm) / (2 * h)
            an = ds[i].real if comp == 0 else ds[i].imag
            assert abs(fd - an) <= 1e-5 * max(1.0, abs(an)), (i, comp, fd, an)
            checked += 1
    assert checked >= 40


@pytest.mark.parametrize("flags", [0, 1, 2, 3])
def test_adjoint_ref_finite_differences(oracle, flags):
    """dL/ds_ref against central differences of the fp64 forward (Eq. 12a)."""
    rng = np.random.default_rng(40 + flags)
    N, lag0, nlags, p0, nbins = 40, -2, 7, -3, 9
    ss = scenes.cn(rng, (N,))
    sr = scenes.cn(rng, (N,))
    A = oracle.caf(ss, sr, lag0, nlags, p0, nbins, flags=flags)
    mask = np.zeros(A.shape, bool)
    mask[1:6, 1:8] = True
    L, gA = oracle.masked_abs_loss_grad(A, mask)
    dref = oracle.caf_adjoint_ref(ss, sr, lag0, nlags, p0, nbins, gA, flags=flags)
    zs = np.stack([oracle.lagprod(ss, sr, l, flags=flags) for l in range(lag0, lag0 + nlags)])
    zr = np.abs(zs.real[zs.real != 0]).min()
    zi = np.abs(zs.imag[zs.imag != 0]).min()
    checked = 0
    for j in range(N):
        margin = min(abs(sr[j].real), abs(sr[j].imag), zr, zi)
        h = min(0.25 * margin, 1e-4)
        if h < 1e-7:
            continue
        for comp, unit in ((0, 1.0), (1, 1j)):
            rp, rm = sr.copy(), sr.copy()
            rp[j] += h * unit
            rm[j] -= h * unit
            Lp = np.sum(np.abs(oracle.caf(ss, rp, lag0, nlags, p0, nbins, flags=flags))[mask])
            Lm = np.sum(np.abs(oracle.caf(ss, rm, lag0, nlags, p0, nbins, flags=flags))[mask])
            fd = (Lp - Lm) / (2 * h)
            an = dref[j].real if comp == 0 else dref[j].imag
            assert abs(fd - an) <= 1e-5 * max(1.0, abs(an)), (j, comp, fd, an)
            checked += 1
    assert checked >= 30
    # the non-circular window leaves the first and last samples of s_ref unread at some lags
    assert np.any(dref != 0)


def test_adjoints_against_torch_autograd(oracle):
    """Both adjoints against torch autograd through a plain elementwise forward of
    Eq. 1-2 / 6 / 12a (sign and abs only: autograd's own derivative rules)."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(77)
    N, lag0, nlags, p0, nbins = 24, -3, 6, 2, 7
    ss = scenes.cn(rng, (N,))
    sr = scenes.cn(rng, (N,))
    gA = scenes.cn(rng, (nlags, nbins))

    def ot(a, b):  # Eq. 1-2
        return torch.sign(a * b) * (torch.abs(a) + torch.abs(b))

    def cot(ar, ai, br, bi):  # Eq. 6
        return ot(ar, br) - ot(ai, bi), ot(ar, bi) + ot(ai, br)

    t = lambda v: torch.tensor(v, dtype=torch.float64, requires_grad=True)
    sr_r, sr_i, ss_r, ss_i = t(sr.real), t(sr.imag), t(ss.real), t(ss.imag)
    n = torch.arange(N, dtype=torch.float64)
    loss = 0.0
    for a in range(nlags):
        l = lag0 + a
        idx = [i - l for i in range(N)]
        ok = torch.tensor([0 <= j < N for j in idx])
        jj = torch.tensor([min(max(j, 0), N - 1) for j in idx])
        cr = torch.where(ok, sr_r[jj], torch.zeros(()))
        ci = torch.where(ok, -sr_i[jj], torch.zeros(()))
        zr, zi = cot(ss_r, ss_i, cr, ci)
        for k in range(nbins):
            p = p0 + k
            th = 2 * np.pi * ((n * p) % N) / N
            wr, wi = torch.cos(th), -torch.sin(th)
            # the axis twiddles are exactly 0 (a (x) 0 = 0), not the 1e-16 of cos/sin
            wr = torch.where(wr.abs() < 1e-12, torch.zeros(()), wr)
            wi = torch.where(wi.abs() < 1e-12, torch.zeros(()), wi)
            Ar, Ai = cot(zr, zi, wr, wi)
            loss = loss + gA[a, k].real * Ar.sum() + gA[a, k].imag * Ai.sum()
    loss.backward()
    want_ref = sr_r.grad.numpy() + 1j * sr_i.grad.numpy()
    want_surv = ss_r.grad.numpy() + 1j * ss_i.grad.numpy()
    got_ref = oracle.caf_adjoint_ref(ss, sr, lag0, nlags, p0, nbins, gA)
    got_surv = oracle.caf_adjoint(ss, sr, lag0, nlags, p0, nbins, gA)
    np.testing.assert_allclose(got_ref, want_ref, rtol=0, atol=1e-9)
    np.testing.assert_allclose(got_surv, want_surv, rtol=0, atol=1e-9)


def test_adjoint_sampled_matches_full(oracle):
    """The sampled adjoints return the full adjoints' values at the listed indices."""
    rng = np.random.default_rng(91)
    N, lag0, nlags, p0, nbins = 57, -4, 9, 5, 11
    ss = scenes.cn(rng, (N,))
    sr = scenes.cn(rng, (N,))
    gA = scenes.cn(rng, (nlags, nbins))
    idx = np.array([0, 3, 17, 56, 40])
    for flags in (0, 3):
        full_s = oracle.caf_adjoint(ss, sr, lag0, nlags, p0, nbins, gA, flags=flags)
        full_r = oracle.caf_adjoint_ref(ss, sr, lag0, nlags, p0, nbins, gA, flags=flags)
        assert np.array_equal(oracle.caf_adjoint_at(ss, sr, lag0, nlags, p0, nbins, gA, "surv", idx, flags),
                              full_s[idx])
        assert np.array_equal(oracle.caf_adjoint_at(ss, sr, lag0, nlags, p0, nbins, gA, "ref", idx, flags),
                              full_r[idx])


def test_lags_at_the_int32_limits(oracle):
    """Lags are taken as int64 by the oracle: windows ending at 2^31 - 1 or
    starting at -2^31 meet no sample (exact zeros, adjoints included), and with
    the circular flag they reduce modulo N, so they equal the reduced window."""
    rng = np.random.default_rng(92)
    N, nlags, p0, nbins = 40, 3, -5, 9
    ss = scenes.cn(rng, (N,))
    sr = scenes.cn(rng, (N,))
    gA = scenes.cn(rng, (nlags, nbins))
    circ = oracle.F_CIRCULAR_LAG
    for lag0 in (2**31 - nlags, -2**31):
        assert np.all(oracle.caf(ss, sr, lag0, nlags, p0, nbins) == 0)
        assert np.all(oracle.caf_adjoint(ss, sr, lag0, nlags, p0, nbins, gA) == 0)
        assert np.all(oracle.caf_adjoint_ref(ss, sr, lag0, nlags, p0, nbins, gA) == 0)
        red = lag0 % N
        assert red + nlags <= N  # no wrap inside the reduced window
        np.testing.assert_array_equal(oracle.caf(ss, sr, lag0, nlags, p0, nbins, flags=circ),
                                      oracle.caf(ss, sr, red, nlags, p0, nbins, flags=circ))
        np.testing.assert_array_equal(oracle.caf_adjoint(ss, sr, lag0, nlags, p0, nbins, gA, flags=circ),
                                      oracle.caf_adjoint(ss, sr, red, nlags, p0, nbins, gA, flags=circ))
        np.testing.assert_array_equal(oracle.caf_adjoint_ref(ss, sr, lag0, nlags, p0, nbins, gA, flags=circ),
                                      oracle.caf_adjoint_ref(ss, sr, red, nlags, p0, nbins, gA, flags=circ))
        assert np.any(oracle.caf(ss, sr, lag0, nlags, p0, nbins, flags=circ) != 0)
