"""The fp32 evaluation orders of the complex (x) (Eq. 6) that the kernels use,
emulated on the CPU and compared bit for bit with the oracle's fp32 lag
product, which rounds each real a (x) b = sgn(ab)(|a| + |b|) (Eq. 1-2) once
and then forms the difference and the sum.

The kernels' form: each real (x) starts as the inner fma(sgn b, |a|, b) =
sgn(b)(|a| + |b|), rounded once; scaling it by sgn a (+-1 or a zero) is
exact, so the difference and the sum of Eq. 6 take one fma each, whose addend
is the other term scaled by one more fma with a +0 addend.  The claim under
test: the same bits as the per-term rounding, signed zeros, subnormals and
exact cancellations included.

Emulation: every fma here has a factor in {-1, -0, +0, +1}, so its product is
exact and it is one rounded addition of two fp32 values; evaluating that
addition in fp64 and rounding to fp32 rounds it correctly (53 >= 2 * 24 + 2,
so the double rounding is innocuous).  No code is shared with the CUDA path.
"""
import numpy as np
import pytest

F32, F64 = np.float32, np.float64


def _sgn(v):
    """sgn(v) as the kernels form it: +-1 with v's sign, or a zero of v's sign."""
    return np.copysign((v != 0).astype(F32), v).astype(F32)


def _fma(s, b, c):
    """fma(s, b, c) for s in {-1, -0, +0, +1}: one correctly rounded addition."""
    return (s.astype(F64) * b.astype(F64) + c.astype(F64)).astype(F32)


def cox_fma(a, b):
    """Eq. 6 in the kernels' fma form on complex64 arrays a, b."""
    ar, ai, br, bi = a.real, a.imag, b.real, b.imag
    sar, sai, sbr, sbi = _sgn(ar), _sgn(ai), _sgn(br), _sgn(bi)
    i1 = _fma(sbr, np.abs(ar), br)  # sgn b_r (|a_r| + |b_r|)
    i2 = _fma(sbi, np.abs(ai), bi)  # sgn b_i (|a_i| + |b_i|)
    i3 = _fma(sbr, np.abs(ai), br)  # sgn b_r (|a_i| + |b_r|)
    i4 = _fma(sbi, np.abs(ar), bi)  # sgn b_i (|a_r| + |b_i|)
    z = np.zeros_like(ar)
    n2 = _fma(-sai, i2, z)          # -(a_i (x) b_i)
    t4 = _fma(sar, i4, z)           # a_r (x) b_i
    out = np.empty(a.shape, np.complex64)
    out.real = _fma(sar, i1, n2)
    out.imag = _fma(sai, i3, t4)
    return out


def _operands(rng, n):
    """CN values over 12 decades, with zeros of both signs, subnormals, the
    smallest normal, and exact cancellations mixed in."""
    special = np.array([0.0, -0.0, 1.0, -1.0, 0.5, -0.5, 1e-40, -1e-40, 3e-45, -3e-45, 2.0**-126, 1.5, 0.75],
                       dtype=F32)

    def part():
        x = rng.standard_normal(n).astype(F32) * (F32(10.0) ** rng.integers(-6, 6, n).astype(F32))
        m = rng.random(n) < 0.3
        x[m] = special[rng.integers(0, special.size, int(m.sum()))]
        return x

    s = (part() + 1j * part()).astype(np.complex64)
    r = (part() + 1j * part()).astype(np.complex64)
    k = rng.random(n) < 0.05  # s_i = s_r, r_i = r_r: Im of s (x) conj(r), or Re of s (x) r, cancels exactly
    s.imag[k] = s.real[k]
    r.imag[k] = r.real[k]
    return s, r


def _bits(z):
    return np.ascontiguousarray(z, np.complex64).view(np.uint32)


@pytest.mark.parametrize("flags", [0, 1])  # conj(s_ref), or s_ref itself (NDFT_F_NO_CONJ_REF)
def test_fma_form_matches_the_oracles_fp32_lag_product(oracle, flags):
    rng = np.random.default_rng(160 + flags)
    n = 400_000
    ss, sr = _operands(rng, n)
    want = oracle.lagprod_f32(ss, sr, 0, flags=flags)  # lag 0: s_surv[i] (x) c(s_ref[i])
    ref = sr if flags else np.conj(sr).astype(np.complex64)
    got = cox_fma(ss, ref)
    assert np.array_equal(_bits(got), _bits(want))
    # the cases the claim is about were exercised: zero results (all +0) and subnormal operands
    zeros = got.real == 0
    assert zeros.sum() > 1000 and not np.signbit(got.real[zeros]).any()
    assert ((ss.real != 0) & (np.abs(ss.real) < 2.0**-126)).sum() > 1000


def test_fma_form_reduces_to_eq2_on_real_operands(oracle):
    """Imaginary parts zero: Re is a_r (x) b_r of Eq. 2 itself, Im = 0."""
    rng = np.random.default_rng(162)
    ss, sr = _operands(rng, 50_000)
    ss = ss.real.astype(np.complex64)
    sr = sr.real.astype(np.complex64)
    got = cox_fma(ss, sr)
    want = np.array([oracle.otimes(float(a), float(b)) for a, b in zip(ss.real[:2000], sr.real[:2000])])
    np.testing.assert_array_equal(got.real[:2000], want.astype(F32))
    assert np.all(got.imag == 0) and not np.signbit(got.imag).any()
