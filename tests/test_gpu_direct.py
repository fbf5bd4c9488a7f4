"""GPU parity of the plain (direct) form, the NFFT, the tables, the adjoint and
the peak search against the CPU oracle, through the C ABI (via the ctypes
binding).  Sizes span several 64 x 64 tiles and a ragged tail."""
import numpy as np
import pytest

import oracle
from paper_1402_0532_gb300 import scenes

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

TOL = 1e-5  # relative to max |X|, the fp32 bar for the transforms


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1402_0532_gb300 import api as A
    return A


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def relerr(got, ref):
    return float(np.max(np.abs(got - ref)) / max(np.max(np.abs(ref)), 1e-30))


def check_nfft_vs_fp64(got, x, dif):
    """The NFFT gate against fp64: every sign-stable vector within the running
    error bound of the fp64 recursion and within TOL of its max |X|; returns
    the number of vectors left out as ill-conditioned (and prints it)."""
    X, bound, stable = oracle.nfft_bound(x, dif=dif)
    amax = np.maximum(np.abs(X).max(axis=1), 1e-30)
    if stable.any():
        assert oracle.within_bound(got[stable], X[stable], bound[stable]).all()
        assert (np.abs(got - X).max(axis=1) / amax)[stable].max() < TOL
    print(f"NFFT N={x.shape[1]} dif={dif}: {int((~stable).sum())} of {len(stable)} vectors ill-conditioned")
    return int((~stable).sum())


# --------------------------------------------------------------------------------
# tables
# --------------------------------------------------------------------------------
@pytest.mark.parametrize("N", [1, 2, 3, 6, 7, 64, 1000, 1024, 4099, 32767, 65536])
def test_tables_match_oracle(api, N):
    p = api.Plan(N, max_batch=1)
    got = p.twiddles(0).cpu().numpy()
    want = oracle.twiddle_table_f32(N)
    assert np.array_equal(got.view(np.uint32), want.view(np.uint32)), \
        f"{np.count_nonzero(got != want)} fp32 twiddles differ"
    q = api.Plan(N, max_batch=1, prec="q14")
    assert np.array_equal(q.twiddles(1).cpu().numpy(), oracle.twiddle_table_q14(N))


# --------------------------------------------------------------------------------
# NDFT, Eq. 8
# --------------------------------------------------------------------------------
def test_ndft_tone_batch(api):
    """The N = 64 batch of 4096 vectors: vector 0 is the exact tone at k0 = 7."""
    x = scenes.tone_batch()
    ref = oracle.ndft(x.astype(np.complex128))
    p = api.Plan(64, max_batch=4096)
    X = p.ndft(dev(x))
    got = X.cpu().numpy()
    per = np.max(np.abs(got - ref), axis=1) / np.max(np.abs(ref), axis=1)
    assert per.max() < TOL
    idx, _ = api.argmax(X)
    idx = idx.cpu().numpy()
    assert idx[0] == 7
    assert abs(got[0, 7].real - 8.0 / np.tan(np.pi / 64)) < TOL * 163
    # peak locations identical wherever the oracle's top-2 gap exceeds twice the tolerance
    mag = np.abs(ref)
    srt = np.sort(mag, axis=1)
    clear = (srt[:, -1] - srt[:, -2]) > 2 * TOL * srt[:, -1]
    assert clear.sum() > 3000
    assert np.array_equal(idx[clear], np.argmax(mag, axis=1)[clear])


@pytest.mark.parametrize("N,batch,p0,nbins", [(100, 130, -7, 77), (64, 1, 0, 0), (1, 3, 0, 1), (257, 65, 300, 200)])
def test_ndft_ragged(api, N, batch, p0, nbins):
    rng = np.random.default_rng(N + batch)
    x = scenes.cn(rng, (batch, N)).astype(np.complex64)
    x[:, ::9] = 0
    nb = nbins or N
    ref = oracle.ndft(x.astype(np.complex128), p0=p0, nbins=nb)
    p = api.Plan(N, p0=p0, nbins=nbins, max_batch=batch)
    got = p.ndft(dev(x)).cpu().numpy()
    assert got.shape == (batch, nb)
    assert relerr(got, ref) < TOL


@pytest.mark.parametrize("N,batch,p0,nbins", [(96, 70, 5, 90), (64, 130, 0, 0), (7, 3, -2, 5)])
def test_ndft_q14_bit_exact(api, N, batch, p0, nbins):
    rng = np.random.default_rng(7 * N)
    q = scenes.quantize_q14(scenes.cn(rng, (batch, N)) * 0.5)
    q[:, ::5, 1] = 0
    nb = nbins or N
    want, _ = oracle.ndft_q14(q, p0=p0, nbins=nb)
    p = api.Plan(N, p0=p0, nbins=nbins, max_batch=batch, prec="q14")
    got = p.ndft(dev(q)).cpu().numpy()
    assert np.array_equal(got, want)


# --------------------------------------------------------------------------------
# NFFT, Sec. 3
# --------------------------------------------------------------------------------
@pytest.mark.parametrize("N,batch", [(2, 300), (4, 301), (8, 300), (16, 77), (32, 65), (64, 100), (128, 33),
                                     (256, 17), (512, 9), (1024, 40), (2048, 5), (4096, 3), (8192, 3),
                                     (16384, 3), (32768, 3), (64, 40000)])
def test_nfft_bit_exact(api, N, batch):
    """Bit for bit (zero signs, exact cancellations and subnormal inputs
    included) against the oracle's fp32 recursion, for every register-kernel
    size, ragged batches, and a batch large enough
    that each persistent block loops over several vector groups."""
    rng = np.random.default_rng(N)
    x = scenes.cn(rng, (batch, N)).astype(np.complex64)
    x[0] = scenes.exact_tone(N, 1 if N > 1 else 0).astype(np.complex64)
    x[1, ::3] = 0
    x[2, ::5] = np.complex64(complex(-0.0, -0.0))
    x[2, 1::5] = np.complex64(complex(0.0, -0.0))
    if batch > 4:
        # eighths of small integers: many butterflies cancel exactly to zero; and a row
        # of subnormals, whose (x) with a twiddle magnitude is a normal number
        x[3] = (rng.integers(-3, 4, N) + 1j * rng.integers(-3, 4, N)).astype(np.complex64) / 8
        x[4] = (scenes.cn(rng, (N,)) * 1e-39).astype(np.complex64)
    want = oracle.nfft_f32(x)
    p = api.Plan(N, max_batch=batch)
    got = p.nfft(dev(x)).cpu().numpy()
    assert np.array_equal(got.view(np.uint32), want.view(np.uint32))
    # in place
    t = dev(x)
    p.nfft(t, out=t)
    assert np.array_equal(t.cpu().numpy().view(np.uint32), want.view(np.uint32))
    # against the fp64 recursion: on the vectors whose every (x) data operand
    # provably keeps its fp64 sign in fp32 (the oracle's running error bound),
    # within that bound and within the 1e-5 bar; the others are counted and
    # reported, not failed ((x) jumps at zero, so there fp32 and fp64 may
    # legitimately part)
    if N <= 4096:
        check_nfft_vs_fp64(got, x, dif=False)


def test_nfft_hand_cases(api):
    import json
    import os
    h = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "hand_cases.json")))
    for case in h["cases"]:
        x = np.array([complex(a, b) for a, b in case["x"]], np.complex64)[None]
        p = api.Plan(case["N"], max_batch=1)
        np.testing.assert_array_equal(p.nfft(dev(x)).cpu().numpy()[0],
                                      [complex(a, b) for a, b in case["nfft"]])
        np.testing.assert_array_equal(p.ndft(dev(x)).cpu().numpy()[0],
                                      [complex(a, b) for a, b in case["ndft"]])


# --------------------------------------------------------------------------------
# CAF, Eq. 12a
# --------------------------------------------------------------------------------
def test_caf_direct_fp32(api):
    sc = scenes.radar_scene(N=4133, nlags=100, nbins=96, seed=31)
    lag0 = -3
    ref32 = oracle.caf(sc.s_surv, sc.s_ref, lag0, 100, sc.p0, 96, z32=True)
    ref64 = oracle.caf(sc.s_surv, sc.s_ref, lag0, 100, sc.p0, 96)
    p = api.Plan(sc.N, p0=sc.p0, nbins=96, max_lags=128)
    got = p.caf(dev(sc.s_surv), dev(sc.s_ref), lag0, 100).cpu().numpy()
    assert relerr(got, ref32) < TOL
    assert relerr(got, ref64) < 1e-3  # the fp32 lag product may flip a sign near 0
    p.query_error()


@pytest.mark.parametrize("flags", [1, 2])
def test_caf_direct_flags(api, flags):
    sc = scenes.radar_scene(N=700, nlags=40, nbins=33, seed=32)
    ref = oracle.caf(sc.s_surv, sc.s_ref, 650, 40, -16, 33, flags=flags, z32=True)
    p = api.Plan(sc.N, p0=-16, nbins=33, max_lags=40, flags=flags)
    got = p.caf(dev(sc.s_surv), dev(sc.s_ref), 650, 40).cpu().numpy()
    assert relerr(got, ref) < TOL


def test_caf_direct_q14_bit_exact(api):
    sc = scenes.radar_scene(N=1500, nlags=70, nbins=80, seed=33)
    qs, qr = scenes.quantize_q14(sc.s_surv, 0.25), scenes.quantize_q14(sc.s_ref, 0.25)
    want, _ = oracle.caf_q14(qs, qr, 0, 70, -40, 80)
    p = api.Plan(sc.N, p0=-40, nbins=80, max_lags=70, prec="q14")
    got = p.caf(dev(qs), dev(qr), 0, 70).cpu().numpy()
    assert np.array_equal(got, want)


def test_caf_direct_q14_wraps(api):
    """Full-scale inputs: the exact sums leave int32 (the oracle counts the
    cells) and the output holds them modulo 2^32, bit for bit, with or without
    the range check; with NDFT_F_Q14_RANGE ndft_query_error reports
    NDFT_E_OVERFLOW, and the plan reports nothing on a call that stays in range."""
    from paper_1402_0532_gb300 import _lib as L
    N = 16384
    ss = np.full((N, 2), 32767, np.int16)
    sr = np.full((N, 2), -32768, np.int16)
    want, novf = oracle.caf_q14(ss, sr, 0, 3, -1, 3)
    assert novf > 0
    p = api.Plan(N, p0=-1, nbins=3, max_lags=3, prec="q14")
    got = p.caf(dev(ss), dev(sr), 0, 3).cpu().numpy()
    assert np.array_equal(got, want)
    p.query_error()  # no report without the flag
    r = api.Plan(N, p0=-1, nbins=3, max_lags=3, prec="q14", flags=api.F_Q14_RANGE)
    got = r.caf(dev(ss), dev(sr), 0, 3).cpu().numpy()
    assert np.array_equal(got, want)
    with pytest.raises(L.NdftError) as ex:
        r.query_error()
    assert ex.value.status == L.E_OVERFLOW
    # the report was cleared; a call whose sums stay in range reports nothing
    small_s, small_r = ss[:200] // 64, sr[:200] // 64
    q = api.Plan(200, p0=-1, nbins=3, max_lags=3, prec="q14", flags=api.F_Q14_RANGE)
    w2, n2 = oracle.caf_q14(small_s, small_r, 0, 3, -1, 3)
    assert n2 == 0
    assert np.array_equal(q.caf(dev(small_s), dev(small_r), 0, 3).cpu().numpy(), w2)
    q.query_error()


@pytest.mark.parametrize("N,batch,p0,nbins", [(65536, 3, -2, 5), (4099, 70, 100, 129)])
def test_ndft_q14_range_check(api, N, batch, p0, nbins):
    """NDFT in Q1.14 with NDFT_F_Q14_RANGE: the same bits as without it, and
    NDFT_E_OVERFLOW exactly when the oracle counts a wrapped cell."""
    from paper_1402_0532_gb300 import _lib as L
    rng = np.random.default_rng(N)
    if N == 65536:
        q = np.full((batch, N, 2), 32767, np.int16)  # full scale: bin 0 sums 65536 x 49151 > 2^31
        q[1, ::2] = -32768
    else:
        q = scenes.quantize_q14(scenes.cn(rng, (batch, N)) * 0.5)
    want, novf = oracle.ndft_q14(q, p0=p0, nbins=nbins)
    for flags in (0, api.F_Q14_RANGE):
        p = api.Plan(N, p0=p0, nbins=nbins, max_batch=batch, prec="q14", flags=flags)
        got = p.ndft(dev(q)).cpu().numpy()
        assert np.array_equal(got, want)
        if flags and novf > 0:
            with pytest.raises(L.NdftError) as ex:
                p.query_error()
            assert ex.value.status == L.E_OVERFLOW
        else:
            p.query_error()
    assert (novf > 0) == (N == 65536)


# --------------------------------------------------------------------------------
# adjoint
# --------------------------------------------------------------------------------
def test_caf_backward_matches_oracle(api):
    sc = scenes.radar_scene(N=700, nlags=70, nbins=40, seed=34)
    rng = np.random.default_rng(35)
    dA = scenes.cn(rng, (70, 40))
    want = oracle.caf_adjoint(sc.s_surv, sc.s_ref, 2, 70, -20, 40, dA)
    p = api.Plan(sc.N, p0=-20, nbins=40, max_lags=70)
    got = p.caf_backward(dev(sc.s_surv), dev(sc.s_ref), 2, 70, dev(dA.astype(np.complex64))).cpu().numpy()
    assert relerr(got, want) < TOL


# --------------------------------------------------------------------------------
# peak search
# --------------------------------------------------------------------------------
def test_argmax_ties_lowest_index(api):
    X = np.zeros((3, 1000), np.complex64)
    X[0, [5, 900]] = 3 + 4j
    X[1, 999] = 1j
    X[2] = 1
    idx, val = api.argmax(dev(X))
    assert idx.cpu().tolist() == [5, 999, 0]
    assert val.cpu().tolist() == [25.0, 1.0, 1.0]


# --------------------------------------------------------------------------------
# batched CPIs, direct form
# --------------------------------------------------------------------------------
def _pack(scs, q14=False):
    surv, ref, cpis, oo = [], [], [], 0
    so = 0
    for sc in scs:
        a = scenes.quantize_q14(sc.s_surv, 0.25) if q14 else sc.s_surv
        b = scenes.quantize_q14(sc.s_ref, 0.25) if q14 else sc.s_ref
        pad = (-sc.N) % 4
        cpis.append(dict(off_surv=so, off_ref=so, off_out=oo, n=sc.N, lag0=sc.lag0, nlags=sc.nlags, p0=sc.p0,
                         nbins=sc.nbins))
        z = np.zeros((pad, 2), np.int16) if q14 else np.zeros(pad, np.complex64)
        surv += [a, z]
        ref += [b, z]
        so += sc.N + pad
        oo += sc.nlags * sc.nbins
    return np.concatenate(surv), np.concatenate(ref), cpis, oo


@pytest.mark.parametrize("q14", [False, True])
def test_batched_direct(api, q14):
    rng = np.random.default_rng(36)
    scs = [scenes.radar_scene(N=int(n), nlags=int(l), nbins=int(b), rng=rng)
           for n, l, b in ((1000, 70, 64), (1536, 5, 96), (777, 130, 33), (2048, 64, 128), (1111, 1, 7))]
    surv, ref, cpis, total = _pack(scs, q14)
    bp = api.BatchedPlan(cpis, prec="q14" if q14 else "fp32")
    out = torch.zeros((total, 2) if q14 else total, dtype=torch.int32 if q14 else torch.complex64, device="cuda")
    bp(dev(surv), dev(ref), out)
    bp.query_error()
    got = out.cpu().numpy()
    for sc, c in zip(scs, cpis):
        g = got[c["off_out"]: c["off_out"] + sc.nlags * sc.nbins]
        if q14:
            want, _ = oracle.caf_q14(scenes.quantize_q14(sc.s_surv, 0.25), scenes.quantize_q14(sc.s_ref, 0.25),
                                     sc.lag0, sc.nlags, sc.p0, sc.nbins)
            assert np.array_equal(g.reshape(sc.nlags, sc.nbins, 2), want)
        else:
            want = oracle.caf(sc.s_surv, sc.s_ref, sc.lag0, sc.nlags, sc.p0, sc.nbins, z32=True)
            assert relerr(g.reshape(sc.nlags, sc.nbins), want) < TOL


# --------------------------------------------------------------------------------
# argument errors on a live plan
# --------------------------------------------------------------------------------
def test_invalid_arguments(api):
    from paper_1402_0532_gb300 import _lib as L
    p = api.Plan(100, max_batch=4, max_lags=8)
    x = torch.zeros(5, 100, dtype=torch.complex64, device="cuda")
    with pytest.raises(L.NdftError) as e:
        p.ndft(x)  # batch 5 > max_batch 4
    assert e.value.status == L.E_INVALID
    with pytest.raises(L.NdftError):
        p.nfft(x[:4])  # N = 100 is not a power of two
    s = torch.zeros(101, dtype=torch.complex64, device="cuda")
    with pytest.raises(L.NdftError):
        p.caf(s[1:], s[1:], 0, 4)  # misaligned (8-byte offset)
    with pytest.raises(L.NdftError):
        p.caf(s[:100], s[:100], 0, 9)  # nlags > max_lags
    p.query_error()


@pytest.mark.parametrize("N,nbins,batch", [(1024, 32, 16), (4133, 96, 7), (16384, 128, 3)])
def test_direct_ndft_split_sample_axis(api, N, nbins, batch):
    """Small NDFT calls (few bin x column tiles) split their sample axis over
    blocks and sum the partials in order: fp32 within the bar, Q1.14 bit-exact,
    ragged N included; form="auto" picks the tensor cores above N = 64."""
    rng = np.random.default_rng(70 + N % 13)
    x = scenes.cn(rng, (batch, N)).astype(np.complex64)
    p0 = -(nbins // 2)
    p = api.Plan(N, p0=p0, nbins=nbins, max_batch=batch, form="direct", prec="fp32")
    got = p.ndft(dev(x)).cpu().numpy()
    p.query_error()
    assert p.last_launches() == 2  # the split tile kernel and the ordered sum
    ref = oracle.ndft(x.astype(np.complex128), p0=p0, nbins=nbins)
    assert np.max(np.abs(got - ref)) / np.max(np.abs(ref)) < 1e-5
    xq = scenes.quantize_q14(scenes.cn(rng, (batch, N)) * 0.25)
    q = api.Plan(N, p0=p0, nbins=nbins, max_batch=batch, form="direct", prec="q14")
    gq = q.ndft(dev(xq)).cpu().numpy()
    q.query_error()
    assert q.last_launches() == 2
    want, _ = oracle.ndft_q14(xq, p0=p0, nbins=nbins)
    assert np.array_equal(gq, want)
    a = api.Plan(N, p0=p0, nbins=nbins, max_batch=batch, form="auto")
    assert a.form == "ternary" and a.prec == "bf16x2"
