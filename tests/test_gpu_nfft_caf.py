"""GPU parity of the NFFT form (Sec. 3 in place of the NDFT): bins of the NFFT
through ndft_exec, and Eq. 12a with the NFFT over each lag product through
caf_exec.  Both are reproducible bit for bit, so the bar is equality of the bit
patterns with the oracle's fp32 evaluation (lag product and recursion in
fp32, one rounding per operation)."""
import numpy as np
import pytest

import oracle
from paper_1402_0532_gb300 import scenes

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


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


def same_bits(a, b):
    a = np.ascontiguousarray(a, np.complex64)
    b = np.ascontiguousarray(b, np.complex64)
    return a.shape == b.shape and np.array_equal(a.view(np.uint32), b.view(np.uint32))


@pytest.mark.parametrize("N,batch,p0,nbins", [(1, 5, 0, 0), (2, 7, 1, 1), (4, 9, -1, 3), (8, 300, 0, 0),
                                              (64, 100, -32, 64), (1024, 33, -512, 1024), (4096, 5, 100, 7),
                                              (8192, 3, -4096, 8192), (16384, 2, 5, 300), (32768, 3, 0, 0),
                                              (65536, 2, -512, 1024)])
def test_nfft_form_bins(api, N, batch, p0, nbins):
    rng = np.random.default_rng(N + 7)
    x = scenes.cn(rng, (batch, N)).astype(np.complex64)
    if batch > 2:
        x[1, ::3] = 0
        x[2, ::5] = np.complex64(complex(-0.0, -0.0))
    nb = nbins or N
    full = oracle.nfft_f32(x)
    want = full[:, (p0 + np.arange(nb)) % N]
    p = api.Plan(N, p0=p0, nbins=nbins, max_batch=batch, form="nfft", prec="fp32")
    got = p.ndft(dev(x)).cpu().numpy()
    p.query_error()
    assert same_bits(got, want)
    # the plain NFFT entry point on the same plan gives the full natural-order output
    if nb == N and p0 % N == 0:
        assert same_bits(p.nfft(dev(x)).cpu().numpy(), full)


@pytest.mark.parametrize("N,lag0,nlags,p0,nbins,flags", [
    (8, -3, 12, 0, 0, 0), (256, 0, 40, -128, 256, 0), (1024, -5, 77, -512, 1024, 0),
    (4096, 100, 9, 7, 33, 1), (4096, 4000, 9, 0, 16, 2), (8192, 0, 21, -4096, 8192, 0),
    (16384, 37, 5, -512, 1024, 0), (65536, 0, 3, -512, 1024, 0), (65536, 65530, 9, 0, 64, 2),
    # the pruned tail at its limits: exactly 2^LA bins, and a window that wraps past bin 0
    (8192, 5, 7, 100, 1024, 0), (16384, -2, 6, -300, 700, 1),
    # the two-kernel path's comb rows: lags past -N (exact zeros), negative
    # circular lags, circular lags without the conjugate
    (8192, -9000, 4, -64, 128, 0), (8192, -3, 5, -64, 128, 2), (32768, 12345, 4, -512, 1024, 3)])
def test_nfft_form_caf(api, N, lag0, nlags, p0, nbins, flags):
    sc = scenes.radar_scene(N=N, nlags=max(nlags, 1), nbins=min(N, 64), seed=60 + N % 97)
    nb = nbins or N
    want = oracle.caf_nfft(sc.s_surv, sc.s_ref, lag0, nlags, p0, nb, flags=flags, f32=True)
    p = api.Plan(N, p0=p0, nbins=nbins, max_lags=nlags, flags=flags, form="nfft", prec="fp32")
    got = p.caf(dev(sc.s_surv), dev(sc.s_ref), lag0, nlags).cpu().numpy()
    p.query_error()
    assert same_bits(got, want)


def test_nfft_form_caf_full_size_sampled(api):
    """The 65536-sample, 1024-lag surface at the 1024 centred bins (the launch
    configuration of the benchmark line): lags sampled across every chunk of
    the two-kernel path, each row bit for bit."""
    sc = scenes.radar_scene(N=65536)
    p = api.Plan(65536, p0=-512, nbins=1024, max_lags=1024, form="nfft", prec="fp32")
    A = p.caf(dev(sc.s_surv), dev(sc.s_ref), 0, 1024).cpu().numpy()
    p.query_error()
    for lag in (0, 1, 37, 63, 64, 120, 127, 128, 301, 555, 1023):
        want = oracle.caf_nfft(sc.s_surv, sc.s_ref, lag, 1, -512, 1024, f32=True)
        assert same_bits(A[lag:lag + 1], want), lag


@pytest.mark.parametrize("N,dif", [(8192, False), (65536, False), (8192, True), (65536, True)])
def test_nfft_form_lag_rows_at_the_int32_limits(api, N, dif):
    """The two-kernel paths form each vector's lag products from one row of
    each input with the reference offset fixed per lag (DIT: one comb row;
    DIF: the natural row): windows ending at INT32_MAX or starting at
    INT32_MIN give an exactly zero surface, and with F_CIRCULAR_LAG the
    surface of the window reduced modulo N, bit for bit."""
    nl = 3
    rng = np.random.default_rng(86)
    ss = dev(scenes.cn(rng, (N,)).astype(np.complex64))
    sr = dev(scenes.cn(rng, (N,)).astype(np.complex64))
    f = api.F_NFFT_DIF if dif else 0
    for lag0 in (2**31 - nl, -2**31):
        p = api.Plan(N, p0=-64, nbins=128, max_lags=nl, form="nfft", prec="fp32", flags=f)
        assert torch.count_nonzero(p.caf(ss, sr, lag0, nl)).item() == 0
        pc = api.Plan(N, p0=-64, nbins=128, max_lags=nl, form="nfft", prec="fp32", flags=f | api.F_CIRCULAR_LAG)
        got = pc.caf(ss, sr, lag0, nl).cpu().numpy()
        ref = pc.caf(ss, sr, lag0 % N, nl).cpu().numpy()  # lag0 % N + nl <= N: no wrap inside
        pc.query_error()
        assert same_bits(got, ref)
        assert np.count_nonzero(got) > 0


def test_nfft_form_unsupported(api):
    from paper_1402_0532_gb300 import _lib as L
    with pytest.raises(L.NdftError) as e:
        api.Plan(100, max_batch=1, form="nfft", prec="fp32")
    assert e.value.status == L.E_INVALID
    with pytest.raises(L.NdftError) as e:
        api.Plan(131072, max_batch=1, form="nfft", prec="fp32")
    assert e.value.status == L.E_INVALID
    with pytest.raises(L.NdftError) as e:
        api.Plan(64, max_batch=1, form="nfft", prec="bf16x2")
    assert e.value.status == L.E_UNSUPPORTED
    p = api.Plan(64, max_lags=4, form="nfft", prec="fp32")
    s = torch.zeros(64, dtype=torch.complex64, device="cuda")
    dA = torch.zeros(4, 64, dtype=torch.complex64, device="cuda")
    with pytest.raises(L.NdftError) as e:
        p.caf_backward(s, s, 0, 4, dA)
    assert e.value.status == L.E_UNSUPPORTED
