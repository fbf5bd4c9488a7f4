"""Edge cases of the CUDA path against the oracle: the largest transform each
form accepts, an empty batch, a lag window entirely outside the samples
(exact zeros), lag windows at the int32 limits, a single lag, and the adjoints
at the same degenerate inputs."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_1402_0532_gb300 import scenes

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

TOL = 1e-5


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


def test_ternary_largest_n(api):
    """N = 2^18, the tensor-core form's limit: 3 vectors, 64 bins around -32."""
    N = 1 << 18
    x = scenes.cn(np.random.default_rng(80), (3, N)).astype(np.complex64)
    p = api.Plan(N, p0=-32, nbins=64, max_batch=3, form="ternary", prec="bf16x2")
    got = p.ndft(dev(x)).cpu().numpy()
    p.query_error()
    assert relerr(got, oracle.ndft(x, p0=-32, nbins=64)) < TOL


def test_direct_largest_n_caf(api):
    """N = 2^20 in the plain form: 2 lags x 16 bins, sampled against the oracle."""
    N = 1 << 20
    rng = np.random.default_rng(81)
    ss = scenes.cn(rng, (N,)).astype(np.complex64)
    sr = scenes.cn(rng, (N,)).astype(np.complex64)
    p = api.Plan(N, p0=-8, nbins=16, max_lags=2)
    got = p.caf(dev(ss), dev(sr), 3, 2).cpu().numpy()
    p.query_error()
    L, P = np.meshgrid([3, 4], np.arange(-8, 8), indexing="ij")
    want = oracle.caf_cells(ss, sr, L.ravel(), P.ravel(), z32=True).reshape(2, 16)
    assert relerr(got, want) < TOL


def test_direct_largest_n_ndft(api):
    """N = 2^20 NDFT in the plain form (each thread sums all 2^20 samples of its
    cells, in two levels), 2 vectors x 16 bins."""
    N = 1 << 20
    x = scenes.cn(np.random.default_rng(84), (2, N)).astype(np.complex64)
    p = api.Plan(N, p0=-8, nbins=16, max_batch=2)
    got = p.ndft(dev(x)).cpu().numpy()
    p.query_error()
    assert relerr(got, oracle.ndft(x, p0=-8, nbins=16)) < TOL


@pytest.mark.parametrize("form,prec", [("direct", "fp32"), ("ternary", "bf16x2"), ("direct", "q14")])
def test_empty_batch(api, form, prec):
    p = api.Plan(64, max_batch=8, form=form, prec=prec)
    dt = torch.int16 if prec == "q14" else torch.complex64
    x = torch.zeros((0, 64, 2) if prec == "q14" else (0, 64), dtype=dt, device="cuda")
    out = p.ndft(x)
    p.query_error()
    assert out.shape[0] == 0
    assert p.last_launches() == 0


@pytest.mark.parametrize("form,prec", [("direct", "fp32"), ("ternary", "bf16x2"), ("nfft", "fp32"),
                                       ("fft", "fp32")])
def test_lags_outside_the_samples_give_exact_zeros(api, form, prec):
    """Every lag beyond N pairs s_surv with the zero outside [0, N) (Eq. 12a as
    read here), so z_l = s (x) 0 = 0 and the surface is exactly 0."""
    N = 1024
    rng = np.random.default_rng(82)
    ss = dev(scenes.cn(rng, (N,)).astype(np.complex64))
    sr = dev(scenes.cn(rng, (N,)).astype(np.complex64))
    p = api.Plan(N, p0=-16, nbins=32, max_lags=40, form=form, prec=prec)
    A = p.caf(ss, sr, N, 40).cpu().numpy()
    p.query_error()
    assert np.all(A == 0)
    B = p.caf(ss, sr, -N - 5, 3).cpu().numpy()
    assert np.all(B == 0)


I32_MAX, I32_MIN = 2**31 - 1, -2**31


@pytest.mark.parametrize("form,prec", [("direct", "fp32"), ("ternary", "bf16x2"), ("nfft", "fp32"),
                                       ("fft", "fp32")])
def test_lag_windows_at_the_int32_limits(api, form, prec):
    """Windows ending at INT32_MAX or starting at INT32_MIN: without
    F_CIRCULAR_LAG the surface is exactly 0; with it the lags reduce modulo N
    and the surface equals the one at the reduced window.  A window one lag
    past INT32_MAX is an argument error."""
    from paper_1402_0532_gb300 import _lib as L
    N, nl = 1024, 4
    rng = np.random.default_rng(84)
    ss = dev(scenes.cn(rng, (N,)).astype(np.complex64))
    sr = dev(scenes.cn(rng, (N,)).astype(np.complex64))
    for lag0 in (I32_MAX - nl + 1, I32_MIN):
        p = api.Plan(N, p0=-16, nbins=32, max_lags=nl, form=form, prec=prec)
        assert torch.count_nonzero(p.caf(ss, sr, lag0, nl)).item() == 0
        pc = api.Plan(N, p0=-16, nbins=32, max_lags=nl, form=form, prec=prec, flags=api.F_CIRCULAR_LAG)
        got = pc.caf(ss, sr, lag0, nl).cpu().numpy()
        ref = pc.caf(ss, sr, lag0 % N, nl).cpu().numpy()  # lag0 % N + nl <= N: no wrap inside
        pc.query_error()
        assert relerr(got, ref) < 1e-6
    A = torch.zeros(nl * 32, dtype=torch.complex64, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    st = p.lib.caf_exec(p.handle, ctypes.c_void_p(ss.data_ptr()), ctypes.c_void_p(sr.data_ptr()), I32_MAX - nl + 2,
                        nl, ctypes.c_void_p(A.data_ptr()), s)
    assert st == L.E_INVALID


@pytest.mark.parametrize("form,prec", [("direct", "fp32"), ("ternary", "bf16x2")])
def test_adjoints_at_the_int32_lag_limits(api, form, prec):
    """Both gradients at a circular window ending at INT32_MAX against the
    oracle (which takes lags as int64), and exact zeros without wrap."""
    N, nl, p0, nbins = 512, 3, -7, 16
    lag0 = I32_MAX - nl + 1
    rng = np.random.default_rng(85)
    ss = scenes.cn(rng, (N,)).astype(np.complex64)
    sr = scenes.cn(rng, (N,)).astype(np.complex64)
    dA = scenes.cn(rng, (nl, nbins)).astype(np.complex64)
    p = api.Plan(N, p0=p0, nbins=nbins, max_lags=nl, form=form, prec=prec)
    gs, gr = p.caf_backward_inputs(dev(ss), dev(sr), lag0, nl, dev(dA))
    assert torch.count_nonzero(gs).item() == 0 and torch.count_nonzero(gr).item() == 0
    f = api.F_CIRCULAR_LAG
    pc = api.Plan(N, p0=p0, nbins=nbins, max_lags=nl, form=form, prec=prec, flags=f)
    gs, gr = pc.caf_backward_inputs(dev(ss), dev(sr), lag0, nl, dev(dA))
    pc.query_error()
    assert relerr(gs.cpu().numpy(), oracle.caf_adjoint(ss, sr, lag0, nl, p0, nbins, dA, flags=f)) < TOL
    assert relerr(gr.cpu().numpy(), oracle.caf_adjoint_ref(ss, sr, lag0, nl, p0, nbins, dA, flags=f)) < TOL


@pytest.mark.parametrize("form,prec", [("direct", "fp32"), ("ternary", "bf16x2")])
def test_single_lag_and_adjoints(api, form, prec):
    N, lag0, p0, nbins = 777, -5, -3, 9
    rng = np.random.default_rng(83)
    ss = scenes.cn(rng, (N,)).astype(np.complex64)
    sr = scenes.cn(rng, (N,)).astype(np.complex64)
    dA = scenes.cn(rng, (1, nbins)).astype(np.complex64)
    p = api.Plan(N, p0=p0, nbins=nbins, max_lags=1, form=form, prec=prec)
    A = p.caf(dev(ss), dev(sr), lag0, 1).cpu().numpy()
    assert relerr(A, oracle.caf(ss, sr, lag0, 1, p0, nbins, z32=True)) < TOL
    gs, gr = p.caf_backward_inputs(dev(ss), dev(sr), lag0, 1, dev(dA))
    p.query_error()
    assert relerr(gs.cpu().numpy(), oracle.caf_adjoint(ss, sr, lag0, 1, p0, nbins, dA)) < TOL
    assert relerr(gr.cpu().numpy(), oracle.caf_adjoint_ref(ss, sr, lag0, 1, p0, nbins, dA)) < TOL
    # a lag beyond the samples: no sample meets s_ref, both gradients are exactly 0
    gs, gr = p.caf_backward_inputs(dev(ss), dev(sr), N + 1, 1, dev(dA))
    assert torch.count_nonzero(gs).item() == 0 and torch.count_nonzero(gr).item() == 0


def test_n1_both_forms(api):
    """N = 1: W = 1, the NDFT is x (x) 1 and the CAF at lag 0 is (s (x) conj r) (x) 1."""
    x = np.array([[0.5 - 2.0j], [0.0 + 0.0j], [-3.0 + 0.25j]], np.complex64)
    for form, prec in (("direct", "fp32"), ("ternary", "bf16x2")):
        p = api.Plan(1, max_batch=3, form=form, prec=prec)
        got = p.ndft(dev(x)).cpu().numpy()
        p.query_error()
        assert relerr(got, oracle.ndft(x)) < TOL


def test_outputs_aliasing_inputs_are_rejected(api):
    """Outputs that start at an input's address are argument errors: nothing launches."""
    from paper_1402_0532_gb300 import _lib as L
    N = 256
    lib = L.load()
    p = api.Plan(N, p0=-4, nbins=8, max_lags=4, max_batch=4, form="ternary", prec="bf16x2")
    x = torch.zeros(4 * N, dtype=torch.complex64, device="cuda")
    y = torch.zeros(4 * N, dtype=torch.complex64, device="cuda")
    dA = torch.zeros(4 * 8, dtype=torch.complex64, device="cuda")
    ptr = lambda t: ctypes.c_void_p(t.data_ptr())  # noqa: E731
    s = torch.cuda.current_stream().cuda_stream
    assert lib.ndft_exec(p.handle, ptr(x), ptr(x), 4, s) == L.E_INVALID
    assert lib.caf_exec(p.handle, ptr(x), ptr(y), 0, 4, ptr(x), s) == L.E_INVALID
    assert lib.caf_exec(p.handle, ptr(x), ptr(y), 0, 4, ptr(y), s) == L.E_INVALID
    assert lib.caf_backward(p.handle, ptr(x), ptr(y), 0, 4, ptr(dA), ptr(y), s) == L.E_INVALID
    assert lib.caf_backward_inputs(p.handle, ptr(x), ptr(y), 0, 4, ptr(dA), ptr(dA), ptr(x), s) == L.E_INVALID
    out = torch.zeros(4 * N, dtype=torch.complex64, device="cuda")
    assert lib.caf_backward_inputs(p.handle, ptr(x), ptr(y), 0, 4, ptr(dA), ptr(out), ptr(out), s) == L.E_INVALID
    p.query_error()
