"""GPU parity of caf_backward_inputs (both gradients of the nonlinear ambiguity
surface, Eq. 12a, through the derivative of Eq. 1-2) against the fp64 oracle.

G_l[i] = sum_p conj(S[p][i]) dA[l][p] is formed once (tcgen05 on the ternary
form: dA as bf16 hi + lo against exact signs, fp32 accumulation; CUDA cores on
the direct form) and folded into dL/ds_surv and dL/ds_ref by a deterministic
kernel.  The bar is the fp32 one, 1e-5 of max |gradient|; the signs sigma(.)
of the inputs are taken from the same fp32 values on both sides."""
import numpy as np
import pytest

import oracle
from paper_1402_0532_gb300 import scenes

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

TOL = 1e-5
FORMS = [("direct", "fp32"), ("ternary", "bf16x2")]


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


def inputs(N, nlags, nbins, seed):
    rng = np.random.default_rng(seed)
    ss = scenes.cn(rng, (N,)).astype(np.complex64)
    sr = scenes.cn(rng, (N,)).astype(np.complex64)
    dA = scenes.cn(rng, (nlags, nbins)).astype(np.complex64)
    return ss, sr, dA


@pytest.mark.parametrize("form,prec", FORMS)
@pytest.mark.parametrize("N,lag0,nlags,p0,nbins,flags", [
    (700, 2, 70, -20, 40, 0),        # ragged tiles everywhere
    (4133, -3, 300, -48, 96, 0),     # odd N (per-element stores), negative lag0, two lag tiles
    (2048, 10, 257, 0, 512, 1),      # no conjugate of s_ref; 257 lags: a 1-lag tail tile
    (1500, 1400, 33, -7, 17, 2),     # circular lag beyond N/2
    (20000, -1000, 40, 3, 1300, 3),  # both flags; 157 m-tiles (no split) and 82 K blocks: two chains
])
def test_both_gradients_against_oracle(api, form, prec, N, lag0, nlags, p0, nbins, flags):
    ss, sr, dA = inputs(N, nlags, nbins, 60 + N % 11)
    want_s = oracle.caf_adjoint(ss, sr, lag0, nlags, p0, nbins, dA, flags=flags)
    want_r = oracle.caf_adjoint_ref(ss, sr, lag0, nlags, p0, nbins, dA, flags=flags)
    p = api.Plan(N, p0=p0, nbins=nbins, max_lags=nlags, flags=flags, form=form, prec=prec)
    gs, gr = p.caf_backward_inputs(dev(ss), dev(sr), lag0, nlags, dev(dA))
    p.query_error()
    gs, gr = gs.cpu().numpy(), gr.cpu().numpy()
    assert relerr(gr, want_r) < TOL
    assert relerr(gs, want_s) < TOL
    # G is formed once: pack + contraction (ternary), or per lag chunk that the
    # workspace holds one CUDA-core kernel; then one fold per chunk
    n = p.last_launches()
    assert n == 3 if form == "ternary" else (n >= 2 and n % 2 == 0)
    # the ref-only call gives the same ds_ref bit for bit, and is deterministic
    none, gr2 = p.caf_backward_inputs(dev(ss), dev(sr), lag0, nlags, dev(dA), surv=False)
    assert none is None
    assert np.array_equal(gr2.cpu().numpy(), gr)
    # ds_surv agrees with the fused caf_backward to rounding
    gs1 = p.caf_backward(dev(ss), dev(sr), lag0, nlags, dev(dA)).cpu().numpy()
    assert relerr(gs1, want_s) < TOL


def test_lag_chunks_direct(api):
    """A direct plan whose workspace holds G for a single lag: the adjoint runs
    in 40 chunks of one lag, each fold adding to the previous chunks."""
    N, lag0, nlags, p0, nbins = 20000, -5, 40, -4, 8
    ss, sr, dA = inputs(N, nlags, nbins, 71)
    p = api.Plan(N, p0=p0, nbins=nbins, max_lags=nlags)
    gs, gr = p.caf_backward_inputs(dev(ss), dev(sr), lag0, nlags, dev(dA))
    p.query_error()
    assert p.last_launches() == 2 * nlags
    assert relerr(gr.cpu().numpy(), oracle.caf_adjoint_ref(ss, sr, lag0, nlags, p0, nbins, dA)) < TOL
    assert relerr(gs.cpu().numpy(), oracle.caf_adjoint(ss, sr, lag0, nlags, p0, nbins, dA)) < TOL


def test_full_size_sampled(api):
    """The surface of N = 65536 samples, 1024 lags x 1024 bins on the tensor
    cores: both gradients at 48 sampled indices (first and last samples
    included) against the oracle evaluated at those indices only."""
    N, lag0, nlags, p0, nbins = 65536, 0, 1024, -512, 1024
    sc = scenes.radar_scene(N=N, seed=8, nlags=nlags, nbins=nbins)
    rng = np.random.default_rng(12)
    dA = (scenes.cn(rng, (nlags, nbins)) * 1e-3).astype(np.complex64)
    p = api.Plan(N, p0=p0, nbins=nbins, max_lags=nlags, form="ternary", prec="bf16x2")
    gs, gr = p.caf_backward_inputs(dev(sc.s_surv), dev(sc.s_ref), lag0, nlags, dev(dA))
    p.query_error()
    gs, gr = gs.cpu().numpy(), gr.cpu().numpy()
    idx = np.concatenate([[0, 1, N - 1024, N - 1], rng.choice(N, 44, replace=False)])
    ws = oracle.caf_adjoint_at(sc.s_surv, sc.s_ref, lag0, nlags, p0, nbins, dA, "surv", idx)
    wr = oracle.caf_adjoint_at(sc.s_surv, sc.s_ref, lag0, nlags, p0, nbins, dA, "ref", idx)
    assert relerr(gs[idx], ws) < TOL
    assert relerr(gr[idx], wr) < TOL
    # the last nlags - 1 samples of s_ref meet fewer lags; the very last meets lag 0 only
    assert np.all(np.isfinite(gr)) and np.abs(gr[-1]) < np.abs(gr).max()


@pytest.mark.parametrize("form,prec", FORMS)
def test_autograd_wrt_both_inputs(api, form, prec):
    """torch.autograd through CafFunction with requires_grad on s_ref (and on
    both): the loss of the differentiation workload, against the oracle."""
    N, nlags, nbins = 4096, 128, 128
    sc = scenes.radar_scene(N=N, seed=5, nlags=nlags, nbins=nbins)
    plan = api.Plan(N, p0=sc.p0, nbins=nbins, max_lags=nlags, form=form, prec=prec)
    mask = scenes.differentiation_mask(sc)
    for both in (False, True):
        ss = torch.from_numpy(sc.s_surv).cuda().requires_grad_(both)
        sr = torch.from_numpy(sc.s_ref).cuda().requires_grad_(True)
        A = api.caf_autograd(ss, sr, plan, sc.lag0, nlags)
        m = torch.from_numpy(mask).cuda()
        A.abs()[m].sum().backward()
        plan.query_error()
        A64 = oracle.caf(sc.s_surv, sc.s_ref, sc.lag0, nlags, sc.p0, nbins)
        _, gA = oracle.masked_abs_loss_grad(A64, mask)
        want_r = oracle.caf_adjoint_ref(sc.s_surv, sc.s_ref, sc.lag0, nlags, sc.p0, nbins, gA)
        assert relerr(sr.grad.cpu().numpy(), want_r) < 1e-4
        if both:
            want_s = oracle.caf_adjoint(sc.s_surv, sc.s_ref, sc.lag0, nlags, sc.p0, nbins, gA)
            assert relerr(ss.grad.cpu().numpy(), want_s) < 1e-4
        else:
            assert ss.grad is None
