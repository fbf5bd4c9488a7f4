"""Exec calls allocate nothing and never synchronise, so a CUDA graph can
capture them: for every form (and the backward calls), a captured call
replayed on new inputs gives the eager call's result bit for bit."""
import numpy as np
import pytest

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


def capture(fn):
    """Warm up on a side stream (kernel attributes are set outside the capture), then capture."""
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        fn()
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        fn()
    return g


@pytest.mark.parametrize("form,prec,tile", [("direct", "fp32", 0), ("ternary", "bf16x2", 0),
                                            ("ternary", "bf16x2", 258), ("nfft", "fp32", 0),
                                            ("fft", "fp32", 0), ("direct", "q14", 0)])
def test_caf_in_a_graph(api, form, prec, tile):
    N, nlags, nbins = 8192, 80, 96
    plan = api.Plan(N, p0=-48, nbins=nbins, max_lags=nlags, form=form, prec=prec)
    if tile:
        plan.set_tuning(1, tile)
    q14 = prec == "q14"

    def inputs(seed):
        sc = scenes.radar_scene(N=N, nlags=nlags, nbins=nbins, seed=seed)
        if q14:
            return (torch.from_numpy(scenes.quantize_q14(sc.s_surv, 0.25)).cuda(),
                    torch.from_numpy(scenes.quantize_q14(sc.s_ref, 0.25)).cuda())
        return torch.from_numpy(sc.s_surv).cuda(), torch.from_numpy(sc.s_ref).cuda()
    ss, sr = inputs(100)
    A = torch.empty((nlags, nbins, 2) if q14 else (nlags, nbins), dtype=torch.int32 if q14 else torch.complex64,
                    device="cuda")
    g = capture(lambda: plan.caf(ss, sr, 3, nlags, out=A))
    for seed in (101, 102):
        s2, r2 = inputs(seed)
        ss.copy_(s2)
        sr.copy_(r2)
        g.replay()
        torch.cuda.synchronize()
        want = plan.caf(s2, r2, 3, nlags).cpu().numpy()
        assert np.array_equal(A.cpu().numpy(), want)
    plan.query_error()


@pytest.mark.parametrize("tile", [0, 258])
def test_two_part_caf_in_a_graph(api, tile):
    """A tensor-core call of 600 lags as two column parts (key 5 = 0), the second
    part's packing on the plan's side stream (forked from and joined back into
    the capturing stream): the captured call replays the eager result bit for bit."""
    N, nlags, nbins = 8192, 600, 64
    plan = api.Plan(N, p0=-32, nbins=nbins, max_lags=nlags, form="ternary", prec="bf16x2")
    plan.set_tuning(5, 0)
    if tile:
        plan.set_tuning(1, tile)

    def inputs(seed):
        sc = scenes.radar_scene(N=N, nlags=nlags, nbins=nbins, seed=seed)
        return torch.from_numpy(sc.s_surv).cuda(), torch.from_numpy(sc.s_ref).cuda()
    ss, sr = inputs(110)
    A = torch.empty((nlags, nbins), dtype=torch.complex64, device="cuda")
    g = capture(lambda: plan.caf(ss, sr, -5, nlags, out=A))
    for seed in (111, 112):
        s2, r2 = inputs(seed)
        ss.copy_(s2)
        sr.copy_(r2)
        g.replay()
        torch.cuda.synchronize()
        want = plan.caf(s2, r2, -5, nlags).cpu().numpy()
        assert np.array_equal(A.cpu().numpy(), want)
    assert plan.last_launches() == 6  # two parts: packing, contraction, ordered split-K sum each
    plan.query_error()


@pytest.mark.parametrize("form,prec", [("direct", "fp32"), ("ternary", "bf16x2")])
def test_backward_in_a_graph(api, form, prec):
    N, nlags, nbins = 4096, 64, 64
    plan = api.Plan(N, p0=-32, nbins=nbins, max_lags=nlags, form=form, prec=prec)
    rng = np.random.default_rng(103)
    ss = torch.from_numpy(scenes.cn(rng, (N,)).astype(np.complex64)).cuda()
    sr = torch.from_numpy(scenes.cn(rng, (N,)).astype(np.complex64)).cuda()
    dA = torch.from_numpy(scenes.cn(rng, (nlags, nbins)).astype(np.complex64)).cuda()
    ds = torch.empty(N, dtype=torch.complex64, device="cuda")
    res = {}

    def step():
        plan.caf_backward(ss, sr, 0, nlags, dA, out=ds)
        res["both"] = plan.caf_backward_inputs(ss, sr, 0, nlags, dA)
    g = capture(step)
    dA.copy_(torch.from_numpy(scenes.cn(rng, (nlags, nbins)).astype(np.complex64)))
    g.replay()
    torch.cuda.synchronize()
    want = plan.caf_backward(ss, sr, 0, nlags, dA).cpu().numpy()
    ws, wr = plan.caf_backward_inputs(ss, sr, 0, nlags, dA)
    assert np.array_equal(ds.cpu().numpy(), want)
    assert np.array_equal(res["both"][0].cpu().numpy(), ws.cpu().numpy())
    assert np.array_equal(res["both"][1].cpu().numpy(), wr.cpu().numpy())
    plan.query_error()


def test_nfft_and_ndft_in_a_graph(api):
    x = torch.from_numpy(scenes.cn_batch(batch=512, N=4096)).cuda()
    pn = api.Plan(4096, max_batch=512)
    pt = api.Plan(4096, p0=-64, nbins=128, max_batch=512, form="ternary", prec="bf16x2")
    y = torch.empty_like(x)
    z = torch.empty(512, 128, dtype=torch.complex64, device="cuda")

    def step():
        pn.nfft(x, out=y)
        pt.ndft(x, out=z)
    g = capture(step)
    x.copy_(torch.from_numpy(scenes.cn_batch(batch=512, N=4096, seed=7)))
    g.replay()
    torch.cuda.synchronize()
    assert np.array_equal(y.cpu().numpy(), pn.nfft(x).cpu().numpy())
    assert np.array_equal(z.cpu().numpy(), pt.ndft(x).cpu().numpy())


def test_autograd_forward_backward_in_a_graph(api):
    """The differentiation workload (Eq. 12a forward, loss sum |A| over a mask,
    backward through CafFunction) captured once and replayed: the gradient
    equals the eager one bit for bit."""
    sc = scenes.radar_scene(N=4096, seed=4, nlags=128, nbins=128)
    plan = api.Plan(sc.N, p0=sc.p0, nbins=128, max_lags=128, form="ternary", prec="bf16x2")
    mask = torch.from_numpy(scenes.differentiation_mask(sc).astype(np.float32)).cuda()
    sr = torch.from_numpy(sc.s_ref).cuda()
    s = torch.from_numpy(sc.s_surv).cuda().requires_grad_(True)

    def step():
        s.grad = None
        (api.caf_autograd(s, sr, plan, 0, 128).abs() * mask).sum().backward()
    step()
    eager = s.grad.detach().clone()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        step()
    torch.cuda.current_stream().wait_stream(side)
    s.grad = None
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        (api.caf_autograd(s, sr, plan, 0, 128).abs() * mask).sum().backward()
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(s.grad, eager)
    plan.query_error()
