"""Differentiation workload: forward + backward through torch.autograd.Function.

N = 16384, 512 lags x 512 Doppler bins (-256..255), the radar scene with seed 4,
loss = sum of |A| over the 32 x 32 mask centred on the first echo (lags
21..52, bins -11..20).  The gradient with respect to s_surv is checked
against the fp64 oracle's gradient and against central finite differences of
the fp64 forward, with a step below every distance to a zero crossing."""
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


@pytest.fixture(scope="module")
def scene():
    return scenes.radar_scene(N=16384, seed=4, nlags=512, nbins=512)


@pytest.mark.parametrize("form,prec", [("direct", "fp32"), ("ternary", "bf16x2")])
def test_autograd_matches_oracle_gradient(api, scene, form, prec):
    sc = scene
    mask = scenes.differentiation_mask(sc)
    assert mask.sum() == 32 * 32
    rows, cols = np.nonzero(mask)
    l0, l1, b0, b1 = rows.min(), rows.max() + 1, cols.min(), cols.max() + 1
    assert (l0 + sc.lag0, l1 - 1 + sc.lag0, b0 + sc.p0, b1 - 1 + sc.p0) == (21, 52, -11, 20)

    plan = api.Plan(sc.N, p0=sc.p0, nbins=sc.nbins, max_lags=sc.nlags, form=form, prec=prec)
    ss = torch.from_numpy(sc.s_surv).cuda().requires_grad_(True)
    sr = torch.from_numpy(sc.s_ref).cuda()
    A = api.caf_autograd(ss, sr, plan, sc.lag0, sc.nlags)
    m = torch.from_numpy(mask).cuda()
    loss = A.abs()[m].sum()
    loss.backward()
    g = ss.grad.cpu().numpy().astype(np.complex128)
    plan.query_error()

    # fp64 oracle: forward on the mask cells, then the adjoint over the mask rectangle
    L = np.arange(l0, l1) + sc.lag0
    P = np.arange(b0, b1) + sc.p0
    LL, PP = np.meshgrid(L, P, indexing="ij")
    Am = oracle.caf_cells(sc.s_surv, sc.s_ref, LL.ravel(), PP.ravel()).reshape(LL.shape)
    Lref, gA = oracle.masked_abs_loss_grad(Am, np.ones(Am.shape, bool))
    want = oracle.caf_adjoint(sc.s_surv, sc.s_ref, int(L[0]), L.size, int(P[0]), P.size, gA)
    assert abs(float(loss) - Lref) < 1e-4 * Lref
    assert np.max(np.abs(g - want)) < 1e-4 * np.max(np.abs(want))


def test_gradient_against_finite_differences(api, scene):
    """Central differences of the fp64 forward at sampled coordinates, each step
    below a quarter of the distance of s_surv[i] and of every z_l[i] (mask lags)
    to 0, so no operand of (x) changes sign inside the stencil."""
    sc = scene
    mask = scenes.differentiation_mask(sc)
    rows, cols = np.nonzero(mask)
    L = np.arange(rows.min(), rows.max() + 1) + sc.lag0
    P = np.arange(cols.min(), cols.max() + 1) + sc.p0
    LL, PP = np.meshgrid(L, P, indexing="ij")

    plan = api.Plan(sc.N, p0=sc.p0, nbins=sc.nbins, max_lags=sc.nlags)
    ss = torch.from_numpy(sc.s_surv).cuda().requires_grad_(True)
    sr = torch.from_numpy(sc.s_ref).cuda()
    A = api.caf_autograd(ss, sr, plan, sc.lag0, sc.nlags)
    A.abs()[torch.from_numpy(mask).cuda()].sum().backward()
    g = ss.grad.cpu().numpy()

    s64 = sc.s_surv.astype(np.complex128)
    zs = np.stack([oracle.lagprod(s64, sc.s_ref, int(l)) for l in L])

    def loss(s):
        return float(np.abs(oracle.caf_cells(s, sc.s_ref, LL.ravel(), PP.ravel())).sum())

    rng = np.random.default_rng(44)
    cand = rng.choice(np.arange(60, sc.N), 400, replace=False)
    checked = 0
    for i in cand:
        zi = zs[:, i]
        margin = min(abs(s64[i].real), abs(s64[i].imag), np.abs(zi.real).min(), np.abs(zi.imag).min())
        h = min(0.25 * margin, 1e-3)
        if h < 1e-6:
            continue
        for comp, unit in ((0, 1.0), (1, 1j)):
            sp, sm = s64.copy(), s64.copy()
            sp[i] += h * unit
            sm[i] -= h * unit
            fd = (loss(sp) - loss(sm)) / (2 * h)
            an = g[i].real if comp == 0 else g[i].imag
            assert abs(fd - an) <= 1e-3 * max(1.0, abs(fd)), (i, comp, fd, an)
            checked += 1
        if checked >= 64:
            break
    assert checked >= 64
