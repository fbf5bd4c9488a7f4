"""The 2-SM pair tile of the tensor-core form (tcgen05 cta_group::2, tuning key
1 = 258): the same units, chains and fold order as the one-CTA 256-row tile
with one row pair per bin (tuning key 6 = 1), so with the same split of the
sample axis the surface is bit-identical to it; and within the fp32 bar of the
oracle."""
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


@pytest.mark.parametrize("N,nlags,nbins,split", [(9000, 300, 200, 3), (4133, 257, 96, 1), (2048, 64, 77, 2),
                                                 (700, 70, 40, 1)])
def test_pair_tile_bit_identical_caf(api, N, nlags, nbins, split):
    sc = scenes.radar_scene(N=N, nlags=nlags, nbins=nbins, seed=47 + N % 5)
    out = []
    for tile in (256, 258):
        p = api.Plan(N, p0=sc.p0, nbins=nbins, max_lags=nlags, form="ternary", prec="bf16x2")
        p.set_tuning(0, split)
        p.set_tuning(1, tile)
        p.set_tuning(6, 1)  # one row pair per bin on both tiles: the pair tile has no conjugate pairing
        out.append(p.caf(dev(sc.s_surv), dev(sc.s_ref), 0, nlags).cpu().numpy())
        p.query_error()
    assert np.array_equal(out[0], out[1])
    lags = np.array([0, nlags - 1, 37 % nlags, 5])
    bins = np.array([0, sc.p0, sc.p0 + nbins - 1, 5])
    ref = oracle.caf_cells(sc.s_surv, sc.s_ref, lags, bins, z32=True)
    assert np.max(np.abs(out[1][lags, bins - sc.p0] - ref)) / np.max(np.abs(out[1])) < TOL


def test_pair_tile_ndft_and_default_split(api):
    """A batched NDFT with ragged bins on the pair tile (automatic split), against the oracle."""
    x = scenes.cn(np.random.default_rng(48), (300, 100)).astype(np.complex64)
    q = api.Plan(100, p0=-7, nbins=77, max_batch=300, form="ternary", prec="bf16x2")
    q.set_tuning(1, 258)
    got = q.ndft(dev(x)).cpu().numpy()
    q.query_error()
    assert relerr(got, oracle.ndft(x.astype(np.complex128), p0=-7, nbins=77)) < TOL


def test_pair_tile_bounded_waits(api):
    """With the operand loads starved every wait of both CTAs runs out, the
    kernel returns NDFT_E_TIMEOUT, and the plan then reproduces its surface."""
    import time
    from paper_1402_0532_gb300 import _lib as L
    sc = scenes.radar_scene(N=4096, nlags=256, nbins=256, seed=49)
    p = api.Plan(4096, p0=sc.p0, nbins=256, max_lags=256, form="ternary", prec="bf16x2")
    p.set_tuning(1, 258)
    ss, sr = dev(sc.s_surv), dev(sc.s_ref)
    want = p.caf(ss, sr, 0, 256).cpu().numpy()
    p.query_error()
    p.set_tuning(4, 1)
    t0 = time.time()
    p.caf(ss, sr, 0, 256)
    with pytest.raises(L.NdftError) as e:
        p.query_error()
    assert e.value.status == L.E_TIMEOUT
    assert time.time() - t0 < 30
    p.set_tuning(4, 0)
    got = p.caf(ss, sr, 0, 256).cpu().numpy()
    p.query_error()
    assert np.array_equal(got, want)
