"""GPU parity of the conjugate-paired tensor-core contraction.

W^(-c i) = conj(W^(c i)) (Eq. 8) and sigma(conj w) = conj(sigma(w)) (Eq. 2),
so bins +c and -c of the NDFT come from one pair of real contractions,
U = S_r v + F_r sigma(v) and V = S_i v + F_i sigma(v): X[+c] = U + jV,
X[-c] = U - jV; bin 0 is the packing kernel's sum of v + sigma(v).  Every case
is checked against the fp64 oracle at the fp32 bar (1e-5 of max |X|), with the
paired path forced (tuning key 6 = 2; its A operand from the plan's table on
the 2-SM pair tile, the default, or on the one-CTA tile, key 1 = 256, or
generated on chip, key 7 = 1; its B operand packed by a kernel, formed inside
the pair tile (key 8 = 2) or packed by the pair tile's own warps ahead of its
loads (key 8 = 3)) and cross-checked against the unpaired rows (key 6 = 1) on the
same inputs: centred and full windows, windows that
wrap past bin 0, contain N/2 or give an odd number of paired frequencies (the
element-wise fold-out), ragged N, both CAF flags and several sample-axis
splits."""
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


# (key 6, key 7, key 1, key 8) -> tile: paired with A from the table on the
# 2-SM pair (default), the same with B formed in the tile or packed ahead by
# it, A from the table on one CTA, A generated on chip; unpaired
COMBOS = ((2, 0, 0, 1), (2, 0, 0, 2), (2, 0, 0, 3), (2, 0, 256, 0), (2, 1, 0, 0), (1, 0, 0, 0))
TILE = {(2, 0, 0, 1): 258, (2, 0, 0, 2): 258, (2, 0, 0, 3): 258, (2, 0, 256, 0): 256, (2, 1, 0, 0): 256,
        (1, 0, 0, 0): 256}


def configure(p, key, atab, tile, bgen):
    p.set_tuning(6, key)
    p.set_tuning(7, atab)
    p.set_tuning(1, tile)
    p.set_tuning(8, bgen)


def bin0_index(N, p0, nbins):
    """Index of bin 0 (frequency 0) in the window, or None."""
    k = (-p0) % N
    return k if k < nbins else None


def slots(N, p0, nbins):
    p = (p0 + np.arange(nbins)) % N
    return int(np.max(np.minimum(p, N - p)))


@pytest.mark.parametrize("N,batch,p0,nbins", [
    (64, 300, 0, 0),          # full window, N/2 self-conjugate
    (1024, 600, 0, 0),
    (1000, 77, -500, 1000),   # centred, even N
    (999, 40, -499, 999),     # centred, odd N (no N/2 bin)
    (100, 130, -7, 77),       # asymmetric: N/2 inside, most bins unpaired
    (4133, 9, 4128, 20),      # wraps past bin 0
    (300, 33, -15, 31),       # odd slot count: element-wise fold-out
    (4, 5, 0, 0), (2, 3, 0, 0), (3, 7, 0, 0),
])
def test_paired_ndft(api, N, batch, p0, nbins):
    rng = np.random.default_rng(60 + N)
    x = scenes.cn(rng, (batch, N)).astype(np.complex64)
    x[:, ::7] = 0
    if batch > 2:
        x[1, :] = 0
    nb = nbins or N
    ref = oracle.ndft(x.astype(np.complex128), p0=p0, nbins=nb)
    outs = {}
    for combo in COMBOS:
        p = api.Plan(N, p0=p0, nbins=nbins, max_batch=batch, form="ternary", prec="bf16x2")
        assert p.query(0) == slots(N, p0, nb)
        configure(p, *combo)
        got = p.ndft(dev(x)).cpu().numpy()
        p.query_error()
        assert p.query(1) == (2 if combo[0] == 2 else 1)
        assert p.query(3) == TILE[combo]
        assert relerr(got, ref) < TOL, combo
        outs[combo] = got
    for combo in COMBOS[1:]:
        assert np.max(np.abs(outs[COMBOS[0]] - outs[combo])) / np.max(np.abs(ref)) < 2 * TOL, combo
    # B formed in the tile or packed ahead by it: the same operand as the
    # packing kernel's, so every bin but 0 (whose sum is grouped per split or
    # per item instead of per packing tile) is the same to the bit
    same = np.ones(nb, bool)
    k0 = bin0_index(N, p0, nb)
    if k0 is not None:
        same[k0] = False
    a = np.ascontiguousarray(outs[(2, 0, 0, 1)][:, same])
    for bmode in (2, 3):
        b = np.ascontiguousarray(outs[(2, 0, 0, bmode)][:, same])
        assert np.array_equal(a.view(np.uint32), b.view(np.uint32)), bmode


@pytest.mark.parametrize("N,lag0,nlags,p0,nbins,flags", [
    (4133, -3, 100, -48, 96, 0),
    (700, 650, 40, -16, 33, 1),
    (700, 650, 40, -16, 33, 2),
    (2048, 0, 300, -1024, 2048, 0),   # every bin of N, lags in two n-tiles
    (513, -600, 3, 250, 20, 0),       # lags entirely before the samples: exact zeros
])
def test_paired_caf(api, N, lag0, nlags, p0, nbins, flags):
    sc = scenes.radar_scene(N=N, nlags=min(nlags, 64), nbins=min(nbins, 64), seed=61 + N % 97)
    ref = oracle.caf(sc.s_surv, sc.s_ref, lag0, nlags, p0, nbins, flags=flags, z32=True)
    outs = {}
    for combo in COMBOS:
        p = api.Plan(N, p0=p0, nbins=nbins, max_lags=nlags, flags=flags, form="ternary", prec="bf16x2")
        configure(p, *combo)
        got = p.caf(dev(sc.s_surv), dev(sc.s_ref), lag0, nlags).cpu().numpy()
        p.query_error()
        assert p.query(1) == (2 if combo[0] == 2 else 1)
        assert p.query(3) == TILE[combo]
        if np.max(np.abs(ref)) == 0:
            assert np.max(np.abs(got)) == 0
        else:
            assert relerr(got, ref) < TOL, combo
        outs[combo] = got
    same = np.ones(nbins, bool)
    k0 = bin0_index(N, p0, nbins)
    if k0 is not None:
        same[k0] = False
    a = np.ascontiguousarray(outs[(2, 0, 0, 1)][:, same])
    for bmode in (2, 3):
        b = np.ascontiguousarray(outs[(2, 0, 0, bmode)][:, same])
        assert np.array_equal(a.view(np.uint32), b.view(np.uint32)), bmode


@pytest.mark.parametrize("split,atab,tile,bgen", [
    (0, 0, 0, 0), (1, 0, 0, 0), (3, 0, 0, 0), (19, 0, 0, 0), (0, 1, 0, 0), (19, 1, 0, 0),
    (0, 0, 256, 0), (3, 0, 256, 0), (19, 0, 256, 0), (7, 0, 258, 0),
    (0, 0, 0, 2), (1, 0, 0, 2), (5, 0, 0, 2), (19, 0, 0, 2),
    (0, 0, 0, 3), (1, 0, 0, 3), (5, 0, 0, 3), (8, 0, 0, 3), (19, 0, 0, 3)])
def test_paired_caf_splits_sampled(api, split, atab, tile, bgen):
    """The headline layout at N = 16384: 1024 lags x bins -512..511 (512 paired
    frequencies, bin 0 from the DC sums), every sample-axis split count giving
    the same cells within the bar; the default choice pairs."""
    sc = scenes.radar_scene(N=16384, nlags=1024, nbins=1024, seed=62)
    p = api.Plan(sc.N, p0=-512, nbins=1024, max_lags=1024, form="ternary", prec="bf16x2")
    assert p.query(0) == 512
    p.set_tuning(0, split)
    p.set_tuning(7, atab)  # 0: A tiles from the plan's table, 1: generated on chip
    p.set_tuning(1, tile)  # 0 / 258: the 2-SM pair tile with the table, 256: one CTA
    p.set_tuning(8, bgen)  # 2: B formed inside the pair tile, 3: packed ahead by it
    A = p.caf(dev(sc.s_surv), dev(sc.s_ref), 0, 1024)
    idx, _ = api.argmax(A.reshape(1, -1))
    got = A.cpu().numpy()
    p.query_error()
    assert p.query(1) == 2
    if split:
        assert p.query(2) == split
    rng = np.random.default_rng(63)
    lags = np.concatenate([[0, 0, 0, 37, 120, 301, 1023, 255, 256, 511, 512], rng.integers(0, 1024, 40)])
    bins = np.concatenate([[0, -512, 511, 5, -12, 40, -1, 1, -511, 255, -256], rng.integers(-512, 512, 40)])
    ref = oracle.caf_cells(sc.s_surv, sc.s_ref, lags, bins, z32=True)
    peak = np.max(np.abs(got))
    assert np.max(np.abs(got[lags, bins + 512] - ref)) / peak < TOL
    assert int(idx[0]) == 512  # the direct path at lag 0, bin 0


@pytest.mark.parametrize("bmode", [0, 1])
def test_paired_deterministic_and_graph(api, bmode):
    """Two calls give the same bits, and a CUDA-graph replay of the paired call
    on new inputs equals an eager call on them (B packed by a kernel, and packed
    just in time inside the pair tile, the default)."""
    sc = scenes.radar_scene(N=8192, nlags=256, nbins=512, seed=64)
    p = api.Plan(sc.N, p0=-256, nbins=512, max_lags=256, form="ternary", prec="bf16x2")
    p.set_tuning(8, bmode)
    ss, sr = dev(sc.s_surv), dev(sc.s_ref)
    a1 = p.caf(ss, sr, 0, 256).cpu().numpy()
    a2 = p.caf(ss, sr, 0, 256).cpu().numpy()
    assert p.query(1) == 2 and p.query(3) == 258  # the 2-SM pair tile, a cluster launch
    assert np.array_equal(a1.view(np.uint32), a2.view(np.uint32))
    out = torch.empty((256, 512), dtype=torch.complex64, device="cuda")
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        p.caf(ss, sr, 0, 256, out=out)  # warm-up on the capture stream
    torch.cuda.current_stream().wait_stream(s)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        p.caf(ss, sr, 0, 256, out=out)
    sc2 = scenes.radar_scene(N=8192, nlags=256, nbins=512, seed=65)
    ss.copy_(dev(sc2.s_surv))
    sr.copy_(dev(sc2.s_ref))
    g.replay()
    torch.cuda.synchronize()
    want = p.caf(ss, sr, 0, 256).cpu().numpy()
    assert np.array_equal(out.cpu().numpy().view(np.uint32), want.view(np.uint32))


@pytest.mark.parametrize("N,lag0,nlags,p0,nbins,flags", [
    (4133, -3, 100, -48, 96, 0),      # centred window, ragged sample tile
    (700, 650, 40, -16, 33, 1),       # odd window, no conjugation
    (700, 650, 40, -16, 33, 2),       # circular lags
    (1024, 0, 300, 0, 1024, 0),       # every bin of N (N/2 self-conjugate), lags over two column tiles
    (999, 2, 37, 100, 60, 0),         # asymmetric window: most frequencies have one bin only
])
def test_paired_adjoint(api, N, lag0, nlags, p0, nbins, flags):
    """The adjoint contraction with conjugate pairing: W^(-c i) = conj(W^(c i))
    makes bins +c and -c of dA enter G as S_r u + ... with u, v = dA[+c] +- dA[-c]
    (one row per sample, half the multiply-adds); dL/ds_surv (the fused fold) and
    both gradients (G stored, then folded) against the fp64 oracle adjoints,
    forced on (key 6 = 2; the sign rows from the plan's table for one or both
    contractions, key 10 = 0 / 2, or generated on chip, key 10 = 1, the same
    bits) and off (key 6 = 1)."""
    sc = scenes.radar_scene(N=N, nlags=min(nlags, 64), nbins=min(nbins, 64), seed=66 + N % 11)
    rng = np.random.default_rng(67)
    dA = scenes.cn(rng, (nlags, nbins))
    want_s = oracle.caf_adjoint(sc.s_surv, sc.s_ref, lag0, nlags, p0, nbins, dA, flags=flags)
    want_r = oracle.caf_adjoint_ref(sc.s_surv, sc.s_ref, lag0, nlags, p0, nbins, dA, flags=flags)
    outs = {}
    for key, gen in ((2, 0), (2, 2), (2, 1), (1, 0)):
        p = api.Plan(N, p0=p0, nbins=nbins, max_lags=nlags, flags=flags, form="ternary", prec="bf16x2")
        p.set_tuning(6, key)
        p.set_tuning(10, gen)
        ss, sr, d = dev(sc.s_surv), dev(sc.s_ref), dev(dA.astype(np.complex64))
        g = p.caf_backward(ss, sr, lag0, nlags, d).cpu().numpy()
        p.query_error()
        assert p.query(1) == (2 if key == 2 else 1)
        assert relerr(g, want_s) < TOL, key
        gs, gr = p.caf_backward_inputs(ss, sr, lag0, nlags, d)
        p.query_error()
        assert p.query(1) == (2 if key == 2 else 1)
        assert relerr(gs.cpu().numpy(), want_s) < TOL, key
        assert relerr(gr.cpu().numpy(), want_r) < TOL, key
        outs[(key, gen)] = (g, gs.cpu().numpy(), gr.cpu().numpy())
    for other in ((2, 1), (2, 2)):
        for a, b in zip(outs[(2, 0)], outs[other]):
            a, b = np.ascontiguousarray(a), np.ascontiguousarray(b)
            assert np.array_equal(a.view(np.uint32), b.view(np.uint32)), other


def test_paired_adjoint_headline_sampled(api):
    """Both gradients of the 65536-sample, 1024 x 1024 surface through the paired
    adjoint (the default there) at sampled indices against the oracle."""
    sc = scenes.radar_scene(N=65536)
    rng = np.random.default_rng(68)
    dA = (scenes.cn(rng, (1024, 1024)) * (rng.random((1024, 1024)) < 0.01)).astype(np.complex64)
    p = api.Plan(sc.N, p0=-512, nbins=1024, max_lags=1024, form="ternary", prec="bf16x2")
    gs, gr = p.caf_backward_inputs(dev(sc.s_surv), dev(sc.s_ref), 0, 1024, dev(dA))
    p.query_error()
    assert p.query(1) == 2
    idx = np.concatenate([[0, 1, 37, 65535, 1023, 1024], rng.integers(0, 65536, 26)])
    ws = oracle.caf_adjoint_at(sc.s_surv, sc.s_ref, 0, 1024, -512, 1024, dA, "surv", idx)
    wr = oracle.caf_adjoint_at(sc.s_surv, sc.s_ref, 0, 1024, -512, 1024, dA, "ref", idx)
    gs, gr = gs.cpu().numpy(), gr.cpu().numpy()
    assert np.max(np.abs(gs[idx] - ws)) / np.max(np.abs(gs)) < TOL
    assert np.max(np.abs(gr[idx] - wr)) / np.max(np.abs(gr)) < TOL
