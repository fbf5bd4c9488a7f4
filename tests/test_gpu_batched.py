"""Batched CPIs: many uneven coherent processing intervals in one persistent
launch sequence, captured in a CUDA graph.  Parity against the oracle per CPI,
graph replay against eager execution, and the full 256-CPI workload
(N_c ~ U{1024..32768}, L_c ~ U{64..1024}, 1024 bins) on sampled cells."""
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


def pack(scs, q14=False):
    surv, ref, cpis, oo, so = [], [], [], 0, 0
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


def small_scenes():
    rng = np.random.default_rng(36)
    return [scenes.radar_scene(N=int(n), nlags=int(l), nbins=int(b), rng=rng)
            for n, l, b in ((1000, 70, 64), (1536, 5, 96), (777, 130, 33), (2048, 300, 128), (1111, 1, 7))]


@pytest.mark.parametrize("pairing", [0, 1])
def test_batched_ternary_small(api, pairing):
    """The tensor-core batch as conjugate-paired calls per CPI (the default
    when every window pairs) and as one persistent unpaired contraction over
    all CPIs (tuning key 6 = 1), each CPI against the oracle."""
    scs = small_scenes()
    surv, ref, cpis, total = pack(scs)
    bp = api.BatchedPlan(cpis, form="ternary", prec="bf16x2")
    bp.set_tuning(6, pairing)
    out = torch.zeros(total, dtype=torch.complex64, device="cuda")
    bp(dev(surv), dev(ref), out)
    bp.query_error()
    got = out.cpu().numpy()
    for sc, c in zip(scs, cpis):
        g = got[c["off_out"]: c["off_out"] + sc.nlags * sc.nbins].reshape(sc.nlags, sc.nbins)
        want = oracle.caf(sc.s_surv, sc.s_ref, sc.lag0, sc.nlags, sc.p0, sc.nbins, z32=True)
        assert np.max(np.abs(g - want)) / np.max(np.abs(want)) < TOL


@pytest.mark.parametrize("pairing", [0, 1])
def test_batched_ternary_uniform_bins(api, pairing):
    """CPIs that share an even nbins use one output tensor map for the bulk-copy
    fold-out of the unpaired contraction; lag counts that are not multiples of
    16 end in column groups that are written element by element (so no CPI's
    copy runs into the next surface).  Long CPIs make several accumulation
    chains per unit.  Paired per-CPI calls (default) and unpaired (key 6 = 1)."""
    rng = np.random.default_rng(37)
    scs = [scenes.radar_scene(N=int(n), nlags=int(l), nbins=40, rng=rng)
           for n, l in ((9000, 5), (1536, 17), (12000, 33), (2048, 300), (700, 1), (16384, 16))]
    surv, ref, cpis, total = pack(scs)
    bp = api.BatchedPlan(cpis, form="ternary", prec="bf16x2")
    bp.set_tuning(6, pairing)
    out = torch.zeros(total, dtype=torch.complex64, device="cuda")
    guard = torch.full((total + 64,), complex(7.0, -7.0), dtype=torch.complex64, device="cuda")
    bp(dev(surv), dev(ref), guard[:total])
    bp(dev(surv), dev(ref), out)
    bp.query_error()
    got = out.cpu().numpy()
    assert np.all(guard[total:].cpu().numpy() == complex(7.0, -7.0))  # nothing past the last surface
    assert np.array_equal(guard[:total].cpu().numpy(), got)  # the stale contents do not leak in
    for sc, c in zip(scs, cpis):
        g = got[c["off_out"]: c["off_out"] + sc.nlags * sc.nbins].reshape(sc.nlags, sc.nbins)
        want = oracle.caf(sc.s_surv, sc.s_ref, sc.lag0, sc.nlags, sc.p0, sc.nbins, z32=True)
        assert np.max(np.abs(g - want)) / np.max(np.abs(want)) < TOL


def test_batched_q14_range_check(api):
    """Batched Q1.14 with NDFT_F_Q14_RANGE: every CPI bit for bit against the
    oracle as without the flag, no report on in-range data, and NDFT_E_OVERFLOW
    once one CPI's inputs are at full scale."""
    from paper_1402_0532_gb300 import _lib as L
    scs = small_scenes()
    surv, ref, cpis, total = pack(scs, q14=True)
    bp = api.BatchedPlan(cpis, form="direct", prec="q14", flags=api.F_Q14_RANGE)
    out = torch.zeros((total, 2), dtype=torch.int32, device="cuda")
    bp(dev(surv), dev(ref), out)
    bp.query_error()
    got = out.cpu().numpy()
    for sc, c in zip(scs, cpis):
        qs, qr = scenes.quantize_q14(sc.s_surv, 0.25), scenes.quantize_q14(sc.s_ref, 0.25)
        want, novf = oracle.caf_q14(qs, qr, sc.lag0, sc.nlags, sc.p0, sc.nbins)
        assert novf == 0
        g = got[c["off_out"]: c["off_out"] + sc.nlags * sc.nbins].reshape(sc.nlags, sc.nbins, 2)
        assert np.array_equal(g, want)
    # a full-scale CPI of 65536 samples: its bin-0 sums leave int32
    n = 65536
    big = [{"off_surv": 0, "off_ref": 0, "off_out": 0, "n": n, "lag0": 0, "nlags": 2, "p0": -1, "nbins": 3}]
    fs = np.full((n, 2), 32767, np.int16)
    fr = np.full((n, 2), -32768, np.int16)
    want, novf = oracle.caf_q14(fs, fr, 0, 2, -1, 3)
    assert novf > 0
    bq = api.BatchedPlan(big, form="direct", prec="q14", flags=api.F_Q14_RANGE)
    o2 = torch.zeros((6, 2), dtype=torch.int32, device="cuda")
    bq(dev(fs), dev(fr), o2)
    assert np.array_equal(o2.cpu().numpy().reshape(2, 3, 2), want)
    with pytest.raises(L.NdftError) as ex:
        bq.query_error()
    assert ex.value.status == L.E_OVERFLOW


@pytest.mark.parametrize("form,prec", [("direct", "fp32"), ("ternary", "bf16x2"), ("direct", "q14")])
def test_batched_graph_replay_equals_eager(api, form, prec):
    q14 = prec == "q14"
    surv, ref, cpis, total = pack(small_scenes(), q14=q14)
    bp = api.BatchedPlan(cpis, form=form, prec=prec)
    shape = (total, 2) if q14 else (total,)
    dt = torch.int32 if q14 else torch.complex64
    ds, dr = dev(surv), dev(ref)
    eager = torch.zeros(shape, dtype=dt, device="cuda")
    bp(ds, dr, eager)
    torch.cuda.synchronize()
    out = torch.zeros(shape, dtype=dt, device="cuda")
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        bp(ds, dr, out)  # warm the kernels' attributes outside capture
    torch.cuda.current_stream().wait_stream(s)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        bp(ds, dr, out)
    out.zero_()
    g.replay()
    g.replay()
    torch.cuda.synchronize()
    bp.query_error()
    assert torch.equal(out, eager)


@pytest.fixture(scope="module")
def cpi256():
    return scenes.cpi_batch()


@pytest.mark.parametrize("form,prec", [("ternary", "bf16x2"), ("direct", "fp32"), ("direct", "q14")])
def test_full_256_cpi_batch_sampled(api, cpi256, form, prec):
    scs = cpi256
    assert len(scs) == 256
    q14 = prec == "q14"
    surv, ref, cpis, total = pack(scs, q14=q14)
    bp = api.BatchedPlan(cpis, form=form, prec=prec)
    shape = (total, 2) if q14 else (total,)
    out = torch.zeros(shape, dtype=torch.int32 if q14 else torch.complex64, device="cuda")
    bp(dev(surv), dev(ref), out)
    bp.query_error()
    got = out.cpu().numpy()
    rng = np.random.default_rng(60)
    # every CPI: its four corner cells (first / last lag x first / last bin), the
    # direct path and 4 random cells
    for c in range(256):
        sc, cp = scs[c], cpis[c]
        last_l, last_b = sc.nlags - 1, sc.p0 + sc.nbins - 1
        lags = np.concatenate([[0, 0, last_l, last_l, 0], rng.integers(0, sc.nlags, 4)])
        bins = np.concatenate([[sc.p0, last_b, sc.p0, last_b, 0], rng.integers(sc.p0, sc.p0 + sc.nbins, 4)])
        idx = cp["off_out"] + lags * sc.nbins + (bins - sc.p0)
        if q14:
            qs, qr = scenes.quantize_q14(sc.s_surv, 0.25), scenes.quantize_q14(sc.s_ref, 0.25)
            for l, b, i in zip(lags, bins, idx):
                want, _ = oracle.caf_q14(qs, qr, int(l), 1, int(b), 1)
                assert np.array_equal(got[i], want[0, 0]), (c, l, b)
        else:
            want = oracle.caf_cells(sc.s_surv, sc.s_ref, lags, bins, z32=True)
            peak = abs(oracle.caf_cells(sc.s_surv, sc.s_ref, [0], [0], z32=True)[0])
            assert np.max(np.abs(got[idx] - want)) / peak < TOL, c


def test_batched_unpaired_operand_kept_only_when_modest(api, cpi256):
    """A paired tensor-core batch keeps the whole batch's unpaired operand
    beside its two paired slices only while it is at most 4 GiB: the 256-CPI
    workload's (41 GB) is not kept, so key 6 = 1 is refused, and the plan
    stays usable with the paired calls."""
    from paper_1402_0532_gb300 import _lib as L
    surv, ref, cpis, total = pack(cpi256[:4])
    small = api.BatchedPlan(cpis, form="ternary", prec="bf16x2")
    small.set_tuning(6, 1)
    out = torch.zeros(total, dtype=torch.complex64, device="cuda")
    small(dev(surv), dev(ref), out)  # small batch: the unpaired operand is kept
    small.query_error()
    surv, ref, cpis, total = pack(cpi256)
    bp = api.BatchedPlan(cpis, form="ternary", prec="bf16x2")
    assert bp.nbytes() < 4 << 30
    out = torch.zeros(total, dtype=torch.complex64, device="cuda")
    bp.set_tuning(6, 1)
    with pytest.raises(L.NdftError) as ex:
        bp(dev(surv), dev(ref), out)
    assert ex.value.status == L.E_UNSUPPORTED
    bp.set_tuning(6, 0)
    bp(dev(surv), dev(ref), out)
    bp.query_error()
