"""GPU parity of the tensor-core (ternary GEMM) form against the CPU oracle.

The form computes X = S v + F sigma(v) with bf16 hi+lo operands and fp32
accumulation; the bar is the fp32 one, 1e-5 of max |X| (against the oracle
with the lag product formed in fp32, the element-wise stage both forms share)."""
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


def test_ternary_small_ndft(api):
    rng = np.random.default_rng(40)
    x = scenes.cn(rng, (300, 64)).astype(np.complex64)
    p = api.Plan(64, max_batch=300, form="ternary", prec="bf16x2")
    got = p.ndft(dev(x)).cpu().numpy()
    p.query_error()
    ref = oracle.ndft(x.astype(np.complex128))
    assert relerr(got, ref) < TOL


def test_ternary_angle_table(api):
    N = 65536
    p = api.Plan(N, max_lags=1, form="ternary", prec="bf16x2")
    t = p.twiddles(2).cpu().numpy()
    nth = (N - 1) // 256 + 1
    a = np.concatenate([np.pi / 2 * (256 * np.arange(nth)) / N, np.pi / 2 * np.arange(256) / N])
    assert np.max(np.abs(t.real - np.cos(a))) < 1e-7 and np.max(np.abs(t.imag - np.sin(a))) < 1e-7
    assert t[0] == 1 and t[nth] == 1


@pytest.mark.parametrize("N,batch,p0,nbins", [(100, 130, -7, 77), (1024, 600, 0, 0), (9, 5, 2, 5), (1, 4, 0, 1)])
def test_ternary_ndft_ragged(api, N, batch, p0, nbins):
    rng = np.random.default_rng(41 + N)
    x = scenes.cn(rng, (batch, N)).astype(np.complex64)
    x[:, ::7] = 0
    nb = nbins or N
    ref = oracle.ndft(x.astype(np.complex128), p0=p0, nbins=nb)
    p = api.Plan(N, p0=p0, nbins=nbins, max_batch=batch, form="ternary", prec="bf16x2")
    got = p.ndft(dev(x)).cpu().numpy()
    p.query_error()
    assert relerr(got, ref) < TOL


def test_ternary_tone_batch_peak(api):
    x = scenes.tone_batch()
    ref = oracle.ndft(x.astype(np.complex128))
    p = api.Plan(64, max_batch=4096, form="ternary", prec="bf16x2")
    X = p.ndft(dev(x))
    got = X.cpu().numpy()
    per = np.max(np.abs(got - ref), axis=1) / np.max(np.abs(ref), axis=1)
    assert per.max() < TOL
    idx, _ = api.argmax(X)
    assert int(idx[0]) == 7


def test_ternary_caf(api):
    sc = scenes.radar_scene(N=4133, nlags=100, nbins=96, seed=31)
    ref = oracle.caf(sc.s_surv, sc.s_ref, -3, 100, sc.p0, 96, z32=True)
    p = api.Plan(sc.N, p0=sc.p0, nbins=96, max_lags=128, form="ternary", prec="bf16x2")
    got = p.caf(dev(sc.s_surv), dev(sc.s_ref), -3, 100).cpu().numpy()
    p.query_error()
    assert relerr(got, ref) < TOL


@pytest.mark.parametrize("flags", [1, 2])
def test_ternary_caf_flags(api, flags):
    sc = scenes.radar_scene(N=700, nlags=40, nbins=33, seed=32)
    ref = oracle.caf(sc.s_surv, sc.s_ref, 650, 40, -16, 33, flags=flags, z32=True)
    p = api.Plan(sc.N, p0=-16, nbins=33, max_lags=40, flags=flags, form="ternary", prec="bf16x2")
    got = p.caf(dev(sc.s_surv), dev(sc.s_ref), 650, 40).cpu().numpy()
    assert relerr(got, ref) < TOL


def test_ternary_caf_split_k_sampled(api):
    """A long sample axis (split into many K ranges) on sampled cells."""
    sc = scenes.radar_scene(N=16384, nlags=300, nbins=256, seed=42)
    p = api.Plan(sc.N, p0=sc.p0, nbins=256, max_lags=300, form="ternary", prec="bf16x2")
    A = p.caf(dev(sc.s_surv), dev(sc.s_ref), 0, 300)
    got = A.cpu().numpy()
    p.query_error()
    rng = np.random.default_rng(43)
    lags = np.concatenate([[0, 37, 120, 299], rng.integers(0, 300, 60)])
    bins = np.concatenate([[0, 5, -12, 127], rng.integers(-128, 128, 60)])
    ref = oracle.caf_cells(sc.s_surv, sc.s_ref, lags, bins, z32=True)
    peak = abs(oracle.caf_cells(sc.s_surv, sc.s_ref, [0], [0], z32=True)[0])
    err = np.max(np.abs(got[lags, bins - sc.p0] - ref))
    assert err / peak < TOL
    # the direct form agrees too
    pd = api.Plan(sc.N, p0=sc.p0, nbins=256, max_lags=300)
    Ad = pd.caf(dev(sc.s_surv), dev(sc.s_ref), 0, 300).cpu().numpy()
    assert np.max(np.abs(Ad - got)) / peak < 2 * TOL


@pytest.mark.parametrize("parts", [0, 1, 512])
def test_ternary_two_column_parts(api, parts):
    """Key 5 = 0 runs calls of at least 512 lags as two column parts (the second
    part packed under the first part's contraction on the plan's side stream);
    one part (key 5 = 1, the default) and an explicit first part of 512 lags
    give the same surface within the bar, ragged in lags, bins and samples."""
    sc = scenes.radar_scene(N=9000, nlags=700, nbins=200, seed=47)
    rng = np.random.default_rng(48)
    lags = np.concatenate([[0, 255, 256, 511, 512, 699], rng.integers(0, 700, 40)])
    bins = np.concatenate([[0, 5, -12, 99, -100, 40], rng.integers(-100, 100, 40)])
    ref = oracle.caf_cells(sc.s_surv, sc.s_ref, np.asarray(lags) - 4, bins, z32=True)
    p = api.Plan(sc.N, p0=sc.p0, nbins=200, max_lags=700, form="ternary", prec="bf16x2")
    p.set_tuning(5, parts)
    A = p.caf(dev(sc.s_surv), dev(sc.s_ref), -4, 700).cpu().numpy()
    p.query_error()
    # one part: the paired contraction packing its own B operand, then the fold;
    # two parts: packing, contraction and ordered split-K sum each
    assert p.last_launches() == (2 if parts == 1 else 6)
    peak = np.max(np.abs(A))
    assert np.max(np.abs(A[lags, bins - sc.p0] - ref)) / peak < TOL
    # the NDFT of 700 vectors the same way
    x = scenes.cn(np.random.default_rng(49), (700, 300)).astype(np.complex64)
    q = api.Plan(300, p0=-7, nbins=77, max_batch=700, form="ternary", prec="bf16x2")
    q.set_tuning(5, parts)
    got = q.ndft(dev(x)).cpu().numpy()
    want = oracle.ndft(x.astype(np.complex128), p0=-7, nbins=77)
    assert relerr(got, want) < TOL


@pytest.mark.parametrize("tile", [256, 128, 258])
@pytest.mark.parametrize("chunk", [64, 16])
def test_ternary_tile_variants(api, tile, chunk):
    """Every tile shape (256 rows; 128 rows with two accumulators; the 256-row
    tile on a 2-SM pair) and chain length gives the same
    surface within the bar, on a ragged problem with split sample axis."""
    sc = scenes.radar_scene(N=9000, nlags=300, nbins=200, seed=45)
    lags = np.array([0, 37, 120, 299, 5, 250])
    bins = np.array([0, 5, -12, 99, -100, 40])
    ref = oracle.caf_cells(sc.s_surv, sc.s_ref, lags, bins, z32=True)
    p = api.Plan(sc.N, p0=sc.p0, nbins=200, max_lags=300, form="ternary", prec="bf16x2")
    p.set_tuning(1, tile)
    p.set_tuning(2, chunk)
    A = p.caf(dev(sc.s_surv), dev(sc.s_ref), 0, 300).cpu().numpy()
    p.query_error()
    assert np.isfinite(A).all()
    peak = np.max(np.abs(A))
    assert np.max(np.abs(A[lags, bins - sc.p0] - ref)) / peak < TOL
    x = scenes.cn(np.random.default_rng(46), (300, 100)).astype(np.complex64)
    q = api.Plan(100, p0=-7, nbins=77, max_batch=300, form="ternary", prec="bf16x2")
    q.set_tuning(1, tile)
    q.set_tuning(2, chunk)
    got = q.ndft(dev(x)).cpu().numpy()
    want = oracle.ndft(x.astype(np.complex128), p0=-7, nbins=77)
    assert relerr(got, want) < TOL


def test_ternary_bounded_waits_time_out(api):
    """Failure detection without a fault: with the test-only key that starves
    the contraction of its operand loads, every bounded wait of the kernel runs
    out (about 2 s), the kernel returns, and the plan's error word reports
    NDFT_E_TIMEOUT; the context and the plan stay usable and the next normal
    call reproduces the surface bit for bit."""
    import time
    from paper_1402_0532_gb300 import _lib as L
    sc = scenes.radar_scene(N=4096, nlags=64, nbins=64, seed=49)
    p = api.Plan(sc.N, p0=-32, nbins=64, max_lags=64, form="ternary", prec="bf16x2")
    ss, sr = dev(sc.s_surv), dev(sc.s_ref)
    A = p.caf(ss, sr, 0, 64).cpu().numpy()
    p.query_error()
    p.set_tuning(4, 1)
    t0 = time.time()
    p.caf(ss, sr, 0, 64)
    with pytest.raises(L.NdftError) as e:
        p.query_error()
    assert e.value.status == L.E_TIMEOUT
    assert time.time() - t0 < 60
    p.query_error()  # the error word was cleared by the read
    p.set_tuning(4, 0)
    B = p.caf(ss, sr, 0, 64).cpu().numpy()
    p.query_error()
    assert np.array_equal(A.view(np.uint32), B.view(np.uint32))


def test_plan_allocation_failure_is_reported(api):
    """A plan whose workspace cannot be allocated (a 4.4 TB packed operand)
    fails with NDFT_E_NOMEM and leaves the device usable."""
    from paper_1402_0532_gb300 import _lib as L
    with pytest.raises(L.NdftError) as e:
        api.Plan(1 << 18, max_lags=1 << 20, form="ternary", prec="bf16x2")
    assert e.value.status == L.E_NOMEM
    x = scenes.cn(np.random.default_rng(52), (4, 64)).astype(np.complex64)
    q = api.Plan(64, max_batch=4, form="ternary", prec="bf16x2")
    assert relerr(q.ndft(dev(x)).cpu().numpy(), oracle.ndft(x.astype(np.complex128))) < TOL


@pytest.mark.parametrize("N,lag0,nlags,p0,nbins,flags", [(700, 2, 70, -20, 40, 0), (4133, -3, 300, -48, 96, 0),
                                                         (2048, 10, 257, 0, 512, 1), (1500, 1400, 33, -7, 17, 2)])
def test_ternary_adjoint_tensor_cores(api, N, lag0, nlags, p0, nbins, flags):
    """caf_backward on a tensor-core plan runs the transposed ternary contraction
    on tcgen05 (dA as bf16 hi + lo against exact signs); against the fp64 oracle
    adjoint within the fp32 bar, ragged tiles and the flags included."""
    sc = scenes.radar_scene(N=N, nlags=nlags, nbins=min(nbins, 64), seed=53 + N % 7)
    rng = np.random.default_rng(54)
    dA = scenes.cn(rng, (nlags, nbins))
    want = oracle.caf_adjoint(sc.s_surv, sc.s_ref, lag0, nlags, p0, nbins, dA, flags=flags)
    p = api.Plan(N, p0=p0, nbins=nbins, max_lags=nlags, flags=flags, form="ternary", prec="bf16x2")
    got = p.caf_backward(dev(sc.s_surv), dev(sc.s_ref), lag0, nlags, dev(dA.astype(np.complex64))).cpu().numpy()
    p.query_error()
    assert p.last_launches() == 3  # pack, contraction, ordered sum of the partials
    assert relerr(got, want) < TOL
