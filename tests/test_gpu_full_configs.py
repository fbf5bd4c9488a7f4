"""Parity at the full sizes of the benchmark's workloads, in the launch
configurations the benchmark times:

* the NFFT of 65536 vectors of N = 1024 (every vector, bit for bit against
  the oracle's fp32 recursion) and the NDFT of the same batch in both forms
  (sampled vectors against the fp64 oracle, within 1e-5 of each vector's
  max |X|, and their peaks wherever the oracle's top two are separated);
* the CAF surface of 65536 samples, 1024 lags x 1024 bins in both forms (and
  the tensor-core form with and without the conjugate pairing): every bin of
  38 lag rows, including every tile boundary, against the fp64 oracle (lag
  product in fp32, the stage both forms share), within 1e-5 of max |A|, with
  per-row peaks.
"""
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


@pytest.fixture(scope="module")
def batch():
    return scenes.cn_batch()


def test_nfft_full_batch_bit_exact(api, batch):
    p = api.Plan(1024, max_batch=batch.shape[0])
    got = p.nfft(torch.from_numpy(batch).cuda()).cpu().numpy()
    p.query_error()
    want = oracle.nfft_f32(batch)
    assert np.array_equal(got.view(np.uint32), want.view(np.uint32))
    # every vector whose (x) operands provably keep their fp64 signs in fp32:
    # within the running error bound of the fp64 recursion and within 1e-5 of
    # its max |X|; the rest are counted as ill-conditioned
    X, bound, stable = oracle.nfft_bound(batch)
    assert stable.mean() > 0.9
    assert oracle.within_bound(got[stable], X[stable], bound[stable]).all()
    amax = np.abs(X).max(axis=1)
    assert (np.abs(got - X).max(axis=1) / amax)[stable].max() < TOL
    print(f"NFFT 65536 x 1024: {int((~stable).sum())} vectors ill-conditioned")


@pytest.mark.parametrize("form,prec", [("direct", "fp32"), ("ternary", "bf16x2")])
def test_ndft_full_batch_sampled(api, batch, form, prec):
    p = api.Plan(1024, max_batch=batch.shape[0], form=form, prec=prec)
    X = p.ndft(torch.from_numpy(batch).cuda())
    idx, _ = api.argmax(X)
    got = X.cpu().numpy()
    idx = idx.cpu().numpy()
    p.query_error()
    rng = np.random.default_rng(50)
    rows = np.unique(np.concatenate([np.arange(16), rng.integers(0, batch.shape[0], 112), [batch.shape[0] - 1]]))
    ref = oracle.ndft(batch[rows].astype(np.complex128))
    amax = np.max(np.abs(ref), axis=1)
    err = np.max(np.abs(got[rows] - ref), axis=1) / amax
    assert err.max() < TOL
    # peaks: equal wherever the oracle's top two magnitudes are separated by more than the bar
    mag = np.sort(np.abs(ref), axis=1)
    clear = (mag[:, -1] - mag[:, -2]) > 2 * TOL * amax
    assert clear.sum() > len(rows) // 2
    assert np.array_equal(idx[rows][clear], np.argmax(np.abs(ref), axis=1)[clear])


@pytest.fixture(scope="module")
def surface():
    return scenes.radar_scene(N=65536)


# lag rows checked in full (all 1024 bins): the direct path and the echoes, the
# first and last lag, and both sides of every 64-lag tile boundary of the plain
# form and every 128-lag (256-column) tile boundary of the paired contraction
ROW_LAGS = np.array(sorted({0, 1, 37, 63, 64, 120, 127, 128, 129, 191, 192, 255, 256, 301, 320, 383, 384, 447,
                            448, 511, 512, 575, 576, 639, 640, 703, 704, 767, 768, 831, 832, 895, 896, 959,
                            960, 1000, 1022, 1023}))


@pytest.fixture(scope="module")
def surface_rows(surface):
    """The oracle (lag product in fp32, the element-wise stage both forms share)
    on every bin of ROW_LAGS."""
    sc = surface
    L, B = np.meshgrid(ROW_LAGS, np.arange(-512, 512), indexing="ij")
    return oracle.caf_cells(sc.s_surv, sc.s_ref, L.ravel(), B.ravel(), z32=True).reshape(len(ROW_LAGS), 1024)


@pytest.mark.parametrize("form,prec,pair", [("direct", "fp32", 0), ("ternary", "bf16x2", 0), ("ternary", "bf16x2", 1)])
def test_caf_full_surface_lag_rows(api, surface, surface_rows, form, prec, pair):
    """The 65536-sample surface, 1024 lags x bins -512..511, in the launch
    configuration the benchmark times (the tensor-core form conjugate-paired by
    default; pair = 1 forces one row pair per bin): every bin of 38 lag rows
    within 1e-5 of max |A|, each row's peak bin equal to the oracle's wherever
    its top two magnitudes are separated by more than the bar, and the
    surface's peak at the direct path."""
    sc = surface
    p = api.Plan(sc.N, p0=-512, nbins=1024, max_lags=1024, form=form, prec=prec)
    if pair:
        p.set_tuning(6, 1)
    A = p.caf(torch.from_numpy(sc.s_surv).cuda(), torch.from_numpy(sc.s_ref).cuda(), 0, 1024)
    idx, _ = api.argmax(A.reshape(1, -1))
    rows_idx, _ = api.argmax(A)
    got = A.cpu().numpy()
    rows_idx = rows_idx.cpu().numpy()
    p.query_error()
    if form == "ternary":
        assert p.query(1) == (1 if pair else 2)
    ref = surface_rows
    amax = np.max(np.abs(got))
    err = np.max(np.abs(got[ROW_LAGS] - ref)) / amax
    print(f"{form}/{prec}/pair-off={pair}: max error over {ref.size} cells {err:.3e} of max|A|")
    assert err < TOL
    mag = np.sort(np.abs(ref), axis=1)
    clear = (mag[:, -1] - mag[:, -2]) > 2 * TOL * amax
    assert clear.sum() >= len(ROW_LAGS) // 2
    assert np.array_equal(rows_idx[ROW_LAGS][clear], np.argmax(np.abs(ref), axis=1)[clear])
    # the surface's peak is the direct path (lag 0, bin 0)
    assert int(idx[0]) == 0 * 1024 + 512
