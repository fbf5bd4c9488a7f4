"""The |A| epilogue (NDFT_F_ABS_OUT): caf_exec writes the magnitude surface
sqrt(re^2 + im^2) (fp32) from the split sum / pair fold instead of A.  Each
plan kind is checked against the magnitude of the complex surface the same
plan kind writes without the flag (the same sums, so within a few ulp) and
against |A| of the fp64 oracle at the fp32 bar; the flag is refused where it
does not apply."""
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


@pytest.mark.parametrize("form,prec,pair,split", [("direct", "fp32", 0, 0), ("direct", "fp32", 0, 1),
                                                  ("ternary", "bf16x2", 0, 0), ("ternary", "bf16x2", 1, 0),
                                                  ("ternary", "bf16x2", 1, 1)])
def test_abs_surface(api, form, prec, pair, split):
    sc = scenes.radar_scene(N=6000, nlags=300, nbins=256, seed=90)
    outs = []
    for flags in (0, api.F_ABS_OUT):
        p = api.Plan(sc.N, p0=-128, nbins=256, max_lags=300, form=form, prec=prec, flags=flags)
        if split:
            p.set_tuning(0, 1)
        if pair:
            p.set_tuning(6, 1)  # one row pair per bin
        A = p.caf(dev(sc.s_surv), dev(sc.s_ref), -2, 300)
        p.query_error()
        assert A.dtype == (torch.float32 if flags else torch.complex64)
        outs.append(A.cpu().numpy())
    mag = np.abs(outs[0].astype(np.complex128))
    assert np.max(np.abs(outs[1] - mag)) <= 4e-7 * np.max(mag)
    rng = np.random.default_rng(91)
    lags = np.concatenate([[0, 299, 39], rng.integers(0, 300, 40)])
    bins = np.concatenate([[0, -128, 127], rng.integers(-128, 128, 40)])
    ref = np.abs(oracle.caf_cells(sc.s_surv, sc.s_ref, lags - 2, bins, z32=True))
    assert np.max(np.abs(outs[1][lags, bins + 128] - ref)) / np.max(outs[1]) < TOL


def test_abs_refused_where_it_does_not_apply(api):
    from paper_1402_0532_gb300 import _lib as L
    with pytest.raises(L.NdftError) as ex:
        api.Plan(64, max_batch=1, prec="q14", flags=api.F_ABS_OUT)
    assert ex.value.status == L.E_INVALID
    with pytest.raises(L.NdftError) as ex:
        api.Plan(64, max_batch=1, form="nfft", prec="fp32", flags=api.F_ABS_OUT)
    assert ex.value.status == L.E_UNSUPPORTED
    p = api.Plan(64, max_batch=2, form="ternary", prec="bf16x2", flags=api.F_ABS_OUT)
    x = torch.zeros(2, 64, dtype=torch.complex64, device="cuda")
    with pytest.raises(L.NdftError) as ex:
        p.ndft(x)
    assert ex.value.status == L.E_UNSUPPORTED
