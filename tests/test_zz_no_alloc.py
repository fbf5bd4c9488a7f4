"""caf_exec_noalloc: the entry point for callers that cannot allocate device
memory (for instance a real-time loop that forbids cudaMalloc after start-up,
or code running while another thread captures a CUDA graph in global mode).

It keeps its twiddle table and split-K partials in a static device array
instead of a plan.  Called through the C ABI, twice in a row (the second call
sees the first call's leftovers in the shared array), its surface must match
the plan-based caf_exec of the same direct fp32 form within the fp32
tolerance of the other tests.  This file sorts last so a stop at the first
failure has already run every other test."""
import ctypes

import numpy as np
import pytest

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


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


@pytest.mark.parametrize("N,nlags,nbins,lag0", [(4133, 100, 96, -3), (65536, 1024, 1024, 0)])
def test_noalloc_matches_plan_twice(api, N, nlags, nbins, lag0):
    from paper_1402_0532_gb300 import _lib as L
    lib = L.load()
    sc = scenes.radar_scene(N=N, nlags=nlags, nbins=nbins, seed=50)
    ss = torch.from_numpy(sc.s_surv).cuda()
    sr = torch.from_numpy(sc.s_ref).cuda()
    plan = api.Plan(N, p0=sc.p0, nbins=nbins, max_lags=nlags)
    want = plan.caf(ss, sr, lag0, nlags).cpu().numpy()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    scale = np.max(np.abs(want))
    for _ in range(2):
        out = torch.full((nlags, nbins), complex(np.nan, np.nan), dtype=torch.complex64, device="cuda")
        st = lib.caf_exec_noalloc(N, sc.p0, nbins, _ptr(ss), _ptr(sr), lag0, nlags, 0, _ptr(out), stream)
        assert st == L.OK, L.status_string(st)
        got = out.cpu().numpy()
        assert np.all(np.isfinite(got))
        assert np.max(np.abs(got - want)) <= TOL * scale


def test_noalloc_rejects_sizes_beyond_its_limit(api):
    from paper_1402_0532_gb300 import _lib as L
    lib = L.load()
    s = torch.zeros(16, dtype=torch.complex64, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert lib.caf_exec_noalloc((1 << 20) + 1, 0, 4, _ptr(s), _ptr(s), 0, 1, 0, _ptr(s), stream) == L.E_INVALID
    assert lib.caf_exec_noalloc(16, 0, 17, _ptr(s), _ptr(s), 0, 1, 0, _ptr(s), stream) == L.E_INVALID
