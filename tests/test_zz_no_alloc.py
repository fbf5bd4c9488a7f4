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


def _call(lib, L, sc, N, p0, nbins, ss, sr, lag0, nlags, flags):
    out = torch.full((nlags, nbins), complex(np.nan, np.nan), dtype=torch.complex64, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    st = lib.caf_exec_noalloc(N, p0, nbins, _ptr(ss), _ptr(sr), lag0, nlags, flags, _ptr(out), stream)
    assert st == L.OK, L.status_string(st)
    got = out.cpu().numpy()
    assert np.all(np.isfinite(got))
    return got


# Shapes called in turn, each twice, so that every call finds another shape's
# table and partials (or its own) left in the shared array: a large surface
# (many split partials), a small ragged one with another bin window, and one
# whose single split does not fit beside the table (2048 x 2048 cells, 32 MiB
# per split), so the kernel writes the surface directly.
SHAPES = [(65536, 1024, 1024, 0, -512), (4133, 100, 96, -3, -48), (4096, 2048, 2048, -5, -1024),
          (65536, 1024, 1024, 0, -512)]


@pytest.mark.parametrize("flags", [0, 3])
def test_noalloc_matches_plan_twice(api, flags):
    from paper_1402_0532_gb300 import _lib as L
    lib = L.load()
    for N, nlags, nbins, lag0, p0 in SHAPES:
        sc = scenes.radar_scene(N=N, nlags=min(nlags, 1024), nbins=min(nbins, 1024), seed=50 + N % 7)
        ss = torch.from_numpy(sc.s_surv).cuda()
        sr = torch.from_numpy(sc.s_ref).cuda()
        plan = api.Plan(N, p0=p0, nbins=nbins, max_lags=nlags, flags=flags)
        want = plan.caf(ss, sr, lag0, nlags).cpu().numpy()
        scale = np.max(np.abs(want))
        for _ in range(2):
            got = _call(lib, L, sc, N, p0, nbins, ss, sr, lag0, nlags, flags)
            assert np.max(np.abs(got - want)) <= TOL * scale, (N, nlags, nbins)
        del plan


@pytest.mark.parametrize("flags", [0, 1, 2, 3])
def test_noalloc_against_oracle(api, flags):
    """Sampled cells of two shapes (including the first and last lag and bin)
    against the fp64 oracle with the lag product in fp32, for every flag
    combination (s_ref conjugated or not, zero-padded or circular)."""
    import oracle
    from paper_1402_0532_gb300 import _lib as L
    lib = L.load()
    rng = np.random.default_rng(70 + flags)
    for N, nlags, nbins, lag0, p0 in SHAPES[:3]:
        sc = scenes.radar_scene(N=N, nlags=min(nlags, 1024), nbins=min(nbins, 1024), seed=51 + N % 5)
        ss = torch.from_numpy(sc.s_surv).cuda()
        sr = torch.from_numpy(sc.s_ref).cuda()
        got = _call(lib, L, sc, N, p0, nbins, ss, sr, lag0, nlags, flags)
        a = np.concatenate([[0, 0, nlags - 1, nlags - 1], rng.integers(0, nlags, 28)])
        k = np.concatenate([[0, nbins - 1, 0, nbins - 1], rng.integers(0, nbins, 28)])
        want = oracle.caf_cells(sc.s_surv, sc.s_ref, a + lag0, k + p0, flags=flags, z32=True)
        peak = np.max(np.abs(got))
        assert np.max(np.abs(got[a, k] - want)) <= TOL * peak, (N, flags)


def test_noalloc_rejects_sizes_beyond_its_limit(api):
    from paper_1402_0532_gb300 import _lib as L
    lib = L.load()
    s = torch.zeros(16, dtype=torch.complex64, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert lib.caf_exec_noalloc((1 << 20) + 1, 0, 4, _ptr(s), _ptr(s), 0, 1, 0, _ptr(s), stream) == L.E_INVALID
    assert lib.caf_exec_noalloc(16, 0, 17, _ptr(s), _ptr(s), 0, 1, 0, _ptr(s), stream) == L.E_INVALID
