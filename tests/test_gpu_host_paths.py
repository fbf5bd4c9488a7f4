"""The host-to-host entry points: caf_from_host (copy in, caf_exec, copy out)
and its pipelined form over a sequence of inputs (one compute stream, or two
with a twin plan) give the device path's surfaces bit for bit."""
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


@pytest.mark.parametrize("form,prec", [("ternary", "bf16x2"), ("direct", "fp32")])
def test_host_paths_match_device_path(api, form, prec):
    N, nlags, nbins = 8192, 96, 128
    scs = [scenes.radar_scene(N=N, nlags=nlags, nbins=nbins, seed=90 + k) for k in range(5)]
    plan = api.Plan(N, p0=scs[0].p0, nbins=nbins, max_lags=nlags, form=form, prec=prec)
    want = [plan.caf(torch.from_numpy(sc.s_surv).cuda(), torch.from_numpy(sc.s_ref).cuda(), 0, nlags)
            .cpu().numpy() for sc in scs]
    ins = [(torch.from_numpy(sc.s_surv).pin_memory(), torch.from_numpy(sc.s_ref).pin_memory()) for sc in scs]
    one = torch.empty(nlags, nbins, dtype=torch.complex64).pin_memory()
    plan.caf_from_host(ins[2][0], ins[2][1], 0, nlags, one)
    assert np.array_equal(one.numpy(), want[2])
    outs = [torch.empty(nlags, nbins, dtype=torch.complex64).pin_memory() for _ in scs]
    staging = {}
    plan.caf_from_host_many(ins, 0, nlags, outs, staging)
    for o, w in zip(outs, want):
        assert np.array_equal(o.numpy(), w)
    # again with the same staging, one output buffer reused: it ends with the last surface
    plan.caf_from_host_many(ins[::-1], 0, nlags, one, staging)
    assert np.array_equal(one.numpy(), want[0])
    # consecutive steps on two streams with a twin plan: the same surfaces, twice over
    # the same staging (the twin and its stream are made once)
    outs2 = [torch.empty(nlags, nbins, dtype=torch.complex64).pin_memory() for _ in scs]
    st2 = {}
    plan.caf_from_host_many(ins, 0, nlags, outs2, st2, overlap=True)
    for o, w in zip(outs2, want):
        assert np.array_equal(o.numpy(), w)
    twin = st2["twin"]
    plan.caf_from_host_many(ins[::-1], 0, nlags, outs2, st2, overlap=True)
    assert st2["twin"] is twin
    for o, w in zip(outs2, want[::-1]):
        assert np.array_equal(o.numpy(), w)
    plan.query_error()


def test_twin_plan_keeps_the_tuning(api):
    """twin() copies the descriptor and every tuning setting: same surface bit for bit."""
    from paper_1402_0532_gb300 import autotune as at
    N, nlags, nbins = 8192, 64, 128
    sc = scenes.radar_scene(N=N, nlags=nlags, nbins=nbins, seed=97)
    ss, sr = torch.from_numpy(sc.s_surv).cuda(), torch.from_numpy(sc.s_ref).cuda()
    plan = api.Plan(N, p0=sc.p0, nbins=nbins, max_lags=nlags, form="ternary", prec="bf16x2")
    plan.set_tuning(at.ROWS, 128)
    plan.set_tuning(at.CHUNK, 32)
    twin = plan.twin()
    assert twin._tuning == plan._tuning and twin.handle.value != plan.handle.value
    a = plan.caf(ss, sr, 0, nlags).cpu().numpy()
    b = twin.caf(ss, sr, 0, nlags).cpu().numpy()
    assert np.array_equal(a, b)
    twin.query_error()
