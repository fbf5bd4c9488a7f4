"""The index-checked build (libndft_checked.so, NDFT_CHECKED=1): its packing,
fold, epilogue and direct-tile kernels test every computed global index
against their problem's extents and report a failed test through the plan's
error word.  A child process with the checked library runs every form of the
path (paired and unpaired tensor-core CAF, two column parts, the NDFT, the
plain form in fp32 and Q1.14, a batched plan); no call may report an error and
every result must equal, bit for bit, the normal build's on the same inputs."""
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CASES = r"""
import numpy as np, torch
from paper_1402_0532_gb300 import api, scenes

def run_all():
    out = {}
    sc = scenes.radar_scene(N=4133, nlags=300, nbins=96, seed=31)
    ss, sr = torch.from_numpy(sc.s_surv).cuda(), torch.from_numpy(sc.s_ref).cuda()
    for name, form, prec, tune in (("paired", "ternary", "bf16x2", {}), ("unpaired", "ternary", "bf16x2", {6: 1}),
                                   ("parts", "ternary", "bf16x2", {5: 0, 6: 1}), ("direct", "direct", "fp32", {})):
        p = api.Plan(sc.N, p0=-48, nbins=96, max_lags=600, form=form, prec=prec)
        for k, v in tune.items():
            p.set_tuning(k, v)
        out[name] = p.caf(ss, sr, -3, 600).cpu().numpy()
        p.query_error()
    qs = torch.from_numpy(scenes.quantize_q14(sc.s_surv, 0.25)).cuda()
    qr = torch.from_numpy(scenes.quantize_q14(sc.s_ref, 0.25)).cuda()
    p = api.Plan(sc.N, p0=-48, nbins=96, max_lags=300, prec="q14")
    out["q14"] = p.caf(qs, qr, 0, 300).cpu().numpy()
    p.query_error()
    x = torch.from_numpy(scenes.cn(np.random.default_rng(5), (300, 1024)).astype(np.complex64)).cuda()
    p = api.Plan(1024, max_batch=300, form="ternary", prec="bf16x2")
    out["ndft"] = p.ndft(x).cpu().numpy()
    p.query_error()
    rng = np.random.default_rng(6)
    scs = [scenes.radar_scene(N=int(n), nlags=int(l), nbins=64, rng=rng) for n, l in ((1000, 70), (2048, 130))]
    surv = np.concatenate([s.s_surv for s in scs] + [np.zeros(8, np.complex64)])
    ref = np.concatenate([s.s_ref for s in scs] + [np.zeros(8, np.complex64)])
    cpis = [{"off_surv": 0, "off_ref": 0, "off_out": 0, "n": 1000, "lag0": 0, "nlags": 70, "p0": -32, "nbins": 64},
            {"off_surv": 1000, "off_ref": 1000, "off_out": 70 * 64, "n": 2048, "lag0": 0, "nlags": 130, "p0": -32,
             "nbins": 64}]
    for form, prec in (("direct", "fp32"), ("ternary", "bf16x2")):
        bp = api.BatchedPlan(cpis, form=form, prec=prec)
        o = torch.zeros(200 * 64, dtype=torch.complex64, device="cuda")
        bp(torch.from_numpy(surv).cuda(), torch.from_numpy(ref).cuda(), o)
        bp.query_error()
        out["batched_" + form] = o.cpu().numpy()
    return out
"""

CHILD = r"""
import sys; sys.path.insert(0, sys.argv[1])
import numpy as np
exec(open(sys.argv[2]).read())
res = run_all()
np.savez(sys.argv[3], **res)
"""


@pytest.fixture(scope="module")
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1402_0532_gb300 import build
    return build.build(checked=True)


def test_checked_build_matches_normal_build(built, tmp_path):
    assert os.path.exists(built)
    cases = tmp_path / "cases.py"
    cases.write_text(CASES)
    env = dict(os.environ, NDFT_CHECKED="1")
    r = subprocess.run([sys.executable, "-c", CHILD, ROOT, str(cases), str(tmp_path / "checked.npz")], env=env,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]  # query_error raises on any recorded index failure
    env = dict(os.environ, NDFT_CHECKED="0")
    r = subprocess.run([sys.executable, "-c", CHILD, ROOT, str(cases), str(tmp_path / "normal.npz")], env=env,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    a, b = np.load(tmp_path / "checked.npz"), np.load(tmp_path / "normal.npz")
    assert sorted(a.files) == sorted(b.files)
    for k in a.files:
        assert np.array_equal(a[k].view(np.uint8), b[k].view(np.uint8)), k
