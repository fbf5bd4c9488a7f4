"""NDFT_LOG: with the variable set the library writes one line per plan and per
exec call on stderr (what ran: form, contraction variant, splits, launches);
unset, it writes nothing.  Run in child processes so the environment is read
fresh."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CHILD = r"""
import sys; sys.path.insert(0, sys.argv[1])
import numpy as np, torch
from paper_1402_0532_gb300 import api, scenes
sc = scenes.radar_scene(N=4096, nlags=64, nbins=128, seed=3)
p = api.Plan(4096, p0=-64, nbins=128, max_lags=64, form="ternary", prec="bf16x2")
p.caf(torch.from_numpy(sc.s_surv).cuda(), torch.from_numpy(sc.s_ref).cuda(), 0, 64)
torch.cuda.synchronize()
"""


def run(env_value):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    env = dict(os.environ)
    env.pop("NDFT_LOG", None)
    if env_value is not None:
        env["NDFT_LOG"] = env_value
    r = subprocess.run([sys.executable, "-c", CHILD, ROOT], env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    return [ln for ln in r.stderr.splitlines() if ln.startswith("[ndft]")]


def test_log_lines_when_set():
    lines = run("1")
    assert any(ln.startswith("[ndft] ndft_plan N=4096 bins=128@-64") and "form=ternary" in ln for ln in lines)
    caf = [ln for ln in lines if ln.startswith("[ndft] caf_exec")]
    assert len(caf) == 1 and "variant=paired" in caf[0] and "status=0" in caf[0] and "cols=64" in caf[0]


def test_no_log_when_unset():
    assert run(None) == []
    assert run("0") == []
