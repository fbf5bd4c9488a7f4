"""The detection study of Sec. 5.2 on the stereo-FM scene (Table 3 geometry),
run through the CUDA library: the surfaces of Eq. 12a (NDFT on the tensor
cores, and through the NFFT) and Eq. 12b, read for detections.  Qualitative
outcomes that hold in every noise case of Tables 1-2, and the same reading
as the oracle's on one scene."""
import numpy as np
import pytest

import oracle
from paper_1402_0532_gb300 import detection, scenes

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def rows():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    return detection.fm_study(envs=("2t1c",), forms=("ternary", "nfft", "fft"), linear=False)


def test_eq12a_detects_every_obstacle(rows):
    assert [r["noise"] for r in rows] == ["awgn3", "awgn6", "eps0.9", "eps0.8"]
    for r in rows:
        # the NDFT form of Eq. 12a: both targets and the clutter, under AWGN and
        # under epsilon-contaminated noise alike
        assert all(r["ternary"]["detected"]), r
        assert r["ternary"]["floor_db"] < -3.0
        # through the NFFT both moving targets stand out
        assert r["nfft"]["detected"][:2] == [True, True], r
        assert all(r["fft"]["detected"]), r


def test_readings_match_the_oracle(rows):
    sc = scenes.fm_scene("2t1c", "eps0.9")
    p0 = -256
    # the NFFT form is bit-exact against the fp32 oracle
    want = detection.evaluate(np.abs(oracle.caf_nfft(sc.s_surv, sc.s_ref, 0, 64, p0, 512, f32=True)), 0, p0,
                              sc.obstacles)
    got = rows[2]["nfft"]
    assert got["detected"] == want["detected"]
    assert got["floor_db"] == pytest.approx(want["floor_db"], abs=1e-4)
    # the tensor-core NDFT against the fp64 NDFT oracle (lag product in fp32, as on the GPU)
    want = detection.evaluate(np.abs(oracle.caf(sc.s_surv, sc.s_ref, 0, 64, p0, 512, z32=True)), 0, p0,
                              sc.obstacles)
    got = rows[2]["ternary"]
    assert got["detected"] == want["detected"]
    assert got["floor_db"] == pytest.approx(want["floor_db"], abs=1e-3)
    np.testing.assert_allclose(got["peaks"], want["peaks"], rtol=1e-5)
