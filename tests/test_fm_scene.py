"""The stereo-FM scene of Sec. 5 (Eq. 11-16, Table 3) and the detection reading
of Tables 1-2: closed forms, the echo model and the noise statistics (CPU)."""
import numpy as np
import pytest

from paper_1402_0532_gb300 import detection, scenes


def test_message_closed_form_eq11():
    t = np.array([0.0, 1.0 / (4 * scenes.PILOT_HZ), 1.0 / scenes.PILOT_HZ])
    z = np.zeros(3)
    # x1 = x2 = 0: only the 3 f_p and f_p tones
    want = 0.25 * np.cos(2 * np.pi * 3 * scenes.PILOT_HZ * t) + 0.1 * np.cos(2 * np.pi * scenes.PILOT_HZ * t)
    np.testing.assert_allclose(scenes.fm_stereo_message(z, z, t), want, atol=1e-15)
    # x1 = 1, x2 = -1 at t = 0: 0.5 * 2 on the subcarrier + 0.25 + 0.1
    assert scenes.fm_stereo_message(np.ones(1), -np.ones(1), np.zeros(1))[0] == pytest.approx(1.35)
    # x1 = x2 = 1 at a quarter pilot period: 1.8 + 0.5 * 0 * cos(pi) + 0.25 cos(3 pi / 2) + 0.1 cos(pi / 2)
    assert scenes.fm_stereo_message(np.ones(1), np.ones(1), t[1:2])[0] == pytest.approx(1.8, abs=1e-12)


def test_fm_signal_eq12_unit_modulus_and_phase():
    rng = np.random.default_rng(3)
    s = scenes.fm_stereo(rng, 4096, kf=0.5)
    np.testing.assert_allclose(np.abs(s), 1.0, atol=1e-12)
    # the phase is 2 pi k_f m: redraw the same channel data and compare
    rng = np.random.default_rng(3)
    x1, x2 = rng.uniform(-1, 1, 4096), rng.uniform(-1, 1, 4096)
    m = scenes.fm_stereo_message(x1, x2, np.arange(4096) / scenes.FS_HZ)
    np.testing.assert_allclose(s, np.exp(1j * np.pi * m), atol=1e-12)


def test_bistatic_delays_table3():
    # excess paths sqrt(200), sqrt(500) + 10, sqrt(28^2 + 23^2) + sqrt(28^2 + 33^2) - 10 km
    paths = [np.sqrt(200.0), np.sqrt(500.0) + 10.0, np.hypot(28, 23) + np.hypot(28, 33) - 10.0]
    for (x, y, _), km in zip(scenes.FM_ENVIRONMENTS["2t1c"], paths):
        assert scenes.bistatic_delay_samples(x, y) == pytest.approx(km / 299792.458 * 200e3, rel=1e-12)
    d = [int(round(scenes.bistatic_delay_samples(x, y))) for x, y, _ in scenes.FM_ENVIRONMENTS["2t1c"]]
    assert d == [9, 22, 46]


@pytest.mark.parametrize("eps,s1,s2", [(0.9, 0.25, 10.0), (0.8, 0.5, 20.0)])
def test_eps_contaminated_statistics(eps, s1, s2):
    rng = np.random.default_rng(5)
    n = 1_000_000
    v = scenes.eps_contaminated(rng, n, eps, s1, s2)
    var = eps * s1 ** 2 + (1 - eps) * s2 ** 2
    assert abs(v.mean()) < 5 * np.sqrt(var / n)
    assert v.var() == pytest.approx(var, rel=0.01)
    # outliers: the share beyond 5 s1 is (1 - eps) P(|N(0, s2^2)| > 5 s1) (nominal part ~ 6e-7)
    from math import erf, sqrt
    tail = (1 - eps) * (1 - erf(5 * s1 / s2 / sqrt(2)))
    assert np.mean(np.abs(v) > 5 * s1) == pytest.approx(tail, rel=0.02)


@pytest.mark.parametrize("env", ["2t1c", "4t2c", "1t3c"])
def test_scene_echo_model_eq16(env):
    """s_surv / gain minus the echoes of Eq. 13 / 16 leaves exactly the noise
    (AWGN at 3 dB: power 10^-0.3 per complex sample)."""
    N = 8192
    sc = scenes.fm_scene(env, "awgn3", N=N, seed=21)
    rng = np.random.default_rng(21)
    s = scenes.fm_stereo(rng, N + 64, sc.kf, t0=-64)
    np.testing.assert_allclose(sc.s_ref, s[64:], atol=1e-6)
    t = np.arange(N) / scenes.FS_HZ
    echoes = sum(s[64 - d: 64 - d + N] * np.exp(2j * np.pi * fd * t) for d, fd, _, _ in sc.obstacles)
    resid = sc.s_surv / sc.gain - echoes
    assert np.mean(np.abs(resid) ** 2) == pytest.approx(10 ** -0.3, rel=0.05)
    kinds = [k for _, _, _, k in sc.obstacles]
    assert kinds.count("target") == int(env[0]) and kinds.count("clutter") == int(env[2])
    assert all(0 <= d < 64 for d, _, _, _ in sc.obstacles)


def test_detection_reading():
    A = np.ones((16, 32))
    obstacles = [(3, 0.0, 2.0, "target"), (10, 0.0, -5.0, "clutter")]  # p0 = -8: columns 10 and 3
    A[3, 10] = 8.0
    A[10, 4] = 4.0     # inside the second window (column 3 +- 2)
    A[14, 30] = 5.0    # the largest side lobe
    r = detection.evaluate(A, 0, -8, obstacles)
    assert r["peaks"] == [8.0, 4.0] and r["sidelobe"] == 5.0
    assert r["detected"] == [True, False] and r["masked"] == ["clutter"]
    assert r["floor_db"] == pytest.approx(20 * np.log10(5.0 / 8.0))
    # a side lobe inside a window does not count as a side lobe
    A[14, 30] = 1.0
    A[2, 12] = 7.0
    r = detection.evaluate(A, 0, -8, obstacles)
    assert r["sidelobe"] == 1.0 and r["detected"] == [True, True]
