"""Seeded synthetic inputs shared by the tests, the smoke check and the benchmark.

This module only draws numbers; it holds none of the transform's arithmetic.
The paper's own scene (a stereo-FM broadcast, Sec. 5, Eq. 13-16) leaves the
modulation index, the channel data and the integration length unstated, so
the radar workloads below stand in for it with band-limited complex noise as
the illuminator, delayed and Doppler-shifted echoes (the echo model of
Eq. 15-16) and additive complex Gaussian noise.  All randomness comes from
``numpy.random.default_rng`` (PCG64) with the stated seeds.

Workloads (sizes and seeds):

* ``tone_batch``      -- 4096 vectors of N = 64: vector 0 is exp(j 2 pi 7 n / 64)
                         with exact values on the axes, the rest CN(0, 1), seed 0.
* ``cn_batch``        -- 65536 vectors of N = 1024, CN(0, 1), seed 1.
* ``radar_scene``     -- N = 65536, band-limited reference (|f| <= 0.4 fs),
                         echoes at delays 37/120/301 samples, Doppler bins
                         5/-12/40, levels -20/-30/-35 dB, noise power 10, seed 2.
* ``cpi_batch``       -- 256 scenes with N_c ~ U{1024..32768}, L_c ~ U{64..1024},
                         1024 Doppler bins, one child seed of SeedSequence(3) each.
* ``radar_scene(N=16384, seed=4)`` -- the differentiation workload.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

Q14_ONE = 1 << 14


def cn(rng: np.random.Generator, shape) -> np.ndarray:
    """Circular complex normal CN(0, 1): (N(0,1) + j N(0,1)) / sqrt(2), complex128."""
    g = rng.standard_normal(tuple(shape) + (2,))
    return (g[..., 0] + 1j * g[..., 1]) / np.sqrt(2.0)


def exact_tone(N: int, k0: int) -> np.ndarray:
    """exp(+j 2 pi k0 n / N), n < N, with the angle reduced to a quadrant in
    integers so that samples on the axes are exactly 0 / +-1 (complex128)."""
    n = np.arange(N, dtype=np.int64)
    m = (k0 * n) % N
    u = 4 * m
    q = u // N
    r = u - q * N
    a = (np.pi / 2) * (r / N)
    c, s = np.cos(a), np.sin(a)
    ct = np.select([q == 0, q == 1, q == 2], [c, -s, -c], s)
    st = np.select([q == 0, q == 1, q == 2], [s, c, -s], -c)
    return (ct + 0.0) + 1j * (st + 0.0)


def tone_batch(batch: int = 4096, N: int = 64, k0: int = 7, seed: int = 0) -> np.ndarray:
    """complex64 [batch, N]: row 0 the exact tone at bin k0, rows 1.. CN(0, 1)."""
    rng = np.random.default_rng(seed)
    x = cn(rng, (batch, N))
    x[0] = exact_tone(N, k0)
    return x.astype(np.complex64)


def cn_batch(batch: int = 65536, N: int = 1024, seed: int = 1) -> np.ndarray:
    """complex64 [batch, N] of CN(0, 1)."""
    rng = np.random.default_rng(seed)
    return cn(rng, (batch, N)).astype(np.complex64)


@dataclass
class Scene:
    s_surv: np.ndarray  # complex64 [N]
    s_ref: np.ndarray   # complex64 [N]
    N: int
    lag0: int
    nlags: int
    p0: int
    nbins: int
    delays: tuple
    dopplers: tuple


def bandlimited_reference(rng: np.random.Generator, N: int, frac: float = 0.4) -> np.ndarray:
    """CN(0,1) noise, spectrum zeroed where |f| > frac * fs, renormalised to unit power."""
    s = cn(rng, (N,))
    S = np.fft.fft(s)
    f = np.fft.fftfreq(N)
    S[np.abs(f) > frac] = 0.0
    s = np.fft.ifft(S)
    return s / np.sqrt(np.mean(np.abs(s) ** 2))


def radar_scene(N: int = 65536, seed: int = 2, nlags: int = 1024, nbins: int = 1024,
                delays=(37, 120, 301), dopplers=(5, -12, 40), levels_db=(-20.0, -30.0, -35.0),
                noise_power: float = 10.0, rng: np.random.Generator | None = None) -> Scene:
    """Direct path (delay 0, 0 dB) plus delayed, Doppler-shifted echoes plus CN noise
    (the surveillance model of Eq. 15-16 with a noise-free reference, Sec. 5.2)."""
    rng = np.random.default_rng(seed) if rng is None else rng
    s_ref = bandlimited_reference(rng, N)
    i = np.arange(N, dtype=np.int64)
    s_surv = s_ref.copy()
    for d, fd, lv in zip(delays, dopplers, levels_db):
        a = 10.0 ** (lv / 20.0)
        delayed = np.zeros(N, np.complex128)
        if d < N:
            delayed[d:] = s_ref[: N - d]
        phase = np.exp(2j * np.pi * ((fd * i) % N) / N)
        s_surv = s_surv + a * delayed * phase
    s_surv = s_surv + np.sqrt(noise_power) * cn(rng, (N,))
    return Scene(s_surv.astype(np.complex64), s_ref.astype(np.complex64), N, 0, nlags,
                 -(nbins // 2), nbins, tuple(delays), tuple(dopplers))


def cpi_batch(n_cpi: int = 256, seed: int = 3, nbins: int = 1024, n_range=(1024, 32768),
              lag_range=(64, 1024)) -> list[Scene]:
    """Uneven CPIs: per CPI c the child seed SeedSequence(seed).spawn(n_cpi)[c] draws
    N_c, L_c and then the scene itself."""
    kids = np.random.SeedSequence(seed).spawn(n_cpi)
    out = []
    for c in range(n_cpi):
        rng = np.random.default_rng(kids[c])
        N = int(rng.integers(n_range[0], n_range[1], endpoint=True))
        L = int(rng.integers(lag_range[0], lag_range[1], endpoint=True))
        out.append(radar_scene(N=N, nlags=L, nbins=nbins, rng=rng))
    return out


def quantize_q14(v: np.ndarray, scale: float = 1.0) -> np.ndarray:
    """Q1.14: int16 pairs [..., 2] = clamp(round-half-even(2^14 scale v), -32768, 32767)."""
    v = np.asarray(v) * scale
    q = np.stack([v.real, v.imag], axis=-1) * Q14_ONE
    return np.clip(np.rint(q), -32768, 32767).astype(np.int16)


def differentiation_mask(scene: Scene, half: int = 16) -> np.ndarray:
    """Boolean [nlags, nbins] mask, 2*half x 2*half, centred on the first echo."""
    m = np.zeros((scene.nlags, scene.nbins), bool)
    l0 = scene.delays[0] - scene.lag0 - half
    b0 = scene.dopplers[0] - scene.p0 - half
    m[max(l0, 0):l0 + 2 * half, max(b0, 0):b0 + 2 * half] = True
    return m


# ---------------------------------------------------------------------------
# The paper's own scene (Sec. 5): a stereo-FM illuminator, Eq. 11-12, echoes
# of targets and clutter placed by a bistatic geometry (Eq. 13-16, Table 3),
# additive white Gaussian or epsilon-contaminated Gaussian noise, s_ref noise
# free.  Quantities the paper leaves open are fixed here and listed with the
# scene: the distribution of the channel data x1, x2 (i.i.d. uniform on
# [-1, 1] per sample), the modulation index k_f (0.5), the CPI length
# (65536 samples), integer-sample delays (the bistatic delay rounded to the
# nearest sample at fs), the SNR reference (noise power relative to one echo
# of unit power), and the positions of the obstacles beyond Table 3.
# ---------------------------------------------------------------------------
FS_HZ = 200e3        # sampling frequency (Sec. 5)
PILOT_HZ = 19e3      # stereo pilot f_p (Eq. 11)
C_KM_S = 299792.458  # propagation speed
TX_KM = (0.0, 10.0)  # Table 3
RX_KM = (0.0, 0.0)

# (x km, y km, Doppler Hz); clutter has Doppler 0.  "2t1c" is Table 3; the other
# two environments of Tables 1-2 have no published geometry and are chosen here.
FM_ENVIRONMENTS = {
    "2t1c": [(10.0, 0.0, 200.0), (20.0, 0.0, 157.0), (28.0, 33.0, 0.0)],
    "4t2c": [(10.0, 0.0, 200.0), (20.0, 0.0, 157.0), (6.0, -18.0, -120.0), (5.0, 12.0, 80.0),
             (28.0, 33.0, 0.0), (-12.0, 20.0, 0.0)],
    "1t3c": [(10.0, 0.0, 200.0), (28.0, 33.0, 0.0), (-12.0, 20.0, 0.0), (-20.0, -5.0, 0.0)],
}

# noise cases of Tables 1-2: AWGN at an SNR in dB, or epsilon-contaminated
# Gaussian (eps, sigma1, sigma2)
FM_NOISES = {"awgn3": ("awgn", 3.0), "awgn6": ("awgn", 6.0),
             "eps0.9": ("eps", (0.9, 0.25, 10.0)), "eps0.8": ("eps", (0.8, 0.5, 20.0))}


def fm_stereo_message(x1: np.ndarray, x2: np.ndarray, t: np.ndarray) -> np.ndarray:
    """Eq. 11: sum / difference channels, the difference on the 2 f_p subcarrier,
    plus the 3 f_p and f_p tones."""
    fp = PILOT_HZ
    return (0.9 * (x1 + x2) + 0.5 * (x1 - x2) * np.cos(2 * np.pi * 2 * fp * t)
            + 0.25 * np.cos(2 * np.pi * 3 * fp * t) + 0.1 * np.cos(2 * np.pi * fp * t))


def fm_stereo(rng: np.random.Generator, n: int, kf: float = 0.5, t0: int = 0) -> np.ndarray:
    """Eq. 12: s = cos(2 pi k_f m) + j sin(2 pi k_f m) at fs, samples t0 .. t0 + n - 1
    (complex128, unit modulus).  x1, x2 i.i.d. uniform on [-1, 1]."""
    t = (t0 + np.arange(n)) / FS_HZ
    x1 = rng.uniform(-1.0, 1.0, n)
    x2 = rng.uniform(-1.0, 1.0, n)
    return np.exp(1j * 2 * np.pi * kf * fm_stereo_message(x1, x2, t))


def bistatic_delay_samples(x_km: float, y_km: float) -> float:
    """Excess path |Tx P| + |P Rx| - |Tx Rx| over the propagation speed, in samples at fs."""
    d = lambda a, b: float(np.hypot(a[0] - b[0], a[1] - b[1]))
    p = (x_km, y_km)
    return (d(TX_KM, p) + d(p, RX_KM) - d(TX_KM, RX_KM)) / C_KM_S * FS_HZ


def eps_contaminated(rng: np.random.Generator, n: int, eps: float, s1: float, s2: float) -> np.ndarray:
    """Real samples of the mixture eps N(0, s1^2) + (1 - eps) N(0, s2^2): each sample
    is nominal with probability eps and an outlier otherwise."""
    nominal = rng.random(n) < eps
    return np.where(nominal, rng.normal(0.0, s1, n), rng.normal(0.0, s2, n))


@dataclass
class FMScene:
    s_surv: np.ndarray  # complex64 [N], the input gain applied
    s_ref: np.ndarray   # complex64 [N], noise free
    N: int
    obstacles: list     # (delay samples, Doppler Hz, Doppler bin p = f N / fs, "target" | "clutter")
    gain: float
    kf: float
    noise: str


def fm_scene(env: str = "2t1c", noise: str = "eps0.9", N: int = 65536, kf: float = 0.5, gain: float = 64.0,
             seed: int = 9) -> FMScene:
    """Eq. 16: s_surv = sum_m K s_ref(t - tau_m) exp(j 2 pi f_m t) + noise, K = 1, scaled by
    `gain` (the x64 input level of Sec. 5.2); s_ref = s(t) of Eq. 12 without noise.  The
    illuminator is drawn for the 64 samples before the CPI as well, so that every echo
    has a full record."""
    rng = np.random.default_rng(seed)
    pre = 64
    s = fm_stereo(rng, N + pre, kf, t0=-pre)
    s_ref = s[pre:]
    t = np.arange(N) / FS_HZ
    s_surv = np.zeros(N, np.complex128)
    obstacles = []
    for x, y, fd in FM_ENVIRONMENTS[env]:
        d = int(round(bistatic_delay_samples(x, y)))
        assert 0 <= d < pre
        s_surv += s[pre - d: pre - d + N] * np.exp(2j * np.pi * fd * t)
        obstacles.append((d, fd, fd * N / FS_HZ, "clutter" if fd == 0.0 else "target"))
    kind, par = FM_NOISES[noise]
    if kind == "awgn":
        pw = 10.0 ** (-par / 10.0)
        s_surv += np.sqrt(pw) * cn(rng, (N,))
    else:
        s_surv += eps_contaminated(rng, N, *par) + 1j * eps_contaminated(rng, N, *par)
    return FMScene((gain * s_surv).astype(np.complex64), s_ref.astype(np.complex64), N, obstacles, gain, kf,
                   noise)
