"""Target detection on an ambiguity surface and the robustness study of Sec. 5.2.

The paper reads targets and clutter off the peaks of |A| (Fig. 3-6) and
reports, per environment and noise case, whether every obstacle was detected
and a side-lobe floor in dB (Tables 1-2) without defining either.  Here:

* an obstacle's window is its delay +- 1 lag and its Doppler bin (f N / fs,
  rounded) +- 2 bins; its peak is the largest |A| inside the window;
* the side-lobe level is the largest |A| outside every obstacle window;
* an obstacle is detected when its peak exceeds the side-lobe level,
  masked otherwise;
* side-lobe floor = 20 log10(side-lobe level / largest obstacle peak) dB.

The study runs each surface through the CUDA library (the paper's forms of
Eq. 12a and Eq. 12b); the linear cross-ambiguity function of Eq. 11, the
paper's point of comparison, is formed with torch.fft for context only.
"""
from __future__ import annotations

import numpy as np


def evaluate(Amag: np.ndarray, lag0: int, p0: int, obstacles, lag_half: int = 1, bin_half: int = 2) -> dict:
    """Detection reading of |A| ([nlags, nbins], lags lag0.., bins p0..) for the
    obstacles (delay, Doppler Hz, Doppler bin, kind) of a scene."""
    A = np.asarray(Amag, dtype=np.float64)
    nl, nb = A.shape
    outside = np.ones(A.shape, bool)
    peaks = []
    for d, _, pb, _ in obstacles:
        r0, r1 = max(d - lag_half - lag0, 0), min(d + lag_half - lag0 + 1, nl)
        c = int(round(pb)) - p0
        c0, c1 = max(c - bin_half, 0), min(c + bin_half + 1, nb)
        if r0 >= r1 or c0 >= c1:
            raise ValueError("obstacle outside the surface")
        peaks.append(float(A[r0:r1, c0:c1].max()))
        outside[r0:r1, c0:c1] = False
    side = float(A[outside].max())
    detected = [p > side for p in peaks]
    return {"peaks": peaks, "sidelobe": side, "detected": detected,
            "masked": [o[3] for o, ok in zip(obstacles, detected) if not ok],
            "floor_db": 20.0 * np.log10(side / max(peaks)) if max(peaks) > 0 else float("inf")}


def linear_caf(s_surv, s_ref, nlags: int, p0: int, nbins: int):
    """Eq. 11 (torch tensors on one device): A[l][p] = sum_i s_surv[i] conj(s_ref[i - l])
    W^(i p), lags 0 .. nlags - 1, by torch.fft.  Comparison only."""
    import torch
    N = s_surv.numel()
    Z = torch.zeros(nlags, N, dtype=s_surv.dtype, device=s_surv.device)
    for l in range(nlags):
        Z[l, l:] = s_surv[l:] * torch.conj(s_ref[:N - l])
    X = torch.fft.fft(Z, dim=1)
    idx = (p0 + torch.arange(nbins, device=s_surv.device)) % N
    return X[:, idx]


def fm_study(envs=("2t1c", "4t2c", "1t3c"), noises=("awgn3", "awgn6", "eps0.9", "eps0.8"), N: int = 65536,
             nlags: int = 64, nbins: int = 512, forms=("ternary", "nfft", "fft"), linear: bool = True,
             seed: int = 9, device=None) -> list[dict]:
    """The Table 1-2 grid on the stereo-FM scene: for every environment and noise
    case, the surface of each form (Eq. 12a on the tensor cores or through the
    NFFT, Eq. 12b) over lags 0 .. nlags - 1 and the nbins centred Doppler bins,
    read by `evaluate`."""
    import torch

    from . import api, scenes
    dev = torch.device("cuda", torch.cuda.current_device()) if device is None else device
    p0 = -(nbins // 2)
    precs = {"ternary": "bf16x2", "direct": "fp32", "nfft": "fp32", "fft": "fp32"}
    plans = {f: api.Plan(N, p0=p0, nbins=nbins, max_lags=nlags, form=f, prec=precs[f], device=dev) for f in forms}
    rows = []
    for env in envs:
        for noise in noises:
            sc = scenes.fm_scene(env, noise, N=N, seed=seed)
            ss = torch.from_numpy(sc.s_surv).to(dev)
            sr = torch.from_numpy(sc.s_ref).to(dev)
            out = {"env": env, "noise": noise}
            for f, plan in plans.items():
                A = plan.caf(ss, sr, 0, nlags)
                out[f] = evaluate(A.abs().cpu().numpy(), 0, p0, sc.obstacles)
            if linear:
                out["linear"] = evaluate(linear_caf(ss, sr, nlags, p0, nbins).abs().cpu().numpy(), 0, p0,
                                         sc.obstacles)
            rows.append(out)
    for plan in plans.values():
        plan.query_error()
    return rows
