"""Sensitivity loss of the harmonic sums to where a pulsar's frequency falls within a frequency bin.

The experiment of the paper's Sec. 4.1 ("Artificial data without noise"): a pulse train from the
modified von Mises distribution (Eq. 10), sampled for T = 20 s at t_s = 64 us (bin width
W_f = 1/T = 0.05 Hz), its power spectrum, and the harmonic sum at the pulsar's fundamental; the
pulsar frequency steps from the centre of bin n0 to the centre of bin n0 + 1 in 50 steps, and the
sensitivity loss of a form is l(f) = RSNR(f) / RSNR(f at the centre of n0) (Eq. 11).

This is a harness around the hot path: the time series and the FFT run in torch on the GPU; every
harmonic sum (simple, greedy and the optimal form) runs in libhs.  The recovered SNR (RSNR) of a
form at frequency f is its largest SNR over the fundamentals n0 and n0 + 1 (the two bins the
pulsar's fundamental occupies across the sweep), with SNR_h = S_h / sqrt(h): the data are
noise-free, so the normalisation only has to grow like an h-term sum's noise; l(f) is a ratio and
does not depend on its scale.

    python -m paper_2202_12817_gb300.sensitivity      # prints the loss table (needs a GPU)
"""
from __future__ import annotations

import math

import numpy as np

T_OBS = 20.0          # s
T_SAMP = 64e-6        # s
STEPS = 50
KAPPA = 88.0          # von Mises shape: 4 % duty cycle (FWHM), ~30 harmonics above 1e-4 of the first


def von_mises_series(f_r: float, n: int, t_samp: float = T_SAMP, kappa: float = KAPPA, amplitude: float = 1.0,
                     phase: float = 0.0, xp=np, device=None):
    """Eq. 10: a (exp(k cos(2 pi f_r t + phi)) - exp(-k)) / (I0(k) - exp(-k)), t = 0, t_s, ...
    Evaluated in float64 (numpy, or torch when ``xp`` is torch) and returned as float64."""
    i0 = float(np.i0(kappa))
    if xp is np:
        t = np.arange(n, dtype=np.float64) * t_samp
        return amplitude * (np.exp(kappa * np.cos(2 * np.pi * f_r * t + phase)) - math.exp(-kappa)) / (i0 - math.exp(-kappa))
    torch = xp
    t = torch.arange(n, dtype=torch.float64, device=device) * t_samp
    return amplitude * (torch.exp(kappa * torch.cos(2 * math.pi * f_r * t + phase)) - math.exp(-kappa)) / (
        i0 - math.exp(-kappa))


def sweep_frequencies(n0: int, steps: int = STEPS, t_obs: float = T_OBS):
    """Pulsar frequencies from the centre of bin n0 to the centre of bin n0 + 1 (steps + 1 values)."""
    w = 1.0 / t_obs
    return [(n0 + i / steps) * w for i in range(steps + 1)]


def unit_norm(H: int):
    """mu_h = 0, sigma_h = sqrt(h): SNR_h = S_h / sqrt(h)."""
    return np.zeros(H, np.float32), np.sqrt(np.arange(1, H + 1, dtype=np.float64)).astype(np.float32)


def loss_curves(n0: int = 2000, H: int = 32, steps: int = STEPS, device: int = 0, kappa: float = KAPPA):
    """RSNR and sensitivity loss of the simple, greedy and optimal forms across one bin, on the GPU.
    Returns {"freq_hz": [...], "offset_bins": [...], form_name: {"rsnr": [...], "loss": [...]}}."""
    import torch

    from . import GREEDY, OPTIMAL, SIMPLE, Plan

    dev = torch.device("cuda", device)
    n = int(round(T_OBS / T_SAMP))
    nbins = n // 2 + 1
    plan = Plan(H, SIMPLE | GREEDY | OPTIMAL, lengths=[nbins], device=device)
    mu, sg = (torch.from_numpy(a).to(dev) for a in unit_norm(H))
    norm = (mu, sg)
    freqs = sweep_frequencies(n0, steps)
    out = {"freq_hz": freqs, "offset_bins": [i / steps for i in range(steps + 1)]}
    names = {SIMPLE: "simple", GREEDY: "greedy", OPTIMAL: "optimal"}
    rs = {f: [] for f in names}
    for f_r in freqs:
        x = von_mises_series(f_r, n, xp=torch, device=dev)
        p = (torch.fft.rfft(x).abs() ** 2 / n).float().contiguous()
        res = plan.forward(p, norm, norm, optimal_norm=norm, path=False, argmax=False)
        for f in names:
            snr = res[f].snr[n0:n0 + 2]
            rs[f].append(float(snr.max().item()))
    plan.close()
    for f, name in names.items():
        r = np.asarray(rs[f])
        out[name] = {"rsnr": r.tolist(), "loss": (r / r[0]).tolist()}
    return out


def main():
    res = loss_curves()
    print("offset  " + "  ".join(f"{k:>8s}" for k in ("simple", "greedy", "optimal")))
    for i, off in enumerate(res["offset_bins"]):
        print(f"{off:6.2f}  " + "  ".join(f"{res[k]['loss'][i]:8.4f}" for k in ("simple", "greedy", "optimal")))
    for k in ("simple", "greedy", "optimal"):
        print(f"{k}: largest loss {1 - min(res[k]['loss']):.3f}")


if __name__ == "__main__":
    main()
