"""Seeded synthetic inputs for harmonic-sum workloads.

This module only *draws inputs*: exponential / chi-square noise power spectra, injected pulse
trains, drifting signals in an f-fdot plane and batches of uneven length.  It holds none of the
harmonic-sum arithmetic, so both the FP64 oracle (``oracle/``) and the CUDA path consume it
without sharing any of the method's code.

Signal model (input recipe, not the method):
  * noise: i.i.d. Exponential(1) power, i.e. |complex Gaussian|^2 with unit mean; for the f-fdot
    plane chi-square with 2 dof = 2 * Exponential(1);
  * a pulsar with fundamental ``f0`` (in bins, fractional) and duty cycle ``delta`` puts power
    ``A * exp(-(pi * delta * k)^2)`` (the power envelope of a Gaussian pulse of that duty cycle) at
    harmonic ``k``, in the bin nearest ``k * f0`` (numpy ``rint``: round half to even).

Host arrays are numpy float32; the device variants draw the noise with a seeded
``torch.Generator`` on the target device and add the same host-drawn pulsar parameters.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

SEED_BASE = 2202_12817


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


# --------------------------------------------------------------------------------------------
# pulsar descriptions
# --------------------------------------------------------------------------------------------
@dataclass(frozen=True)
class Pulsar:
    f0: float          # fundamental frequency in bins (fractional)
    duty: float        # duty cycle (fraction of the period)
    amplitude: float = 8.0

    def harmonic_bins_and_powers(self, n_bins: int):
        """Bins round(k*f0) < n_bins and the powers A*exp(-(pi*duty*k)^2) placed there."""
        if self.f0 <= 0:
            return np.zeros(0, np.int64), np.zeros(0, np.float64)
        kmax = int(math.floor((n_bins - 0.5) / self.f0)) + 1
        k = np.arange(1, kmax + 1, dtype=np.float64)
        bins = np.rint(k * self.f0).astype(np.int64)
        keep = (bins >= 0) & (bins < n_bins)
        k, bins = k[keep], bins[keep]
        powers = self.amplitude * np.exp(-(math.pi * self.duty * k) ** 2)
        return bins, powers


def random_pulsars(count: int, n_bins: int, seed: int, f_lo: float = 100.0,
                   f_hi: float | None = None, duty_lo: float = 0.02, duty_hi: float = 0.2,
                   amplitude: float = 8.0) -> list[Pulsar]:
    """``count`` pulsars with f0 ~ U[f_lo, f_hi) (default f_hi = n_bins/32), duty ~ U[duty_lo, duty_hi)."""
    g = rng(seed)
    if f_hi is None:
        f_hi = n_bins / 32.0
    f0 = g.uniform(f_lo, f_hi, size=count)
    duty = g.uniform(duty_lo, duty_hi, size=count)
    return [Pulsar(float(a), float(b), amplitude) for a, b in zip(f0, duty)]


def inject(x: np.ndarray, pulsars) -> np.ndarray:
    """Add each pulsar's harmonic powers to the host float32 spectrum ``x`` in place."""
    n = x.shape[0]
    for p in pulsars:
        bins, powers = p.harmonic_bins_and_powers(n)
        acc = np.zeros(bins.shape[0], np.float64)
        acc[:] = powers
        # float32 additions, one harmonic at a time, in ascending k (duplicates handled by add.at)
        np.add.at(x, bins, acc.astype(np.float32))
    return x


# --------------------------------------------------------------------------------------------
# 1D spectra
# --------------------------------------------------------------------------------------------
def exp_noise(n: int, seed: int) -> np.ndarray:
    return rng(seed).standard_exponential(int(n), dtype=np.float32)


def spectrum(n: int, seed: int, pulsars=()) -> np.ndarray:
    x = exp_noise(n, seed)
    return inject(x, pulsars)


def small_int_spectrum(n: int, seed: int, hi: int = 8) -> np.ndarray:
    """Integer powers 0..hi-1 as float32: sums stay exact in FP32 and ties are dense."""
    return rng(seed).integers(0, hi, size=int(n)).astype(np.float32)


# Workload recipes -----------------------------------------------------------------------------
CONFIG1_N = 131072
CONFIG1_PULSAR = Pulsar(1234.37, 0.05, 8.0)


def single_pulse_spectrum(seed: int = SEED_BASE + 1) -> np.ndarray:
    """N = 131072 Exponential(1) spectrum with the pulse train f0 = 1234.37 bins, duty 0.05, A = 8."""
    return spectrum(CONFIG1_N, seed, [CONFIG1_PULSAR])


LONG_N = 1 << 23


def long_spectrum_pulsars(seed: int = SEED_BASE + 2, n: int = LONG_N, count: int = 16):
    return random_pulsars(count, n, seed + 1000)


def long_spectrum(seed: int = SEED_BASE + 2, n: int = LONG_N) -> np.ndarray:
    """N = 2^23 Exponential(1) spectrum with 16 pulsars (f0 ~ U[100, N/32), duty ~ U[0.02, 0.2))."""
    return spectrum(n, seed, long_spectrum_pulsars(seed, n))


# --------------------------------------------------------------------------------------------
# uneven batches of DM-trial spectra
# --------------------------------------------------------------------------------------------
@dataclass
class Batch:
    lengths: np.ndarray               # int64 [B]
    offsets: np.ndarray               # int64 [B+1] element offsets (aligned)
    pulsar_of: dict = field(default_factory=dict)   # trial -> Pulsar
    seed: int = 0
    ids: np.ndarray | None = None     # trial k draws the noise of trial ids[k] of the full batch

    @property
    def total(self) -> int:
        return int(self.offsets[-1])

    def trial_id(self, k: int) -> int:
        return int(self.ids[k]) if self.ids is not None else int(k)


def sub_batch(b: Batch, indices) -> Batch:
    """Trials ``indices`` of ``b`` packed in that order (a rank's shard): trial k of the result
    holds exactly trial indices[k] of ``b`` (same noise seed, same pulsar)."""
    ids = np.asarray(indices, np.int64)
    lengths = np.asarray(b.lengths, np.int64)[ids]
    pulsar_of = {k: b.pulsar_of[int(i)] for k, i in enumerate(ids) if int(i) in b.pulsar_of}
    src = np.array([b.trial_id(int(i)) for i in ids], np.int64)
    return Batch(lengths, pack_offsets(lengths), pulsar_of, b.seed, src)


def pack_offsets(lengths, align: int = 32) -> np.ndarray:
    """Concatenation offsets, each spectrum starting at a multiple of ``align`` elements."""
    lengths = np.asarray(lengths, np.int64)
    off = np.zeros(lengths.shape[0] + 1, np.int64)
    pos = 0
    for i, n in enumerate(lengths):
        start = -(-pos // align) * align
        off[i] = start
        pos = start + int(n)
    off[-1] = pos      # total extent: end of the last spectrum (no trailing padding)
    return off


def uneven_batch(count: int = 2048, seed: int = SEED_BASE + 3,
                 choices=(1 << 20, 1 << 21, 1 << 22, 1 << 23), pulsar_fraction: float = 0.05,
                 align: int = 32) -> Batch:
    """Lengths drawn uniformly from ``choices``; ``pulsar_fraction`` of the trials carry one pulsar."""
    g = rng(seed)
    lengths = g.choice(np.asarray(choices, np.int64), size=count)
    n_pulsar = int(round(pulsar_fraction * count))
    with_pulsar = g.choice(count, size=n_pulsar, replace=False) if n_pulsar else []
    pulsar_of = {}
    for i in sorted(int(t) for t in with_pulsar):
        pulsar_of[i] = random_pulsars(1, int(lengths[i]), seed + 7919 * (i + 1))[0]
    return Batch(lengths, pack_offsets(lengths, align), pulsar_of, seed)


def batch_trial(b: Batch, i: int) -> np.ndarray:
    """Host copy of trial ``i`` of a batch (noise seeded per trial, plus its pulsar if any)."""
    p = [b.pulsar_of[i]] if i in b.pulsar_of else []
    return spectrum(int(b.lengths[i]), b.seed * 4099 + b.trial_id(i), p)


def batch_host(b: Batch) -> np.ndarray:
    out = np.zeros(b.total, np.float32)
    for i in range(b.lengths.shape[0]):
        out[b.offsets[i]:b.offsets[i] + b.lengths[i]] = batch_trial(b, i)
    return out


# --------------------------------------------------------------------------------------------
# device-side generation (large workloads): torch is only the random source and the container
# --------------------------------------------------------------------------------------------
def _torch():
    import torch
    return torch


def device_noise(n: int, seed: int, device, scale: float = 1.0, out=None):
    torch = _torch()
    g = torch.Generator(device=device)
    g.manual_seed(int(seed) & 0x7FFFFFFFFFFFFFFF)
    t = out if out is not None else torch.empty(int(n), dtype=torch.float32, device=device)
    t.exponential_(1.0, generator=g)
    if scale != 1.0:
        t.mul_(scale)
    return t


def device_inject(t, pulsars, base: int = 0):
    """Add pulsar powers to a device float32 view ``t`` (bins relative to ``base``)."""
    torch = _torch()
    n = t.shape[0]
    for p in pulsars:
        bins, powers = p.harmonic_bins_and_powers(n)
        if bins.size == 0:
            continue
        idx = torch.from_numpy(bins + base).to(t.device)
        val = torch.from_numpy(powers.astype(np.float32)).to(t.device)
        t.index_add_(0, idx - base, val)
    return t


def device_spectrum(n: int, seed: int, pulsars, device):
    t = device_noise(n, seed, device)
    return device_inject(t, pulsars)


def device_batch(b: Batch, device, dtype=None):
    """Whole uneven batch on the device: per-trial seeded noise + pulsars, packed at ``b.offsets``."""
    torch = _torch()
    out = torch.zeros(b.total, dtype=torch.float32, device=device)
    for i in range(b.lengths.shape[0]):
        view = out[int(b.offsets[i]):int(b.offsets[i]) + int(b.lengths[i])]
        device_noise(view.shape[0], b.seed * 4099 + b.trial_id(i), device, out=view)
        if i in b.pulsar_of:
            device_inject(view, [b.pulsar_of[i]])
    return out if dtype is None else out.to(dtype)


# --------------------------------------------------------------------------------------------
# f-fdot plane (2D)
# --------------------------------------------------------------------------------------------
@dataclass(frozen=True)
class Track:
    f0: float       # fundamental frequency bin (fractional)
    z0: int         # fdot row offset of the fundamental (rows are z = -z0_row..)
    amplitude: float = 8.0
    duty: float = 0.05


def random_tracks(count: int, n_freq: int, seed: int, f_lo: float = 1000.0,
                  f_hi: float | None = None, zmax: int = 11) -> list[Track]:
    g = rng(seed)
    if f_hi is None:
        f_hi = (n_freq - 1 - 8) / 8.0
    f0 = g.uniform(f_lo, f_hi, size=count)
    z0 = g.integers(-zmax, zmax + 1, size=count)
    return [Track(float(a), int(b)) for a, b in zip(f0, z0)]


def track_points(tr: Track, n_freq: int, n_rows: int, z0_row: int, kmax: int = 8):
    """(row, col, power) triples of a drifting signal: harmonic k is centred at (k*z0, k*f0) and
    smeared along u in [-k, k] rows with weight exp(-(u/k)^2), its column sliding by u/2."""
    rows, cols, vals = [], [], []
    for k in range(1, kmax + 1):
        a_k = tr.amplitude * math.exp(-(math.pi * tr.duty * k) ** 2)
        for u in range(-k, k + 1):
            r = z0_row + k * tr.z0 + u
            c = int(np.rint(k * tr.f0 + 0.5 * u))
            if 0 <= r < n_rows and 0 <= c < n_freq:
                rows.append(r)
                cols.append(c)
                vals.append(a_k * math.exp(-(u / k) ** 2))
    return np.asarray(rows, np.int64), np.asarray(cols, np.int64), np.asarray(vals, np.float64)


def plane(n_freq: int, n_rows: int, z0_row: int, seed: int, tracks=()) -> np.ndarray:
    """Host chi-square(2) f-fdot plane [n_rows][n_freq] (row-major, f contiguous) with tracks."""
    p = rng(seed).standard_exponential((int(n_rows), int(n_freq)), dtype=np.float32)
    p *= np.float32(2.0)
    for tr in tracks:
        r, c, v = track_points(tr, n_freq, n_rows, z0_row)
        np.add.at(p, (r, c), v.astype(np.float32))
    return p


def device_plane(n_freq: int, n_rows: int, z0_row: int, seed: int, tracks, device):
    torch = _torch()
    t = torch.empty(int(n_rows) * int(n_freq), dtype=torch.float32, device=device)
    device_noise(t.shape[0], seed, device, scale=2.0, out=t)
    for tr in tracks:
        r, c, v = track_points(tr, n_freq, n_rows, z0_row)
        if r.size:
            idx = torch.from_numpy(r * n_freq + c).to(device)
            t.index_add_(0, idx, torch.from_numpy(v.astype(np.float32)).to(device))
    return t.view(int(n_rows), int(n_freq))


PLANE_N_FREQ = 1 << 21
PLANE_N_ROWS = 201
PLANE_Z0_ROW = 100


# --------------------------------------------------------------------------------------------
# whitening / gradient inputs
# --------------------------------------------------------------------------------------------
def whitening(n: int, seed: int | None = None, lo: float = 0.5, hi: float = 1.5) -> np.ndarray:
    """Per-bin whitening weights: ones when ``seed`` is None, else U[lo, hi)."""
    if seed is None:
        return np.ones(int(n), np.float32)
    return rng(seed).uniform(lo, hi, size=int(n)).astype(np.float32)


def upstream_grad(n: int, seed: int) -> np.ndarray:
    """A seeded dL/dSNR vector (standard normal) for adjoint tests."""
    return rng(seed).standard_normal(int(n)).astype(np.float32)
