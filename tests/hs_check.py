"""Shared helpers of the GPU parity tests: run the CUDA path through the C ABI and compare it
with the FP64 oracle.

Comparison rules:
  * drift paths: bit-exact (comparisons are on stored values, exact in every dtype);
  * SNR: |snr_gpu - snr_ref| <= RTOL * (|S_ref| + |mu_h|) / sigma_h at the reference best h,
    i.e. 1e-5 relative to the un-cancelled magnitude (S_ref = snr_ref * sigma_h + mu_h);
  * best h and argmax: exact, except where the two competing reference SNRs differ by less
    than that tolerance (either answer is then correct); such near-ties are counted and must
    stay rare.
"""
import numpy as np

RTOL = 1e-5


def tol_at(ref_snr, bh, mu, sigma):
    """The SNR tolerance per fundamental (mu/sigma FP64 arrays [H] or [F, H])."""
    mu = np.asarray(mu, np.float64)
    sigma = np.asarray(sigma, np.float64)
    idx = bh.astype(np.int64) - 1
    if mu.ndim == 1:
        m, s = mu[idx], sigma[idx]
    else:
        r = np.arange(bh.shape[0])
        m, s = mu[r, idx], sigma[r, idx]
    S = ref_snr * s + m
    return RTOL * (np.abs(S) + np.abs(m)) / s + 1e-30


def compare_form(gpu_snr, gpu_bh, ref_snr, ref_bh, ref_all, mu, sigma, gpu_path=None, ref_path=None,
                 max_near_tie_rate=1e-3, what=""):
    """Returns the number of accepted near-ties; raises AssertionError on any other mismatch."""
    gpu_snr = np.asarray(gpu_snr, np.float64)
    gpu_bh = np.asarray(gpu_bh).astype(np.int64)
    ref_bh = np.asarray(ref_bh).astype(np.int64)
    assert gpu_snr.shape == ref_snr.shape, (what, gpu_snr.shape, ref_snr.shape)
    if gpu_path is not None:
        bad = np.nonzero(np.asarray(gpu_path, np.uint64) != np.asarray(ref_path, np.uint64))[0]
        assert bad.size == 0, f"{what}: {bad.size} paths differ, first at {bad[:5]}"
    assert np.all((gpu_bh >= 1) & (gpu_bh <= ref_all.shape[1])), what
    tol = tol_at(ref_snr, ref_bh, mu, sigma)
    diff_h = np.nonzero(gpu_bh != ref_bh)[0]
    near = 0
    if diff_h.size:
        alt = ref_all[diff_h, gpu_bh[diff_h] - 1]
        ok = np.abs(alt - ref_snr[diff_h]) <= tol[diff_h]
        assert ok.all(), f"{what}: best_h differs beyond near-ties at {diff_h[~ok][:5]}"
        near = int(diff_h.size)
        assert near <= max(2, max_near_tie_rate * gpu_snr.size), f"{what}: {near} near-ties"
    err = np.abs(gpu_snr - ref_snr)
    bad = np.nonzero(err > tol)[0]
    assert bad.size == 0, (f"{what}: snr beyond tolerance at {bad[:5]} gpu={gpu_snr[bad[:5]]} "
                           f"ref={ref_snr[bad[:5]]} tol={tol[bad[:5]]}")
    return near


def compare_argmax(gpu_key, ref_snr, gpu_snr, mu, sigma, ref_bh, decode, what=""):
    """Per-spectrum argmax: the GPU's bin carries the GPU's own snr, and is the oracle's argmax
    unless the two reference SNRs are within tolerance."""
    snr_k, n_k = decode(gpu_key)
    assert 0 <= n_k < ref_snr.shape[0], what
    assert np.float32(snr_k) == np.float32(gpu_snr[n_k]), (what, snr_k, gpu_snr[n_k])
    n_ref = int(np.argmax(ref_snr))
    if n_k != n_ref:
        tol = tol_at(ref_snr[[n_ref]], ref_bh[[n_ref]], mu, sigma)[0]
        assert abs(ref_snr[n_k] - ref_snr[n_ref]) <= 2 * tol, (what, n_k, n_ref)
        return 1
    return 0


def path_view(t, H):
    """Device path tensor -> numpy uint32 view."""
    a = t.cpu().numpy()
    if a.dtype == np.int16:
        return a.view(np.uint16).astype(np.uint32)
    if a.dtype == np.int32:
        return a.view(np.uint32)
    return a.astype(np.uint32)
