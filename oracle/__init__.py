"""FP64 CPU oracle for the harmonic sum -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline / reference leg
may import this package.  The product path (``paper_2202_12817_gb300``) never does, and this
package imports nothing from it: the two share only the seeded input generators in
``synth``.

The arithmetic lives in ``hs_oracle.c`` (plain C, FP64, single thread), compiled with gcc into
``liboracle.so`` next to it.  Every function cites the passage of arXiv:2202.12817 it follows:

  simple_1d   Eq. 3 (simple harmonic sum) + Eq. 2 (SNR of partial sums, max over H)
  greedy_1d   Eq. 5 + Algorithm 2 (greedy drift tracking, optional fundamental comparison)
  greedy_2d   the 1D greedy rule lifted to a 3x3 f-fdot neighbourhood (the paper names the
              higher-dimensional sum but gives no algorithm: centre first, then the 8
              neighbours in raster order, a strictly larger value replacing the best)
  backward_1d adjoint of the forward with the chosen path and best h held fixed
  dp_1d       optimal partial sums over all monotone drift paths (Sec. 2.2 drift tree)
  optimal_1d  dp_1d for every fundamental + Eq. 2's maximum over h (the optimal form)
  tail_1d     fundamentals past the full-harmonic domain with the orders that fit (all forms)
  brute_1d/2d exhaustive enumeration of drift paths (tiny inputs)
  sectors_1d  distinct 32-B input sectors read (compulsory input bytes)
  sectors_2d  the same for the 2D greedy form over an f-fdot plane
  norm_*      closed-form mean / sigma of partial sums of i.i.d. exponential noise

Every function is pinned by ``tests/test_oracle_*.py`` against values the paper or the
mathematics fixes; none is "parity unpinned".
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hs_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


_FLAGS = ["-O2", "-fPIC", "-shared", "-std=c11", "-fno-fast-math", "-ffp-contract=off"]
LIB_OMP = os.path.join(_HERE, "liboracle_omp.so")


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc (portable flags only: it also builds on the Arm GPU host),
    and, where the compiler has OpenMP, liboracle_omp.so: the same source with its loops over
    fundamentals spread over threads (the all-core CPU baseline; never used by the tests)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", *_FLAGS, "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    if force or not os.path.exists(LIB_OMP) or os.path.getmtime(LIB_OMP) < os.path.getmtime(_SRC):
        tmp = LIB_OMP + f".tmp{os.getpid()}"
        r = subprocess.run(["gcc", *_FLAGS, "-fopenmp", "-o", tmp, _SRC, "-lm"], capture_output=True, text=True)
        if r.returncode == 0:
            os.replace(tmp, LIB_OMP)
    return _LIB


_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_I32 = ctypes.c_int32


_use_omp = False


def use_openmp(on: bool = True) -> bool:
    """Route every call to liboracle_omp.so (the all-core CPU baseline) instead of the
    single-threaded oracle; call before the first oracle call.  False when that build is missing."""
    global _use_omp
    build()
    _use_omp = bool(on) and os.path.exists(LIB_OMP)
    return _use_omp


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(LIB_OMP if _use_omp else _LIB)
            L.hso_nf_1d.restype = _I64
            L.hso_nf_1d.argtypes = [_I64, _I32]
            L.hso_simple_1d.restype = ctypes.c_int
            L.hso_simple_1d.argtypes = [_P, _P, _I32, _I64, _I32, _P, _P, _I64, _P, _P, _P]
            L.hso_greedy_1d.restype = ctypes.c_int
            L.hso_greedy_1d.argtypes = [_P, _P, _I32, _I64, _I32, _I32, _P, _P, _I64, _P, _P, _P, _P]
            L.hso_greedy_1d_list.restype = ctypes.c_int
            L.hso_greedy_1d_list.argtypes = [_P, _P, _I32, _I64, _I32, _I32, _P, _P, _I64, _P, _P, _P, _P]
            L.hso_greedy_2d.restype = ctypes.c_int
            L.hso_greedy_2d.argtypes = [_P, _I64, _I64, _I64, _I32, _I64, _I64, _I64, _I64, _P, _P,
                                        _P, _P, _P, _P]
            L.hso_backward_1d.restype = ctypes.c_int
            L.hso_backward_1d.argtypes = [_I32, _I64, _I32, _I64, _P, _P, _P, _P, _P]
            L.hso_dp_1d.restype = ctypes.c_int
            L.hso_dp_1d.argtypes = [_P, _P, _I32, _I64, _I32, _I32, _I64, _P]
            L.hso_tail_1d.restype = ctypes.c_int
            L.hso_tail_1d.argtypes = [_I32, _P, _P, _I32, _I64, _I32, _I32, _P, _P, _I64, _I64, _P, _P, _P, _P]
            L.hso_optimal_1d.restype = ctypes.c_int
            L.hso_optimal_1d.argtypes = [_P, _P, _I32, _I64, _I32, _I32, _P, _P, _I64, _P, _P, _P]
            L.hso_brute_1d.restype = ctypes.c_int
            L.hso_brute_1d.argtypes = [_P, _P, _I32, _I64, _I32, _I32, _I64, _P, _P, _P]
            L.hso_brute_2d.restype = ctypes.c_int
            L.hso_brute_2d.argtypes = [_P, _I64, _I64, _I64, _I32, _I64, _I64, _P, _P, _P]
            L.hso_sectors_1d.restype = _I64
            L.hso_sectors_1d.argtypes = [_I32, _I32, _I64, _I32, _I32, _I64, _P]
            L.hso_sectors_2d.restype = _I64
            L.hso_sectors_2d.argtypes = [_I64, _I64, _I64, _I32, _I64, _I64, _I64, _I64, _P]
            _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _f32(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float32)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _check(rc, what):
    if rc != 0:
        raise ValueError(f"oracle {what}: invalid arguments")


def nf_1d(n: int, H: int) -> int:
    """Fundamental count floor((N-1)/H) (0 when N < H+1)."""
    return int(lib().hso_nf_1d(int(n), int(H)))


def simple_1d(p, H, mu, sigma, w=None, round_w=True, nf=None, want_all=False):
    """Simple HS (Eq. 3) + max SNR (Eq. 2).  Returns (snr f64[nf], best_h u8[nf][, snr_all [nf,H]])."""
    p = _f32(p)
    w = _f32(w)
    n = p.shape[0]
    nf = nf_1d(n, H) if nf is None else int(nf)
    snr = np.empty(nf, np.float64)
    bh = np.empty(nf, np.uint8)
    allv = np.empty((nf, H), np.float64) if want_all else None
    mu, sigma = _f64(mu), _f64(sigma)
    _check(lib().hso_simple_1d(_ptr(p), _ptr(w), int(round_w), n, int(H), _ptr(mu), _ptr(sigma), nf,
                               _ptr(snr), _ptr(bh), _ptr(allv)), "simple_1d")
    return (snr, bh, allv) if want_all else (snr, bh)


def greedy_1d(p, H, mu, sigma, mitigation=True, w=None, round_w=True, nf=None, want_all=False):
    """Greedy HS (Eq. 5, Algorithm 2) + max SNR.  Returns (snr, best_h, path u32[nf][, snr_all])."""
    p = _f32(p)
    w = _f32(w)
    n = p.shape[0]
    nf = nf_1d(n, H) if nf is None else int(nf)
    snr = np.empty(nf, np.float64)
    bh = np.empty(nf, np.uint8)
    path = np.empty(nf, np.uint32)
    allv = np.empty((nf, H), np.float64) if want_all else None
    mu, sigma = _f64(mu), _f64(sigma)
    _check(lib().hso_greedy_1d(_ptr(p), _ptr(w), int(round_w), n, int(H), int(bool(mitigation)),
                               _ptr(mu), _ptr(sigma), nf, _ptr(snr), _ptr(bh), _ptr(path), _ptr(allv)),
           "greedy_1d")
    return (snr, bh, path, allv) if want_all else (snr, bh, path)


def greedy_1d_list(p, H, mu, sigma, fund, mitigation=True, w=None, round_w=True):
    """Greedy HS of the listed fundamentals only.  Returns (snr, best_h, path) in list order."""
    p = _f32(p)
    w = _f32(w)
    fund = np.ascontiguousarray(fund, np.int64)
    cnt = fund.shape[0]
    snr = np.empty(cnt, np.float64)
    bh = np.empty(cnt, np.uint8)
    path = np.empty(cnt, np.uint32)
    mu, sigma = _f64(mu), _f64(sigma)
    _check(lib().hso_greedy_1d_list(_ptr(p), _ptr(w), int(round_w), p.shape[0], int(H), int(bool(mitigation)),
                                    _ptr(mu), _ptr(sigma), cnt, _ptr(fund), _ptr(snr), _ptr(bh), _ptr(path)),
           "greedy_1d_list")
    return snr, bh, path


def domain_2d(n_freq, n_rows, z0_row, H):
    """(f_lo, f_hi, z_lo, z_hi): every read of every order stays inside the plane."""
    f_lo, f_hi = 1, (n_freq - 1 - H) // H
    z_lo = -((z0_row - H) // H)
    z_hi = (n_rows - 1 - z0_row - H) // H
    return f_lo, f_hi, z_lo, z_hi


def greedy_2d(plane, z0_row, H, mu, sigma, dom=None, want_all=False):
    """2D greedy HS.  plane float32 [n_rows][n_freq].  Returns (snr, best_h, path) flattened z-major."""
    plane = _f32(plane)
    n_rows, n_freq = plane.shape
    f_lo, f_hi, z_lo, z_hi = dom if dom is not None else domain_2d(n_freq, n_rows, z0_row, H)
    cnt = (f_hi - f_lo + 1) * (z_hi - z_lo + 1)
    snr = np.empty(cnt, np.float64)
    bh = np.empty(cnt, np.uint8)
    path = np.empty(cnt, np.uint32)
    allv = np.empty((cnt, H), np.float64) if want_all else None
    mu, sigma = _f64(mu), _f64(sigma)
    _check(lib().hso_greedy_2d(_ptr(plane), n_freq, n_rows, int(z0_row), int(H), f_lo, f_hi, z_lo, z_hi,
                               _ptr(mu), _ptr(sigma), _ptr(snr), _ptr(bh), _ptr(path), _ptr(allv)),
           "greedy_2d")
    return (snr, bh, path, allv) if want_all else (snr, bh, path)


def backward_1d(form, n, H, best_h, sigma, g, path=None):
    """dL/dx (f64[n]) of one spectrum for upstream dL/dSNR ``g`` (form 1 simple, 2 greedy)."""
    best_h = np.ascontiguousarray(best_h, np.uint8)
    nf = best_h.shape[0]
    path = None if path is None else np.ascontiguousarray(path, np.uint32)
    g = _f64(g)
    sigma = _f64(sigma)
    out = np.empty(int(n), np.float64)
    _check(lib().hso_backward_1d(int(form), int(n), int(H), nf, _ptr(best_h), _ptr(path), _ptr(sigma),
                                 _ptr(g), _ptr(out)), "backward_1d")
    return out


def dp_1d(p, H, fund, mitigation=True, w=None, round_w=True):
    p = _f32(p)
    w = _f32(w)
    out = np.empty(int(H), np.float64)
    _check(lib().hso_dp_1d(_ptr(p), _ptr(w), int(round_w), p.shape[0], int(H), int(bool(mitigation)),
                           int(fund), _ptr(out)), "dp_1d")
    return out


def tail_1d(form, p, H, mu, sigma, mitigation=True, w=None, round_w=True, lo=None, hi=None, want_all=False):
    """Fundamentals n in [lo, hi) (default [N_f, N-1)) past the full-harmonic domain, each form
    summing only its orders whose reads fit (simple h n <= N-1; greedy/optimal h n + h <= N-1).
    Returns (snr, best_h, path (greedy, else None)[, snr_all with NaN for excluded orders])."""
    p = _f32(p)
    w = _f32(w)
    n = p.shape[0]
    lo = nf_1d(n, H) if lo is None else int(lo)
    hi = n - 1 if hi is None else int(hi)
    k = max(hi - lo, 0)
    snr = np.empty(k, np.float64)
    bh = np.empty(k, np.uint8)
    path = np.zeros(k, np.uint32) if form == 2 else None
    allv = np.empty((k, H), np.float64) if want_all else None
    mu, sigma = _f64(mu), _f64(sigma)
    _check(lib().hso_tail_1d(int(form), _ptr(p), _ptr(w), int(round_w), n, int(H), int(bool(mitigation)),
                             _ptr(mu), _ptr(sigma), lo, hi, _ptr(snr), _ptr(bh), _ptr(path), _ptr(allv)), "tail_1d")
    return (snr, bh, path, allv) if want_all else (snr, bh, path)


def tail_orders(form, n, H, f):
    """Orders summed for fundamental f of an n-bin spectrum in the truncated tail."""
    lim = (H if f == 0 else (n - 1) // f) if form == 1 else (n - 1) // (f + 1)
    return min(lim, H)


def optimal_1d(p, H, mu, sigma, mitigation=True, w=None, round_w=True, nf=None, want_all=False):
    """Optimal form: the DP optimum S*_h over monotone drift paths (Sec. 2.2) + max SNR (Eq. 2).
    Returns (snr f64[nf], best_h u8[nf][, snr_all [nf,H]])."""
    p = _f32(p)
    w = _f32(w)
    n = p.shape[0]
    nf = nf_1d(n, H) if nf is None else int(nf)
    snr = np.empty(nf, np.float64)
    bh = np.empty(nf, np.uint8)
    allv = np.empty((nf, H), np.float64) if want_all else None
    mu, sigma = _f64(mu), _f64(sigma)
    _check(lib().hso_optimal_1d(_ptr(p), _ptr(w), int(round_w), n, int(H), int(bool(mitigation)),
                                _ptr(mu), _ptr(sigma), nf, _ptr(snr), _ptr(bh), _ptr(allv)), "optimal_1d")
    return (snr, bh, allv) if want_all else (snr, bh)


def brute_1d(p, H, fund, mitigation=True, w=None, round_w=True):
    """Returns (best_sum f64[H], rule_path, rule_count)."""
    p = _f32(p)
    w = _f32(w)
    out = np.empty(int(H), np.float64)
    rp = np.zeros(1, np.uint32)
    rc = np.zeros(1, np.int64)
    _check(lib().hso_brute_1d(_ptr(p), _ptr(w), int(round_w), p.shape[0], int(H), int(bool(mitigation)),
                              int(fund), _ptr(out), _ptr(rp), _ptr(rc)), "brute_1d")
    return out, int(rp[0]), int(rc[0])


def brute_2d(plane, z0_row, H, f, z):
    plane = _f32(plane)
    n_rows, n_freq = plane.shape
    out = np.empty(int(H), np.float64)
    rp = np.zeros(1, np.uint32)
    rc = np.zeros(1, np.int64)
    _check(lib().hso_brute_2d(_ptr(plane), n_freq, n_rows, int(z0_row), int(H), int(f), int(z),
                              _ptr(out), _ptr(rp), _ptr(rc)), "brute_2d")
    return out, int(rp[0]), int(rc[0])


def sectors_1d(forms, elem_bytes, n, H, path=None, mitigation=True, nf=None):
    nf = nf_1d(n, H) if nf is None else int(nf)
    path = None if path is None else np.ascontiguousarray(path, np.uint32)
    r = lib().hso_sectors_1d(int(forms), int(elem_bytes), int(n), int(H), int(bool(mitigation)), nf,
                             _ptr(path))
    if r < 0:
        raise ValueError("oracle sectors_1d: invalid arguments")
    return int(r)


def sectors_2d(n_freq, n_rows, z0_row, H, path, dom=None):
    """Distinct 32-B sectors of a float32 plane read by the 2D greedy form along ``path``."""
    f_lo, f_hi, z_lo, z_hi = dom if dom is not None else domain_2d(n_freq, n_rows, z0_row, H)
    path = np.ascontiguousarray(path, np.uint32)
    r = lib().hso_sectors_2d(int(n_freq), int(n_rows), int(z0_row), int(H), f_lo, f_hi, z_lo, z_hi, _ptr(path))
    if r < 0:
        raise ValueError("oracle sectors_2d: invalid arguments")
    return int(r)


# ---------------------------------------------------------------------------------------------
# closed-form normalisation for i.i.d. exponential noise (Eq. 2's mu_H, sigma_H)
# ---------------------------------------------------------------------------------------------
def _harmonic(m):
    return sum(1.0 / k for k in range(1, m + 1))


def _harmonic2(m):
    return sum(1.0 / (k * k) for k in range(1, m + 1))


def norm_exponential(form, dims, H, mitigation=True, mean1=1.0):
    """(mu[H], sigma[H]) in FP64 of partial sums of h terms when every summed term is an
    independent draw: Exp(mean1) (simple), max of 2 (greedy step; the un-mitigated
    fundamental is a single draw) or max of 9 (2D greedy step).  The maximum of m i.i.d.
    Exp(1) has mean H_m and variance sum_{k<=m} 1/k^2."""
    h = np.arange(1, H + 1, dtype=np.float64)
    if dims == 1 and form == 1:
        mu, var = h, h.copy()
    elif dims == 1 and form == 2:
        m2, v2 = _harmonic(2), _harmonic2(2)
        if mitigation:
            mu, var = m2 * h, v2 * h
        else:
            mu, var = 1.0 + m2 * (h - 1), 1.0 + v2 * (h - 1)
    elif dims == 2 and form == 2:
        mu, var = _harmonic(9) * h, _harmonic2(9) * h
    else:
        raise ValueError("unsupported form/dims")
    return mu * mean1, np.sqrt(var) * mean1
