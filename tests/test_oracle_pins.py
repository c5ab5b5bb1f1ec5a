"""Pins of the FP64 oracle against what the paper and the mathematics fix (CPU only).

Each test checks the oracle against something other than itself: the paper's worked
example, closed-form noise statistics, exhaustive enumeration, special cases with a known
answer and finite differences.  A dropped term, a wrong index, a flipped comparison or a
transposed operand in ``oracle/hs_oracle.c`` fails at least one of them.
"""
import json
import math
import os

import numpy as np
import pytest

import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def unit_norm(H):
    return np.zeros(H), np.ones(H)


def drift_of(path, H):
    """Drift after each order: D_k = popcount(path & ((1 << k) - 1))."""
    return [bin(int(path) & ((1 << k) - 1)).count("1") for k in range(1, H + 1)]


# ----------------------------------------------------------------------------------------
# special cases
# ----------------------------------------------------------------------------------------
def test_h1_returns_input(oracle_lib):
    o = oracle_lib
    x = synth.spectrum(1000, 11)
    mu, sg = unit_norm(1)
    nf = o.nf_1d(x.size, 1)
    assert nf == x.size - 1
    s, bh = o.simple_1d(x, 1, mu, sg)
    assert np.array_equal(s, x[:nf].astype(np.float64)) and np.all(bh == 1)
    g, bh, path = o.greedy_1d(x, 1, mu, sg, mitigation=False)
    assert np.array_equal(g, x[:nf].astype(np.float64)) and np.all(path == 0)
    g, bh, path = o.greedy_1d(x, 1, mu, sg, mitigation=True)
    assert np.array_equal(g, np.maximum(x[:nf], x[1:nf + 1]).astype(np.float64))
    assert np.array_equal(path, (x[1:nf + 1] > x[:nf]).astype(np.uint32))


def test_domain(oracle_lib):
    o = oracle_lib
    assert o.nf_1d(131072, 32) == 4095
    assert o.nf_1d(1 << 23, 32) == 262143
    assert o.nf_1d(33, 32) == 1 and o.nf_1d(32, 32) == 0
    # the greedy form's largest read, H*n + H, is the last bin for the largest n
    N, H = 1000, 7
    nf = o.nf_1d(N, H)
    assert H * (nf - 1) + H <= N - 1 < H * nf + H


def test_monotone_spectra(oracle_lib):
    o = oracle_lib
    N, H = 4096, 16
    mu, sg = unit_norm(H)
    dec = (N - np.arange(N)).astype(np.float32)          # strictly decreasing: never drift
    s_all = o.simple_1d(dec, H, mu, sg, want_all=True)[2]
    g_all = o.greedy_1d(dec, H, mu, sg, want_all=True)[3]
    path = o.greedy_1d(dec, H, mu, sg)[2]
    assert np.all(path == 0)
    assert np.array_equal(s_all, g_all)
    n = np.arange(s_all.shape[0])[:, None]
    h = np.arange(1, H + 1)[None, :]
    assert np.array_equal(s_all, N * h - n * h * (h + 1) / 2)    # sum_k (N - k n)
    inc = np.arange(N).astype(np.float32)                  # strictly increasing: drift every order
    g_all = o.greedy_1d(inc, H, mu, sg, want_all=True)[3]
    path = o.greedy_1d(inc, H, mu, sg)[2]
    assert np.all(path == (1 << H) - 1)
    assert np.array_equal(g_all, (n + 1) * h * (h + 1) / 2)       # sum_k (k n + k)
    path_nm = o.greedy_1d(inc, H, mu, sg, mitigation=False)[2]
    assert np.all(path_nm == (1 << H) - 2)


def test_snr_normalisation_and_best_h(oracle_lib):
    """Eq. 2: SNR_h = (S_h - mu_h) / sigma_h, max over h, lowest h on ties."""
    o = oracle_lib
    N, H = 2048, 8
    x = synth.small_int_spectrum(N, 5)
    mu = np.arange(1, H + 1) * 3.5
    sg = np.sqrt(np.arange(1, H + 1)) * 2.0
    for fn in (lambda m, s: o.simple_1d(x, H, m, s, want_all=True),
               lambda m, s: o.greedy_1d(x, H, m, s, want_all=True)):
        raw = fn(np.zeros(H), np.ones(H))[-1]                 # raw partial sums S_h
        out = fn(mu, sg)
        snr, bh, allv = out[0], out[1], out[-1]
        np.testing.assert_allclose(allv, (raw - mu) / sg, rtol=0, atol=1e-12)
        first_max = np.argmax(allv, axis=1) + 1               # numpy argmax = lowest index on ties
        assert np.array_equal(bh, first_max)
        assert np.array_equal(snr, allv[np.arange(allv.shape[0]), bh - 1])
    # ties: an all-zero spectrum with zero mean gives equal SNRs -> best h is 1
    z = np.zeros(300, np.float32)
    assert np.all(o.greedy_1d(z, 8, np.zeros(8), np.ones(8))[1] == 1)
    assert np.all(o.simple_1d(z, 8, np.zeros(8), np.ones(8))[1] == 1)


def test_greedy_strict_tie_keeps_drift(oracle_lib):
    """A tie x[m+1] == x[m] keeps the drift (the comparison is strict, Algorithm 2)."""
    o = oracle_lib
    x = np.ones(200, np.float32)
    assert np.all(o.greedy_1d(x, 8, *unit_norm(8))[2] == 0)


# ----------------------------------------------------------------------------------------
# the paper's worked example and the injected pulse train
# ----------------------------------------------------------------------------------------
def _sinc2(d):
    d = np.asarray(d, np.float64)
    out = np.ones_like(d)
    nz = d != 0
    out[nz] = (np.sin(np.pi * d[nz]) / (np.pi * d[nz])) ** 2
    return out


def test_fig2_drift(oracle_lib):
    """Sec. 2.2 / Fig. 2: a 10.1245 Hz pulsar in 0.05 Hz bins drifts by {0,1,1,2,2} bins."""
    o = oracle_lib
    gold = json.load(open(os.path.join(GOLD, "fig2_drift.json")))
    f_bins = gold["pulsar_hz"] / gold["bin_width_hz"]
    H = len(gold["orders"])
    N = 4096
    j = np.arange(N)
    x = np.zeros(N)
    for h in gold["orders"]:
        x += _sinc2(j - h * f_bins)        # noise-free DFT power of each harmonic
    x = x.astype(np.float32)
    n = gold["fundamental_bin"]
    assert [int(np.argmax(x[h * n - 5:h * n + 6]) + h * n - 5) for h in gold["orders"]] == gold["nearest_bins"]
    path = o.greedy_1d(x, H, *unit_norm(H))[2]
    assert drift_of(path[n], H) == gold["drift"]
    # the simple sum stays on the integer multiples: it collects the fundamental only
    s = o.simple_1d(x, H, *unit_norm(H), want_all=True)[2]
    g = o.greedy_1d(x, H, *unit_norm(H), want_all=True)[3]
    assert g[n, -1] > s[n, -1] + 1.5


def test_pulse_train_noise_free(oracle_lib):
    o = oracle_lib
    gold = json.load(open(os.path.join(GOLD, "pulse_train_1234.json")))
    H, n = gold["H"], gold["fundamental_bin"]
    pul = synth.Pulsar(gold["f0_bins"], gold["duty"], gold["amplitude"])
    x = synth.inject(np.zeros(synth.CONFIG1_N, np.float32), [pul])
    s_all = o.simple_1d(x, H, *unit_norm(H), want_all=True)[2]
    g_all = o.greedy_1d(x, H, *unit_norm(H), want_all=True)[3]
    path = o.greedy_1d(x, H, *unit_norm(H))[2]
    assert drift_of(path[n], H)[:8] == gold["drift_first_8"]
    k = np.arange(1, H + 1)
    expect = np.cumsum(gold["amplitude"] * np.exp(-(np.pi * gold["duty"] * k) ** 2))
    np.testing.assert_allclose(g_all[n], expect, rtol=1e-6)       # float32-stored powers
    assert abs(g_all[n, -1] - 41.13516668) < 1e-4
    np.testing.assert_allclose(s_all[n], np.full(H, expect[0]), rtol=1e-6)
    assert abs(s_all[n, 0] - 7.80502323) < 1e-5


def test_pulse_train_recovered_in_noise(oracle_lib):
    o = oracle_lib
    x = synth.single_pulse_spectrum()
    H = 32
    mu_s, sg_s = o.norm_exponential(1, 1, H)
    mu_g, sg_g = o.norm_exponential(2, 1, H)
    ss, _ = o.simple_1d(x, H, mu_s, sg_s)
    gs, gh, _ = o.greedy_1d(x, H, mu_g, sg_g)
    assert int(np.argmax(gs)) == 1234
    assert gs[1234] > ss[1234]
    assert gh[1234] > 1          # several harmonics add SNR (power ~ noise mean past k ~ 8)


# ----------------------------------------------------------------------------------------
# noise statistics (Eq. 2's mu_H, sigma_H for exponential noise)
# ----------------------------------------------------------------------------------------
def _moment_check(samples, mean, var, nsig=5.0):
    m = samples.mean(axis=0)
    v = samples.var(axis=0, ddof=1)
    cnt = samples.shape[0]
    se_m = np.sqrt(var / cnt)
    c = samples - m
    m4 = (c ** 4).mean(axis=0)
    se_v = np.sqrt(np.maximum(m4 - v ** 2, 1e-30) / cnt)
    assert np.all(np.abs(m - mean) < nsig * se_m), (m, mean)
    assert np.all(np.abs(v - var) < nsig * se_v), (v, var)


def test_exp_noise_moments(oracle_lib):
    """Simple: S_h ~ Gamma(h, 1) (mean h, var h).  Greedy: each order adds the max of two fresh
    Exp(1) draws (mean 3/2, var 5/4) -- fresh because order h reads bins > n past order h-1."""
    o = oracle_lib
    N, H = 1 << 21, 32
    x = synth.exp_noise(N, 99)
    h = np.arange(1, H + 1, dtype=np.float64)
    s_all = o.simple_1d(x, H, *unit_norm(H), want_all=True)[2][2:]
    _moment_check(s_all, h, h)
    g_all = o.greedy_1d(x, H, *unit_norm(H), want_all=True)[3][2:]
    _moment_check(g_all, 1.5 * h, 1.25 * h)
    g_nm = o.greedy_1d(x, H, *unit_norm(H), mitigation=False, want_all=True)[3][2:]
    _moment_check(g_nm, 1 + 1.5 * (h - 1), 1 + 1.25 * (h - 1))
    # closed forms used for normalisation agree with the measured moments
    for form, mit, samp in ((1, True, s_all), (2, True, g_all), (2, False, g_nm)):
        mu, sg = o.norm_exponential(form, 1, H, mitigation=mit)
        _moment_check(samp, mu, sg ** 2)


def test_snr_standardised_on_noise(oracle_lib):
    o = oracle_lib
    N, H = 1 << 20, 16
    x = synth.exp_noise(N, 7)
    mu, sg = o.norm_exponential(2, 1, H)
    allv = o.greedy_1d(x, H, mu, sg, want_all=True)[3][2:]
    assert np.all(np.abs(allv.mean(axis=0)) < 0.02)
    assert np.all(np.abs(allv.std(axis=0) - 1) < 0.02)


# ----------------------------------------------------------------------------------------
# exhaustive search and the optimal path
# ----------------------------------------------------------------------------------------
@pytest.mark.parametrize("mitigation", [True, False])
@pytest.mark.parametrize("seed", [1, 2, 3])
def test_brute_force_bounds_and_reproduces_greedy(oracle_lib, mitigation, seed):
    o = oracle_lib
    N, H = 96, 7
    for x in (synth.exp_noise(N, seed), synth.small_int_spectrum(N, seed, 4)):
        g_all = o.greedy_1d(x, H, *unit_norm(H), mitigation=mitigation, want_all=True)
        paths, allv = g_all[2], g_all[3]
        for n in range(o.nf_1d(N, H)):
            best, rule_path, rule_count = o.brute_1d(x, H, n, mitigation=mitigation)
            dp = o.dp_1d(x, H, n, mitigation=mitigation)
            assert rule_count == 1
            assert rule_path == paths[n]
            np.testing.assert_allclose(best, dp, rtol=0, atol=1e-12)
            assert np.all(allv[n] <= best + 1e-12)


@pytest.mark.parametrize("mitigation", [True, False])
def test_optimal_form_is_the_brute_force_optimum(oracle_lib, mitigation):
    """optimal_1d's every-order sums are the exhaustive maxima over drift paths (tiny inputs),
    bound the greedy and simple sums from above, and its best h follows Eq. 2's maximum rule."""
    o = oracle_lib
    N, H = 96, 7
    for seed in (4, 5):
        x = synth.exp_noise(N, seed)
        _, _, opt_all = o.optimal_1d(x, H, *unit_norm(H), mitigation=mitigation, want_all=True)
        g_all = o.greedy_1d(x, H, *unit_norm(H), mitigation=mitigation, want_all=True)[3]
        s_all = o.simple_1d(x, H, *unit_norm(H), want_all=True)[2]
        for n in range(o.nf_1d(N, H)):
            best = o.brute_1d(x, H, n, mitigation=mitigation)[0]
            np.testing.assert_allclose(opt_all[n], best, rtol=0, atol=1e-12)
        assert np.all(opt_all >= g_all - 1e-12) and np.all(opt_all >= s_all - 1e-12)
        mu = np.linspace(0.5, 4.0, H)
        sg = np.linspace(1.0, 2.5, H)
        snr, bh, allv = o.optimal_1d(x, H, mu, sg, mitigation=mitigation, want_all=True)
        for n in range(allv.shape[0]):
            v = allv[n]
            h = 0
            for k in range(1, H):
                if v[k] > v[h]:
                    h = k
            assert bh[n] == h + 1 and snr[n] == v[h]
            np.testing.assert_allclose(v, (opt_all[n] - mu) / sg, rtol=1e-12)


def test_optimal_form_special_cases(oracle_lib):
    """H = 1 with mitigation: max(x[n], x[n+1]); an increasing spectrum: every increment (the
    greedy path is then optimal); the noise-free pulse train: the optimum collects every harmonic
    peak, as the greedy does (41.135167 at H = 32, n = 1234)."""
    o = oracle_lib
    x = synth.exp_noise(1000, 9)
    s1 = o.optimal_1d(x, 1, *unit_norm(1), want_all=True)[2][:, 0]
    np.testing.assert_array_equal(s1, np.maximum(x[:-1], x[1:]).astype(np.float64)[:s1.size])
    s1u = o.optimal_1d(x, 1, *unit_norm(1), mitigation=False, want_all=True)[2][:, 0]
    np.testing.assert_array_equal(s1u, x[:s1u.size].astype(np.float64))
    inc = np.arange(1, 801, dtype=np.float32)
    H = 8
    g = o.greedy_1d(inc, H, *unit_norm(H), want_all=True)[3]
    opt = o.optimal_1d(inc, H, *unit_norm(H), want_all=True)[2]
    np.testing.assert_array_equal(opt, g)
    gold = json.load(open(os.path.join(GOLD, "pulse_train_1234.json")))
    H, n = gold["H"], gold["fundamental_bin"]
    pul = synth.Pulsar(gold["f0_bins"], gold["duty"], gold["amplitude"])
    xp = synth.inject(np.zeros(synth.CONFIG1_N, np.float32), [pul])
    opt = o.optimal_1d(xp, H, *unit_norm(H), nf=n + 1, want_all=True)[2]
    assert abs(opt[n, -1] - 41.13516668) < 1e-4


@pytest.mark.parametrize("mitigation", [True, False])
def test_tail_reduces_to_full_forms_where_they_fit(oracle_lib, mitigation):
    """Below N_f every order fits, so the truncated-tail rule gives the full forms exactly."""
    o = oracle_lib
    N, H = 3001, 16
    x = synth.exp_noise(N, 12)
    nf = o.nf_1d(N, H)
    mu, sg = np.linspace(1.0, 9.0, H), np.linspace(1.0, 3.0, H)
    s, b = o.simple_1d(x, H, mu, sg)
    g, gb, gp = o.greedy_1d(x, H, mu, sg, mitigation=mitigation)
    q, qb = o.optimal_1d(x, H, mu, sg, mitigation=mitigation)
    ts, tb, _ = o.tail_1d(1, x, H, mu, sg, lo=0, hi=nf)
    tg, tgb, tgp = o.tail_1d(2, x, H, mu, sg, mitigation=mitigation, lo=0, hi=nf)
    tq, tqb, _ = o.tail_1d(4, x, H, mu, sg, mitigation=mitigation, lo=0, hi=nf)
    np.testing.assert_array_equal(ts, s), np.testing.assert_array_equal(tb, b)
    np.testing.assert_array_equal(tg, g), np.testing.assert_array_equal(tgb, gb)
    np.testing.assert_array_equal(tgp, gp)
    np.testing.assert_array_equal(tq, q), np.testing.assert_array_equal(tqb, qb)


def test_tail_order_counts_are_the_largest_that_fit(oracle_lib):
    """On a strictly increasing spectrum the greedy increments at every order, so its last bin
    is H_n n + H_n: inside the spectrum, while one more order would leave it; the simple form's
    last bin H_n n likewise."""
    o = oracle_lib
    N, H = 2000, 32
    x = np.arange(1, N + 1, dtype=np.float32)
    lo = o.nf_1d(N, H)
    _, gb, gp, gall = o.tail_1d(2, x, H, *unit_norm(H), want_all=True)
    _, sb, _, sall = o.tail_1d(1, x, H, *unit_norm(H), want_all=True)
    for i, n in enumerate(range(lo, N - 1)):
        hg = int(np.sum(~np.isnan(gall[i])))
        assert hg == o.tail_orders(2, N, H, n)
        assert hg * n + hg <= N - 1 and (hg + 1) * (n + 1) > N - 1 or hg == H
        assert gp[i] == (1 << hg) - 1 and gb[i] == hg       # increasing: every increment, last order best
        hs_ = int(np.sum(~np.isnan(sall[i])))
        assert hs_ * n <= N - 1 and ((hs_ + 1) * n > N - 1 or hs_ == H)
        assert sb[i] == hs_


def test_tail_pulse_train(oracle_lib):
    """A noise-free pulse train whose fundamental lies past N_f: at n = 200 of a 4096-bin
    spectrum (N_f = 127 at H = 32) the greedy, simple and optimal forms all keep
    floor(4095 / 201) = 20 and floor(4095 / 200) = 20 orders, and each sums the first 20
    harmonic powers 8 exp(-(pi 0.05 k)^2)."""
    o = oracle_lib
    N, H, n = 4096, 32, 200
    x = synth.inject(np.zeros(N, np.float32), [synth.Pulsar(200.0, 0.05, 8.0)])
    k = np.arange(1, 21)
    want = np.sum(np.float32(8.0 * np.exp(-(np.pi * 0.05 * k) ** 2)).astype(np.float64))
    lo = o.nf_1d(N, H)
    assert lo == 127
    for form in (1, 2, 4):
        _, b, _, allv = o.tail_1d(form, x, H, *unit_norm(H), lo=n, hi=n + 1, want_all=True)
        assert int(np.sum(~np.isnan(allv[0]))) == 20
        assert abs(allv[0, 19] - want) < 1e-9 and b[0] == 20


def test_greedy_list_is_the_greedy_form_of_the_listed_fundamentals(oracle_lib):
    """hso_greedy_1d_list runs the same per-fundamental steps as hso_greedy_1d, in list order,
    with or without whitening and mitigation; a fundamental outside [0, N_f) is refused."""
    o = oracle_lib
    N, H = 5000, 13
    x = synth.spectrum(N, 41, [synth.Pulsar(77.3, 0.05)])
    w = synth.whitening(N, 3)
    mu, sg = o.norm_exponential(2, 1, H)
    nf = o.nf_1d(N, H)
    fund = np.random.default_rng(2).integers(0, nf, 300)
    for mit in (True, False):
        for wv, rw in ((None, True), (w, True), (w, False)):
            s, b, pa = o.greedy_1d(x, H, mu, sg, mitigation=mit, w=wv, round_w=rw)
            s2, b2, p2 = o.greedy_1d_list(x, H, mu, sg, fund, mitigation=mit, w=wv, round_w=rw)
            assert np.array_equal(s2, s[fund]) and np.array_equal(b2, b[fund]) and np.array_equal(p2, pa[fund])
    with pytest.raises(ValueError):
        o.greedy_1d_list(x, H, mu, sg, [nf])


def test_path_invariants(oracle_lib):
    """d_m(h) = h-1 between fundamentals (Sec. 2.2); the fundamental comparison adds at most 1."""
    o = oracle_lib
    N, H = 1 << 16, 32
    x = synth.exp_noise(N, 3)
    for mit in (True, False):
        path = o.greedy_1d(x, H, *unit_norm(H), mitigation=mit)[2]
        for k in (1, 2, 5, 17, 32):
            mask = np.uint32((1 << k) - 1) if k < 32 else np.uint32(0xFFFFFFFF)
            D = np.array([bin(int(v)).count("1") for v in (path & mask)])
            assert D.max() <= (k if mit else k - 1)
        if not mit:
            assert np.all((path & 1) == 0)


# ----------------------------------------------------------------------------------------
# adjoint vs finite differences (FP64, whitening kept exact so the forward is piecewise linear)
# ----------------------------------------------------------------------------------------
@pytest.mark.parametrize("form", [1, 2])
def test_backward_matches_finite_differences(oracle_lib, form):
    o = oracle_lib
    N, H = 1024, 8
    p = synth.exp_noise(N, 21)
    w = synth.whitening(N, 22)
    mu, sg = o.norm_exponential(form, 1, H)
    nf = o.nf_1d(N, H)
    g = synth.upstream_grad(nf, 23).astype(np.float64)

    def fwd(wv):
        if form == 1:
            s, bh = o.simple_1d(p, H, mu, sg, w=wv, round_w=False)
            return s, bh, None
        return o.greedy_1d(p, H, mu, sg, w=wv, round_w=False)

    s0, bh0, path0 = fwd(w)
    gx = o.backward_1d(form, N, H, bh0, sg, g, path0)
    gw = gx * p                                    # dL/dw = p * dL/dx for x = w p
    eps = 1e-3
    rs = np.random.default_rng(5)
    js = rs.choice(H * nf, size=120, replace=False)
    checked = 0
    for j in js:
        wp, wm = w.astype(np.float64).copy(), w.astype(np.float64).copy()
        wp[j] += eps
        wm[j] -= eps
        outp, outm = fwd(wp.astype(np.float32)), fwd(wm.astype(np.float32))
        # keep w in float32 for the oracle input: use the exact float32 perturbation size
        dw = float(np.float32(wp[j])) - float(np.float32(wm[j]))
        same = all(np.array_equal(a, b) for a, b in zip(outp[1:], (bh0, path0)) if b is not None) and \
            all(np.array_equal(a, b) for a, b in zip(outm[1:], (bh0, path0)) if b is not None)
        if not same:
            continue
        fd = (np.dot(g, outp[0]) - np.dot(g, outm[0])) / dw
        assert abs(fd - gw[j]) <= 1e-7 * max(1.0, abs(gw[j])), (j, fd, gw[j])
        checked += 1
    assert checked > 60


def test_backward_counts_each_chosen_bin(oracle_lib):
    """With g = sigma_{h*}, dL/dx counts how many (n, k <= h*) chose each bin."""
    o = oracle_lib
    N, H = 512, 6
    x = synth.exp_noise(N, 8)
    mu, sg = o.norm_exponential(2, 1, H)
    _, bh, path = o.greedy_1d(x, H, mu, sg)
    g = sg[bh.astype(np.int64) - 1]
    gx = o.backward_1d(2, N, H, bh, sg, g, path)
    assert np.isclose(gx.sum(), bh.astype(np.int64).sum())
    assert np.all(gx == np.round(gx))
    gx_s = o.backward_1d(1, N, H, bh, sg, g)
    n = np.arange(bh.size)
    assert gx_s[0] == bh.astype(np.int64)[0]              # fundamental 0 puts all its orders on bin 0
    assert gx_s[n[1:]].min() >= 1                          # every fundamental's own bin (k = 1)


# ----------------------------------------------------------------------------------------
# 2D
# ----------------------------------------------------------------------------------------
def test_2d_domain(oracle_lib):
    assert oracle_lib.domain_2d(1 << 21, 201, 100, 8) == (1, 262142, -11, 11)


@pytest.mark.parametrize("seed", [4, 5])
def test_2d_brute_force(oracle_lib, seed):
    o = oracle_lib
    H, z0 = 3, 6
    pl = synth.plane(40, 2 * z0 + 1, z0, seed)
    pl_int = np.floor(pl).astype(np.float32)             # dense ties exercise the raster rule
    for P in (pl, pl_int):
        dom = o.domain_2d(P.shape[1], P.shape[0], z0, H)
        snr, bh, path, allv = o.greedy_2d(P, z0, H, *unit_norm(H), want_all=True)
        f_lo, f_hi, z_lo, z_hi = dom
        nff = f_hi - f_lo + 1
        for z in range(z_lo, z_hi + 1):
            for f in range(f_lo, f_hi + 1, 3):
                i = (z - z_lo) * nff + (f - f_lo)
                best, rp, rc = o.brute_2d(P, z0, H, f, z)
                assert rc == 1 and rp == path[i]
                assert np.all(allv[i] <= best + 1e-12)


def test_2d_noise_moments(oracle_lib):
    """chi-square(2) noise: each 2D order adds the max of 9 fresh draws of mean 2
    (fresh for f >= 4): mean 2 H_9 per order, variance 4 sum_{k<=9} 1/k^2 per order."""
    o = oracle_lib
    H, z0 = 4, 20
    pl = synth.plane(1 << 15, 2 * z0 + 1, z0, 31)
    dom = o.domain_2d(pl.shape[1], pl.shape[0], z0, H)
    dom = (4, dom[1], dom[2], dom[3])
    allv = o.greedy_2d(pl, z0, H, *unit_norm(H), dom=dom, want_all=True)[3]
    h = np.arange(1, H + 1, dtype=np.float64)
    H9 = sum(1.0 / k for k in range(1, 10))
    S9 = sum(1.0 / k ** 2 for k in range(1, 10))
    # rows of different z share no bins for f >= 4 only within a row band; moments are robust
    _moment_check(allv, 2 * H9 * h, 4 * S9 * h, nsig=6)
    mu, sg = o.norm_exponential(2, 2, H, mean1=2.0)
    _moment_check(allv, mu, sg ** 2, nsig=6)


def test_2d_noise_free_track(oracle_lib):
    """A signal whose harmonic k sits at (k*zf, k*ff) with |fractional parts| < 1/2 is followed
    bin by bin: the drift at order k is (round(k*ff) - k*f, round(k*zf) - k*z)."""
    o = oracle_lib
    H, z0, nfreq = 8, 100, 1 << 14
    ff, zf = 1000.3, -3.4
    f, z = 1000, -3
    pl = np.zeros((2 * z0 + 1, nfreq), np.float32)
    amp = [8 * math.exp(-(math.pi * 0.05 * k) ** 2) for k in range(1, H + 1)]
    for k in range(1, H + 1):
        pl[z0 + int(round(k * zf)), int(round(k * ff))] += amp[k - 1]
    dom = o.domain_2d(nfreq, 2 * z0 + 1, z0, H)
    snr, bh, path, allv = o.greedy_2d(pl, z0, H, *unit_norm(H), want_all=True)
    i = (z - dom[2]) * (dom[1] - dom[0] + 1) + (f - dom[0])
    np.testing.assert_allclose(allv[i], np.cumsum(np.float32(amp).astype(np.float64)), rtol=1e-12)
    df = dz = 0
    for k in range(1, H + 1):
        code = (int(path[i]) >> (4 * (k - 1))) & 0xF
        df += code % 3 - 1
        dz += code // 3 - 1
        assert df == int(round(k * ff)) - k * f and dz == int(round(k * zf)) - k * z


# ----------------------------------------------------------------------------------------
# sector footprint (compulsory input bytes)
# ----------------------------------------------------------------------------------------
def test_sector_footprint(oracle_lib):
    o = oracle_lib
    N, H = 1 << 14, 1
    nf = o.nf_1d(N, H)
    assert o.sectors_1d(1, 4, N, H) == -(-nf // 8)            # order 1 reads bins 0..nf-1
    assert o.sectors_1d(1, 2, N, H) == -(-nf // 16)
    # strictly increasing input: greedy reads h n + d, d = h-1 and h -> bins up to H n + H
    H = 4
    inc = np.arange(N, dtype=np.float32)
    path = o.greedy_1d(inc, H, *unit_norm(H))[2]
    nf = o.nf_1d(N, H)
    reads = set()
    for n in range(nf):
        reads.update({n, n + 1})
        for h in range(2, H + 1):
            reads.update({h * n + h - 1, h * n + h})
    assert o.sectors_1d(2, 4, N, H, path=path) == len({r // 8 for r in reads})
    # on noise, fused simple + greedy at H = 32 touch most (not all) sectors; the greedy form
    # alone touches a subset of the fused footprint, which contains the simple one
    x = synth.exp_noise(1 << 20, 1)
    path = o.greedy_1d(x, 32, *unit_norm(32))[2]
    both = o.sectors_1d(3, 4, 1 << 20, 32, path=path)
    g = o.sectors_1d(2, 4, 1 << 20, 32, path=path)
    s = o.sectors_1d(1, 4, 1 << 20, 32)
    assert max(g, s) <= both <= (1 << 20) // 8
    assert both > 0.95 * (1 << 20) // 8


def test_sector_footprint_2d(oracle_lib):
    """H = 1: the reads are exactly the 3x3 neighbourhoods of the fundamentals, so rows
    z0 + z - 1 .. z0 + z + 1 are read over columns f_lo - 1 .. f_hi + 1 (closed form)."""
    o = oracle_lib
    n_freq, n_rows, z0 = 4096, 21, 10
    pl = synth.plane(n_freq, n_rows, z0, 3)
    dom = o.domain_2d(n_freq, n_rows, z0, 1)
    path = o.greedy_2d(pl, z0, 1, *unit_norm(1))[2]
    f_lo, f_hi, z_lo, z_hi = dom
    rows = (z_hi + 1) - (z_lo - 1) + 1
    per_row = (f_hi + 1) // 8 - (f_lo - 1) // 8 + 1
    assert o.sectors_2d(n_freq, n_rows, z0, 1, path) == rows * per_row
    # higher orders only add sectors of the plane; never more than the plane holds
    path8 = o.greedy_2d(pl, z0, 3, *unit_norm(3))[2]
    c = o.sectors_2d(n_freq, n_rows, z0, 3, path8)
    assert 0 < c <= n_rows * n_freq // 8


def _ramp_plane(n_freq, n_rows, sf, sz):
    """Plane whose value strictly increases (s = +1) or decreases (s = -1) along f and z, or is
    constant (s = 0 for both): values r n_freq + c are exact in float32 for these sizes."""
    r = np.arange(n_rows, dtype=np.float64)[:, None]
    c = np.arange(n_freq, dtype=np.float64)[None, :]
    return (sz * r * n_freq + sf * c).astype(np.float32)


# (sign along f, sign along z) -> the 3x3 offset every order takes: the largest neighbour is the
# corner the ramp climbs towards; on a constant plane no neighbour is strictly larger than the
# centre, so the centre is kept
_RAMPS = [((1, 1), (1, 1)), ((-1, -1), (-1, -1)), ((1, -1), (1, -1)), ((-1, 1), (-1, 1)), ((0, 0), (0, 0))]


@pytest.mark.parametrize("H", [2, 3, 5, 8])
@pytest.mark.parametrize("signs,offset", _RAMPS)
def test_sector_footprint_2d_along_known_paths(oracle_lib, H, signs, offset):
    """On a ramp every order moves by the same 3x3 offset (of, oz), so the greedy path is known
    without the oracle: code (oz + 1) * 3 + (of + 1) at every order, and order h is centred at
    (h f + (h - 1) of, h z + (h - 1) oz).  The sector count must equal the number of distinct
    32-byte sectors of the 3x3 neighbourhoods along those paths, listed here in Python."""
    o = oracle_lib
    n_freq, n_rows, z0 = 512, 57, 28
    pl = _ramp_plane(n_freq, n_rows, *signs)
    of, oz = offset
    code = (oz + 1) * 3 + (of + 1)
    f_lo, f_hi, z_lo, z_hi = o.domain_2d(n_freq, n_rows, z0, H)
    path = o.greedy_2d(pl, z0, H, *unit_norm(H))[2]
    want = sum(code << (4 * (h - 1)) for h in range(1, H + 1))
    assert np.all(path == want)
    per_row = -(-n_freq // 8)
    sectors = set()
    for z in range(z_lo, z_hi + 1):
        for f in range(f_lo, f_hi + 1):
            for h in range(1, H + 1):
                cf, cr = h * f + (h - 1) * of, z0 + h * z + (h - 1) * oz
                for a in (-1, 0, 1):
                    for b in (-1, 0, 1):
                        sectors.add((cr + a) * per_row + (cf + b) // 8)
    assert o.sectors_2d(n_freq, n_rows, z0, H, path) == len(sectors)
    # a sub-domain counts only its own fundamentals' reads
    dom = (f_lo, min(f_hi, f_lo + 7), 0, 0)
    sub = o.greedy_2d(pl, z0, H, *unit_norm(H), dom=dom)[2]
    sec0 = set()
    for f in range(dom[0], dom[1] + 1):
        for h in range(1, H + 1):
            cf, cr = h * f + (h - 1) * of, z0 + (h - 1) * oz
            for a in (-1, 0, 1):
                for b in (-1, 0, 1):
                    sec0.add((cr + a) * per_row + (cf + b) // 8)
    assert o.sectors_2d(n_freq, n_rows, z0, H, sub, dom=dom) == len(sec0)


@pytest.mark.parametrize("signs,offset", _RAMPS)
def test_2d_brute_force_best_sum_closed_form(oracle_lib, signs, offset):
    """Exhaustive 2D enumeration on a ramp: the partial sum of h terms along any offset sequence
    is sum_k value(z0 + k z + Dz_k, k f + Df_k) with D the running sum of the offsets, which the
    ramp maximises by moving towards its top corner at every order.  So the best h-term sum is
    that closed form (exact in FP64), exactly one sequence obeys the greedy rule, and it is the
    all-(of, oz) path."""
    o = oracle_lib
    n_freq, n_rows, z0, H = 256, 41, 20, 5
    pl = _ramp_plane(n_freq, n_rows, *signs)
    sf, sz = signs
    of, oz = offset
    code = (oz + 1) * 3 + (of + 1)
    f_lo, f_hi, z_lo, z_hi = o.domain_2d(n_freq, n_rows, z0, H)
    for f, z in ((f_lo, z_lo), (f_hi, z_hi), ((f_lo + f_hi) // 2, 0), (f_lo + 3, z_hi - 1)):
        best, rule_path, rule_count = o.brute_2d(pl, z0, H, f, z)
        want, acc = [], 0.0
        for k in range(1, H + 1):
            r, c = z0 + k * z + k * oz, k * f + k * of
            acc += sz * r * n_freq + sf * c
            want.append(acc)
        assert np.array_equal(best, np.array(want)), (f, z, best, want)
        assert rule_count == 1
        assert rule_path == sum(code << (4 * (h - 1)) for h in range(1, H + 1))
    # a plane with one bright bin off the ramp's path: the optimum detours through it when that
    # pays, so best_sum exceeds the greedy sum by exactly the detour's gain (here the bright bin
    # sits at order 2 one column left of the greedy's (+1, +1) step on a constant plane)
    flat = np.zeros((n_rows, n_freq), np.float32)
    f, z = 10, 1
    flat[z0 + 2 * z, 2 * f - 1] = 5.0          # reachable at order 2 only by offset (-1, 0)
    best, rule_path, rule_count = o.brute_2d(flat, z0, H, f, z)
    assert np.array_equal(best, np.array([0.0, 5.0, 5.0, 5.0, 5.0]))
    # the greedy sees the bright bin in its order-2 neighbourhood and takes it
    assert rule_count == 1 and ((rule_path >> 4) & 0xF) == 3


def test_golden_footprints_match_oracle(oracle_lib):
    """tests/golden/footprints.json (the benchmark's compulsory input bytes) is what the
    oracle counts for the benchmark spectrum."""
    gold = json.load(open(os.path.join(GOLD, "footprints.json")))
    x = synth.long_spectrum()
    path = oracle_lib.greedy_1d(x, 32, *unit_norm(32))[2]
    assert gold["long"]["fused"]["sectors"] == oracle_lib.sectors_1d(3, 4, x.size, 32, path=path)
    assert gold["long"]["simple"]["sectors"] == oracle_lib.sectors_1d(1, 4, x.size, 32)


def test_openmp_build_matches_the_oracle(oracle_lib, tmp_path):
    """The all-core CPU baseline (liboracle_omp.so, the same source with its loops over
    fundamentals split over OpenMP threads) returns what the single-threaded oracle returns."""
    import subprocess
    import sys
    o = oracle_lib
    if not os.path.exists(o.LIB_OMP):
        pytest.skip("no OpenMP in this compiler")
    x = synth.spectrum(40000, 12, [synth.Pulsar(123.4, 0.05)])
    pl = synth.plane(2048, 41, 20, 8)
    np.save(tmp_path / "x.npy", x)
    np.save(tmp_path / "pl.npy", pl)
    code = (
        "import os, sys, numpy as np\n"
        "os.environ['OMP_NUM_THREADS'] = '4'\n"
        "import oracle\n"
        "assert oracle.use_openmp()\n"
        "x = np.load(sys.argv[1] + '/x.npy'); pl = np.load(sys.argv[1] + '/pl.npy')\n"
        "z, one = np.zeros(32), np.ones(32)\n"
        "s = oracle.simple_1d(x, 32, z, one, want_all=True)\n"
        "g = oracle.greedy_1d(x, 32, z, one, want_all=True)\n"
        "q = oracle.greedy_2d(pl, 20, 3, z[:3], one[:3], want_all=True)\n"
        "np.savez(sys.argv[1] + '/out.npz', *s, *g, *q)\n")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    subprocess.check_call([sys.executable, "-c", code, str(tmp_path)], cwd=root)
    got = np.load(tmp_path / "out.npz")
    z, one = np.zeros(32), np.ones(32)
    want = [*o.simple_1d(x, 32, z, one, want_all=True), *o.greedy_1d(x, 32, z, one, want_all=True),
            *o.greedy_2d(pl, 20, 3, z[:3], one[:3], want_all=True)]
    for i, w in enumerate(want):
        assert np.array_equal(got[f"arr_{i}"], w), i
