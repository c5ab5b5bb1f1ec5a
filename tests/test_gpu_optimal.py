"""GPU parity of the optimal form (the dynamic programme over monotone drift paths, Sec. 2.2)
against the FP64 oracle, through the C ABI (hs_run_optimal)."""
import numpy as np
import pytest
import torch

import synth
from hs_check import compare_argmax, compare_form, path_view

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda", 0)
TORCH_DT = {0: torch.float32, 1: torch.float16, 2: torch.bfloat16}


def drifts(path, H):
    """D_k = popcount(path & ((1 << k) - 1)) for k = 1..H, per fundamental: int64 [F, H]."""
    p = path.astype(np.uint64)
    out = np.zeros((p.size, H), np.int64)
    acc = np.zeros(p.size, np.int64)
    for k in range(1, H + 1):
        acc += ((p >> np.uint64(k - 1)) & np.uint64(1)).astype(np.int64)
        out[:, k - 1] = acc
    return out


def path_sums(x, H, path, bh):
    """FP64 sum of x[k n + D_k] over k <= best h along each reported path."""
    n = np.arange(path.size, dtype=np.int64)
    d = drifts(path, H)
    xs = x.astype(np.float64)
    tot = np.zeros(path.size)
    for k in range(1, H + 1):
        sel = bh >= k
        tot[sel] += xs[k * n[sel] + d[sel, k - 1]]
    return tot


def opt_case(hs, o, spectra, H, mitigation=True, dtype=0, w=None, per_spec_norm=False, seed=0):
    lengths = [len(s) for s in spectra]
    flags = (0 if mitigation else hs.FLAG_NO_MITIGATION) | (hs.FLAG_WHITENING if w is not None else 0)
    flags |= hs.FLAG_PER_SPECTRUM_NORM if per_spec_norm else 0
    plan = hs.Plan(H, hs.OPTIMAL, lengths=lengths, dtype=dtype, flags=flags)
    buf = torch.zeros(plan.extent, dtype=TORCH_DT[dtype])
    refs = []
    for s, x in enumerate(spectra):
        t = torch.from_numpy(np.ascontiguousarray(x, np.float32)).to(TORCH_DT[dtype])
        buf[int(plan.input_offsets[s]):int(plan.input_offsets[s]) + len(x)] = t
        refs.append(t.float().numpy())
    rng = np.random.default_rng(seed)
    # mu/sigma of the optimum have no closed form: any positive table exercises Eq. 2
    mu = np.linspace(1.6, 1.6 * H, H).astype(np.float32)
    sg = np.sqrt(np.linspace(1.3, 1.3 * H, H)).astype(np.float32)
    if per_spec_norm:
        mu = (mu[None, :] * rng.uniform(0.8, 1.2, (len(spectra), 1))).astype(np.float32)
        sg = (sg[None, :] * rng.uniform(0.8, 1.2, (len(spectra), 1))).astype(np.float32)
    nrm = (torch.from_numpy(mu).to(DEV), torch.from_numpy(sg).to(DEV))
    wd = None if w is None else torch.from_numpy(w).to(DEV)
    out = plan.forward(buf.to(DEV), w=wd, optimal_norm=nrm)[hs.OPTIMAL]
    torch.cuda.synchronize()
    hs.check_device_error(plan)
    snr_all = out.snr.cpu().numpy()
    bh_all = out.best_h.cpu().numpy()
    path_all = path_view(out.path, H)
    near = 0
    for s, x in enumerate(refs):
        a, b = int(plan.fund_offsets[s]), int(plan.fund_offsets[s + 1])
        mu_s = mu[s] if per_spec_norm else mu
        sg_s = sg[s] if per_spec_norm else sg
        r_snr, r_bh, r_all = o.optimal_1d(x, H, mu_s, sg_s, mitigation=mitigation, w=w, want_all=True)
        g_snr, g_bh, g_path = snr_all[a:b], bh_all[a:b], path_all[a:b]
        near += compare_form(g_snr, g_bh, r_snr, r_bh, r_all, mu_s, sg_s, what=f"optimal spectrum {s}")
        # the reported path is a valid drift path of the reported order ...
        assert np.all((g_path >> g_bh.astype(np.uint32)) == 0), "path bits beyond best h"
        if not mitigation:
            assert np.all((g_path & 1) == 0), "increment at order 1 without mitigation"
        # ... and an optimal one: its FP64 sum is the oracle's optimum of that order
        xs = x if w is None else (w.astype(np.float32) * x).astype(np.float32)
        got = path_sums(xs, H, g_path, g_bh.astype(np.int64))
        _, _, sums = o.optimal_1d(x, H, np.zeros(H), np.ones(H), mitigation=mitigation, w=w, want_all=True)
        opt = sums[np.arange(g_bh.size), g_bh.astype(np.int64) - 1]
        np.testing.assert_allclose(got, opt, rtol=1e-5, atol=1e-6, err_msg=f"spectrum {s}: path not optimal")
        compare_argmax(out.argmax.cpu().numpy()[s], r_snr, g_snr, mu_s, sg_s, r_bh, hs.decode_argmax,
                       what=f"optimal argmax {s}")
    plan.close()
    return near, out


@pytest.mark.parametrize("H", [1, 2, 7, 8, 16, 31, 32])
@pytest.mark.parametrize("mitigation", [True, False])
def test_optimal_matches_oracle(hs, oracle_lib, H, mitigation):
    x = synth.spectrum(30001, 200 + H, [synth.Pulsar(211.37, 0.05), synth.Pulsar(97.9, 0.1)])
    opt_case(hs, oracle_lib, [x], H, mitigation=mitigation)


@pytest.mark.parametrize("dtype", [0, 1, 2])
def test_optimal_batch_dtypes(hs, oracle_lib, dtype):
    xs = [synth.spectrum(n, 10 + n % 7) for n in (33, 4097, 20000, 9, 65536)]
    opt_case(hs, oracle_lib, xs, 8, dtype=dtype, per_spec_norm=True)
    opt_case(hs, oracle_lib, xs[:3], 32, dtype=dtype)


def test_optimal_whitening(hs, oracle_lib):
    N = 16384
    w = synth.whitening(N, 3)
    xs = [synth.spectrum(N, 70 + i, [synth.Pulsar(123.4 + i, 0.05)]) for i in range(3)]
    opt_case(hs, oracle_lib, xs, 32, w=w)


def test_optimal_small_integers_bit_exact(hs, oracle_lib):
    """Integer powers: FP32 sums along every path are exact, so with mu = 0, sigma = 1 the
    optimum is bit-exact and dense ties exercise the lowest-h rule."""
    N, H = 20011, 32
    x = synth.small_int_spectrum(N, 11)
    plan = hs.Plan(H, hs.OPTIMAL, lengths=[N])
    z, one = torch.zeros(H, device=DEV), torch.ones(H, device=DEV)
    out = plan.forward(torch.from_numpy(x).to(DEV), optimal_norm=(z, one))[hs.OPTIMAL]
    r_snr, r_bh = oracle_lib.optimal_1d(x, H, np.zeros(H), np.ones(H))
    assert np.array_equal(out.snr.cpu().numpy().astype(np.float64), r_snr)
    assert np.array_equal(out.best_h.cpu().numpy(), r_bh)
    plan.close()


def test_optimal_bounds_greedy_and_simple(hs, oracle_lib):
    """On the same input the optimum's SNR at any order is at least the greedy's and the simple
    form's (every path they take is a monotone drift path) -- checked with a common mu, sigma."""
    N, H = 50001, 32
    x = synth.spectrum(N, 5, [synth.Pulsar(300.2, 0.05)])
    plan = hs.Plan(H, hs.SIMPLE | hs.GREEDY | hs.OPTIMAL, lengths=[N])
    z, one = torch.zeros(H, device=DEV), torch.ones(H, device=DEV)
    out = plan.forward(torch.from_numpy(x).to(DEV), (z, one), (z, one), optimal_norm=(z, one))
    so, go, oo = (out[f].snr.cpu().numpy().astype(np.float64) for f in (hs.SIMPLE, hs.GREEDY, hs.OPTIMAL))
    # mu = 0, sigma = 1: the maxima over h are the order-H sums of nonnegative powers
    assert np.all(oo >= go * (1 - 1e-6)) and np.all(oo >= so * (1 - 1e-6))
    plan.close()


def test_optimal_adjoint(hs, oracle_lib):
    """hs_backward of the optimal form scatters along the reported optimal path, as the oracle's
    adjoint does for that path."""
    N, H = 40001, 24
    x = synth.spectrum(N, 8, [synth.Pulsar(157.3, 0.05)])
    plan = hs.Plan(H, hs.OPTIMAL, lengths=[N])
    mu = np.linspace(1.6, 1.6 * H, H).astype(np.float32)
    sg = np.sqrt(np.linspace(1.3, 1.3 * H, H)).astype(np.float32)
    nrm = (torch.from_numpy(mu).to(DEV), torch.from_numpy(sg).to(DEV))
    xd = torch.from_numpy(x).to(DEV)
    out = plan.forward(xd, optimal_norm=nrm)[hs.OPTIMAL]
    g = synth.upstream_grad(plan.total_fundamentals, 31)
    gin = torch.zeros(plan.extent, dtype=torch.float32, device=DEV)
    hs.backward(plan, hs.OPTIMAL, torch.from_numpy(g).to(DEV), out, xd, None, gin, None)
    torch.cuda.synchronize()
    ref = oracle_lib.backward_1d(2, N, H, out.best_h.cpu().numpy(), sg, g.astype(np.float64),
                                 path_view(out.path, H))
    scale = np.abs(g).max() / sg.min() * H
    np.testing.assert_allclose(gin.cpu().numpy()[:N], ref, rtol=1e-5, atol=1e-6 * scale)
    plan.close()


def test_optimal_full_size(hs, oracle_lib):
    """The 2^23-bin H = 32 benchmark spectrum: sampled fundamentals against the oracle."""
    x = synth.long_spectrum()
    H = 32
    plan = hs.Plan(H, hs.OPTIMAL, lengths=[x.size])
    mu = np.linspace(1.6, 1.6 * H, H).astype(np.float32)
    sg = np.sqrt(np.linspace(1.3, 1.3 * H, H)).astype(np.float32)
    nrm = (torch.from_numpy(mu).to(DEV), torch.from_numpy(sg).to(DEV))
    out = plan.forward(torch.from_numpy(x).to(DEV), optimal_norm=nrm)[hs.OPTIMAL]
    snr = out.snr.cpu().numpy()
    bh = out.best_h.cpu().numpy()
    rng = np.random.default_rng(3)
    nf = plan.total_fundamentals
    pick = np.unique(np.concatenate([rng.integers(0, nf, 3000), np.arange(nf - 2000, nf)]))
    from hs_check import tol_at
    for n in pick:
        sums = oracle_lib.dp_1d(x, H, int(n))
        v = (sums - mu) / sg
        h = 0
        for k in range(1, H):
            if v[k] > v[h]:
                h = k
        tol = tol_at(np.array([v[h]]), np.array([h + 1]), mu, sg)[0]
        assert abs(snr[n] - v[h]) <= tol, (n, snr[n], v[h])
        assert bh[n] == h + 1 or abs(v[bh[n] - 1] - v[h]) <= tol, (n, bh[n], h + 1)
    plan.close()
