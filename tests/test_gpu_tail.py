"""GPU parity of the truncated tail (HS_FLAG_TRUNCATE_TAIL): fundamentals N_f <= n < N - 1 with
the orders that fit, every form, against the FP64 oracle through the C ABI."""
import numpy as np
import pytest
import torch

import synth
from hs_check import compare_argmax, compare_form, path_view

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda", 0)
TORCH_DT = {0: torch.float32, 1: torch.float16, 2: torch.bfloat16}


def oracle_full(o, form, x, H, mu, sg, mitigation, w):
    """Main domain then tail, concatenated: (snr, best_h, path, snr_all)."""
    nf = o.nf_1d(len(x), H)
    if form == 1:
        s, b, a = o.simple_1d(x, H, mu, sg, w=w, want_all=True)
        p = None
    elif form == 2:
        s, b, p, a = o.greedy_1d(x, H, mu, sg, mitigation=mitigation, w=w, want_all=True)
    else:
        s, b, a = o.optimal_1d(x, H, mu, sg, mitigation=mitigation, w=w, want_all=True)
        p = None
    ts, tb, tp, ta = o.tail_1d(form, x, H, mu, sg, mitigation=mitigation, w=w, want_all=True)
    # excluded orders (NaN) can never be the best: give compare_form -inf there
    ta = np.where(np.isnan(ta), -np.inf, ta)
    return (np.concatenate([s, ts]), np.concatenate([b, tb]),
            None if p is None else np.concatenate([p, tp]), np.concatenate([a, ta]))


def tail_case(hs, o, spectra, H, forms, mitigation=True, dtype=0, w=None, tuning=None, per_spec_norm=False):
    lengths = [len(s) for s in spectra]
    flags = hs.FLAG_TRUNCATE_TAIL | (0 if mitigation else hs.FLAG_NO_MITIGATION)
    flags |= hs.FLAG_WHITENING if w is not None else 0
    flags |= hs.FLAG_PER_SPECTRUM_NORM if per_spec_norm else 0
    plan = hs.Plan(H, forms, lengths=lengths, dtype=dtype, flags=flags)
    if tuning is not None:
        plan.tuning = tuning
    assert list(plan.counts) == [n - 1 for n in lengths]
    buf = torch.zeros(plan.extent, dtype=TORCH_DT[dtype])
    refs = []
    for s, x in enumerate(spectra):
        t = torch.from_numpy(np.ascontiguousarray(x, np.float32)).to(TORCH_DT[dtype])
        buf[int(plan.input_offsets[s]):int(plan.input_offsets[s]) + len(x)] = t
        refs.append(t.float().numpy())
    norms = {}
    for f in (1, 2, 4):
        if forms & f:
            if f == 4:
                mu = np.linspace(1.6, 1.6 * H, H).astype(np.float32)
                sg = np.sqrt(np.linspace(1.3, 1.3 * H, H)).astype(np.float32)
            else:
                mu, sg = hs.norm_exponential(f, 1, H, mitigation)
            if per_spec_norm:   # one row per spectrum, scaled per spectrum
                g = np.random.default_rng(77 + f)
                mu = (mu[None, :] * g.uniform(0.8, 1.2, (len(spectra), 1))).astype(np.float32)
                sg = (sg[None, :] * g.uniform(0.8, 1.2, (len(spectra), 1))).astype(np.float32)
            norms[f] = (mu, sg)
    dn = {f: (torch.from_numpy(m).to(DEV), torch.from_numpy(s).to(DEV)) for f, (m, s) in norms.items()}
    wd = None if w is None else torch.from_numpy(w).to(DEV)
    out = plan.forward(buf.to(DEV), dn.get(1), dn.get(2), w=wd, optimal_norm=dn.get(4))
    torch.cuda.synchronize()
    hs.check_device_error(plan)
    for s, x in enumerate(refs):
        a, b = int(plan.fund_offsets[s]), int(plan.fund_offsets[s + 1])
        for f in norms:
            mu, sg = norms[f]
            if per_spec_norm:
                mu, sg = mu[s], sg[s]
            r_snr, r_bh, r_path, r_all = oracle_full(o, f, x, H, mu, sg, mitigation, w)
            io = out[f]
            g_path = path_view(io.path, H)[a:b] if f == 2 else None
            compare_form(io.snr.cpu().numpy()[a:b], io.best_h.cpu().numpy()[a:b], r_snr, r_bh, r_all, mu, sg,
                         g_path, r_path, what=f"tail spectrum {s} form {f}")
            compare_argmax(io.argmax.cpu().numpy()[s], r_snr, io.snr.cpu().numpy()[a:b], mu, sg, r_bh,
                           hs.decode_argmax, what=f"tail argmax {s}/{f}")
    return plan, out, buf


@pytest.mark.parametrize("H", [2, 7, 16, 32])
@pytest.mark.parametrize("mitigation", [True, False])
def test_tail_all_forms(hs, oracle_lib, H, mitigation):
    x = synth.spectrum(9001, 40 + H, [synth.Pulsar(61.7, 0.05), synth.Pulsar(777.3, 0.08)])
    plan, _, _ = tail_case(hs, oracle_lib, [x], H, hs.SIMPLE | hs.GREEDY | hs.OPTIMAL, mitigation=mitigation)
    plan.close()


@pytest.mark.parametrize("dtype", [0, 1, 2])
def test_tail_batch_dtypes_and_shapes(hs, oracle_lib, dtype):
    xs = [synth.spectrum(n, 90 + n % 13) for n in (33, 2050, 4097, 70001, 34)]
    for t in (None, dict(kernel=0, threads=128), dict(kernel=3, threads=64, fund_per_thread=2),
              dict(kernel=6, threads=256, ctas_per_sm=4, dynamic=1), dict(kernel=7, threads=128),
              dict(kernel=2, threads=128, stages=12, stage_kb=17, producers=4)):
        plan, _, _ = tail_case(hs, oracle_lib, xs, 32, hs.SIMPLE | hs.GREEDY, dtype=dtype, tuning=t)
        plan.close()
    plan, _, _ = tail_case(hs, oracle_lib, xs, 8, hs.GREEDY, dtype=dtype)
    plan.close()


def test_tail_per_spectrum_norm(hs, oracle_lib):
    """Per-spectrum normalisation rows reach both kinds of tail tile (generic and one-order),
    several one-order tiles per spectrum, uneven lengths (spectrum found by binary search)."""
    xs = [synth.spectrum(n, 500 + n % 17, [synth.Pulsar(41.3, 0.06)]) for n in (5000, 40000, 20011, 9000)]
    plan, _, _ = tail_case(hs, oracle_lib, xs, 16, hs.SIMPLE | hs.GREEDY, per_spec_norm=True)
    plan.close()


def test_tail_whitening(hs, oracle_lib):
    N = 8192
    w = synth.whitening(N, 6)
    xs = [synth.spectrum(N, 300 + i, [synth.Pulsar(500.5 + i, 0.05)]) for i in range(3)]
    plan, _, _ = tail_case(hs, oracle_lib, xs, 16, hs.SIMPLE | hs.GREEDY | hs.OPTIMAL, w=w)
    plan.close()


def test_tail_pulse_train(hs, oracle_lib):
    """Noise-free harmonics of a fundamental past N_f (n = 200 of 4096 bins, H = 32): every form
    sums the 20 orders that fit (the oracle pin of the same case) and reports best h = 20."""
    N, H, n = 4096, 32, 200
    x = synth.inject(np.zeros(N, np.float32), [synth.Pulsar(200.0, 0.05, 8.0)])
    plan = hs.Plan(H, hs.SIMPLE | hs.GREEDY | hs.OPTIMAL, lengths=[N], flags=hs.FLAG_TRUNCATE_TAIL)
    z, one = torch.zeros(H, device=DEV), torch.ones(H, device=DEV)
    out = plan.forward(torch.from_numpy(x).to(DEV), (z, one), (z, one), optimal_norm=(z, one))
    k = np.arange(1, 21)
    want = np.sum(np.float32(8.0 * np.exp(-(np.pi * 0.05 * k) ** 2)).astype(np.float64))
    for f in (hs.SIMPLE, hs.GREEDY, hs.OPTIMAL):
        assert int(out[f].best_h.cpu().numpy()[n]) == 20
        assert abs(float(out[f].snr.cpu().numpy()[n]) - want) <= 1e-5 * want
    plan.close()


@pytest.mark.parametrize("form", [1, 2, 4])
def test_tail_adjoint(hs, oracle_lib, form):
    """The adjoint covers tail fundamentals: their bins follow their (shorter) chains."""
    N, H = 12001, 16
    x = synth.spectrum(N, 17, [synth.Pulsar(1000.2, 0.05)])
    plan, out, buf = tail_case(hs, oracle_lib, [x], H, form)
    io = out[form]
    g = synth.upstream_grad(plan.total_fundamentals, 41)
    gin = torch.zeros(plan.extent, dtype=torch.float32, device=DEV)
    hs.backward(plan, form, torch.from_numpy(g).to(DEV), io, buf.to(DEV), None, gin, None)
    torch.cuda.synchronize()
    sg = io.sigma.cpu().numpy()
    path = path_view(io.path, H) if form != 1 else None
    ref = oracle_lib.backward_1d(1 if form == 1 else 2, N, H, io.best_h.cpu().numpy(), sg,
                                 g.astype(np.float64), path)
    scale = np.abs(g).max() / sg.min() * H
    np.testing.assert_allclose(gin.cpu().numpy()[:N], ref, rtol=1e-5, atol=1e-6 * scale)
    plan.close()
