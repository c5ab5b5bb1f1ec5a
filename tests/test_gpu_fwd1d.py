"""GPU parity of the 1D forward (simple + greedy) against the FP64 oracle, through the C ABI."""
import numpy as np
import pytest
import torch

import synth
from hs_check import compare_argmax, compare_form, path_view

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda", 0)
TORCH_DT = {0: torch.float32, 1: torch.float16, 2: torch.bfloat16}


def stored(x, dtype):
    """Round host float32 values to the stored type; return (device-ready tensor, exact f32 view)."""
    t = torch.from_numpy(np.ascontiguousarray(x, np.float32)).to(TORCH_DT[dtype])
    return t, t.float().numpy()


def run_case(hs, o, spectra, H, forms=3, dtype=0, mitigation=True, w=None, tuning=None, flags=0,
             offsets=None, per_spec_norm=False, seed=0, check_argmax=True):
    lengths = [len(s) for s in spectra]
    if not mitigation:
        flags |= hs.FLAG_NO_MITIGATION
    if w is not None:
        flags |= hs.FLAG_WHITENING
    if per_spec_norm:
        flags |= hs.FLAG_PER_SPECTRUM_NORM
    plan = hs.Plan(H, forms, lengths=lengths, dtype=dtype, offsets=offsets, flags=flags)
    if tuning is not None:
        plan.tuning = tuning
    B = len(spectra)
    buf = torch.zeros(plan.extent, dtype=TORCH_DT[dtype])
    refs = []
    for s, x in enumerate(spectra):
        t, xf = stored(x, dtype)
        off = int(plan.input_offsets[s])
        buf[off:off + len(x)] = t
        refs.append(xf)
    xd = buf.to(DEV)
    wd = None if w is None else torch.from_numpy(w).to(DEV)
    rng = np.random.default_rng(seed)
    norms = {}
    for form in (1, 2):
        if not forms & form:
            continue
        mu, sg = hs.norm_exponential(form, 1, H, mitigation)
        if per_spec_norm:
            mu = (mu[None, :] * rng.uniform(0.8, 1.2, (B, 1))).astype(np.float32)
            sg = (sg[None, :] * rng.uniform(0.8, 1.2, (B, 1))).astype(np.float32)
        norms[form] = (mu, sg)
    ios = {f: (torch.from_numpy(m).to(DEV), torch.from_numpy(s).to(DEV)) for f, (m, s) in norms.items()}
    out = plan.forward(xd, ios.get(1), ios.get(2), w=wd)
    torch.cuda.synchronize()
    hs.check_device_error(plan)
    near = 0
    for s in range(B):
        a, b = int(plan.fund_offsets[s]), int(plan.fund_offsets[s + 1])
        for form in (1, 2):
            if not forms & form:
                continue
            mu, sg = norms[form]
            mu_s = mu[s] if per_spec_norm else mu
            sg_s = sg[s] if per_spec_norm else sg
            io = out[form]
            if form == 1:
                r_snr, r_bh, r_all = o.simple_1d(refs[s], H, mu_s, sg_s, w=w, want_all=True)
                r_path = g_path = None
            else:
                r_snr, r_bh, r_path, r_all = o.greedy_1d(refs[s], H, mu_s, sg_s, mitigation=mitigation, w=w,
                                                         want_all=True)
                g_path = path_view(io.path, H)[a:b]
            g_snr = io.snr.cpu().numpy()[a:b]
            g_bh = io.best_h.cpu().numpy()[a:b]
            near += compare_form(g_snr, g_bh, r_snr, r_bh, r_all, mu_s, sg_s, g_path, r_path,
                                 what=f"spectrum {s} form {form}")
            if check_argmax and io.argmax is not None:
                key = io.argmax.cpu().numpy()[s]
                compare_argmax(key, r_snr, g_snr, mu_s, sg_s, r_bh, hs.decode_argmax, what=f"argmax {s}/{form}")
    plan.close()
    return near


TUNINGS = [dict(kernel=0, threads=256),
           dict(kernel=1, threads=256),
           dict(kernel=1, threads=128, ctas_per_sm=2),
           dict(kernel=0, threads=64, ctas_per_sm=1, dynamic=1),
           dict(kernel=1, threads=192, ctas_per_sm=3, dynamic=1),
           dict(kernel=2, threads=128, stages=12, stage_kb=17, producers=4),
           dict(kernel=2, threads=64, stages=4, stage_kb=9, producers=2, ctas_per_sm=3),
           dict(kernel=2, threads=256, stages=6, stage_kb=33, producers=6, ctas_per_sm=1, prefetch=1),
           dict(kernel=2, threads=96, stages=3, stage_kb=13, producers=1, ctas_per_sm=2),
           dict(kernel=2, threads=448, stages=3, stage_kb=57, producers=3),
           dict(kernel=3, threads=128, fund_per_thread=2),
           dict(kernel=3, threads=64, fund_per_thread=2, ctas_per_sm=5),
           dict(kernel=4, threads=128),
           dict(kernel=5, threads=256, ctas_per_sm=3, dynamic=1),
           dict(kernel=6, threads=256),
           dict(kernel=6, threads=128, ctas_per_sm=8, prefetch=1),
           dict(kernel=7, threads=64, ctas_per_sm=6, dynamic=1, prefetch=1),
           dict(kernel=7, threads=256, ctas_per_sm=2),
           dict(kernel=7, threads=128, ctas_per_sm=16, prefetch=1),
           dict(kernel=6, threads=192, ctas_per_sm=3, dynamic=1),
           dict(kernel=3, threads=128, fund_per_thread=2, prefetch=2),
           dict(kernel=0, threads=256, prefetch=2),
           dict(kernel=6, threads=128, prefetch=3),
           dict(kernel=7, threads=64, ctas_per_sm=8, prefetch=2)]
# one launch shape per kernel id, for the tests that sweep ids
BY_KERNEL = {1: TUNINGS[1], 2: TUNINGS[5], 3: TUNINGS[10], 6: TUNINGS[14], 7: TUNINGS[16]}


@pytest.mark.parametrize("tuning", TUNINGS)
@pytest.mark.parametrize("H", [1, 2, 7, 8, 9, 16, 17, 31, 32])
def test_fused_f32_shapes(hs, oracle_lib, H, tuning):
    x = synth.spectrum(40001, 100 + H, [synth.Pulsar(211.37, 0.05), synth.Pulsar(97.9, 0.1)])
    run_case(hs, oracle_lib, [x], H, tuning=tuning)


@pytest.mark.parametrize("kernel", [1, 2, 3, 6, 7])
@pytest.mark.parametrize("forms", [1, 2, 3])
@pytest.mark.parametrize("mitigation", [True, False])
@pytest.mark.parametrize("dtype", [0, 1, 2])
def test_forms_dtypes(hs, oracle_lib, forms, mitigation, dtype, kernel):
    x = synth.single_pulse_spectrum()
    t = BY_KERNEL[kernel]
    run_case(hs, oracle_lib, [x], 32, forms=forms, dtype=dtype, mitigation=mitigation, tuning=t)


@pytest.mark.parametrize("dtype", [0, 1, 2])
@pytest.mark.parametrize("n", [4097, 4098, 4099, 40003])
def test_window_unaligned_tails(hs, oracle_lib, dtype, n):
    """Spectra whose last window ends off a 16-byte boundary at the very end of the input
    buffer: the bulk copy stops at the last whole 16-byte unit and the rest is loaded directly."""
    xs = [synth.spectrum(n - 7, 3), synth.spectrum(n, 4)]
    for t in (TUNINGS[5], TUNINGS[6], TUNINGS[14], TUNINGS[16], TUNINGS[18]):
        run_case(hs, oracle_lib, xs, 7, dtype=dtype, tuning=t)
        run_case(hs, oracle_lib, xs, 32, dtype=dtype, tuning=t)


@pytest.mark.parametrize("kernel", [0, 1, 3, 6, 7])
@pytest.mark.parametrize("N", [65536, 65533])
def test_whitening(hs, oracle_lib, kernel, N):
    """N = 65533: w and the spectra end off a 16-byte boundary."""
    w = synth.whitening(N, 5)
    xs = [synth.spectrum(N, 50 + i, [synth.Pulsar(300.4 + 17 * i, 0.07)]) for i in range(3)]
    for dtype in (0, 1, 2):
        for forms in (3, 2):
            run_case(hs, oracle_lib, xs, 16, w=w, dtype=dtype, forms=forms,
                     tuning=dict(kernel=kernel, threads=256, fund_per_thread=2 if kernel == 3 else 1))


def test_small_and_degenerate_lengths(hs, oracle_lib):
    """N = H+1 (one fundamental), ragged tails, many tiny spectra in one batch."""
    H = 8
    lens = [9, 10, 17, 31, 33, 64, 65, 255, 257, 1000, 2049, 4097]
    xs = [synth.spectrum(n, 900 + n) for n in lens]
    for t in TUNINGS:
        run_case(hs, oracle_lib, xs, H, tuning=t)


def test_uneven_batch_per_spectrum_norm(hs, oracle_lib):
    b = synth.uneven_batch(count=24, seed=77, choices=(1 << 12, 1 << 13, 1 << 15, 1 << 17), pulsar_fraction=0.25)
    xs = [synth.batch_trial(b, i) for i in range(24)]
    for t in (TUNINGS[1], TUNINGS[4], TUNINGS[5], TUNINGS[8], TUNINGS[15], TUNINGS[16], TUNINGS[20],
              TUNINGS[21], TUNINGS[22], TUNINGS[23]):
        run_case(hs, oracle_lib, xs, 16, per_spec_norm=True, tuning=t)
        run_case(hs, oracle_lib, xs, 16, dtype=1, tuning=t)


def test_custom_offsets(hs, oracle_lib):
    xs = [synth.spectrum(5000, 1), synth.spectrum(3000, 2), synth.spectrum(7001, 3)]
    run_case(hs, oracle_lib, xs, 12, offsets=[12000, 0, 4000])


def test_small_integer_spectra_bit_exact(hs, oracle_lib):
    """Integer powers: FP32 sums are exact, so with mu = 0, sigma = 1 the SNR is bit-exact."""
    N, H = 30011, 32
    x = synth.small_int_spectrum(N, 9)
    plan = hs.Plan(H, 3, lengths=[N])
    z = torch.zeros(H, device=DEV)
    one = torch.ones(H, device=DEV)
    out = plan.forward(torch.from_numpy(x).to(DEV), (z, one), (z, one))
    rs, rbh = oracle_lib.simple_1d(x, H, np.zeros(H), np.ones(H))
    gs, gbh, gp = oracle_lib.greedy_1d(x, H, np.zeros(H), np.ones(H))
    assert np.array_equal(out[1].snr.cpu().numpy().astype(np.float64), rs)
    assert np.array_equal(out[2].snr.cpu().numpy().astype(np.float64), gs)
    assert np.array_equal(out[1].best_h.cpu().numpy(), rbh)       # dense ties: lowest h
    assert np.array_equal(out[2].best_h.cpu().numpy(), gbh)
    assert np.array_equal(path_view(out[2].path, H), gp)


def test_h1_returns_input(hs):
    N = 10000
    x = synth.spectrum(N, 4)
    z, one = torch.zeros(1, device=DEV), torch.ones(1, device=DEV)
    xd = torch.from_numpy(x).to(DEV)
    for flags, expect in ((0, np.maximum(x[:-1], x[1:])), (hs.FLAG_NO_MITIGATION, x[:-1])):
        plan = hs.Plan(1, 3, lengths=[N], flags=flags)
        out = plan.forward(xd, (z, one), (z, one))
        assert np.array_equal(out[1].snr.cpu().numpy(), x[:-1])
        assert np.array_equal(out[2].snr.cpu().numpy(), expect)


def test_pulse_train_recovered(hs, oracle_lib):
    x = synth.single_pulse_spectrum()
    plan = hs.Plan(32, 3, lengths=[x.size])
    ns = [torch.from_numpy(a).to(DEV) for a in hs.norm_exponential(1, 1, 32)]
    ng = [torch.from_numpy(a).to(DEV) for a in hs.norm_exponential(2, 1, 32)]
    out = plan.forward(torch.from_numpy(x).to(DEV), ns, ng)
    snr, n = hs.decode_argmax(out[2].argmax.cpu().numpy()[0])
    assert n == 1234


def test_checked_mode_and_graph(hs, oracle_lib):
    x = synth.spectrum(100003, 12)
    near = run_case(hs, oracle_lib, [x], 24, flags=hs.FLAG_CHECKED)
    assert near <= 2
    # graph replay: repeated runs and a changed output buffer give the same answers
    plan = hs.Plan(24, 3, lengths=[x.size], flags=hs.FLAG_GRAPH)
    ns = [torch.from_numpy(a).to(DEV) for a in hs.norm_exponential(1, 1, 24)]
    ng = [torch.from_numpy(a).to(DEV) for a in hs.norm_exponential(2, 1, 24)]
    xd = torch.from_numpy(x).to(DEV)
    ref = plan.forward(xd, ns, ng)
    for _ in range(3):
        again = plan.forward(xd, ns, ng)
        for f in (1, 2):
            assert torch.equal(again[f].snr, ref[f].snr)
            assert torch.equal(again[f].argmax, ref[f].argmax)


def test_autotune(hs, oracle_lib):
    b = synth.uneven_batch(count=6, seed=5, choices=(1 << 16, 1 << 18))
    xs = [synth.batch_trial(b, i) for i in range(6)]
    run_case(hs, oracle_lib, xs, 16, flags=hs.FLAG_AUTOTUNE)


@pytest.mark.parametrize("dtype", [0, 1])
def test_autotune_whitening(hs, oracle_lib, dtype):
    """The autotuner times a whitening plan's candidates on the path hs_run takes (the whitened
    copy, then the plain FP32 pass) and the chosen shape still agrees with the oracle."""
    N = 1 << 18
    w = synth.whitening(N, 9)
    xs = [synth.spectrum(N, 60 + i, [synth.Pulsar(501.2 + 13 * i, 0.06)]) for i in range(4)]
    run_case(hs, oracle_lib, xs, 16, w=w, dtype=dtype, flags=hs.FLAG_AUTOTUNE)


def test_long_spectrum_full_size(hs, oracle_lib):
    """The 2^23-bin, H = 32 single-spectrum workload in the default launch configuration."""
    x = synth.long_spectrum()
    near = run_case(hs, oracle_lib, [x], 32)
    assert near <= 5


@pytest.mark.parametrize("t", [TUNINGS[14], TUNINGS[15], TUNINGS[16], TUNINGS[19]])
def test_long_spectrum_full_size_pair(hs, oracle_lib, t):
    """The same workload through the paired-lane kernels (persistent, dynamic, L2 prefetch)."""
    x = synth.long_spectrum()
    near = run_case(hs, oracle_lib, [x], 32, tuning=t)
    assert near <= 5


@pytest.mark.parametrize("limit_us", [2000, 50000])
def test_bounded_wait_reports_timeout(hs, oracle_lib, limit_us):
    """A wait that nothing completes gives up after its limit and reports HS_ERR_DEVICE_TIMEOUT
    through the plan's error word; the context and the plan stay usable afterwards."""
    import time
    x = synth.spectrum(20000, 5)
    plan = hs.Plan(16, hs.SIMPLE | hs.GREEDY, lengths=[len(x)])
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    hs.selftest_timeout(plan, limit_us)
    with pytest.raises(hs.HSError) as e:
        hs.check_device_error(plan)
    waited = time.perf_counter() - t0
    assert e.value.status == 6                     # HS_ERR_DEVICE_TIMEOUT
    assert waited >= limit_us * 1e-6 * 0.9 and waited < 5.0
    hs.check_device_error(plan)                    # the error word was cleared
    plan.close()
    run_case(hs, oracle_lib, [x], 16)              # and the device still computes


@pytest.mark.parametrize("dtype", [0, 1, 2])
@pytest.mark.parametrize("flags", [0, 128])
def test_whitening_copy_equals_multiply_on_load(hs, oracle_lib, dtype, flags):
    """A whitening plan given a workspace writes fl32(w p) into it and runs the plain FP32 pass on
    that copy; without one (the fixed-scratch entry point) the pass multiplies as it loads.  Both
    give the same outputs bit for bit (the truncated tail included), and the oracle agrees."""
    N, B, H = 40013, 3, 16
    xs = [synth.spectrum(N, 810 + i, [synth.Pulsar(91.3 + 7 * i, 0.05)]) for i in range(B)]
    w = synth.whitening(N, 44)
    if not flags:      # (the tail's oracle comparison with whitening is in test_gpu_tail.py)
        assert run_case(hs, oracle_lib, xs, H, dtype=dtype, w=w) <= 4
    plan = hs.Plan(H, hs.SIMPLE | hs.GREEDY, lengths=[N] * B, dtype=dtype, flags=hs.FLAG_WHITENING | flags)
    assert plan.workspace_bytes >= plan.extent * 4
    buf = torch.zeros(plan.extent, dtype=TORCH_DT[dtype])
    for s, x in enumerate(xs):
        o = int(plan.input_offsets[s])
        buf[o:o + N] = stored(x, dtype)[0]
    xd, wd = buf.to(DEV), torch.from_numpy(w).to(DEV)
    ns = [torch.from_numpy(a).to(DEV) for a in hs.norm_exponential(hs.SIMPLE, 1, H)]
    ng = [torch.from_numpy(a).to(DEV) for a in hs.norm_exponential(hs.GREEDY, 1, H)]
    outs = []
    for how in ("copy", "on load"):
        s_io, g_io = plan.alloc_form(*ns, path=False), plan.alloc_form(*ng)
        if how == "copy":
            hs.run(plan, xd, wd, s_io, g_io)
        else:
            hs.run_fixed_scratch(plan, xd, wd, s_io, g_io)
        torch.cuda.synchronize()
        hs.check_device_error(plan)
        outs.append([s_io.snr, s_io.best_h, s_io.argmax, g_io.snr, g_io.best_h, g_io.path, g_io.argmax])
    for a, b in zip(*outs):
        assert torch.equal(a, b)
    plan.close()


@pytest.mark.parametrize("tuning", [None, dict(kernel=0, threads=128, ctas_per_sm=4, dynamic=1)])
def test_whitening_workspace_off_16_bytes(hs, tuning):
    """A workspace that is 8- but not 16-byte aligned cannot take the whitened copy's 16-byte
    stores: the pass then multiplies as it loads (the dynamic schedule's counter still lives at
    its start), with the same outputs bit for bit as with an aligned workspace."""
    N, B, H = 40013, 2, 16
    xs = [synth.spectrum(N, 850 + i, [synth.Pulsar(61.3 + 5 * i, 0.05)]) for i in range(B)]
    plan = hs.Plan(H, hs.SIMPLE | hs.GREEDY, lengths=[N] * B, flags=hs.FLAG_WHITENING)
    if tuning:
        plan.tuning = tuning
    buf = torch.zeros(plan.extent, dtype=torch.float32)
    for s, x in enumerate(xs):
        o = int(plan.input_offsets[s])
        buf[o:o + N] = torch.from_numpy(x)
    xd, wd = buf.to(DEV), torch.from_numpy(synth.whitening(N, 47)).to(DEV)
    ns = [torch.from_numpy(a).to(DEV) for a in hs.norm_exponential(hs.SIMPLE, 1, H)]
    ng = [torch.from_numpy(a).to(DEV) for a in hs.norm_exponential(hs.GREEDY, 1, H)]
    big = torch.zeros(plan.workspace_bytes + 256, dtype=torch.uint8, device=DEV)
    outs = []
    for ws in (big[:plan.workspace_bytes], big[8:8 + plan.workspace_bytes]):
        s_io, g_io = plan.alloc_form(*ns, path=False), plan.alloc_form(*ng)
        hs.run(plan, xd, wd, s_io, g_io, workspace=ws)
        torch.cuda.synchronize()
        hs.check_device_error(plan)
        outs.append([s_io.snr, s_io.best_h, s_io.argmax, g_io.snr, g_io.best_h, g_io.path, g_io.argmax])
    assert big.data_ptr() % 256 == 0
    for a, b in zip(*outs):
        assert torch.equal(a, b)
    plan.close()
