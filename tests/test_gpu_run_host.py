"""hs_run_host (input from page-locked host memory, copied in chunks while earlier chunks run)
gives bit for bit the outputs of hs_run on the same input, on the device and in the host copies."""
import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda", 0)
TORCH_DT = {0: torch.float32, 1: torch.float16, 2: torch.bfloat16}


def layout(plan, spectra, dtype):
    buf = torch.zeros(plan.extent, dtype=TORCH_DT[dtype])
    for s, x in enumerate(spectra):
        off = int(plan.input_offsets[s])
        buf[off:off + len(x)] = torch.from_numpy(np.ascontiguousarray(x, np.float32)).to(TORCH_DT[dtype])
    return buf


def norms(hs, plan, form, mitigation=True, per_spec=False):
    mu, sg = hs.norm_exponential(form, plan.dims, plan.H, mitigation, 1.0 if plan.dims == 1 else 2.0)
    if per_spec:
        g = np.random.default_rng(form)
        mu = (mu[None, :] * g.uniform(0.8, 1.2, (plan.B, 1))).astype(np.float32)
        sg = (sg[None, :] * g.uniform(0.8, 1.2, (plan.B, 1))).astype(np.float32)
    return torch.from_numpy(mu).to(DEV), torch.from_numpy(sg).to(DEV)


def same(a, b, what):
    if a is None and b is None:
        return
    assert torch.equal(a.cpu(), b.cpu()), what


def check(hs, plan, buf, w=None, per_spec=False, mitigation=True):
    forms = plan.forms
    ns = norms(hs, plan, 1, mitigation, per_spec) if forms & 1 else None
    ng = norms(hs, plan, 2, mitigation, per_spec) if forms & 2 else None
    ref_s = plan.alloc_form(*ns, path=False) if ns else None
    ref_g = plan.alloc_form(*ng) if ng else None
    dev = buf.to(DEV)
    wd = None if w is None else torch.from_numpy(w).to(DEV)
    hs.run(plan, dev, wd, ref_s, ref_g)
    out_s = plan.alloc_form(*ns, path=False) if ns else None
    out_g = plan.alloc_form(*ng) if ng else None
    host_s = plan.alloc_form_host(path=False) if ns else None
    host_g = plan.alloc_form_host() if ng else None
    hbuf = buf.pin_memory()
    dbuf = torch.full_like(dev, 7)       # stale contents: every bin read must come from the copy
    for _ in range(2):                   # twice: the second call reuses the plan's streams and events
        hs.run_host(plan, hbuf, dbuf, wd, out_s, out_g, host_s, host_g)
        torch.cuda.synchronize()
        hs.check_device_error(plan)
        assert torch.equal(dbuf.cpu(), buf)
        for ref, out, host, name in ((ref_s, out_s, host_s, "simple"), (ref_g, out_g, host_g, "greedy")):
            if ref is None:
                continue
            for field in ("snr", "best_h", "path", "argmax"):
                r = getattr(ref, field)
                if r is None:
                    continue
                same(r, getattr(out, field), f"{name} {field} (device)")
                same(r, getattr(host, field), f"{name} {field} (host copy)")


@pytest.mark.parametrize("chunks", [0, 1, 7, 16])
def test_long_spectrum_chunks(hs, chunks):
    """32 MiB: the default (two chunks of fundamentals) and other chunk counts, paired lanes."""
    x = synth.long_spectrum()
    plan = hs.Plan(32, hs.SIMPLE | hs.GREEDY, lengths=[len(x)])
    plan.host_chunks = chunks
    check(hs, plan, layout(plan, [x], 0))


@pytest.mark.parametrize("tuning", [dict(kernel=0, threads=256), dict(kernel=3, threads=128, fund_per_thread=2),
                                    dict(kernel=2, threads=128, stages=12, stage_kb=17, producers=4),
                                    dict(kernel=6, threads=128, ctas_per_sm=8, dynamic=1),
                                    dict(kernel=7, threads=64, ctas_per_sm=6, dynamic=1),
                                    dict(kernel=1, threads=192, ctas_per_sm=3, dynamic=1)])
@pytest.mark.parametrize("forms", [1, 2, 3])
def test_launch_shapes(hs, tuning, forms):
    x = synth.spectrum(3 * (1 << 21) + 77, 5, synth.random_pulsars(4, 3 << 21, 6))
    plan = hs.Plan(32, forms, lengths=[len(x)])
    plan.tuning = tuning
    check(hs, plan, layout(plan, [x], 0))


@pytest.mark.parametrize("chunks", [0, 16])
@pytest.mark.parametrize("dtype", [0, 1])
def test_batch_groups(hs, dtype, chunks):
    b = synth.uneven_batch(count=40, seed=91, choices=(1 << 17, 1 << 19, 1 << 20, 1 << 21), pulsar_fraction=0.2)
    xs = [synth.batch_trial(b, i) for i in range(40)]
    plan = hs.Plan(16, hs.SIMPLE | hs.GREEDY, lengths=[len(x) for x in xs], dtype=dtype,
                   flags=hs.FLAG_PER_SPECTRUM_NORM)
    plan.host_chunks = chunks
    check(hs, plan, layout(plan, xs, dtype), per_spec=True)


def test_truncated_tail_and_unmitigated(hs):
    """With the tail the outputs come back after the whole pass."""
    x = synth.spectrum((1 << 22) + 5, 8, synth.random_pulsars(3, 1 << 22, 9))
    plan = hs.Plan(24, hs.SIMPLE | hs.GREEDY, lengths=[len(x)], flags=hs.FLAG_TRUNCATE_TAIL | hs.FLAG_NO_MITIGATION)
    check(hs, plan, layout(plan, [x], 0), mitigation=False)


def test_whitening_bf16(hs):
    N = 1 << 21
    w = synth.whitening(N, 3)
    xs = [synth.spectrum(N, 30 + i) for i in range(6)]
    plan = hs.Plan(32, hs.GREEDY, lengths=[N] * 6, dtype=hs.BF16, flags=hs.FLAG_WHITENING)
    check(hs, plan, layout(plan, xs, 2), w=w)


def test_unordered_offsets_single_chunk(hs):
    xs = [synth.spectrum(1 << 21, 40 + i) for i in range(5)]
    offs = [4 << 21, 0, 2 << 21, 1 << 21, 3 << 21]
    plan = hs.Plan(16, hs.SIMPLE | hs.GREEDY, lengths=[len(x) for x in xs], offsets=offs)
    check(hs, plan, layout(plan, xs, 0))


@pytest.mark.parametrize("n_freq,tuning", [(5003, None), (5008, dict(kernel=2, threads=512))])
def test_plane(hs, n_freq, tuning):
    """A plane goes in one copy; then kernel 1 or the column sweep (here at the 16-column band
    width the plane takes; its rows must be a multiple of 16 bytes) runs as under hs_run."""
    z0 = 30
    pl = synth.plane(n_freq, 2 * z0 + 1, z0, 12, synth.random_tracks(3, n_freq, 8, f_lo=50, zmax=3))
    plan = hs.Plan(4, hs.GREEDY, dims=2, n_freq=n_freq, n_rows=2 * z0 + 1, z0_row=z0)
    if tuning:
        plan.tuning = tuning
        assert plan.tuning.kernel == 2
    check(hs, plan, torch.from_numpy(pl).reshape(-1))


def test_rejects_same_buffer(hs):
    x = synth.spectrum(10000, 1)
    plan = hs.Plan(8, hs.GREEDY, lengths=[len(x)])
    ng = norms(hs, plan, 2)
    out = plan.alloc_form(*ng)
    buf = torch.from_numpy(x).to(DEV)
    with pytest.raises(hs.HSError):
        hs.run_host(plan, buf, buf, None, None, out)


def test_graph_capture_and_replay(hs):
    """hs_run_host records into a CUDA graph (after a first call has created the plan's copy
    streams and events); each replay copies the current contents of the pinned buffer."""
    N, H = (1 << 22) + 11, 32
    plan = hs.Plan(H, hs.SIMPLE | hs.GREEDY, lengths=[N])
    ns, ng = norms(hs, plan, 1), norms(hs, plan, 2)
    out_s, out_g = plan.alloc_form(*ns, path=False), plan.alloc_form(*ng)
    host_s, host_g = plan.alloc_form_host(path=False), plan.alloc_form_host()
    ref_s, ref_g = plan.alloc_form(*ns, path=False), plan.alloc_form(*ng)
    hbuf = torch.zeros(plan.extent, dtype=torch.float32).pin_memory()
    dbuf = torch.zeros(plan.extent, dtype=torch.float32, device=DEV)
    ws = plan.workspace(DEV)
    side = torch.cuda.Stream(DEV)
    with torch.cuda.stream(side):
        hs.run_host(plan, hbuf, dbuf, None, out_s, out_g, host_s, host_g, ws, side)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=side):
        hs.run_host(plan, hbuf, dbuf, None, out_s, out_g, host_s, host_g, ws, side)
    for seed in (3, 4):
        x = synth.spectrum(N, seed, synth.random_pulsars(3, N, seed + 10))
        hbuf[:N] = torch.from_numpy(x)
        g.replay()
        torch.cuda.synchronize()
        hs.run(plan, torch.from_numpy(x).to(DEV), None, ref_s, ref_g)
        torch.cuda.synchronize()
        for ref, out, host in ((ref_s, out_s, host_s), (ref_g, out_g, host_g)):
            for field in ("snr", "best_h", "path", "argmax"):
                r = getattr(ref, field)
                if r is not None:
                    same(r, getattr(out, field), f"replay {seed} {field}")
                    same(r, getattr(host, field), f"replay {seed} {field} (host)")


@pytest.mark.parametrize("H,lengths,dtype,chunks", [(1, [2], 0, 0), (8, [9], 0, 3), (8, [9, 10, 17], 1, 3),
                                                    (32, [40001], 2, 5), (5, [(1 << 21) + 3], 1, 3)])
def test_edge_shapes(hs, H, lengths, dtype, chunks):
    """One fundamental (N = H + 1), H = 1, odd 16-bit lengths, several tiny spectra, more chunks
    asked for than there are tiles."""
    xs = [synth.spectrum(n, 60 + i) for i, n in enumerate(lengths)]
    plan = hs.Plan(H, hs.SIMPLE | hs.GREEDY, lengths=lengths, dtype=dtype)
    plan.host_chunks = chunks
    check(hs, plan, layout(plan, xs, dtype))


def test_partial_host_outputs(hs):
    """Host copies of some fields only (no path, no argmax, SNR only for the simple form)."""
    N, H = (1 << 22) + 1, 16
    x = synth.spectrum(N, 77, synth.random_pulsars(2, N, 78))
    plan = hs.Plan(H, hs.SIMPLE | hs.GREEDY, lengths=[N])
    ns, ng = norms(hs, plan, 1), norms(hs, plan, 2)
    ref_s, ref_g = plan.alloc_form(*ns, path=False), plan.alloc_form(*ng)
    dev = torch.from_numpy(x).to(DEV)
    hs.run(plan, dev, None, ref_s, ref_g)
    out_s, out_g = plan.alloc_form(*ns, path=False), plan.alloc_form(*ng, path=False, argmax=False)
    full_s = plan.alloc_form_host(path=False, argmax=False)
    host_s = hs.FormIO(None, None, full_s.snr, None, None, None)
    host_g = plan.alloc_form_host(path=True, argmax=True)
    hs.run_host(plan, torch.from_numpy(x).pin_memory(), torch.empty_like(dev), None, out_s, out_g, host_s, host_g)
    torch.cuda.synchronize()
    same(ref_s.snr, host_s.snr, "simple snr")
    same(ref_g.snr, host_g.snr, "greedy snr")
    same(ref_g.best_h, host_g.best_h, "greedy best_h")
    same(ref_g.snr, out_g.snr, "greedy snr (device)")
