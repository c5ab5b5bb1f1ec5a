"""The column-sweep 2D kernel (kernel 2 of a 2D plan) against the FP64 oracle, and bit for bit
against the register-resident kernel 1 on the same plane: band widths, CTA sizes, stored types,
planes with gaps between the anchors of two orders, dense ties, graph replay and the fallback
without a workspace."""
import numpy as np
import pytest
import torch

import synth
from test_gpu_2d_bwd import run_2d

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda", 0)


@pytest.mark.parametrize("stage_kb", [0, 1, 2, 4, 8])
@pytest.mark.parametrize("threads", [256, 512])
def test_sweep_band_widths(hs, oracle_lib, stage_kb, threads):
    """H = 8 on 61 rows; band widths 16..128 columns (0 = the default) on an 80000-column plane:
    the sweep starts at f = 64 Wb, so every band width leaves both prefix chains and sweep chains."""
    z0 = 30
    pl = synth.plane(80000, 2 * z0 + 1, z0, 90 + stage_kb, synth.random_tracks(4, 80000, 7, f_lo=50, zmax=3))
    run_2d(hs, oracle_lib, pl, z0, 8, tuning=dict(kernel=2, threads=threads, stage_kb=stage_kb))


@pytest.mark.parametrize("producers", [2, 5])
def test_sweep_longer_prefix(hs, oracle_lib, producers):
    """tuning.producers moves the start of the sweep to f = 64 producers Wb: more chains run whole
    in registers, the sweep's first band starts later; the outputs do not change."""
    z0 = 30
    pl = synth.plane(120000, 2 * z0 + 1, z0, 170 + producers, synth.random_tracks(4, 120000, 23, f_lo=50, zmax=3))
    run_2d(hs, oracle_lib, pl, z0, 8, tuning=dict(kernel=2, threads=512, stage_kb=1, producers=producers))


@pytest.mark.parametrize("H", [1, 2, 3, 5, 6, 7, 8])
def test_sweep_orders(hs, oracle_lib, H):
    z0 = 24
    pl = synth.plane(65536, 2 * z0 + 1, z0, 110 + H, synth.random_tracks(3, 65536, 8, f_lo=50, zmax=2))
    run_2d(hs, oracle_lib, pl, z0, H, tuning=dict(kernel=2, threads=512, stage_kb=2))


@pytest.mark.parametrize("ctas_per_sm", [1, 2])
def test_sweep_persistent_grid(hs, oracle_lib, ctas_per_sm):
    z0 = 40
    pl = synth.plane(1 << 17, 2 * z0 + 1, z0, 131 + ctas_per_sm, synth.random_tracks(5, 1 << 17, 9, f_lo=60, zmax=4))
    run_2d(hs, oracle_lib, pl, z0, 6, tuning=dict(kernel=2, threads=256, stage_kb=2, ctas_per_sm=ctas_per_sm))


@pytest.mark.parametrize("dtype", [1, 2])
@pytest.mark.parametrize("H", [4, 8])
def test_sweep_reduced_precision(hs, oracle_lib, H, dtype):
    z0 = 30
    pl = synth.plane(48000, 2 * z0 + 1, z0, 150 + H, synth.random_tracks(3, 48000, 19, f_lo=50, zmax=3))
    run_2d(hs, oracle_lib, pl, z0, H, dtype=dtype, tuning=dict(kernel=2, threads=512, stage_kb=2))


def test_sweep_gap_between_orders(hs, oracle_lib):
    """f_hi = 1200 with 16-column bands: the sweep covers f in [1024, 1200], so order 1 anchors
    end at 1200 and order 2 anchors start at 2048 -- the bands between hold no event."""
    pl = synth.plane(2404, 9, 4, 5)
    run_2d(hs, oracle_lib, pl, 4, 2, tuning=dict(kernel=2, threads=256, stage_kb=1))


def test_sweep_asymmetric_rows(hs, oracle_lib):
    """z0 off centre: the staged rows start above row 0 and stop below the last row."""
    pl = synth.plane(33000, 201, 150, 12, synth.random_tracks(3, 33000, 21, f_lo=50, zmax=2))
    run_2d(hs, oracle_lib, pl, 150, 6, tuning=dict(kernel=2, threads=512))


def test_sweep_integer_ties(hs, oracle_lib):
    """Small integers: dense ties exercise the strict raster-order rule on staged values."""
    pl = np.floor(synth.plane(36000, 41, 20, 6) * 0.7).astype(np.float32)
    run_2d(hs, oracle_lib, pl, 20, 5, tuning=dict(kernel=2, threads=512, stage_kb=1))
    run_2d(hs, oracle_lib, pl, 20, 5, dtype=2, tuning=dict(kernel=2, threads=256, stage_kb=3))


def _outputs(hs, plan, pl_dev, H, fixed=False):
    mu, sg = hs.norm_exponential(2, 2, H, True, 2.0)
    ng = (torch.from_numpy(mu).to(DEV), torch.from_numpy(sg).to(DEV))
    if fixed:
        g = plan.alloc_form(*ng)
        hs.run_fixed_scratch(plan, pl_dev, None, None, g)
    else:
        g = plan.forward(pl_dev, None, ng)[hs.GREEDY]
    torch.cuda.synchronize()
    hs.check_device_error(plan)
    return [t.cpu() for t in (g.snr, g.best_h, g.path, g.argmax)]


@pytest.mark.parametrize("dtype", [0, 1])
def test_sweep_equals_kernel1(hs, dtype):
    """201 x 2^18 plane, H = 8: kernel 2 gives kernel 1's outputs bit for bit in four launch shapes; the
    plan's default for this plane (211 MB, under 8 L2 sizes) is kernel 1 (the sweep's default launch is
    checked on the full 201 x 2^21 plane in test_gpu_2d_bwd.py)."""
    n_freq = 1 << 18
    tracks = synth.random_tracks(8, n_freq, 333)
    pl = torch.from_numpy(synth.plane(n_freq, 201, 100, 334, tracks))
    if dtype:
        pl = pl.half()
    pl_dev = pl.to(DEV)
    outs = []
    for t in (dict(kernel=1, threads=256), dict(kernel=2, threads=512), dict(kernel=2, threads=256, stage_kb=2),
              dict(kernel=2, threads=1024, producers=4), None):
        plan = hs.Plan(8, hs.GREEDY, dims=2, n_freq=n_freq, n_rows=201, z0_row=100, dtype=dtype)
        if t is not None:
            plan.tuning = t
        else:
            assert plan.tuning.kernel == 1 and plan.tuning.threads == 256
        outs.append(_outputs(hs, plan, pl_dev, 8))
        plan.close()
    for o in outs[1:]:
        for a, b in zip(outs[0], o):
            assert torch.equal(a, b)


def test_sweep_graph_replay_and_fixed_scratch(hs):
    """Graph replay reads the plane's current contents; without a workspace (the fixed-scratch
    entry point) kernel 2 runs as kernel 1 with the same outputs."""
    n_freq, z0, H = 60000, 30, 8
    ref_plan = hs.Plan(H, hs.GREEDY, dims=2, n_freq=n_freq, n_rows=2 * z0 + 1, z0_row=z0)
    ref_plan.tuning = dict(kernel=1, threads=256)
    plan = hs.Plan(H, hs.GREEDY, dims=2, n_freq=n_freq, n_rows=2 * z0 + 1, z0_row=z0, flags=hs.FLAG_GRAPH)
    plan.tuning = dict(kernel=2, threads=512)
    pl_dev = torch.empty((2 * z0 + 1) * n_freq, dtype=torch.float32, device=DEV)
    for seed in (1, 2, 3):
        pl_dev.copy_(torch.from_numpy(synth.plane(n_freq, 2 * z0 + 1, z0, seed, synth.random_tracks(2, n_freq, seed))
                                      .reshape(-1)))
        ref = _outputs(hs, ref_plan, pl_dev, H)
        for a, b in zip(ref, _outputs(hs, plan, pl_dev, H)):
            assert torch.equal(a, b)
    nog = hs.Plan(H, hs.GREEDY, dims=2, n_freq=n_freq, n_rows=2 * z0 + 1, z0_row=z0)
    nog.tuning = dict(kernel=2, threads=512)
    for a, b in zip(ref, _outputs(hs, nog, pl_dev, H, fixed=True)):
        assert torch.equal(a, b)


@pytest.mark.parametrize("stages", [3, 4])
@pytest.mark.parametrize("dtype", [0, 1])
def test_sweep_stages(hs, oracle_lib, stages, dtype):
    """Three or four buffers: the control warp runs up to three bands ahead of the compute warps."""
    z0 = 30
    pl = synth.plane(96000, 2 * z0 + 1, z0, 170 + stages, synth.random_tracks(4, 96000, 23, f_lo=50, zmax=3))
    run_2d(hs, oracle_lib, pl, z0, 8, dtype=dtype, tuning=dict(kernel=2, threads=512, stage_kb=2, stages=stages))


def test_sweep_stops_on_a_recorded_timeout(hs):
    """A timeout already recorded in the plan's error word (as after another CTA's wait ran out):
    a CTA whose next band still waits on a dependency stops instead of reading chain state that
    was never written.  The pass ends, reports HS_ERR_DEVICE_TIMEOUT, and the plan then gives the
    outputs of kernel 1 again."""
    n_freq, z0, H = 1 << 18, 100, 8
    pl_dev = torch.from_numpy(synth.plane(n_freq, 2 * z0 + 1, z0, 335, synth.random_tracks(4, n_freq, 336))).to(DEV)
    ref_plan = hs.Plan(H, hs.GREEDY, dims=2, n_freq=n_freq, n_rows=2 * z0 + 1, z0_row=z0)
    ref_plan.tuning = dict(kernel=1, threads=256)
    ref = _outputs(hs, ref_plan, pl_dev, H)
    plan = hs.Plan(H, hs.GREEDY, dims=2, n_freq=n_freq, n_rows=2 * z0 + 1, z0_row=z0)
    plan.tuning = dict(kernel=2, threads=512)
    mu, sg = hs.norm_exponential(2, 2, H, True, 2.0)
    g = plan.alloc_form(torch.from_numpy(mu).to(DEV), torch.from_numpy(sg).to(DEV))
    hs.selftest_timeout(plan, 1000)          # records the timeout; the pass is queued after it
    hs.run(plan, pl_dev, None, None, g)
    with pytest.raises(hs.HSError) as e:
        hs.check_device_error(plan)
    assert e.value.status == 6               # HS_ERR_DEVICE_TIMEOUT
    for a, b in zip(ref, _outputs(hs, plan, pl_dev, H)):
        assert torch.equal(a, b)
    plan.close()
    ref_plan.close()
