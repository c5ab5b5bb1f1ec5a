#!/usr/bin/env python3
"""Throughput of the GB300 harmonic sum (bins x harmonics / s) against the HBM roofline.

Default workload (one step = one fused simple + greedy pass, one kernel): a single FP32 power
spectrum of 2^23 bins, H = 32, Exponential(1) noise with 16 injected pulsars (f0 ~ U[100, N/32),
duty ~ U[0.02, 0.2)), 262143 fundamentals.  The spectrum (32 MiB) fits in L2, so L2 is flushed
(a write of max(2 x L2, 256 MiB)) before every timed step, and every step is timed alone with
CUDA events on the stream hs_run launches on.

The same line carries a ``workloads`` object with every other configuration, each timed in the
same run with its own roofline, clocks and CPU baseline (``--extras none`` skips them):
  long16              the headline spectrum stored in FP16 (FP32 accumulation)
  batch / batch16     2048 uneven spectra (2^20..2^23 bins), H = 16, 5 % with a pulsar, one
                      launch replayed from a CUDA graph, launch shape autotuned (the line names it);
                      FP32 / FP16 storage (inputs 32 / 16 GB, larger than L2: no flush)
  plane / plane16     2D greedy over an f-fdot plane 201 x 2^21 (z = -100..100), H = 8,
                      chi-square(2) noise + 8 drifting signals (1.69 GB FP32, larger than L2)
  grad                one training step of a learnable per-bin whitening: 256 spectra x 2^20
                      bins, H = 32, greedy forward, loss = -sum of the top-16 SNRs per spectrum
                      (torch.topk), hand-written adjoint to dL/dw
  table2              the paper's throughput configuration (Table 2): 1024 spectra x 131072 bins, H = 32,
                      greedy; also with every bin a fundamental (truncated tail), in Gbin/s
Any of them (and longbf16, the headline spectrum in BF16) can also be the headline of a run of
its own (--workload).

CPU baseline: the FP64 oracle on a bounded sample of the same input, on one thread (the oracle
proper) and on every core of the host (the same source built with OpenMP over fundamentals,
timed in a subprocess); ``cores`` is the thread count of ``value``.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload ...] [--extras all|none]
    python bench.py --impl reference      # the FP64 oracle on the host cores, same metric

N > 1 (torchrun): spectra of a batch (batch, batch16, table2, grad) are independent units, sharded
over ranks longest-first with no data-path collective (per-spectrum argmax keys are gathered once
after the timed steps); the training step all-reduces dL/dw (its one exchange) inside each step.
One spectrum or one plane does not shard: every rank runs a replica.  value = units of all ranks /
max-over-ranks time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "bins×harmonics/s and HBM GB/s (% of peak), greedy vs simple HS at H=32"
UNIT = "bins*harmonics/s"
GOLDEN = os.path.join(ROOT, "tests", "golden", "footprints.json")
PROFILE_TRAFFIC = os.path.join(ROOT, "profiles", "traffic.json")
# sources of the kernel each workload times (the ncu counters under profiles/ hold for them only)
KERNEL_SOURCES = {
    "long": ["hs_fwd1d.cuh", "hs_fwd1d_pair.cuh", "hs_fwd1d_f32.cu", "hs_internal.cuh"],
    "long16": ["hs_fwd1d.cuh", "hs_fwd1d_pair.cuh", "hs_fwd1d_f16.cu", "hs_internal.cuh"],
    "longbf16": ["hs_fwd1d.cuh", "hs_fwd1d_pair.cuh", "hs_fwd1d_bf16.cu", "hs_internal.cuh"],
    "batch": ["hs_fwd1d.cuh", "hs_fwd1d_win.cuh", "hs_fwd1d_pair.cuh", "hs_fwd1d_f32.cu", "hs_internal.cuh"],
    "batch16": ["hs_fwd1d.cuh", "hs_fwd1d_win.cuh", "hs_fwd1d_pair.cuh", "hs_fwd1d_f16.cu", "hs_internal.cuh"],
    "table2": ["hs_fwd1d.cuh", "hs_fwd1d_win.cuh", "hs_fwd1d_pair.cuh", "hs_fwd1d_f32.cu", "hs_internal.cuh"],
    "plane": ["hs_fwd2d.cu", "hs_fwd2d.cuh", "hs_fwd2d_sweep.cu", "hs_fwd2d_sweep.cuh", "hs_fwd1d.cuh",
              "hs_fwd1d_win.cuh", "hs_internal.cuh"],
    "plane16": ["hs_fwd2d.cu", "hs_fwd2d.cuh", "hs_fwd1d.cuh", "hs_internal.cuh"],
    "planebf16": ["hs_fwd2d.cu", "hs_fwd2d.cuh", "hs_fwd1d.cuh", "hs_internal.cuh"],
    "grad": ["hs_bwd1d.cu", "hs_fwd1d.cuh", "hs_fwd1d_f32.cu", "hs_internal.cuh", "hs_prewhiten.cuh"],
}


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def kernel_hash(wl: str) -> str:
    """Hash of the sources of the kernel a workload times."""
    h = hashlib.sha256()
    for f in KERNEL_SOURCES.get(wl, []):
        p = os.path.join(ROOT, "paper_2202_12817_gb300", "csrc", f)
        if os.path.exists(p):
            h.update(open(p, "rb").read())
    return h.hexdigest()[:16]


def load_json(path):
    try:
        return json.load(open(path))
    except Exception:
        return None


NOMINAL_HBM_GBS = 7900.0   # GB300 HBM3e, nominal


def measured_peaks():
    p = load_json(os.path.join(ROOT, "MEASURED_PEAKS.json"))
    if p and "hbm_gbs" in p:
        return float(p["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# ---------------------------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------------------------
# oracle timing (CPU baseline / reference arm): the only place bench.py runs oracle/
# ---------------------------------------------------------------------------------------------
def oracle_rate_1d(x_host, H, budget_s=8.0, frac=1.0, forms=3):
    """Time the FP64 single-thread oracle (simple and/or greedy) on the first ``frac`` of the
    spectrum's fundamentals, repeated until ``budget_s``; returns (units/s, sample text)."""
    import oracle
    oracle.build()
    nf = max(1, int(oracle.nf_1d(x_host.size, H) * frac))
    mu_s, sg_s = oracle.norm_exponential(1, 1, H)
    mu_g, sg_g = oracle.norm_exponential(2, 1, H)
    reps, t0 = 0, time.perf_counter()
    while True:
        if forms & 1:
            oracle.simple_1d(x_host, H, mu_s, sg_s, nf=nf)
        if forms & 2:
            oracle.greedy_1d(x_host, H, mu_g, sg_g, nf=nf)
        reps += 1
        el = time.perf_counter() - t0
        if el >= budget_s:
            break
    what = {1: "simple", 2: "greedy", 3: "simple + greedy"}[forms]
    return reps * nf * H / el, f"{reps} x fundamentals [0, {nf}) of a {x_host.size}-bin spectrum, {what}, 1 thread"


def plane_sample(plane_host, H, f_count=16384):
    """The columns of the plane that the fundamentals f < f_lo + f_count read (every z): a
    bounded CPU-baseline sample of the 2D workload."""
    ncols = min(plane_host.shape[1], H * (1 + f_count) + H + 1)
    return np.ascontiguousarray(plane_host[:, :ncols])


def oracle_rate_2d(plane_host, z0_row, H, budget_s=8.0):
    """Time the single-thread oracle over every fundamental of `plane_host` (a column slice)."""
    import oracle
    oracle.build()
    f_lo, f_hi, z_lo, z_hi = oracle.domain_2d(plane_host.shape[1], plane_host.shape[0], z0_row, H)
    dom = (f_lo, f_hi, z_lo, z_hi)
    mu, sg = oracle.norm_exponential(2, 2, H, mean1=2.0)
    reps, t0 = 0, time.perf_counter()
    while True:
        oracle.greedy_2d(plane_host, z0_row, H, mu, sg, dom=dom)
        reps += 1
        el = time.perf_counter() - t0
        if el >= budget_s:
            break
    units = reps * (f_hi - f_lo + 1) * (z_hi - z_lo + 1) * H
    return units / el, (f"{reps} x every (f, z) fundamental of a {plane_host.shape[0]} x {plane_host.shape[1]} "
                        "plane, 1 thread")


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def oracle_rate_all_cores(spec, budget_s):
    """The oracle built with OpenMP over fundamentals, on every core of the host, in a subprocess
    (its OpenMP runtime stays out of this process); None when that build is unavailable."""
    import tempfile
    threads = host_cores()
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "input.npy")
        np.save(path, spec["x"])
        cmd = [sys.executable, "-m", "oracle.timing", "--input", path, "--dims", str(spec["dims"]),
               "--H", str(spec["H"]), "--threads", str(threads), "--budget", str(budget_s)]
        if spec["dims"] == 1:
            cmd += ["--forms", str(spec.get("forms", 3)), "--frac", str(spec.get("frac", 1.0))]
        else:
            cmd += ["--z0", str(spec["z0"])]
        try:
            r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=120 + 4 * budget_s)
            return json.loads(r.stdout.strip().splitlines()[-1])
        except Exception as e:
            log("all-core oracle timing failed:", e)
            return None


def cpu_baseline(spec, budget_one, budget_all):
    """cpu_baseline object: value = the oracle on every host core (cores = its threads), with the
    single-thread oracle beside it."""
    if spec["dims"] == 1:
        v1, s1 = oracle_rate_1d(spec["x"], spec["H"], budget_s=budget_one, frac=spec.get("frac", 1.0),
                                forms=spec.get("forms", 3))
    else:
        v1, s1 = oracle_rate_2d(spec["x"], spec["z0"], spec["H"], budget_s=budget_one)
    one = {"value": v1, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": s1}
    allc = oracle_rate_all_cores(spec, budget_all)
    if not allc or allc.get("threads", 1) <= 1:
        out = dict(one)
        out["cpu_model"] = allc.get("cpu") if allc else None
        out["all_cores"] = None
        return out
    return {"value": allc["rate"], "unit": UNIT, "cores": int(allc["threads"]), "kind": "oracle",
            "sample": allc["sample"] + " (the oracle's source built with OpenMP over fundamentals)",
            "cpu_model": allc.get("cpu"), "single_thread": one}


# ---------------------------------------------------------------------------------------------
# distributed plumbing
# ---------------------------------------------------------------------------------------------
def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", str(rank)))
    return rank, world, local


def init_dist(world, backend):
    import torch.distributed as dist
    if world > 1 and not dist.is_initialized():
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group(backend)
    return dist if world > 1 else None


def max_over_ranks(v, dist, device):
    if dist is None:
        return v
    from paper_2202_12817_gb300 import dist as hsd
    return hsd.max_over_ranks(v, device)


# ---------------------------------------------------------------------------------------------
# compulsory bytes
# ---------------------------------------------------------------------------------------------
def out_bytes_1d(nf, H, forms):
    pb = 4 if H > 16 else (2 if H > 8 else 1)
    b = 0
    if forms & 1:
        b += nf * 5
    if forms & 2:
        b += nf * (5 + pb)
    return b


def long_alg_bytes(H, forms, elem, nf):
    """Compulsory bytes of one pass over the benchmark spectrum: its distinct 32-B sectors that
    the forms read (oracle-counted, tests/golden/footprints.json) + outputs + mu/sigma."""
    gold = (load_json(GOLDEN) or {}).get("long", {})
    fp = gold.get({1: "simple", 2: "greedy", 3: "fused"}[forms])
    if fp is not None:
        in_bytes, how = int(fp["sectors" if elem == 4 else "sectors_16bit"]) * 32, "oracle sector footprint"
    else:
        in_bytes, how = synth.LONG_N * elem, "whole input"
    return in_bytes + out_bytes_1d(nf, H, forms) + 2 * 4 * H * (2 if forms == 3 else 1), how


def batch_alg_bytes(lengths, H, elem, nf):
    gold = (load_json(GOLDEN) or {}).get("batch_H16_fraction", {})
    key = "fused" if elem == 4 else "fused_16bit"
    tot, how = 0.0, "oracle sector footprint per length"
    for n in lengths:
        fr = gold.get(str(int(n)), {}).get(key)
        if fr is None:
            fr, how = 1.0, "whole input"
        tot += fr * n * elem
    return int(tot) + out_bytes_1d(nf, H, 3) + 4 * 4 * H, how


# ---------------------------------------------------------------------------------------------
# timing helper
# ---------------------------------------------------------------------------------------------
def time_steps(torch, step, K, stream, flush=None):
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    for i in range(K):
        if flush is not None:
            flush.fill_(float(i & 7))
        ev[i][0].record(stream)
        step()
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in ev]


def traffic_entry(wl, tuning):
    """The committed ncu capture of this workload's timed kernel (profiles/traffic.json holds one or
    more per workload, one per captured launch shape) whose sources and launch shape are the ones
    that ran; None when there is none."""
    ents = (load_json(PROFILE_TRAFFIC) or {}).get(wl) or []
    if isinstance(ents, dict):
        ents = [ents]
    h = kernel_hash(wl)
    for e in ents:
        if e.get("kernel_hash") == h and e.get("tuning") == tuning:
            return e
    return None


def roofline(alg_bytes, ms, peak, peak_kind, wl, how, tuning=None):
    """roofline entry; `traffic` = DRAM bytes per launch from the committed ncu capture of this
    workload, reported only while the kernel's sources and launch shape are those captured."""
    achieved = alg_bytes / (ms / 1e3) / 1e9
    pk = traffic_entry(wl, tuning) or {}
    fresh = bool(pk)
    return {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
            "frac": round(achieved / peak, 4), "traffic": pk.get("dram_bytes_per_launch") if fresh else None,
            "algorithmic_bytes": int(alg_bytes), "bytes_basis": how, "peak_kind": peak_kind,
            "peak_nominal": NOMINAL_HBM_GBS, "frac_nominal": round(achieved / NOMINAL_HBM_GBS, 4),
            "kernel": pk.get("kernel") if fresh else None}


def plane_launch_text(t):
    """What one 2D step launches, from the plan's launch shape."""
    if t.get("kernel") == 2:
        return ("column sweep (kernel 2): one persistent CTA of %d threads per SM takes bands of anchor columns, "
                "each staged once for all orders; chains f < %d band widths run whole in registers first"
                % (t.get("threads", 0), 64 * max(1, t.get("producers", 0))))
    return "one thread per (f, z) chain (kernel %d), CTAs over %s fastest" % (
        t.get("kernel", 0), "z rows" if t.get("kernel") == 1 else "f tiles")


def launch_text(t):
    """What one step launches, from the plan's (autotuned) launch shape."""
    if t.get("ctas_per_sm", 0) > 0:
        sched = "a persistent grid of %d CTAs per SM, %s" % (
            t["ctas_per_sm"], "tiles from an atomic counter" if t.get("dynamic") else "tiles strided over the grid")
    else:
        sched = "one CTA per tile"
    return "one launch of kernel %d (%s) replayed from a CUDA graph" % (t.get("kernel", 0), sched)


# ---------------------------------------------------------------------------------------------
# workloads: each returns (result dict without clocks, clock summary, cpu-baseline function)
# ---------------------------------------------------------------------------------------------
def wl_long(args, hs, torch, dev, world, dist):
    wl = args.workload
    H = 32
    dtype = {"long": hs.F32, "long16": hs.F16, "longbf16": hs.BF16}[wl]
    elem = 4 if dtype == hs.F32 else 2
    x32 = synth.device_spectrum(synth.LONG_N, synth.SEED_BASE + 2, synth.long_spectrum_pulsars(), dev)
    x = x32 if dtype == hs.F32 else x32.to(torch.float16 if dtype == hs.F16 else torch.bfloat16)
    plan = hs.Plan(H, hs.SIMPLE | hs.GREEDY, lengths=[synth.LONG_N], dtype=dtype, device=dev.index)
    if args.tuning:
        plan.tuning = json.loads(args.tuning)
    nf = plan.total_fundamentals
    ns = [torch.from_numpy(a).to(dev) for a in hs.norm_exponential(hs.SIMPLE, 1, H)]
    ng = [torch.from_numpy(a).to(dev) for a in hs.norm_exponential(hs.GREEDY, 1, H)]
    s_io = plan.alloc_form(*ns, path=False, argmax=True)
    g_io = plan.alloc_form(*ng, path=True, argmax=True)
    ws = plan.workspace(dev)
    stream = torch.cuda.current_stream(dev)
    l2 = torch.cuda.get_device_properties(dev).L2_cache_size
    flush = torch.empty(max(2 * l2, 256 << 20) // 4, dtype=torch.float32, device=dev)

    def step():
        hs.run(plan, x, None, s_io, g_io, ws, stream)

    for _ in range(args.warmup):
        flush.fill_(1.0)
        step()
    torch.cuda.synchronize(dev)
    if dist:
        dist.barrier()
    torch.cuda.synchronize(dev)
    with ClockSampler(dev.index) as clk:
        t0 = time.perf_counter()
        times = time_steps(torch, step, args.steps, stream, flush)
        wall = time.perf_counter() - t0
    if dist:
        dist.barrier()
    ms = sum(times) / len(times)
    ms_max = max_over_ranks(ms, dist, dev)
    units = nf * H
    peak, peak_kind = measured_peaks()
    alg, how = long_alg_bytes(H, 3, elem, nf)

    # each form alone (separate plans, same input), reported beside the fused pass
    per_form = {}
    for form, name in ((hs.SIMPLE, "simple"), (hs.GREEDY, "greedy")):
        p2 = hs.Plan(H, form, lengths=[synth.LONG_N], dtype=dtype, device=dev.index)
        if args.tuning:
            p2.tuning = json.loads(args.tuning)
        io = p2.alloc_form(*(ns if form == hs.SIMPLE else ng), path=form == hs.GREEDY, argmax=True)
        ws2 = p2.workspace(dev)

        def st2():
            hs.run(p2, x, None, io if form == 1 else None, io if form == 2 else None, ws2, stream)

        for _ in range(3):
            flush.fill_(1.0)
            st2()
        ft = time_steps(torch, st2, min(args.steps, 300), stream, flush)
        fms = sum(ft) / len(ft)
        fb, _ = long_alg_bytes(H, form, elem, nf)
        per_form[name] = {"value": units / (fms / 1e3), "ms": round(fms, 5),
                          "hbm_gbs": round(fb / (fms / 1e3) / 1e9, 1), "frac": round(fb / (fms / 1e3) / 1e9 / peak, 4),
                          "tuning": p2.tuning.as_dict()}
        p2.close()

    # the optimal form (dynamic programme over drift paths) on the same input, for reference
    po = hs.Plan(H, hs.OPTIMAL, lengths=[synth.LONG_N], dtype=dtype, device=dev.index)
    no = [torch.from_numpy(a).to(dev) for a in (np.linspace(1.6, 1.6 * H, H).astype(np.float32),
                                                np.sqrt(np.linspace(1.3, 1.3 * H, H)).astype(np.float32))]
    io_o = po.alloc_form(*no, path=True, argmax=True)

    def st_opt():
        hs.run_optimal(po, x, None, io_o, stream)

    for _ in range(3):
        flush.fill_(1.0)
        st_opt()
    ot = time_steps(torch, st_opt, min(args.steps, 100), stream, flush)
    oms = sum(ot) / len(ot)
    per_form["optimal"] = {"value": units / (oms / 1e3), "ms": round(oms, 5),
                           "note": "DP optimum over monotone drift paths, one warp per fundamental"}
    po.close()

    # the fused pass with the input left in L2 between steps (labelled context, not the headline)
    for _ in range(3):
        step()
    wt = time_steps(torch, step, min(args.steps, 300), stream)
    w_ms = sum(wt) / len(wt)

    # end to end through the C ABI with host buffers: hs_run_host copies the pinned spectrum in
    # chunks and runs each chunk's fundamentals once their bins have arrived, and copies every
    # output back to pinned host memory, all inside the timed region
    xh = x.cpu().pin_memory()
    host_s, host_g = plan.alloc_form_host(path=False), plan.alloc_form_host()
    outs_h = [t for t in (host_s.snr, host_s.best_h, host_s.argmax, host_g.snr, host_g.best_h, host_g.path,
                          host_g.argmax)]
    xd2 = torch.empty_like(x)

    def e2e_step():
        hs.run_host(plan, xh, xd2, None, s_io, g_io, host_s, host_g, ws, stream)

    # the same with one copy before the pass and the outputs copied after it (context)
    dev_outs = (s_io.snr, s_io.best_h, s_io.argmax, g_io.snr, g_io.best_h, g_io.path, g_io.argmax)

    def serial_step():
        xd2.copy_(xh, non_blocking=True)
        hs.run(plan, xd2, None, s_io, g_io, ws, stream)
        for hbuf, dbuf in zip(outs_h, dev_outs):
            hbuf.copy_(dbuf, non_blocking=True)

    for _ in range(2):
        e2e_step()
        serial_step()
    et = time_steps(torch, e2e_step, max(3, min(args.steps, 30)), stream)
    e_ms = max_over_ranks(sum(et) / len(et), dist, dev)
    st_ = time_steps(torch, serial_step, max(3, min(args.steps, 30)), stream)
    s_ms = sum(st_) / len(st_)

    result = {
        "metric": METRIC, "value": world * units / (ms_max / 1e3), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": {hs.F32: "f32", hs.F16: "f16 storage, f32 accumulate", hs.BF16: "bf16 storage, f32 accumulate"}[dtype],
        "data": "synthetic",
        "config": {"workload": "single spectrum of 2^23 bins (%s), H=32, 16 pulsars, simple+greedy fused"
                               % {hs.F32: "FP32", hs.F16: "FP16", hs.BF16: "BF16"}[dtype],
                   "bins": synth.LONG_N, "H": H, "fundamentals": int(nf),
                   "parallelism": "replicas" if world > 1 else "1 GPU",
                   "l2": "flushed before every timed step (write of max(2 x L2, 256 MiB))",
                   "tuning": plan.tuning.as_dict()},
        "roofline": roofline(alg, ms, peak, peak_kind, wl, how, plan.tuning.as_dict()),
        "per_form": per_form,
        "warm_l2": {"value": world * units / (w_ms / 1e3), "unit": UNIT, "ms": round(w_ms, 5),
                    "note": "input left in L2 between steps (no flush): context, not the headline"},
        "e2e": {"value": world * units / (e_ms / 1e3), "unit": UNIT,
                "h2d_bytes_per_step": int(x.numel() * x.element_size()),
                "d2h_bytes_per_step": int(sum(t.numel() * t.element_size() for t in outs_h)),
                "ms": round(e_ms, 5), "api": "hs_run_host (chunked copies overlapped with the pass)",
                "copy_then_run": {"value": world * units / (s_ms / 1e3), "ms": round(s_ms, 5)}},
        # per step: k_fwd_reset (argmax keys) + the fused pass
        "gpu_launches": 2 * args.steps, "wall_s_timed_region": round(wall, 3),
    }
    return result, clk.summary(), {"dims": 1, "x": x.float().cpu().numpy(), "H": H, "forms": 3}


def wl_batch(args, hs, torch, dev, world, dist):
    from paper_2202_12817_gb300 import dist as hsd
    H = 16
    dtype = hs.F16 if args.workload == "batch16" else hs.F32
    elem = 4 if dtype == hs.F32 else 2
    b = synth.uneven_batch(count=args.batch_spectra)
    B = len(b.lengths)
    rank = dist.get_rank() if dist else 0
    # N > 1: this rank's spectra (longest-processing-time shards), drawn and packed on its GPU
    mine = hsd.shard_for_rank(b.lengths, world, rank) if world > 1 else list(range(B))
    lb = synth.sub_batch(b, mine) if world > 1 else b
    x = synth.device_batch(lb, dev, dtype=torch.float16 if dtype == hs.F16 else None)
    plan = hs.Plan(H, hs.SIMPLE | hs.GREEDY, lengths=lb.lengths, dtype=dtype, offsets=lb.offsets[:-1],
                   flags=hs.FLAG_GRAPH | (0 if args.tuning else hs.FLAG_AUTOTUNE), device=dev.index)
    if args.tuning:
        plan.tuning = json.loads(args.tuning)
    nf = plan.total_fundamentals
    nf_all = int(sum((int(n) - 1) // H for n in b.lengths))
    ns = [torch.from_numpy(a).to(dev) for a in hs.norm_exponential(hs.SIMPLE, 1, H)]
    ng = [torch.from_numpy(a).to(dev) for a in hs.norm_exponential(hs.GREEDY, 1, H)]
    s_io = plan.alloc_form(*ns, path=False, argmax=True)
    g_io = plan.alloc_form(*ng, path=True, argmax=True)
    ws = plan.workspace(dev)
    stream = torch.cuda.current_stream(dev)

    def compute(idx):
        hs.run(plan, x, None, s_io, g_io, ws, stream)
        return g_io.argmax.view(torch.int64)

    def step():
        hsd.batch_step(mine, B, compute, gather=False)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)
    if dist:
        dist.barrier()
    steps = min(args.steps, 40)
    with ClockSampler(dev.index) as clk:
        t0 = time.perf_counter()
        times = time_steps(torch, step, steps, stream)
        wall = time.perf_counter() - t0
    ms = sum(times) / len(times)
    ms_max = max_over_ranks(ms, dist, dev)
    gathered = None
    if world > 1:
        # the per-spectrum argmax keys of every rank, in global spectrum order (after the timed steps)
        gathered = int(hsd.batch_step(mine, B, compute).shape[0])
    peak, peak_kind = measured_peaks()
    alg, how = batch_alg_bytes(lb.lengths, H, elem, nf)
    tun = plan.tuning.as_dict()
    result = {
        "metric": METRIC, "value": nf_all * H / (ms_max / 1e3), "unit": UNIT, "n_gpus": world,
        "steps": steps, "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True,
        "scaling": "weak" if world == 1 else "strong",
        "vs_baseline": None, "dtype": "f32" if dtype == hs.F32 else "f16 storage, f32 accumulate",
        "data": "synthetic",
        "config": {"workload": f"{B} uneven spectra (2^20..2^23 bins, {'FP32' if dtype == hs.F32 else 'FP16'}), "
                               f"H=16, 5% with a pulsar, {launch_text(tun)}",
                   "bins": int(sum(b.lengths)), "H": H, "fundamentals": nf_all, "spectra": B,
                   "parallelism": f"LPT shards over {world} ranks ({len(mine)} spectra on rank 0)" if world > 1
                   else "1 GPU", "gathered_argmax_spectra": gathered,
                   "l2": "inputs larger than L2 (no flush)", "tuning": tun},
        "roofline": roofline(alg, ms, peak, peak_kind, args.workload, how, tun),
        # per step: k_fwd_reset + the pass, replayed from one graph
        "gpu_launches": 2 * steps, "wall_s_timed_region": round(wall, 3),
    }
    i0 = int(np.argmax(lb.lengths))
    off = int(lb.offsets[i0])
    xs_host = x[off:off + int(lb.lengths[i0])].float().cpu().numpy()
    return result, clk.summary(), {"dims": 1, "x": xs_host, "H": H, "forms": 3}


def wl_plane(args, hs, torch, dev, world, dist):
    H = 8
    wl = args.workload
    dtype = {"plane": hs.F32, "plane16": hs.F16, "planebf16": hs.BF16}[wl]
    elem = 4 if dtype == hs.F32 else 2
    tracks = synth.random_tracks(8, synth.PLANE_N_FREQ, synth.SEED_BASE + 4 + 1000)
    pl = synth.device_plane(synth.PLANE_N_FREQ, synth.PLANE_N_ROWS, synth.PLANE_Z0_ROW, synth.SEED_BASE + 4,
                            tracks, dev)
    if dtype != hs.F32:
        pl = pl.to(torch.float16 if dtype == hs.F16 else torch.bfloat16)
    plan = hs.Plan(H, hs.GREEDY, dims=2, n_freq=synth.PLANE_N_FREQ, n_rows=synth.PLANE_N_ROWS,
                   z0_row=synth.PLANE_Z0_ROW, dtype=dtype, device=dev.index)
    if args.tuning:
        plan.tuning = json.loads(args.tuning)
    nfund = plan.total_fundamentals
    ng = [torch.from_numpy(a).to(dev) for a in hs.norm_exponential(hs.GREEDY, 2, H, True, 2.0)]
    g_io = plan.alloc_form(*ng, path=True, argmax=True)
    stream = torch.cuda.current_stream(dev)

    def step():
        hs.run(plan, pl, None, None, g_io, None, stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)
    if dist:
        dist.barrier()
    steps = min(args.steps, 200)
    with ClockSampler(dev.index) as clk:
        t0 = time.perf_counter()
        times = time_steps(torch, step, steps, stream)
        wall = time.perf_counter() - t0
    ms = sum(times) / len(times)
    ms_max = max_over_ranks(ms, dist, dev)
    peak, peak_kind = measured_peaks()
    gold = (load_json(GOLDEN) or {}).get("plane", {})
    if "sectors" in gold:
        # the FP32 footprint; a 16-bit plane touches the same bins in half the bytes
        alg = int(gold["sectors"]) * 32 * elem // 4
        how = "oracle sector footprint" + ("" if elem == 4 else " of the FP32 plane x 1/2")
    else:
        alg, how = synth.PLANE_N_FREQ * synth.PLANE_N_ROWS * elem, "whole input"
    alg += nfund * (4 + 1 + 4) + 2 * 4 * H
    result = {
        "metric": METRIC, "value": world * nfund * H / (ms_max / 1e3), "unit": UNIT, "n_gpus": world,
        "steps": steps, "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": {hs.F32: "f32", hs.F16: "f16 storage, f32 accumulate", hs.BF16: "bf16 storage, f32 accumulate"}[dtype],
        "data": "synthetic",
        "config": {"workload": "2D greedy over an f-fdot plane 201 x 2^21 (%s), H=8, 8 drifting signals"
                               % {hs.F32: "FP32", hs.F16: "FP16", hs.BF16: "BF16"}[dtype],
                   "fundamentals": int(nfund), "H": H, "domain": list(plan.domain), "tuning": plan.tuning.as_dict(),
                   "launch": plane_launch_text(plan.tuning.as_dict()), "l2": "input larger than L2 (no flush)"},
        "roofline": roofline(alg, ms, peak, peak_kind, wl, how, plan.tuning.as_dict()),
        "gpu_launches": steps, "wall_s_timed_region": round(wall, 3),
    }
    return result, clk.summary(), {"dims": 2, "x": plane_sample(pl.float().cpu().numpy(), H), "H": H,
                                   "z0": synth.PLANE_Z0_ROW}


def wl_grad(args, hs, torch, dev, world, dist):
    from paper_2202_12817_gb300 import dist as hsd
    B_all, N, H, K = 256, 1 << 20, 32, 16
    rank = dist.get_rank() if dist else 0
    mine = hsd.shard_for_rank([N] * B_all, world, rank) if world > 1 else list(range(B_all))
    B = len(mine)
    p = torch.empty(B * N, dtype=torch.float32, device=dev)
    for k, i in enumerate(mine):
        view = p[k * N:(k + 1) * N]
        synth.device_noise(N, synth.SEED_BASE + 5 + 7 * i, dev, out=view)
        synth.device_inject(view, [synth.random_pulsars(1, N, synth.SEED_BASE + 5000 + i)[0]])
    w = torch.ones(N, dtype=torch.float32, device=dev, requires_grad=True)
    plan = hs.Plan(H, hs.GREEDY, lengths=[N] * B, flags=hs.FLAG_WHITENING, device=dev.index)
    if args.tuning:
        plan.tuning = json.loads(args.tuning)
    mu, sg = [torch.from_numpy(a).to(dev) for a in hs.norm_exponential(hs.GREEDY, 1, H)]
    nf = plan.total_fundamentals // B
    stream = torch.cuda.current_stream(dev)
    fwd_t, bwd_t = [], []

    def compute():
        snr, bh, path = hs.HarmonicSum.apply(p, w, plan, hs.GREEDY, mu, sg)
        loss = -snr.view(B, nf).topk(K, dim=1).values.sum()
        return loss

    def step(timed=False):
        w.grad = None
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record(stream)
        loss = compute()
        e1.record(stream)

        def local_grad():
            loss.backward()
            return w.grad

        # N > 1: the step's one exchange, the sum of dL/dw over ranks
        if world > 1:
            hsd.grad_step(local_grad)
        else:
            local_grad()
        e2.record(stream)
        if timed:
            fwd_t.append((e0, e1))
            bwd_t.append((e1, e2))

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)
    if dist:
        dist.barrier()
    steps = min(args.steps, 100)
    with ClockSampler(dev.index) as clk:
        t0 = time.perf_counter()
        for _ in range(steps):
            step(True)
        torch.cuda.synchronize(dev)
        wall = time.perf_counter() - t0
    f_ms = sum(a.elapsed_time(b) for a, b in fwd_t) / steps
    b_ms = sum(a.elapsed_time(b) for a, b in bwd_t) / steps
    ms = f_ms + b_ms
    ms_max = max_over_ranks(ms, dist, dev)
    units = B_all * nf * H
    peak, peak_kind = measured_peaks()
    frac = (load_json(GOLDEN) or {}).get("grad_H32_fraction", {}).get(str(N), {}).get("fused", 1.0)
    fwd_bytes = B * N * 4 * frac + N * 4 + B * nf * (4 + 1 + 4)
    bwd_bytes = B * N * 4 + B * nf * (4 + 1 + 4) + N * 4
    result = {
        "metric": METRIC, "value": units / (ms_max / 1e3), "unit": UNIT, "n_gpus": world,
        "steps": steps, "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True,
        "scaling": "weak" if world == 1 else "strong", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "training step: 256 spectra x 2^20 bins, H=32, learnable whitening, greedy "
                               "forward + top-16 loss (torch.topk) + adjoint to dL/dw", "H": H, "spectra": B_all,
                   "parallelism": f"LPT shards over {world} ranks + all-reduce of dL/dw" if world > 1 else "1 GPU",
                   "fwd_ms": round(f_ms, 4), "bwd_ms": round(b_ms, 4), "l2": "inputs larger than L2 (no flush)",
                   "tuning": plan.tuning.as_dict()},
        "roofline": roofline(fwd_bytes + bwd_bytes, ms, peak, peak_kind, "grad",
                             "fwd: oracle sector fraction x input + w + outputs; bwd: input + forward outputs + dL/dw",
                             plan.tuning.as_dict()),
        # per step: the whitened copy, the forward pass, the adjoint's marking pass, the adjoint and
        # (spectra summed in more than one group) the reduction of the partial dL/dw
        "gpu_launches": (4 + (1 if B > 1 else 0)) * steps, "wall_s_timed_region": round(wall, 3),
    }
    return result, clk.summary(), {"dims": 1, "x": p[:N].detach().cpu().numpy(), "H": H, "forms": 2}


def wl_table2(args, hs, torch, dev, world, dist):
    """The paper's own throughput configuration (Table 2): 1024 FP32 power spectra of 131072 bins,
    H = 32, greedy form; Exp(1) noise, one pulsar in every spectrum.  Timed twice: over the fundamentals
    with all H orders, and with the truncated tail (every bin but the last a fundamental, the paper's
    loop over all bins), whose fundamentals per second are the paper's "Gbin/s" under that reading.
    N > 1: the spectra are sharded over the ranks."""
    from paper_2202_12817_gb300 import dist as hsd
    B_all, N, H = 1024, 1 << 17, 32
    rank = dist.get_rank() if dist else 0
    mine = hsd.shard_for_rank([N] * B_all, world, rank) if world > 1 else list(range(B_all))
    B = len(mine)
    b = synth.Batch(np.full(B, N, np.int64), synth.pack_offsets(np.full(B, N, np.int64), 32), {}, synth.SEED_BASE + 6)
    x = torch.zeros(b.total, dtype=torch.float32, device=dev)
    for k, i in enumerate(mine):
        view = x[int(b.offsets[k]):int(b.offsets[k]) + N]
        synth.device_noise(N, synth.SEED_BASE + 6 + 13 * i, dev, out=view)
        synth.device_inject(view, [synth.random_pulsars(1, N, synth.SEED_BASE + 6000 + i)[0]])
    mu, sg = [torch.from_numpy(a).to(dev) for a in hs.norm_exponential(hs.GREEDY, 1, H)]
    stream = torch.cuda.current_stream(dev)
    out = {}
    clk_all = None
    for name, flags in (("main", 0), ("all_bins", hs.FLAG_TRUNCATE_TAIL)):
        plan = hs.Plan(H, hs.GREEDY, lengths=b.lengths, offsets=b.offsets[:-1],
                       flags=flags | (0 if args.tuning else hs.FLAG_AUTOTUNE), device=dev.index)
        if args.tuning:
            plan.tuning = json.loads(args.tuning)
        io = plan.alloc_form(mu, sg, path=True, argmax=True)
        ws = None if not plan.workspace_bytes else plan.workspace(dev)

        def compute(idx):
            hs.run(plan, x, None, None, io, ws, stream)
            return io.argmax.view(torch.int64)

        def step():
            hsd.batch_step(mine, B_all, compute, gather=False)

        for _ in range(args.warmup):
            step()
        torch.cuda.synchronize(dev)
        if dist:
            dist.barrier()
        steps = min(args.steps, 100)
        with ClockSampler(dev.index) as clk:
            times = time_steps(torch, step, steps, stream)
        clk_all = clk.summary() if clk_all is None else clk_all
        ms_local = sum(times) / len(times)
        ms = max_over_ranks(ms_local, dist, dev)
        # fundamentals of all ranks: every spectrum has the same count
        out[name] = {"ms": ms, "ms_local": ms_local, "fundamentals": plan.total_fundamentals // B * B_all,
                     "tuning": plan.tuning.as_dict()}
        plan.close()
    m, a = out["main"], out["all_bins"]
    units = m["fundamentals"] * H
    peak, peak_kind = measured_peaks()
    alg = B * N * 4 + m["fundamentals"] // B_all * B * (4 + 1 + 4) + 2 * 4 * H
    result = {
        "metric": METRIC, "value": units / (m["ms"] / 1e3), "unit": UNIT, "n_gpus": world,
        "steps": min(args.steps, 100), "warmup": args.warmup, "ms_per_step": m["ms"], "higher_is_better": True,
        "scaling": "weak" if world == 1 else "strong", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "the paper's Table 2 configuration: 1024 spectra x 131072 bins (FP32), H=32, greedy",
                   "spectra": B_all, "bins": N, "H": H, "l2": "input (512 MiB) larger than L2 (no flush)",
                   "parallelism": f"LPT shards over {world} ranks" if world > 1 else "1 GPU",
                   "gbin_per_s_full_harmonic_fundamentals": m["fundamentals"] / (m["ms"] / 1e3) / 1e9,
                   "gbin_per_s_every_bin_truncated_tail": a["fundamentals"] / (a["ms"] / 1e3) / 1e9,
                   "ms_every_bin_truncated_tail": a["ms"],
                   "paper_v100_greedy_gbin_per_s": 8.64,
                   "tuning": m["tuning"], "tuning_every_bin": a["tuning"]},
        "roofline": roofline(alg, m["ms_local"], peak, peak_kind, "table2", "whole input + outputs", m["tuning"]),
        # per step: k_fwd_reset + the pass
        "gpu_launches": 2 * min(args.steps, 100),
    }
    return result, clk_all, {"dims": 1, "x": x[:N].cpu().numpy(), "H": H, "forms": 2}


WORKLOADS = {"long": wl_long, "long16": wl_long, "longbf16": wl_long, "batch": wl_batch, "batch16": wl_batch,
             "plane": wl_plane, "plane16": wl_plane, "planebf16": wl_plane, "grad": wl_grad, "table2": wl_table2}


EXTRAS = ("long16", "batch", "batch16", "plane", "plane16", "grad", "table2")


def reference_arm(args, rank, world):
    """The FP64 oracle on the host cores (all of them where the OpenMP build of the oracle exists,
    else one thread); each step runs the whole headline workload (one thread: 1/32 of its
    fundamentals).  Under torchrun rank 0 alone runs it."""
    if rank != 0:
        return
    import oracle
    H = 32
    x = synth.long_spectrum()
    threads = host_cores()
    if threads > 1:
        os.environ["OMP_NUM_THREADS"] = str(threads)
    omp = oracle.use_openmp(threads > 1)
    threads = threads if omp else 1
    nf = oracle.nf_1d(x.size, H)
    frac = 1.0 if omp else 1.0 / 32
    for _ in range(args.warmup):
        oracle_rate_1d(x, H, budget_s=0.0, frac=frac / 4)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle_rate_1d(x, H, budget_s=0.0, frac=frac)
    el = time.perf_counter() - t0
    v = args.steps * int(nf * frac) * H / el
    from oracle.timing import cpu_model
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "single spectrum of 2^23 bins (FP32), H=32, 16 pulsars, simple+greedy fused",
                   "H": H},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle", "cpu_model": cpu_model(),
                         "sample": f"each step: fundamentals [0, {int(nf * frac)}) of the 2^23-bin spectrum, "
                                   f"simple + greedy, FP64, {threads} thread(s)"
                                   + (" (the oracle's source built with OpenMP over fundamentals)" if omp else "")},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="long", choices=sorted(WORKLOADS))
    ap.add_argument("--extras", default="all", choices=["all", "none"],
                    help="with the headline workload, also time every other configuration (the line's "
                         "'workloads' object)")
    ap.add_argument("--tuning", default=None, help="JSON hs_tuning override")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--batch-spectra", type=int, default=2048,
                    help="spectra of the batch workloads (2048 = the benchmark; fewer only for profiling)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    rank, world, local = dist_env()

    if args.impl == "reference":
        reference_arm(args, rank, world)
        return

    import copy

    import torch
    import paper_2202_12817_gb300 as hs
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    dist = init_dist(world, "nccl")
    result, clocks, cpu_spec = WORKLOADS[args.workload](args, hs, torch, dev, world, dist)
    result["clocks"] = clocks
    want_cpu = rank == 0 and world == 1 and not args.no_cpu_baseline
    result["cpu_baseline"] = cpu_baseline(cpu_spec, 8.0, 5.0) if want_cpu else None
    del cpu_spec
    torch.cuda.empty_cache()
    if args.workload == "long" and args.extras == "all" and not args.tuning:
        extras = {}
        for name in EXTRAS:
            sub = copy.copy(args)
            sub.workload = name
            r, clk, spec = WORKLOADS[name](sub, hs, torch, dev, world, dist)
            entry = {k: r[k] for k in ("value", "unit", "ms_per_step", "steps", "warmup", "scaling", "dtype", "config",
                                       "roofline", "gpu_launches")}
            entry["clocks"] = clk
            entry["cpu_baseline"] = cpu_baseline(spec, 3.0, 3.0) if want_cpu else None
            extras[name] = entry
            del r, spec
            torch.cuda.synchronize(dev)
            torch.cuda.empty_cache()
        result["workloads"] = extras
    if rank == 0:
        print(json.dumps(result))
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
