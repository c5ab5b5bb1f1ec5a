#!/usr/bin/env python3
"""Throughput of the GB300 harmonic sum (bins x harmonics / s) against the HBM roofline.

Default workload (one step = one fused simple + greedy pass): a single FP32 power spectrum of
2^23 bins, H = 32, Exponential(1) noise with 16 injected pulsars (f0 ~ U[100, N/32), duty
~ U[0.02, 0.2)), 262143 fundamentals.  L2 is flushed (a 2 x L2 write) before every timed step;
each step is timed alone with CUDA events on the stream hs_run launches on.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload long|long16|batch|plane|grad]
    python bench.py --impl reference      # the FP64 oracle on the host cores, same metric

N > 1 (torchrun): replicas only -- every rank runs the whole workload on its own GPU (the
harmonic sum of one spectrum has no exchange step); value = units of all ranks / max time.
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
KERNEL_SOURCES = ["hs_fwd1d.cuh", "hs_fwd1d_f32.cu", "hs_fwd1d_f16.cu", "hs_fwd1d_bf16.cu", "hs_fwd2d.cu",
                  "hs_bwd1d.cu", "hs_internal.cuh", "hs_api.cu"]


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def kernel_hash() -> str:
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        p = os.path.join(ROOT, "paper_2202_12817_gb300", "csrc", f)
        if os.path.exists(p):
            h.update(open(p, "rb").read())
    return h.hexdigest()[:16]


def load_json(path):
    try:
        return json.load(open(path))
    except Exception:
        return None


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
def oracle_rate(x_host, H, budget_s=8.0, frac=1.0):
    """Time the FP64 single-thread oracle (simple + greedy) on the first ``frac`` of the
    spectrum's fundamentals, repeated until ``budget_s``; returns (units/s, sample text)."""
    import oracle
    oracle.build()
    nf_all = oracle.nf_1d(x_host.size, H)
    nf = max(1, int(nf_all * frac))
    mu_s, sg_s = oracle.norm_exponential(1, 1, H)
    mu_g, sg_g = oracle.norm_exponential(2, 1, H)
    reps, t0 = 0, time.perf_counter()
    while True:
        oracle.simple_1d(x_host, H, mu_s, sg_s, nf=nf)
        oracle.greedy_1d(x_host, H, mu_g, sg_g, nf=nf)
        reps += 1
        el = time.perf_counter() - t0
        if el >= budget_s:
            break
    units = reps * nf * H
    return units / el, f"{reps} x fundamentals [0, {nf}) of the {x_host.size}-bin spectrum, simple + greedy, 1 thread"


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
    import torch
    t = torch.tensor([v], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------------------------------------
# workloads
# ---------------------------------------------------------------------------------------------
def algorithmic_bytes_1d(n_bins, H, forms, elem, nf, B=1, key="long"):
    """Compulsory bytes of one pass: distinct 32-B input sectors read (oracle-counted for the
    benchmark spectrum, stored in tests/golden/footprints.json; else the whole input) + outputs
    (snr 4 B + best_h 1 B per form, greedy path 4 B for H > 16) + mu/sigma tables."""
    gold = load_json(GOLDEN) or {}
    fp = gold.get(key, {}).get({1: "simple", 2: "greedy", 3: "fused"}[forms])
    if fp is not None and elem == 4:
        in_bytes, how = int(fp["sectors"]) * 32, "oracle sector footprint"
    elif fp is not None:
        in_bytes, how = int(fp["sectors_16bit"]) * 32, "oracle sector footprint"
    else:
        in_bytes, how = n_bins * elem, "whole input"
    pb = 4 if H > 16 else (2 if H > 8 else 1)
    out = 0
    if forms & 1:
        out += nf * 5
    if forms & 2:
        out += nf * (5 + pb)
    norms = 2 * 4 * H * (2 if forms == 3 else 1) * B
    return in_bytes + out + norms, how


def run_device(args, hs, torch, dev, rank, world, dist):
    wl = args.workload
    H = 32
    elem = 4
    dtype = hs.F32
    if wl in ("long", "long16", "longbf16"):
        N = synth.LONG_N
        dtype = {"long": hs.F32, "long16": hs.F16, "longbf16": hs.BF16}[wl]
        elem = 4 if dtype == hs.F32 else 2
        x32 = synth.device_spectrum(N, synth.SEED_BASE + 2, synth.long_spectrum_pulsars(), dev)
        x = x32 if dtype == hs.F32 else x32.to(torch.float16 if dtype == hs.F16 else torch.bfloat16)
        lengths = [N]
        desc = f"single FP32 spectrum 2^23 bins, H=32, 16 pulsars" if dtype == hs.F32 else \
            f"single spectrum 2^23 bins stored {'FP16' if dtype == hs.F16 else 'BF16'}, H=32"
        host_for_oracle = x32
    elif wl == "batch":
        H = 16
        b = synth.uneven_batch()
        x = synth.device_batch(b, dev)
        lengths = list(b.lengths)
        desc = "2048 uneven FP32 spectra (2^20..2^23 bins), H=16, 5% with a pulsar"
        host_for_oracle = None
    else:
        raise SystemExit(f"unknown workload {wl}")
    flags = hs.FLAG_GRAPH if wl == "batch" else 0
    offsets = None
    if wl == "batch":
        offsets = b.offsets[:-1]
    plan = hs.Plan(H, hs.SIMPLE | hs.GREEDY, lengths=lengths, dtype=dtype, offsets=offsets, flags=flags,
                   device=dev.index)
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
    K = args.steps
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    if dist:
        dist.barrier()
    torch.cuda.synchronize(dev)
    with ClockSampler(dev.index) as clk:
        t0 = time.perf_counter()
        for i in range(K):
            flush.fill_(float(i & 7))
            ev[i][0].record(stream)
            step()
            ev[i][1].record(stream)
        torch.cuda.synchronize(dev)
        wall = time.perf_counter() - t0
    if dist:
        dist.barrier()
    times = [a.elapsed_time(b) for a, b in ev]
    ms = sum(times) / K
    ms_max = max_over_ranks(ms, dist, dev)
    units = nf * H
    value = world * units / (ms_max / 1e3)
    fkey = "long" if wl.startswith("long") else wl
    alg, how = algorithmic_bytes_1d(plan.extent, H, 3, elem, nf, plan.B, key=fkey)
    peak, peak_kind = measured_peaks()
    achieved = alg / (ms / 1e3) / 1e9
    prof = load_json(PROFILE_TRAFFIC) or {}
    traffic = None
    pk = prof.get(wl)
    if pk and pk.get("kernel_hash") == kernel_hash():
        traffic = pk.get("dram_bytes_per_launch")

    # per-form separate passes (simple only, greedy only) on the same input
    per_form = {}
    for form, name in ((hs.SIMPLE, "simple"), (hs.GREEDY, "greedy")):
        p2 = hs.Plan(H, form, lengths=lengths, dtype=dtype, offsets=offsets, device=dev.index)
        if args.tuning:
            p2.tuning = json.loads(args.tuning)
        io = p2.alloc_form(*(ns if form == hs.SIMPLE else ng), path=form == hs.GREEDY, argmax=True)
        ws2 = p2.workspace(dev)
        for _ in range(3):
            flush.fill_(1.0)
            hs.run(p2, x, None, io if form == 1 else None, io if form == 2 else None, ws2, stream)
        reps = min(K, 200)
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
        for i in range(reps):
            flush.fill_(float(i & 7))
            evs[i][0].record(stream)
            hs.run(p2, x, None, io if form == 1 else None, io if form == 2 else None, ws2, stream)
            evs[i][1].record(stream)
        torch.cuda.synchronize(dev)
        fms = sum(a.elapsed_time(b) for a, b in evs) / reps
        fb, _ = algorithmic_bytes_1d(plan.extent, H, form, elem, nf, plan.B, key=fkey)
        per_form[name] = {"value": units / (fms / 1e3), "ms": round(fms, 5),
                          "hbm_gbs": round(fb / (fms / 1e3) / 1e9, 1),
                          "frac": round(fb / (fms / 1e3) / 1e9 / peak, 4)}
        p2.close()

    # end to end through the C ABI with host buffers: pinned H2D of the spectrum, run,
    # D2H of every output, all inside the timed region
    xh = x.cpu().pin_memory()
    outs_h = [torch.empty_like(t, device="cpu").pin_memory() for t in
              (s_io.snr, s_io.best_h, s_io.argmax, g_io.snr, g_io.best_h, g_io.path, g_io.argmax)]
    xd2 = torch.empty_like(x)
    e_reps = max(3, min(K, 20))
    for i in range(e_reps + 2):
        if i == 2:
            torch.cuda.synchronize(dev)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
        xd2.copy_(xh, non_blocking=True)
        hs.run(plan, xd2, None, s_io, g_io, ws, stream)
        for hbuf, dbuf in zip(outs_h, (s_io.snr, s_io.best_h, s_io.argmax, g_io.snr, g_io.best_h, g_io.path,
                                       g_io.argmax)):
            hbuf.copy_(dbuf, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    e_ms = max_over_ranks(e0.elapsed_time(e1) / e_reps, dist, dev)
    h2d = x.numel() * x.element_size()
    d2h = sum(t.numel() * t.element_size() for t in outs_h)

    result = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": args.warmup,
        "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {hs.F32: "f32", hs.F16: "f16 storage, f32 accumulate",
                  hs.BF16: "bf16 storage, f32 accumulate"}[dtype],
        "data": "synthetic",
        "config": {"workload": desc, "bins": int(plan.extent), "H": H, "fundamentals": int(nf),
                   "forms": "simple+greedy fused (one kernel)", "parallelism": "replicas" if world > 1 else "1 GPU",
                   "l2": "flushed before every timed step (write of max(2 x L2, 256 MiB))",
                   "tuning": plan.tuning.as_dict()},
        "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                     "frac": round(achieved / peak, 4), "traffic": traffic,
                     "algorithmic_bytes": int(alg), "bytes_basis": how, "peak_kind": peak_kind},
        "per_form": per_form,
        "e2e": {"value": world * units / (e_ms / 1e3), "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h)},
        "gpu_launches": K,
        "wall_s_timed_region": round(wall, 3),
    }
    return result, clk.summary(), host_for_oracle


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="long", choices=["long", "long16", "longbf16", "batch"])
    ap.add_argument("--tuning", default=None, help="JSON hs_tuning override")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    rank, world, local = dist_env()

    if args.impl == "reference":
        # the FP64 oracle on the host cores; under torchrun only rank 0 works
        if rank != 0:
            return
        H = 32
        x = synth.long_spectrum()
        import oracle
        nf = oracle.nf_1d(x.size, H)
        frac = 1.0 / 32
        for _ in range(args.warmup):
            oracle_rate(x, H, budget_s=0.0, frac=frac / 4)
        t0 = time.perf_counter()
        units = 0
        for _ in range(args.steps):
            r, sample = oracle_rate(x, H, budget_s=0.0, frac=frac)
            units += int(nf * frac) * H
        el = time.perf_counter() - t0
        v = units / el
        print(json.dumps({
            "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "single FP32 spectrum 2^23 bins, H=32, 16 pulsars", "H": H},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"each step: fundamentals [0, {int(nf * frac)}) of the 2^23-bin spectrum, "
                                       "simple + greedy, single-thread FP64"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))
        return

    import torch
    import paper_2202_12817_gb300 as hs
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    dist = init_dist(world, "nccl")
    result, clocks, host_src = run_device(args, hs, torch, dev, rank, world, dist)
    result["clocks"] = clocks
    if rank == 0 and world == 1 and not args.no_cpu_baseline and host_src is not None:
        xh = host_src.cpu().numpy()
        v, sample = oracle_rate(xh, result["config"]["H"], budget_s=10.0)
        result["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample}
    elif rank == 0:
        result["cpu_baseline"] = None
    if rank == 0:
        print(json.dumps(result))
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
