"""Timing of the FP64 oracle for the benchmark's CPU baseline -- TEST INFRASTRUCTURE ONLY.

Run by ``bench.py`` in a subprocess, so that the OpenMP runtime of the all-core build never
shares a process with torch's:

    python -m oracle.timing --input x.npy --H 32 --forms 3 --threads T --budget S [--frac F]
    python -m oracle.timing --input plane.npy --dims 2 --z0 100 --H 8 --threads T --budget S

threads = 1 times liboracle.so (the oracle proper, one thread); threads > 1 times
liboracle_omp.so, the same source with its loops over fundamentals spread over `threads`
OpenMP threads.  The oracle runs repeatedly over a bounded sample of the input (the first
`frac` of a spectrum's fundamentals, or every fundamental of a plane: the caller passes a slice
of the columns of a larger plane)
until `budget` seconds have passed.  Prints one JSON line: units (bins x harmonics) per second,
the threads used, the sample and the host CPU model.
"""
from __future__ import annotations

import argparse
import json
import os
import platform
import subprocess
import sys
import time


def cpu_model() -> str:
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "hardware")):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return platform.processor() or platform.machine()


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--input", required=True)
    ap.add_argument("--dims", type=int, default=1)
    ap.add_argument("--H", type=int, required=True)
    ap.add_argument("--forms", type=int, default=3)
    ap.add_argument("--threads", type=int, default=1)
    ap.add_argument("--budget", type=float, default=5.0)
    ap.add_argument("--frac", type=float, default=1.0)
    ap.add_argument("--z0", type=int, default=0)
    a = ap.parse_args(argv)
    if a.threads > 1:
        os.environ["OMP_NUM_THREADS"] = str(a.threads)
    import numpy as np
    import oracle
    omp = oracle.use_openmp(a.threads > 1)
    threads = a.threads if omp else 1
    x = np.load(a.input)
    H = a.H
    reps, t0 = 0, time.perf_counter()
    if a.dims == 1:
        nf = max(1, int(oracle.nf_1d(x.size, H) * a.frac))
        mu_s, sg_s = oracle.norm_exponential(1, 1, H)
        mu_g, sg_g = oracle.norm_exponential(2, 1, H)
        while True:
            if a.forms & 1:
                oracle.simple_1d(x, H, mu_s, sg_s, nf=nf)
            if a.forms & 2:
                oracle.greedy_1d(x, H, mu_g, sg_g, nf=nf)
            reps += 1
            el = time.perf_counter() - t0
            if el >= a.budget:
                break
        what = {1: "simple", 2: "greedy", 3: "simple + greedy"}[a.forms]
        units = reps * nf * H
        sample = f"{reps} x fundamentals [0, {nf}) of a {x.size}-bin spectrum, {what}"
    else:
        f_lo, f_hi, z_lo, z_hi = oracle.domain_2d(x.shape[1], x.shape[0], a.z0, H)
        dom = (f_lo, f_hi, z_lo, z_hi)
        mu, sg = oracle.norm_exponential(2, 2, H, mean1=2.0)
        while True:
            oracle.greedy_2d(x, a.z0, H, mu, sg, dom=dom)
            reps += 1
            el = time.perf_counter() - t0
            if el >= a.budget:
                break
        units = reps * (f_hi - f_lo + 1) * (z_hi - z_lo + 1) * H
        sample = f"{reps} x every (f, z) fundamental of a {x.shape[0]} x {x.shape[1]} plane"
    print(json.dumps({"rate": units / el, "threads": threads, "sample": sample + f", {threads} thread(s)",
                      "cpu": cpu_model(), "seconds": el}))


if __name__ == "__main__":
    sys.exit(main())
