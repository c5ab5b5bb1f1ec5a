"""Reduced-precision storage: the SNR error of FP16 / BF16 spectra (FP32 accumulation) against
the FP64 oracle on the original FP32 values, per workload shape.

Paths, best h and argmax are checked exactly against the oracle fed the same rounded values in
test_gpu_fwd1d; here the comparison is with the un-rounded input, so the numbers measure what
16-bit storage costs.  With HS_REPORT_DIR set, the figures are also written to
$HS_REPORT_DIR/precision_report.json.
"""
import json
import os

import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda", 0)
REPORT_DIR = os.environ.get("HS_REPORT_DIR")


def _run(hs, x, H, dtype):
    plan = hs.Plan(H, hs.SIMPLE | hs.GREEDY, lengths=[x.size], dtype=dtype)
    t = {0: torch.float32, 1: torch.float16, 2: torch.bfloat16}[dtype]
    ns = [torch.from_numpy(a).to(DEV) for a in hs.norm_exponential(1, 1, H)]
    ng = [torch.from_numpy(a).to(DEV) for a in hs.norm_exponential(2, 1, H)]
    out = plan.forward(torch.from_numpy(x).to(t).to(DEV), ns, ng)
    torch.cuda.synchronize()
    res = {f: (out[f].snr.cpu().numpy().astype(np.float64), out[f].best_h.cpu().numpy(),
               hs.decode_argmax(out[f].argmax.cpu().numpy()[0])[1]) for f in (1, 2)}
    plan.close()
    return res


@pytest.mark.parametrize("name", ["single_131072", "long_2p23"])
def test_reduced_precision_error(hs, oracle_lib, name):
    x = synth.single_pulse_spectrum() if name == "single_131072" else synth.long_spectrum()
    H = 32
    o = oracle_lib
    ref = {}
    mu_s, sg_s = hs.norm_exponential(1, 1, H)
    mu_g, sg_g = hs.norm_exponential(2, 1, H)
    ref[1] = o.simple_1d(x, H, mu_s, sg_s)
    ref[2] = o.greedy_1d(x, H, mu_g, sg_g)[:2]
    report = {}
    for dtype, dname in ((0, "f32"), (1, "f16"), (2, "bf16")):
        got = _run(hs, x, H, dtype)
        for form, fname in ((1, "simple"), (2, "greedy")):
            r_snr, r_bh = ref[form]
            g_snr, g_bh, g_arg = got[form]
            mu, sg = (mu_s, sg_s) if form == 1 else (mu_g, sg_g)
            idx = r_bh.astype(np.int64) - 1
            scale = (np.abs(r_snr * sg[idx] + mu[idx]) + np.abs(mu[idx])) / sg[idx]
            err = np.abs(g_snr - r_snr)
            entry = {"max_abs_snr_err": float(err.max()), "max_rel_err_vs_unc_magnitude": float((err / scale).max()),
                     "best_h_change_rate": float(np.mean(g_bh != r_bh)),
                     "argmax_same": bool(g_arg == int(np.argmax(r_snr)))}
            # median error over all fundamentals (most keep the FP32 path)
            entry["median_abs_snr_err"] = float(np.median(err))
            report[f"{dname}/{fname}"] = entry
    if REPORT_DIR and os.path.isdir(REPORT_DIR):
        path = os.path.join(REPORT_DIR, "precision_report.json")
        prev = json.load(open(path)) if os.path.exists(path) else {}
        prev[name] = report
        json.dump(prev, open(path, "w"), indent=1)
    for key, entry in report.items():
        if key.startswith("f32/"):
            assert entry["max_rel_err_vs_unc_magnitude"] <= 1e-5, (key, entry)
            continue
        # 16-bit storage rounds each value by up to 2^-11 (FP16) / 2^-8 (BF16) relative, which
        # also flips near-tied greedy comparisons, so a few fundamentals take a different path
        # (a large error there); the detection itself -- the per-spectrum argmax -- survives,
        # best h rarely changes and the typical error is the storage rounding
        assert entry["argmax_same"], (key, entry)
        assert entry["best_h_change_rate"] < 0.05, (key, entry)
        assert entry["median_abs_snr_err"] < (0.01 if key.startswith("f16") else 0.05), (key, entry)
