"""Writes footprints.json: the compulsory input bytes of the benchmark workloads, counted by the
FP64 oracle (distinct 32-byte sectors of the stored spectrum that the simple and/or greedy forms
read, with the greedy drift paths the oracle computes).  Calls only oracle/ and synth.

    python tests/golden/make_footprints.py
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
import synth  # noqa: E402


def footprint(x32, H):
    z = np.zeros(H)
    o = np.ones(H)
    path32 = oracle.greedy_1d(x32, H, z, o)[2]
    x16 = x32.astype(np.float16).astype(np.float32)
    path16 = oracle.greedy_1d(x16, H, z, o)[2]
    out = {}
    for name, forms in (("simple", 1), ("greedy", 2), ("fused", 3)):
        out[name] = {"sectors": oracle.sectors_1d(forms, 4, x32.size, H, path=path32),
                     "sectors_16bit": oracle.sectors_1d(forms, 2, x32.size, H, path=path16)}
    return out


def plane_footprint():
    H = 8
    tracks = synth.random_tracks(8, synth.PLANE_N_FREQ, synth.SEED_BASE + 4 + 1000)
    pl = synth.plane(synth.PLANE_N_FREQ, synth.PLANE_N_ROWS, synth.PLANE_Z0_ROW, synth.SEED_BASE + 4, tracks)
    path = oracle.greedy_2d(pl, synth.PLANE_Z0_ROW, H, np.zeros(H), np.ones(H))[2]
    return {"sectors": oracle.sectors_2d(synth.PLANE_N_FREQ, synth.PLANE_N_ROWS, synth.PLANE_Z0_ROW, H, path),
            "n_freq": synth.PLANE_N_FREQ, "n_rows": synth.PLANE_N_ROWS, "H": H}


def length_fractions(H=16, lengths=(1 << 20, 1 << 21, 1 << 22, 1 << 23)):
    """Fraction of a noise spectrum's 32-B sectors the fused pass reads, per spectrum length."""
    out = {}
    for n in lengths:
        x = synth.spectrum(n, 77 + n)
        path = oracle.greedy_1d(x, H, np.zeros(H), np.ones(H))[2]
        x16 = x.astype(np.float16).astype(np.float32)
        path16 = oracle.greedy_1d(x16, H, np.zeros(H), np.ones(H))[2]
        out[str(n)] = {"fused": oracle.sectors_1d(3, 4, n, H, path=path) / (n / 8),
                       "fused_16bit": oracle.sectors_1d(3, 2, n, H, path=path16) / (n / 16)}
    return out


def main():
    res = {"_about": "distinct 32-B sectors read per pass (oracle-counted); 'sectors' for FP32 "
                     "storage, 'sectors_16bit' for FP16 storage of the same spectrum",
           "long": dict(bins=synth.LONG_N, H=32, **footprint(synth.long_spectrum(), 32)),
           "plane": plane_footprint(),
           "batch_H16_fraction": length_fractions(16),
           "grad_H32_fraction": length_fractions(32, (1 << 20,))}
    json.dump(res, open(os.path.join(HERE, "footprints.json"), "w"), indent=1)
    print(json.dumps(res, indent=1))


if __name__ == "__main__":
    main()
