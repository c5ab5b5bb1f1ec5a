"""Seeded random configurations of the 1D forward against the FP64 oracle: batch shape and
layout, H, forms, stored type, mitigation, per-spectrum normalisation, whitening and launch shape
drawn together, so combinations that the grid tests do not list are exercised as well."""
import numpy as np
import pytest

import synth
from test_gpu_fwd1d import TUNINGS, run_case

pytestmark = pytest.mark.gpu


def draw_case(seed: int):
    g = np.random.default_rng(seed)
    H = int(g.integers(1, 33))
    forms = int(g.choice([1, 2, 3]))
    dtype = int(g.choice([0, 1, 2]))
    mitigation = bool(g.random() < 0.7)
    B = int(g.integers(1, 6))
    whiten = bool(g.random() < 0.25)
    if whiten:
        lengths = [int(g.integers(H + 1, 50000))] * B
    else:
        # a mix of tiny spectra (a few fundamentals, ragged last tile) and long ones
        lengths = [int(g.integers(H + 1, H + 300)) if g.random() < 0.35 else int(g.integers(H + 1, 70000))
                   for _ in range(B)]
    per_spec = bool(g.random() < 0.3)
    choices = [t for t in TUNINGS if not (whiten and t["kernel"] == 2)]
    tuning = choices[int(g.integers(len(choices)))] if g.random() < 0.8 else None
    offsets = None
    if B > 1 and g.random() < 0.3:
        # a custom layout: spectra in shuffled order with gaps, each start on a 32-element boundary
        order = g.permutation(B)
        offsets = [0] * B
        pos = 0
        for s in order:
            pos += 32 * int(g.integers(0, 4))
            offsets[s] = pos
            pos = (pos + lengths[s] + 31) // 32 * 32
    spectra = []
    for s, n in enumerate(lengths):
        pulsars = synth.random_pulsars(int(g.integers(0, 3)), n, seed * 31 + s, f_lo=2.0, f_hi=max(3.0, n / 40))
        spectra.append(synth.spectrum(n, seed * 17 + s, pulsars))
    w = synth.whitening(lengths[0], seed) if whiten else None
    return dict(spectra=spectra, H=H, forms=forms, dtype=dtype, mitigation=mitigation, w=w, tuning=tuning,
                offsets=offsets, per_spec_norm=per_spec)


@pytest.mark.parametrize("case", range(48))
def test_fuzz_forward(hs, oracle_lib, case):
    c = draw_case(2202_12817 + case)
    run_case(hs, oracle_lib, c["spectra"], c["H"], forms=c["forms"], dtype=c["dtype"], mitigation=c["mitigation"],
             w=c["w"], tuning=c["tuning"], offsets=c["offsets"], per_spec_norm=c["per_spec_norm"], seed=case)
