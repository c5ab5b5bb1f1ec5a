"""Seeded random configurations of the optimal form and of the truncated tail against the FP64
oracle: H, forms, stored type, mitigation, per-spectrum normalisation, whitening, batch shape and
launch shape drawn together (the optimal kernel's unrolled H = 8 / 16 / 32 instances and its
generic loop, the tail kernel's chains and spectrum order)."""
import numpy as np
import pytest

import synth
from test_gpu_fwd1d import TUNINGS
from test_gpu_optimal import opt_case
from test_gpu_tail import tail_case

pytestmark = pytest.mark.gpu


def draw(seed: int, forms_choices):
    g = np.random.default_rng(seed)
    H = int(g.choice([8, 16, 32])) if g.random() < 0.5 else int(g.integers(1, 33))
    forms = int(g.choice(forms_choices))
    dtype = int(g.choice([0, 1, 2]))
    mitigation = bool(g.random() < 0.7)
    B = int(g.integers(1, 5))
    whiten = bool(g.random() < 0.25)
    if whiten:
        lengths = [int(g.integers(H + 2, 30000))] * B
    else:
        lengths = [int(g.integers(H + 2, H + 400)) if g.random() < 0.3 else int(g.integers(H + 2, 40000))
                   for _ in range(B)]
    spectra = []
    for s, n in enumerate(lengths):
        pulsars = synth.random_pulsars(int(g.integers(0, 3)), n, seed * 29 + s, f_lo=2.0, f_hi=max(3.0, n / 40))
        spectra.append(synth.spectrum(n, seed * 13 + s, pulsars))
    w = synth.whitening(lengths[0], seed) if whiten else None
    per_spec = bool(g.random() < 0.3)
    tuning = None
    if g.random() < 0.6:
        choices = [t for t in TUNINGS if not (whiten and t["kernel"] == 2)]
        tuning = choices[int(g.integers(len(choices)))]
    return dict(spectra=spectra, H=H, forms=forms, dtype=dtype, mitigation=mitigation, w=w, per_spec=per_spec,
                tuning=tuning)


@pytest.mark.parametrize("case", range(24))
def test_fuzz_optimal(hs, oracle_lib, case):
    c = draw(2202_12817 + 1000 + case, [4])
    opt_case(hs, oracle_lib, c["spectra"], c["H"], mitigation=c["mitigation"], dtype=c["dtype"], w=c["w"],
             per_spec_norm=c["per_spec"], seed=case)


@pytest.mark.parametrize("case", range(24))
def test_fuzz_truncated_tail(hs, oracle_lib, case):
    c = draw(2202_12817 + 2000 + case, [1, 2, 3, 4, 7])
    plan, _, _ = tail_case(hs, oracle_lib, c["spectra"], c["H"], c["forms"], mitigation=c["mitigation"],
                           dtype=c["dtype"], w=c["w"], tuning=c["tuning"] if c["forms"] & 3 else None)
    plan.close()
