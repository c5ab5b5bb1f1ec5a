"""hs_run_fixed_scratch -- the forward pass for callers that cannot allocate device memory.

Plug-ins whose host framework owns every allocation, or real-time pipelines that forbid
allocation once running, may pass only their input and output buffers.  This entry point
takes the scratch hs_run receives as `workspace` (the dynamic schedule's tile counter) from a
fixed array inside the library instead.  The test calls it through the C ABI twice in a row
and checks that its outputs match hs_run's, with the tolerance the other parity tests use
(the launches are identical, so the results are in fact bit-equal).
"""
import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda", 0)


def _outputs(io):
    out = [io.snr.cpu().numpy(), io.best_h.cpu().numpy(), io.argmax.cpu().numpy()]
    if io.path is not None:
        out.append(io.path.cpu().numpy())
    return out


@pytest.mark.parametrize("tuning", [dict(kernel=0, threads=128, ctas_per_sm=2, dynamic=1),
                                    dict(kernel=1, threads=256, ctas_per_sm=1, dynamic=1)])
def test_fixed_scratch_matches_hs_run(hs, tuning):
    lengths = [50000, 70001, 4099, 131072]
    xs = [synth.spectrum(n, 500 + i, [synth.Pulsar(101.7 + 13 * i, 0.06)]) for i, n in enumerate(lengths)]
    plan = hs.Plan(16, hs.SIMPLE | hs.GREEDY, lengths=lengths)
    plan.tuning = tuning              # the schedule that keeps its tile counter in scratch memory
    buf = torch.zeros(plan.extent, dtype=torch.float32)
    for s, x in enumerate(xs):
        o = int(plan.input_offsets[s])
        buf[o:o + len(x)] = torch.from_numpy(x)
    x = buf.to(DEV)
    ns = [torch.from_numpy(a).to(DEV) for a in hs.norm_exponential(hs.SIMPLE, 1, 16)]
    ng = [torch.from_numpy(a).to(DEV) for a in hs.norm_exponential(hs.GREEDY, 1, 16)]
    ref_s, ref_g = plan.alloc_form(*ns, path=False), plan.alloc_form(*ng)
    hs.run(plan, x, None, ref_s, ref_g)
    torch.cuda.synchronize()
    want = _outputs(ref_s) + _outputs(ref_g)
    for call in range(2):             # the second call starts from the first call's scratch
        s_io, g_io = plan.alloc_form(*ns, path=False), plan.alloc_form(*ng)
        hs.run_fixed_scratch(plan, x, None, s_io, g_io)
        torch.cuda.synchronize()
        hs.check_device_error(plan)
        got = _outputs(s_io) + _outputs(g_io)
        for a, b, what in zip(got, want, ["snr", "best_h", "argmax", "snr", "best_h", "argmax", "path"]):
            if what == "snr":
                np.testing.assert_allclose(a, b, rtol=1e-5, atol=0, err_msg=f"call {call} {what}")
            else:
                assert np.array_equal(a, b), f"call {call} {what}"
    plan.close()
