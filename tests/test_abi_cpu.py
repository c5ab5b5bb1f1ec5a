"""The C-ABI library without a GPU: it loads, exports every symbol hs.h declares, validates
plans on the host (HS_FLAG_NO_DEVICE) and its host helpers agree with the oracle."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def hs():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2202_12817_gb300 as m
    return m


def declared_functions():
    txt = open(os.path.join(ROOT, "include", "hs.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(hs_[a-z0-9_]+)\s*\(", txt)))


def test_exports_every_declared_symbol(hs):
    names = declared_functions()
    assert len(names) >= 14
    L = ctypes.CDLL(hs.LIB_PATH)
    for n in names:
        assert hasattr(L, n), n
    assert hs.lib().hs_version() == b"1.0.0"


def test_status_strings(hs):
    for s in range(8):
        assert hs.status_string(s) not in ("", "unknown status")
    assert hs.status_string(99) == "unknown status"


@pytest.mark.parametrize("form,dims,mit,mean1", [(1, 1, True, 1.0), (2, 1, True, 1.0), (2, 1, False, 1.0),
                                                 (2, 2, True, 2.0), (1, 1, True, 3.5)])
def test_norm_exponential_matches_oracle(hs, oracle_lib, form, dims, mit, mean1):
    H = 8 if dims == 2 else 32
    mu, sg = hs.norm_exponential(form, dims, H, mit, mean1)
    rmu, rsg = oracle_lib.norm_exponential(form, dims, H, mitigation=mit, mean1=mean1)
    np.testing.assert_allclose(mu, rmu, rtol=1e-7)
    np.testing.assert_allclose(sg, rsg, rtol=1e-7)


def test_norm_exponential_rejects(hs):
    with pytest.raises(hs.HSError):
        hs.norm_exponential(1, 2, 8)          # 2D has only the greedy form
    with pytest.raises(hs.HSError) as e:
        hs.norm_exponential(hs.OPTIMAL, 1, 8)  # the optimum over paths has no closed form
    assert e.value.status == 2
    with pytest.raises(hs.HSError):
        hs.norm_exponential(2, 1, 33)
    with pytest.raises(hs.HSError):
        hs.norm_exponential(2, 1, 4, True, -1.0)


def plan(hs, **kw):
    kw.setdefault("flags", 0)
    kw["flags"] |= hs.FLAG_NO_DEVICE
    return hs.Plan(**kw)


def test_plan_counts_offsets(hs):
    lens = [131072, 1000, 33, 40]
    p = plan(hs, H=32, forms=3, lengths=lens)
    assert list(p.counts) == [(n - 1) // 32 for n in lens]
    assert list(p.fund_offsets) == [0] + list(np.cumsum(p.counts))
    off = p.input_offsets
    assert off[0] == 0 and all(o % 32 == 0 for o in off[:-1])
    assert all(off[i] >= off[i - 1] + lens[i - 1] for i in range(1, len(lens)))
    assert off[-1] == off[-2] + lens[-1]
    assert p.path_bytes == 4 and p.workspace_bytes > 0
    assert plan(hs, H=8, forms=2, lengths=[100]).path_bytes == 1
    assert plan(hs, H=16, forms=2, lengths=[100]).path_bytes == 2


def test_plan_2d_domain(hs):
    p = plan(hs, H=8, forms=hs.GREEDY, dims=2, n_freq=1 << 21, n_rows=201, z0_row=100)
    assert p.domain == (1, 262142, -11, 11)
    assert p.total_fundamentals == 262142 * 23


def test_host_chunks_setting(hs):
    p = plan(hs, H=32, forms=3, lengths=[1 << 23])
    for k in (0, 1, 4, 16):
        p.host_chunks = k
        assert p.host_chunks == k
    for bad in (-1, 17):
        with pytest.raises(hs.HSError):
            p.host_chunks = bad


def test_plan_2d_reduced_precision(hs):
    """2D plans take FP16 / BF16 planes with the same domain as FP32."""
    for dt in (hs.F16, hs.BF16):
        p = plan(hs, H=8, forms=hs.GREEDY, dims=2, n_freq=1 << 21, n_rows=201, z0_row=100, dtype=dt)
        assert p.domain == (1, 262142, -11, 11) and p.extent == 201 << 21


def test_plan_2d_domain_matches_oracle(hs, oracle_lib):
    for nf, nr, z0, H in [(5000, 41, 20, 3), (1000, 30, 10, 4), (777, 9, 4, 1)]:
        p = plan(hs, H=H, forms=hs.GREEDY, dims=2, n_freq=nf, n_rows=nr, z0_row=z0)
        assert p.domain == oracle_lib.domain_2d(nf, nr, z0, H) or nr != 2 * z0 + 1


@pytest.mark.parametrize("kw", [
    dict(H=0, forms=3, lengths=[100]),
    dict(H=33, forms=3, lengths=[100]),
    dict(H=8, forms=0, lengths=[100]),
    dict(H=8, forms=8, lengths=[100]),
    dict(H=4, forms=6, dims=2, n_freq=1000, n_rows=41, z0_row=20),   # 2D has no optimal form
    dict(H=8, forms=3, lengths=[8]),                       # N < H + 1: no fundamental
    dict(H=8, forms=3, lengths=[100], dtype=3),
    dict(H=8, forms=3, lengths=[100, 100], offsets=[0, 3]),   # misaligned offset
    dict(H=8, forms=3, lengths=[100, 100], offsets=[0, 64]),  # overlapping spectra
    dict(H=8, forms=3, lengths=[100, 96], flags=1 << 2),      # whitening needs equal lengths
    dict(H=8, forms=3, lengths=[100], flags=1 << 12),         # unknown flag
    dict(H=9, forms=2, dims=2, n_freq=1000, n_rows=41, z0_row=20),
    dict(H=4, forms=1, dims=2, n_freq=1000, n_rows=41, z0_row=20),
    dict(H=4, forms=2, dims=2, n_freq=1000, n_rows=5, z0_row=2),   # no z fits
    dict(H=4, forms=2, dims=3, n_freq=1000, n_rows=41, z0_row=20),
    dict(H=4, forms=2, dims=2, n_freq=1000, n_rows=41, z0_row=20, dtype=3),
])
def test_plan_rejects(hs, kw):
    with pytest.raises(hs.HSError) as e:
        plan(hs, **kw)
    assert e.value.status in (1, 2)


def test_offsets_accepted(hs):
    p = plan(hs, H=8, forms=3, lengths=[100, 100], offsets=[128, 0])
    assert list(p.input_offsets[:2]) == [128, 0] and p.extent == 228
    p = plan(hs, H=8, forms=3, lengths=[100, 100], offsets=[0, 104], dtype=hs.F16)
    assert p.extent == 204


def test_run_without_device(hs):
    p = plan(hs, H=8, forms=3, lengths=[100])
    L = hs.lib()
    assert L.hs_run(p.handle, 16, None, None, None, None, None) == 7
    assert L.hs_backward(p.handle, 2, 16, None, None, None, None, None, None, None) == 7
    assert L.hs_check_device_error(p.handle, None) == 7
    assert L.hs_run(None, 16, None, None, None, None, None) == 1


def test_tuning_validation(hs):
    p = plan(hs, H=8, forms=3, lengths=[10000])
    t = p.tuning
    assert t.threads in (64, 128, 256) and t.fund_per_thread == 1
    assert t.kernel == 6 and t.threads == 128          # FP32: paired lanes
    t16 = plan(hs, H=8, forms=3, lengths=[10000], dtype=hs.F16).tuning
    assert t16.kernel == 0 and t16.threads == 128
    p.tuning = dict(kernel=0, threads=128, fund_per_thread=1, ctas_per_sm=4, dynamic=1)
    assert p.tuning.as_dict() == dict(kernel=0, threads=128, fund_per_thread=1, ctas_per_sm=4, dynamic=1,
                                      stages=0, stage_kb=0, prefetch=0, producers=0)
    with pytest.raises(hs.HSError):      # L2 prefetch belongs to the window and paired-lane kernels
        p.tuning = dict(kernel=0, threads=128, prefetch=1)
    p.tuning = dict(kernel=6, threads=128, ctas_per_sm=8, dynamic=1, prefetch=1)
    p.tuning = dict(kernel=7, threads=64)
    with pytest.raises(hs.HSError):      # no kernel 8
        p.tuning = dict(kernel=8, threads=128)
    p.tuning = dict(kernel=2, threads=128, stages=2, stage_kb=24, prefetch=1, producers=2)
    p.tuning = dict(kernel=3, threads=128, fund_per_thread=2)
    p.tuning = dict(kernel=2, threads=256, stages=2, stage_kb=96, producers=1)
    big = plan(hs, H=32, forms=3, lengths=[100000])
    with pytest.raises(hs.HSError):      # order-32 window of a 256-wide tile needs ~32 KiB
        big.tuning = dict(kernel=2, threads=256, stages=4, stage_kb=24, producers=2)
    with pytest.raises(hs.HSError):      # more than 227 KiB of shared memory
        big.tuning = dict(kernel=2, threads=128, stages=16, stage_kb=17, producers=4)
    with pytest.raises(hs.HSError):      # more producer warps than slots
        big.tuning = dict(kernel=2, threads=128, stages=4, stage_kb=17, producers=5)
    with pytest.raises(hs.HSError):      # more than 640 threads
        big.tuning = dict(kernel=2, threads=512, stages=3, stage_kb=66, producers=5)
    big.tuning = dict(kernel=2, threads=512, stages=3, stage_kb=66, producers=3)
    white = plan(hs, H=8, forms=3, lengths=[1000, 1000], flags=hs.FLAG_WHITENING)
    assert white.tuning.kernel == 0
    with pytest.raises(hs.HSError) as e:
        white.tuning = dict(kernel=2, threads=128, stages=2, stage_kb=16, producers=1)
    assert e.value.status == 2
    for bad in (dict(kernel=2, threads=128, fund_per_thread=1, ctas_per_sm=0, dynamic=0),
                dict(kernel=0, threads=100, fund_per_thread=1, ctas_per_sm=0, dynamic=0),
                dict(kernel=0, threads=512, fund_per_thread=1, ctas_per_sm=0, dynamic=0),
                dict(kernel=2, threads=544, stages=2, stage_kb=80, producers=1),
                dict(kernel=0, threads=128, fund_per_thread=1, ctas_per_sm=0, dynamic=1),
                dict(kernel=2, threads=128, stages=1, stage_kb=48, producers=1),
                dict(kernel=2, threads=128, stages=17, stage_kb=8, producers=1),
                dict(kernel=2, threads=128, stages=4, stage_kb=8, producers=0),
                dict(kernel=3, threads=128, fund_per_thread=1),
                dict(kernel=0, threads=128, fund_per_thread=2)):
        with pytest.raises(hs.HSError):
            p.tuning = bad


def test_decode_argmax(hs):
    for snr, n in [(3.25, 17), (-2.5, 0), (0.0, 4095), (1e6, 123456)]:
        u = np.frombuffer(np.float32(snr).tobytes(), np.uint32)[0]
        o = (u & 0x7FFFFFFF) | 0x80000000 if not (u & 0x80000000) else (~u & 0xFFFFFFFF)
        key = (int(o) << 32) | (0xFFFFFFFF - n)
        assert hs.decode_argmax(np.int64(np.uint64(key).astype(np.int64))) == (np.float32(snr), n)
        assert hs.decode_argmax(key) == (np.float32(snr), n)


def test_plan_create_without_gpu_fails_cleanly(hs):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(hs.HSError) as e:
        hs.Plan(H=8, forms=3, lengths=[100])
    assert e.value.status == 4


def test_tuning_2d_block_order(hs):
    """Kernels 0 (f-tiles fastest) and 1 (z rows fastest, the default) take 256 threads and
    nothing else; a plane too small for the column sweep refuses kernel 2."""
    p = hs.Plan(4, hs.GREEDY, dims=2, n_freq=1000, n_rows=41, z0_row=20, flags=hs.FLAG_NO_DEVICE)
    assert p.tuning.kernel == 1 and p.tuning.threads == 256
    p.tuning = dict(kernel=0, threads=256)
    assert p.tuning.kernel == 0
    for bad in (dict(kernel=2, threads=256), dict(kernel=1, threads=128), dict(kernel=1, threads=256, dynamic=1)):
        with pytest.raises(hs.HSError):
            p.tuning = bad
    p.close()


def test_tuning_2d_sweep(hs):
    """The column sweep (kernel 2): its workspace holds 16 bytes of chain state per sweep chain
    (f >= 64 x 16, the narrowest band) plus one flag per band; it takes 256, 512 or 1024 threads,
    band widths that are multiples of 16 columns (at most 240) whose buffers fit in shared memory,
    2..4 stages;
    it is refused for checked plans and for rows whose byte stride is not a multiple of 16."""
    n_freq, n_rows, z0, H = 1 << 21, 201, 100, 8
    p = hs.Plan(H, hs.GREEDY, dims=2, n_freq=n_freq, n_rows=n_rows, z0_row=z0, flags=hs.FLAG_NO_DEVICE)
    f_lo, f_hi, z_lo, z_hi = p.domain
    nz, f_s = z_hi - z_lo + 1, 64 * 16
    nbands = H * f_hi // 16 - f_s // 16 + 1
    assert p.workspace_bytes == nz * (f_hi - f_s + 1) * 16 + (4 * (2 + nbands) + 255) // 256 * 256
    assert p.tuning.kernel == 1                       # without a device (no L2 size) the default is kernel 1
    # a buffer holds the band's tile, 193 staged rows x (Wb + 16) columns: 2 x 128-column bands fit
    # in 227 KiB of shared memory, 3 x 64 and 4 x 48 too
    for ok in (dict(kernel=2, threads=512), dict(kernel=2, threads=256, stage_kb=2, stages=3),
               dict(kernel=2, threads=1024, stage_kb=4, ctas_per_sm=1), dict(kernel=2, threads=512, stage_kb=1, stages=4),
               dict(kernel=2, threads=512, stage_kb=8), dict(kernel=2, threads=512, stage_kb=4, stages=3),
               dict(kernel=2, threads=512, stage_kb=3, stages=4)):
        p.tuning = ok
        assert p.tuning.kernel == 2
    for bad in (dict(kernel=2, threads=128), dict(kernel=2, threads=512, stages=1), dict(kernel=2, threads=512, stages=5),
                dict(kernel=2, threads=512, stage_kb=10), dict(kernel=2, threads=512, stage_kb=4, stages=4),
                dict(kernel=2, threads=512, stage_kb=16),
                dict(kernel=2, threads=512, dynamic=1), dict(kernel=1, threads=256, stages=2)):
        with pytest.raises(hs.HSError):
            p.tuning = bad
    p.close()
    for kw in (dict(n_freq=n_freq + 1), dict(flags=hs.FLAG_CHECKED)):
        args = dict(n_freq=n_freq, n_rows=n_rows, z0_row=z0, flags=0)
        args.update(kw)
        q = hs.Plan(H, hs.GREEDY, dims=2, n_freq=args["n_freq"], n_rows=n_rows, z0_row=z0,
                    flags=hs.FLAG_NO_DEVICE | args["flags"])
        assert q.workspace_bytes == 0
        with pytest.raises(hs.HSError):
            q.tuning = dict(kernel=2, threads=512)
        q.close()


def test_sweep_default_band_width_narrows_to_the_plane(hs):
    """stage_kb = 0 takes 112-column bands for FP32 where the plane has chains beyond the 64-band-width
    register prefix, else the widest narrower multiple of 16 that has some (33000 x 201 rows, H = 6:
    f_hi = 5498, so 112 (f_s = 7168) is too wide but 80 (f_s = 5120) is not); nothing fits a plane
    whose chains all lie in the prefix of the narrowest band."""
    p = plan(hs, H=6, forms=hs.GREEDY, dims=2, n_freq=33000, n_rows=201, z0_row=150)
    assert p.domain[1] == 5498
    p.tuning = dict(kernel=2, threads=512)
    assert p.tuning.kernel == 2 and p.tuning.stage_kb == 0
    with pytest.raises(hs.HSError):
        p.tuning = dict(kernel=2, threads=512, stage_kb=7)       # 112 columns given explicitly
    p.tuning = dict(kernel=2, threads=512, stage_kb=5)           # 80 columns: f_s = 5120 <= 5498
    q = plan(hs, H=6, forms=hs.GREEDY, dims=2, n_freq=6000, n_rows=201, z0_row=150)
    with pytest.raises(hs.HSError):                               # f_hi = 998 < 64 x 16
        q.tuning = dict(kernel=2, threads=512)


def test_selftest_timeout_needs_device(hs):
    p = plan(hs, H=8, forms=hs.GREEDY, lengths=[1000])
    with pytest.raises(hs.HSError) as e:
        hs.selftest_timeout(p, 1000, stream=0)
    assert e.value.status == 7     # HS_ERR_NO_DEVICE
