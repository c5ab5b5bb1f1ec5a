"""The N > 1 host path on CPU: two gloo ranks shard an uneven batch longest-first, run the
forward of their spectra, gather the per-spectrum results in global order and all-reduce the
training step's dL/dw, through the same helpers (``shard_for_rank``, ``batch_step``,
``grad_step``) that bench.py runs under torchrun.  The per-rank compute is the FP64 oracle (the CPU stand-in for the GPU
forward / adjoint, which these ranks cannot run); what is tested is the sharding and the
exchanges, against a single-process run of the whole batch."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

import synth


def _key(snr):
    """Per-spectrum argmax as the library's 64-bit key (ordered float32 snr, ~index)."""
    s32 = snr.astype(np.float32)
    n = int(np.argmax(s32))
    u = int(np.frombuffer(np.float32(s32[n]).tobytes(), np.uint32)[0])
    o = (~u & 0xFFFFFFFF) if u & 0x80000000 else (u | 0x80000000)
    return np.int64(np.uint64((o << 32) | (0xFFFFFFFF - n)).astype(np.int64))


def _batch():
    b = synth.uneven_batch(count=9, seed=31, choices=(1024, 2048, 4096, 8192), pulsar_fraction=0.34)
    xs = [synth.batch_trial(b, i) for i in range(9)]
    return b, xs


def _rank_work(oracle, xs, idx, H, w):
    mu, sg = oracle.norm_exponential(2, 1, H)
    keys, gw = [], np.zeros(len(w))
    for i in idx:
        snr, bh, path = oracle.greedy_1d(xs[i], H, mu, sg)
        keys.append(_key(snr))
        g = np.zeros(snr.size)
        g[np.argsort(-snr, kind="stable")[:4]] = -1.0
        gx = oracle.backward_1d(2, xs[i].size, H, bh, sg, g, path)
        gw[:len(gx)] += gx[:len(w)] * xs[i][:len(w)]
    return np.array(keys, np.int64), gw


def _worker(rank, world, port, out_dir):
    import torch.distributed as dist

    import oracle
    from paper_2202_12817_gb300 import dist as hsd
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    b, xs = _batch()
    H = 8
    w = np.ones(1024)
    # the helpers bench.py runs under torchrun, with the oracle as each rank's compute
    mine = hsd.shard_for_rank(b.lengths, world, rank)
    # each rank draws only its own trials, packed as synth.sub_batch lays them out (as on a GPU)
    sb = synth.sub_batch(b, mine)
    xs_local = [synth.batch_trial(sb, k) for k in range(len(mine))]
    assert all(np.array_equal(a, xs[i]) for a, i in zip(xs_local, mine))
    local_ids = list(range(len(mine)))

    def forward(idx):
        assert list(idx) == list(mine)
        return torch.from_numpy(_rank_work(oracle, xs_local, local_ids, H, w)[0])

    all_keys = hsd.batch_step(mine, len(xs), forward)
    gw_t = hsd.grad_step(lambda: torch.from_numpy(_rank_work(oracle, xs_local, local_ids, H, w)[1]))
    local = hsd.batch_step(mine, len(xs), forward, gather=False)
    assert local.shape[0] == len(mine)
    tmax = hsd.max_over_ranks(float(rank + 1))
    np.savez(os.path.join(out_dir, f"rank{rank}.npz"), keys=all_keys.numpy(), gw=gw_t.numpy(), tmax=tmax,
             shard=np.array(mine))
    dist.barrier()
    dist.destroy_process_group()


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def test_lpt_shards():
    from paper_2202_12817_gb300 import dist as hsd
    lengths = [1 << 23, 1 << 20, 1 << 21, 1 << 23, 1 << 22, 1 << 20, 1 << 21]
    for world in (1, 2, 3, 8):
        shards = hsd.lpt_shards(lengths, world)
        flat = sorted(i for s in shards for i in s)
        assert flat == list(range(len(lengths)))
        loads = hsd.shard_loads(lengths, shards)
        assert max(loads) - min(loads) <= max(lengths)          # LPT balance bound
        assert shards == hsd.lpt_shards(lengths, world)         # deterministic
    # longest first: the two 2^23 spectra go to different ranks
    s2 = hsd.lpt_shards(lengths, 2)
    assert (0 in s2[0]) != (3 in s2[0])
    with pytest.raises(ValueError):
        hsd.lpt_shards(lengths, 0)


def test_two_gloo_ranks_match_single_process(tmp_path, oracle_lib):
    world = 2
    mp.spawn(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    b, xs = _batch()
    keys_ref, gw_ref = _rank_work(oracle_lib, xs, list(range(len(xs))), 8, np.ones(1024))
    shards = []
    for r in range(world):
        d = np.load(tmp_path / f"rank{r}.npz")
        assert np.array_equal(d["keys"], keys_ref)          # gathered in global order on every rank
        np.testing.assert_allclose(d["gw"], gw_ref, rtol=1e-12, atol=1e-12)
        assert float(d["tmax"]) == 2.0
        shards.append(list(d["shard"]))
    assert sorted(i for s in shards for i in s) == list(range(len(xs)))
