"""Sharding DM-trial batches across GPUs (one process per GPU, torch.distributed).

The harmonic sum of one spectrum needs the whole spectrum (a fundamental range [a, b) reads
bins up to H b + H), so a single spectrum or plane runs as independent replicas.  Batches of
independent spectra shard with no data-path collective:

  * ``lpt_shards`` assigns spectra to ranks longest-first (work is proportional to length),
    deterministically, so every rank computes the same assignment without communicating
    (``shard_for_rank`` is one rank's share);
  * ``batch_step`` and ``grad_step`` are the steps the benchmark runs under torchrun, with the
    per-rank compute passed in (the library's kernels on a GPU, the oracle in the CPU tests);
  * after each rank's forward, ``gather_by_spectrum`` collects per-spectrum results (e.g. the
    argmax keys) into global spectrum order on every rank;
  * the training step's only exchange is ``allreduce_sum`` of dL/dw over ranks (each rank's
    adjoint already summed its own spectra);
  * ``max_over_ranks`` is the timing reduction of the benchmark.

The functions take torch tensors on any device; with the ``gloo`` backend they run on CPU.
"""
from __future__ import annotations

import heapq

import numpy as np


def lpt_shards(lengths, world: int):
    """Longest-processing-time assignment: spectra sorted by length (descending, index
    ascending on ties) go one by one to the least-loaded rank (lowest rank on ties).
    Returns ``world`` sorted lists of spectrum indices."""
    if world < 1:
        raise ValueError("world must be >= 1")
    lengths = np.asarray(lengths, dtype=np.int64)
    order = sorted(range(lengths.shape[0]), key=lambda i: (-int(lengths[i]), i))
    heap = [(0, r) for r in range(world)]
    shards = [[] for _ in range(world)]
    for i in order:
        load, r = heapq.heappop(heap)
        shards[r].append(i)
        heapq.heappush(heap, (load + int(lengths[i]), r))
    return [sorted(s) for s in shards]


def shard_loads(lengths, shards):
    lengths = np.asarray(lengths, dtype=np.int64)
    return [int(lengths[s].sum()) if s else 0 for s in shards]


def shard_for_rank(lengths, world: int, rank: int):
    """This rank's spectra under ``lpt_shards`` (sorted global indices)."""
    return lpt_shards(lengths, world)[rank]


def batch_step(mine, num_spectra: int, compute, group=None, gather: bool = True):
    """One sharded forward over a batch: ``compute(mine)`` runs this rank's spectra and returns
    their per-spectrum results (a tensor with one row per spectrum, in ``mine`` order), with no
    collective; with ``gather`` they are then collected into global spectrum order on every rank."""
    local = compute(mine)
    if not gather:
        return local
    return gather_by_spectrum(local, mine, num_spectra, group)


def grad_step(compute, group=None):
    """One sharded training step: ``compute()`` runs forward, loss and adjoint over this rank's
    spectra and returns its dL/dw (the sum over its spectra); the step's one exchange sums it
    over ranks."""
    return allreduce_sum(compute(), group)


def gather_by_spectrum(local_values, my_indices, num_spectra: int, group=None):
    """All-gather per-spectrum values (1 row per spectrum this rank owns, in ``my_indices``
    order) into a [num_spectra, ...] tensor in global spectrum order on every rank."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    idx = torch.as_tensor(my_indices, dtype=torch.int64, device=local_values.device)
    counts = torch.tensor([idx.numel()], dtype=torch.int64, device=local_values.device)
    all_counts = [torch.zeros_like(counts) for _ in range(world)]
    dist.all_gather(all_counts, counts, group=group)
    maxc = int(max(c.item() for c in all_counts))
    pad_v = torch.zeros((maxc,) + tuple(local_values.shape[1:]), dtype=local_values.dtype,
                        device=local_values.device)
    pad_i = torch.full((maxc,), -1, dtype=torch.int64, device=local_values.device)
    pad_v[:idx.numel()] = local_values
    pad_i[:idx.numel()] = idx
    vals = [torch.zeros_like(pad_v) for _ in range(world)]
    ids = [torch.zeros_like(pad_i) for _ in range(world)]
    dist.all_gather(vals, pad_v, group=group)
    dist.all_gather(ids, pad_i, group=group)
    out = torch.zeros((num_spectra,) + tuple(local_values.shape[1:]), dtype=local_values.dtype,
                      device=local_values.device)
    for v, i in zip(vals, ids):
        keep = i >= 0
        out[i[keep]] = v[keep]
    return out


def allreduce_sum(t, group=None):
    """Sum a tensor (dL/dw of each rank's spectra) over ranks, in place; returns it."""
    import torch.distributed as dist
    dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return t


def max_over_ranks(value: float, device="cpu", group=None) -> float:
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())
