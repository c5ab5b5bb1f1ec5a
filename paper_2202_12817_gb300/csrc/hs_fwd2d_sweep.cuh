// Column-sweep schedule of the 2D greedy sum (kernel 2 of a 2D plan).
//
// Order h of chain (f, z) reads the 3x3 neighbourhood of (h f + df, h z + dz), so the plane value
// at column c and row z0 + r is read at order h by the chains near (c / h, r / h), for every h.
// One thread per chain carrying all orders in registers reads those values at unrelated times,
// and on a plane larger than L2 each order fetches its own copy from DRAM.  The sweep instead
// orders the work by the anchor column h f: band j holds every event (f, z, h) with h f in
// [j Wb, j Wb + Wb).  A CTA stages the band's columns of the rows the domain can reach (plus a
// halo of kSweepHalo columns on each side, >= H) in shared memory with one 2D bulk tensor copy,
// and runs all of the band's events from there; between orders a chain's state (sum, running
// maximum, path, drift, best order) waits in global memory (L2), read and written there directly.  Order h - 1 of a chain f >= Wb lies
// in an earlier band (its anchor is h f - f), so a band depends only on earlier bands -- for each
// order on at most two of them: CTAs take bands in order from a ticket counter and wait (bounded)
// on the done flags of the bands holding the previous orders of their chains.  Chains with f < f_s stay out of the sweep and run whole in
// registers in a few prefix tasks.
#pragma once

#include <cuda.h>

#include "hs_internal.cuh"

namespace hs {

constexpr int kSweepHalo = 8;          // staged columns on each side of a band (>= kMaxH2D)
constexpr int kSweepMaxBox = 256;      // tensor-copy box limit per dimension
constexpr int kSweepMaxStages = 4;     // buffers (bands in flight per CTA)
constexpr int kSweepRing = 64;         // finished bands queued for the publisher

struct Sweep2DArgs {
    Fwd2DArgs a;          // plane, domain, outputs, error word (zfast unused)
    int64_t f_s;          // chains f in [f_lo, f_s): prefix tasks; f in [f_s, f_hi]: the sweep
    int64_t n_prefix;     // prefix tasks (one chain per thread)
    int64_t band_lo;      // first band; band j covers anchors [(band_lo + j) Wb, ... + Wb)
    int64_t nbands;
    int32_t Wb;           // anchor columns per band (multiple of 16)
    int32_t r_lo, nr;     // staged rows [r_lo, r_lo + nr)
    int32_t box_bytes;    // bytes of one staged tile, nr x (Wb + 2 kSweepHalo) elements
    int32_t buf_bytes;    // box_bytes rounded up to 128: one buffer
    int32_t nbuf;         // buffers, 2..kSweepMaxStages
    int64_t nfs;          // chains in the sweep, f_hi + 1 - f_s: the row stride of `state`
    int4 *state;          // [z - z_lo][f - f_s] chain state between orders (z-major: the chains of
                          // adjacent f that adjacent compute threads run are adjacent)
    unsigned *sync;       // [0] ticket counter, [1] unused, [2 + j] band j done
};

// Kernel entry per stored type; launched as (const __grid_constant__ CUtensorMap, Sweep2DArgs)
// with nbuf x buf_bytes of dynamic shared memory and kSweepThreads threads: warp 0 claims bands,
// waits on their dependencies and issues their copies up to nbuf - 1 bands ahead, warp 1
// publishes finished bands, the other warps compute.
const void *fwd2d_sweep_kernel(int dtype);
constexpr int kSweepThreads = 512;
constexpr int kSweepMaxThreads = 1024;

}  // namespace hs
