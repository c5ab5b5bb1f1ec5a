// One order of the 2D greedy chain: the 1D greedy rule (Eq. 5, Algorithm 2) lifted to a 3x3
// neighbourhood.  The paper names the higher-dimensional sum (acceleration search) without
// giving an algorithm; the rule used here is: the best value starts at the centre, the 8
// neighbours are scanned in raster order (dz = -1..1 outer, df = -1..1 inner) and replace it
// only when strictly larger.  The winner's raster code (0..8, dz-major) moves the drift by
// (code % 3 - 1, code / 3 - 1) and is recorded in 4 bits per order.
#pragma once

#include "hs_internal.cuh"

namespace hs {

struct Chain2D {
    float sum;      // accumulated power along the path
    float best;     // running maximum of the normalised sum
    uint32_t bits;  // 4-bit raster code per order
    int df, dz;     // drift in f and z
    int bh;         // order of the running maximum
};

// Step order h of chain `c` on the neighbourhood c[0..8] (raster order around
// (h f + df, h z + dz)); rs / murs: 1/sigma_h and mu_h / sigma_h of that order.
__device__ __forceinline__ void chain2d_step(Chain2D &c, int h, const float (&v9)[9], float rs, float murs)
{
    float v = v9[4];
    int code = 4;
#pragma unroll
    for (int k = 0; k < 9; ++k)
        if (k != 4 && v9[k] > v) { v = v9[k]; code = k; }
    c.sum += v;
    c.df += code % 3 - 1;
    c.dz += code / 3 - 1;
    c.bits |= static_cast<uint32_t>(code) << (4 * (h - 1));
    const float snr = fmaf(c.sum, rs, -murs);
    if (h == 1 || snr > c.best) { c.best = snr; c.bh = h; }
}

}  // namespace hs
