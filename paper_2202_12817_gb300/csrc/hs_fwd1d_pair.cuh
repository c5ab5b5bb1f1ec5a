// 1D forward kernel with paired lanes (kernels 6, 7): the simple form (Eq. 3) and the greedy
// form (Eq. 5 / Algorithm 2) of one fundamental are computed by two adjacent lanes of a warp, and
// at every order both lanes' reads are issued by the same load instruction.  Kernel 7 gives each
// lane two fundamentals, so a spectrum needs half the lanes and every lane has two loads in flight.
//
// Why: random gathers from L2 are limited by the number of 128-byte-line requests the SMs can
// issue (about 0.9 per clock per SM on GB300, whatever the number of 32-byte sectors each
// request carries).  The direct kernel reads x[h n] (simple) and x[m] (greedy) in separate
// instructions, so a line holding both is requested twice; here the two lanes' addresses meet in
// one instruction and the line is requested once.  Loads stay 4 bytes wide (16-byte random
// gathers run slower on GB300).
#pragma once

#include "hs_fwd1d.cuh"

namespace hs {

// A load the compiler may not merge with an earlier load of the same address.
__device__ __forceinline__ int64_t ld_volatile_i64(const int64_t *p)
{
    return *reinterpret_cast<const volatile int64_t *>(p);
}

// CH: fundamentals (chains) per lane, interleaved order by order so that each lane keeps CH
// loads in flight; a tile is CH x (fundamentals per CTA pass).  32 registers a thread at most,
// so every thread slot of an SM is usable.
template <typename T, int FORMS, bool WHITEN, int CH>
__global__ void __launch_bounds__(256, 8) k_fwd1d_pair(const Fwd1DArgs a)
{
    // per (order, form): {1/sigma, mu/sigma}; SNR = S * rs - murs (one FMA)
    __shared__ float2 tab[kMaxH1D][2];
    __shared__ unsigned long long red[2][8];
    __shared__ long long s_tile;
    constexpr bool kBoth = FORMS == (HS_FORM_SIMPLE | HS_FORM_GREEDY);
    const int H = a.H;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // form of this lane: with both forms, even lanes simple and odd lanes greedy, two lanes per
    // fundamental; with one form, one lane per fundamental
    const bool greedy = kBoth ? (lane & 1) != 0 : FORMS == HS_FORM_GREEDY;
    const int role = greedy ? 1 : 0;
    const int fpp = kBoth ? static_cast<int>(blockDim.x >> 1) : static_cast<int>(blockDim.x);   // per pass
    const int li = kBoth ? static_cast<int>(threadIdx.x >> 1) : static_cast<int>(threadIdx.x);
    const bool pair1 = greedy && a.mitigation != 0;   // order 1 compares x[n], x[n+1]

    if (a.pf_chunk > 0 && threadIdx.x == 0) {
        // the input fits comfortably in L2: bring this CTA's share in before the gathers need it
        int64_t lo = static_cast<int64_t>(blockIdx.x) * a.pf_chunk;
        const int64_t hi = lo + a.pf_chunk < a.pf_bytes ? lo + a.pf_chunk : a.pf_bytes;
        const unsigned char *src = static_cast<const unsigned char *>(a.x);
        for (; lo + 16 <= hi; lo += 65536) {
            const int64_t nb = (hi - lo < 65536 ? hi - lo : 65536) & ~static_cast<int64_t>(15);
            asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src + lo), "r"(static_cast<uint32_t>(nb))
                         : "memory");
        }
    }

    int loaded_spec = -1;
    int64_t tile = blockIdx.x;
    if (a.tile_counter) {
        if (threadIdx.x == 0) {
            wait_prior_grid();
            s_tile = static_cast<long long>(atomicAdd(a.tile_counter, 1ull));
        }
        __syncthreads();
        tile = s_tile;
    }
    while (tile < a.total_tiles) {
        // the fused one-chain kernel (kernel 6, the default for one FP32 spectrum) keeps the search:
        // the division path would push it past its 32 registers
        constexpr bool kSearchOnly = kBoth && CH == 1;
        const int s = tile_spectrum(a.tile_start, a.B, tile, kSearchOnly ? 0u : a.tiles_per_spec, a.inv_tiles_per_spec);
        prefetch_next_spectrum(a, s, tile);
        if (s != loaded_spec) {
            if (loaded_spec >= 0) __syncthreads();
            const int64_t no = a.per_spectrum_norm ? static_cast<int64_t>(s) * H : 0;
            for (int i = threadIdx.x; i < 2 * H; i += blockDim.x) {
                const int f = i / H, h = i - f * H;
                // select the pointers, not the parameter struct (indexing it would copy it to local memory)
                const float *sg = f ? a.g.sigma : a.s.sigma;
                const float *mu = f ? a.g.mu : a.s.mu;
                if ((FORMS >> f) & 1) {
                    const float rs = __frcp_rn(__ldg(sg + no + h));
                    tab[h][f] = make_float2(rs, __fmul_rn(__ldg(mu + no + h), rs));
                }
            }
            __syncthreads();
            loaded_spec = s;
        }
        const int64_t nf = __ldg(a.nf_main + s);
        const int64_t n0 = (tile - __ldg(a.tile_start + s)) * (CH * fpp) + li;
        const T *x = static_cast<const T *>(a.x) + __ldg(a.in_off + s);
        const float *wv = a.w;
        // spectra hold fewer than 2^31 bins: every index of the spectrum fits in 32 bits.  A
        // fundamental past the end of the spectrum runs the chain of fundamental 0 (reads in range)
        // and writes nothing.
        uint32_t n32[CH], hn[CH], d[CH], bits[CH];
        float S[CH];
        RunMax rm[CH];
#pragma unroll
        for (int c = 0; c < CH; ++c) {
            const int64_t n = n0 + static_cast<int64_t>(c) * fpp;
            const bool valid = n < nf;
            if (a.checked && valid && static_cast<int64_t>(H) * n + H > __ldg(a.in_len + s) - 1)
                set_error(a.err, kErrBounds);
            n32[c] = valid ? static_cast<uint32_t>(n) : 0u;
            hn[c] = n32[c];
        }
        // order 1: the two lanes of a fundamental load in the same instruction, so bins of both
        // forms that share a 128-byte line cost one L2 request; a simple lane's second value is
        // its first (no load), so its comparison never increments
        float va[CH], vb[CH];
#pragma unroll
        for (int c = 0; c < CH; ++c) {
            va[c] = ld_x<T, WHITEN>(x, wv, n32[c]);
            vb[c] = pair1 ? ld_x<T, WHITEN>(x, wv, n32[c] + 1) : va[c];
        }
        float2 t = tab[0][role];
#pragma unroll
        for (int c = 0; c < CH; ++c) {
            const bool inc = vb[c] > va[c];
            S[c] = inc ? vb[c] : va[c];
            d[c] = inc ? 1u : 0u;
            bits[c] = d[c];
            rm[c].first(fmaf(S[c], t.x, -t.y));
        }
        for (int h = 2; h <= H; ++h) {
#pragma unroll
            for (int c = 0; c < CH; ++c) {
                hn[c] += n32[c];
                const uint32_t m = hn[c] + d[c];   // simple lanes: d stays 0
                va[c] = ld_x<T, WHITEN>(x, wv, m);
                vb[c] = greedy ? ld_x<T, WHITEN>(x, wv, m + 1) : va[c];
            }
            t = tab[h - 1][role];
#pragma unroll
            for (int c = 0; c < CH; ++c) {
                const bool inc = vb[c] > va[c];
                S[c] += inc ? vb[c] : va[c];
                d[c] += inc;
                bits[c] |= static_cast<uint32_t>(inc) << (h - 1);
                rm[c].step(fmaf(S[c], t.x, -t.y), h);
            }
        }
        unsigned long long key = 0ull;
        // the tile's offsets are read again rather than kept live through the order loop (the
        // loop then fits the 32 registers a thread has at full occupancy without spilling)
        const int64_t nf2 = ld_volatile_i64(a.nf_main + s);
        const int64_t n02 = (tile - ld_volatile_i64(a.tile_start + s)) * (CH * fpp) + li;
        const int64_t fbase2 = ld_volatile_i64(a.fund_off + s);
#pragma unroll
        for (int c = 0; c < CH; ++c) {
            const int64_t n = n02 + static_cast<int64_t>(c) * fpp;
            if (n < nf2) {
                const int64_t o = fbase2 + n;
                (greedy ? a.g.snr : a.s.snr)[o] = rm[c].best;
                (greedy ? a.g.best_h : a.s.best_h)[o] = static_cast<uint8_t>(rm[c].bh);
                if (greedy && a.g.path) store_path(a.g.path, a.path_bytes, o, bits[c]);
                const unsigned long long kk = argmax_key(rm[c].best, n);
                key = kk > key ? kk : key;
            }
        }
        if (a.s.argmax || a.g.argmax) {
            // per-form block maximum of the argmax key, then one atomicMax per form and CTA
#pragma unroll
            for (int o = kBoth ? 2 : 1; o < 32; o <<= 1) {
                const unsigned long long k2 = __shfl_xor_sync(0xffffffffu, key, o);
                key = k2 > key ? k2 : key;
            }
            if (lane < (kBoth ? 2 : 1)) red[role][warp] = key;
            __syncthreads();
            if (threadIdx.x < 2 && ((FORMS >> threadIdx.x) & 1)) {
                unsigned long long *dst = (threadIdx.x ? a.g.argmax : a.s.argmax);
                if (dst) {
                    unsigned long long mx = 0ull;
                    for (int i = 0; i < static_cast<int>(blockDim.x >> 5); ++i)
                        mx = red[threadIdx.x][i] > mx ? red[threadIdx.x][i] : mx;
                    if (mx != 0ull) {
                        wait_prior_grid();
                        argmax_update(dst + s, mx);
                    }
                }
            }
        }
        if (a.tile_counter) {
            __syncthreads();
            if (threadIdx.x == 0) s_tile = static_cast<long long>(atomicAdd(a.tile_counter, 1ull));
            __syncthreads();
            tile = s_tile;
        } else {
            tile += gridDim.x;
            if (tile < a.total_tiles) __syncthreads();
        }
    }
}

template <typename T, int CH>
static const void *fwd1d_pair_kernel_ch(int forms, int whitening)
{
    if (whitening) {
        switch (forms) {
        case 1: return reinterpret_cast<const void *>(&k_fwd1d_pair<T, 1, true, CH>);
        case 2: return reinterpret_cast<const void *>(&k_fwd1d_pair<T, 2, true, CH>);
        case 3: return reinterpret_cast<const void *>(&k_fwd1d_pair<T, 3, true, CH>);
        }
    } else {
        switch (forms) {
        case 1: return reinterpret_cast<const void *>(&k_fwd1d_pair<T, 1, false, CH>);
        case 2: return reinterpret_cast<const void *>(&k_fwd1d_pair<T, 2, false, CH>);
        case 3: return reinterpret_cast<const void *>(&k_fwd1d_pair<T, 3, false, CH>);
        }
    }
    return nullptr;
}

// kernel 6: one fundamental per lane; kernel 7: two, interleaved
template <typename T>
static const void *fwd1d_pair_kernel_for(int forms, int whitening, int kernel)
{
    return kernel == 6 ? fwd1d_pair_kernel_ch<T, 1>(forms, whitening) : fwd1d_pair_kernel_ch<T, 2>(forms, whitening);
}

}  // namespace hs
