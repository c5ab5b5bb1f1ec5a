// Truncated tail of the 1D forward (HS_FLAG_TRUNCATE_TAIL): fundamentals N_f <= n < N - 1.
#pragma once

#include <type_traits>

#include "hs_fwd1d.cuh"

namespace hs {

constexpr int kTailChains = 4;      // tail fundamentals per thread (a tile is kTailThreads x 4)
constexpr int kTailAhead = 8;       // the tail prefetches the spectrum this many places ahead
static_assert(kTailTile == kTailThreads * kTailChains, "host tail tiling and kernel chains disagree");

// ---------------------------------------------------------------------------------------
// The truncated tail (HS_FLAG_TRUNCATE_TAIL), fundamentals N_f <= n < N - 1 whose higher
// orders would read past the end of the spectrum.  Each form keeps the orders whose every
// possible read fits: simple h n <= N - 1, greedy h n + h <= N - 1 (drift at most h - 1 after
// order h - 1, plus the compared neighbour).  Two kinds of tile, run by one kernel
// (k_fwd1d_tail): below n1 = floor((N - 1) / 2) + 1 the orders that fit vary (tail_orders);
// from n1 on both forms keep order 1 only (tail_one_order).
// ---------------------------------------------------------------------------------------

// Generic tile `tile` (of the tail_tile_start numbering) of spectrum s: kTailThreads x
// kTailChains consecutive fundamentals N_f <= n < n1, both forms in one thread.  Most of them
// have a few orders only, so a thread's time is a short chain of dependent loads: each thread
// runs kTailChains fundamentals (n, n + 32, ...) interleaved order by order to keep that many
// chains in flight.  The tiles of spectrum s bring spectrum s - kTailAhead into L2, one share
// each.
template <typename T, int FORMS, bool WHITEN>
__device__ __forceinline__ void tail_orders(const Fwd1DArgs &a, const int s, const int64_t tile, NormSmem &nm,
                                            unsigned long long *red)
{
    constexpr int CH = kTailChains;
    constexpr bool kS = (FORMS & HS_FORM_SIMPLE) != 0;
    constexpr bool kG = (FORMS & HS_FORM_GREEDY) != 0;
    const int H = a.H;
    const int64_t t0 = __ldg(a.tail_tile_start + s), t1 = __ldg(a.tail_tile_start + s + 1);
    const int64_t fbase = __ldg(a.fund_off + s);
    const int64_t len = __ldg(a.in_len + s);
    // these fundamentals end at n1 = floor((N - 1) / 2) + 1 (or N - 1); from n1 on both forms keep
    // order 1 only (tail_one_order)
    const int64_t n_all = __ldg(a.fund_off + s + 1) - fbase, n1 = (len - 1) / 2 + 1;
    const int64_t nf = n_all < n1 ? n_all : n1;
    // warp w runs the 32 CH fundamentals [32 CH w, 32 CH (w + 1)) of the tile, chain c of lane l at 32 c + l, so a
    // thread's chains have nearly the same order counts
    const int64_t nbase = __ldg(a.nf_main + s) + (tile - t0) * (static_cast<int64_t>(blockDim.x) * CH) +
                          (threadIdx.x >> 5) * (32 * CH) + (threadIdx.x & 31);
    const T *x = static_cast<const T *>(a.x) + __ldg(a.in_off + s);
    const float *wv = a.w;
    RunMax ms[CH], mg[CH];
    uint32_t bits[CH], d[CH], n32[CH], hn[CH];
    float ss[CH], sg[CH];
    int Hs[CH], Hg[CH];
    int Hmax = 0;
#pragma unroll
    for (int c = 0; c < CH; ++c) {
        const int64_t n = nbase + static_cast<int64_t>(c) * 32;
        ms[c] = RunMax{0.f, 1};
        mg[c] = RunMax{0.f, 1};
        bits[c] = 0;
        d[c] = 0;
        // orders of each form (n >= N_f >= 1 here); a fundamental past N - 2 takes no orders
        const bool valid = n < nf;
        const int64_t hs_ = valid ? (len - 1) / n : 0, hg_ = valid ? (len - 1) / (n + 1) : 0;
        Hs[c] = kS ? static_cast<int>(hs_ < H ? hs_ : H) : 0;
        Hg[c] = kG ? static_cast<int>(hg_ < H ? hg_ : H) : 0;
        const int hm = Hs[c] > Hg[c] ? Hs[c] : Hg[c];
        Hmax = hm > Hmax ? hm : Hmax;
        n32[c] = valid ? static_cast<uint32_t>(n) : 0u;
        hn[c] = n32[c];
    }
    // order 1 of every chain is loaded before the normalisation table, so the two latencies overlap
    float x0[CH], x1[CH];
#pragma unroll
    for (int c = 0; c < CH; ++c) {
        x0[c] = Hg[c] > 0 || Hs[c] > 0 ? ld_x<T, WHITEN>(x, wv, n32[c]) : 0.f;
        x1[c] = (kG && a.mitigation && Hg[c] > 0) ? ld_x<T, WHITEN>(x, wv, n32[c] + 1) : x0[c];
    }
    const int64_t no = a.per_spectrum_norm ? static_cast<int64_t>(s) * H : 0;
    if (kS) load_norm(nm, 0, a.s.mu + no, a.s.sigma + no, H);
    if (kG) load_norm(nm, 1, a.g.mu + no, a.g.sigma + no, H);
    if (threadIdx.x == 0 && s >= kTailAhead) {
        // share (t1 - 1 - tile) of spectrum s - kTailAhead, in 16-byte units
        const int sp = s - kTailAhead;
        const int64_t nb = __ldg(a.in_len + sp) * a.elem_bytes, nt = t1 - t0;
        const int64_t chunk = ((nb + nt - 1) / nt + 15) & ~static_cast<int64_t>(15);
        int64_t lo = (t1 - 1 - tile) * chunk;
        const int64_t hi = lo + chunk < nb ? lo + chunk : nb;
        const unsigned char *src = static_cast<const unsigned char *>(a.x) + __ldg(a.in_off + sp) * a.elem_bytes;
        for (; lo + 16 <= hi; lo += 65536) {
            const int64_t b = (hi - lo < 65536 ? hi - lo : 65536) & ~static_cast<int64_t>(15);
            asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src + lo), "r"(static_cast<uint32_t>(b)) : "memory");
        }
    }
    __syncthreads();
#pragma unroll
    for (int c = 0; c < CH; ++c) {
        ss[c] = x0[c];
        sg[c] = x0[c];
        if (kG && x1[c] > x0[c]) {
            d[c] = 1;
            sg[c] = x1[c];
            bits[c] = 1u;
        }
        if (kS) ms[c].first(fmaf(ss[c], nm.rs[0][0], -nm.murs[0][0]));
        if (kG) mg[c].first(fmaf(sg[c], nm.rs[1][0], -nm.murs[1][0]));
    }
    for (int h = 2; h <= Hmax; ++h) {
        float vs[CH], va[CH], vb[CH];
#pragma unroll
        for (int c = 0; c < CH; ++c) {
            hn[c] += n32[c];
            if (kS && h <= Hs[c]) vs[c] = ld_x<T, WHITEN>(x, wv, hn[c]);
            if (kG && h <= Hg[c]) {
                va[c] = ld_x<T, WHITEN>(x, wv, hn[c] + d[c]);
                vb[c] = ld_x<T, WHITEN>(x, wv, hn[c] + d[c] + 1);
            }
        }
#pragma unroll
        for (int c = 0; c < CH; ++c) {
            if (kS && h <= Hs[c]) {
                ss[c] += vs[c];
                ms[c].step(fmaf(ss[c], nm.rs[0][h - 1], -nm.murs[0][h - 1]), h);
            }
            if (kG && h <= Hg[c]) {
                const bool inc = vb[c] > va[c];
                sg[c] += inc ? vb[c] : va[c];
                d[c] += inc;
                bits[c] |= static_cast<uint32_t>(inc) << (h - 1);
                mg[c].step(fmaf(sg[c], nm.rs[1][h - 1], -nm.murs[1][h - 1]), h);
            }
        }
    }
    unsigned long long ks = 0ull, kg = 0ull;
#pragma unroll
    for (int c = 0; c < CH; ++c) {
        const int64_t n = nbase + static_cast<int64_t>(c) * 32;
        if (n >= nf) continue;
        const int64_t o = fbase + n;
        if (kS) {
            a.s.snr[o] = ms[c].best;
            a.s.best_h[o] = static_cast<uint8_t>(ms[c].bh);
            const unsigned long long k = argmax_key(ms[c].best, n);
            ks = k > ks ? k : ks;
        }
        if (kG) {
            a.g.snr[o] = mg[c].best;
            a.g.best_h[o] = static_cast<uint8_t>(mg[c].bh);
            if (a.g.path) store_path(a.g.path, a.path_bytes, o, bits[c]);
            const unsigned long long k = argmax_key(mg[c].best, n);
            kg = k > kg ? k : kg;
        }
    }
    if (kS && a.s.argmax) block_argmax(ks, a.s.argmax + s, red);
    if (kG && a.g.argmax) {
        if (kS && a.s.argmax) __syncthreads();
        block_argmax(kg, a.g.argmax + s, red);
    }
}

// One-order tiles: max(n1, N_f) <= n < N - 1 with n1 = floor((N - 1) / 2) + 1, where h n > N - 1
// for h >= 2, so both forms keep order 1 only (greedy: its mitigation comparison of x[n] and
// x[n + 1]).  The same steps as tail_orders' order 1, streamed: kTail1Tile consecutive
// fundamentals of one spectrum in rounds of kTailThreads x kTail1Chains, each round's loads
// issued before the previous round's stores, so one DRAM latency per round overlaps the other's
// work; coalesced loads and stores, one argmax update per form and CTA.
constexpr int kTail1Chains = 4;     // one-order fundamentals per thread and round
constexpr int kTail1Rounds = kTail1Tile / (kTailThreads * kTail1Chains);
static_assert(kTail1Rounds * kTailThreads * kTail1Chains == kTail1Tile, "one-order tile and rounds disagree");

// One round's loads: x[n] and, for the greedy mitigation, x[n + 1] of the thread's fundamentals.
template <typename T, bool WHITEN, bool MIT>
__device__ __forceinline__ void tail1_load(const T *x, const float *wv, uint32_t nb, uint32_t nf, float (&x0)[kTail1Chains],
                                           float (&x1)[kTail1Chains])
{
#pragma unroll
    for (int c = 0; c < kTail1Chains; ++c) {
        const uint32_t n = nb + c * kTailThreads;
        const uint32_t nl = n < nf ? n : 0u;
        x0[c] = n < nf ? ld_x<T, WHITEN>(x, wv, nl) : 0.f;
        x1[c] = MIT && n < nf ? ld_x<T, WHITEN>(x, wv, nl + 1) : x0[c];
    }
}

// One-order tile `tile` (of the tail1_tile_start numbering) of spectrum s.
template <typename T, int FORMS, bool WHITEN>
__device__ __forceinline__ void tail_one_order(const Fwd1DArgs &a, const int s, const int64_t tile,
                                               unsigned long long *red)
{
    constexpr int CH = kTail1Chains;
    constexpr bool kS = (FORMS & HS_FORM_SIMPLE) != 0;
    constexpr bool kG = (FORMS & HS_FORM_GREEDY) != 0;
    const int H = a.H;
    const int64_t t0 = __ldg(a.tail1_tile_start + s);
    const int64_t fbase = __ldg(a.fund_off + s);
    const int64_t len = __ldg(a.in_len + s);
    // N < 2^31, so every bin index of the spectrum fits in 32 bits
    const uint32_t nf = static_cast<uint32_t>(len - 1);   // N - 1
    const uint32_t n1 = static_cast<uint32_t>((len - 1) / 2 + 1), nm = static_cast<uint32_t>(__ldg(a.nf_main + s));
    const uint32_t nbase = (n1 > nm ? n1 : nm) + static_cast<uint32_t>(tile - t0) * kTail1Tile + threadIdx.x;
    const T *x = static_cast<const T *>(a.x) + __ldg(a.in_off + s);
    const float *wv = a.w;
    // order 1's normalisation, formed as the other kernels form it (1/sigma rounded, mu/sigma as mu * that)
    const int64_t no = a.per_spectrum_norm ? static_cast<int64_t>(s) * H : 0;
    float rs_s = 0.f, mr_s = 0.f, rs_g = 0.f, mr_g = 0.f;
    if (kS) {
        rs_s = __frcp_rn(__ldg(a.s.sigma + no));
        mr_s = __fmul_rn(__ldg(a.s.mu + no), rs_s);
    }
    if (kG) {
        rs_g = __frcp_rn(__ldg(a.g.sigma + no));
        mr_g = __fmul_rn(__ldg(a.g.mu + no), rs_g);
    }
    float *snr_s = kS ? a.s.snr + fbase : nullptr;
    float *snr_g = kG ? a.g.snr + fbase : nullptr;
    uint8_t *bh_s = kS ? a.s.best_h + fbase : nullptr;
    uint8_t *bh_g = kG ? a.g.best_h + fbase : nullptr;
    const int pb = kG && a.g.path ? a.path_bytes : 0;
    unsigned char *pth = pb ? static_cast<unsigned char *>(a.g.path) + fbase * pb : nullptr;
    // per-thread argmax as (ordered SNR bits, bin): a thread's bins ascend, so a strictly larger
    // value replaces and equal values keep the lower bin, as the 64-bit key order does
    uint32_t os = 0u, og = 0u, bs = 0xffffffffu, bg = 0xffffffffu;
    const auto body = [&](uint32_t nb, const float (&x0)[CH], const float (&x1)[CH]) {
#pragma unroll
        for (int c = 0; c < CH; ++c) {
            const uint32_t n = nb + c * kTailThreads;
            if (n >= nf) continue;
            const float v0 = x0[c], v1 = x1[c];
            if (kS) {
                const float snr = fmaf(v0, rs_s, -mr_s);
                snr_s[n] = snr;
                bh_s[n] = 1;
                const uint32_t o = ordered_bits(snr);
                if (bs == 0xffffffffu || o > os) { os = o; bs = n; }
            }
            if (kG) {
                const bool inc = v1 > v0;
                const float snr = fmaf(inc ? v1 : v0, rs_g, -mr_g);
                snr_g[n] = snr;
                bh_g[n] = 1;
                if (pb == 4) reinterpret_cast<uint32_t *>(pth)[n] = inc ? 1u : 0u;
                else if (pb == 2) reinterpret_cast<uint16_t *>(pth)[n] = inc ? 1u : 0u;
                else if (pb == 1) pth[n] = inc ? 1u : 0u;
                const uint32_t o = ordered_bits(snr);
                if (bg == 0xffffffffu || o > og) { og = o; bg = n; }
            }
        }
    };
    // rounds alternate between two register sets: round r + 1's loads go out before round r's stores
    const auto rounds = [&](auto mit) {
        constexpr bool M = decltype(mit)::value;
        constexpr uint32_t R = kTailThreads * CH;
        float xa0[CH], xa1[CH], xb0[CH], xb1[CH];
        tail1_load<T, WHITEN, M>(x, wv, nbase, nf, xa0, xa1);
#pragma unroll
        for (int r = 0; r < kTail1Rounds; r += 2) {
            const uint32_t nb = nbase + r * R;
            if (r + 1 < kTail1Rounds) tail1_load<T, WHITEN, M>(x, wv, nb + R, nf, xb0, xb1);
            body(nb, xa0, xa1);
            if (r + 1 < kTail1Rounds) {
                if (r + 2 < kTail1Rounds) tail1_load<T, WHITEN, M>(x, wv, nb + 2 * R, nf, xa0, xa1);
                body(nb + R, xb0, xb1);
            }
        }
    };
    if (kG && a.mitigation) rounds(std::true_type{});
    else rounds(std::false_type{});
    const unsigned long long ks = bs == 0xffffffffu ? 0ull : (static_cast<unsigned long long>(os) << 32) | (0xffffffffu - bs);
    const unsigned long long kg = bg == 0xffffffffu ? 0ull : (static_cast<unsigned long long>(og) << 32) | (0xffffffffu - bg);
    if (kS && a.s.argmax) block_argmax(ks, a.s.argmax + s, red);
    if (kG && a.g.argmax) {
        if (kS && a.s.argmax) __syncthreads();
        block_argmax(kg, a.g.argmax + s, red);
    }
}

// ---------------------------------------------------------------------------------------
// kernel: the whole truncated tail in one launch.  Spectrum s owns T_s = G_s + O_s consecutive
// CTAs of the launch, its G_s generic tiles followed by its O_s one-order tiles; the CTAs run
// from the last spectrum down (the main pass that precedes this kernel leaves the last spectra
// in L2), and within a spectrum the one-order tiles, which stream, start with the generic ones,
// whose chains of gathers are latency-bound, and read the same lines of the spectrum.
// ---------------------------------------------------------------------------------------
template <typename T, int FORMS, bool WHITEN>
__global__ void __launch_bounds__(kTailThreads) k_fwd1d_tail(const Fwd1DArgs a)
{
    __shared__ NormSmem nm;
    __shared__ unsigned long long red[32];
    const int64_t q = a.tail_tiles + a.tail1_tiles - 1 - static_cast<int64_t>(blockIdx.x);
    // the spectrum whose CTAs hold q: by a division when every spectrum has the same tile counts,
    // else a binary search over the summed prefixes
    const unsigned per = a.tail_tiles_per_spec + a.tail1_tiles_per_spec;
    int s = 0;
    int64_t c0 = 0;
    if (a.B > 1) {
        if (per > 0) {
            const unsigned u = static_cast<unsigned>(q) / per;
            s = u < static_cast<unsigned>(a.B) ? static_cast<int>(u) : a.B - 1;
            c0 = static_cast<int64_t>(s) * per;
        } else {
            int lo = 0, hi = a.B - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (__ldg(a.tail_tile_start + mid) + __ldg(a.tail1_tile_start + mid) <= q) lo = mid;
                else hi = mid - 1;
            }
            s = lo;
            c0 = __ldg(a.tail_tile_start + s) + __ldg(a.tail1_tile_start + s);
        }
    }
    const int64_t g0 = __ldg(a.tail_tile_start + s), gn = __ldg(a.tail_tile_start + s + 1) - g0;
    const int64_t j = q - c0;
    if (j < gn) tail_orders<T, FORMS, WHITEN>(a, s, g0 + j, nm, red);
    else tail_one_order<T, FORMS, WHITEN>(a, s, __ldg(a.tail1_tile_start + s) + (j - gn), red);
}

template <typename T>
static const void *fwd1d_tail_kernel_for(int forms, int whitening)
{
    if (whitening) {
        switch (forms) {
        case 1: return reinterpret_cast<const void *>(&k_fwd1d_tail<T, 1, true>);
        case 2: return reinterpret_cast<const void *>(&k_fwd1d_tail<T, 2, true>);
        case 3: return reinterpret_cast<const void *>(&k_fwd1d_tail<T, 3, true>);
        }
    } else {
        switch (forms) {
        case 1: return reinterpret_cast<const void *>(&k_fwd1d_tail<T, 1, false>);
        case 2: return reinterpret_cast<const void *>(&k_fwd1d_tail<T, 2, false>);
        case 3: return reinterpret_cast<const void *>(&k_fwd1d_tail<T, 3, false>);
        }
    }
    return nullptr;
}

}  // namespace hs
