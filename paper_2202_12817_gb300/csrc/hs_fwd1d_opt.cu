// Optimal partial sums of the 1D harmonic sum (HS_FORM_OPTIMAL): for every fundamental n and
// order h, S*_h[n] = max over monotone drift paths of sum_{k<=h} x[k n + D_k], with
// D_k - D_{k-1} in {0, 1}, D_0 = 0 and D_1 = 0 without scalloping-loss mitigation -- the
// best partial sum over the bin choices that the greedy form (Eq. 5 / Algorithm 2) makes one
// order at a time (Sec. 2.2, Sec. 3).  The SNR, its maximum over h (Eq. 2) and the best h
// follow as for the other forms; the path reported is an optimal path of the best h.
//
// Dynamic programme over the drift, one warp per fundamental: lane d holds
//   best[h][d] = x[h n + d] + max(best[h-1][d], best[h-1][d-1])
// and the path that reaches it, for d = 0..31 (lane 31 also holds d = 32, reachable only at
// order 32 with mitigation).  Each order's reads x[h n .. h n + h] are consecutive (one
// coalesced load) and do not depend on the programme's state, so they are issued ahead of the
// arithmetic.  Each lane keeps the running SNR maximum of its own state with its path; one warp
// reduction at the end gives the best h and drift, whose lane holds the path.  Ties keep the
// drift (no increment), and among the drifts whose SNR at the best h equals the maximum the
// lowest is reported.
#include "hs_fwd1d.cuh"

namespace hs {

// HC > 0: H = HC known at compile time and no truncated-tail fundamentals, so the orders are
// unrolled completely (no loop or bounds tests between orders); HC = 0: any H, tail included.
// H = 8 and 32 fit in 48 registers, so five CTAs share an SM; the others keep four.
template <typename T, bool WHITEN, int HC>
__global__ void __launch_bounds__(256, (HC == 8 || HC == 32) ? 5 : 4) k_fwd1d_opt(const Fwd1DArgs a, const FormArgs o, int64_t F, int64_t chunk)
{
    __shared__ int tab_spec[8];           // spectrum whose table each warp last loaded
    __shared__ float2 wtab[8][kMaxH1D];   // per warp: (1/sigma, mu/sigma) of that spectrum
    const int H = HC > 0 ? HC : a.H;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const bool mit = a.mitigation != 0;
    const float NEG = -INFINITY;
    if (lane == 0) tab_spec[warp] = -1;
    __syncwarp();
    const int64_t gw = static_cast<int64_t>(blockIdx.x) * (blockDim.x >> 5) + warp;
    int64_t i = gw * chunk;
    const int64_t iend = i + chunk < F ? i + chunk : F;
    int s = -1;
    int64_t fb = 0, fe = 0;
    unsigned long long kmax = 0ull;   // running argmax key of spectrum s
    for (; i < iend; ++i) {
        if (i >= fe) {
            // next spectrum: flush the argmax of the previous one, locate the new one
            if (s >= 0 && o.argmax && lane == 0 && kmax != 0ull) argmax_update(o.argmax + s, kmax);
            kmax = 0ull;
            int lo = 0, hi = a.B - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (__ldg(a.fund_off + mid) <= i) lo = mid;
                else hi = mid - 1;
            }
            s = lo;
            fb = __ldg(a.fund_off + s);
            fe = __ldg(a.fund_off + s + 1);
            if (tab_spec[warp] != s) {
                const int64_t no = a.per_spectrum_norm ? static_cast<int64_t>(s) * H : 0;
                if (lane < H) {
                    const float rs = __frcp_rn(__ldg(o.sigma + no + lane));
                    wtab[warp][lane] = make_float2(rs, __fmul_rn(__ldg(o.mu + no + lane), rs));
                }
                __syncwarp();
                if (lane == 0) tab_spec[warp] = s;
                __syncwarp();
            }
            if (i >= fe) continue;   // empty range (cannot happen: every spectrum has N_f >= 1)
        }
        const int64_t n = i - fb;
        const T *x = static_cast<const T *>(a.x) + __ldg(a.in_off + s);
        // orders of this fundamental: all H, or in the truncated tail those with h n + h <= N - 1
        int Hn = H;
        if (HC == 0 && n >= __ldg(a.nf_main + s)) {
            const int64_t lim = (__ldg(a.in_len + s) - 1) / (n + 1);
            Hn = static_cast<int>(lim < H ? lim : H);
        }
        if (a.checked && lane == 0 && static_cast<int64_t>(Hn) * n + Hn > __ldg(a.in_len + s) - 1)
            set_error(a.err, kErrBounds);
        const uint32_t n32 = static_cast<uint32_t>(n);
        const float *wv = a.w;
        // Lane d holds the best sum ending at drift d and the path reaching it (bit k-1 set:
        // increment at order k).  A state that no path reaches holds -inf: its bins are not
        // read (the queue below holds -inf there), so no state needs a separate validity test.
        // Order 1: drift 0, or drift 1 through the mitigation increment.
        const int dmax1 = mit ? 1 : 0;
        const int lk = lane + 1 - dmax1;         // first order at which drift `lane` is reachable
        float best = lane <= dmax1 ? ld_x<T, WHITEN>(x, wv, n32 + lane) : NEG;
        uint32_t pth = (mit && lane == 1) ? 1u : 0u;
        // Each lane keeps the running maximum over h of its own state's SNR (first strictly larger
        // wins) and the path that gave it; fl((S - mu)/sigma) = fma(S, rs, -murs) is monotone in
        // S, so the maximum over lanes at the end is the maximum over h of the SNR of S*_h.
        float2 t = wtab[warp][0];
        float lsnr = lane <= dmax1 ? fmaf(best, t.x, -t.y) : NEG;
        int lh = 1, ld = lane;
        uint32_t lpath = pth;
        uint32_t bit = 1u;                       // 1 << (h - 1)
        // the values of the next PF orders, loaded ahead (the reads do not depend on the
        // programme): at the start of the block of orders h0 .. h0 + PF - 1, q[j] holds order
        // h0 + j; lane d of order k reads x[k n + d] when drift d is reachable at order k
        constexpr int PF = WHITEN ? 8 : 10;   // whitening keeps the registers for w
        float q[PF];
#pragma unroll
        for (int j = 0; j < PF; ++j) {
            const int k = 2 + j;
            q[j] = (k <= Hn && k >= lk) ? ld_x<T, WHITEN>(x, wv, static_cast<uint32_t>(k) * n32 + lane) : NEG;
        }
        uint32_t kn = static_cast<uint32_t>(2 + PF) * n32;   // (order entering the queue) x n
        // order h: best[h][d] = x[h n + d] + max(best[h-1][d], best[h-1][d-1]); ties keep the drift
        auto order = [&](int h, float v) {
            bit <<= 1;
            const float up = __shfl_up_sync(0xffffffffu, best, 1);     // lane 0 reads its own: no increment
            const uint32_t upp = __shfl_up_sync(0xffffffffu, pth, 1);
            const bool inc = up > best;
            best = (inc ? up : best) + v;
            pth = inc ? (upp | bit) : pth;
            const float2 tt = wtab[warp][h - 1];
            const float snr = fmaf(best, tt.x, -tt.y);
            if (snr > lsnr) {
                lsnr = snr;
                lh = h;
                lpath = pth;
            }
        };
        // with mitigation, order 32 also reaches drift 32 (lane 31's second state): that order is
        // taken after the loop
        const bool peel = mit && Hn == 32;
        const int Hl = peel ? 31 : Hn;
        const float v32 = (peel && lane == 31) ? ld_x<T, WHITEN>(x, wv, 32u * n32 + 32u) : NEG;
        if constexpr (HC > 0) {
#pragma unroll
            for (int h = 2; h <= HC; ++h) {
                if (HC == 32 && h == 32 && peel) break;
                const int j = (h - 2) % PF;
                const float v = q[j];
                if (h + PF <= HC) q[j] = h + PF >= lk ? ld_x<T, WHITEN>(x, wv, kn + lane) : NEG;
                kn += n32;
                order(h, v);
            }
        } else {
            for (int h0 = 2; h0 <= Hl; h0 += PF) {
#pragma unroll
                for (int j = 0; j < PF; ++j) {
                    const int h = h0 + j;
                    if (h > Hl) break;
                    const float v = q[j];
                    const int k = h + PF;
                    q[j] = (k <= Hn && k >= lk) ? ld_x<T, WHITEN>(x, wv, kn + lane) : NEG;
                    kn += n32;
                    order(h, v);
                }
            }
        }
        if (peel) {
            const float prev = best;             // lane 31: best sum at drift 31 after order 31
            const uint32_t pprev = pth;
            order(32, q[(32 - 2) % PF]);         // the loop stopped at order 32 = h0 + (32 - 2) % PF
            t = wtab[warp][31];
            if (lane == 31) {                    // drift 32: its only predecessor is drift 31
                const float s32 = fmaf(prev + v32, t.x, -t.y);
                if (s32 > lsnr) {
                    lsnr = s32;
                    lh = 32;
                    ld = 32;
                    lpath = pprev | (1u << 31);
                }
            }
        }
        // the warp's maximum: largest SNR, then lowest h, then lowest drift; its lane holds the path
        unsigned long long key = (static_cast<unsigned long long>(ordered_bits(lsnr)) << 32) |
                                 (static_cast<unsigned long long>(63 - lh) << 6) | static_cast<unsigned long long>(63 - ld);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            const unsigned long long k2 = __shfl_xor_sync(0xffffffffu, key, off);
            key = k2 > key ? k2 : key;
        }
        const unsigned int kb = static_cast<unsigned int>(key >> 32);
        const float bsnr = __uint_as_float((kb & 0x80000000u) ? (kb & 0x7fffffffu) : ~kb);
        const int bh = 63 - static_cast<int>((key >> 6) & 63u);
        const int bd = 63 - static_cast<int>(key & 63u);
        const uint32_t path = __shfl_sync(0xffffffffu, lpath, bd & 31);
        if (lane == 0) {
            const int64_t oi = fb + n;
            o.snr[oi] = bsnr;
            o.best_h[oi] = static_cast<uint8_t>(bh);
            if (o.path) store_path(o.path, a.path_bytes, oi, path);
            const unsigned long long key = argmax_key(bsnr, n);
            kmax = key > kmax ? key : kmax;
        }
    }
    if (s >= 0 && o.argmax && lane == 0 && kmax != 0ull) argmax_update(o.argmax + s, kmax);
}

// H = 32 without the truncated tail: two consecutive fundamentals A = n and B = n + 1 of one
// spectrum per warp.  Up to order 15 a fundamental has at most 16 drift states, so orders 1..15
// run A on lanes 0-15 and B on lanes 16-31 (16-lane shuffles); orders 16..32 then run A and B in
// turn on the whole warp.  Orders keep one queue whose slot (k - 2) % PF holds order k: while
// the last orders of phase 1 free their slots, A's orders 16.. enter them in the same mapping,
// and while A's last orders free theirs, B's orders 16.. enter them shifted by R_B = 17 % PF, so
// each pair waits once for its first loads.  A fundamental without a partner in its spectrum
// runs as A with a copy of itself as B, whose outputs are not written.  Four CTAs per SM with a
// 12-order queue (233 us on the 2^23-bin spectrum, against 304 us one fundamental per warp); the
// register cap spills a little, which costs less than a shorter queue or a fifth CTA.
template <typename T, bool WHITEN>
__global__ void __launch_bounds__(256, 4) k_fwd1d_opt_pair(const Fwd1DArgs a, const FormArgs o, int64_t F, int64_t chunk)
{
    constexpr int H = 32, P1 = 15, PF = 12, RB = 17 % PF;
    // the queue's first fill (orders 2 .. PF + 1) must lie in phase 1, whose lanes read other bins
    static_assert(PF <= P1 - 1, "phase-1 queue reaches past order 15");
    __shared__ int tab_spec[8];
    __shared__ float2 wtab[8][kMaxH1D];
    // B's phase-1 states (lanes 16-31) wait here while A runs its orders 16..32
    __shared__ float sb_best[8][16], sb_lsnr[8][16];
    __shared__ uint32_t sb_pth[8][16], sb_lpath[8][16];
    __shared__ int sb_lh[8][16];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int half = lane >> 4, hl = lane & 15;
    const bool mit = a.mitigation != 0;
    const float NEG = -INFINITY;
    if (lane == 0) tab_spec[warp] = -1;
    __syncwarp();
    const int64_t gw = static_cast<int64_t>(blockIdx.x) * (blockDim.x >> 5) + warp;
    int64_t i = gw * chunk;
    const int64_t iend = i + chunk < F ? i + chunk : F;
    int s = -1;
    int64_t fb = 0, fe = 0;
    unsigned long long kmax = 0ull;
    const float *wv = a.w;
    const int dmax1 = mit ? 1 : 0;
    const int lk = lane + 1 - dmax1;      // phase 2: first order at which drift `lane` is reachable
    const int lkP = hl + 1 - dmax1;       // phase 1: the same for drift hl
    while (i < iend) {
        if (i >= fe) {
            if (s >= 0 && o.argmax && lane == 0 && kmax != 0ull) argmax_update(o.argmax + s, kmax);
            kmax = 0ull;
            int lo = 0, hi = a.B - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (__ldg(a.fund_off + mid) <= i) lo = mid;
                else hi = mid - 1;
            }
            s = lo;
            fb = __ldg(a.fund_off + s);
            fe = __ldg(a.fund_off + s + 1);
            if (tab_spec[warp] != s) {
                const int64_t no = a.per_spectrum_norm ? static_cast<int64_t>(s) * H : 0;
                const float rs = __frcp_rn(__ldg(o.sigma + no + lane));
                wtab[warp][lane] = make_float2(rs, __fmul_rn(__ldg(o.mu + no + lane), rs));
                __syncwarp();
                if (lane == 0) tab_spec[warp] = s;
                __syncwarp();
            }
        }
        const bool pairB = i + 1 < iend && i + 1 < fe;   // B is a real fundamental of this spectrum
        const int64_t n = i - fb;
        const T *x = static_cast<const T *>(a.x) + __ldg(a.in_off + s);
        if (a.checked && lane == 0 && static_cast<int64_t>(H) * (n + (pairB ? 1 : 0)) + H > __ldg(a.in_len + s) - 1)
            set_error(a.err, kErrBounds);
        const uint32_t nA = static_cast<uint32_t>(n), nB = pairB ? nA + 1 : nA;
        const uint32_t nP = half ? nB : nA;   // this lane's fundamental in phase 1

        // ---- phase 1: orders 1..15, A on lanes 0-15, B on lanes 16-31, drift hl
        float best = hl <= dmax1 ? ld_x<T, WHITEN>(x, wv, nP + hl) : NEG;
        uint32_t pth = (mit && hl == 1) ? 1u : 0u;
        float2 t = wtab[warp][0];
        float lsnr = hl <= dmax1 ? fmaf(best, t.x, -t.y) : NEG;
        int lh = 1, ld = lane;
        uint32_t lpath = pth;
        uint32_t bit = 1u;
        float q[PF];
#pragma unroll
        for (int j = 0; j < PF; ++j) {
            const int k = 2 + j;
            q[j] = k >= lkP ? ld_x<T, WHITEN>(x, wv, static_cast<uint32_t>(k) * nP + hl) : NEG;
        }
        auto step = [&](int h, float v, int width) {
            bit <<= 1;
            const float up = __shfl_up_sync(0xffffffffu, best, 1, width);   // a segment's first lane reads its own
            const uint32_t upp = __shfl_up_sync(0xffffffffu, pth, 1, width);
            const bool inc = up > best;
            best = (inc ? up : best) + v;
            pth = inc ? (upp | bit) : pth;
            const float2 tt = wtab[warp][h - 1];
            const float snr = fmaf(best, tt.x, -tt.y);
            if (snr > lsnr) {
                lsnr = snr;
                lh = h;
                lpath = pth;
            }
        };
#pragma unroll
        for (int h = 2; h <= P1; ++h) {
            const int j = (h - 2) % PF;
            const float v = q[j];
            const int k = h + PF;
            if (k <= P1) q[j] = k >= lkP ? ld_x<T, WHITEN>(x, wv, static_cast<uint32_t>(k) * nP + hl) : NEG;
            else q[j] = k >= lk ? ld_x<T, WHITEN>(x, wv, static_cast<uint32_t>(k) * nA + lane) : NEG;   // A's order k
            step(h, v, 16);
        }
        // B's phase-1 states wait in shared memory (drift = hl) until B's turn
        if (half) {
            sb_best[warp][hl] = best;
            sb_pth[warp][hl] = pth;
            sb_lsnr[warp][hl] = lsnr;
            sb_lh[warp][hl] = lh;
            sb_lpath[warp][hl] = lpath;
        }
        __syncwarp();

        // ---- phase 2: orders 16..32 of one fundamental on the whole warp, then its result
        auto phase2 = [&](uint32_t nF, bool isA, bool write) {
            const bool peel = mit;   // order 32 also reaches drift 32 (lane 31's second state)
            const float v32 = (peel && lane == 31) ? ld_x<T, WHITEN>(x, wv, 32u * nF + 32u) : NEG;
#pragma unroll
            for (int h = P1 + 1; h <= H; ++h) {
                const int j = (h - 2 + (isA ? 0 : RB)) % PF;
                const float v = q[j];
                const int k = h + PF;
                if (k <= H) q[j] = k >= lk ? ld_x<T, WHITEN>(x, wv, static_cast<uint32_t>(k) * nF + lane) : NEG;
                else if (isA) {
                    const int k2 = k - H + P1;   // B's orders 16 .. 25
                    q[j] = k2 >= lk ? ld_x<T, WHITEN>(x, wv, static_cast<uint32_t>(k2) * nB + lane) : NEG;
                }
                if (h == H && peel) {
                    const float prev = best;
                    const uint32_t pprev = pth;
                    step(H, v, 32);
                    const float2 tt = wtab[warp][H - 1];
                    if (lane == 31) {
                        const float s32 = fmaf(prev + v32, tt.x, -tt.y);
                        if (s32 > lsnr) {
                            lsnr = s32;
                            lh = H;
                            ld = 32;
                            lpath = pprev | (1u << 31);
                        }
                    }
                } else {
                    step(h, v, 32);
                }
            }
            unsigned long long key = (static_cast<unsigned long long>(ordered_bits(lsnr)) << 32) |
                                     (static_cast<unsigned long long>(63 - lh) << 6) |
                                     static_cast<unsigned long long>(63 - ld);
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                const unsigned long long k2 = __shfl_xor_sync(0xffffffffu, key, off);
                key = k2 > key ? k2 : key;
            }
            const unsigned int kb = static_cast<unsigned int>(key >> 32);
            const float bsnr = __uint_as_float((kb & 0x80000000u) ? (kb & 0x7fffffffu) : ~kb);
            const int bh = 63 - static_cast<int>((key >> 6) & 63u);
            const int bd = 63 - static_cast<int>(key & 63u);
            const uint32_t path = __shfl_sync(0xffffffffu, lpath, bd & 31);
            if (write && lane == 0) {
                const int64_t nn = static_cast<int64_t>(nF);
                const int64_t oi = fb + nn;
                o.snr[oi] = bsnr;
                o.best_h[oi] = static_cast<uint8_t>(bh);
                if (o.path) store_path(o.path, a.path_bytes, oi, path);
                const unsigned long long k3 = argmax_key(bsnr, nn);
                kmax = k3 > kmax ? k3 : kmax;
            }
        };
        // A: its phase-1 states stay on lanes 0-15; lanes 16-31 start unreachable
        if (half) {
            best = NEG;
            pth = 0u;
            lsnr = NEG;
            lh = 1;
            lpath = 0u;
        }
        ld = lane;
        phase2(nA, true, true);
        // B: its phase-1 states return to lanes 0-15
        best = half ? NEG : sb_best[warp][hl];
        pth = half ? 0u : sb_pth[warp][hl];
        lsnr = half ? NEG : sb_lsnr[warp][hl];
        lh = half ? 1 : sb_lh[warp][hl];
        lpath = half ? 0u : sb_lpath[warp][hl];
        ld = lane;
        bit = 1u << (P1 - 1);
        phase2(nB, false, pairB);
        __syncwarp();   // the next pair's B states may overwrite the slots
        i += pairB ? 2 : 1;
    }
    if (s >= 0 && o.argmax && lane == 0 && kmax != 0ull) argmax_update(o.argmax + s, kmax);
}

template <typename T, bool WHITEN>
static const void *opt_kernel_h(int H, int tail)
{
    if (!tail && H == 32) return reinterpret_cast<const void *>(&k_fwd1d_opt_pair<T, WHITEN>);
    if (!tail && H == 16) return reinterpret_cast<const void *>(&k_fwd1d_opt<T, WHITEN, 16>);
    if (!tail && H == 8) return reinterpret_cast<const void *>(&k_fwd1d_opt<T, WHITEN, 8>);
    return reinterpret_cast<const void *>(&k_fwd1d_opt<T, WHITEN, 0>);
}

const void *fwd1d_opt_kernel(int dtype, int whitening, int H, int tail)
{
    if (dtype == HS_F32) return whitening ? opt_kernel_h<float, true>(H, tail) : opt_kernel_h<float, false>(H, tail);
    if (dtype == HS_F16) return whitening ? opt_kernel_h<__half, true>(H, tail) : opt_kernel_h<__half, false>(H, tail);
    if (dtype == HS_BF16)
        return whitening ? opt_kernel_h<__nv_bfloat16, true>(H, tail) : opt_kernel_h<__nv_bfloat16, false>(H, tail);
    return nullptr;
}

}  // namespace hs
