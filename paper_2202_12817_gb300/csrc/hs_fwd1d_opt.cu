// Optimal partial sums of the 1D harmonic sum (HS_FORM_OPTIMAL): for every fundamental n and
// order h, S*_h[n] = max over monotone drift paths of sum_{k<=h} x[k n + D_k], with
// D_k - D_{k-1} in {0, 1}, D_0 = 0 and D_1 = 0 without scalloping-loss mitigation -- the
// "optimal partial sum" over the bin choices the greedy form (Eq. 5 / Algorithm 2) makes
// one order at a time (Sec. 2.2, Sec. 3).  The SNR, its maximum over h (Eq. 2) and the best h
// follow as for the other forms; the path reported is an optimal path of the best h.
//
// Dynamic programme over the drift, one warp per fundamental: lane d holds
//   best[h][d] = x[h n + d] + max(best[h-1][d], best[h-1][d-1]),
// for d = 0..31 (lane 31 also holds d = 32, reachable only at order 32 with mitigation).
// Each order's reads x[h n .. h n + h] are consecutive (one coalesced load) and do not depend
// on the programme's state, so they are issued ahead of the arithmetic.  Ties keep the drift
// (no increment), and among equal optima at the best h the lowest drift is reported.
#include "hs_fwd1d.cuh"

namespace hs {

template <typename T, bool WHITEN>
__global__ void __launch_bounds__(256) k_fwd1d_opt(const Fwd1DArgs a, const FormArgs o, int64_t F, int64_t chunk)
{
    __shared__ int tab_spec[8];           // spectrum whose table each warp last loaded
    __shared__ float2 wtab[8][kMaxH1D];   // per warp: (1/sigma, mu/sigma) of that spectrum
    const int H = a.H;
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
            if (s >= 0 && o.argmax && lane == 0 && kmax != 0ull) atomicMax(o.argmax + s, kmax);
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
        if (n >= __ldg(a.nf_main + s)) {
            const int64_t lim = (__ldg(a.in_len + s) - 1) / (n + 1);
            Hn = static_cast<int>(lim < H ? lim : H);
        }
        if (a.checked && lane == 0 && static_cast<int64_t>(Hn) * n + Hn > __ldg(a.in_len + s) - 1)
            set_error(a.err, kErrBounds);
        const uint32_t n32 = static_cast<uint32_t>(n);
        const float *wv = a.w;
        // order 1: drift 0, or 1 with mitigation
        const int dmax1 = mit ? 1 : 0;
        float best = lane <= dmax1 ? ld_x<T, WHITEN>(x, wv, n32 + lane) : NEG;
        uint32_t bits = 0;                       // lane d: increments chosen into state d, bit h-1
        float b32 = NEG;                         // lane 31: state d = 32 (order 32 with mitigation)
        unsigned int cu = ordered_bits(best);
        unsigned int m = __reduce_max_sync(0xffffffffu, cu);
        uint32_t win = __ballot_sync(0xffffffffu, cu == m);
        float2 t = wtab[warp][0];
        float bsnr = fmaf(__uint_as_float((m & 0x80000000u) ? (m & 0x7fffffffu) : ~m), t.x, -t.y);
        int bh = 1, bd = __ffs(win) - 1;
        int dmax = dmax1;
        uint32_t hn = n32;
        // the values of the next PF orders, loaded ahead (the reads do not depend on the
        // programme); lane d of order k reads x[k n + d] when drift d is reachable at order k
        constexpr int PF = 4;
        float q[PF];
#pragma unroll
        for (int j = 0; j < PF; ++j) {
            const int k = 2 + j, dk = dmax1 + 1 + j;
            q[j] = (k <= Hn && lane <= dk) ? ld_x<T, WHITEN>(x, wv, static_cast<uint32_t>(k) * n32 + lane) : NEG;
        }
        // drift 32 exists only at order 32 with mitigation: lane 31 loads it at the start
        const float v32 = (Hn == 32 && mit && lane == 31) ? ld_x<T, WHITEN>(x, wv, 32u * n32 + 32u) : NEG;
        for (int h = 2; h <= Hn; ++h) {
            hn += n32;
            const int dnew = dmax + 1;           // largest drift reachable at order h
            const float v = q[0];
#pragma unroll
            for (int j = 0; j + 1 < PF; ++j) q[j] = q[j + 1];
            {
                const int k = h + PF, dk = dnew + PF;   // order entering the queue
                q[PF - 1] = (k <= Hn && lane <= dk) ? ld_x<T, WHITEN>(x, wv, hn + static_cast<uint32_t>(PF) * n32 + lane)
                                                   : NEG;
            }
            float up = __shfl_up_sync(0xffffffffu, best, 1);
            if (lane == 0) up = NEG;
            const float stay = lane <= dmax ? best : NEG;
            const bool inc = up > stay;          // ties keep the drift
            const float take = inc ? up : stay;
            const float prev31 = best;
            best = (lane <= dnew && take != NEG) ? take + v : NEG;
            bits |= static_cast<uint32_t>(inc) << (h - 1);
            if (lane == 31 && dnew == 32) b32 = prev31 + v32;   // only predecessor: drift 31
            cu = ordered_bits(best);
            if (lane == 31 && dnew == 32) {
                const unsigned int c32 = ordered_bits(b32);
                cu = c32 > cu ? c32 : cu;
            }
            m = __reduce_max_sync(0xffffffffu, cu);
            t = wtab[warp][h - 1];
            const float sh = __uint_as_float((m & 0x80000000u) ? (m & 0x7fffffffu) : ~m);
            const float snr = fmaf(sh, t.x, -t.y);
            if (snr > bsnr) {
                bsnr = snr;
                bh = h;
                win = __ballot_sync(0xffffffffu, ordered_bits(best) == m);
                // lowest drift holding the optimum; drift 32 only when it alone does
                bd = win ? __ffs(win) - 1 : 32;
            }
            dmax = dnew;
        }
        // an optimal path of order bh: walk the recorded increments back from drift bd
        uint32_t path = 0;
        int d = bd;
        for (int k = bh; k >= 2; --k) {
            const uint32_t bk = __shfl_sync(0xffffffffu, bits, d & 31);
            const bool step = (d == 32) || ((bk >> (k - 1)) & 1u);
            if (step) {
                path |= 1u << (k - 1);
                --d;
            }
        }
        if (d == 1) path |= 1u;   // order 1 chose drift 1 (mitigation)
        if (lane == 0) {
            const int64_t oi = fb + n;
            o.snr[oi] = bsnr;
            o.best_h[oi] = static_cast<uint8_t>(bh);
            if (o.path) store_path(o.path, a.path_bytes, oi, path);
            const unsigned long long key = argmax_key(bsnr, n);
            kmax = key > kmax ? key : kmax;
        }
    }
    if (s >= 0 && o.argmax && lane == 0 && kmax != 0ull) atomicMax(o.argmax + s, kmax);
}

const void *fwd1d_opt_kernel(int dtype, int whitening)
{
    if (dtype == HS_F32) return whitening ? reinterpret_cast<const void *>(&k_fwd1d_opt<float, true>)
                                          : reinterpret_cast<const void *>(&k_fwd1d_opt<float, false>);
    if (dtype == HS_F16) return whitening ? reinterpret_cast<const void *>(&k_fwd1d_opt<__half, true>)
                                          : reinterpret_cast<const void *>(&k_fwd1d_opt<__half, false>);
    if (dtype == HS_BF16) return whitening ? reinterpret_cast<const void *>(&k_fwd1d_opt<__nv_bfloat16, true>)
                                           : reinterpret_cast<const void *>(&k_fwd1d_opt<__nv_bfloat16, false>);
    return nullptr;
}

}  // namespace hs
