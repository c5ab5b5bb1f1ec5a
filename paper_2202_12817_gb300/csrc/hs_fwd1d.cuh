// 1D forward harmonic-sum kernels (simple form, Eq. 3; greedy form, Eq. 5 / Algorithm 2),
// templated on the stored type, the forms computed in one pass and whitening.  Included by
// one translation unit per stored type.
#pragma once

#include "hs_internal.cuh"

namespace hs {

// ---------------------------------------------------------------------------------------
// loads
// ---------------------------------------------------------------------------------------
template <typename T, typename I>
__device__ __forceinline__ float ld_raw(const T *p, I j);

template <>
__device__ __forceinline__ float ld_raw<float, int64_t>(const float *p, int64_t j)
{
    return __ldg(p + j);
}
template <>
__device__ __forceinline__ float ld_raw<float, uint32_t>(const float *p, uint32_t j)
{
    return __ldg(p + j);
}
template <typename I>
__device__ __forceinline__ float ld_half_bits(const __half *p, I j)
{
    unsigned short b = __ldg(reinterpret_cast<const unsigned short *>(p) + j);
    return __half2float(__ushort_as_half(b));
}
template <typename I>
__device__ __forceinline__ float ld_bf16_bits(const __nv_bfloat16 *p, I j)
{
    unsigned short b = __ldg(reinterpret_cast<const unsigned short *>(p) + j);
    return __uint_as_float(static_cast<unsigned int>(b) << 16);
}
template <>
__device__ __forceinline__ float ld_raw<__half, int64_t>(const __half *p, int64_t j) { return ld_half_bits(p, j); }
template <>
__device__ __forceinline__ float ld_raw<__half, uint32_t>(const __half *p, uint32_t j) { return ld_half_bits(p, j); }
template <>
__device__ __forceinline__ float ld_raw<__nv_bfloat16, int64_t>(const __nv_bfloat16 *p, int64_t j)
{
    return ld_bf16_bits(p, j);
}
template <>
__device__ __forceinline__ float ld_raw<__nv_bfloat16, uint32_t>(const __nv_bfloat16 *p, uint32_t j)
{
    return ld_bf16_bits(p, j);
}

// Loaded power x[j]: the stored value, or fl32(w[j] * p[j]) with whitening.
template <typename T, bool WHITEN, typename I>
__device__ __forceinline__ float ld_x(const T *p, const float *w, I j)
{
    float v = ld_raw<T, I>(p, j);
    if constexpr (WHITEN) v = __fmul_rn(__ldg(w + j), v);
    return v;
}

// ordered-float key: larger float -> larger unsigned
__device__ __forceinline__ unsigned int ordered_bits(float f)
{
    unsigned int u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

__device__ __forceinline__ unsigned long long argmax_key(float snr, int64_t n)
{
    return (static_cast<unsigned long long>(ordered_bits(snr)) << 32) |
           static_cast<unsigned long long>(0xffffffffu - static_cast<unsigned int>(n));
}

__device__ __forceinline__ void set_error(int *err, int code)
{
    if (err) atomicCAS(err, kErrNone, code);
}

// Programmatic dependent launch: a 1D pass launched right after k_fwd_reset may start while that
// kernel still clears the argmax keys and the tile counter; every access to those waits here
// first.  Returns at once when the kernel was launched without the attribute or the reset is done.
__device__ __forceinline__ void wait_prior_grid() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// atomicMax of a per-spectrum argmax key, skipped when the key already stored is at least as
// large: keys only grow during a pass, so a smaller or equal key can never win, and on a spectrum
// of thousands of CTAs only the few that raise the running maximum reach the L2 atomic unit (the
// others would serialise there on one address).  Called after wait_prior_grid().
__device__ __forceinline__ void argmax_update(unsigned long long *dst, unsigned long long key)
{
    const unsigned long long cur = *reinterpret_cast<volatile unsigned long long *>(dst);
    if (key > cur) atomicMax(dst, key);
}

// Block-wide max of a 64-bit key, then one atomicMax per CTA.
__device__ __forceinline__ void block_argmax(unsigned long long key, unsigned long long *dst,
                                             unsigned long long *scratch /*[32] smem*/)
{
    for (int o = 16; o > 0; o >>= 1) {
        unsigned long long k2 = __shfl_xor_sync(0xffffffffu, key, o);
        key = k2 > key ? k2 : key;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) scratch[warp] = key;
    __syncthreads();
    if (warp == 0) {
        const int nw = (blockDim.x + 31) >> 5;
        key = lane < nw ? scratch[lane] : 0ull;
        for (int o = 16; o > 0; o >>= 1) {
            unsigned long long k2 = __shfl_xor_sync(0xffffffffu, key, o);
            key = k2 > key ? k2 : key;
        }
        if (lane == 0 && key != 0ull) {
            wait_prior_grid();
            argmax_update(dst, key);
        }
    }
}

// Next-spectrum L2 prefetch: tile i of the T_s tiles of spectrum s brings share i of spectrum
// s+1's input bytes into L2 (cp.async.bulk.prefetch, 16-byte units), so that when spectrum s+1's
// tiles start, their dependent chains of gathers hit L2 instead of DRAM.
__device__ __forceinline__ void prefetch_next_spectrum(const Fwd1DArgs &a, int s, int64_t tile)
{
    if (!a.pf_next || threadIdx.x != 0 || s + 1 >= a.B) return;
    const int64_t t0 = __ldg(a.tile_start + s), nt = __ldg(a.tile_start + s + 1) - t0;
    const int64_t nb = __ldg(a.in_len + s + 1) * a.elem_bytes;
    const int64_t chunk = ((nb + nt - 1) / nt + 15) & ~static_cast<int64_t>(15);
    int64_t lo = (tile - t0) * chunk;
    const int64_t hi = lo + chunk < nb ? lo + chunk : nb;
    const unsigned char *src = static_cast<const unsigned char *>(a.x) + __ldg(a.in_off + s + 1) * a.elem_bytes;
    for (; lo + 16 <= hi; lo += 65536) {
        const int64_t b = (hi - lo < 65536 ? hi - lo : 65536) & ~static_cast<int64_t>(15);
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src + lo), "r"(static_cast<uint32_t>(b)) : "memory");
    }
}

// spectrum owning a tile: largest s with tile_start[s] <= t.  `per` > 0: every spectrum has that
// many tiles (a plan whose spectra all have one length; the host passes it below 2^22 tiles, with
// inv = fl(1/per)), so it is x / per for x = t - tile_start[0] (tile_start[0] is 0, or minus a
// chunk's first tile): a single-precision estimate, within one of x / per there, and an exact
// integer correction.  Otherwise a binary search, a chain of log2 B dependent loads.
__device__ __forceinline__ int tile_spectrum(const int64_t *tile_start, int B, int64_t t, unsigned per, float inv)
{
    if (B == 1) return 0;
    if (per > 0) {
        const unsigned x = static_cast<unsigned>(t - __ldg(tile_start));
        unsigned g = __float2uint_rz(__uint2float_rn(x) * inv);
        if (g * per > x) --g;
        else if ((g + 1) * per <= x) ++g;
        return g < static_cast<unsigned>(B) ? static_cast<int>(g) : B - 1;
    }
    int lo = 0, hi = B - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (__ldg(tile_start + mid) <= t) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Normalisation table in shared memory: rs = 1/sigma, murs = mu * rs, so that
// SNR = S * rs - murs (one FMA); error relative to (|S| + |mu|) / sigma stays ~3 ulp.
struct NormSmem {
    float rs[2][kMaxH1D];
    float murs[2][kMaxH1D];
};

__device__ __forceinline__ void load_norm(NormSmem &nm, int slot, const float *mu, const float *sigma,
                                          int H)
{
    for (int h = threadIdx.x; h < H; h += blockDim.x) {
        float rs = __frcp_rn(__ldg(sigma + h));
        nm.rs[slot][h] = rs;
        nm.murs[slot][h] = __fmul_rn(__ldg(mu + h), rs);
    }
}

__device__ __forceinline__ void store_path(void *path, int bytes, int64_t i, uint32_t bits)
{
    if (bytes == 4) static_cast<uint32_t *>(path)[i] = bits;
    else if (bytes == 2) static_cast<uint16_t *>(path)[i] = static_cast<uint16_t>(bits);
    else if (bytes == 1) static_cast<uint8_t *>(path)[i] = static_cast<uint8_t>(bits);
}

// One running SNR maximum (Eq. 2): start at h = 1, strictly larger replaces.
struct RunMax {
    float best;
    int bh;
    __device__ __forceinline__ void first(float snr) { best = snr; bh = 1; }
    __device__ __forceinline__ void step(float snr, int h)
    {
        if (snr > best) { best = snr; bh = h; }
    }
};

// ---------------------------------------------------------------------------------------
// greedy candidate selection for the look-ahead kernel
// ---------------------------------------------------------------------------------------
template <int J>
__device__ __forceinline__ float pick(const float (&v)[J], int r)
{
    float out = v[0];
#pragma unroll
    for (int i = 1; i < J; ++i) out = (r == i) ? v[i] : out;
    return out;
}

// ---------------------------------------------------------------------------------------
// kernel: one thread per fundamental, tiles of blockDim.x fundamentals.
//   LOOKAHEAD = 1: every order loads its two candidates after the previous comparison
//                  (a chain of H dependent loads per fundamental);
//   LOOKAHEAD = G > 1: with the drift d known before order h0, all candidates of orders
//                  h0..h0+G-1 ((h0+j) n + d + [0, j+1]) are loaded at once and the G
//                  comparisons run from registers: H/G dependent rounds.
// ---------------------------------------------------------------------------------------
template <typename T, int FORMS, bool WHITEN, int LOOKAHEAD>
__global__ void __launch_bounds__(256) k_fwd1d(const Fwd1DArgs a)
{
    __shared__ NormSmem nm;
    __shared__ unsigned long long red[32];
    __shared__ long long s_tile;
    constexpr bool kS = (FORMS & HS_FORM_SIMPLE) != 0;
    constexpr bool kG = (FORMS & HS_FORM_GREEDY) != 0;
    const int H = a.H;
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
        const int s = tile_spectrum(a.tile_start, a.B, tile, a.tiles_per_spec, a.inv_tiles_per_spec);
        prefetch_next_spectrum(a, s, tile);
        if (s != loaded_spec) {
            if (loaded_spec >= 0) __syncthreads();
            const int64_t no = a.per_spectrum_norm ? static_cast<int64_t>(s) * H : 0;
            if (kS) load_norm(nm, 0, a.s.mu + no, a.s.sigma + no, H);
            if (kG) load_norm(nm, 1, a.g.mu + no, a.g.sigma + no, H);
            __syncthreads();
            loaded_spec = s;
        }
        const int64_t fbase = __ldg(a.fund_off + s);
        const int64_t nf = __ldg(a.nf_main + s);
        const int64_t n = (tile - __ldg(a.tile_start + s)) * blockDim.x + threadIdx.x;
        const bool valid = n < nf;
        const T *x = static_cast<const T *>(a.x) + __ldg(a.in_off + s);
        if (a.checked && valid) {
            // every read of both forms lies in [0, H n + H]; checked mode verifies the domain
            const int64_t len = __ldg(a.in_len + s);
            if (static_cast<int64_t>(H) * n + H > len - 1) set_error(a.err, kErrBounds);
        }
        RunMax ms{0.f, 1}, mg{0.f, 1};
        uint32_t bits = 0;
        if (valid) {
            // spectra hold fewer than 2^31 bins, so every index of the spectrum fits in 32 bits
            const uint32_t n32 = static_cast<uint32_t>(n);
            const float *wv = a.w;
            // ---- order 1 ----
            const float x0 = ld_x<T, WHITEN>(x, wv, n32);
            float ss = x0, sg = x0;
            uint32_t d = 0;
            if (kG && a.mitigation) {
                const float b = ld_x<T, WHITEN>(x, wv, n32 + 1);
                if (b > x0) { d = 1; sg = b; bits = 1u; }
            }
            if (kS) ms.first(fmaf(ss, nm.rs[0][0], -nm.murs[0][0]));
            if (kG) mg.first(fmaf(sg, nm.rs[1][0], -nm.murs[1][0]));
            uint32_t hn = n32;            // h n, stepped by n per order
            if constexpr (LOOKAHEAD <= 1) {
                for (int h = 2; h <= H; ++h) {
                    hn += n32;
                    if (kS) {
                        ss += ld_x<T, WHITEN>(x, wv, hn);
                        ms.step(fmaf(ss, nm.rs[0][h - 1], -nm.murs[0][h - 1]), h);
                    }
                    if (kG) {
                        const uint32_t m = hn + d;
                        const float va = ld_x<T, WHITEN>(x, wv, m);
                        const float vb = ld_x<T, WHITEN>(x, wv, m + 1);
                        const bool inc = vb > va;
                        sg += inc ? vb : va;
                        d += inc;
                        bits |= static_cast<uint32_t>(inc) << (h - 1);
                        mg.step(fmaf(sg, nm.rs[1][h - 1], -nm.murs[1][h - 1]), h);
                    }
                }
            } else {
                constexpr int G = LOOKAHEAD;
                for (int h0 = 2; h0 <= H; h0 += G) {
                    float sv[G];
                    float v[G][G + 1];
                    // issue every load of the group before any comparison
#pragma unroll
                    for (int j = 0; j < G; ++j) {
                        const int h = h0 + j;
                        if (h <= H) {
                            const uint32_t hnj = hn + static_cast<uint32_t>(j + 1) * n32;
                            if (kS) sv[j] = ld_x<T, WHITEN>(x, wv, hnj);
                            if (kG) {
#pragma unroll
                                for (int i = 0; i <= j + 1; ++i) v[j][i] = ld_x<T, WHITEN>(x, wv, hnj + d + i);
                            }
                        }
                    }
                    uint32_t r = 0;
#pragma unroll
                    for (int j = 0; j < G; ++j) {
                        const int h = h0 + j;
                        if (h <= H) {
                            if (kS) {
                                ss += sv[j];
                                ms.step(fmaf(ss, nm.rs[0][h - 1], -nm.murs[0][h - 1]), h);
                            }
                            if (kG) {
                                float va = v[j][0], vb = v[j][1];
#pragma unroll
                                for (int i = 1; i <= j; ++i) {
                                    va = (r == static_cast<uint32_t>(i)) ? v[j][i] : va;
                                    vb = (r == static_cast<uint32_t>(i)) ? v[j][i + 1] : vb;
                                }
                                const bool inc = vb > va;
                                sg += inc ? vb : va;
                                r += inc;
                                bits |= static_cast<uint32_t>(inc) << (h - 1);
                                mg.step(fmaf(sg, nm.rs[1][h - 1], -nm.murs[1][h - 1]), h);
                            }
                        }
                    }
                    d += r;
                    hn += static_cast<uint32_t>(G) * n32;
                }
            }
            const int64_t o = fbase + n;
            if (kS) {
                a.s.snr[o] = ms.best;
                a.s.best_h[o] = static_cast<uint8_t>(ms.bh);
            }
            if (kG) {
                a.g.snr[o] = mg.best;
                a.g.best_h[o] = static_cast<uint8_t>(mg.bh);
                if (a.g.path) store_path(a.g.path, a.path_bytes, o, bits);
            }
        }
        if (kS && a.s.argmax)
            block_argmax(valid ? argmax_key(ms.best, n) : 0ull, a.s.argmax + s, red);
        if (kG && a.g.argmax) {
            if (kS && a.s.argmax) __syncthreads();
            block_argmax(valid ? argmax_key(mg.best, n) : 0ull, a.g.argmax + s, red);
        }
        // next tile
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

// ---------------------------------------------------------------------------------------
// kernel: two fundamentals per thread (n0 + t and n0 + t + blockDim.x), their greedy chains
// interleaved order by order for instruction-level parallelism; a tile is 2 x blockDim.x
// fundamentals, so half as many threads cover a spectrum (one wave on the GPU where one
// fundamental per thread would need a second).
// ---------------------------------------------------------------------------------------
template <typename T, int FORMS, bool WHITEN>
__global__ void __launch_bounds__(256) k_fwd1d_x2(const Fwd1DArgs a)
{
    __shared__ NormSmem nm;
    __shared__ unsigned long long red[32];
    constexpr bool kS = (FORMS & HS_FORM_SIMPLE) != 0;
    constexpr bool kG = (FORMS & HS_FORM_GREEDY) != 0;
    constexpr int F = 2;
    const int H = a.H;
    int loaded_spec = -1;
    for (int64_t tile = blockIdx.x; tile < a.total_tiles; tile += gridDim.x) {
        const int s = tile_spectrum(a.tile_start, a.B, tile, a.tiles_per_spec, a.inv_tiles_per_spec);
        prefetch_next_spectrum(a, s, tile);
        if (s != loaded_spec) {
            if (loaded_spec >= 0) __syncthreads();
            const int64_t no = a.per_spectrum_norm ? static_cast<int64_t>(s) * H : 0;
            if (kS) load_norm(nm, 0, a.s.mu + no, a.s.sigma + no, H);
            if (kG) load_norm(nm, 1, a.g.mu + no, a.g.sigma + no, H);
            __syncthreads();
            loaded_spec = s;
        }
        const int64_t fbase = __ldg(a.fund_off + s);
        const int64_t nf = __ldg(a.nf_main + s);
        const int64_t n0 = (tile - __ldg(a.tile_start + s)) * (F * blockDim.x) + threadIdx.x;
        const T *x = static_cast<const T *>(a.x) + __ldg(a.in_off + s);
        const float *wv = a.w;
        uint32_t n[F];
        bool valid[F];
        float ss[F], sg[F], bs[F], bg[F];
        int hs_[F], hg[F];
        uint32_t d[F], bits[F], hn[F];
#pragma unroll
        for (int i = 0; i < F; ++i) {
            const int64_t ni = n0 + static_cast<int64_t>(i) * blockDim.x;
            valid[i] = ni < nf;
            if (a.checked && valid[i] && static_cast<int64_t>(H) * ni + H > __ldg(a.in_len + s) - 1)
                set_error(a.err, kErrBounds);   // every read lies in [0, H n + H]
            n[i] = valid[i] ? static_cast<uint32_t>(ni) : 0u;   // invalid lanes read bin 0 (harmless)
            const float x0 = ld_x<T, WHITEN>(x, wv, n[i]);
            ss[i] = x0;
            sg[i] = x0;
            d[i] = 0;
            bits[i] = 0;
            if (kG && a.mitigation) {
                const float b = ld_x<T, WHITEN>(x, wv, n[i] + 1);
                if (b > x0) { d[i] = 1; sg[i] = b; bits[i] = 1u; }
            }
            bs[i] = fmaf(ss[i], nm.rs[0][0], -nm.murs[0][0]);
            bg[i] = fmaf(sg[i], nm.rs[1][0], -nm.murs[1][0]);
            hs_[i] = 1;
            hg[i] = 1;
            hn[i] = n[i];
        }
        for (int h = 2; h <= H; ++h) {
            const float rs0 = nm.rs[0][h - 1], mr0 = nm.murs[0][h - 1];
            const float rs1 = nm.rs[1][h - 1], mr1 = nm.murs[1][h - 1];
            float xs[F], va[F], vb[F];
#pragma unroll
            for (int i = 0; i < F; ++i) {       // all loads of this order first
                hn[i] += n[i];
                if (kS) xs[i] = ld_x<T, WHITEN>(x, wv, hn[i]);
                if (kG) {
                    va[i] = ld_x<T, WHITEN>(x, wv, hn[i] + d[i]);
                    vb[i] = ld_x<T, WHITEN>(x, wv, hn[i] + d[i] + 1);
                }
            }
#pragma unroll
            for (int i = 0; i < F; ++i) {
                if (kS) {
                    ss[i] += xs[i];
                    const float v = fmaf(ss[i], rs0, -mr0);
                    if (v > bs[i]) { bs[i] = v; hs_[i] = h; }
                }
                if (kG) {
                    const bool inc = vb[i] > va[i];
                    sg[i] += inc ? vb[i] : va[i];
                    d[i] += inc;
                    bits[i] |= static_cast<uint32_t>(inc) << (h - 1);
                    const float v = fmaf(sg[i], rs1, -mr1);
                    if (v > bg[i]) { bg[i] = v; hg[i] = h; }
                }
            }
        }
        unsigned long long ks = 0ull, kg = 0ull;
#pragma unroll
        for (int i = 0; i < F; ++i) {
            if (!valid[i]) continue;
            const int64_t o = fbase + n[i];
            if (kS) {
                a.s.snr[o] = bs[i];
                a.s.best_h[o] = static_cast<uint8_t>(hs_[i]);
                const unsigned long long kk = argmax_key(bs[i], n[i]);
                ks = kk > ks ? kk : ks;
            }
            if (kG) {
                a.g.snr[o] = bg[i];
                a.g.best_h[o] = static_cast<uint8_t>(hg[i]);
                if (a.g.path) store_path(a.g.path, a.path_bytes, o, bits[i]);
                const unsigned long long kk = argmax_key(bg[i], n[i]);
                kg = kk > kg ? kk : kg;
            }
        }
        if (kS && a.s.argmax) block_argmax(ks, a.s.argmax + s, red);
        if (kG && a.g.argmax) {
            if (kS && a.s.argmax) __syncthreads();
            block_argmax(kg, a.g.argmax + s, red);
        }
        if (tile + gridDim.x < a.total_tiles) __syncthreads();
    }
}

// ---------------------------------------------------------------------------------------
// dispatch for one stored type
// ---------------------------------------------------------------------------------------
// kernel ids: 0 = direct gather; 1 = look-ahead over 4 orders; 3 = two fundamentals per thread;
// 4, 5 = look-ahead over 2, 3 orders; 2 = shared-memory windows (hs_fwd1d_win.cuh);
// 6, 7 = paired lanes, one lane per form and fundamental (hs_fwd1d_pair.cuh), one or two
// fundamentals per lane
template <typename T, int FORMS, bool WHITEN>
static const void *fwd1d_kernel_ptr(int kernel)
{
    switch (kernel) {
    case 0: return reinterpret_cast<const void *>(&k_fwd1d<T, FORMS, WHITEN, 1>);
    case 1: return reinterpret_cast<const void *>(&k_fwd1d<T, FORMS, WHITEN, 4>);
    case 3: return reinterpret_cast<const void *>(&k_fwd1d_x2<T, FORMS, WHITEN>);
    case 4: return reinterpret_cast<const void *>(&k_fwd1d<T, FORMS, WHITEN, 2>);
    case 5: return reinterpret_cast<const void *>(&k_fwd1d<T, FORMS, WHITEN, 3>);
    default: return nullptr;
    }
}

template <typename T>
static const void *fwd1d_win_kernel_for(int forms);
template <typename T>
static const void *fwd1d_pair_kernel_for(int forms, int whitening, int kernel);

template <typename T>
static const void *fwd1d_kernel_for(int forms, int whitening, int kernel)
{
    if (kernel == 2) return whitening ? nullptr : fwd1d_win_kernel_for<T>(forms);
    if (kernel == 6 || kernel == 7) return fwd1d_pair_kernel_for<T>(forms, whitening, kernel);
    if (whitening) {
        switch (forms) {
        case 1: return fwd1d_kernel_ptr<T, 1, true>(kernel);
        case 2: return fwd1d_kernel_ptr<T, 2, true>(kernel);
        case 3: return fwd1d_kernel_ptr<T, 3, true>(kernel);
        }
    } else {
        switch (forms) {
        case 1: return fwd1d_kernel_ptr<T, 1, false>(kernel);
        case 2: return fwd1d_kernel_ptr<T, 2, false>(kernel);
        case 3: return fwd1d_kernel_ptr<T, 3, false>(kernel);
        }
    }
    return nullptr;
}

}  // namespace hs
