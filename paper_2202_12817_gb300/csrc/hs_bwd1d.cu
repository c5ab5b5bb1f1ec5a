// Adjoint of the 1D forward (simple and greedy forms) with the drift path and the best
// harmonic count held fixed -- a subgradient through the maximum of Eq. 2:
//   dL/dx[j] = sum over (n, k <= h*(n)) with b_k(n) = j of g[n] / sigma[h*(n) - 1],
//   b_k(n) = k n (simple) or k n + popcount(path[n] & ((1 << k) - 1)) (greedy).
//
// Gather formulation, deterministic without float atomics: a CTA owns bins [J, J + L) of a
// spectrum and, for k = 1..H, visits the fundamentals whose order-k bin can fall in that
// range (greedy: n in [ceil(J/k) - 1, floor((J+L-1)/k)]; simple: multiples) -- about L ln H
// candidates instead of L H bin-order pairs.  All candidates' target bins and values are
// staged in shared memory with coalesced loads, then added into per-bin 64-bit fixed-point
// accumulators with shared-memory integer atomics: the values are scaled by a power of two
// set by the block's largest |value| (resolution 2^-55 of it), integer addition is
// associative, so the gradient is bit-reproducible whatever the order of the additions, and
// more accurate than an FP32 running sum.  dL/dw sums the spectra in order: within a group of
// spectra per CTA, then the groups' partial sums in order.
//
// Sparse upstream gradients (a top-k loss leaves most g[n] = 0): a first pass marks, per spectrum,
// the bin blocks that receive at least one contribution (those of b_k(n), k <= h*(n), for every n
// with g[n] != 0) and lists the fundamentals with g[n] != 0 while there are at most
// kBwdListCap of them.  The adjoint kernel skips the candidate staging of unmarked blocks, whose
// dL/dx is exactly zero, and in a listed spectrum stages only the listed fundamentals' bins.
// Either way a block sums the same set of nonzero contributions, exactly, so the result does
// not depend on the path taken.
#include <type_traits>

#include "hs_fwd1d.cuh"

namespace hs {

template <typename T>
__device__ __forceinline__ float ld_plain(const void *p, int64_t j)
{
    return ld_raw<T, int64_t>(static_cast<const T *>(p), j);
}

// RN(v * 2^e2) for a 64-bit integer v, with integer operations only (FP64 arithmetic is slow on
// GB300): the 24 leading bits of |v| rounded to nearest-even on the rest, assembled into the
// float's fields -- one rounding.  Results outside FP32's normal range go through ldexpf (a
// subnormal result may then be rounded twice).
__device__ __forceinline__ float fixed_to_float(long long v, int e2)
{
    if (v == 0) return 0.f;
    const unsigned long long u = v < 0 ? 0ull - static_cast<unsigned long long>(v) : static_cast<unsigned long long>(v);
    const int msb = 63 - __clzll(static_cast<long long>(u));   // |v| in [2^msb, 2^(msb+1))
    uint32_t m;                                                 // rounded significand, leading 1 at bit 23
    if (msb <= 23) {
        m = static_cast<uint32_t>(u) << (23 - msb);
    } else {
        const int sh = msb - 23;
        const unsigned long long q = u >> sh;
        const unsigned long long rem = u - (q << sh);
        const unsigned long long half = 1ull << (sh - 1);
        m = static_cast<uint32_t>(q);
        if (rem > half || (rem == half && (m & 1u))) ++m;      // a carry to 2^24 bumps the exponent below
    }
    const int be = msb + e2 + 127;                              // biased exponent of the result
    if (be <= 0 || be >= 254) return ldexpf(__ll2float_rn(v), e2);
    const uint32_t bits = (static_cast<uint32_t>(be - 1) << 23) + m;
    return __uint_as_float(bits | (v < 0 ? 0x80000000u : 0u));
}

__device__ __forceinline__ uint32_t ld_path(const void *path, int bytes, int64_t i)
{
    if (bytes == 4) return __ldg(static_cast<const uint32_t *>(path) + i);
    if (bytes == 2) return __ldg(static_cast<const uint16_t *>(path) + i);
    return __ldg(static_cast<const uint8_t *>(path) + i);
}

// Candidates of order k for the bin block [J, J + Lr): greedy n in [ceil(J/k) - 1, floor((J+Lr-1)/k)],
// simple n in [ceil(J/k), floor((J+Lr-1)/k)], clipped to [0, nf).
__device__ __forceinline__ void cand_range(int form, int64_t J, int64_t Jend, int k, int64_t nf, int64_t &lo,
                                           int64_t &hi)
{
    if (Jend + k < 0x7fffffff) {   // 32-bit division where the bins allow it
        hi = static_cast<uint32_t>(Jend - 1) / static_cast<uint32_t>(k);
        lo = static_cast<uint32_t>(J + k - 1) / static_cast<uint32_t>(k);
    } else {
        hi = (Jend - 1) / k;
        lo = (J + k - 1) / k;
    }
    if (hi > nf - 1) hi = nf - 1;
    lo -= (form == HS_FORM_GREEDY ? 1 : 0);
    if (lo < 0) lo = 0;
}

// Four consecutive stored values p[j..j+3] as float; `nv` (< 4 at a ragged block end) of them are
// read, the rest are 0.  j is a multiple of 4 and p + j is 16-byte (FP32) / 8-byte (16-bit) aligned.
template <typename T>
__device__ __forceinline__ void ld4(const void *p, int64_t j, int nv, float (&v)[4])
{
    const T *q = static_cast<const T *>(p) + j;
    if (nv >= 4) {
        if constexpr (sizeof(T) == 4) {
            const float4 f = __ldg(reinterpret_cast<const float4 *>(q));
            v[0] = f.x; v[1] = f.y; v[2] = f.z; v[3] = f.w;
        } else {
            const uint2 u = __ldg(reinterpret_cast<const uint2 *>(q));
            const unsigned short h[4] = {static_cast<unsigned short>(u.x & 0xffffu), static_cast<unsigned short>(u.x >> 16),
                                         static_cast<unsigned short>(u.y & 0xffffu), static_cast<unsigned short>(u.y >> 16)};
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                if constexpr (std::is_same<T, __half>::value) v[i] = __half2float(__ushort_as_half(h[i]));
                else v[i] = __uint_as_float(static_cast<unsigned int>(h[i]) << 16);
            }
        }
    } else {
#pragma unroll
        for (int i = 0; i < 4; ++i) v[i] = i < nv ? ld_raw<T, int64_t>(q, i) : 0.f;
    }
}

// Shared memory: acc[L] (int64 fixed point), then per candidate (k, n) of the block its target
// bin offset (int16, -1 = no contribution in this block) and value g[n] * fl(1 / sigma[h*(n)-1]).
// Grid: x = bin block [J, J + L), y = group of spectra [y G, y G + G).  With dL/dw requested,
// the group's sum over its spectra (in order) goes to dw_partial[y] (or straight to grad_w
// when there is one group); k_bwd_dw_reduce then adds the groups in order.  Thread t owns bins
// J + 4t .. J + 4t + 3 of the epilogue (L = 4 x blockDim.x) and keeps their dL/dw sum in registers.
template <int FORM, typename T, bool WHITEN>
// Four CTAs per SM (64 registers): the streaming epilogue needs the warps (0.376 ms vs 0.431 ms at
// 78 registers and three CTAs on the 256 x 2^20 training step; five CTAs spill and take 0.526 ms).
__global__ void __launch_bounds__(256, 4) k_bwd1d(const Bwd1DArgs a)
{
    extern __shared__ __align__(16) unsigned char bsm[];
    const int L = a.block_bins;
    long long *acc = reinterpret_cast<long long *>(bsm);
    float *cval = reinterpret_cast<float *>(acc + L);
    int16_t *coff = reinterpret_cast<int16_t *>(cval + a.max_cand);
    __shared__ uint8_t s_act[256];   // active flags of the next (up to) 256 spectra of the group
    __shared__ int kofs[kMaxH1D + 1];
    __shared__ long long klo[kMaxH1D];
    __shared__ float s_rsig[kMaxH1D];   // 1 / sigma_h
    __shared__ unsigned int s_maxbits;
    __shared__ int s_nlist;
    const bool want_w = a.grad_w != nullptr;
    const int s_begin = static_cast<int>(blockIdx.y) * a.group;
    const int s_end = min(a.B, s_begin + a.group);
    const int64_t J = static_cast<int64_t>(blockIdx.x) * L;
    const int H = a.H;
    const int t4 = 4 * static_cast<int>(threadIdx.x);   // this thread's first bin of the epilogue
    float dw[4] = {0.f, 0.f, 0.f, 0.f};                 // its dL/dw partial sums (grad_w mode)

    // epilogue of one spectrum's block for this thread's four bins, given their dL/dx values
    auto epilogue = [&](int64_t base, int Lr, const float (&gx)[4], const float (&pv)[4]) {
        const int nv = Lr - t4;
        if (nv <= 0) return;
        if (a.grad_in) {
            float o[4];
            float wv[4] = {1.f, 1.f, 1.f, 1.f};
            if (WHITEN) ld4<float>(a.w, J + t4, nv, wv);
#pragma unroll
            for (int i = 0; i < 4; ++i) o[i] = WHITEN ? __fmul_rn(wv[i], gx[i]) : gx[i];
            float *dst = a.grad_in + base + J + t4;
            if (nv >= 4 && (reinterpret_cast<uintptr_t>(dst) & 15) == 0) {
                *reinterpret_cast<float4 *>(dst) = make_float4(o[0], o[1], o[2], o[3]);
            } else {
#pragma unroll
                for (int i = 0; i < 4; ++i)
                    if (i < nv) dst[i] = o[i];
            }
        }
        if (want_w) {
#pragma unroll
            for (int i = 0; i < 4; ++i)
                if (i < nv) dw[i] = __fadd_rn(dw[i], __fmul_rn(pv[i], gx[i]));
        }
    };

    for (int s = s_begin; s < s_end; ++s) {
        if (a.active && ((s - s_begin) & 255) == 0) {
            // stage the active flags of the next 256 spectra (one load each, all in flight at once)
            __syncthreads();
            const int sj = s + static_cast<int>(threadIdx.x);
            if (threadIdx.x < 256)
                s_act[threadIdx.x] = sj < s_end ? a.active[static_cast<int64_t>(sj) * a.nblk + blockIdx.x] : 0;
            __syncthreads();
        }
        const int64_t len = __ldg(a.in_len + s);
        if (J >= len) continue;   // uniform across the CTA
        const int Lr = static_cast<int>(len - J < L ? len - J : L);
        const int64_t Jend = J + Lr;   // exclusive
        const int64_t base = __ldg(a.in_off + s);
        // uniform across the CTA: does any contribution land in this block?
        const bool active = !a.active || s_act[(s - s_begin) & 255] != 0;
        if (!active) {
            // dL/dx is exactly zero here: the same epilogue with gx = 0 (w * 0, p * 0 keep their
            // signed zeros and non-finite products as the full path would).  A run of such
            // spectra issues its loads of p together.
            constexpr int R = 4;
            int r = 1;
            while (r < R && s + r < s_end && ((s + r - s_begin) & 255) != 0 && !s_act[(s + r - s_begin) & 255] &&
                   __ldg(a.in_len + s + r) == len)
                ++r;
            float pv[R][4];
            const float zero[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int q = 0; q < R; ++q) {
                if (q < r) {
                    if (want_w && t4 < Lr) ld4<T>(a.p, __ldg(a.in_off + s + q) + J + t4, Lr - t4, pv[q]);
                    else pv[q][0] = pv[q][1] = pv[q][2] = pv[q][3] = 0.f;
                }
            }
#pragma unroll
            for (int q = 0; q < R; ++q)
                if (q < r) epilogue(__ldg(a.in_off + s + q), Lr, zero, pv[q]);
            s += r - 1;
            continue;
        }
        // this spectrum's p for the epilogue, loaded before the candidate search hides its latency
        float pv[4] = {0.f, 0.f, 0.f, 0.f};
        if (want_w && t4 < Lr) ld4<T>(a.p, base + J + t4, Lr - t4, pv);
        const int64_t fb = __ldg(a.fund_off + s);
        const int64_t nf = __ldg(a.fund_off + s + 1) - fb;
        if (threadIdx.x < 32) {
            // lane k-1 sizes the candidate range of order k; a warp prefix sum places the ranges
            const int k = threadIdx.x + 1;
            int cnt = 0;
            int64_t lo = 0;
            if (k <= H) {
                int64_t hi;
                cand_range(FORM, J, Jend, k, nf, lo, hi);
                cnt = hi >= lo ? static_cast<int>(hi - lo + 1) : 0;
                klo[k - 1] = lo;
                s_rsig[k - 1] = __frcp_rn(__ldg(a.sigma + (a.per_spectrum_norm ? static_cast<int64_t>(s) * H : 0) + k - 1));
            }
            int incl = cnt;
            for (int o = 1; o < 32; o <<= 1) {
                const int v = __shfl_up_sync(0xffffffffu, incl, o);
                if (threadIdx.x >= o) incl += v;
            }
            if (k <= H) kofs[k - 1] = incl - cnt;
            if (k == H) kofs[H] = incl;
            if (threadIdx.x == 0) {
                s_maxbits = 0u;
                s_nlist = 0;
            }
        }
        for (int i = threadIdx.x; i < L; i += blockDim.x) acc[i] = 0;
        __syncthreads();
        const int nz = a.nz_count ? __ldg(a.nz_count + s) : kBwdListCap + 1;
        unsigned int mybits = 0u;
        int total;
        if (nz <= kBwdListCap) {
            // listed spectrum: each (listed fundamental, order) pair whose bin lands in the block
            // appends its contribution
            const int *lst = a.nz_list + static_cast<int64_t>(s) * kBwdListCap;
            for (int q = threadIdx.x; q < nz * H; q += blockDim.x) {
                const int e = q / H, kq = q - e * H + 1;
                const int64_t nn = __ldg(lst + e);
                const int hb = __ldg(a.best_h + fb + nn);
                if (kq > hb || hb > H) continue;
                int64_t j = static_cast<int64_t>(kq) * nn;
                if (FORM == HS_FORM_GREEDY) {
                    const uint32_t pa = ld_path(a.path, a.path_bytes, fb + nn);
                    j += __popc(pa & ((kq >= 32) ? 0xffffffffu : ((1u << kq) - 1u)));
                }
                if (j < J || j >= Jend) continue;
                const float c = __ldg(a.grad_snr + fb + nn) * s_rsig[hb - 1];
                const int slot = atomicAdd(&s_nlist, 1);
                coff[slot] = static_cast<int16_t>(j - J);
                cval[slot] = c;
                const unsigned int bits = __float_as_uint(fabsf(c));
                mybits = bits > mybits ? bits : mybits;
            }
            __syncthreads();
            total = s_nlist;
        } else {
        total = kofs[H];
        // stage every candidate's target offset and value; the (k, n) space is flattened and each
        // thread issues the loads of four candidates before using any of them
        int k = 1;
        for (int e0 = threadIdx.x; e0 < total; e0 += 4 * blockDim.x) {
            int kk[4], hb[4];
            int64_t nn[4];
            uint32_t pa[4];
            float gg[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int e = e0 + u * blockDim.x;
                hb[u] = 0;
                if (e < total) {
                    while (kofs[k] <= e) ++k;   // e grows with u and e0, so k only advances
                    kk[u] = k;
                    nn[u] = klo[k - 1] + (e - kofs[k - 1]);
                    hb[u] = __ldg(a.best_h + fb + nn[u]);
                    pa[u] = FORM == HS_FORM_GREEDY ? ld_path(a.path, a.path_bytes, fb + nn[u]) : 0u;
                    gg[u] = __ldg(a.grad_snr + fb + nn[u]);
                }
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int e = e0 + u * blockDim.x;
                if (e < total) {
                    int16_t off = -1;
                    float c = 0.f;
                    const int kq = kk[u];
                    if (kq <= hb[u] && hb[u] <= H) {   // best_h outside 1..H contributes nothing
                        int64_t j = static_cast<int64_t>(kq) * nn[u];
                        if (FORM == HS_FORM_GREEDY)
                            j += __popc(pa[u] & ((kq >= 32) ? 0xffffffffu : ((1u << kq) - 1u)));
                        if (j >= J && j < Jend) {
                            off = static_cast<int16_t>(j - J);
                            c = gg[u] * s_rsig[hb[u] - 1];
                            const unsigned int bits = __float_as_uint(fabsf(c));
                            mybits = bits > mybits ? bits : mybits;   // order of non-negative floats
                        }
                    }
                    coff[e] = off;
                    cval[e] = c;
                }
            }
        }
        }
        mybits = __reduce_max_sync(0xffffffffu, mybits);
        if ((threadIdx.x & 31) == 0) atomicMax(&s_maxbits, mybits);
        __syncthreads();
        // Exact accumulation: every value becomes an integer multiple of 2^(e-55), e the exponent of
        // the block's largest |value|, so at most 2 H values per bin sum below 2^62 and integer
        // addition makes the result independent of the order of the additions.
        const float vmax = __uint_as_float(s_maxbits);
        const bool finite = vmax > 0.f && vmax < INFINITY;
        const int ex = finite ? ilogbf(vmax) : 0;
        // value -> round(value * 2^(55-ex)); the scale is split in two exact power-of-two steps so
        // that neither factor overflows for tiny blocks (ex < -72)
        const int sh = 55 - ex, sh1 = sh > 100 ? 100 : sh;
        const float up1 = ldexpf(1.0f, sh1), up2 = ldexpf(1.0f, sh - sh1);
        if (finite)
            for (int e = threadIdx.x; e < total; e += blockDim.x) {
                const int o = coff[e];
                if (o >= 0)
                    atomicAdd(reinterpret_cast<unsigned long long *>(acc + o),
                              static_cast<unsigned long long>(__float2ll_rn(__fmul_rn(__fmul_rn(cval[e], up1), up2))));
            }
        __syncthreads();
        {
            float gx[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int i = 0; i < 4; ++i)
                if (t4 + i < Lr) gx[i] = fixed_to_float(acc[t4 + i], ex - 55);
            epilogue(base, Lr, gx, pv);
        }
        __syncthreads();
    }
    if (want_w) {
        const int64_t len = a.n_common;
        float *dst = gridDim.y == 1 ? a.grad_w : a.dw_partial + static_cast<int64_t>(blockIdx.y) * len;
#pragma unroll
        for (int i = 0; i < 4; ++i)
            if (J + t4 + i < len) dst[J + t4 + i] = dw[i];
    }
}

// Marks active[s][j / L] for every chosen bin j = b_k(n), k <= h*(n), of every fundamental with a
// nonzero upstream gradient (grid-stride over all fundamentals of the plan).  A warp's fundamentals
// are consecutive, so at one order their bins fall in one or two blocks and the byte stores of a
// warp mostly hit one sector.
template <int FORM>
__global__ void __launch_bounds__(256) k_bwd_mark(const Bwd1DArgs a, int64_t F)
{
    const int L = a.block_bins;
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < F;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        if (!(__ldg(a.grad_snr + i) != 0.f)) continue;   // NaN gradients are marked too
        const int hb = __ldg(a.best_h + i);
        if (hb < 1 || hb > a.H) continue;                  // contributes nothing
        // spectrum owning output i: largest s with fund_off[s] <= i
        int lo = 0, hi = a.B - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (__ldg(a.fund_off + mid) <= i) lo = mid;
            else hi = mid - 1;
        }
        const int64_t n = i - __ldg(a.fund_off + lo);
        const int pos = atomicAdd(a.nz_count + lo, 1);
        if (pos < kBwdListCap) a.nz_list[static_cast<int64_t>(lo) * kBwdListCap + pos] = static_cast<int>(n);
        const uint32_t pa = FORM == HS_FORM_GREEDY ? ld_path(a.path, a.path_bytes, i) : 0u;
        uint8_t *row = a.active + static_cast<int64_t>(lo) * a.nblk;
        int64_t prev = -1;
        for (int k = 1; k <= hb; ++k) {
            int64_t j = static_cast<int64_t>(k) * n;
            if (FORM == HS_FORM_GREEDY) j += __popc(pa & ((k >= 32) ? 0xffffffffu : ((1u << k) - 1u)));
            const int64_t blk = j / L;
            if (blk != prev) {
                row[blk] = 1;
                prev = blk;
            }
        }
    }
}

const void *bwd_mark_kernel(int form)
{
    return form == HS_FORM_GREEDY ? reinterpret_cast<const void *>(&k_bwd_mark<HS_FORM_GREEDY>)
                                  : reinterpret_cast<const void *>(&k_bwd_mark<HS_FORM_SIMPLE>);
}

// grad_w[j] = sum over groups g (in order) of dw_partial[g][j]
__global__ void k_bwd_dw_reduce(const float *__restrict__ part, int groups, int64_t n, float *__restrict__ grad_w)
{
    for (int64_t j = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; j < n;
         j += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        float acc = 0.f;
        for (int g = 0; g < groups; ++g) acc = __fadd_rn(acc, __ldg(part + g * n + j));
        grad_w[j] = acc;
    }
}

const void *bwd_dw_reduce_kernel() { return reinterpret_cast<const void *>(&k_bwd_dw_reduce); }

template <int FORM, typename T>
static const void *bwd_ptr(int whitening)
{
    return whitening ? reinterpret_cast<const void *>(&k_bwd1d<FORM, T, true>)
                     : reinterpret_cast<const void *>(&k_bwd1d<FORM, T, false>);
}

const void *bwd1d_kernel(int form, int dtype, int whitening)
{
    if (form == HS_FORM_SIMPLE) {
        if (dtype == HS_F32) return bwd_ptr<HS_FORM_SIMPLE, float>(whitening);
        if (dtype == HS_F16) return bwd_ptr<HS_FORM_SIMPLE, __half>(whitening);
        if (dtype == HS_BF16) return bwd_ptr<HS_FORM_SIMPLE, __nv_bfloat16>(whitening);
    } else if (form == HS_FORM_GREEDY) {
        if (dtype == HS_F32) return bwd_ptr<HS_FORM_GREEDY, float>(whitening);
        if (dtype == HS_F16) return bwd_ptr<HS_FORM_GREEDY, __half>(whitening);
        if (dtype == HS_BF16) return bwd_ptr<HS_FORM_GREEDY, __nv_bfloat16>(whitening);
    }
    return nullptr;
}

}  // namespace hs
