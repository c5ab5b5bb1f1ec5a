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
#include "hs_fwd1d.cuh"

namespace hs {

template <typename T>
__device__ __forceinline__ float ld_plain(const void *p, int64_t j)
{
    return ld_raw<T, int64_t>(static_cast<const T *>(p), j);
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

// Shared memory: acc[L] (int64 fixed point), dwacc[L], then per candidate (k, n) of the block
// its target bin offset (int16, -1 = no contribution in this block) and value
// g[n] * fl(1 / sigma[h*(n)-1]).
// Grid: x = bin block [J, J + L), y = group of spectra [y G, y G + G).  With dL/dw requested,
// the group's sum over its spectra (in order) goes to dw_partial[y] (or straight to grad_w
// when there is one group); k_bwd_dw_reduce then adds the groups in order.
template <int FORM, typename T, bool WHITEN>
__global__ void __launch_bounds__(256) k_bwd1d(const Bwd1DArgs a)
{
    extern __shared__ __align__(16) unsigned char bsm[];
    const int L = a.block_bins;
    long long *acc = reinterpret_cast<long long *>(bsm);
    float *dwacc = reinterpret_cast<float *>(acc + L);
    float *cval = dwacc + L;
    int16_t *coff = reinterpret_cast<int16_t *>(cval + a.max_cand);
    __shared__ int kofs[kMaxH1D + 1];
    __shared__ long long klo[kMaxH1D];
    __shared__ float s_rsig[kMaxH1D];   // 1 / sigma_h
    __shared__ unsigned int s_maxbits;
    const bool want_w = a.grad_w != nullptr;
    const int s_begin = static_cast<int>(blockIdx.y) * a.group;
    const int s_end = min(a.B, s_begin + a.group);
    const int64_t J = static_cast<int64_t>(blockIdx.x) * L;
    const int H = a.H;
    if (want_w)
        for (int i = threadIdx.x; i < L; i += blockDim.x) dwacc[i] = 0.f;

    for (int s = s_begin; s < s_end; ++s) {
        const int64_t len = __ldg(a.in_len + s);
        if (J >= len) continue;   // uniform across the CTA
        const int Lr = static_cast<int>(len - J < L ? len - J : L);
        const int64_t Jend = J + Lr;   // exclusive
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
            if (threadIdx.x == 0) s_maxbits = 0u;
        }
        for (int i = threadIdx.x; i < L; i += blockDim.x) acc[i] = 0;
        __syncthreads();
        const int total = kofs[H];
        // stage every candidate's target offset and value; the (k, n) space is flattened and each
        // thread issues the loads of four candidates before using any of them
        unsigned int mybits = 0u;
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
        mybits = __reduce_max_sync(0xffffffffu, mybits);
        if ((threadIdx.x & 31) == 0) atomicMax(&s_maxbits, mybits);
        __syncthreads();
        // Exact accumulation: every value becomes an integer multiple of 2^(e-55), e the exponent of
        // the block's largest |value|, so at most 2 H values per bin sum below 2^62 and integer
        // addition makes the result independent of the order of the additions.
        const float vmax = __uint_as_float(s_maxbits);
        const bool finite = vmax > 0.f && vmax < INFINITY;
        const int ex = finite ? ilogbf(vmax) : 0;
        const float up = ldexpf(1.0f, 55 - ex);
        if (finite)
            for (int e = threadIdx.x; e < total; e += blockDim.x) {
                const int o = coff[e];
                if (o >= 0)
                    atomicAdd(reinterpret_cast<unsigned long long *>(acc + o),
                              static_cast<unsigned long long>(__float2ll_rn(cval[e] * up)));
            }
        __syncthreads();
        const double down = ldexp(1.0, ex - 55);
        const int64_t base = __ldg(a.in_off + s);
        for (int i = threadIdx.x; i < Lr; i += blockDim.x) {
            const float gx = static_cast<float>(static_cast<double>(acc[i]) * down);
            if (a.grad_in) a.grad_in[base + J + i] = WHITEN ? __fmul_rn(__ldg(a.w + J + i), gx) : gx;
            if (want_w) dwacc[i] = __fadd_rn(dwacc[i], __fmul_rn(ld_plain<T>(a.p, base + J + i), gx));
        }
        __syncthreads();
    }
    if (want_w) {
        const int64_t len = a.n_common;
        float *dst = gridDim.y == 1 ? a.grad_w : a.dw_partial + static_cast<int64_t>(blockIdx.y) * len;
        for (int i = threadIdx.x; i < L && J + i < len; i += blockDim.x) dst[J + i] = dwacc[i];
    }
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
