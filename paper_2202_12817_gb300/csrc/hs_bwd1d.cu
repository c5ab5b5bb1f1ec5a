// Adjoint of the 1D forward (simple and greedy forms) with the drift path and the best
// harmonic count held fixed -- a subgradient through the maximum of Eq. 2:
//   dL/dx[j] = sum over (n, k <= h*(n)) with b_k(n) = j of g[n] / sigma[h*(n) - 1],
//   b_k(n) = k n (simple) or k n + popcount(path[n] & ((1 << k) - 1)) (greedy).
//
// Gather formulation, deterministic without float atomics: a CTA owns bins [J, J + L) of a
// spectrum and, for k = 1..H, visits the fundamentals whose order-k bin can fall in that
// range (greedy: n in [ceil(J/k) - 1, floor((J+L-1)/k)]; simple: multiples).  Two greedy
// fundamentals n, n+1 can hit the same bin at one k (D_k(n) = k, D_k(n+1) = 0), so each k is
// split into an even-n and an odd-n pass separated by a barrier; within a pass every bin is
// written by at most one thread.  The order of additions to every bin is therefore fixed:
// k ascending, even n before odd n.
#include "hs_fwd1d.cuh"

namespace hs {

template <typename T>
__device__ __forceinline__ float ld_plain(const void *p, int64_t j)
{
    return ld_raw<T>(static_cast<const T *>(p), j);
}

__device__ __forceinline__ uint32_t ld_path(const void *path, int bytes, int64_t i)
{
    if (bytes == 4) return __ldg(static_cast<const uint32_t *>(path) + i);
    if (bytes == 2) return __ldg(static_cast<const uint16_t *>(path) + i);
    return __ldg(static_cast<const uint8_t *>(path) + i);
}

template <int FORM, typename T, bool WHITEN>
__global__ void __launch_bounds__(256) k_bwd1d(const Bwd1DArgs a)
{
    extern __shared__ float sm[];
    const int L = a.block_bins;
    float *acc = sm;
    float *dwacc = sm + L;
    const bool all_spec = a.grad_w != nullptr;
    const int s_begin = all_spec ? 0 : static_cast<int>(blockIdx.y);
    const int s_end = all_spec ? a.B : s_begin + 1;
    const int64_t J = static_cast<int64_t>(blockIdx.x) * L;
    const int H = a.H;
    if (all_spec)
        for (int i = threadIdx.x; i < L; i += blockDim.x) dwacc[i] = 0.f;

    for (int s = s_begin; s < s_end; ++s) {
        const int64_t len = __ldg(a.in_len + s);
        if (J >= len) continue;   // uniform across the CTA
        const int Lr = static_cast<int>(len - J < L ? len - J : L);
        for (int i = threadIdx.x; i < L; i += blockDim.x) acc[i] = 0.f;
        __syncthreads();
        const int64_t fb = __ldg(a.fund_off + s);
        const int64_t nf = __ldg(a.fund_off + s + 1) - fb;
        const float *sig = a.sigma + (a.per_spectrum_norm ? static_cast<int64_t>(s) * H : 0);
        const int64_t Jend = J + Lr;   // exclusive
        for (int k = 1; k <= H; ++k) {
            int64_t n_hi = (Jend - 1) / k;
            if (n_hi > nf - 1) n_hi = nf - 1;
            if (FORM == HS_FORM_GREEDY) {
                int64_t n_lo = (J + k - 1) / k - 1;
                if (n_lo < 0) n_lo = 0;
                const uint32_t mask = (k >= 32) ? 0xffffffffu : ((1u << k) - 1u);
                for (int par = 0; par < 2; ++par) {
                    const int64_t first = n_lo + ((par - n_lo) & 1);
                    for (int64_t n = first + 2 * static_cast<int64_t>(threadIdx.x); n <= n_hi;
                         n += 2 * static_cast<int64_t>(blockDim.x)) {
                        const int hb = __ldg(a.best_h + fb + n);
                        if (k > hb || hb > H) continue;   // best_h outside 1..H contributes nothing
                        const int64_t j = static_cast<int64_t>(k) * n +
                                          __popc(ld_path(a.path, a.path_bytes, fb + n) & mask);
                        if (j >= J && j < Jend)
                            acc[j - J] += __fdiv_rn(__ldg(a.grad_snr + fb + n), __ldg(sig + hb - 1));
                    }
                    __syncthreads();
                }
            } else {
                const int64_t n_lo = (J + k - 1) / k;
                for (int64_t n = n_lo + threadIdx.x; n <= n_hi; n += blockDim.x) {
                    const int hb = __ldg(a.best_h + fb + n);
                    if (k > hb || hb > H) continue;
                    const int64_t j = static_cast<int64_t>(k) * n;
                    acc[j - J] += __fdiv_rn(__ldg(a.grad_snr + fb + n), __ldg(sig + hb - 1));
                }
                __syncthreads();
            }
        }
        const int64_t base = __ldg(a.in_off + s);
        for (int i = threadIdx.x; i < Lr; i += blockDim.x) {
            const float gx = acc[i];
            if (a.grad_in) a.grad_in[base + J + i] = WHITEN ? __fmul_rn(__ldg(a.w + J + i), gx) : gx;
            if (all_spec) dwacc[i] = __fadd_rn(dwacc[i], __fmul_rn(ld_plain<T>(a.p, base + J + i), gx));
        }
        __syncthreads();
    }
    if (all_spec) {
        const int64_t len = a.n_common;
        for (int i = threadIdx.x; i < L && J + i < len; i += blockDim.x) a.grad_w[J + i] = dwacc[i];
    }
}

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
