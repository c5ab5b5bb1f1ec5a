// Small kernels that run before a 1D forward pass: the clear of the argmax keys and the tile
// counter (k_fwd_reset) and the whitened copy of a whitening plan's input (k_prewhiten).
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

// A stored 16-bit value widened exactly to FP32.
template <typename T>
__device__ __forceinline__ float widen16(unsigned int bits);
template <>
__device__ __forceinline__ float widen16<__half>(unsigned int bits)
{
    return __half2float(__ushort_as_half(static_cast<unsigned short>(bits)));
}
template <>
__device__ __forceinline__ float widen16<__nv_bfloat16>(unsigned int bits)
{
    return __uint_as_float(bits << 16);
}

// Clears the per-spectrum argmax keys of both forms and the dynamic schedule's tile counter before
// a 1D pass.  Its first instruction lets the pass that follows it on the stream start at once
// (programmatic dependent launch); the pass waits for this kernel only before its first argmax
// update or tile-counter fetch, so the clear costs no serialisation gap.
__global__ void k_fwd_reset(unsigned long long *s_key, unsigned long long *g_key, int64_t B,
                            unsigned long long *counter)
{
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < B; i += stride) {
        if (s_key) s_key[i] = 0ull;
        if (g_key) g_key[i] = 0ull;
    }
    if (counter && blockIdx.x == 0 && threadIdx.x == 0) *counter = 0ull;
}

// Whitened copy of a whitening plan's input: X[o_s + j] = fl32(w[j] p_s[j]) for every spectrum s
// (offset o_s) and bin j < N, the product each pass kernel would form as it loads (the same single
// rounding, so the pass on X gives the same outputs bit for bit).  Four bins per thread where the
// input is 16-byte aligned (offsets and w are; N may leave a ragged tail).  Also clears the argmax
// keys and the tile counter, as k_fwd_reset does.
template <typename T>
__global__ void __launch_bounds__(256) k_prewhiten(const T *p, const float *w, float *X, const int64_t *in_off,
                                                   int32_t B, int64_t N, unsigned long long *s_key,
                                                   unsigned long long *g_key, unsigned long long *counter)
{
    if (blockIdx.x == 0) {
        for (int i = threadIdx.x; i < B; i += blockDim.x) {
            if (s_key) s_key[i] = 0ull;
            if (g_key) g_key[i] = 0ull;
        }
        if (counter && threadIdx.x == 0) *counter = 0ull;
    }
    const int64_t cps = (N + 1023) / 1024;   // 1024-bin chunks per spectrum
    const int64_t total = cps * B;
    for (int64_t c = blockIdx.x; c < total; c += gridDim.x) {
        const int64_t sp = c / cps;
        const int64_t j0 = (c - sp * cps) * 1024 + 4 * threadIdx.x;
        const int64_t o = __ldg(in_off + sp);
        if (j0 + 3 < N) {
            const float4 wv = __ldg(reinterpret_cast<const float4 *>(w + j0));
            float v0, v1, v2, v3;
            if constexpr (sizeof(T) == 4) {
                const float4 q = __ldg(reinterpret_cast<const float4 *>(p + o + j0));
                v0 = q.x; v1 = q.y; v2 = q.z; v3 = q.w;
            } else {
                const uint2 q = __ldg(reinterpret_cast<const uint2 *>(p + o + j0));
                v0 = widen16<T>(q.x & 0xffffu); v1 = widen16<T>(q.x >> 16);
                v2 = widen16<T>(q.y & 0xffffu); v3 = widen16<T>(q.y >> 16);
            }
            *reinterpret_cast<float4 *>(X + o + j0) =
                make_float4(__fmul_rn(wv.x, v0), __fmul_rn(wv.y, v1), __fmul_rn(wv.z, v2), __fmul_rn(wv.w, v3));
        } else {
            for (int64_t j = j0; j < N && j < j0 + 4; ++j) {
                float v;
                if constexpr (sizeof(T) == 4) v = __ldg(reinterpret_cast<const float *>(p) + o + j);
                else v = widen16<T>(__ldg(reinterpret_cast<const unsigned short *>(p) + o + j));
                X[o + j] = __fmul_rn(__ldg(w + j), v);
            }
        }
    }
}
