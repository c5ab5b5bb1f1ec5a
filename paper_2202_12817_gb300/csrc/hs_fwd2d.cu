// 2D greedy harmonic sum over an f-fdot plane, one thread per (f, z) chain carried in registers
// through all orders (kernels 0 and 1 of the 2D plan); the per-order rule is chain2d_step.
// The plane is stored as FP32, FP16 or BF16; each value is widened exactly to FP32, so the
// comparisons are those of the stored values and the sum accumulates in FP32.
#include "hs_fwd1d.cuh"
#include "hs_fwd2d.cuh"

namespace hs {

template <typename T>
__global__ void __launch_bounds__(256) k_fwd2d(const Fwd2DArgs a)
{
    __shared__ float rs[kMaxH2D], murs[kMaxH2D];
    __shared__ unsigned long long red[32];
    const int H = a.H;
    if (threadIdx.x < H) {
        const float r = __frcp_rn(__ldg(a.g.sigma + threadIdx.x));
        rs[threadIdx.x] = r;
        murs[threadIdx.x] = __fmul_rn(__ldg(a.g.mu + threadIdx.x), r);
    }
    __syncthreads();
    // block order: f-tiles fastest (grid.x = f-tile), or z rows fastest (grid.x = z), which keeps
    // the fundamentals of neighbouring z -- whose low orders read overlapping rows -- co-resident
    const int64_t ft = a.zfast ? blockIdx.y : blockIdx.x;
    const int64_t fi = ft * blockDim.x + threadIdx.x;
    const int64_t zi = a.zfast ? blockIdx.x : blockIdx.y;
    const bool valid = fi < a.nff;
    const int64_t o = zi * a.nff + fi;
    float best = 0.f;
    if (valid) {
        const int64_t f = a.f_lo + fi, z = a.z_lo + zi;
        const int64_t nfq = a.n_freq;
        Chain2D c{0.f, 0.f, 0u, 0, 0, 1};
        for (int h = 1; h <= H; ++h) {
            const int64_t cf = h * f + c.df;
            const int64_t cr = a.z0_row + h * z + c.dz;
            if (a.checked) {
                if (cr - 1 < 0 || cr + 1 > a.n_rows - 1 || cf - 1 < 0 || cf + 1 > nfq - 1) {
                    set_error(a.err, kErrBounds);
                    break;
                }
            }
            const T *r0 = static_cast<const T *>(a.plane) + (cr - 1) * nfq + cf;   // row z - 1, column cf
            float v9[9];
#pragma unroll
            for (int r = 0; r < 3; ++r)
#pragma unroll
                for (int q = 0; q < 3; ++q) v9[3 * r + q] = ld_raw<T, int64_t>(r0 + r * nfq, q - 1);
            chain2d_step(c, h, v9, rs[h - 1], murs[h - 1]);
        }
        best = c.best;
        a.g.snr[o] = best;
        a.g.best_h[o] = static_cast<uint8_t>(c.bh);
        if (a.g.path) static_cast<uint32_t *>(a.g.path)[o] = c.bits;
    }
    if (a.g.argmax) block_argmax(valid ? argmax_key(best, o) : 0ull, a.g.argmax, red);
}

const void *fwd2d_kernel(int dtype)
{
    switch (dtype) {
    case HS_F32: return reinterpret_cast<const void *>(&k_fwd2d<float>);
    case HS_F16: return reinterpret_cast<const void *>(&k_fwd2d<__half>);
    case HS_BF16: return reinterpret_cast<const void *>(&k_fwd2d<__nv_bfloat16>);
    }
    return nullptr;
}

}  // namespace hs
