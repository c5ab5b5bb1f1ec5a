// 2D greedy harmonic sum over an f-fdot plane: the 1D greedy rule (Eq. 5, Algorithm 2)
// lifted to a 3x3 neighbourhood at (h f + df, h z + dz).  The paper names the
// higher-dimensional sum (acceleration search) without giving an algorithm; the rule here
// is: best value starts at the centre, the 8 neighbours are scanned in raster order
// (dz = -1..1 outer, df = -1..1 inner) and replace it only when strictly larger.
// The plane is stored as FP32, FP16 or BF16; each value is widened exactly to FP32, so the
// comparisons are those of the stored values and the sum accumulates in FP32.
#include "hs_fwd1d.cuh"

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
        int64_t df = 0, dz = 0;
        float sum = 0.f;
        uint32_t bits = 0;
        int bh = 1;
        for (int h = 1; h <= H; ++h) {
            const int64_t cf = h * f + df;
            const int64_t cr = a.z0_row + h * z + dz;
            if (a.checked) {
                if (cr - 1 < 0 || cr + 1 > a.n_rows - 1 || cf - 1 < 0 || cf + 1 > nfq - 1) {
                    set_error(a.err, kErrBounds);
                    break;
                }
            }
            const T *r0 = static_cast<const T *>(a.plane) + (cr - 1) * nfq + cf;   // row z - 1, column cf
            const T *r1 = r0 + nfq;
            const T *r2 = r1 + nfq;
            const float c00 = ld_raw<T, int64_t>(r0, -1), c01 = ld_raw<T, int64_t>(r0, 0), c02 = ld_raw<T, int64_t>(r0, 1);
            const float c10 = ld_raw<T, int64_t>(r1, -1), c11 = ld_raw<T, int64_t>(r1, 0), c12 = ld_raw<T, int64_t>(r1, 1);
            const float c20 = ld_raw<T, int64_t>(r2, -1), c21 = ld_raw<T, int64_t>(r2, 0), c22 = ld_raw<T, int64_t>(r2, 1);
            float v = c11;
            int code = 4;
            if (c00 > v) { v = c00; code = 0; }
            if (c01 > v) { v = c01; code = 1; }
            if (c02 > v) { v = c02; code = 2; }
            if (c10 > v) { v = c10; code = 3; }
            if (c12 > v) { v = c12; code = 5; }
            if (c20 > v) { v = c20; code = 6; }
            if (c21 > v) { v = c21; code = 7; }
            if (c22 > v) { v = c22; code = 8; }
            sum += v;
            df += code % 3 - 1;
            dz += code / 3 - 1;
            bits |= static_cast<uint32_t>(code) << (4 * (h - 1));
            const float snr = fmaf(sum, rs[h - 1], -murs[h - 1]);
            if (h == 1 || snr > best) { best = snr; bh = h; }
        }
        a.g.snr[o] = best;
        a.g.best_h[o] = static_cast<uint8_t>(bh);
        if (a.g.path) static_cast<uint32_t *>(a.g.path)[o] = bits;
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
