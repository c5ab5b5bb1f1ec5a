// 1D forward kernels instantiated for stored type __nv_bfloat16.
#include "hs_fwd1d.cuh"
#include "hs_fwd1d_win.cuh"
#include "hs_fwd1d_pair.cuh"
#include "hs_fwd1d_tail.cuh"

namespace hs {
const void *fwd1d_kernel_bf16(int forms, int whitening, int kernel)
{
    return fwd1d_kernel_for<__nv_bfloat16>(forms, whitening, kernel);
}
const void *fwd1d_tail_kernel_bf16(int forms, int whitening)
{
    return fwd1d_tail_kernel_for<__nv_bfloat16>(forms, whitening);
}
}  // namespace hs
