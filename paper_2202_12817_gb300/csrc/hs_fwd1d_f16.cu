// 1D forward kernels instantiated for stored type __half.
#include "hs_fwd1d.cuh"
#include "hs_fwd1d_win.cuh"
#include "hs_fwd1d_pair.cuh"
#include "hs_fwd1d_tail.cuh"

namespace hs {
const void *fwd1d_kernel_f16(int forms, int whitening, int kernel)
{
    return fwd1d_kernel_for<__half>(forms, whitening, kernel);
}
const void *fwd1d_tail_kernel_f16(int forms, int whitening)
{
    return fwd1d_tail_kernel_for<__half>(forms, whitening);
}
}  // namespace hs
