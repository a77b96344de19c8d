// Instantiations of the batched kernel for CTAs of 4 warps (one
// translation unit per CTA shape, so they compile in parallel).
#include "batch_kernel.cuh"

namespace admm_impl {

void *batch_fn_w4(int mb, bool roll)
{
    if (mb > 4) return (void *)batch_kernel<4, 8, false>; // no staging for m > 4
    return roll ? (void *)batch_kernel<4, 4, true> : (void *)batch_kernel<4, 4, false>;
}

} // namespace admm_impl
