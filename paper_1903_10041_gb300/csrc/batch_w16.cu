// Instantiations of the batched kernel for CTAs of 16 warps (one
// translation unit per CTA shape, so they compile in parallel).
#include "batch_kernel.cuh"

namespace admm_impl {

void *batch_fn_w16(int mb, bool roll)
{
    if (mb > 4) return (void *)batch_kernel<16, 8, false>; // no staging for m > 4
    return roll ? (void *)batch_kernel<16, 4, true> : (void *)batch_kernel<16, 4, false>;
}

} // namespace admm_impl
