// Instantiations of the batched kernel for CTAs of 16 warps (one
// translation unit per CTA shape, so they compile in parallel).
#include "batch_kernel.cuh"

namespace admm_impl {

void *batch_fn_w16(int mb)
{
    return mb <= 4 ? (void *)batch_kernel<16, 4> : (void *)batch_kernel<16, 8>;
}

} // namespace admm_impl
