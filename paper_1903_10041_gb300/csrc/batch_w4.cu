// Instantiations of the batched kernel for CTAs of 4 warps (one
// translation unit per CTA shape, so they compile in parallel).
#include "batch_kernel.cuh"

namespace admm_impl {

void *batch_fn_w4(int mb)
{
    return mb <= 4 ? (void *)batch_kernel<4, 4> : (void *)batch_kernel<4, 8>;
}

} // namespace admm_impl
