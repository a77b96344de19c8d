// Device helpers shared by the solver kernels: bounded grid barrier,
// deterministic warp/block reductions, L2-coherent loads.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace admm_impl {

__device__ __forceinline__ unsigned long long globaltimer_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ int ld_volatile_i32(const int *p)
{
    return *(const volatile int *)p;
}

// Bounds-checked builds (compiled with -DADMM_DEBUG_BOUNDS, libadmm_debug.so):
// an element-array index is checked against the instance's range of that
// array before the access; an index outside it is recorded in *rec (array
// id in the top byte, the index below; the first violation wins) and
// replaced by 0, so the access stays inside the allocation and the kernel
// carries on.  The host turns a record into ADMM_EBOUNDS.  Release builds
// use the index as it is.
#ifdef ADMM_DEBUG_BOUNDS
__device__ __forceinline__ size_t dbg_index(size_t idx, size_t need, size_t len, unsigned long long *rec, int id)
{
    if (idx + need <= len) return idx;
    if (rec) atomicCAS(rec, 0ull, ((unsigned long long)(id + 1) << 56) | (idx & 0x00FFFFFFFFFFFFFFull));
    return 0;
}
#define ADMM_IDX(idx, need, len, rec, id) ::admm_impl::dbg_index((idx), (need), (len), (rec), (id))
#else
#define ADMM_IDX(idx, need, len, rec, id) (idx)
#endif
// array ids of the bounds records
enum { DBG_COL = 0, DBG_X = 1, DBG_COEF = 2, DBG_BOUND = 3, DBG_SELFTEST = 15 };

// Loads that bypass L1: data written by other SMs since this SM last cached it.
__device__ __forceinline__ double ldcg(const double *p) { return __ldcg(p); }

// Grid-wide barrier for a cooperative launch.  `bar` counts arrivals and is
// zeroed before the launch; barrier number b (1, 2, ...) waits for b * grid
// arrivals.  The wait is bounded: after spin_ns nanoseconds it records
// timeout_code in *status and returns false; it also returns false as soon
// as another CTA has recorded an error.  Never traps.
__device__ __forceinline__ bool grid_barrier(unsigned *bar, unsigned target, int *status,
                                             long long spin_ns, int timeout_code)
{
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(bar, 1u);
        unsigned long long t0 = globaltimer_ns();
        int ok = 1;
        for (unsigned spins = 1;; ++spins) {
            unsigned v = ld_acquire_u32(bar);
            if ((int)(v - target) >= 0)
                break;
            if ((spins & 15) == 0) { // error flag and time limit every 16 polls
                if (ld_volatile_i32(status) != 0) { ok = 0; break; }
                if ((long long)(globaltimer_ns() - t0) > spin_ns) {
                    atomicCAS(status, 0, timeout_code);
                    ok = 0;
                    break;
                }
            }
            __nanosleep(32); // leave issue slots to co-resident CTAs still computing
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

template <class T> __device__ __forceinline__ T warp_sum(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
template <class T> __device__ __forceinline__ T warp_max(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
// Maxima of non-negative doubles (residual terms, absolute values): for
// x, y >= 0 the order of their IEEE-754 bit patterns read as signed 64-bit
// integers is the order of the values, so these run on the integer pipes
// instead of the FP64 pipe (1/64 of the FP32 rate on this GPU).
__device__ __forceinline__ double max_nonneg(double a, double b)
{
    return __longlong_as_double(max(__double_as_longlong(a), __double_as_longlong(b)));
}
__device__ __forceinline__ double warp_max_nonneg(double v)
{
    long long b = __double_as_longlong(v);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) b = max(b, __shfl_xor_sync(0xffffffffu, b, o));
    return __longlong_as_double(b);
}
template <class T> __device__ __forceinline__ T warp_min(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

__device__ __forceinline__ double clampd(double v, double lo, double hi)
{
    return v < lo ? lo : (v > hi ? hi : v);
}
__device__ __forceinline__ float clampf(float v, float lo, float hi)
{
    return v < lo ? lo : (v > hi ? hi : v);
}

} // namespace admm_impl
