// Algorithm 1 + clamp on many independent quartics (the quartic benchmark
// of Sec. III-C): admm_quartic_min (FP64, the solver's FP64 minimiser) and
// admm_quartic_min_f32 (FP32 on packed column pairs, the solver's mixed
// minimiser, branch decisions as FP64 would take them).  Each thread takes
// consecutive elements (pairs in FP32) in a grid-stride loop: 7 streams of
// one value each, coalesced; the kernels are HBM bound once the minimiser
// is cheap enough.  Invalid elements (A < 0, A = C = 0, lo > hi, non-finite)
// get x = NaN and are counted.
#include <algorithm>
#include <cstdint>
#include <cstdio>

#include <cuda_runtime.h>

#include "internal.h"
#include "trace.h"
#include "quartic32.cuh"

using namespace admm_impl;

namespace {

__device__ __forceinline__ bool quartic_ok(double A, double B, double C, double D, double lo, double hi)
{
    return isfinite(A) && isfinite(B) && isfinite(C) && isfinite(D) && !isnan(lo) && !isnan(hi) && A >= 0.0 &&
           (A > 0.0 || C > 0.0) && lo <= hi;
}

__global__ void __launch_bounds__(256) quartic_many_f64(const double *A, const double *B, const double *C,
                                                        const double *D, const double *lo, const double *hi,
                                                        int64_t count, int mode, double *x, int *bad)
{
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < count;
         t += (int64_t)gridDim.x * blockDim.x) {
        const double a = A[t], b = B[t], c = C[t], d = D[t], l = lo[t], h = hi[t];
        if (quartic_ok(a, b, c, d, l, h)) {
            x[t] = quartic_min64_seeded(a, b, c, d, l, h, mode);
        } else {
            x[t] = NAN;
            atomicAdd(bad, 1);
        }
    }
}

__global__ void __launch_bounds__(256) quartic_many_f32(const float *A, const float *B, const float *C,
                                                        const float *D, const float *lo, const float *hi,
                                                        int64_t count, int mode, float *x, int *bad)
{
    const int64_t pairs = count / 2;
    unsigned esc = 0;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < pairs;
         t += (int64_t)gridDim.x * blockDim.x) {
        const float2 a = ((const float2 *)A)[t], b = ((const float2 *)B)[t], c = ((const float2 *)C)[t],
                     d = ((const float2 *)D)[t], l = ((const float2 *)lo)[t], h = ((const float2 *)hi)[t];
        const bool okx = quartic_ok(a.x, b.x, c.x, d.x, l.x, h.x), oky = quartic_ok(a.y, b.y, c.y, d.y, l.y, h.y);
        float2 r;
        if (okx && oky) {
            r = quartic_min32x2(a, b, c, d, l, h, mode, esc);
        } else {
            r.x = okx ? quartic_min32(a.x, b.x, c.x, d.x, l.x, h.x, mode, esc) : NAN;
            r.y = oky ? quartic_min32(a.y, b.y, c.y, d.y, l.y, h.y, mode, esc) : NAN;
            atomicAdd(bad, (okx ? 0 : 1) + (oky ? 0 : 1));
        }
        ((float2 *)x)[t] = r;
    }
    if (count % 2 == 1 && blockIdx.x == 0 && threadIdx.x == 0) {
        const int64_t t = count - 1;
        if (quartic_ok(A[t], B[t], C[t], D[t], lo[t], hi[t])) {
            x[t] = quartic_min32(A[t], B[t], C[t], D[t], lo[t], hi[t], mode, esc);
        } else {
            x[t] = NAN;
            atomicAdd(bad, 1);
        }
    }
}

int quartic_grid(int64_t work)
{
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const int64_t want = (work + 255) / 256;
    return (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)std::max(nsm, 1) * 8));
}

template <class T>
admm_status quartic_min_impl(const T *A, const T *B, const T *C, const T *D, const T *lo, const T *hi, int64_t count,
                             T *x, int32_t xmin_mode, int32_t on_device, void *stream)
{
    TraceRange trace_("admm_quartic_min");
    clear_last_error();
    if (count < 0 || (count > 0 && (!A || !B || !C || !D || !lo || !hi || !x)))
        return set_last_error("NULL array or negative count"), ADMM_EINVAL;
    if (xmin_mode != ADMM_XMIN_EXACT && xmin_mode != ADMM_XMIN_PAPER)
        return set_last_error("bad xmin_mode"), ADMM_EINVAL;
    if (count == 0) return ADMM_OK;
    if (on_device) { // the kernel dereferences these: they must be device-accessible
        const void *ptrs[7] = {A, B, C, D, lo, hi, x};
        for (const void *ptr : ptrs) {
            cudaPointerAttributes at{};
            if (cudaPointerGetAttributes(&at, ptr) != cudaSuccess ||
                (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged)) {
                cudaGetLastError(); // clear a sticky query error
                return set_last_error("on_device = 1 but an array is not device memory"), ADMM_EINVAL;
            }
        }
    }
    if (sizeof(T) == 4 && on_device &&
        ((uintptr_t)A | (uintptr_t)B | (uintptr_t)C | (uintptr_t)D | (uintptr_t)lo | (uintptr_t)hi | (uintptr_t)x) % 8)
        return set_last_error("FP32 device arrays must be 8-byte aligned"), ADMM_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t bytes = sizeof(T) * (size_t)count;
    T *d[7] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    int *dbad = nullptr;
    cudaError_t e = cudaMallocAsync(&dbad, sizeof(int), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(dbad, 0, sizeof(int), st);
    const T *src[6] = {A, B, C, D, lo, hi};
    if (!on_device)
        for (int t = 0; t < 7 && e == cudaSuccess; ++t) {
            e = cudaMallocAsync(&d[t], bytes, st);
            if (e == cudaSuccess && t < 6) e = cudaMemcpyAsync(d[t], src[t], bytes, cudaMemcpyHostToDevice, st);
        }
    if (e == cudaSuccess) {
        const T *a[6];
        for (int t = 0; t < 6; ++t) a[t] = on_device ? src[t] : d[t];
        T *xo = on_device ? x : d[6];
        if constexpr (sizeof(T) == 8)
            quartic_many_f64<<<quartic_grid(count), 256, 0, st>>>(a[0], a[1], a[2], a[3], a[4], a[5], count,
                                                                  xmin_mode, xo, dbad);
        else
            quartic_many_f32<<<quartic_grid(count / 2 + 1), 256, 0, st>>>(a[0], a[1], a[2], a[3], a[4], a[5],
                                                                          count, xmin_mode, xo, dbad);
        e = cudaGetLastError();
        if (e == cudaSuccess && !on_device) e = cudaMemcpyAsync(x, d[6], bytes, cudaMemcpyDeviceToHost, st);
    }
    int hbad = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hbad, dbad, sizeof(int), cudaMemcpyDeviceToHost, st);
    for (T *p : d)
        if (p) cudaFreeAsync(p, st);
    if (dbad) cudaFreeAsync(dbad, st);
    const cudaError_t es = cudaStreamSynchronize(st);
    if (e == cudaSuccess) e = es;
    if (e != cudaSuccess) {
        set_last_error(cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? ADMM_ENOMEM : ADMM_ECUDA;
    }
    if (hbad > 0) {
        char m[96];
        snprintf(m, sizeof m, "%d invalid quartics (x = NaN there)", hbad);
        set_last_error(m);
        return ADMM_EINVAL;
    }
    return ADMM_OK;
}

} // namespace

extern "C" {

admm_status admm_quartic_min(const double *A, const double *B, const double *C, const double *D, const double *lo,
                             const double *hi, int64_t count, double *x, int32_t xmin_mode, int32_t on_device,
                             void *stream)
{
    return quartic_min_impl<double>(A, B, C, D, lo, hi, count, x, xmin_mode, on_device, stream);
}

admm_status admm_quartic_min_f32(const float *A, const float *B, const float *C, const float *D, const float *lo,
                                 const float *hi, int64_t count, float *x, int32_t xmin_mode, int32_t on_device,
                                 void *stream)
{
    return quartic_min_impl<float>(A, B, C, D, lo, hi, count, x, xmin_mode, on_device, stream);
}

} // extern "C"
