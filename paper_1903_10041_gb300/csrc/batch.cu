// Batched solve: host-side launch helpers, kernel selection and the
// receding-horizon shift kernels.  The persistent kernel itself is in
// batch_kernel.cuh, instantiated per CTA shape in batch_w4/8/16.cu.
#include <algorithm>

#include "batch.h"
#include "common.cuh"
#include "mixed_elem.cuh"

namespace admm_impl {

void *batch_pick(int warps, int mb, bool roll)
{
    switch (warps) {
    case 4: return batch_fn_w4(mb, roll);
    case 16: return batch_fn_w16(mb, roll);
    default: return batch_fn_w8(mb, roll);
    }
}

namespace {

// Receding-horizon warm start (Sec. II, Alg. 2): the previous solution of a
// controller moved one step forward in place (x_k <- x_{k+1}, last step
// kept; the same for s and mu), x_1^(i) reset to the mean of the new first
// moves, cold flag cleared.  One CTA per instance.
// row[k] <- row[k + 1] for k < n - 1, by one warp: each round reads 32 * 4
// values ahead of the ones it overwrites (left to right, so every value is
// read before it is replaced).
__device__ __forceinline__ void warp_shift_left(float *row, int n)
{
    const int lane = threadIdx.x & 31;
    for (int k0 = 0; k0 < n - 1; k0 += 128) {
        float v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int k = k0 + u * 32 + lane;
            v[u] = k < n - 1 ? row[k + 1] : 0.0f;
        }
        __syncwarp();
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int k = k0 + u * 32 + lane;
            if (k < n - 1) row[k] = v[u];
        }
        __syncwarp();
    }
}

__global__ void shift_state_kernel(const BatchInst *inst, const int *ids, int count, float *x, float *s, float *s_lo,
                                   float *mu, float *mu_lo, double *scal)
{
    for (int t = blockIdx.x; t < count; t += gridDim.x) {
        const BatchInst I = inst[ids[t]];
        const int n = I.n, rows_e = I.m * I.q;
        // rows of x, then rows of s, s_lo, mu, mu_lo; each shifted left by one (a warp per row)
        for (int r = threadIdx.x >> 5; r < rows_e + 4 * I.q; r += blockDim.x >> 5) {
            float *row;
            if (r < rows_e) row = x + I.off_e + (int64_t)r * I.ld;
            else {
                const int c = (r - rows_e) / I.q, j = (r - rows_e) % I.q;
                float *base = c == 0 ? s : (c == 1 ? s_lo : (c == 2 ? mu : mu_lo));
                row = base + I.off_c + (int64_t)j * I.ld;
            }
            warp_shift_left(row, n);
        }
        __syncthreads();
        double *sc = scal + I.off_scal;
        const int mq = I.m * I.q;
        if (threadIdx.x < I.m) {
            const int i = threadIdx.x;
            double sum = 0.0;
            for (int j = 0; j < I.q; ++j) sum += (double)x[I.off_e + ((int64_t)i * I.q + j) * I.ld];
            sc[5 * mq + i] = sum / (double)I.q;
        }
        if (threadIdx.x == 0) sc[5 * mq + I.m + 4] = 0.0;
        __syncthreads();
    }
}

// Receding-horizon step request: the whole instance (coefficients, bounds,
// demand, x, s, mu) moves one step forward in place; the new last step's
// data comes from `payload` (per instance, FP32: f2 f1 f0 g2 g1 g0 [m][q],
// lo hi [m], y [q]; an instance with scenario-shared maps takes scenario
// 0's maps for every scenario); x at the new last step is clamped to its
// new bounds;
// sum_k beta_0 is recomputed; x_1^(i) = mean of the new first moves; cold
// flag cleared.  One CTA per instance.
__global__ void shift_step_kernel(const BatchInst *inst, const int *ids, int count, const float *payload,
                                  int payload_stride, float *f2, float *f1, float *f0, float *g2, float *g1, float *g0,
                                  float *lo, float *hi, float *y, float *x, float *s, float *s_lo, float *mu,
                                  float *mu_lo, double *sumg0, double *scal, double *out)
{
    for (int t = blockIdx.x; t < count; t += gridDim.x) {
        const int id = ids[t];
        const BatchInst I = inst[id];
        const int n = I.n, m = I.m, q = I.q, mq = m * q;
        const float *pl = payload + (size_t)t * payload_stride;
        for (int u = threadIdx.x; u < kInfo; u += blockDim.x) out[(size_t)id * kInfo + u] = 0.0; // fresh record
        float *erows[7] = {f2, f1, f0, g2, g1, g0, x};
        float *crows[5] = {y, s, s_lo, mu, mu_lo};
        const int nrows = 7 * mq + 2 * m + 5 * q;
        for (int r = threadIdx.x >> 5; r < nrows; r += blockDim.x >> 5) { // a warp per row
            float *row;
            if (r < 7 * mq) row = erows[r / mq] + I.off_e + (int64_t)(r % mq) * I.ld;
            else if (r < 7 * mq + 2 * m) {
                const int rr = r - 7 * mq;
                row = (rr < m ? lo : hi) + I.off_b + (int64_t)(rr % m) * I.ld;
            } else {
                const int rr = r - 7 * mq - 2 * m;
                row = crows[rr / q] + I.off_c + (int64_t)(rr % q) * I.ld;
            }
            warp_shift_left(row, n);
        }
        __syncthreads();
        // the new last step (shared maps: scenario 0's maps of the step data in every scenario's row)
        const int last = n - 1;
        for (int u = threadIdx.x; u < mq; u += blockDim.x) {
            const int64_t e = I.off_e + (int64_t)u * I.ld + last;
            const int v = I.cs ? u / q * q : u;
            f2[e] = pl[0 * mq + v];
            f1[e] = pl[1 * mq + v];
            f0[e] = pl[2 * mq + v];
            g2[e] = pl[3 * mq + v];
            g1[e] = pl[4 * mq + v];
            g0[e] = pl[5 * mq + v];
        }
        for (int i = threadIdx.x; i < m; i += blockDim.x) {
            lo[I.off_b + (int64_t)i * I.ld + last] = pl[6 * mq + i];
            hi[I.off_b + (int64_t)i * I.ld + last] = pl[6 * mq + m + i];
        }
        for (int j = threadIdx.x; j < q; j += blockDim.x) y[I.off_c + (int64_t)j * I.ld + last] = pl[6 * mq + 2 * m + j];
        __syncthreads();
        for (int u = threadIdx.x; u < mq; u += blockDim.x) {
            const int i = u / q;
            const int64_t e = I.off_e + (int64_t)u * I.ld + last;
            const float l = lo[I.off_b + (int64_t)i * I.ld + last], h = hi[I.off_b + (int64_t)i * I.ld + last];
            x[e] = x[e] < l ? l : (x[e] > h ? h : x[e]);
        }
        // sum_k beta_0 per pair (one warp per pair, fixed order)
        const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
        for (int u = w; u < mq; u += nw) {
            double acc = 0.0;
            for (int k = lane; k < n; k += 32) acc += (double)g0[I.off_e + (int64_t)u * I.ld + k];
            acc = warp_sum(acc);
            if (lane == 0) sumg0[I.off_pair + u] = acc;
        }
        __syncthreads();
        double *sc = scal + I.off_scal;
        if (threadIdx.x < m) {
            const int i = threadIdx.x;
            double sum = 0.0;
            for (int j = 0; j < q; ++j) sum += (double)x[I.off_e + ((int64_t)i * q + j) * I.ld];
            sc[5 * mq + i] = sum / (double)q;
        }
        if (threadIdx.x == 0) sc[5 * mq + m + 4] = 0.0;
        __syncthreads();
    }
}

// One CTA per finished instance: x rows [m q][ld] (FP32) -> [m q][n] FP64,
// then x_1 from the scalar state.
__global__ void gather_x_kernel(const BatchInst *inst, const int *ids, const int64_t *dst, int count, const float *x,
                                const double *scal, double *out)
{
    for (int t = blockIdx.x; t < count; t += gridDim.x) {
        const BatchInst I = inst[ids[t]];
        const int64_t rows = (int64_t)I.m * I.q, ne = rows * I.n;
        double *o = out + dst[t];
        for (int64_t e = threadIdx.x; e < ne; e += blockDim.x) {
            const int64_t r = e / I.n;
            const int k = (int)(e - r * I.n);
            o[e] = (double)x[I.off_e + r * I.ld + k];
        }
        for (int i = threadIdx.x; i < I.m; i += blockDim.x) o[ne + i] = scal[I.off_scal + 5 * rows + i];
    }
}

} // namespace

void launch_gather_x(const BatchInst *inst, const int *ids, const int64_t *dst, int count, const float *x,
                     const double *scal, double *out, cudaStream_t st)
{
    if (count > 0) gather_x_kernel<<<std::min(count, 4096), 256, 0, st>>>(inst, ids, dst, count, x, scal, out);
}

void launch_shift_step(const BatchInst *inst, const int *ids, int count, const float *payload, int payload_stride,
                       float *f2, float *f1, float *f0, float *g2, float *g1, float *g0, float *lo, float *hi,
                       float *y, float *x, float *s, float *s_lo, float *mu, float *mu_lo, double *sumg0,
                       double *scal, double *out, cudaStream_t st)
{
    if (count > 0)
        shift_step_kernel<<<std::min(count, 1024), 256, 0, st>>>(inst, ids, count, payload, payload_stride, f2, f1, f0,
                                                                 g2, g1, g0, lo, hi, y, x, s, s_lo, mu, mu_lo, sumg0,
                                                                 scal, out);
}

void launch_shift_state(const BatchInst *inst, const int *ids, int count, float *x, float *s, float *s_lo, float *mu,
                        float *mu_lo, double *scal, cudaStream_t st)
{
    if (count > 0) shift_state_kernel<<<std::min(count, 1024), 256, 0, st>>>(inst, ids, count, x, s, s_lo, mu, mu_lo, scal);
}

// Shared memory (doubles) of one team: scalar state, double-buffered records
// of `items` work items, per-warp column maxima, x at k = 0, scratch, and
// the FP32 zeta + lambda and x1 + nu vectors.
static size_t team_doubles(int m, int q, int items, int nwt)
{
    const int mq = m * q;
    return (size_t)scal_size(m, q) + 2 * (size_t)items * m * 4 + 4 * (size_t)nwt + 24 + mq + kMaxM + kWarpsMax * 8 +
           2 * ((mq + 1) / 2) + 8;
}

size_t batch_slice_doubles(int max_m, int max_q)
{
    // a one-warp team has one segment per row
    return (team_doubles(max_m, max_q, max_q, 1) + 3) / 4 * 4;
}

size_t batch_cluster_team_doubles(int max_m, int max_q, int warps, int cluster)
{
    // at most q + W items (W = warps x cluster)
    return team_doubles(max_m, max_q, max_q + warps * cluster, warps);
}

size_t batch_smem_bytes(int warps, size_t slice_doubles)
{
    return sizeof(double) * slice_doubles * (size_t)warps;
}

BatchSmem batch_cta_smem(int max_m, int max_q, int warps, int cluster, bool warp_teams, size_t slice_doubles)
{
    const size_t team = sizeof(double) * batch_cluster_team_doubles(max_m, max_q, warps, cluster);
    const size_t off = (team + 15) / 16 * 16;
    // the stage region of 32-float2 slots per warp (m <= 4 kernel: the larger of the double stage,
    // 2 (4 m + 1), and the rolling stage, 5 + 7 m; see stage_vec32, roll_issue_col), then 11
    // floats per thread for the check-only lane maxima
    const size_t stages = batch_mbound(max_m) == 4
                              ? (size_t)warps * stage_region_slots<4>() * 32 * sizeof(float2) +
                                    (size_t)warps * 32 * 11 * sizeof(float)
                              : 0;
    size_t bytes = off + stages;
    if (warp_teams) bytes = std::max(bytes, batch_smem_bytes(warps, slice_doubles));
    return {bytes, (int)off};
}

int batch_blocks_per_sm(int warps, int mb, size_t smem, bool roll)
{
    void *fn = batch_pick(warps, mb, roll);
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return 0;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, warps * 32, smem) != cudaSuccess) return 0;
    return nb;
}

// The kernel's shared-memory attribute is set by batch_blocks_per_sm, which
// the host calls before launching (and before any graph capture).
cudaError_t launch_batch(int warps, int mb, int grid, int cluster, const BatchArgs &a, size_t smem, bool roll,
                         cudaStream_t st)
{
    void *fn = batch_pick(warps, mb, roll);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(warps * 32);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cluster > 1 ? cluster : 1;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    void *args[] = {(void *)&a};
    return cudaLaunchKernelExC(&cfg, fn, args);
}

int batch_max_clusters(int warps, int mb, int cluster, size_t smem, bool roll)
{
    void *fn = batch_pick(warps, mb, roll);
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return 0;
    if (cluster > 8 && cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess)
        return 0;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(cluster * 152);
    cfg.blockDim = dim3(warps * 32);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int nc = 0;
    if (cudaOccupancyMaxActiveClusters(&nc, fn, &cfg) != cudaSuccess) return 0;
    return nc;
}

} // namespace admm_impl
