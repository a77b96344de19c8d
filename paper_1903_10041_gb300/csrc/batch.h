// Internal declarations of the batched solve kernel (batch.cu) for the host
// code of the batch and serving APIs.  Not part of the public interface.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "internal.h"

namespace admm_impl {

constexpr int kWarpsMax = 16; // largest CTA of the batched kernel, in warps
// Elements per array of a batch or server store: the kernel indexes the
// arrays with 32-bit unsigned offsets from their bases.
constexpr int64_t kBatchArrayMax = 0xFFFFFFFFll;

// One instance of a batch: sizes and offsets into the packed arrays.
struct BatchInst {
    int n, m, q, ld;          // ld: row stride (multiple of 4)
    int64_t off_e;            // element arrays f2 f1 f0 g2 g1 g0 x: [m][q][ld] at off_e
    int64_t off_b;            // bound arrays lo hi: [m][ld] at off_b
    int64_t off_c;            // column arrays y s s_lo mu mu_lo: [q][ld] at off_c
    int off_pair;             // sumg0: [m*q] at off_pair
    int off_scal;             // scalar state: scal_size(m, q) doubles at off_scal
    int off_src;              // c: [m] at off_src
    int cs;                   // 1: f2..g0 shared by the scenarios (stored repeated; a step request
                              //    writes scenario 0's new maps to every scenario's row)
};

struct BatchArgs {
    const BatchInst *inst;
    const int *orderX;        // instances solved by cluster teams (all CTAs of a cluster), in queue order
    const int *orderL;        // instances solved by whole-CTA teams, in queue order
    const int *orderS;        // instances solved by one-warp teams, in queue order
    int nX, nL, nS;
    const int *nLS;           // if non-null, {nX, nL, nS} are read from device memory (graph replays)
    int *qX, *qL, *qS;        // queue heads (zeroed before the launch)
    const float *f2, *f1, *f0, *g2, *g1, *g0, *lo, *hi, *y;
    float *x, *s, *s_lo, *mu, *mu_lo;
    const double *c, *sumg0;
    double *scal;             // per-instance scalar state (in/out)
    double *out;              // per-instance record [id][kInfo]; [0] iterations so far, [14] finished
    int slice_doubles;        // shared memory per warp-team slice
    int stage_off;            // bytes from the CTA's shared memory to its coefficient stages (m <= 4 kernels)
    unsigned long long *dbg;  // bounds record of checked builds (see ADMM_IDX), else unused
    int iter_budget;          // > 0: stop every instance after this many more iterations
    const float *tick_work;   // if non-null (with iter_budget > 0): time-balanced budget, below
    const int *tick_rounds;   // if non-null and > 1: CTA and warp teams take each instance up to this many
                              // times per launch, in round-robin order (serving ticks, below)
    int *lock;                // per instance: 1 while a team runs it (round-robin launches)
    double r_tol, s_tol, tau;
    double adapt_target;      // r_tol / s_tol of the settings (Sec. IV-A ratio rule)
    int adapt_start;          // the adaptation applies at check iterations t >= adapt_start
    int max_iter, check_every, xmin_mode, sweep, adapt;
};

// Time-balanced iteration budget (serving ticks): an instance whose team
// spends `cost` element updates per thread and iteration runs
// floor(*tick_work / cost) iterations (at least 1), so every team of a tick
// works for about the same time and small instances are not held to the
// pace of the largest one.  The host sets *tick_work to iter_budget times
// the largest cost in the tick.  Where a tick ends does not change any
// result: an instance resumes from its saved state bit for bit.  With
// round-robin slices (below) a cluster team's instance, taken once per
// tick, runs R slices' worth of iterations in its one pass.
__host__ __device__ inline float team_iter_cost(int n, int m, int q, int team_threads)
{
    return (float)((double)n * m * q / team_threads) + 4.0f; // + per-iteration fixed work
}

// Round-robin ticks: when a tick has more instances than teams, one pass
// per instance leaves teams idle in the last, partial round.  With
// *tick_rounds = R > 1 the queue holds every instance R times (instance
// order repeated), each pass running a slice of the budget, so teams stay
// busy to within one slice.  A team that draws an instance another team is
// running skips it; state moves between SMs through L2 (the element update
// reads mutable state with L1-bypassing loads).
//
// Kernel variant (register arrays for M sources) of a batch or server: 4 for
// every m <= 4, else 8.  It must not depend on which instances share a
// launch, so that an instance gives the same bits alone and in any mix.
inline int batch_mbound(int max_m) { return max_m <= 4 ? 4 : 8; }

// Settings a batch or server accepts; false with the reason in why.
bool batch_params_ok(const admm_params *p, std::string &why);

size_t batch_slice_doubles(int max_m, int max_q);
// The persistent kernel for CTAs of 4, 8 or 16 warps and source bound mbound.
// roll: the rolling-stage instantiation (every input through cp.async; for launches whose
// instances never move to another SM, i.e. batches; servers take the double stage).
void *batch_fn_w4(int mbound, bool roll);
void *batch_fn_w8(int mbound, bool roll);
void *batch_fn_w16(int mbound, bool roll);
// Shared memory (doubles) a CTA or cluster team needs in each of its CTAs.
size_t batch_cluster_team_doubles(int max_m, int max_q, int warps, int cluster);
size_t batch_smem_bytes(int warps, size_t slice_doubles);
// Dynamic shared memory of one CTA: the CTA or cluster team's region, then
// (m <= 4 kernel) two coefficient stages per warp at byte offset stage_off;
// the per-warp slices of one-warp teams, when used, overlap both (a CTA runs
// its one-warp teams only after its CTA-team work).
struct BatchSmem {
    size_t bytes;
    int stage_off;
};
BatchSmem batch_cta_smem(int max_m, int max_q, int warps, int cluster, bool warp_teams, size_t slice_doubles);
int batch_blocks_per_sm(int warps, int mbound, size_t smem, bool roll = false);
// Launch with clusters of `cluster` CTAs (1 = no clusters); grid is a multiple of it.
cudaError_t launch_batch(int warps, int mbound, int grid, int cluster, const BatchArgs &a, size_t smem, bool roll,
                         cudaStream_t st);
// Co-resident clusters of that size (0 if it cannot launch).
int batch_max_clusters(int warps, int mbound, int cluster, size_t smem, bool roll = false);
// Moves data and state of instances ids[0..count-1] one step forward,
// writes the new last step from payload + t * payload_stride and clears the
// result record out[id].
void launch_shift_step(const BatchInst *inst, const int *ids, int count, const float *payload, int payload_stride,
                       float *f2, float *f1, float *f0, float *g2, float *g1, float *g0, float *lo, float *hi,
                       float *y, float *x, float *s, float *s_lo, float *mu, float *mu_lo, double *sumg0,
                       double *scal, double *out, cudaStream_t st);
// Gathers x (as FP64, rows of n) followed by x_1 (m values) of instances
// ids[0..count-1] into out + dst[t], for one device-to-host copy.
void launch_gather_x(const BatchInst *inst, const int *ids, const int64_t *dst, int count, const float *x,
                     const double *scal, double *out, cudaStream_t st);
// Moves the state of instances ids[0..count-1] one step forward (receding horizon).
void launch_shift_state(const BatchInst *inst, const int *ids, int count, float *x, float *s, float *s_lo, float *mu,
                        float *mu_lo, double *scal, cudaStream_t st);

} // namespace admm_impl
