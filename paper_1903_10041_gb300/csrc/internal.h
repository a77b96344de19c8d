// Internal declarations shared by the host C ABI and the kernel translation
// units.  Not part of the public interface.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/admm.h"

namespace admm_impl {

constexpr int kBlock = 256;          // threads per CTA of the mixed-precision solve kernel
constexpr int kBlockF64 = 384;       // threads per CTA of the FP64 solve kernel
constexpr int kSingleWarpsMax = 12;  // most warps per CTA of the single-instance kernels
constexpr int kMaxM = ADMM_MAX_M;
constexpr int kInfo = 16;            // doubles of the per-solve info record
constexpr int kMixedVW = 2; // columns per thread in the mixed kernels (one float2 pair)

// Stop test of the mixed-precision solves: r < r_tol and sigma <
// kMixedSigmaStop * s_tol (Alg. 2 step 3 with a margin on sigma).  x is
// stored in FP32; at the stop of these problems sigma is the binding
// residual (r is orders of magnitude below r_tol), and the FP32 rounding of x
// leaves the KKT residual of eq. (2) at the mixed stop up to 1e-6 above that
// of the FP64 solve stopped at the same thresholds.  Stopping at 0.85 s_tol
// removes that excess; it stays above sigma's FP32 floor (about m ulps of x
// in the demand term, 7.2e-7 for m = 4 and x in [1, 2)), so mixed solves
// still reach it.  The penalty adaptation of Sec. IV-A keeps using the ratio
// r_tol / s_tol of the settings.
constexpr double kMixedSigmaStop = 0.85;
inline double stop_r_tol(int precision, double r_tol) { return (void)precision, r_tol; }
inline double stop_s_tol(int precision, double s_tol)
{
    return precision == ADMM_FP64 ? s_tol : kMixedSigmaStop * s_tol;
}

// Offsets into the scalar state vector (doubles), for mq = m*q pairs:
//   [0, 5mq)        lam, zeta, h, p, nu   (pair arrays, mq each)
//   [5mq, 5mq+m)    x1
//   [5mq+m, +4)     rho_1..rho_4
//   [5mq+m+4]       cold flag (1.0 = zero start, z = 0)
//   [5mq+m+5]       pending mu divisor (1.0 = none)
inline __host__ __device__ int scal_size(int m, int q) { return 5 * m * q + m + 6; }

// info record written by a solve:
//   0 iters, 1 converged, 2 r, 3 sigma, 4..7 r terms, 8..10 sigma terms,
//   11 objective, 12 status, 13 cubic decisions escalated to FP64 (mixed)
struct SingleArgs {
    int n, m, q, ld;           // ld: padded row stride of the [*][n] arrays
    int rs;                    // row length of the column space: n (FP64) or ld (mixed, padded)
    int cq, cj;                // coefficient row of pair (i, j): i * cq + j * cj ((q, 1), or (1, 0) when shared)
    int64_t ncols;             // q * rs columns (j, k)
    int64_t chunk;             // flat split: columns per CTA (contiguous in j-major order)
    int pieces;                // > 0: row-aligned split, CTA b takes piece b % pieces of row b / pieces
    int nbmax;                 // max CTAs whose columns touch one row
    int grid;                  // CTAs
    const void *f2, *f1, *f0, *g2, *g1, *g0, *lo, *hi, *y;   // storage type of the precision
    const double *c, *sumg0;   // [m], [mq]
    void *x, *s, *mu;          // state arrays (storage type)
    void *s_lo, *mu_lo;        // mixed: low parts of the float-float column state s, mu
    double *scal;              // scalar state, in/out
    double *part;              // [2][q][nbmax][m][4] partial records (gsum, dmax, dmin, x0), row-major by
                               // row j and position b - b0(j) of the CTA among those touching row j
    double *cpart;             // [2][grid][4] per-CTA column maxima and objective partials
    unsigned *bar;             // barrier counter (zeroed before the launch)
    int *status;               // 0 or an admm_status set by a device wait
    double *info;              // out [kInfo]
    unsigned long long *dbg;   // bounds record of checked builds (see ADMM_IDX), else unused
    double r_tol, s_tol, tau;
    double adapt_target;       // r_tol / s_tol of the settings (Sec. IV-A ratio rule)
    int adapt_start;           // the adaptation applies at check iterations t >= adapt_start
    int max_iter, check_every, xmin_mode, sweep, adapt;
    long long spin_ns;         // bound of one barrier wait
};

// Launch the persistent single-instance solve kernel (cooperative launch);
// minb selects the register-budget variant (1 or 2 CTAs per SM).
cudaError_t launch_single(int precision, int minb, const SingleArgs &a, size_t smem, cudaStream_t st);
// Max co-resident CTAs per SM of that kernel for the given dynamic smem.
int single_blocks_per_sm(int precision, int m, int minb, size_t smem);
// Launch shape of a solve: CTAs, columns per CTA (a multiple of the vector
// width in mixed precision), kernel variant, and the most CTAs touching one
// row j (records per row).  grid = 0: the kernel cannot be resident.
struct SingleShape {
    int grid;
    int64_t chunk;
    int pieces;
    int minb;
    int nbmax;
};

// Column bound t (0..p) of the row-aligned split of a row of rs columns
// into p pieces, on multiples of `unit`.
inline __host__ __device__ int64_t piece_bound(int t, int64_t rs, int p, int unit)
{
    return (int64_t)t * rs / p / unit * unit;
}
SingleShape single_shape(int precision, int m, int q, int64_t rs, int nsm, size_t smem);
// Dynamic shared memory the single-instance kernel needs.
size_t single_smem_bytes(int m, int q, int precision);
// Index of the kernel variant used for m sources (template bound).
int single_mbound(int m);
// Threads per CTA of the single-instance kernel of a precision.
int single_threads(int precision);
// Row copies with conversion (device to device): rows x n values from a
// source with row stride sld into a destination with row stride dld.
void convert_rows_f32_to_f64(double *dst, int64_t dld, const float *src, int64_t sld, int n, int64_t rows,
                             cudaStream_t st);
void convert_rows_f64_to_f32(float *dst, int64_t dld, const double *src, int64_t sld, int n, int64_t rows,
                             cudaStream_t st);
// Float-float column arrays (hi + lo) <-> FP64 rows.
void convert_rows_ff_to_f64(double *dst, int64_t dld, const float *hi, const float *lo, int64_t sld, int n,
                            int64_t rows, cudaStream_t st);
void split_rows_f64_to_ff(float *hi, float *lo, int64_t dld, const double *src, int64_t sld, int n, int64_t rows,
                          cudaStream_t st);
// Thread-local message returned by admm_last_error().
void set_last_error(const char *msg);
void clear_last_error();

} // namespace admm_impl
