// Device store of many instances for the batched and serving solvers:
// packed FP32 arrays with one offset-range allocator per array family, so
// instances of any size can be placed, solved and released while others
// are in flight (admission is by free space in the store).
#pragma once
#include <map>
#include <string>
#include <vector>

#include "batch.h"

namespace admm_impl {

// First-fit allocator of aligned ranges in [0, cap), with coalescing frees.
class RangeAlloc {
  public:
    void init(int64_t cap);
    int64_t alloc(int64_t len, int64_t align); // -1 if no room
    void release(int64_t off, int64_t len);
    int64_t capacity() const { return cap_; }
    int64_t free_total() const;
    int64_t largest_free() const;

  private:
    int64_t cap_ = 0;
    std::map<int64_t, int64_t> free_; // start -> length
};

// Sizes of an instance in each array family.
struct InstSizes {
    int64_t e, b, c, p, s, m;
};
InstSizes inst_sizes(int n, int m, int q);

// Host-side check and FP32 packing of one instance (FP64 host arrays in the
// dense layout of admm.h).  Fills the staging vectors and sumg0; returns
// false with a message on invalid data.
struct Staged {
    int n = 0, m = 0, q = 0, ld = 0;
    int cs = 0;                // 1: f2..g0 given once per source ([m][n]), repeated over the scenarios here
    std::vector<float> e[7];   // f2 f1 f0 g2 g1 g0 x0   [m][q][ld]
    std::vector<float> b[2];   // lo hi                  [m][ld]
    std::vector<float> y;      // [q][ld]
    std::vector<double> sumg0; // [m*q]
    std::vector<double> c;     // [m]
};
bool stage_instance(const admm_problem &P, Staged &out, std::string &why);

struct Store {
    int64_t cap_e = 0, cap_b = 0, cap_c = 0, cap_p = 0, cap_s = 0, cap_m = 0;
    float *f2 = nullptr, *f1 = nullptr, *f0 = nullptr, *g2 = nullptr, *g1 = nullptr, *g0 = nullptr, *x = nullptr;
    float *lo = nullptr, *hi = nullptr;
    float *y = nullptr, *s = nullptr, *s_lo = nullptr, *mu = nullptr, *mu_lo = nullptr;
    double *sumg0 = nullptr, *scal = nullptr, *c = nullptr;
    RangeAlloc ae, ab, ac, ap, as, am;

    cudaError_t allocate(int64_t e, int64_t b, int64_t c, int64_t p, int64_t s, int64_t m);
    void free_all();
    // Reserves room for an instance; false (nothing reserved) if it does not fit.
    bool place(int n, int m, int q, BatchInst &out);
    void release(const BatchInst &I);
    // Copies a staged instance into its place and sets its zero start
    // (rho from params).  Uses `pinned` (>= the instance's float count) as
    // the staging buffer; synchronous on `st`.
    cudaError_t upload(const BatchInst &I, const Staged &S, const admm_params &prm, float *pinned, size_t pinned_n,
                       cudaStream_t st);
    void fill_args(BatchArgs &a) const;
};

// Dense FP64 state of one instance <-> its place in the store.
cudaError_t store_get_state(const Store &S, const BatchInst &I, admm_state *out, double *tmp, cudaStream_t st);
cudaError_t store_set_state(const Store &S, const BatchInst &I, const admm_state *in, double *tmp, cudaStream_t st);

} // namespace admm_impl
