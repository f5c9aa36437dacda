// Internal declarations shared by the CUDA translation units of libkb.
//
// Data layout in HBM
//   * Graph: the off-diagonal part of L in CSR (int32 rowptr/col, FP32 weights
//     w_ij = -L_ij > 0, weights omitted when all are 1) plus the diagonal excess
//     r_i = L_ii - sum_j w_ij (omitted when it is zero everywhere, i.e. L = D - W).
//     Then (L x)_i = sum_j w_ij (x_i - x_j) + r_i x_i   (difference form).
//   * Blocks of the Krylov process: n x W row-major FP32 (or FP64 for the plain FP64
//     mode), W = the block width M rounded up to 16/32/64/128; the padding columns hold
//     zeros throughout.  One row of a block is W*4 bytes, read with 16-byte vector loads.
//   * Small matrices (Gram partials, H blocks, R factors) are W x W row-major.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cstdint>
#include <cstddef>
#include <string>
#include <vector>

#include "kb.h"

namespace kb {

// ------------------------------------------------------------------ graph
struct GraphDev {
    int64_t n = 0;
    int64_t nnz = 0;                  // stored off-diagonal entries
    const int32_t *rowptr = nullptr;  // n+1
    const int32_t *col = nullptr;     // nnz
    const float *w = nullptr;         // nnz or nullptr (unit weights)
    const float *rdiag = nullptr;     // n or nullptr (zero diagonal excess)
};

}  // namespace kb

struct kb_graph {
    kb::GraphDev dev;
    int32_t *d_rowptr = nullptr;
    int32_t *d_col = nullptr;
    float *d_w = nullptr;
    float *d_rdiag = nullptr;
    double lambda = 0.0;     // Gershgorin bound
    double lambda_proj = 0.0;// spectral bound for the Lanczos projected step: the Gershgorin
                             // bound, or for a unit-weight D - A the smaller edge bound
                             // max over edges (d_i + d_j) (Anderson and Morley)
    int device = 0;
    int32_t unit_weights = 0;
    int32_t zero_excess = 0;
};

namespace kb {

// ------------------------------------------------------------------ errors
void set_error(const std::string &msg);
int fail(int code, const std::string &msg);
int cuda_fail(cudaError_t e, const char *what);

#define KB_CUDA_TRY(expr)                                      \
    do {                                                       \
        cudaError_t _e = (expr);                               \
        if (_e != cudaSuccess) return ::kb::cuda_fail(_e, #expr); \
    } while (0)

// ------------------------------------------------------------------ device control block
// One per solve, in device memory.  Kernels after a stop or a breakdown return early.
struct Ctrl {
    int32_t status;          // KB_OK / KB_ERR_BREAKDOWN
    int32_t stop;            // 1 once the process stopped (invariant space or breakdown)
    int32_t steps;           // blocks entering the result
    int32_t breakdown_step;  // -1 or step index
    double est_change;       // stopping rule: relative change at the last check, -1 if none
    int32_t from_check;      // stopping rule: buffer of the check whose U_k is the result, or -1
    int32_t reserved;
};

// Makes a device current for the lifetime of the object and restores the caller's current
// device afterwards (entry points switch to the graph's device and must not leave the
// calling thread on it).
class DeviceGuard {
  public:
    DeviceGuard() { ok_ = cudaGetDevice(&prev_) == cudaSuccess; }
    cudaError_t set(int dev) { return cudaSetDevice(dev); }
    ~DeviceGuard() {
        if (ok_) cudaSetDevice(prev_);
    }
    DeviceGuard(const DeviceGuard &) = delete;
    DeviceGuard &operator=(const DeviceGuard &) = delete;

  private:
    int prev_ = 0;
    bool ok_ = false;
};

// ------------------------------------------------------------------ profiling (events)
struct KernelClass {
    enum : int { SPMM = 0, ROWBLOCK, REDUCE, SMALL, PROJECTED, ASSEMBLE, OTHER, COUNT };
};
// Work counters a profiled launch fills on the device: rows it processed and, for the
// SpMM, stored nonzeros of those rows (one atomicAdd per CTA).  nullptr when not profiling.
struct ProfCount {
    unsigned long long *rows = nullptr;
    unsigned long long *nnz = nullptr;
};
// prof_begin returns the counters of this launch (nullptr fields when not profiling).
ProfCount prof_begin(int cls, cudaStream_t s);
// Records the end event (when profiling) and always adds nlaunch to the launch counter.
// With work counters, the launch's algorithmic bytes are fixed + rows * per_row +
// nnz * per_nnz and its flops rows * flops_per_row, rows/nnz read from the device counters
// when the profile is read; otherwise the full-size alg_bytes / alg_flops are used.
void prof_end(int cls, cudaStream_t s, double alg_bytes, double alg_flops, int nlaunch = 1,
              double per_row = 0.0, double per_nnz = 0.0, double flops_per_row = 0.0,
              double fixed = 0.0);
void count_launches(int k);
bool prof_on();

// ------------------------------------------------------------------ frontier restriction
// Krylov blocks started from E_W are exactly zero outside the (k-1)-hop ball of W at step
// k.  gen[i] (uint8) is the hop distance of row i from W (255 = not reached yet); tgen[t]
// is the minimum over the 32-row activity tile t.  Kernels given tgen skip tiles whose
// minimum exceeds their limit.
constexpr int ACT_ROWS = 32;
constexpr int FRONTIER_MAX_HOPS = 250;
__device__ __forceinline__ int tile_min_gen(const int32_t *tgen, int64_t r0, int rows) {
    int m = 0x7fffffff;
    for (int64_t t = r0 / ACT_ROWS; t <= (r0 + rows - 1) / ACT_ROWS; ++t) m = min(m, __ldg(tgen + t));
    return m;
}

// ------------------------------------------------------------------ storage / compute types
// Blocks are stored as T and computed in Cmp<T>::type: FP32 blocks in FP32, FP64 blocks in
// FP64, BF16 blocks in FP32 (the BF16 basis mode: half the bytes per block row, FP32
// accumulation).  Small matrices and Gram partials are always of the compute type.
template <typename T> struct Cmp { using type = T; };
template <> struct Cmp<__nv_bfloat16> { using type = float; };

// ------------------------------------------------------------------ double-float sums
// FP64 arithmetic is slow on this part, so reductions of FP32 data accumulate in an
// unevaluated pair hi + lo of floats (about 48 significant bits) on the FP32 pipe.
// two_sum is the error-free transformation of Knuth (s + e == a + b exactly); merging two
// pairs renormalises with Dekker's fast two-sum.  The pairs are stored as 8-byte DF values
// where the FP64 path stores doubles.
struct DF {
    float hi, lo;
};
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}
__device__ __forceinline__ void df_add(DF &a, float b) {
    float s, e;
    two_sum(a.hi, b, s, e);
    a.hi = s;
    a.lo += e;
}
__device__ __forceinline__ void df_merge(DF &a, const DF &b) {
    float s, e;
    two_sum(a.hi, b.hi, s, e);
    const float lo = a.lo + b.lo + e;
    a.hi = s + lo;
    a.lo = lo - (a.hi - s);
}
__device__ __forceinline__ double df_value(const DF &a) { return double(a.hi) + double(a.lo); }

// ------------------------------------------------------------------ launch helpers
int num_sms();
inline int width_for(int M) { return M <= 16 ? 16 : M <= 32 ? 32 : M <= 64 ? 64 : 128; }

// SpMM epilogue parameters (linear combination, used by gbl/sbl/cheb/cheb2/cbl):
//   out_i[c] = c1[c]*(L x)_i[c] + c0[c]*x_i[c] + c2[c]*y_i[c] + s3*z_i[c] + (marker_i==c)*wE
// c0/c1/c2 come from device arrays (length W) when the pointer is set, else the scalars.
template <typename T>
struct LinEpi {
    const double *a1 = nullptr, *a0 = nullptr, *a2 = nullptr;
    double s1 = 1.0, s0 = 0.0, s2 = 0.0, s3 = 0.0;
    const T *y = nullptr;
    const T *z = nullptr;
    const int32_t *marker = nullptr;
    double wE = 0.0;
    T *out = nullptr;                 // internal n x W output (used when yout is null)
    float *yout = nullptr;            // final FP32 output with leading dimension ldo, mo columns
    double *dot_partials = nullptr;   // [grid][W]: sum_i x_i[c] * out_i[c] (DF pairs when
                                      // the arithmetic is FP32, doubles for FP64)
    const Ctrl *ctrl = nullptr;
    const int32_t *tgen = nullptr;    // frontier tiles (nullptr: all rows)
    const uint8_t *gen = nullptr;     // hop distance per row (with tgen): a warp whose rows
                                      // all lie beyond the limit skips them
    int limit = 0;                    // process tiles with tgen <= limit
    int zero_inactive = 0;            // write zeros for skipped tiles (final output)
    const int32_t *alist = nullptr;   // with tgen: the 32-row frontier tiles with tgen <= limit in
    const int32_t *acount = nullptr;  // increasing order and their number (device); the kernel
                                      // then visits only the row tiles they cover (ignored when
                                      // zero_inactive is set: every tile is written then)
    ProfCount prof;
};

// ldo <= 0: output is an internal n x W block; otherwise out has leading dimension ldo
// and only columns < mo are written.  n_dense_in counts the dense inputs besides x
// (y, z) for the algorithmic byte count.
template <typename T>
int launch_spmm(const GraphDev &g, int W, const T *x, const LinEpi<T> &e, cudaStream_t s,
                int *grid_out, int64_t M_alg, int n_dense_in, int64_t ldo = 0, int mo = 0);
template <typename T>
int spmm_max_grid(int W);

// Tall-skinny row-block kernels (tiled SIMT, FP32 or FP64), W x W matrices row-major:
//   PROJ    : G = Qa^T X                                         (no write)
//   UPD     : out = X - Qa*Ca - Qb*Cb (Qa may be null) ; write ; G = out^T out
//   MULGRAM : out = X*Ca ; write ; G = out^T out
//   MUL     : out = X*Ca ; write
//   ASM     : y[:, :mo] = sum_{k < nblk} basis_k * Ca_k  (Ca stacked nblk*W x W), nblk
//             capped by ctrl->steps
// In-place out == x is allowed (a tile's output rows depend only on its input rows).
//   ASMSUB  : out = X - sum_{k < nblk} basis_k * Ca_k ; write ; G = out^T out
//             (full reorthogonalisation against the stored blocks)
enum RowMode { RB_PROJ = 0, RB_UPD = 1, RB_MULGRAM = 2, RB_MUL = 3, RB_ASM = 4, RB_ASMSUB = 5 };
template <typename T>
struct RowArgs {
    using C = typename Cmp<T>::type;
    int64_t n = 0;
    const T *x = nullptr;
    const T *qa = nullptr;
    const T *qb = nullptr;
    const C *ca = nullptr;
    const C *cb = nullptr;
    T *out = nullptr;
    C *partials = nullptr;          // [grid][W*W]
    const T *basis = nullptr;       // ASM
    int64_t block_stride = 0;
    int nblk = 0;
    float *y = nullptr;
    int64_t ldy = 0;
    int mo = 0;
    const Ctrl *ctrl = nullptr;
    const int32_t *tgen = nullptr;    // frontier tiles (nullptr: all rows)
    int limit = 0;                    // process tiles with tgen <= limit (ASM: all tiles)
    const int32_t *alist = nullptr;   // as LinEpi::alist (not used by ASM, which writes every
    const int32_t *acount = nullptr;  // row of its output)
    int kbase = 0;                    // ASM: index of the first block (frontier reach)
    int accumulate = 0;               // ASM: y += product (the accumulator starts from y)
    const int32_t *skip = nullptr;    // the launch does nothing when *skip != 0 (device flag)
    ProfCount prof;
};
template <typename T>
int launch_rowblock(int mode, int W, const RowArgs<T> &a, cudaStream_t s, int *grid_out,
                    int64_t M_alg);
template <typename T>
int rowblock_max_grid(int W);
// Tensor-core (tcgen05) variant of PROJ, UPD, MULGRAM and MUL for FP32 blocks of width 64
// (rowblock_tc.cu); launch_rowblock uses it where rowblock_tc_supported says so.  Gram
// partials: grid <= max_grid rows of [W*W].
bool rowblock_tc_supported(int mode, int W);
bool rowblock_tc_enabled();   // KB_TENSOR_CORES=1 in the environment
int launch_rowblock_tc(int mode, const RowArgs<float> &a, cudaStream_t s, int max_grid, int *grid_out);
int rowblock_tc_max_grid();

// Host coefficient math shared by the entry points (krylov.cu).  lobatto_coeffs_into: the
// Lobatto interpolation coefficients c_0..c_m of phi (or sqrt(phi)) on [0, lam] into the
// caller's arrays f (samples) and c, m + 1 doubles each, without allocating.  validate_phi:
// KB_OK, or KB_ERR_ARG for a bad kernel choice or non-finite / non-positive parameters.
void lobatto_coeffs_into(kb_phi phi, const kb_params &p, int m, double lam, bool sqrt_phi, double *f,
                         double *c);
int validate_phi(kb_phi phi, const kb_params &p);

// Deterministic FP64 reduction of [nparts][len] partials into out[len]; when out_p is set
// the sums are also written there rounded to P.  Nothing is done when *skip != 0.
template <typename P>
int launch_reduce(const P *parts, int nparts, int len, double *out, cudaStream_t s,
                  const Ctrl *ctrl, P *out_p = nullptr, const int32_t *skip = nullptr);

}  // namespace kb
