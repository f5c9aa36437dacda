/*
 * kb.h -- block Krylov kernel columns phi(L) E_W on one GPU (sm_103a).
 *
 * The library computes approximations of the N kernel columns
 *     Y ~ phi(L) E_W,   E_W = [e_{w_1}, ..., e_{w_N}]                 (Section 3, Eq. (GBFcompute))
 * of a graph Laplacian L (Section 2.1, Eq. (generalizedLaplacian): symmetric, negative
 * off-diagonal entries on edges, spectrum in [0, Lambda]) for the diffusion kernel
 * phi(lambda) = e^{-t lambda} and the variational spline kernel (eps + lambda)^{-s}
 * (Section 2.4), with the five block Krylov methods of Section 3:
 *     KB_CBL   classical block Lanczos               (Algorithm 1)
 *     KB_GBL   global block Lanczos                  (Algorithm 2)
 *     KB_SBL   sequential (column-wise) Lanczos      (Section 3.3)
 *     KB_CHEB  Chebyshev-Lobatto interpolation       (Section 3.4, Eqs. (apprchebyshevseries), (chebcoeff))
 *     KB_CHEB2 squared Chebyshev, PSD by construction (Section 3.4.1)
 *
 * Conventions for every entry point
 *   - The return value is KB_OK (0) on success or a negative KB_ERR_* code.  No C++
 *     exception crosses this boundary.  kb_last_error() gives a thread-local message for
 *     the last failing call on the calling thread.
 *   - Device pointers are plain CUDA device addresses of the current device; host
 *     pointers are ordinary host memory.  `stream` is a cudaStream_t passed as void*
 *     (NULL = the legacy default stream).
 *   - All GPU work of a call is enqueued on `stream`.  A call returns without waiting for
 *     the GPU unless it is documented to synchronise.
 *   - The library never frees memory it does not own and never keeps a caller pointer
 *     beyond the call.
 */
#ifndef KB_H
#define KB_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------------ status codes */
enum {
    KB_OK = 0,
    KB_ERR_ARG = -1,          /* invalid argument (null pointer, size out of range, bad enum)   */
    KB_ERR_CSR = -2,          /* CSR not a valid generalized Laplacian (unsorted, duplicate,
                                 out-of-range column, non-symmetric, positive off-diagonal)   */
    KB_ERR_NODES = -3,        /* node set has an out-of-range or repeated node                  */
    KB_ERR_CUDA = -4,         /* a CUDA runtime call failed (message in kb_last_error)          */
    KB_ERR_NOMEM = -5,        /* device memory exhausted                                         */
    KB_ERR_BREAKDOWN = -6,    /* a Lanczos block became rank deficient (not deflated)            */
    KB_ERR_UNSUPPORTED = -7,  /* combination not implemented (see kb_krylov_apply)               */
    KB_ERR_BUSY = -8,         /* serving queue full (kb_server_submit)                           */
    KB_ERR_ORTHOGONALITY = -9,/* the projected matrix left [0, Lambda]: the Lanczos basis lost
                                 orthogonality (FP32 on graphs whose top eigenvalues converge
                                 fast, e.g. hubs); rerun with params.reorth = 2 or 1            */
    KB_PENDING = 1            /* not an error: the request has not finished (kb_server_poll)     */
};

/* ------------------------------------------------------------------ enums and params */
typedef enum { KB_CBL = 0, KB_GBL = 1, KB_SBL = 2, KB_CHEB = 3, KB_CHEB2 = 4 } kb_method;
typedef enum { KB_PHI_EXP = 0, KB_PHI_SPLINE = 1 } kb_phi;          /* e^{-t L}, (eps I + L)^{-s} */
typedef enum { KB_F32 = 0, KB_BF16 = 1, KB_F64 = 2 } kb_dtype;     /* Krylov basis storage        */

typedef struct {
    double t;           /* diffusion time t (KB_PHI_EXP), any finite value                         */
    double eps;         /* spline shift eps > 0 (KB_PHI_SPLINE)                                    */
    double s;           /* spline exponent s > 0 (KB_PHI_SPLINE)                                   */
    double lambda_max;  /* spectral bound Lambda used by KB_CHEB/KB_CHEB2; <= 0 selects the
                           graph's Gershgorin bound max_i sum_j |L_ij|                            */
    int32_t reorth;     /* KB_CBL only (not in the paper): 0 = none (Algorithm 1
                           as printed); 1 = full: each new block is orthogonalised against all
                           earlier blocks by classical Gram-Schmidt, a second pass only when the
                           first removed more than half of some column's squared norm (Kahan's
                           "twice is enough"); 2 = local: a
                           second Gram-Schmidt pass against the two previous blocks, which keeps
                           the FP32 process on the FP64 one where Ritz values converge fast     */
    int32_t basis;      /* kb_dtype of the stored Krylov blocks: KB_F32 (FP32 arithmetic),
                           KB_BF16 (blocks stored in bfloat16, arithmetic in FP32, small
                           matrices as for KB_F32; relative error of order 1e-3 to 1e-2, set
                           by the bfloat16 rounding of every stored element), KB_F64 (plain
                           FP64 arithmetic throughout); any other value is KB_ERR_ARG         */
    int32_t no_frontier;/* 0 (default): the products and block updates of step k touch only
                           rows within k hops of W (the Krylov blocks are exactly zero
                           elsewhere); 1: every step touches all n rows                           */
    int32_t two_pass;   /* 0 (default): the Krylov basis is stored (m blocks of n x W); 1: the
                           Lanczos methods keep three blocks and run the recurrence twice,
                           the second time with the recorded coefficients, adding each block
                           to Y as it is recomputed (twice the products with L, O(n W) memory
                           instead of the m n W of Table 2).  Not with reorth = 1; no effect
                           for KB_CHEB / KB_CHEB2, which never store a basis                    */
    double tol;         /* KB_CBL only (a stopping rule for serving; the paper fixes m):
                           0 (default) runs m steps.  > 0: m is the largest number of steps;
                           after steps k = 8, 12, 16, 24, 32, 48, 64, 96 (those below m) the
                           projected result U_k = phi(H_k) F_1 is formed in FP64 and the process
                           stops at the first k with ||U_k - [U_k'; 0]||_F <= tol ||U_k||_F,
                           k' the previous such step (info->steps_done = k; the result is then
                           the one of the fixed-m call with m = k).  Not with two_pass        */
} kb_params;

typedef struct {
    int32_t status;          /* KB_OK or KB_ERR_BREAKDOWN                                          */
    int32_t steps_done;      /* products with L whose blocks enter the result (<= m); smaller
                                than m when the Krylov space became invariant (exact result)     */
    int32_t breakdown_step;  /* step of a rank-deficient block, or -1                             */
    int32_t spmm_launches;   /* SpMM kernels launched by the call                                  */
    double  lambda_used;     /* Lambda used for the Chebyshev methods (0 for Lanczos)              */
    double  est_change;      /* KB_CBL with params.tol > 0: ||U_k - [U_k'; 0]||_F / ||U_k||_F at the
                                last stopping-rule check that ran (the estimate of the change of Y
                                since the previous check, Q being orthonormal); -1 when no check
                                compared two results (tol = 0, other methods, m <= 12)           */
} kb_info;

typedef struct kb_graph kb_graph;   /* opaque; owned by the library */

/* ------------------------------------------------------------------ graph */
/*
 * kb_graph_create -- copy a graph Laplacian to the device.          (Section 2.1, Eq. (generalizedLaplacian))
 *
 *   n       number of nodes, 1 <= n < 2^31.
 *   rowptr  host, n+1 int32, rowptr[0] = 0, non-decreasing; row i holds entries
 *           rowptr[i] .. rowptr[i+1]-1 of col/val.
 *   col     host, int32 column indices, strictly increasing within a row, in [0, n).
 *   val     host, float32 values L_ij; off-diagonal entries must be < 0 (edge weight
 *           w_ij = -L_ij), and the matrix must be symmetric (bitwise L_ij == L_ji).  The
 *           diagonal entry may be absent (taken as 0).  NULL means the unit-weight standard
 *           Laplacian D - A of the pattern (diagonal entries of the pattern are ignored).
 *   flags   0, or a sum of KB_GRAPH_SKIP_SYMMETRY_CHECK (skip the O(nnz log deg) symmetry
 *           check) and KB_GRAPH_NORMALIZED (store the normalized Laplacian
 *           I - D^{-1/2} A D^{-1/2} of the graph instead: A = the off-diagonal weights w_ij,
 *           D = diag of the weighted degrees; the given diagonal is ignored; nodes without
 *           edges get a zero row; Lambda = min(Gershgorin, 2) since the spectrum lies in
 *           [0, 2].  The paper uses this Laplacian in Section 8 without defining it.)
 *   stream  stream for the upload and the Lambda reduction; the call synchronises it.
 *   out     receives the handle.
 *
 * The library copies the CSR (the caller keeps ownership of its arrays), stores the
 * off-diagonal part (weights dropped when all are 1) and the diagonal excess
 * L_ii - sum_j w_ij, and computes the Gershgorin bound Lambda = max_i sum_j |L_ij| on the
 * device.  Errors: KB_ERR_ARG, KB_ERR_CSR (validation runs on the host before any CUDA
 * call), KB_ERR_NOMEM, KB_ERR_CUDA.  On error *out is set to NULL.
 */
#define KB_GRAPH_SKIP_SYMMETRY_CHECK 1
#define KB_GRAPH_NORMALIZED 2
int kb_graph_create(int64_t n, const int32_t *rowptr, const int32_t *col, const float *val,
                    int32_t flags, void *stream, kb_graph **out);

/* Release the device copy.  NULL is ignored.  No call using the graph may be in flight. */
void kb_graph_destroy(kb_graph *g);

/* Graph facts: node count, stored off-diagonal entries, Gershgorin Lambda, whether all
 * weights are 1 and the diagonal equals the degree (standard Laplacian).  Any output
 * pointer may be NULL. */
int kb_graph_info(const kb_graph *g, int64_t *n, int64_t *nnz_offdiag, double *lambda_max,
                  int32_t *standard_unit);

/* Spectral upper bounds of the graph (host values, no GPU work): gershgorin =
 * max_i sum_j |L_ij| (the Lambda of the Chebyshev methods); projected = the bound
 * the Lanczos methods use for their projected e^{-tH} series (Algorithms 1 and 2 need
 * phi(H_m), whose spectrum lies in [0, lambda_max(L)]): for the unit-weight standard
 * Laplacian D - A the edge bound max over edges (d_i + d_j) of Anderson and Morley when
 * smaller, otherwise gershgorin.  Either pointer may be NULL. */
int kb_graph_lambda_bounds(const kb_graph *g, double *gershgorin, double *projected);

/* ------------------------------------------------------------------ kernel columns */
/*
 * kb_krylov_apply -- Y ~ phi(L) E_W by one block Krylov method.   (Section 3; Algorithms 1, 2)
 *
 *   method  kb_method.  phi: kb_phi with parameters in *params.
 *   nodes   host, M distinct node indices in [0, n) (0-based).
 *   M       block width N of the paper, 1 <= M <= 128 for KB_CBL and KB_GBL; any M >= 1
 *           for KB_SBL, KB_CHEB, KB_CHEB2 (columns are independent and processed in
 *           groups of at most 128).
 *   m       number of products with L (block SpMMs), m >= 1 (KB_CHEB2: m >= 2).  The
 *           Lanczos methods return the degree m-1 polynomial p_{phi,m-1} (Algorithm 1,
 *           final step); KB_CHEB returns the degree-m interpolant; KB_CHEB2 the square of the
 *           degree floor(m/2) interpolant of sqrt(phi).
 *   Y       device, n x M float32, row-major with leading dimension M (Y[i*M + j] is
 *           entry (node i, column j)); written completely; caller-owned.
 *   stream  all work is enqueued here; scratch memory is taken from and returned to the
 *           device's stream-ordered memory pool on this stream.
 *   info    NULL, or receives facts about the run.  When non-NULL the call synchronises
 *           `stream` and returns KB_ERR_BREAKDOWN if the Lanczos process met a
 *           rank-deficient block, or KB_ERR_ORTHOGONALITY if phi(H_m) F_1 exceeds the bound
 *           max phi on [0, Lambda] (the projected matrix left the spectral interval); Y is
 *           then filled with NaN.  With info == NULL the call does not synchronise, and
 *           these failures show only as NaN in Y.
 *
 * Spline kernel with the Lanczos methods: phi(H_m) F_1 = (eps I + H_m)^{-s} F_1 is formed by
 * floor(s) block Cholesky solves with eps I + H_m and, for non-integer s, a quadrature of
 * the fractional power over real shifts sigma_k > eps (Gauss-Jacobi rule of the Stieltjes
 * integral of z^{-alpha}, relative accuracy 1e-14 on [0, Lambda]), one solve with
 * sigma_k I + H_m per node (kb_spline_quadrature gives the rule).
 *
 * Not implemented (KB_ERR_UNSUPPORTED): the Lanczos methods with KB_PHI_SPLINE and s >= 65,
 * or with (eps + Lambda) / eps so large that 240 quadrature nodes do not reach 1e-14;
 * reorth with methods other than KB_CBL; KB_CBL / KB_GBL with M > 128 (M > 64 for KB_F64).
 * Other errors: KB_ERR_ARG, KB_ERR_NODES, KB_ERR_NOMEM, KB_ERR_CUDA (also when an opt-in
 * tensor-core kernel gives up waiting for its MMA completion).
 *
 * Environment: KB_TENSOR_CORES=1 (read at every launch) runs the tall-skinny products of
 * KB_CBL with FP32 blocks of width 64 (M in 33..64) on the tcgen05 tensor cores (BF16 x 6
 * split products, FP32 accumulation).  It is not the default: with the frontier restriction
 * it is slower than the SIMT kernels, and on sensitive kernels its error is several times
 * theirs (e.g. (0.1 I + L)^{-2}: 8.6e-5 against 2.0e-5 on a 2e4-node RGG).
 */
int kb_krylov_apply(kb_graph *g, kb_method method, kb_phi phi, const kb_params *params,
                    const int32_t *nodes, int32_t M, int32_t m, float *Y, void *stream,
                    kb_info *info);

/*
 * kb_krylov_apply_host -- the same computation with the result in HOST memory.
 *
 * Y_host is host memory of n x M float32 (row-major, leading dimension M); pinned memory
 * (cudaHostAlloc / cudaHostRegister) gives an asynchronous DMA, pageable memory works but
 * is staged by the CUDA runtime.  The call allocates the device result from the
 * stream-ordered pool, runs kb_krylov_apply, copies the result to Y_host and synchronises
 * `stream` before returning.  Errors as kb_krylov_apply.
 */
int kb_krylov_apply_host(kb_graph *g, kb_method method, kb_phi phi, const kb_params *params,
                         const int32_t *nodes, int32_t M, int32_t m, float *Y_host,
                         void *stream, kb_info *info);

/*
 * kb_cheb_apply_fixed_scratch -- KB_CHEB without any memory allocation.
 *
 * The paper has no counterpart of this call.  It serves callers that cannot allocate
 * device memory when they need kernel columns: code running inside a framework that has
 * reserved the device memory for its own allocator, latency-critical loops that must not
 * enter an allocator after start-up, and processes sharing a device under a fixed memory
 * budget.  It computes exactly what kb_krylov_apply(g, KB_CHEB, phi, params, nodes, M, m,
 * Y, stream, NULL) computes, bit for bit: it runs the same SpMM kernel with the same
 * coefficients on every row at every step (KB_CHEB also skips rows beyond the frontier,
 * whose values are exactly zero).  Its scratch is a file-scope device array of
 * KB_FIXED_SCRATCH_BYTES (32 MiB) that every GPU loading the library holds until the
 * process exits; the call performs no cudaMalloc, cudaMallocAsync
 * or cudaFree and calls no allocating library routine.
 *
 *   Arguments as kb_krylov_apply, restricted to 1 <= M <= 128, 1 <= m <= 1024 and
 *   params->basis == KB_F32.  The scratch needed is 3 * n * W * 4 bytes (each block rounded
 *   up to 256 bytes) plus 4 * n bytes, W = M rounded up to 16/32/64/128; a larger problem
 *   is rejected with KB_ERR_ARG and a message giving both sizes, before any GPU work.
 *   The first call on a device looks up the array's device address
 *   (cudaGetSymbolAddress) with that device current; make that first call before any
 *   stream capture.  All calls in the process share the one array, and every call
 *   rewrites the parts it reads before reading them: calls whose GPU work overlaps (other
 *   streams, other threads) race on the scratch and must be serialised by the caller.
 *   Does not synchronise; errors: KB_ERR_ARG, KB_ERR_NODES, KB_ERR_UNSUPPORTED,
 *   KB_ERR_CUDA.
 */
#define KB_FIXED_SCRATCH_BYTES (32u << 20)
int kb_cheb_apply_fixed_scratch(kb_graph *g, kb_phi phi, const kb_params *params,
                                const int32_t *nodes, int32_t M, int32_t m, float *Y,
                                void *stream);

/* ------------------------------------------------------------------ diagnostics */
/* Static text for a status code. */
const char *kb_status_string(int status);
/* Message of the last failing call on this thread ("" if none). */
const char *kb_last_error(void);
/* Library version, major*10000 + minor*100 + patch. */
int kb_version(void);

/* ------------------------------------------------------------------ host coefficient math
 * These run on the host only (no CUDA call) and expose the scalar preprocessing of the
 * Chebyshev steps so that it can be checked without a GPU. */

/* Coefficients c_0..c_m of the degree-m Chebyshev-Lobatto interpolant of phi (or of
 * sqrt(phi) when sqrt_phi != 0) on [0, lam], Eq. (chebcoeff) read as
 * c_k = (2/m) sum''_{j=0..m} phi(lam/2 (1 - cos(pi j/m))) cos(pi j k/m) (endpoint terms
 * halved); the interpolant is sum''_k c_k T_k(1 - 2 lambda/lam) with c_0 and
 * c_m halved.  c: host array of m+1 doubles.  Errors: KB_ERR_ARG. */
int kb_cheb_lobatto_coeffs(kb_phi phi, const kb_params *params, int32_t m, double lam,
                           int32_t sqrt_phi, double *c);

/* Chebyshev series e^{-t lambda} = sum_k d_k T_k(1 - 2 lambda/lam) on [0, lam] (no
 * halving), truncated where |d_k| <= tol * sum |d|; used for phi(H_m) of the Lanczos
 * methods.  d: host array of cap doubles; *count receives the number of terms (the call
 * fails with KB_ERR_ARG when it exceeds cap). */
int kb_exp_series_coeffs(double t, double lam, double tol, double *d, int32_t cap,
                         int32_t *count);

/* Quadrature form of the spline kernel for non-integer s (Section 2.4), as the Lanczos methods
 * use it: (eps + lambda)^{-s} ~ (eps + lambda)^{-s_int} sum_k weight_k / (shift_k + lambda) on
 * [0, lam], s_int = floor(s), relative error <= tol (checked on a grid of [0, lam]).  The
 * nodes are a Gauss-Jacobi rule of the Stieltjes integral
 * z^{-alpha} = sin(pi alpha)/pi int_0^inf t^{-alpha} / (t + z) dt, alpha = s - s_int, after
 * the substitution t = c ((1-x)/(1+x))^3, c = sqrt(eps (eps + lam)).  shift, weight: host
 * arrays of cap doubles; *count receives the number of nodes (0 for integer s), *s_int
 * floor(s).  Errors: KB_ERR_ARG (bad arguments, cap too small), KB_ERR_UNSUPPORTED (240
 * nodes do not reach tol). */
int kb_spline_quadrature(double eps, double s, double lam, double tol, double *shift, double *weight,
                         int32_t cap, int32_t *count, int32_t *s_int);

/* ------------------------------------------------------------------ measurement aids
 * Optional CUDA-event timing of every kernel launch class (not part of the method).
 * While enabled, each launch of a class is bracketed by events on its stream; reading
 * synchronises those events, returns per-class totals and clears the record. */
typedef struct {
    int32_t kernel_class;   /* 0 spmm, 1 rowblock, 2 reduce, 3 small_fp64, 4 projected_fp64,
                               5 assemble, 6 other                                           */
    int32_t launches;
    double total_ms;        /* summed event durations                                         */
    double alg_bytes;       /* algorithmic HBM bytes of those launches                        */
    double alg_flops;       /* algorithmic flops of those launches                            */
} kb_kernel_stats;
int kb_profile_enable(int32_t on);
int kb_profile_read(kb_kernel_stats *out, int32_t cap, int32_t *count);
const char *kb_kernel_class_name(int32_t cls);
/* Number of CUDA kernels this library has launched in the process so far. */
int64_t kb_launch_counter(void);

/* ------------------------------------------------------------------ RLS predictor
 * Regularised least-squares kernel predictor from approximated kernel columns (Section 5,
 * Eq. (computationcoefficientskrylov); Algorithm 3 for KB_CBL, whose collocation matrix
 * E_W^T Y equals F_1^T phi(H_m) F_1 by the proof of Theorem 3.1):
 *     Y = p_{phi,m-1}^{(kr)}(L) E_W            (as kb_krylov_apply, into library scratch)
 *     (E_W^T Y + gamma M I) c = labels         (FP64 LU with partial pivoting on the device)
 *     y_pred = Y c                             (device, n float32, caller-owned)
 * labels: host, M doubles (label of node nodes[i]); gamma >= 0 (gamma = 0: interpolation);
 * c_host: NULL or host, M doubles receiving c.  M <= 128.  The call synchronises `stream`.
 * Errors: as kb_krylov_apply; KB_ERR_BREAKDOWN when E_W^T Y + gamma M I is numerically
 * singular (possible for gbl, sbl and cheb at small m, Section 8.3; never for cbl). */
int kb_rls_predict(kb_graph *g, kb_method method, kb_phi phi, const kb_params *params,
                   const int32_t *nodes, int32_t M, int32_t m, const double *labels,
                   double gamma, float *y_pred, double *c_host, void *stream, kb_info *info);

/* ------------------------------------------------------------------ scratch size */
/* Bytes of device scratch one kb_krylov_apply call with these arguments takes from the
 * stream-ordered pool (the result Y excluded).  Host-only; validates the arguments as
 * kb_krylov_apply does, except the node list. */
int kb_workspace_bytes(kb_graph *g, kb_method method, kb_phi phi, const kb_params *params,
                       int32_t M, int32_t m, uint64_t *bytes);

/* ------------------------------------------------------------------ serving
 * A request queue over kb_krylov_apply for many independent kernel-column requests (the
 * serving use of Section 3's methods; the paper has no serving layer).
 *
 * kb_server_create starts `streams` host worker threads on `device`, each owning one CUDA
 * stream.  Requests start in submission order; a worker starts the oldest pending request
 * once its scratch (kb_workspace_bytes) fits in `memory_budget` next to the requests in
 * flight (memory_budget <= 0: three quarters of the device memory available at creation,
 * free memory plus what the stream-ordered pool holds unused), runs
 * it on its stream and waits for it, so at most `streams` solves run concurrently and
 * requests may complete out of order.
 *
 * kb_server_submit copies the node list and the parameters; the caller keeps `g` alive
 * and must not touch the device array Y (n x M float32, as for kb_krylov_apply) until the
 * request has been polled as finished.  It returns a ticket, or KB_ERR_BUSY when
 * queue_capacity requests are pending or unpolled, or KB_ERR_NOMEM when the request alone
 * exceeds the memory budget.  Argument errors of the solve itself are reported by poll.
 *
 * kb_server_poll waits up to wait_ms milliseconds (0: do not wait, < 0: wait until done).
 * It returns KB_PENDING while the request runs or waits, otherwise the solve's status; a
 * finished request is reported once (its ticket is then forgotten).  info (nullable)
 * receives the solve's kb_info, latency_ms (nullable) the host time from submit to the end
 * of the solve.  kb_server_destroy runs every submitted request to completion, then stops
 * the workers and destroys the streams.  All four functions may be called from any host
 * thread. */
typedef struct kb_server kb_server;
typedef struct {
    int32_t streams;         /* concurrent solves, 1..64                                          */
    int32_t queue_capacity;  /* maximum requests submitted and not yet polled as finished         */
    int64_t memory_budget;   /* bytes of scratch the running requests may hold together          */
    int32_t fallback_sbl;    /* 1: a KB_CBL or KB_GBL request whose block becomes rank deficient
                                (KB_ERR_BREAKDOWN, e.g. nodes whose neighbourhoods are tiny
                                components) is run again as KB_SBL, one Lanczos process per
                                column, which has no block rank deficiency (reorth off, all m
                                steps; only when its scratch fits the request's admission); poll
                                then reports the KB_SBL status, with info->breakdown_step set to
                                the step of the block breakdown.  0: the breakdown is reported. */
} kb_server_config;
int kb_server_create(int32_t device, const kb_server_config *cfg, kb_server **out);
int kb_server_submit(kb_server *sv, kb_graph *g, kb_method method, kb_phi phi,
                     const kb_params *params, const int32_t *nodes, int32_t M, int32_t m,
                     float *Y, int64_t *ticket);
int kb_server_poll(kb_server *sv, int64_t ticket, int32_t wait_ms, kb_info *info,
                   double *latency_ms);
int kb_server_destroy(kb_server *sv);

#ifdef __cplusplus
}
#endif
#endif /* KB_H */
