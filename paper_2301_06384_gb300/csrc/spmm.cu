// Block SpMM with the Laplacian: out = epilogue(L x), x an n x W row-major block.
//
// This is the "MV" of Table 1 (Section 7), the operation the paper names the most
// expensive for large graphs; every method performs m of them per solve.
//
// Layout and schedule (GB300): one warp per row.  The W columns of a row are split into
// float4 (or 2 x double2) chunks, W/4 lanes cover one row of x, and the 32/(W/4) lane
// groups of the warp walk the row's neighbours in parallel, each group gathering one full
// neighbour row with 16-byte loads.  The groups are reduced with xor shuffles, so every
// group ends with (L x)_i for its 4 columns; group 0 applies the fused epilogue and
// stores.  The grid is persistent (a multiple of the SM count) and strides over rows.
//
// The Laplacian is applied in difference form (L x)_i = sum_j w_ij (x_i - x_j) + r_i x_i,
// which gives L 1 = 0 exactly for D - A and drops the diagonal load for standard
// Laplacians.
#include "kb_internal.cuh"

namespace kb {
namespace {

template <typename T> struct V4;
template <> struct V4<float> {
    float v[4];
    __device__ __forceinline__ static V4 load(const float *p) {
        float4 t = __ldg(reinterpret_cast<const float4 *>(p));
        return V4{{t.x, t.y, t.z, t.w}};
    }
    __device__ __forceinline__ void store(float *p) const {
        *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
    }
};
template <> struct V4<double> {
    double v[4];
    __device__ __forceinline__ static V4 load(const double *p) {
        double2 a = __ldg(reinterpret_cast<const double2 *>(p));
        double2 b = __ldg(reinterpret_cast<const double2 *>(p + 2));
        return V4{{a.x, a.y, b.x, b.y}};
    }
    __device__ __forceinline__ void store(double *p) const {
        reinterpret_cast<double2 *>(p)[0] = make_double2(v[0], v[1]);
        reinterpret_cast<double2 *>(p)[1] = make_double2(v[2], v[3]);
    }
};

constexpr int SPMM_THREADS = 256;

template <typename T, int W>
__global__ void __launch_bounds__(SPMM_THREADS)
k_spmm(GraphDev g, const T *__restrict__ x, LinEpi<T> e, int64_t ldo, int mo) {
    constexpr int LPR = W / 4;       // lanes per row
    constexpr int G = 32 / LPR;      // neighbour slots per warp
    if (e.ctrl && e.ctrl->stop) return;
    __shared__ float sc1[W], sc0[W], sc2[W];
    __shared__ double sdot[SPMM_THREADS / 32][W];
    for (int c = threadIdx.x; c < W; c += blockDim.x) {
        sc1[c] = e.a1 ? e.a1[c] : e.s1;
        sc0[c] = e.a0 ? e.a0[c] : e.s0;
        sc2[c] = e.a2 ? e.a2[c] : e.s2;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int grp = lane / LPR;
    const int c4 = (lane % LPR) * 4;
    const int64_t warp = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = (int64_t(gridDim.x) * blockDim.x) >> 5;
    T dot[4] = {0, 0, 0, 0};
    T c1[4], c0[4], c2[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) { c1[q] = sc1[c4 + q]; c0[q] = sc0[c4 + q]; c2[q] = sc2[c4 + q]; }
    const T s3 = T(e.s3);

    for (int64_t row = warp; row < g.n; row += nwarps) {
        const int beg = __ldg(g.rowptr + row);
        const int end = __ldg(g.rowptr + row + 1);
        const V4<T> xi = V4<T>::load(x + row * W + c4);
        T acc[4] = {0, 0, 0, 0};
        for (int p = beg + grp; p < end; p += G) {
            const int j = __ldg(g.col + p);
            const T w = g.w ? T(__ldg(g.w + p)) : T(1);
            const V4<T> xj = V4<T>::load(x + int64_t(j) * W + c4);
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[q] = fma(w, xi.v[q] - xj.v[q], acc[q]);
        }
#pragma unroll
        for (int off = LPR; off < 32; off <<= 1)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[q] += __shfl_xor_sync(0xffffffffu, acc[q], off);
        if (g.rdiag) {
            const T r = T(__ldg(g.rdiag + row));
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[q] = fma(r, xi.v[q], acc[q]);
        }
        if (grp == 0) {
            T o[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) o[q] = c1[q] * acc[q] + c0[q] * xi.v[q];
            if (e.y) {
                const V4<T> yi = V4<T>::load(e.y + row * W + c4);
#pragma unroll
                for (int q = 0; q < 4; ++q) o[q] = fma(c2[q], yi.v[q], o[q]);
            }
            if (e.z) {
                const V4<T> zi = V4<T>::load(e.z + row * W + c4);
#pragma unroll
                for (int q = 0; q < 4; ++q) o[q] = fma(s3, zi.v[q], o[q]);
            }
            if (e.marker) {
                const int mk = __ldg(e.marker + row);
                if (mk >= c4 && mk < c4 + 4) o[mk - c4] += T(e.wE);
            }
            if (!e.yout) {
                V4<T> ov;
#pragma unroll
                for (int q = 0; q < 4; ++q) ov.v[q] = o[q];
                ov.store(e.out + row * W + c4);
            } else {
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    if (c4 + q < mo) e.yout[row * ldo + c4 + q] = float(o[q]);
            }
            if (e.dot_partials) {
#pragma unroll
                for (int q = 0; q < 4; ++q) dot[q] = fma(xi.v[q], o[q], dot[q]);
            }
        }
    }
    if (e.dot_partials) {
        const int wib = threadIdx.x >> 5;
        if (grp == 0)
#pragma unroll
            for (int q = 0; q < 4; ++q) sdot[wib][c4 + q] = double(dot[q]);
        __syncthreads();
        for (int c = threadIdx.x; c < W; c += blockDim.x) {
            double s = 0.0;
            for (int w2 = 0; w2 < SPMM_THREADS / 32; ++w2) s += sdot[w2][c];
            e.dot_partials[int64_t(blockIdx.x) * W + c] = s;
        }
    }
}

template <typename T, int W>
int launch_w(const GraphDev &g, const T *x, const LinEpi<T> &e, int64_t ldo, int mo,
             cudaStream_t s, int *grid_out) {
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_spmm<T, W>, SPMM_THREADS, 0);
    if (per_sm < 1) per_sm = 1;
    int64_t need = (g.n + (SPMM_THREADS / 32) - 1) / (SPMM_THREADS / 32);
    int grid = int(std::min<int64_t>(need, int64_t(num_sms()) * per_sm));
    if (grid < 1) grid = 1;
    if (grid_out) *grid_out = grid;
    k_spmm<T, W><<<grid, SPMM_THREADS, 0, s>>>(g, x, e, ldo, mo);
    return 0;
}

}  // namespace

// Maximum grid of the SpMM (size of its dot-partial buffer), per W.
template <typename T>
int spmm_max_grid(int W);

template <typename T>
int launch_spmm(const GraphDev &g, int W, const T *x, const LinEpi<T> &e, cudaStream_t s,
                int *grid_out, int64_t M_alg, int n_dense_in, int64_t ldo, int mo) {
    if (ldo <= 0) { ldo = W; mo = W; }
    prof_begin(KernelClass::SPMM, s);
    switch (W) {
        case 16: launch_w<T, 16>(g, x, e, ldo, mo, s, grid_out); break;
        case 32: launch_w<T, 32>(g, x, e, ldo, mo, s, grid_out); break;
        case 64: launch_w<T, 64>(g, x, e, ldo, mo, s, grid_out); break;
        case 128: launch_w<T, 128>(g, x, e, ldo, mo, s, grid_out); break;
        default: return fail(KB_ERR_ARG, "unsupported block width");
    }
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) return cuda_fail(err, "k_spmm launch");
    // algorithmic bytes: CSR (+weights, +diagonal excess) once, the gathered block once,
    // the other dense inputs once each, the output once; flops 2 per nonzero per column
    double csr = 4.0 * double(g.n + 1) + 4.0 * double(g.nnz) + (g.w ? 4.0 * double(g.nnz) : 0.0) +
                 (g.rdiag ? 4.0 * double(g.n) : 0.0);
    double blk = double(g.n) * double(M_alg) * double(sizeof(T));
    prof_end(KernelClass::SPMM, s, csr + blk * (2 + n_dense_in),
             3.0 * double(g.nnz) * double(M_alg));
    return 0;
}

template <typename T>
int spmm_max_grid(int W) {
    int per_sm = 0;
    switch (W) {
        case 16: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_spmm<T, 16>, SPMM_THREADS, 0); break;
        case 32: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_spmm<T, 32>, SPMM_THREADS, 0); break;
        case 64: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_spmm<T, 64>, SPMM_THREADS, 0); break;
        default: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_spmm<T, 128>, SPMM_THREADS, 0); break;
    }
    if (per_sm < 1) per_sm = 1;
    return num_sms() * per_sm;
}

template int launch_spmm<float>(const GraphDev &, int, const float *, const LinEpi<float> &,
                                cudaStream_t, int *, int64_t, int, int64_t, int);
template int launch_spmm<double>(const GraphDev &, int, const double *, const LinEpi<double> &,
                                 cudaStream_t, int *, int64_t, int, int64_t, int);
template int spmm_max_grid<float>(int);
template int spmm_max_grid<double>(int);

}  // namespace kb
