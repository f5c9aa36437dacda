// Block SpMM with the Laplacian: out = epilogue(L x), x an n x W row-major block.
//
// This is the "MV" of Table 1 (Section 7), the operation the paper names the most
// expensive for large graphs; every method performs m of them per solve.
//
// Schedule (GB300).  A row of x is W elements; W/4 lanes cover it with one 16-byte
// vector each (float4, or 2 x double2), so a warp works on 32/(W/4) rows at once, one
// lane group per row.  A group first loads up to W/4 column indices (and weights) of its
// row with one coalesced load, then walks them U at a time: the U neighbour rows are
// gathered with independent 16-byte loads before any is consumed, which keeps 4 x 16 B
// per lane in flight instead of one dependent index->row chain.  Groups of a warp run
// different rows and never wait for each other (group-masked shuffles).  The grid is
// persistent (a multiple of the SM count).
//
// The Laplacian is applied in difference form (L x)_i = sum_j w_ij (x_i - x_j) + r_i x_i,
// which gives L 1 = 0 exactly for D - A and drops the diagonal load for standard
// Laplacians.  Epilogue coefficients arrive in FP64; in the FP32 path each is split into
// a float pair (hi + lo) so that c * (L x) carries only the rounding of the final sum.
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

template <typename T>
__device__ __forceinline__ void split(double d, T &hi, T &lo) {
    hi = T(d);
    lo = T(d - double(hi));
}

constexpr int SPMM_THREADS = 256;
constexpr int UNROLL = 4;

template <typename T, int W>
__global__ void __launch_bounds__(SPMM_THREADS)
k_spmm(GraphDev g, const T *__restrict__ x, LinEpi<T> e, int64_t ldo, int mo) {
    constexpr int LPR = W / 4;       // lanes per row
    constexpr int RPW = 32 / LPR;    // rows per warp
    if (e.ctrl && e.ctrl->stop) return;
    __shared__ double sdot[SPMM_THREADS / 32][W];
    const int lane = threadIdx.x & 31;
    const int sub = lane % LPR;
    const int grp = lane / LPR;
    const int c4 = sub * 4;
    const unsigned gmask = (LPR == 32) ? 0xffffffffu : (((1u << LPR) - 1u) << (grp * LPR));
    T c1h[4], c1l[4], c0[4], c2h[4], c2l[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        split<T>(e.a1 ? e.a1[c4 + q] : e.s1, c1h[q], c1l[q]);
        c0[q] = T(e.a0 ? e.a0[c4 + q] : e.s0);
        split<T>(e.a2 ? e.a2[c4 + q] : e.s2, c2h[q], c2l[q]);
    }
    const T s3 = T(e.s3);
    const T wE = T(e.wE);
    const int64_t warp = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = (int64_t(gridDim.x) * blockDim.x) >> 5;
    T dot[4] = {0, 0, 0, 0};

    for (int64_t base = warp * RPW; base < g.n; base += nwarps * RPW) {
        const int64_t row = base + grp;
        const bool active = row < g.n;
        const int beg = active ? __ldg(g.rowptr + row) : 0;
        const int end = active ? __ldg(g.rowptr + row + 1) : 0;
        V4<T> xi;
        if (active) xi = V4<T>::load(x + row * W + c4);
        else {
#pragma unroll
            for (int q = 0; q < 4; ++q) xi.v[q] = T(0);
        }
        T acc[4] = {0, 0, 0, 0};
        for (int p0 = beg; p0 < end; p0 += LPR) {
            const int myp = p0 + sub;
            const int jj = myp < end ? __ldg(g.col + myp) : 0;
            const T ww = (myp < end && g.w) ? T(__ldg(g.w + myp)) : T(1);
            const int cnt = min(LPR, end - p0);
            for (int q0 = 0; q0 < cnt; q0 += UNROLL) {
                int j[UNROLL];
                T wv[UNROLL];
#pragma unroll
                for (int u = 0; u < UNROLL; ++u) {
                    const int src = grp * LPR + min(q0 + u, LPR - 1);
                    j[u] = __shfl_sync(gmask, jj, src);
                    wv[u] = __shfl_sync(gmask, ww, src);
                }
                V4<T> xj[UNROLL];
#pragma unroll
                for (int u = 0; u < UNROLL; ++u)
                    if (q0 + u < cnt) xj[u] = V4<T>::load(x + int64_t(j[u]) * W + c4);
#pragma unroll
                for (int u = 0; u < UNROLL; ++u)
                    if (q0 + u < cnt)
#pragma unroll
                        for (int q = 0; q < 4; ++q) acc[q] = fma(wv[u], xi.v[q] - xj[u].v[q], acc[q]);
            }
        }
        if (!active) continue;
        if (g.rdiag) {
            const T r = T(__ldg(g.rdiag + row));
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[q] = fma(r, xi.v[q], acc[q]);
        }
        T o[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) o[q] = fma(c1h[q], acc[q], fma(c1l[q], acc[q], c0[q] * xi.v[q]));
        if (e.y) {
            const V4<T> yi = V4<T>::load(e.y + row * W + c4);
#pragma unroll
            for (int q = 0; q < 4; ++q) o[q] = fma(c2h[q], yi.v[q], fma(c2l[q], yi.v[q], o[q]));
        }
        if (e.z) {
            const V4<T> zi = V4<T>::load(e.z + row * W + c4);
#pragma unroll
            for (int q = 0; q < 4; ++q) o[q] = fma(s3, zi.v[q], o[q]);
        }
        if (e.marker) {
            const int mk = __ldg(e.marker + row);
            if (mk >= c4 && mk < c4 + 4) o[mk - c4] += wE;
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
    if (e.dot_partials) {
        double dd[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            dd[q] = double(dot[q]);
#pragma unroll
            for (int off = LPR; off < 32; off <<= 1) dd[q] += __shfl_xor_sync(0xffffffffu, dd[q], off);
        }
        const int wib = threadIdx.x >> 5;
        if (grp == 0)
#pragma unroll
            for (int q = 0; q < 4; ++q) sdot[wib][c4 + q] = dd[q];
        __syncthreads();
        for (int c = threadIdx.x; c < W; c += blockDim.x) {
            double s = 0.0;
            for (int w2 = 0; w2 < SPMM_THREADS / 32; ++w2) s += sdot[w2][c];
            e.dot_partials[int64_t(blockIdx.x) * W + c] = s;
        }
    }
}

template <typename T, int W>
int occupancy_spmm() {
    static int per_sm = -1;
    if (per_sm < 0) {
        int v = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, k_spmm<T, W>, SPMM_THREADS, 0);
        per_sm = v < 1 ? 1 : v;
    }
    return per_sm;
}

template <typename T, int W>
int launch_w(const GraphDev &g, const T *x, const LinEpi<T> &e, int64_t ldo, int mo,
             cudaStream_t s, int *grid_out) {
    constexpr int RPB = (SPMM_THREADS / 32) * (32 / (W / 4));   // rows per block pass
    const int64_t need = (g.n + RPB - 1) / RPB;
    int grid = int(std::min<int64_t>(need, int64_t(num_sms()) * occupancy_spmm<T, W>()));
    if (grid < 1) grid = 1;
    if (grid_out) *grid_out = grid;
    k_spmm<T, W><<<grid, SPMM_THREADS, 0, s>>>(g, x, e, ldo, mo);
    return 0;
}

}  // namespace

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
    // the other dense inputs once each, the output once; flops 3 per nonzero per column
    double csr = 4.0 * double(g.n + 1) + 4.0 * double(g.nnz) + (g.w ? 4.0 * double(g.nnz) : 0.0) +
                 (g.rdiag ? 4.0 * double(g.n) : 0.0);
    double blk = double(g.n) * double(M_alg) * double(sizeof(T));
    prof_end(KernelClass::SPMM, s, csr + blk * (2 + n_dense_in),
             3.0 * double(g.nnz) * double(M_alg));
    return 0;
}

template <typename T>
int spmm_max_grid(int W) {
    switch (W) {
        case 16: return num_sms() * occupancy_spmm<T, 16>();
        case 32: return num_sms() * occupancy_spmm<T, 32>();
        case 64: return num_sms() * occupancy_spmm<T, 64>();
        default: return num_sms() * occupancy_spmm<T, 128>();
    }
}

template int launch_spmm<float>(const GraphDev &, int, const float *, const LinEpi<float> &,
                                cudaStream_t, int *, int64_t, int, int64_t, int);
template int launch_spmm<double>(const GraphDev &, int, const double *, const LinEpi<double> &,
                                 cudaStream_t, int *, int64_t, int, int64_t, int);
template int spmm_max_grid<float>(int);
template int spmm_max_grid<double>(int);

}  // namespace kb
