// Tall-skinny block kernels of the classical block Lanczos step (Algorithm 1: diagonal
// block, three-term update, reduced QR) and of its final assembly: products of n x W
// blocks with W x W matrices and Gram matrices A^T B of n x W blocks.
//
// One CTA of 256 threads owns a tile of TR = 4096/W consecutive rows (16 KB of FP32) at
// a time and walks tiles with a persistent grid-stride loop.  Products are K-chunked:
// 16 columns of the left operand are staged transposed in shared memory next to 16 rows
// of the small matrix, and each thread accumulates a 4 x 4 register tile.  The resulting
// tile is written to HBM and kept in shared memory, where each thread adds its
// (W/16) x (W/16) share of the tile's Gram contribution.  In the FP32 path the Gram is
// accumulated in two levels (per tile, then across tiles) to keep the rounding growth of
// long sums small; each CTA writes its partial Gram, and the partials are summed in FP64
// by k_reduce in a fixed order (deterministic).
#include <type_traits>

#include "kb_internal.cuh"

#include <algorithm>
#include <cstdlib>

namespace kb {
namespace {

constexpr int RB_THREADS = 256;
constexpr int KC = 16;

template <typename T>
__device__ __forceinline__ void ld4(const T *p, T (&v)[4]);
template <>
__device__ __forceinline__ void ld4<float>(const float *p, float (&v)[4]) {
    float4 t = *reinterpret_cast<const float4 *>(p);
    v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
}
template <>
__device__ __forceinline__ void ld4<double>(const double *p, double (&v)[4]) {
    double2 a = reinterpret_cast<const double2 *>(p)[0];
    double2 b = reinterpret_cast<const double2 *>(p)[1];
    v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}
template <typename T>
__device__ __forceinline__ void st4(T *p, const T (&v)[4]);
template <>
__device__ __forceinline__ void st4<float>(float *p, const float (&v)[4]) {
    *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
template <>
__device__ __forceinline__ void st4<double>(double *p, const double (&v)[4]) {
    reinterpret_cast<double2 *>(p)[0] = make_double2(v[0], v[1]);
    reinterpret_cast<double2 *>(p)[1] = make_double2(v[2], v[3]);
}

// Global block access: load 4 stored elements widened to the compute type, store narrowed.
template <typename T>
__device__ __forceinline__ void ldg4(const T *p, typename Cmp<T>::type (&v)[4]) { ld4<T>(p, v); }
template <>
__device__ __forceinline__ void ldg4<__nv_bfloat16>(const __nv_bfloat16 *p, float (&v)[4]) {
    const uint2 raw = *reinterpret_cast<const uint2 *>(p);
    const float2 a = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&raw.x));
    const float2 b = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&raw.y));
    v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}
template <typename T>
__device__ __forceinline__ void stg4(T *p, const typename Cmp<T>::type (&v)[4]) { st4<T>(p, v); }
template <>
__device__ __forceinline__ void stg4<__nv_bfloat16>(__nv_bfloat16 *p, const float (&v)[4]) {
    const __nv_bfloat162 a = __floats2bfloat162_rn(v[0], v[1]);
    const __nv_bfloat162 b = __floats2bfloat162_rn(v[2], v[3]);
    uint2 raw;
    raw.x = *reinterpret_cast<const unsigned int *>(&a);
    raw.y = *reinterpret_cast<const unsigned int *>(&b);
    *reinterpret_cast<uint2 *>(p) = raw;
}

template <typename T, int W>
struct Geo {
    static constexpr int TR = 4096 / W;     // rows per tile
    static constexpr int CG = W / 4;        // float4 column groups
    static constexpr int GR = W / 16;       // Gram sub-block edge per thread
    static constexpr int LDA = TR + 4;      // transposed A chunk row stride
    static constexpr int LDO = W + 4;       // out tile row stride
    static constexpr size_t smem_a = sizeof(typename Cmp<T>::type) * KC * LDA;
    static constexpr size_t smem_c = sizeof(typename Cmp<T>::type) * KC * W;
    static constexpr size_t smem_o = sizeof(typename Cmp<T>::type) * TR * LDO;
    // FP32 Gram of width 128: the cross-tile sums (64 per thread) live in shared memory, so
    // that the kernel fits two CTAs per SM in the register file
    static constexpr bool G2S = W == 128 && sizeof(typename Cmp<T>::type) == 4;
    static constexpr size_t smem_g = G2S ? sizeof(float) * W * W : 0;
    static constexpr size_t smem = smem_a + smem_c + 2 * smem_o + smem_g;
};

template <typename T, int W, int MODE>
__global__ void __launch_bounds__(RB_THREADS)
k_rowblock(RowArgs<T> a) {
    using G = Geo<T, W>;
    constexpr int TR = G::TR, CG = G::CG, GR = G::GR;
    constexpr bool PROD = MODE != RB_PROJ;
    constexpr bool GRAM = MODE == RB_PROJ || MODE == RB_UPD || MODE == RB_MULGRAM || MODE == RB_ASMSUB;
    constexpr bool SUBX = MODE == RB_UPD || MODE == RB_ASMSUB;     // out = X - product
    constexpr bool MULTI = MODE == RB_ASM || MODE == RB_ASMSUB;    // product over basis blocks
    using C = typename Cmp<T>::type;   // arithmetic / shared-memory type
    constexpr bool TWO = sizeof(C) == 4;
    if (MODE != RB_ASM && a.ctrl && a.ctrl->stop) return;
    if (a.skip && *a.skip) return;

    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *sA = reinterpret_cast<C *>(smem_raw);                      // [KC][LDA]
    C *sC = reinterpret_cast<C *>(smem_raw + G::smem_a);          // [KC][W]
    C *sO = reinterpret_cast<C *>(smem_raw + G::smem_a + G::smem_c);            // [TR][LDO]
    C *sQ = reinterpret_cast<C *>(smem_raw + G::smem_a + G::smem_c + G::smem_o);  // [TR][LDO]
    C *sG = reinterpret_cast<C *>(smem_raw + G::smem_a + G::smem_c + 2 * G::smem_o); // [W][W] (G2S)
    constexpr bool G2S = G::G2S;

    const int tid = threadIdx.x;
    // product mapping: consecutive threads share an output column group, so a warp covers
    // few column groups and can skip K-chunks that meet the zero half of a triangular factor
    const int col4 = (tid / (TR / 4)) * 4;
    const int row0 = (tid % (TR / 4)) * 4;
    const int gi0 = (tid / 16) * GR;
    const int gj0 = (tid % 16) * GR;

    // number of K blocks (of width W) of the product
    int nkb = 1;
    if (MODE == RB_UPD) nkb = a.qa ? 2 : 1;
    if (MODE == RB_ASM) nkb = a.ctrl ? min(a.ctrl->steps, a.nblk) : a.nblk;
    if (MODE == RB_ASMSUB) nkb = a.nblk;

    C g1[GR][GR], g2[G2S ? 1 : GR][G2S ? 1 : GR];
#pragma unroll
    for (int i = 0; i < GR; ++i)
#pragma unroll
        for (int j = 0; j < GR; ++j) {
            g1[i][j] = 0;
            if constexpr (G2S) sG[(gi0 + i) * W + gj0 + j] = 0;   // this thread's entries only
            else g2[i][j] = 0;
        }

    const int64_t ntiles = (a.n + TR - 1) / TR;
    unsigned long long my_rows = 0, my_units = 0;
    // active-tile list (not for ASM, which writes every row): only row tiles holding a listed
    // 32-row frontier tile are visited, the first listed entry of a tile taking it
    constexpr int APT = TR / ACT_ROWS > 0 ? TR / ACT_ROWS : 1;
    const bool listed = MODE != RB_ASM && a.alist && a.tgen;
    const int64_t nloop = listed ? int64_t(*a.acount) : ntiles;
    for (int64_t it = blockIdx.x; it < nloop; it += gridDim.x) {
        int64_t tile = it;
        if (listed) {
            tile = __ldg(a.alist + it) / APT;
            if (it > 0 && __ldg(a.alist + it - 1) / APT == tile) continue;
        }
        const int64_t r0 = tile * TR;
        const int rows_t = (a.n - r0 < TR) ? int(a.n - r0) : TR;
        // frontier restriction: a tile beyond the limit is zero in every operand; in the
        // assemblies basis blocks k below the tile's hop distance are zero there
        int kb0 = 0;
        if (a.tgen) {
            const int tmin = tile_min_gen(a.tgen, r0, rows_t);
            if (MODE == RB_ASM) {
                kb0 = min(max(tmin - a.kbase, 0), nkb);
            } else {
                if (tmin > a.limit) continue;
                if (MODE == RB_ASMSUB) kb0 = min(tmin, nkb);
            }
        }
        if (threadIdx.x == 0) { my_rows += rows_t; my_units += (unsigned long long)rows_t * (nkb - kb0); }
        if constexpr (PROD) {
            if (SUBX) {
                // stage the X tile (coalesced); the first __syncthreads of the K loop orders it
                for (int idx = tid; idx < TR * CG; idx += RB_THREADS) {
                    const int r = idx / CG;
                    const int c = (idx % CG) * 4;
                    C xv[4] = {0, 0, 0, 0};
                    if (r0 + r < a.n) ldg4<T>(a.x + (r0 + r) * W + c, xv);
                    st4<C>(sO + r * G::LDO + c, xv);
                }
            }
            C acc[4][4];
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int q = 0; q < 4; ++q) acc[r][q] = 0;
            if (MODE == RB_ASM && a.accumulate) {
                // continue the accumulation of the earlier blocks from y (FP32, as stored)
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    const int64_t row = r0 + row0 + r;
#pragma unroll
                    for (int q = 0; q < 4; ++q)
                        if (row < a.n && col4 + q < a.mo) acc[r][q] = C(a.y[row * a.ldy + col4 + q]);
                }
            }
            for (int kb = kb0; kb < nkb; ++kb) {
                const T *src;
                const C *cmat;
                if (MODE == RB_UPD) {
                    src = (a.qa && kb == 0) ? a.qa : a.qb;
                    cmat = (a.qa && kb == 0) ? a.ca : a.cb;
                } else if (MULTI) {
                    src = a.basis + int64_t(kb) * a.block_stride;
                    cmat = a.ca + int64_t(kb) * W * W;
                } else {
                    src = a.x;
                    cmat = a.ca;
                }
                for (int k0 = 0; k0 < W; k0 += KC) {
                    // stage A[r0:r0+TR, k0:k0+KC] transposed and C[k0:k0+KC, :]
                    for (int idx = tid; idx < TR * (KC / 4); idx += RB_THREADS) {
                        const int r = idx / (KC / 4);
                        const int kq = (idx % (KC / 4)) * 4;
                        C v[4] = {0, 0, 0, 0};
                        if (r0 + r < a.n) ldg4<T>(src + (r0 + r) * W + k0 + kq, v);
#pragma unroll
                        for (int q = 0; q < 4; ++q) sA[(kq + q) * G::LDA + r] = v[q];
                    }
                    for (int idx = tid; idx < KC * CG; idx += RB_THREADS) {
                        const int kr = idx / CG;
                        const int c = (idx % CG) * 4;
                        C v[4];
                        ld4<C>(cmat + (k0 + kr) * W + c, v);
                        st4<C>(sC + kr * W + c, v);
                    }
                    __syncthreads();
                    // R^{-1} (MUL, MULGRAM) is upper triangular: rows k > c contribute nothing
                    // to column c.  H_{k-1,k} (UPD, first K block) is lower triangular: rows
                    // k < c contribute nothing.
                    bool skip = false;
                    if (MODE == RB_MUL || MODE == RB_MULGRAM) skip = k0 > col4 + 3;
                    if (MODE == RB_UPD && a.qa && kb == 0) skip = k0 + KC - 1 < col4;
                    if (!skip)
#pragma unroll
                    for (int k = 0; k < KC; ++k) {
                        C av[4], cv[4];
                        ld4<C>(sA + k * G::LDA + row0, av);
                        ld4<C>(sC + k * W + col4, cv);
#pragma unroll
                        for (int r = 0; r < 4; ++r)
#pragma unroll
                            for (int q = 0; q < 4; ++q) acc[r][q] = fma(av[r], cv[q], acc[r][q]);
                    }
                    __syncthreads();
                }
            }
            // finish the tile: the register tile goes to shared memory (UPD subtracts it from
            // the X tile staged there), then the whole tile is stored with coalesced rows.
            // The barrier matters when the K loop was empty (an assembly tile below every
            // block's reach): without it this tile's writes to sO would race with the slower
            // threads still storing the previous tile from sO.
            __syncthreads();
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                C o[4];
                if (SUBX) {
                    C xv[4];
                    ld4<C>(sO + (row0 + r) * G::LDO + col4, xv);
#pragma unroll
                    for (int q = 0; q < 4; ++q) o[q] = xv[q] - acc[r][q];
                } else {
#pragma unroll
                    for (int q = 0; q < 4; ++q) o[q] = acc[r][q];
                }
                // narrow stored blocks now, so the Gram below is that of the stored values
                if constexpr (!std::is_same<T, C>::value && MODE != RB_ASM) {
#pragma unroll
                    for (int q = 0; q < 4; ++q) o[q] = C(T(o[q]));
                }
                st4<C>(sO + (row0 + r) * G::LDO + col4, o);
            }
            __syncthreads();
            for (int idx = tid; idx < TR * CG; idx += RB_THREADS) {
                const int r = idx / CG;
                const int c = (idx % CG) * 4;
                const int64_t row = r0 + r;
                if (row >= a.n) continue;
                C o[4];
                ld4<C>(sO + r * G::LDO + c, o);
                if (MODE == RB_ASM) {
#pragma unroll
                    for (int q = 0; q < 4; ++q)
                        if (c + q < a.mo) a.y[row * a.ldy + c + q] = float(o[q]);
                } else {
                    stg4<T>(a.out + row * W + c, o);
                }
            }
        } else {
            // PROJ: stage X and Qa tiles
            for (int idx = tid; idx < TR * CG; idx += RB_THREADS) {
                const int r = idx / CG;
                const int c = (idx % CG) * 4;
                C xv[4] = {0, 0, 0, 0}, qv[4] = {0, 0, 0, 0};
                if (r0 + r < a.n) {
                    ldg4<T>(a.x + (r0 + r) * W + c, xv);
                    ldg4<T>(a.qa + (r0 + r) * W + c, qv);
                }
                st4<C>(sO + r * G::LDO + c, xv);
                st4<C>(sQ + r * G::LDO + c, qv);
            }
        }
        if constexpr (GRAM) {
            __syncthreads();
            const C *left = (MODE == RB_PROJ) ? sQ : sO;
            for (int r = 0; r < TR; ++r) {
                C av[GR], bv[GR];
                if constexpr (GR >= 4) {
#pragma unroll
                    for (int q = 0; q < GR; q += 4) {
                        C t4[4];
                        ld4<C>(left + r * G::LDO + gi0 + q, t4);
#pragma unroll
                        for (int u = 0; u < 4; ++u) av[q + u] = t4[u];
                        ld4<C>(sO + r * G::LDO + gj0 + q, t4);
#pragma unroll
                        for (int u = 0; u < 4; ++u) bv[q + u] = t4[u];
                    }
                } else {
#pragma unroll
                    for (int q = 0; q < GR; ++q) {
                        av[q] = left[r * G::LDO + gi0 + q];
                        bv[q] = sO[r * G::LDO + gj0 + q];
                    }
                }
#pragma unroll
                for (int i = 0; i < GR; ++i)
#pragma unroll
                    for (int j = 0; j < GR; ++j) {
                        if (TWO) g1[i][j] = fma(av[i], bv[j], g1[i][j]);
                        else if constexpr (!G2S) g2[i][j] = fma(av[i], bv[j], g2[i][j]);
                    }
            }
            if (TWO) {
#pragma unroll
                for (int i = 0; i < GR; ++i)
#pragma unroll
                    for (int j = 0; j < GR; ++j) {
                        if constexpr (G2S) sG[(gi0 + i) * W + gj0 + j] += g1[i][j];
                        else g2[i][j] += g1[i][j];
                        g1[i][j] = 0;
                    }
            }
            __syncthreads();
        }
    }
    if (threadIdx.x == 0 && a.prof.rows) {
        atomicAdd(a.prof.rows, my_rows);
        atomicAdd(a.prof.nnz, my_units);
    }
    if constexpr (GRAM) {
        C *p = a.partials + int64_t(blockIdx.x) * W * W;
#pragma unroll
        for (int i = 0; i < GR; ++i)
#pragma unroll
            for (int j = 0; j < GR; ++j) {
                if constexpr (G2S) p[(gi0 + i) * W + gj0 + j] = sG[(gi0 + i) * W + gj0 + j];
                else p[(gi0 + i) * W + gj0 + j] = g2[i][j];
            }
    }
}

template <typename T, int W, int MODE>
int occupancy() {
    using G = Geo<T, W>;
    // function-local static: computed once, thread-safe (several serving workers)
    static const int cached = [] {
        cudaFuncSetAttribute(k_rowblock<T, W, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             int(G::smem));
        int per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_rowblock<T, W, MODE>, RB_THREADS,
                                                      G::smem);
        return std::max(per_sm, 1);
    }();
    return cached;
}

template <typename T, int W, int MODE>
int launch_wm(const RowArgs<T> &a, cudaStream_t s, int *grid_out) {
    using G = Geo<T, W>;
    const int per_sm = occupancy<T, W, MODE>();
    const int64_t ntiles = (a.n + G::TR - 1) / G::TR;
    int grid = int(std::min<int64_t>(ntiles, int64_t(num_sms()) * per_sm));
    if (grid < 1) grid = 1;
    if (grid_out) *grid_out = grid;
    k_rowblock<T, W, MODE><<<grid, RB_THREADS, G::smem, s>>>(a);
    return 0;
}

template <typename T, int W>
int launch_w(int mode, const RowArgs<T> &a, cudaStream_t s, int *grid_out) {
    switch (mode) {
        case RB_PROJ: return launch_wm<T, W, RB_PROJ>(a, s, grid_out);
        case RB_UPD: return launch_wm<T, W, RB_UPD>(a, s, grid_out);
        case RB_MULGRAM: return launch_wm<T, W, RB_MULGRAM>(a, s, grid_out);
        case RB_MUL: return launch_wm<T, W, RB_MUL>(a, s, grid_out);
        case RB_ASM: return launch_wm<T, W, RB_ASM>(a, s, grid_out);
        case RB_ASMSUB: return launch_wm<T, W, RB_ASMSUB>(a, s, grid_out);
    }
    return fail(KB_ERR_ARG, "bad row-block mode");
}

template <typename T, int W>
int max_grid_w() {
    int g = num_sms() * std::max({occupancy<T, W, RB_PROJ>(), occupancy<T, W, RB_UPD>(),
                                  occupancy<T, W, RB_MULGRAM>(), occupancy<T, W, RB_MUL>(),
                                  occupancy<T, W, RB_ASMSUB>()});
    if (std::is_same<T, float>::value && W == 64) g = std::max(g, rowblock_tc_max_grid());
    return g;
}

// ---------------------------------------------------------------- deterministic reduction
template <typename P>
__global__ void __launch_bounds__(1024) k_reduce(const P *__restrict__ parts, int nparts, int len,
                                                  double *__restrict__ out, const Ctrl *ctrl,
                                                  P *__restrict__ out_p, const int32_t *skip) {
    // 32 columns per CTA, 32 warps over the partials (two loads in flight per lane), then a
    // fixed-order combination of the warps' sums by warp 0
    if ((ctrl && ctrl->stop) || (skip && *skip)) return;
    __shared__ double s[32][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int e = blockIdx.x * 32 + lane;
    if constexpr (std::is_same<P, float>::value) {
        // double-float accumulation on the FP32 pipe
        DF a0{0.f, 0.f}, a1{0.f, 0.f};
        if (e < len) {
            int p = warp;
            for (; p + nw < nparts; p += 2 * nw) {
                const float v0 = parts[int64_t(p) * len + e], v1 = parts[int64_t(p + nw) * len + e];
                df_add(a0, v0);
                df_add(a1, v1);
            }
            if (p < nparts) df_add(a0, parts[int64_t(p) * len + e]);
        }
        df_merge(a0, a1);
        reinterpret_cast<DF *>(&s[warp][0])[lane] = a0;
        __syncthreads();
        if (warp == 0 && e < len) {
            DF t = reinterpret_cast<const DF *>(&s[0][0])[lane];
            for (int w = 1; w < nw; ++w) df_merge(t, reinterpret_cast<const DF *>(&s[w][0])[lane]);
            const double v = df_value(t);
            out[e] = v;
            if (out_p) out_p[e] = P(v);
        }
    } else {
        double acc = 0.0;
        if (e < len)
            for (int p = warp; p < nparts; p += nw) acc += double(parts[int64_t(p) * len + e]);
        s[warp][lane] = acc;
        __syncthreads();
        if (warp == 0 && e < len) {
            double t = 0.0;
            for (int w = 0; w < nw; ++w) t += s[w][lane];
            out[e] = t;
            if (out_p) out_p[e] = P(t);
        }
    }
}

}  // namespace

// The tensor-core kernels are used when the environment variable KB_TENSOR_CORES is "1"
// at the time of the launch (read on every launch, so a process can switch).  They are not
// the default: with the frontier restriction most launches of a solve cover few tiles, and
// one 192 KB CTA per SM keeps other streams' kernels off the SM (measured slower in the
// multi-stream throughput run).
bool rowblock_tc_enabled() {
    const char *e = std::getenv("KB_TENSOR_CORES");
    return e && e[0] == '1';
}

template <typename T>
int launch_rowblock(int mode, int W, const RowArgs<T> &a, cudaStream_t s, int *grid_out,
                    int64_t M_alg) {
    if (sizeof(typename Cmp<T>::type) == 8 && W > 64) return fail(KB_ERR_UNSUPPORTED, "FP64 blocks wider than 64");
    const int cls = mode == RB_ASM ? KernelClass::ASSEMBLE : KernelClass::ROWBLOCK;
    RowArgs<T> aa = a;
    aa.prof = prof_begin(cls, s);
    int rc = 0;
    bool tc = false;
    // (launches under a device skip flag take the SIMT kernels, which read the flag)
    if constexpr (std::is_same<T, float>::value)
        tc = !a.skip && rowblock_tc_supported(mode, W) && rowblock_tc_enabled();
    if (tc) {
        // FP32 blocks of width 64: tensor-core kernel (rowblock_tc.cu)
        if constexpr (std::is_same<T, float>::value)
            rc = launch_rowblock_tc(mode, aa, s, rowblock_max_grid<T>(W), grid_out);
    } else {
        switch (W) {
            case 16: rc = launch_w<T, 16>(mode, aa, s, grid_out); break;
            case 32: rc = launch_w<T, 32>(mode, aa, s, grid_out); break;
            case 64: rc = launch_w<T, 64>(mode, aa, s, grid_out); break;
            case 128:
                if constexpr (sizeof(typename Cmp<T>::type) == 4) { rc = launch_w<T, 128>(mode, aa, s, grid_out); break; }
                [[fallthrough]];
            default: return fail(KB_ERR_ARG, "unsupported block width");
        }
    }
    if (rc) return rc;
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) return cuda_fail(err, tc ? "k_rowblock_tc launch" : "k_rowblock launch");
    const double blk = double(a.n) * double(M_alg) * sizeof(T);
    const double row = double(M_alg) * sizeof(T);             // bytes of one block row
    const double fr = 2.0 * double(M_alg) * double(M_alg);    // flops of one row times M x M
    double bytes = 0, flops = 0, per_row = 0, per_unit = 0, frow = 0, fixed = 0;
    const double mm = double(a.n) * fr;
    // algorithmic flops count the structure of the small matrices: a product with a
    // triangular factor (H_{k-1,k}, R^{-1}) is half of a general one, a Gram X^T X is
    // symmetric (half); the kernels compute more than this (full products, full Gram)
    switch (mode) {
        case RB_PROJ: bytes = 2 * blk; flops = mm; per_row = 2 * row; frow = fr; break;
        case RB_UPD:
            bytes = (a.qa ? 4 : 3) * blk; flops = (a.qa ? 2.0 : 1.5) * mm;
            per_row = (a.qa ? 4 : 3) * row; frow = (a.qa ? 2.0 : 1.5) * fr; break;
        case RB_MULGRAM: bytes = 2 * blk; flops = mm; per_row = 2 * row; frow = fr; break;
        case RB_MUL: bytes = 2 * blk; flops = 0.5 * mm; per_row = 2 * row; frow = 0.5 * fr; break;
        case RB_ASM:
            // block rows read (counted per tile and block) + the FP32 output written in full
            bytes = (a.nblk + 1) * blk; flops = a.nblk * mm;
            per_unit = row; fixed = double(a.n) * double(M_alg) * 4.0; break;
        case RB_ASMSUB:
            bytes = (a.nblk + 2) * blk; flops = a.nblk * mm + mm;
            per_row = 2 * row; per_unit = row; frow = fr; break;
    }
    prof_end(cls, s, bytes, flops, 1, per_row, per_unit, frow, fixed);
    return 0;
}

template <typename T>
int rowblock_max_grid(int W) {
    switch (W) {
        case 16: return max_grid_w<T, 16>();
        case 32: return max_grid_w<T, 32>();
        case 64: return max_grid_w<T, 64>();
        default:
            if constexpr (sizeof(typename Cmp<T>::type) == 4) return max_grid_w<T, 128>();
            return 0;
    }
}

template <typename P>
int launch_reduce(const P *parts, int nparts, int len, double *out, cudaStream_t s,
                  const Ctrl *ctrl, P *out_p, const int32_t *skip) {
    prof_begin(KernelClass::REDUCE, s);
    k_reduce<P><<<(len + 31) / 32, 1024, 0, s>>>(parts, nparts, len, out, ctrl, out_p, skip);
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) return cuda_fail(err, "k_reduce launch");
    prof_end(KernelClass::REDUCE, s, double(nparts) * len * sizeof(P), 0);
    return 0;
}

template int launch_rowblock<float>(int, int, const RowArgs<float> &, cudaStream_t, int *, int64_t);
template int launch_rowblock<double>(int, int, const RowArgs<double> &, cudaStream_t, int *, int64_t);
template int rowblock_max_grid<float>(int);
template int rowblock_max_grid<double>(int);
template int launch_rowblock<__nv_bfloat16>(int, int, const RowArgs<__nv_bfloat16> &, cudaStream_t, int *, int64_t);
template int rowblock_max_grid<__nv_bfloat16>(int);
template int launch_reduce<float>(const float *, int, int, double *, cudaStream_t, const Ctrl *, float *,
                                  const int32_t *);
template int launch_reduce<double>(const double *, int, int, double *, cudaStream_t, const Ctrl *, double *,
                                   const int32_t *);

}  // namespace kb
