// Block SpMM with the Laplacian: out = epilogue(L x), x an n x W row-major block.
//
// This is the "MV" of Table 1 (Section 7), the operation the paper names the most
// expensive for large graphs; every method performs m of them per solve.
//
// Schedule (GB300).  A CTA owns a tile of consecutive rows at a time (persistent grid,
// a multiple of the SM count).  The tile's row pointers and then all its column indices
// (and weights) are staged in shared memory with coalesced loads, so a row's neighbour
// list costs no dependent global round trip.  A row of x is W elements; W/8 lanes cover it
// with two 16-byte vectors each (float4, or 2 x double2), so each warp works on 32/(W/8)
// rows at once, one lane group per row; a group reads its neighbour indices from shared
// memory (broadcast) and gathers two neighbour rows with independent 16-byte loads before
// consuming them.  The register budget is sized for 5 resident CTAs (40 warps) per SM.  Rows of a tile whose column list does not fit in shared memory
// (hub rows) read their indices from global memory instead.
//
// The Laplacian is applied in difference form (L x)_i = sum_j w_ij (x_i - x_j) + r_i x_i,
// which gives L 1 = 0 exactly for D - A and drops the diagonal load for standard
// Laplacians.  Epilogue coefficients arrive in FP64; in the FP32 path each is split into
// a float pair (hi + lo) so that c * (L x) carries only the rounding of the final sum.
#include <type_traits>

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
template <> struct V4<__nv_bfloat16> {
    // four BF16 values (8 bytes) widened to FP32
    float v[4];
    __device__ __forceinline__ static V4 load(const __nv_bfloat16 *p) {
        const uint2 raw = __ldg(reinterpret_cast<const uint2 *>(p));
        const float2 a = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&raw.x));
        const float2 b = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&raw.y));
        return V4{{a.x, a.y, b.x, b.y}};
    }
    __device__ __forceinline__ void store(__nv_bfloat16 *p) const {
        const __nv_bfloat162 a = __floats2bfloat162_rn(v[0], v[1]);
        const __nv_bfloat162 b = __floats2bfloat162_rn(v[2], v[3]);
        uint2 raw;
        raw.x = *reinterpret_cast<const unsigned int *>(&a);
        raw.y = *reinterpret_cast<const unsigned int *>(&b);
        *reinterpret_cast<uint2 *>(p) = raw;
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

// Schedule parameters (compile-time; the defaults are the measured best on the RGG bench).
#ifndef KB_SPMM_CAP
#define KB_SPMM_CAP 4096
#endif
#ifndef KB_SPMM_VPL
#define KB_SPMM_VPL 2
#endif
#ifndef KB_SPMM_U
#define KB_SPMM_U 4
#endif
#ifndef KB_SPMM_PACKED
#define KB_SPMM_PACKED 1   // FP32 neighbour loop on packed f32x2 pairs
#endif
#ifndef KB_SPMM_IDX32
#define KB_SPMM_IDX32 0
#endif
constexpr int SPMM_THREADS = 256;
constexpr int WARPS = SPMM_THREADS / 32;
constexpr int CAP = KB_SPMM_CAP;   // staged column indices per tile
constexpr int VPL = KB_SPMM_VPL;   // 16-byte vectors per lane (4 VPL elements of a row)
constexpr int U = KB_SPMM_U;       // neighbour rows gathered per lane before use

template <int W>
struct SpmmGeo {
    static constexpr int LPR = W / (4 * VPL) < 1 ? 1 : W / (4 * VPL);   // lanes per row
    static constexpr int RPW = 32 / LPR;                 // rows per warp
    static constexpr int NG = WARPS * RPW;               // lane groups per CTA
    static constexpr int RPG = W >= 64 ? 4 : (W == 32 ? 2 : 1);   // rows per group per tile
    static constexpr int TR = NG * RPG;                  // rows per tile
};

// Resident CTAs per SM the register budget is sized for: the FP32 kernel without column
// dot products fits 5 (40 warps), the others fewer.
// Prefetch the 128-byte line holding p into L2 (no register result, no fault on the
// addresses used here: every caller passes an address inside an allocated array).
__device__ __forceinline__ void prefetch_l2(const void *p) {
    asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

// Packed FP32 pairs (Blackwell add/sub/fma.rn.f32x2): each lane of the pair is rounded as
// the scalar instruction would round it, so the packed neighbour loop gives bit-identical
// sums with half the floating-point instructions.
using f2 = unsigned long long;
__device__ __forceinline__ f2 f2_add(f2 a, f2 b) {
    f2 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2 f2_sub(f2 a, f2 b) {
    f2 d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2 f2_fma(f2 a, f2 b, f2 c) {
    f2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ f2 f2_pack(float lo, float hi) {
    f2 d;
    asm("mov.b64 %0, {%1, %2};" : "=l"(d) : "f"(lo), "f"(hi));
    return d;
}
__device__ __forceinline__ void f2_unpack(f2 v, float &lo, float &hi) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
// 16 bytes of a read-only FP32 row as two packed pairs
__device__ __forceinline__ void ldg_f2x2(const float *p, f2 &a, f2 &b) {
    asm("ld.global.nc.v2.b64 {%0, %1}, [%2];" : "=l"(a), "=l"(b) : "l"(p));
}

// Four consecutive coefficients from shared memory in one 16-byte (FP32) or two 16-byte
// (FP64) loads; c is a multiple of 4 and the arrays are 16-byte aligned.
template <typename C>
__device__ __forceinline__ void lds4(const C *p, C (&v)[4]) {
    if constexpr (sizeof(C) == 4) {
        const float4 t = *reinterpret_cast<const float4 *>(p);
        v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
    } else {
        const double2 a = reinterpret_cast<const double2 *>(p)[0];
        const double2 b = reinterpret_cast<const double2 *>(p)[1];
        v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
    }
}

#ifndef KB_SPMM_OCC
#define KB_SPMM_OCC 4   // FP32 / BF16 kernel without column dots
#endif
#ifndef KB_SPMM_OCC_DOT
#define KB_SPMM_OCC_DOT 4   // FP32 / BF16 kernel with column dots
#endif
template <typename T, bool DOT>
struct SpmmOcc {
    static constexpr int value = sizeof(typename Cmp<T>::type) == 8 ? 3 : (DOT ? KB_SPMM_OCC_DOT : KB_SPMM_OCC);
};

// WGT: the graph stores edge weights (false: unit weights, w_ij = 1).  LST: the launch walks
// the active-tile list (frontier restriction with a list of the active 32-row tiles).
template <typename T, int W, bool DOT, bool WGT, bool LST>
__global__ void __launch_bounds__(SPMM_THREADS, (SpmmOcc<T, DOT>::value))
k_spmm(GraphDev g, const T *__restrict__ x, LinEpi<T> e, int64_t ldo, int mo) {
    using G = SpmmGeo<W>;
    using C = typename Cmp<T>::type;   // arithmetic type
    constexpr int LPR = G::LPR, RPW = G::RPW, NG = G::NG, TR = G::TR, RPG = G::RPG;
    // gathers in flight per lane group: fewer in the variant that also accumulates column
    // dots (its registers hold the dot partials)
    constexpr int UU = DOT ? (U < 2 ? U : 2) : U;
    static_assert(TR >= ACT_ROWS && TR % ACT_ROWS == 0, "row tiles hold whole 32-row frontier tiles");
    if (e.ctrl && e.ctrl->stop) return;
    // (arrays a variant does not use take one element: shared memory left to L1 caches the
    // gathered rows)
    __shared__ int s_rp[TR + 1];
    __shared__ int s_col[CAP];
    __shared__ float s_w[WGT ? CAP : 1];
    __shared__ __align__(16) C s_coef[5][W];       // c1 hi, c1 lo, c0, c2 hi, c2 lo
    __shared__ C s_sc[2];                          // s3, wE in the arithmetic type
    __shared__ double s_dot[DOT ? WARPS : 1][W];
    __shared__ unsigned long long s_cnt[2];       // rows, stored nonzeros processed
    if (threadIdx.x == 0) {
        s_sc[0] = C(e.s3);
        s_sc[1] = C(e.wE);
        s_cnt[0] = 0ull;
        s_cnt[1] = 0ull;
    }
    for (int c = threadIdx.x; c < W; c += blockDim.x) {
        const double d1 = e.a1 ? e.a1[c] : e.s1;
        const double d2 = e.a2 ? e.a2[c] : e.s2;
        const C h1 = C(d1), h2 = C(d2);
        s_coef[0][c] = h1;
        s_coef[1][c] = C(d1 - double(h1));
        s_coef[2][c] = C(e.a0 ? e.a0[c] : e.s0);
        s_coef[3][c] = h2;
        s_coef[4][c] = C(d2 - double(h2));
    }
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int grp = lane / LPR;
    // columns of this lane: 4 consecutive columns in each of VPL slices of 4 * LPR columns,
    // so that one 16-byte load instruction of a lane group reads one contiguous 4 * LPR
    // column span (whole 32-byte sectors) of the gathered row
    const int sub = lane % LPR;
#define KB_COL(v) (((v) * LPR + sub) * 4)
    const int gid = warp * RPW + grp;
    C dot[VPL][4];
#pragma unroll
    for (int v = 0; v < VPL; ++v)
#pragma unroll
        for (int q = 0; q < 4; ++q) dot[v][q] = C(0);
    const int64_t ntiles = (g.n + TR - 1) / TR;
    // with the active-tile list, the unit of work is one listed 32-row tile instead of a
    // TR-row tile: the few active rows of an early step spread over all CTAs
    constexpr bool listed = LST;
    const int64_t nloop = listed ? int64_t(*e.acount) : ntiles;
    // A listed unit is one chunk of 32 rows: its lane groups read their row pointers and
    // column indices straight from global memory, with no shared staging and no barrier, so
    // the warps of a CTA move through their units independently.  The coefficients set above
    // are ordered here.
    if constexpr (listed) __syncthreads();

    for (int64_t it = blockIdx.x; it < nloop; it += gridDim.x) {
        const int64_t r0 = listed ? int64_t(__ldg(e.alist + it)) * ACT_ROWS : it * TR;
        const int urows = listed ? ACT_ROWS : TR;
        const int rows = (g.n - r0 < urows) ? int(g.n - r0) : urows;
        if (e.tgen && tile_min_gen(e.tgen, r0, rows) > e.limit) {
            // every row of the tile is beyond the frontier: its output is exactly zero
            if (e.zero_inactive) {
                if (e.yout) {
                    for (int i = threadIdx.x; i < rows * mo; i += blockDim.x)
                        e.yout[(r0 + i / mo) * ldo + (i % mo)] = 0.f;
                } else {
                    for (int i = threadIdx.x; i < rows * W; i += blockDim.x) e.out[r0 * W + i] = T(0.f);
                }
            }
            continue;
        }
        int base = 0;
        bool staged = false;
        if constexpr (!listed) {
            // ask L2 for the tile's own dense rows now (x_i at the row start, y / z in the
            // epilogue) and for the next tile's row pointers, so that those loads, issued
            // later, do not wait on DRAM
            const char *xb = reinterpret_cast<const char *>(x + r0 * W);
            const int64_t tile_bytes = int64_t(rows) * W * int64_t(sizeof(T));
            constexpr int64_t row_bytes = int64_t(W) * int64_t(sizeof(T));
            for (int64_t off = int64_t(threadIdx.x) * 128; off < tile_bytes; off += int64_t(blockDim.x) * 128) {
                // rows of 32-row frontier tiles beyond the limit are skipped below: no prefetch
                if (e.tgen && __ldg(e.tgen + (r0 + off / row_bytes) / ACT_ROWS) > e.limit) continue;
                prefetch_l2(xb + off);
                if (e.y) prefetch_l2(reinterpret_cast<const char *>(e.y + r0 * W) + off);
                if (e.z) prefetch_l2(reinterpret_cast<const char *>(e.z + r0 * W) + off);
            }
            const int64_t nr0 = r0 + int64_t(gridDim.x) * TR;
            if (threadIdx.x < (TR + 1 + 31) / 32 && nr0 + threadIdx.x * 32 <= g.n)
                prefetch_l2(g.rowptr + nr0 + threadIdx.x * 32);
            __syncthreads();   // previous tile done with the shared arrays
            for (int i = threadIdx.x; i <= rows; i += blockDim.x) s_rp[i] = __ldg(g.rowptr + r0 + i);
            __syncthreads();
            base = s_rp[0];
            const int cnt = s_rp[rows] - base;
            staged = cnt <= CAP;
            if (staged) {
                for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
                    s_col[i] = __ldg(g.col + base + i);
                    if (WGT) s_w[i] = __ldg(g.w + base + i);
                }
            }
            __syncthreads();
        }
#pragma unroll 1
        for (int rr = 0; rr < RPG; ++rr) {
            // rows rr*NG .. rr*NG+NG-1 of the tile (one lane group each); with the frontier
            // restriction a chunk whose 32-row frontier tiles are all beyond the limit is
            // exactly zero and skipped (CTA-uniform)
            const int c0r = rr * NG;
            if (c0r >= rows) break;
            const int crows = rows - c0r < NG ? rows - c0r : NG;
            const int lrow = c0r + gid;
            bool skip_rows = e.tgen && tile_min_gen(e.tgen, r0 + c0r, crows) > e.limit;
            if (!skip_rows && e.gen) {
                // this warp's RPW rows of the chunk: skipped (warp-uniform) when every one
                // of them lies beyond the limit (the rr loop has no barrier)
                const int wr0 = c0r + warp * RPW;
                bool any = false;
#pragma unroll
                for (int q = 0; q < RPW; ++q)
                    if (wr0 + q < rows && int(__ldg(e.gen + r0 + wr0 + q)) <= e.limit) any = true;
                skip_rows = !any;
            } else if (!skip_rows && threadIdx.x == 0 && !listed) {
                s_cnt[0] += unsigned(crows);
                s_cnt[1] += unsigned(s_rp[c0r + crows] - s_rp[c0r]);
            }
            if (skip_rows) {
                if (e.zero_inactive && lrow < rows) {
#pragma unroll
                    for (int v = 0; v < VPL; ++v)
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            const int c = KB_COL(v) + q;
                            if (e.yout) {
                                if (c < mo) e.yout[(r0 + lrow) * ldo + c] = 0.f;
                            } else {
                                e.out[(r0 + lrow) * W + c] = T(0.f);
                            }
                        }
                }
                continue;
            }
            if (e.gen && lane == 0) {
                // rows and stored nonzeros this warp processes
                const int wr0 = c0r + warp * RPW;
                const int wr1 = wr0 + RPW < rows ? wr0 + RPW : rows;
                if (wr1 > wr0) {
                    const int nz = listed ? __ldg(g.rowptr + r0 + wr1) - __ldg(g.rowptr + r0 + wr0)
                                          : s_rp[wr1] - s_rp[wr0];
                    atomicAdd(&s_cnt[0], (unsigned long long)(wr1 - wr0));
                    atomicAdd(&s_cnt[1], (unsigned long long)nz);
                }
            }
            if (lrow >= rows) continue;
            const int64_t row = r0 + lrow;
            const int beg = listed ? __ldg(g.rowptr + row) : s_rp[lrow] - base;
            const int end = listed ? __ldg(g.rowptr + row + 1) : s_rp[lrow + 1] - base;
            V4<T> xi[VPL];
            C acc[VPL][4];
#pragma unroll
            for (int v = 0; v < VPL; ++v) {
                xi[v] = V4<T>::load(x + row * W + KB_COL(v));
#pragma unroll
                for (int q = 0; q < 4; ++q) acc[v][q] = C(0);
            }
            if constexpr (std::is_same<T, float>::value && KB_SPMM_PACKED) {
                // the same sums on packed pairs: acc += w (x_i - x_j), two columns per
                // instruction
                f2 xi2[VPL][2], acc2[VPL][2];
#pragma unroll
                for (int v = 0; v < VPL; ++v) {
                    xi2[v][0] = f2_pack(xi[v].v[0], xi[v].v[1]);
                    xi2[v][1] = f2_pack(xi[v].v[2], xi[v].v[3]);
                    acc2[v][0] = 0ull;
                    acc2[v][1] = 0ull;
                }
                for (int p = beg; p < end; p += UU) {
                    // slots past the row's end gather the row itself (weight 0): x_i - x_i
                    // adds an exact zero, so the unrolled body needs no per-slot branch
                    f2 xj2[UU][VPL][2];
                    f2 wv2[UU];
                    int jj[UU];
#pragma unroll
                    for (int u = 0; u < UU; ++u) {
                        const bool in = p + u < end;
                        jj[u] = in ? (staged ? s_col[p + u] : __ldg(g.col + base + p + u)) : int(row);
                        if (WGT) {
                            const float w = in ? (staged ? s_w[p + u] : __ldg(g.w + base + p + u)) : 0.f;
                            wv2[u] = f2_pack(w, w);
                        }
                    }
#pragma unroll
                    for (int u = 0; u < UU; ++u)
#pragma unroll
                        for (int v = 0; v < VPL; ++v)
                            ldg_f2x2(reinterpret_cast<const float *>(x) + int64_t(jj[u]) * W + KB_COL(v),
                                     xj2[u][v][0], xj2[u][v][1]);
#pragma unroll
                    for (int u = 0; u < UU; ++u)
#pragma unroll
                        for (int v = 0; v < VPL; ++v)
#pragma unroll
                            for (int h = 0; h < 2; ++h) {
                                const f2 d = f2_sub(xi2[v][h], xj2[u][v][h]);
                                acc2[v][h] = WGT ? f2_fma(wv2[u], d, acc2[v][h]) : f2_add(acc2[v][h], d);
                            }
                }
#pragma unroll
                for (int v = 0; v < VPL; ++v) {
                    f2_unpack(acc2[v][0], acc[v][0], acc[v][1]);
                    f2_unpack(acc2[v][1], acc[v][2], acc[v][3]);
                    // x_i again from its packed copy (the scalar copy need not live across
                    // the loop)
                    f2_unpack(xi2[v][0], xi[v].v[0], xi[v].v[1]);
                    f2_unpack(xi2[v][1], xi[v].v[2], xi[v].v[3]);
                }
            } else {
            for (int p = beg; p < end; p += UU) {
                // slots past the row's end gather the row itself (weight 0): x_i - x_i adds
                // an exact zero, so the unrolled body needs no per-slot branch
                V4<T> xj[UU][VPL];
                C wv[UU];
                int jj[UU];
#pragma unroll
                for (int u = 0; u < UU; ++u) {
                    const bool in = p + u < end;
                    jj[u] = in ? (staged ? s_col[p + u] : __ldg(g.col + base + p + u)) : int(row);
                    wv[u] = WGT ? (in ? C(staged ? s_w[p + u] : __ldg(g.w + base + p + u)) : C(0)) : C(1);
                }
#pragma unroll
                for (int u = 0; u < UU; ++u)
#pragma unroll
                    for (int v = 0; v < VPL; ++v)
                        xj[u][v] = V4<T>::load(KB_SPMM_IDX32 ? x + (unsigned(jj[u]) * unsigned(W) + unsigned(KB_COL(v)))
                                                             : x + int64_t(jj[u]) * W + KB_COL(v));
#pragma unroll
                for (int u = 0; u < UU; ++u)
#pragma unroll
                    for (int v = 0; v < VPL; ++v)
#pragma unroll
                        for (int q = 0; q < 4; ++q)
                            acc[v][q] = WGT ? fma(wv[u], xi[v].v[q] - xj[u][v].v[q], acc[v][q])
                                            : acc[v][q] + (xi[v].v[q] - xj[u][v].v[q]);
            }
            }
            const C r = g.rdiag ? C(__ldg(g.rdiag + row)) : C(0);
            const int mk = e.marker ? __ldg(e.marker + row) : -1;
#pragma unroll
            for (int v = 0; v < VPL; ++v) {
                const int c = KB_COL(v);
                C o[4], k1h[4], k1l[4], k0[4];
                lds4(&s_coef[0][c], k1h);
                lds4(&s_coef[1][c], k1l);
                lds4(&s_coef[2][c], k0);
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const C a = fma(r, xi[v].v[q], acc[v][q]);
                    o[q] = fma(k1h[q], a, fma(k1l[q], a, k0[q] * xi[v].v[q]));
                }
                if (e.y) {
                    const V4<T> yi = V4<T>::load(e.y + row * W + c);
                    C k2h[4], k2l[4];
                    lds4(&s_coef[3][c], k2h);
                    lds4(&s_coef[4][c], k2l);
#pragma unroll
                    for (int q = 0; q < 4; ++q) o[q] = fma(k2h[q], yi.v[q], fma(k2l[q], yi.v[q], o[q]));
                }
                if (e.z) {
                    const V4<T> zi = V4<T>::load(e.z + row * W + c);
#pragma unroll
                    for (int q = 0; q < 4; ++q) o[q] = fma(s_sc[0], zi.v[q], o[q]);
                }
                // (constant indices: a computed index would put o in local memory)
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    if (mk == c + q) o[q] += s_sc[1];
                if (!e.yout) {
                    // narrowed blocks: the dot below is that of the stored values
                    if constexpr (!std::is_same<T, C>::value) {
#pragma unroll
                        for (int q = 0; q < 4; ++q) o[q] = C(T(o[q]));
                    }
                    V4<T> ov;
#pragma unroll
                    for (int q = 0; q < 4; ++q) ov.v[q] = o[q];
                    ov.store(e.out + row * W + c);
                } else {
#pragma unroll
                    for (int q = 0; q < 4; ++q)
                        if (c + q < mo) e.yout[row * ldo + c + q] = float(o[q]);
                }
                if (DOT) {
#pragma unroll
                    for (int q = 0; q < 4; ++q) dot[v][q] = fma(xi[v].v[q], o[q], dot[v][q]);
                }
            }
        }
    }
    if (threadIdx.x == 0 && e.prof.rows) {
        atomicAdd(e.prof.rows, s_cnt[0]);
        atomicAdd(e.prof.nnz, s_cnt[1]);
    }
    if constexpr (DOT && std::is_same<C, float>::value) {
        // double-float combination on the FP32 pipe; partials written as DF pairs
        DF *sd = reinterpret_cast<DF *>(&s_dot[0][0]);
#pragma unroll
        for (int v = 0; v < VPL; ++v)
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                DF d{dot[v][q], 0.f};
#pragma unroll
                for (int off = LPR; off < 32; off <<= 1) {
                    const DF o{__shfl_xor_sync(0xffffffffu, d.hi, off), __shfl_xor_sync(0xffffffffu, d.lo, off)};
                    df_merge(d, o);
                }
                if (grp == 0) sd[warp * W + KB_COL(v) + q] = d;
            }
        __syncthreads();
        DF *out = reinterpret_cast<DF *>(e.dot_partials);
        for (int c = threadIdx.x; c < W; c += blockDim.x) {
            DF s = sd[c];
            for (int w2 = 1; w2 < WARPS; ++w2) df_merge(s, sd[w2 * W + c]);
            out[int64_t(blockIdx.x) * W + c] = s;
        }
    } else if constexpr (DOT) {
#pragma unroll
        for (int v = 0; v < VPL; ++v)
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                double dd = double(dot[v][q]);
#pragma unroll
                for (int off = LPR; off < 32; off <<= 1) dd += __shfl_xor_sync(0xffffffffu, dd, off);
                if (grp == 0) s_dot[warp][KB_COL(v) + q] = dd;
            }
        __syncthreads();
        for (int c = threadIdx.x; c < W; c += blockDim.x) {
            double s = 0.0;
            for (int w2 = 0; w2 < WARPS; ++w2) s += s_dot[w2][c];
            e.dot_partials[int64_t(blockIdx.x) * W + c] = s;
        }
    }
}

#undef KB_COL

template <typename T, int W, bool DOT>
int occupancy_spmm() {
    // the weighted and unweighted kernels share the launch bounds
    // function-local static: computed once, thread-safe (several serving workers)
    static const int per_sm = [] {
        int v = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, k_spmm<T, W, DOT, true, false>, SPMM_THREADS, 0);
        return v < 1 ? 1 : v;
    }();
    return per_sm;
}

template <typename T, int W, bool DOT>
int launch_wd(const GraphDev &g, const T *x, const LinEpi<T> &e, int64_t ldo, int mo,
              cudaStream_t s, int *grid_out) {
    const int64_t ntiles = (g.n + SpmmGeo<W>::TR - 1) / SpmmGeo<W>::TR;
    int grid = int(std::min<int64_t>(ntiles, int64_t(num_sms()) * occupancy_spmm<T, W, DOT>()));
    if (grid < 1) grid = 1;
    if (grid_out) *grid_out = grid;
    const bool lst = e.alist && e.tgen && !e.zero_inactive;
    if (g.w) {
        if (lst) k_spmm<T, W, DOT, true, true><<<grid, SPMM_THREADS, 0, s>>>(g, x, e, ldo, mo);
        else k_spmm<T, W, DOT, true, false><<<grid, SPMM_THREADS, 0, s>>>(g, x, e, ldo, mo);
    } else {
        if (lst) k_spmm<T, W, DOT, false, true><<<grid, SPMM_THREADS, 0, s>>>(g, x, e, ldo, mo);
        else k_spmm<T, W, DOT, false, false><<<grid, SPMM_THREADS, 0, s>>>(g, x, e, ldo, mo);
    }
    return 0;
}

template <typename T, int W>
int launch_w(const GraphDev &g, const T *x, const LinEpi<T> &e, int64_t ldo, int mo,
             cudaStream_t s, int *grid_out) {
    return e.dot_partials ? launch_wd<T, W, true>(g, x, e, ldo, mo, s, grid_out)
                          : launch_wd<T, W, false>(g, x, e, ldo, mo, s, grid_out);
}

}  // namespace

template <typename T>
int launch_spmm(const GraphDev &g, int W, const T *x, const LinEpi<T> &e, cudaStream_t s,
                int *grid_out, int64_t M_alg, int n_dense_in, int64_t ldo, int mo) {
    if (ldo <= 0) { ldo = W; mo = W; }
    LinEpi<T> ee = e;
    ee.prof = prof_begin(KernelClass::SPMM, s);
    switch (W) {
        case 16: launch_w<T, 16>(g, x, ee, ldo, mo, s, grid_out); break;
        case 32: launch_w<T, 32>(g, x, ee, ldo, mo, s, grid_out); break;
        case 64: launch_w<T, 64>(g, x, ee, ldo, mo, s, grid_out); break;
        case 128: launch_w<T, 128>(g, x, ee, ldo, mo, s, grid_out); break;
        default: return fail(KB_ERR_ARG, "unsupported block width");
    }
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) return cuda_fail(err, "k_spmm launch");
    // algorithmic bytes: CSR (+weights, +diagonal excess) once, the gathered block once,
    // the other dense inputs once each, the output once; flops 3 per nonzero per column
    double csr = 4.0 * double(g.n + 1) + 4.0 * double(g.nnz) + (g.w ? 4.0 * double(g.nnz) : 0.0) +
                 (g.rdiag ? 4.0 * double(g.n) : 0.0);
    double blk = double(g.n) * double(M_alg) * double(sizeof(T));
    // per processed row: its row pointer (+ diagonal excess), the gathered block counted
    // once, the other dense inputs and the output; per stored nonzero: index (+ weight)
    const double per_row = 4.0 + (g.rdiag ? 4.0 : 0.0) +
                           double(M_alg) * double(sizeof(T)) * (2 + n_dense_in);
    const double per_nnz = 4.0 + (g.w ? 4.0 : 0.0);
    const double flops_per_row = 3.0 * double(M_alg) * double(g.nnz) / double(g.n);
    prof_end(KernelClass::SPMM, s, csr + blk * (2 + n_dense_in), 3.0 * double(g.nnz) * double(M_alg),
             1, per_row, per_nnz, flops_per_row, 4.0);
    return 0;
}

template <typename T>
int spmm_max_grid(int W) {
    // dot partials are written only by the DOT variant; its grid bounds the buffer
    switch (W) {
        case 16: return num_sms() * occupancy_spmm<T, 16, true>();
        case 32: return num_sms() * occupancy_spmm<T, 32, true>();
        case 64: return num_sms() * occupancy_spmm<T, 64, true>();
        default: return num_sms() * occupancy_spmm<T, 128, true>();
    }
}

template int launch_spmm<float>(const GraphDev &, int, const float *, const LinEpi<float> &,
                                cudaStream_t, int *, int64_t, int, int64_t, int);
template int launch_spmm<double>(const GraphDev &, int, const double *, const LinEpi<double> &,
                                 cudaStream_t, int *, int64_t, int, int64_t, int);
template int launch_spmm<__nv_bfloat16>(const GraphDev &, int, const __nv_bfloat16 *,
                                        const LinEpi<__nv_bfloat16> &, cudaStream_t, int *, int64_t,
                                        int, int64_t, int);
template int spmm_max_grid<float>(int);
template int spmm_max_grid<double>(int);
template int spmm_max_grid<__nv_bfloat16>(int);

}  // namespace kb
