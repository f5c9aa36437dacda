// Tall-skinny block kernels of the classical block Lanczos step (Algorithm 1: diagonal
// block, three-term update, reduced QR) on the fifth-generation tensor cores, for FP32
// blocks of width 64:
//   PROJ     G = Qa^T X
//   UPD      out = X - Qa Ca - Qb Cb, G = out^T out      (Qa may be absent)
//   MULGRAM  out = X Ca, G = out^T out
//   MUL      out = X Ca
// (same contract as the SIMT k_rowblock of rowblock.cu, which serves the other widths,
// precisions and the assemblies).
//
// FP32 accuracy from BF16 tensor-core products.  Every FP32 operand value v is split into
// three BF16 parts v = v0 + v1 + v2 + r, |r| <= 2^-24 |v| (each part is the BF16 rounding
// of what the previous parts left), and a product a * c is formed from the six part
// products a_i c_j with i + j <= 2; the dropped terms are of relative size 2^-24.  BF16 x
// BF16 products are exact in FP32 and the tensor core accumulates in FP32 (in TMEM), so
// the result carries FP32-level rounding: on random 128 x 64 by 64 x 64 products its error
// against FP64 is below that of an FP32 FMA loop.
//
// Schedule.  One persistent CTA of 256 threads (8 warps) per SM (the occupancy of a TMEM-
// allocating kernel is one CTA per SM) walks its tiles of 128 rows.  The work is a stream
// of operand tiles (for each tile, each source of the product; PROJ: the pair Qa, X): an
// operand's 16-byte loads are issued into registers one operand ahead, then its three BF16
// parts are stored in one of two shared-memory buffers (K-major 8 x 16-byte core matrices)
// and one thread issues its tcgen05.mma instructions (M = 128 rows, N = 64, K = 16 each;
// 6 part pairs x 4 K steps) into one of two TMEM product accumulators, committed to the
// buffer's mbarrier.  Before a buffer is refilled its mbarrier is awaited; if the operand
// that used it was the last of a tile, that tile's epilogue runs then: the accumulator is
// read with tcgen05.ld (warp w: rows 32 (w%4).., columns 32 (w/4)..), UPD subtracts it
// from the rows of X, the output rows are stored, and for the Gram the output's BF16 parts
// go row-major into core matrices (the MN-major layout) and the Gram tcgen05.mma
// instructions (K = the tile's rows) accumulate G in a third TMEM accumulator across all
// tiles of the CTA, which writes its 64 x 64 partial once at the end (summed over CTAs in
// FP64 by k_reduce, as for the SIMT kernel).  So loads, splits, MMAs and epilogues of
// consecutive operands overlap.  The Gram instruction has M = 128 with the left operand's
// rows 64..127 reading the next 16 KB of shared memory; those accumulator rows are never
// read.
//
// Waits on the mbarriers are bounded; a wait that runs out sets the control block's status
// to KB_ERR_CUDA and stops the process, and every CTA releases its TMEM before returning.
#include <algorithm>
#include <type_traits>

#include "kb_internal.cuh"

namespace kb {
namespace {

constexpr int TC_THREADS = 256;
constexpr int TC_TM = 128;                    // rows per tile = TMEM lanes
constexpr int TC_W = 64;                      // block width (K of the product, N, Gram size)
constexpr int TC_TILE = TC_TM * TC_W * 2;     // bytes of one BF16 part of a tile (16 KB)
constexpr int TC_CMAT = TC_W * TC_W * 2;      // bytes of one BF16 part of a W x W matrix
constexpr int TC_BUF = 3 * TC_TILE;           // the three parts of one operand tile
constexpr int TC_TMEM_COLS = 256;             // product accumulators 0..63, 64..127; Gram 128..191
constexpr long TC_WAIT_LIMIT = 1L << 22;      // mbarrier polls before giving up

template <int MODE>
struct TcCfg {
    static constexpr bool PROD = MODE != RB_PROJ;
    static constexpr bool GRAM = MODE != RB_MUL;
    static constexpr int NO = (PROD && GRAM) ? 1 : 0;     // Gram operand buffer (output parts)
    static constexpr int NB = PROD ? 2 : 4;               // operand buffers (PROJ: two pairs)
    static constexpr int NC = MODE == RB_UPD ? 2 : (PROD ? 1 : 0);
    static constexpr int OFF_OP = NO * TC_BUF;
    static constexpr int OFF_C = OFF_OP + NB * TC_BUF;
    static constexpr int OFF_BAR = OFF_C + NC * 3 * TC_CMAT;
    static constexpr int SMEM = OFF_BAR + 128;
    // the Gram instruction's left operand (M = 128) reaches 32 KB past the start of each of
    // its parts, the right operand (N = 64) 16 KB: both stay inside the buffers
    static constexpr int REACH_LEFT = 2 * TC_TILE + 7 * 256 + 128 + 15 * 2048 + 128;
    static constexpr int REACH_RIGHT = 2 * TC_TILE + 7 * 256 + 128 + 7 * 2048 + 128;
    static_assert(!GRAM || !PROD || REACH_LEFT <= OFF_BAR, "Gram operand reach");
    // PROJ: the left operand of a pair is followed by the pair's right operand
    static_assert(PROD || (REACH_LEFT <= 2 * TC_BUF && REACH_RIGHT <= TC_BUF), "Gram operand reach");
    static_assert(SMEM <= 227 * 1024, "shared memory");
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
// K-major core layout of a rows x 64 operand (row r, k), in BF16 units: core (r/8, k/8) at
// ((r/8) * 8 + k/8) * 128 bytes, row r%8 of the core at 16 (r%8) bytes
__device__ __forceinline__ int kmaj(int r, int k) {
    return ((r >> 3) * 8 + (k >> 3)) * 64 + (r & 7) * 8 + (k & 7);
}
// MN-major core layout of a 128 x 64 tile (row r = K index, column c = M or N index), in
// BF16 units: core (c/8, r/8) at (c/8) * 2048 + (r/8) * 128 bytes, i.e. 16 r + 2 (c%8)
// bytes past the start of the column group
__device__ __forceinline__ int mnmaj(int r, int c) {
    return (c >> 3) * 1024 + r * 8 + (c & 7);
}
// shared-memory matrix descriptor: start, K-direction core stride (LBO), M/N-direction
// core stride (SBO), descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    return uint64_t((saddr >> 4) & 0x3FFF) | (uint64_t((lbo >> 4) & 0x3FFF) << 16) |
           (uint64_t((sbo >> 4) & 0x3FFF) << 32) | (uint64_t(1) << 46);
}
// instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, major-ness, N, M
__host__ __device__ constexpr uint32_t mma_idesc(int M, int N, int a_mn, int b_mn) {
    return (1u << 4) | (1u << 7) | (1u << 10) | (uint32_t(a_mn) << 15) | (uint32_t(b_mn) << 16) |
           (uint32_t(N >> 3) << 17) | (uint32_t(M >> 4) << 24);
}
__device__ __forceinline__ void mma_bf16(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                 " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
                 ::"r"(d), "l"(a), "l"(b), "r"(idesc), "r"(acc));
}
__device__ __forceinline__ void mma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                 ::"r"(smem_u32(bar)));
}
__device__ __forceinline__ bool bar_wait(uint64_t *bar, uint32_t parity) {
    const uint32_t addr = smem_u32(bar);
    for (long i = 0; i < TC_WAIT_LIMIT; ++i) {
        uint32_t ok;
        asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                     " selp.u32 %0, 1, 0, p;\n}\n"
                     : "=r"(ok) : "r"(addr), "r"(parity) : "memory");
        if (ok) return true;
    }
    return false;
}
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// 16 consecutive FP32 columns of this thread's TMEM lane
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float *v) {
    uint32_t r[16];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                   "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int q = 0; q < 16; ++q) v[q] = __uint_as_float(r[q]);
}

// three BF16 parts of v, packed for four consecutive values: p[s] holds part s of v[0..3]
__device__ __forceinline__ void split4(const float (&v)[4], uint2 (&p)[3]) {
    uint32_t w[3][2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        __nv_bfloat16 a[3], b[3];
        float ra = v[2 * h], rb = v[2 * h + 1];
#pragma unroll
        for (int s = 0; s < 3; ++s) {
            a[s] = __float2bfloat16_rn(ra);
            b[s] = __float2bfloat16_rn(rb);
            ra -= __bfloat162float(a[s]);
            rb -= __bfloat162float(b[s]);
        }
#pragma unroll
        for (int s = 0; s < 3; ++s) {
            __nv_bfloat162 t = __halves2bfloat162(a[s], b[s]);
            w[s][h] = *reinterpret_cast<uint32_t *>(&t);
        }
    }
#pragma unroll
    for (int s = 0; s < 3; ++s) p[s] = make_uint2(w[s][0], w[s][1]);
}

// A 128 x 64 FP32 tile (rows r0.. of src, zero past n) is moved in two steps: load_tile
// issues its 16-byte loads into registers (8 per thread), store_tile splits the values and
// stores the three BF16 parts in the K-major (MN = false) or MN-major (MN = true) core
// layout.  The loads of the next operand are issued before the wait for the current MMAs,
// so their latency overlaps the tensor-core work.  A warp covers 8 rows x 16 columns per
// step: lane l takes row 8 g + l/4, columns 16 q + 4 (l%4); each part store of a warp then
// fills 256 contiguous (K-major) or two 128-byte (MN-major) shared-memory spans, without
// bank conflicts.
constexpr int TC_UNITS = (TC_TM / 8) * (TC_W / 16) / (TC_THREADS / 32);   // loads per thread
__device__ __forceinline__ void load_tile(const float *__restrict__ src, int64_t r0, int64_t n,
                                          float4 (&v)[TC_UNITS]) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < TC_UNITS; ++i) {
        const int u = warp + i * (TC_THREADS / 32);
        const int g = u / (TC_W / 16), q = u % (TC_W / 16);
        const int r = g * 8 + (lane >> 2), k = q * 16 + (lane & 3) * 4;
        v[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (r0 + r < n) v[i] = __ldg(reinterpret_cast<const float4 *>(src + (r0 + r) * TC_W + k));
    }
}
template <bool MN>
__device__ __forceinline__ void store_tile(const float4 (&v)[TC_UNITS], __nv_bfloat16 *dst) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < TC_UNITS; ++i) {
        const int u = warp + i * (TC_THREADS / 32);
        const int g = u / (TC_W / 16), q = u % (TC_W / 16);
        const int r = g * 8 + (lane >> 2), k = q * 16 + (lane & 3) * 4;
        const float vv[4] = {v[i].x, v[i].y, v[i].z, v[i].w};
        uint2 p[3];
        split4(vv, p);
        const int o = MN ? mnmaj(r, k) : kmaj(r, k);
#pragma unroll
        for (int s = 0; s < 3; ++s) *reinterpret_cast<uint2 *>(dst + s * (TC_TILE / 2) + o) = p[s];
    }
}

// L2 prefetch of a tile's rows (32 KB: one 128-byte line per thread)
__device__ __forceinline__ void prefetch_tile(const float *src, int64_t r0, int64_t n) {
    if (!src || r0 >= n) return;
    const int64_t rows = n - r0 < TC_TM ? n - r0 : TC_TM;
    const char *b = reinterpret_cast<const char *>(src + r0 * TC_W);
    for (int64_t off = int64_t(threadIdx.x) * 128; off < rows * TC_W * 4; off += TC_THREADS * 128)
        asm volatile("prefetch.global.L2 [%0];" ::"l"(b + off));
}

// part pairs (a_i, c_j), i + j <= 2, smallest first
__constant__ int c_pa[6] = {2, 1, 0, 1, 0, 0};
__constant__ int c_pb[6] = {0, 1, 2, 0, 1, 0};

template <int MODE>
__global__ void __launch_bounds__(TC_THREADS, 1) k_rowblock_tc(RowArgs<float> a) {
    using G = TcCfg<MODE>;
    constexpr int TB = TC_TILE / 2;   // BF16 elements of one part
    if (a.ctrl && a.ctrl->stop) return;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    __nv_bfloat16 *sO = reinterpret_cast<__nv_bfloat16 *>(smem_raw);
    __nv_bfloat16 *sB = reinterpret_cast<__nv_bfloat16 *>(smem_raw + G::OFF_OP);
    __nv_bfloat16 *sC = reinterpret_cast<__nv_bfloat16 *>(smem_raw + G::OFF_C);
    uint64_t *bar_op = reinterpret_cast<uint64_t *>(smem_raw + G::OFF_BAR);        // [2]
    uint64_t *bar_g = reinterpret_cast<uint64_t *>(smem_raw + G::OFF_BAR + 16);
    uint32_t *s_tmem = reinterpret_cast<uint32_t *>(smem_raw + G::OFF_BAR + 24);
    unsigned long long *s_cnt = reinterpret_cast<unsigned long long *>(smem_raw + G::OFF_BAR + 32);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    if (tid == 0) {
        s_cnt[0] = 0ull;
        s_cnt[1] = 0ull;
        for (int i = 0; i < 3; ++i)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar_op + i)));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(smem_u32(s_tmem)), "r"(TC_TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    // sources of the product and their W x W matrices
    const float *src[2] = {a.x, nullptr};
    const float *cm[2] = {a.ca, nullptr};
    int nsrc = G::PROD ? 1 : 2;
    if (MODE == RB_UPD) {
        if (a.qa) { src[0] = a.qa; cm[0] = a.ca; src[1] = a.qb; cm[1] = a.cb; nsrc = 2; }
        else { src[0] = a.qb; cm[0] = a.cb; }
    }
    if (!G::PROD) { src[0] = a.qa; src[1] = a.x; }
    // B operands of the product: C^T (element (n, k) = C[k][n]) in three parts, K-major
    if (G::PROD)
        for (int m = 0; m < nsrc; ++m)
            for (int idx = tid; idx < TC_W * TC_W / 4; idx += TC_THREADS) {
                const int k = idx / (TC_W / 4), n0 = (idx % (TC_W / 4)) * 4;
                const float4 t = __ldg(reinterpret_cast<const float4 *>(cm[m] + k * TC_W + n0));
                const float v[4] = {t.x, t.y, t.z, t.w};
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    float rv = v[q];
#pragma unroll
                    for (int s = 0; s < 3; ++s) {
                        const __nv_bfloat16 h = __float2bfloat16_rn(rv);
                        rv -= __bfloat162float(h);
                        sC[(m * 3 + s) * (TC_CMAT / 2) + kmaj(n0 + q, k)] = h;
                    }
                }
            }
    fence_async_smem();
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = *s_tmem;
    const uint32_t d_gram = tmem + 128;
    const uint32_t id_prod = mma_idesc(TC_TM, TC_W, 0, 0);
    const uint32_t id_gram = mma_idesc(TC_TM, TC_W, 1, 1);
    const uint32_t trow = uint32_t((warp & 3) * 32) << 16;   // this warp's TMEM lanes
    const int ecol = (warp >> 2) * 32;                        // this warp's accumulator columns
    const int erow = (warp & 3) * 32 + lane;                  // this thread's tile row

    const int64_t ntiles = (a.n + TC_TM - 1) / TC_TM;
    // the CTA's tiles inside the frontier (all others are zero in every operand)
    auto next_active = [&](int64_t t) {
        for (; t < ntiles; t += gridDim.x) {
            const int64_t q0 = t * TC_TM;
            const int rr = (a.n - q0 < TC_TM) ? int(a.n - q0) : TC_TM;
            if (!a.tgen || tile_min_gen(a.tgen, q0, rr) <= a.limit) break;
        }
        return t;
    };

    bool failed = false;
    uint32_t n_op[2] = {0u, 0u};   // commits made on bar_op[b]
    uint32_t n_g = 0u;             // Gram instruction groups issued
    // what the last operand in buffer b belonged to (product modes)
    int64_t b_tile[2] = {-1, -1};
    int b_acc[2] = {0, 0};
    bool b_last[2] = {false, false};

    // epilogue of tile te whose product is complete in accumulator acc
    auto epilogue = [&](int64_t te, int acc) -> bool {
        fence_after();
        if (G::GRAM && n_g > 0) {
            // the previous Gram instructions read sO: wait before overwriting it
            if (!bar_wait(bar_g, (n_g - 1u) & 1u)) return false;
        }
        const int64_t row = te * TC_TM + erow;
        const uint32_t dacc = tmem + uint32_t(acc * 64);
#pragma unroll 1
        for (int c0 = ecol; c0 < ecol + 32; c0 += 16) {
            float v[16];
            tmem_ld16(dacc + trow + c0, v);
            if (row < a.n) {
                if (MODE == RB_UPD) {
#pragma unroll
                    for (int c = 0; c < 16; c += 4) {
                        const float4 xv = __ldg(reinterpret_cast<const float4 *>(a.x + row * TC_W + c0 + c));
                        v[c] = xv.x - v[c]; v[c + 1] = xv.y - v[c + 1];
                        v[c + 2] = xv.z - v[c + 2]; v[c + 3] = xv.w - v[c + 3];
                    }
                }
#pragma unroll
                for (int c = 0; c < 16; c += 4)
                    *reinterpret_cast<float4 *>(a.out + row * TC_W + c0 + c) =
                        make_float4(v[c], v[c + 1], v[c + 2], v[c + 3]);
            } else {
#pragma unroll
                for (int c = 0; c < 16; ++c) v[c] = 0.f;
            }
            if constexpr (G::GRAM) {
#pragma unroll
                for (int c = 0; c < 16; c += 8) {
                    uint2 p0[3], p1[3];
                    const float lo[4] = {v[c], v[c + 1], v[c + 2], v[c + 3]};
                    const float hi[4] = {v[c + 4], v[c + 5], v[c + 6], v[c + 7]};
                    split4(lo, p0);
                    split4(hi, p1);
#pragma unroll
                    for (int s = 0; s < 3; ++s)
                        *reinterpret_cast<uint4 *>(sO + s * TB + mnmaj(erow, c0 + c)) =
                            make_uint4(p0[s].x, p0[s].y, p1[s].x, p1[s].y);
                }
            }
        }
        fence_async_smem();
        fence_before();
        __syncthreads();
        if (G::GRAM && tid == 0) {
            fence_after();
            for (int t = 0; t < 6; ++t) {
                const uint32_t a0 = smem_u32(sO + c_pa[t] * TB), b0 = smem_u32(sO + c_pb[t] * TB);
#pragma unroll
                for (int j = 0; j < TC_TM / 16; ++j)
                    mma_bf16(d_gram, smem_desc(a0 + j * 256, 128, 2048), smem_desc(b0 + j * 256, 128, 2048),
                             id_gram, (n_g == 0 && t == 0 && j == 0) ? 0u : 1u);
            }
            mma_commit(bar_g);
        }
        if (G::GRAM) ++n_g;
        return true;
    };

    // operand stream: (tile, source m) in order; pre holds the next operand, in flight
    constexpr int NPRE = G::PROD ? 1 : 2;
    float4 pre[NPRE][TC_UNITS];
    int64_t tile = next_active(blockIdx.x);
    int m = 0;
    int lt = 0;   // local tile count (accumulator choice)
    if (tile < ntiles) {
        load_tile(src[0], tile * TC_TM, a.n, pre[0]);
        if (!G::PROD) load_tile(src[1], tile * TC_TM, a.n, pre[NPRE - 1]);
        if (MODE == RB_UPD) prefetch_tile(a.x, tile * TC_TM, a.n);
    }
    for (uint32_t j = 0;; ++j) {
        const int b = int(j & 1u);
        // free buffer b (pair b for PROJ): wait for the instructions that read it
        if (n_op[b] > 0) {
            const bool ok = bar_wait(bar_op + b, (n_op[b] - 1u) & 1u);
            if (__syncthreads_or(!ok)) { failed = true; break; }
            if (G::PROD && b_last[b]) {
                b_last[b] = false;
                const bool ok2 = epilogue(b_tile[b], b_acc[b]);
                if (__syncthreads_or(!ok2)) { failed = true; break; }
            }
        }
        if (tile >= ntiles) {
            // no operand left: finish the other buffer, then stop
            const int o = b ^ 1;
            if (n_op[o] > 0) {
                const bool ok = bar_wait(bar_op + o, (n_op[o] - 1u) & 1u);
                if (__syncthreads_or(!ok)) { failed = true; break; }
                if (G::PROD && b_last[o]) {
                    b_last[o] = false;
                    const bool ok2 = epilogue(b_tile[o], b_acc[o]);
                    if (__syncthreads_or(!ok2)) { failed = true; break; }
                }
            }
            break;
        }
        if (tid == 0 && m == 0) {
            const int64_t r0 = tile * TC_TM;
            const int rows = (a.n - r0 < TC_TM) ? int(a.n - r0) : TC_TM;
            s_cnt[0] += unsigned(rows);
            s_cnt[1] += unsigned(rows) * unsigned(nsrc);
        }
        if constexpr (G::PROD) {
            __nv_bfloat16 *buf = sB + b * (TC_BUF / 2);
            store_tile<false>(pre[0], buf);
            fence_async_smem();
            fence_before();
            __syncthreads();
            const int acc = lt & 1;
            if (tid == 0) {
                fence_after();
                for (int t = 0; t < 6; ++t) {
                    const uint32_t a0 = smem_u32(buf + c_pa[t] * TB);
                    const uint32_t b0 = smem_u32(sC + (m * 3 + c_pb[t]) * (TC_CMAT / 2));
#pragma unroll
                    for (int jj = 0; jj < TC_W / 16; ++jj)
                        mma_bf16(tmem + uint32_t(acc * 64), smem_desc(a0 + jj * 256, 128, 1024),
                                 smem_desc(b0 + jj * 256, 128, 1024), id_prod, (m == 0 && t == 0 && jj == 0) ? 0u : 1u);
                }
                mma_commit(bar_op + b);
            }
            ++n_op[b];
            b_tile[b] = tile;
            b_acc[b] = acc;
            b_last[b] = (m == nsrc - 1);
            // advance the stream and issue the next operand's loads
            if (m + 1 < nsrc) {
                ++m;
            } else {
                m = 0;
                ++lt;
                tile = next_active(tile + gridDim.x);
                if (MODE == RB_UPD && tile < ntiles) prefetch_tile(a.x, tile * TC_TM, a.n);
            }
            if (tile < ntiles) load_tile(src[m], tile * TC_TM, a.n, pre[0]);
        } else {
            __nv_bfloat16 *bl = sB + (2 * b) * (TC_BUF / 2), *br = sB + (2 * b + 1) * (TC_BUF / 2);
            store_tile<true>(pre[0], bl);
            store_tile<true>(pre[NPRE - 1], br);
            fence_async_smem();
            fence_before();
            __syncthreads();
            if (tid == 0) {
                fence_after();
                for (int t = 0; t < 6; ++t) {
                    const uint32_t a0 = smem_u32(bl + c_pa[t] * TB), b0 = smem_u32(br + c_pb[t] * TB);
#pragma unroll
                    for (int jj = 0; jj < TC_TM / 16; ++jj)
                        mma_bf16(d_gram, smem_desc(a0 + jj * 256, 128, 2048), smem_desc(b0 + jj * 256, 128, 2048),
                                 id_gram, (n_g == 0 && t == 0 && jj == 0) ? 0u : 1u);
                }
                mma_commit(bar_op + b);
            }
            ++n_op[b];
            ++n_g;   // Gram groups issued (PROJ commits them on the pair barriers)
            tile = next_active(tile + gridDim.x);
            if (tile < ntiles) {
                load_tile(src[0], tile * TC_TM, a.n, pre[0]);
                load_tile(src[1], tile * TC_TM, a.n, pre[NPRE - 1]);
            }
        }
    }
    // all Gram instructions complete (product modes: the last Gram commit; PROJ: the pair
    // barriers were awaited above)
    if (!failed && G::PROD && G::GRAM && n_g > 0) {
        const bool ok = bar_wait(bar_g, (n_g - 1u) & 1u);
        if (__syncthreads_or(!ok)) failed = true;
    }
    fence_before();
    __syncthreads();
    fence_after();
    if (failed) {
        if (tid == 0 && a.ctrl) {
            Ctrl *c = const_cast<Ctrl *>(a.ctrl);
            c->status = KB_ERR_CUDA;
            c->stop = 1;
        }
    } else if (G::GRAM && (warp & 3) < 2) {
        // rows 0..63 of the Gram accumulator: this CTA's partial
        float *p = a.partials + int64_t(blockIdx.x) * TC_W * TC_W + int64_t(erow) * TC_W;
#pragma unroll 1
        for (int c0 = ecol; c0 < ecol + 32; c0 += 16) {
            float g[16];
            if (n_g > 0) {
                tmem_ld16(d_gram + trow + c0, g);
            } else {
#pragma unroll
                for (int c = 0; c < 16; ++c) g[c] = 0.f;
            }
#pragma unroll
            for (int c = 0; c < 16; c += 4)
                *reinterpret_cast<float4 *>(p + c0 + c) = make_float4(g[c], g[c + 1], g[c + 2], g[c + 3]);
        }
    }
    if (tid == 0 && a.prof.rows) {
        atomicAdd(a.prof.rows, s_cnt[0]);
        atomicAdd(a.prof.nnz, s_cnt[1]);
    }
    fence_before();
    __syncthreads();
    if (warp == 0) {
        fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_TMEM_COLS));
    }
}

template <int MODE>
void tc_setup() {
    static const cudaError_t attr = cudaFuncSetAttribute(
        k_rowblock_tc<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, TcCfg<MODE>::SMEM);
    (void)attr;
}

template <int MODE>
int launch_tc_mode(const RowArgs<float> &a, cudaStream_t s, int max_grid, int *grid_out) {
    using G = TcCfg<MODE>;
    tc_setup<MODE>();
    const int64_t ntiles = (a.n + TC_TM - 1) / TC_TM;
    int64_t grid = std::min<int64_t>(ntiles, int64_t(num_sms()));   // one CTA per SM
    if (G::GRAM) grid = std::min<int64_t>(grid, max_grid);          // partials buffer rows
    if (grid < 1) grid = 1;
    if (grid_out) *grid_out = int(grid);
    k_rowblock_tc<MODE><<<int(grid), TC_THREADS, G::SMEM, s>>>(a);
    return 0;
}

}  // namespace

bool rowblock_tc_supported(int mode, int W) {
    return W == TC_W && (mode == RB_PROJ || mode == RB_UPD || mode == RB_MULGRAM || mode == RB_MUL);
}

int launch_rowblock_tc(int mode, const RowArgs<float> &a, cudaStream_t s, int max_grid, int *grid_out) {
    switch (mode) {
        case RB_PROJ: return launch_tc_mode<RB_PROJ>(a, s, max_grid, grid_out);
        case RB_UPD: return launch_tc_mode<RB_UPD>(a, s, max_grid, grid_out);
        case RB_MULGRAM: return launch_tc_mode<RB_MULGRAM>(a, s, max_grid, grid_out);
        case RB_MUL: return launch_tc_mode<RB_MUL>(a, s, max_grid, grid_out);
    }
    return fail(KB_ERR_ARG, "bad tensor-core row-block mode");
}

int rowblock_tc_max_grid() { return num_sms(); }

}  // namespace kb
