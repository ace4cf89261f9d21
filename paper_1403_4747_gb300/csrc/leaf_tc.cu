// Tensor-core (tcgen05) form of the per-leaf products for several
// right-hand sides at once (chosen precision):
//   near field (Step 4):  y_B  = A_B X(cols_B)   A_B: n_B x n_cols, row-major per leaf
//   S2M (Step 2, Eq. s2m): q~_B = S~_B X_B        S~ stored [n_B][T] per leaf
//   L2T (Step 3, Eq. l2t): y_B += T~_B p~_B       T~ stored [T][64] per leaf
// Each is a complex GEMM per leaf with the right-hand sides as columns:
// C (64 rows x NC columns) = A (64 x K) B (K x NC), taken as in
// translate_tc.cu with the stacked [Ar; Ai] (M = 128) against [Br Bi]
// (N = 2 NC) and three bf16 products per value (A_hi B_hi + A_hi B_lo +
// A_lo B_hi, FP32 accumulation in tensor memory).
//
// Unlike the translations, neither operand is stored split: the producer
// warps read the FP32 operator and the FP32 vectors (the near-field columns
// through the leaf's column list), split every value into bf16 hi and lo and
// write them straight into the shared-memory K-major core-matrix layout.  So
// the near-field matrix is read once per pass at 8 bytes per entry, the same
// bytes as the one-column CUDA-core kernel, for any number of columns; every
// output value is written once (leaves own disjoint element ranges), with no
// atomics.  Every mbarrier wait is bounded; on timeout the CTA records an
// error, waits (bounded) for its MMAs, frees its tensor memory and returns.
#include <cuda_bf16.h>

#include <algorithm>
#include <vector>

#include "fda_internal.cuh"
#include "tc_util.cuh"

namespace {

using namespace fda_tc;

enum { LT_NEAR = 0, LT_S2M = 1, LT_L2T = 2 };

constexpr int LT_EPC = 16;       // epilogue chunk: accumulator columns staged per pass
constexpr int LT_NPROD = 256;    // producer threads (warps 5-12)
constexpr int LT_THREADS = 416;  // 13 warps: 4 epilogue, 1 MMA, 8 producers

struct leaf_tile {
    int leaf, rt, m0, pad;  // leaf, 64-row tile of the output, first right-hand side
};

// per-level density pointers of the FP32 pass (S2M writes q~, L2T reads p~)
struct leaf_levels {
    c32f *q[FDA_MAX_LEVELS];
    const c32f *p[FDA_MAX_LEVELS];
    int64_t stride[FDA_MAX_LEVELS];  // per right-hand side: boxes x T (leaves are low frequency: one cone)
    int box0[FDA_MAX_LEVELS], T[FDA_MAX_LEVELS];
};

struct leaf_args {
    const leaf_tile *tiles;
    int ntiles;
    const int32_t *leaf_box, *bbeg, *bend, *blev;
    const int64_t *colptr;  // near field: columns of leaf li are cols[colptr[li] .. colptr[li+1])
    const int32_t *cols;
    const int64_t *off;     // near field: first entry of leaf li's block
    const int64_t *loff;    // S~ / T~: first entry of leaf li's operator
    const c32f *A;          // near blocks, S~ or T~ (FP32)
    const c32f *x;          // FP32 input vectors [m][N] (near field, S2M)
    int64_t xstr;
    c64d *y;                // FP64 output [m][N] (near field: overwritten; L2T: added)
    int64_t ldy;
    int mr;
    int *err;
};

// what every role needs to know about a tile
struct tile_info {
    int B, i0, nB, rows, K, l, T;
    int64_t c0, aoff;
};

template <int KIND>
__device__ inline tile_info get_info(const leaf_args &a, const leaf_levels &lv, const leaf_tile &t)
{
    tile_info f;
    f.B = a.leaf_box[t.leaf];
    f.i0 = a.bbeg[f.B];
    f.nB = a.bend[f.B] - f.i0;
    f.l = a.blev[f.B];
    f.T = lv.T[f.l];
    f.c0 = 0;
    if (KIND == LT_NEAR) {
        f.c0 = a.colptr[t.leaf];
        f.K = (int)(a.colptr[t.leaf + 1] - f.c0);
        f.rows = f.nB;
        f.aoff = a.off[t.leaf];
    } else if (KIND == LT_S2M) {
        f.K = f.nB;
        f.rows = f.T;
        f.aoff = a.loff[t.leaf];
    } else {
        f.K = f.T;
        f.rows = f.nB;
        f.aoff = a.loff[t.leaf];
    }
    return f;
}

// operator entry (row r of the output, column k of the contraction)
template <int KIND>
__device__ inline c32f a_at(const leaf_args &a, const tile_info &f, int r, int k)
{
    if (KIND == LT_NEAR) return a.A[f.aoff + (int64_t)r * f.K + k];
    if (KIND == LT_S2M) return a.A[f.aoff + (int64_t)k * f.T + r];
    return a.A[f.aoff + (int64_t)k * 64 + r];
}

// input entry (contraction index k, right-hand side m)
template <int KIND>
__device__ inline c32f b_at(const leaf_args &a, const leaf_levels &lv, const tile_info &f, int k, int m)
{
    if (KIND == LT_NEAR) return a.x[(int64_t)m * a.xstr + __ldg(a.cols + f.c0 + k)];
    if (KIND == LT_S2M) return a.x[(int64_t)m * a.xstr + f.i0 + k];
    return lv.p[f.l][(int64_t)m * lv.stride[f.l] + (int64_t)(f.B - lv.box0[f.l]) * f.T + k];
}

// bf16 hi and lo of two consecutive K values, packed for one 4-byte store each
__device__ inline void split2(float v0, float v1, uint32_t &hi, uint32_t &lo)
{
    const __nv_bfloat16 h0 = __float2bfloat16_rn(v0), h1 = __float2bfloat16_rn(v1);
    const __nv_bfloat16 l0 = __float2bfloat16_rn(v0 - __bfloat162float(h0));
    const __nv_bfloat16 l1 = __float2bfloat16_rn(v1 - __bfloat162float(h1));
    hi = (uint32_t)__bfloat16_as_ushort(h0) | ((uint32_t)__bfloat16_as_ushort(h1) << 16);
    lo = (uint32_t)__bfloat16_as_ushort(l0) | ((uint32_t)__bfloat16_as_ushort(l1) << 16);
}

// Persistent, warp-specialised.  CTA c takes tiles c, c + grid, ...:
//   warps 5-12 (producers): fill ring stage g % ST with the tile's operator
//       rows (64 x 32 of K, split) and its NC input columns (split), zeros
//       beyond K and beyond the last right-hand side; every producer thread
//       fences its stores to the async proxy and arrives on full[b] (count
//       LT_NPROD);
//   warp 4 (MMA): one thread issues the three products per 16 of K into the
//       tile's accumulator slot and commits them to empty[b] and, after the
//       tile's last stage, to accf[slot];
//   warps 0-3 (epilogue, one warp per TMEM lane quarter): combine real and
//       imaginary parts and write the tile's outputs, then arrive on
//       acce[slot] (count 128).
// Operator rows beyond the tile's row count are not written (their products
// land in accumulator rows that are never read).
template <int KIND, int NC, int ST>
__global__ void __launch_bounds__(LT_THREADS, 1) k_leaf_tc(leaf_args a, leaf_levels lv)
{
    extern __shared__ __align__(128) uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
    constexpr int BB = NC * KC * 2;  // one B panel (Br or Bi, hi or lo)
    constexpr int AR = 2 * ABYTES;   // A hi, A lo
    constexpr int STAGE = AR + 4 * BB;
    constexpr int SLOT = 2 * NC;     // TMEM columns of one accumulator slot
    constexpr int TALLOC = 2 * SLOT <= 32 ? 32 : (2 * SLOT <= 64 ? 64 : (2 * SLOT <= 128 ? 128 : 256));
    static_assert(NC % 16 == 0 && NC <= 64, "N = 2 NC must be a multiple of 32 and at most 128");
    float2 *stg = reinterpret_cast<float2 *>(smem + ST * STAGE);  // epilogue staging [EPC][128 lanes]
    __shared__ uint32_t tmem_base;
    __shared__ __align__(8) uint64_t full[ST], empty[ST], accf[2], acce[2];
    __shared__ int abort_flag, n_commit;
    volatile int *abort_v = &abort_flag;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int my_tiles = (int)blockIdx.x < a.ntiles ? (a.ntiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "r"(TALLOC));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        for (int b = 0; b < ST; ++b) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&full[b])), "r"(LT_NPROD));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&empty[b])));
        }
        for (int b = 0; b < 2; ++b) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&accf[b])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&acce[b])), "r"(128));
        }
        asm volatile("fence.mbarrier_init.release.cluster;");
        abort_flag = 0;
        n_commit = 0;
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = tmem_base;

    if (warp >= 5) {
        // ---------------- producers
        // Each thread's loads of a stage are issued together, into registers,
        // before it waits for the ring slot; the split and the shared-memory
        // stores follow.  Item i of thread tp: operator item tp + i LT_NPROD
        // (row, pair of K) and input item tp + i LT_NPROD (column, pair of K).
        constexpr int AI = 64 * 16 / LT_NPROD;  // operator items per thread
        constexpr int BI = NC * 16 / LT_NPROD;  // input items per thread
        static_assert(AI >= 1 && BI >= 1, "at least one item per producer thread");
        const int tp = tid - 160;
        int g = 0;
        bool ok = true;
        // every input item of this thread has the same pair of K in its stage
        // (LT_NPROD is a multiple of 16): for the near field its two column
        // indices are fetched one stage ahead, so the gather of x waits on one
        // memory latency, not two
        const int kp_b = tp & 15;
        for (int j = 0; j < my_tiles && ok; ++j) {
            const leaf_tile t = a.tiles[blockIdx.x + (int64_t)j * gridDim.x];
            const tile_info f = get_info<KIND>(a, lv, t);
            const int nkc = (f.K + KC - 1) / KC;
            const int rmax = min(64, f.rows - 64 * t.rt);
            int cn0 = -1, cn1 = -1;  // near field: column elements of the next stage
            if (KIND == LT_NEAR) {
                const int k = 2 * kp_b;
                if (k < f.K) cn0 = __ldg(a.cols + f.c0 + k);
                if (k + 1 < f.K) cn1 = __ldg(a.cols + f.c0 + k + 1);
            }
            for (int s = 0; s < nkc; ++s, ++g) {
                const int b = g % ST;
                const int k0 = s * KC;
                const int ce0 = cn0, ce1 = cn1;
                c32f av[AI][2], bv[BI][2];
#pragma unroll
                for (int i = 0; i < AI; ++i) {
                    const int e = tp + i * LT_NPROD;
                    const int r = KIND == LT_NEAR ? e >> 4 : e & 63;
                    const int kp = KIND == LT_NEAR ? e & 15 : e >> 6;
                    const int k = k0 + 2 * kp, rg = 64 * t.rt + r;
                    av[i][0] = c32f();
                    av[i][1] = c32f();
                    if (r < rmax) {
                        if (k < f.K) av[i][0] = a_at<KIND>(a, f, rg, k);
                        if (k + 1 < f.K) av[i][1] = a_at<KIND>(a, f, rg, k + 1);
                    }
                }
#pragma unroll
                for (int i = 0; i < BI; ++i) {
                    const int e = tp + i * LT_NPROD;
                    const int n = e >> 4, k = k0 + 2 * (e & 15), m = t.m0 + n;
                    bv[i][0] = c32f();
                    bv[i][1] = c32f();
                    if (m < a.mr) {
                        if (KIND == LT_NEAR) {
                            if (ce0 >= 0) bv[i][0] = a.x[(int64_t)m * a.xstr + ce0];
                            if (ce1 >= 0) bv[i][1] = a.x[(int64_t)m * a.xstr + ce1];
                        } else {
                            if (k < f.K) bv[i][0] = b_at<KIND>(a, lv, f, k, m);
                            if (k + 1 < f.K) bv[i][1] = b_at<KIND>(a, lv, f, k + 1, m);
                        }
                    }
                }
                if (KIND == LT_NEAR) {
                    const int k = k0 + KC + 2 * kp_b;
                    cn0 = k < f.K ? __ldg(a.cols + f.c0 + k) : -1;
                    cn1 = k + 1 < f.K ? __ldg(a.cols + f.c0 + k + 1) : -1;
                }
                const bool fail = g >= ST && !mbar_wait_ab(smem_u32(&empty[b]), ((g - ST) / ST) & 1, abort_v);
                if (bar_any(1, LT_NPROD, fail)) {
                    if (fail && !*abort_v) atomicExch(a.err, 2);
                    *abort_v = 1;
                    ok = false;
                    break;
                }
                uint8_t *st = smem + b * STAGE;
                // operator: Re rows 0-63, Im rows 64-127, hi then lo
#pragma unroll
                for (int i = 0; i < AI; ++i) {
                    const int e = tp + i * LT_NPROD;
                    const int r = KIND == LT_NEAR ? e >> 4 : e & 63;
                    const int kp = KIND == LT_NEAR ? e & 15 : e >> 6;
                    if (r >= rmax) continue;
                    uint32_t rh, rl, ih, il;
                    split2(av[i][0].re, av[i][1].re, rh, rl);
                    split2(av[i][0].im, av[i][1].im, ih, il);
                    const int ore = core_off(r, 2 * kp), oim = core_off(64 + r, 2 * kp);
                    *reinterpret_cast<uint32_t *>(st + ore) = rh;
                    *reinterpret_cast<uint32_t *>(st + oim) = ih;
                    *reinterpret_cast<uint32_t *>(st + ABYTES + ore) = rl;
                    *reinterpret_cast<uint32_t *>(st + ABYTES + oim) = il;
                }
                // inputs: Br hi, Bi hi, Br lo, Bi lo panels of NC rows
                uint8_t *sb = st + AR;
#pragma unroll
                for (int i = 0; i < BI; ++i) {
                    const int e = tp + i * LT_NPROD;
                    uint32_t rh, rl, ih, il;
                    split2(bv[i][0].re, bv[i][1].re, rh, rl);
                    split2(bv[i][0].im, bv[i][1].im, ih, il);
                    const int o = core_off(e >> 4, 2 * (e & 15));
                    *reinterpret_cast<uint32_t *>(sb + o) = rh;
                    *reinterpret_cast<uint32_t *>(sb + BB + o) = ih;
                    *reinterpret_cast<uint32_t *>(sb + 2 * BB + o) = rl;
                    *reinterpret_cast<uint32_t *>(sb + 3 * BB + o) = il;
                }
                // the MMAs read this stage through the async proxy
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&full[b])) : "memory");
            }
        }
    } else if (warp == 4) {
        // ---------------- MMA issue (one thread)
        if (lane == 0) {
            // bf16 x bf16 -> f32, K-major A and B, M = 128, N = 2 NC
            const uint32_t idesc =
                (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)((2 * NC) >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
            int g = 0;
            bool ok = true;
            for (int j = 0; j < my_tiles && ok; ++j) {
                const int slot = j & 1;
                if (j >= 2 && !mbar_wait_ab(smem_u32(&acce[slot]), ((j - 2) >> 1) & 1, abort_v)) {
                    if (!*abort_v) atomicExch(a.err, 3);
                    *abort_v = 1;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;");
                const uint32_t dslot = tmem + slot * SLOT;
                const leaf_tile t = a.tiles[blockIdx.x + (int64_t)j * gridDim.x];
                const tile_info f = get_info<KIND>(a, lv, t);
                const int nkc = (f.K + KC - 1) / KC;
                for (int s = 0; s < nkc; ++s, ++g) {
                    const int b = g % ST;
                    if (!mbar_wait_ab(smem_u32(&full[b]), (g / ST) & 1, abort_v)) {
                        if (!*abort_v) atomicExch(a.err, 1);
                        *abort_v = 1;
                        ok = false;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;");
                    const uint32_t base = smem_u32(smem + b * STAGE);
                    const uint32_t aHi = base, aLo = base + ABYTES, bHi = base + AR, bLo = bHi + 2 * BB;
                    for (int k = 0; k < KC / 16; ++k) {
                        const uint32_t so = k * 256;  // two core matrices along K per k-step
                        const uint32_t en = (s > 0 || k > 0) ? 1u : 0u;
                        asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                                     "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(dslot),
                                     "l"(smem_desc(aHi + so)), "l"(smem_desc(bHi + so)), "r"(idesc), "r"(en));
                        asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                                     "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(dslot),
                                     "l"(smem_desc(aHi + so)), "l"(smem_desc(bLo + so)), "r"(idesc), "r"(1u));
                        asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                                     "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(dslot),
                                     "l"(smem_desc(aLo + so)), "l"(smem_desc(bHi + so)), "r"(idesc), "r"(1u));
                    }
                    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                        smem_u32(&empty[b])));
                    n_commit = g + 1;
                }
                if (!ok) break;
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                    smem_u32(&accf[slot])));
            }
        }
        __syncwarp();
    } else {
        // ---------------- epilogue (warps 0-3 = TMEM lanes 0-127)
        // lane r < 64 holds Ar rows (D1 -> Re, D2 -> Im); lane r >= 64 holds
        // Ai rows (D1 -> Im, D2 -> -Re).  Per chunk of EPC columns every lane
        // stages (D1, D2); then thread (row, half) combines the two lanes of
        // its row for EPC / 2 columns and writes them.
        const int row = (warp & 1) * 32 + lane, half = warp >> 1;
        for (int j = 0; j < my_tiles; ++j) {
            const int slot = j & 1;
            const leaf_tile t = a.tiles[blockIdx.x + (int64_t)j * gridDim.x];
            const tile_info f = get_info<KIND>(a, lv, t);
            const bool have = mbar_wait_ab(smem_u32(&accf[slot]), (j >> 1) & 1, abort_v);
            if (bar_any(2, 128, !have)) {
                if (!have && !*abort_v) atomicExch(a.err, 4);
                *abort_v = 1;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;");
            const uint32_t d1 = tmem + slot * SLOT + ((uint32_t)(warp * 32) << 16), d2 = d1 + NC;
            const int rmax = min(64, f.rows - 64 * t.rt);
            const int ncols = min(NC, a.mr - t.m0);
            for (int c0 = 0; c0 < ncols; c0 += LT_EPC) {
                uint32_t v1[16], v2[16];
                tmem_ld16x2(d1 + c0, d2 + c0, v1, v2);
#pragma unroll
                for (int jj = 0; jj < LT_EPC; ++jj)
                    stg[jj * 128 + tid] = make_float2(__uint_as_float(v1[jj]), __uint_as_float(v2[jj]));
                asm volatile("bar.sync 2, 128;");
                if (row < rmax) {
#pragma unroll
                    for (int jj = half * (LT_EPC / 2); jj < (half + 1) * (LT_EPC / 2); ++jj) {
                        const int n = c0 + jj;
                        if (n < ncols) {
                            const float2 top = stg[jj * 128 + row], bot = stg[jj * 128 + 64 + row];
                            const float re = top.x - bot.y, im = top.y + bot.x;
                            const int64_t m = t.m0 + n;
                            if (KIND == LT_NEAR) {
                                a.y[m * a.ldy + f.i0 + row] = c64d((double)re, (double)im);
                            } else if (KIND == LT_S2M) {
                                lv.q[f.l][m * lv.stride[f.l] + (int64_t)(f.B - lv.box0[f.l]) * f.T + 64 * t.rt + row] =
                                    c32f(re, im);
                            } else {
                                c64d *yp = a.y + m * a.ldy + f.i0 + row;
                                const c64d o = *yp;
                                *yp = c64d(o.re + (double)re, o.im + (double)im);
                            }
                        }
                    }
                }
                asm volatile("bar.sync 2, 128;");
            }
            // this slot is read: the MMAs of tile j + 2 may overwrite it
            asm volatile("tcgen05.fence::before_thread_sync;");
            asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&acce[slot])));
        }
    }
    __syncthreads();
    // drain after an error: the last MMA commit covers every MMA issued before it
    const int nc = n_commit;
    if (*abort_v && nc > 0 && tid == 0) mbar_wait(smem_u32(&empty[(nc - 1) % ST]), ((nc - 1) / ST) & 1);
    asm volatile("tcgen05.fence::after_thread_sync;");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TALLOC));
}

template <int KIND, int NC>
void launch_leaf(const leaf_args &a, const leaf_levels &lv, cudaStream_t s)
{
    constexpr int ST = 4;
    const size_t stage = 2 * (size_t)ABYTES + 4 * (size_t)NC * KC * 2;
    const size_t smem = 128 + ST * stage + (size_t)LT_EPC * 128 * sizeof(float2);
    static int per_sm = 0, nsm = 0;  // resident CTAs per SM for this instantiation
    if (!per_sm) {
        int dev = 0;
        FDA_CUDA(cudaGetDevice(&dev));
        FDA_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
        FDA_CUDA(cudaFuncSetAttribute(k_leaf_tc<KIND, NC, ST>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        FDA_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_leaf_tc<KIND, NC, ST>, LT_THREADS, smem));
        if (per_sm < 1) fda_fail(FDA_ERR_CUDA, "tensor-core leaf kernel does not fit on an SM");
    }
    const int grid = std::min(a.ntiles, per_sm * nsm);
    k_leaf_tc<KIND, NC, ST><<<grid, LT_THREADS, smem, s>>>(a, lv);
}

}  // namespace

// Leaf products on the tensor cores for mr right-hand sides (chosen
// precision).  kind 0: y = A_near x (overwrites y); kind 1: q~ = S~ x at
// the leaves (q32 densities); kind 2: y += T~ p~ (p32 densities).  A: the
// FP32 near-field blocks, S~ or T~ of the side being applied; x: FP32
// [mr][N]; y: FP64 [mr][N].  Tile lists are cut once per (kind, right-hand
// sides, width) and kept for the handle's lifetime (captured graphs point
// into them).
void fda_leaf_tc(fda_handle *h, int kind, const dbuf &A, const c32f *x, c64d *y, int mr)
{
    if (mr < 1) return;
    const int NC = mr <= 16 ? 16 : (mr <= 32 ? 32 : 64);
    fda_handle::leaf_tile_set *ts = nullptr;
    for (auto &t : h->leaf_sets)
        if (t.kind == kind && t.mr == mr && t.nc == NC) ts = &t;
    if (!ts) {
        std::vector<leaf_tile> tiles;
        for (int li = 0; li < h->nleaf; ++li) {
            const int l = h->h_leaf_level[li];
            const int T = (h->lev[l].active ? h->lev[l].T : 0);
            if (kind != LT_NEAR && T == 0) continue;
            const int nrt = kind == LT_S2M ? (T + 63) / 64 : 1;
            for (int rt = 0; rt < nrt; ++rt)
                for (int m0 = 0; m0 < mr; m0 += NC) tiles.push_back(leaf_tile{li, rt, m0, 0});
        }
        h->leaf_sets.emplace_back();
        ts = &h->leaf_sets.back();
        ts->kind = kind;
        ts->mr = mr;
        ts->nc = NC;
        ts->n = (int)tiles.size();
        ts->buf.alloc(sizeof(leaf_tile) * std::max<size_t>(tiles.size(), 1));
        if (!tiles.empty())
            FDA_CUDA(cudaMemcpy(ts->buf.p, tiles.data(), sizeof(leaf_tile) * tiles.size(), cudaMemcpyHostToDevice));
    }
    if (ts->n == 0) return;
    if (!h->tc_err.p) {
        h->tc_err.alloc(sizeof(int));
        FDA_CUDA(cudaMemsetAsync(h->tc_err.p, 0, sizeof(int), h->stream));
    }
    leaf_levels lv;
    for (int l = 0; l < FDA_MAX_LEVELS; ++l) {
        const bool act = l < h->nlev && h->lev[l].active;
        lv.q[l] = act ? h->q32[l].as<c32f>() : nullptr;
        lv.p[l] = act ? h->p32[l].as<c32f>() : nullptr;
        lv.T[l] = act ? h->lev[l].T : 0;
        lv.box0[l] = l < h->nlev ? h->lev[l].box0 : 0;
        lv.stride[l] = act ? (int64_t)h->lev[l].nbox * h->lev[l].ncones * h->lev[l].T : 0;
    }
    leaf_args a;
    a.tiles = ts->buf.as<leaf_tile>();
    a.ntiles = ts->n;
    a.leaf_box = h->leaf_box.as<int32_t>();
    a.bbeg = h->box_begin.as<int32_t>();
    a.bend = h->box_end.as<int32_t>();
    a.blev = h->box_level.as<int32_t>();
    a.colptr = h->nf_colptr.as<int64_t>();
    a.cols = h->nf_cols.as<int32_t>();
    a.off = h->nf_off.as<int64_t>();
    a.loff = h->leaf_op_off.as<int64_t>();
    a.A = A.as<c32f>();
    a.x = x;
    a.xstr = h->N;
    a.y = y;
    a.ldy = h->N;
    a.mr = mr;
    a.err = h->tc_err.as<int>();
    cudaStream_t s = h->stream;
    if (kind == LT_NEAR) {
        if (NC == 16) launch_leaf<LT_NEAR, 16>(a, lv, s);
        else if (NC == 32) launch_leaf<LT_NEAR, 32>(a, lv, s);
        else launch_leaf<LT_NEAR, 64>(a, lv, s);
    } else if (kind == LT_S2M) {
        if (NC == 16) launch_leaf<LT_S2M, 16>(a, lv, s);
        else if (NC == 32) launch_leaf<LT_S2M, 32>(a, lv, s);
        else launch_leaf<LT_S2M, 64>(a, lv, s);
    } else {
        if (NC == 16) launch_leaf<LT_L2T, 16>(a, lv, s);
        else if (NC == 32) launch_leaf<LT_L2T, 32>(a, lv, s);
        else launch_leaf<LT_L2T, 64>(a, lv, s);
    }
    FDA_CHECK_LAUNCH();
}
