// Tensor-core (tcgen05) form of the batched translations (M2M, M2L, L2L) for
// the chosen precision: the operator-grouped tiles of translate.cu as bf16
// tensor-core GEMMs.
//
// A complex tile C (64 rows x NC columns) += A (64 x Tin) B (Tin x NC) is
// computed with the stacked operator [Ar; Ai] (128 rows, M = 128 per
// tcgen05.mma, each operator element stored once) against the column panels
// [Br Bi] (2 NC columns):
//     [D1 D2] = [Ar; Ai] [Br Bi],
//     Cr = D1_top - D2_bottom,  Ci = D2_top + D1_bottom.
// Each FP32 value is split into two bf16 numbers, x = x_hi + x_lo, and the
// products A_hi B_hi + A_hi B_lo + A_lo B_hi are taken with FP32 accumulation
// in tensor memory (about 16 significant bits per operand) as three MMAs per
// 16 of K, each with N = 2 NC.  A CTA tile covers R consecutive 64-row tiles
// of one operator, so every density column gathered into shared memory
// serves R row tiles.
//
// Operands in shared memory use the tcgen05 K-major layout without swizzle:
// 8-row x 16-byte core matrices, LBO = 128 B between core matrices along K,
// SBO = 512 B between 8-row groups (32 complex columns of K per stage); the
// B panels Br hi, Bi hi, Br lo, Bi lo follow one another, so [Br Bi] hi and
// [Br Bi] lo are single operands of 2 NC rows.
// The operator panels are stored in HBM already in that layout (built once in
// setup) and copied to shared memory with cp.async.bulk on an mbarrier; the
// densities, split into bf16 once per level, are gathered column by column
// with 16-byte cp.async copies that arrive on the same mbarrier.  Every
// mbarrier wait is bounded: on timeout the kernel records an error, waits
// (bounded) for its own copies and MMAs, frees its tensor memory and returns.
#include <cuda_bf16.h>

#include <algorithm>
#include <vector>

#include "fda_internal.cuh"
#include "tc_util.cuh"

namespace {

using namespace fda_tc;

struct tc_tile {
    int op, pair0, npair, rt;     // operator, first column, columns, first row tile (64 complex rows)
};

// Densities of one level split once per apply into bf16 hi/lo, laid out
// for the gather: vector v (box, cone, right-hand side) holds per K chunk of
// 32 (stage s) the four panels Re hi, Im hi, Re lo, Im lo of 32 values each,
// 256 contiguous bytes per (vector, stage): 4 Tp bf16 per vector, Tp = T
// rounded up to 32, zero beyond T.
__global__ void k_split_density(const c32f *q, int64_t nvec, int T, int Tp, __nv_bfloat16 *out)
{
    // each thread: entries j, j + 1 (j even) of one vector; their Re hi, Im hi,
    // Re lo, Im lo go out as four bf16 pairs (4-byte stores: j and j + 1 share
    // a K chunk, KC being even). Two 8-byte loads, since v * T + j is odd for
    // odd T and odd v.
    const int hp = Tp / 2;  // entry pairs per vector
    const int64_t total = nvec * hp;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t v = e / hp;
        const int j = 2 * (int)(e - v * hp);
        c32f c0(0.0f, 0.0f), c1(0.0f, 0.0f);
        if (j < T) c0 = q[v * T + j];
        if (j + 1 < T) c1 = q[v * T + j + 1];
        auto split = [](float x0, float x1, uint32_t &hi, uint32_t &lo) {
            const __nv_bfloat16 h0 = __float2bfloat16_rn(x0), h1 = __float2bfloat16_rn(x1);
            const __nv_bfloat16 l0 = __float2bfloat16_rn(x0 - __bfloat162float(h0));
            const __nv_bfloat16 l1 = __float2bfloat16_rn(x1 - __bfloat162float(h1));
            hi = (uint32_t)__bfloat16_as_ushort(h0) | ((uint32_t)__bfloat16_as_ushort(h1) << 16);
            lo = (uint32_t)__bfloat16_as_ushort(l0) | ((uint32_t)__bfloat16_as_ushort(l1) << 16);
        };
        uint32_t rh, rl, ih, il;
        split(c0.re, c1.re, rh, rl);
        split(c0.im, c1.im, ih, il);
        __nv_bfloat16 *o = out + v * 4 * Tp + (j / KC) * 4 * KC + (j % KC);
        *reinterpret_cast<uint32_t *>(o) = rh;
        *reinterpret_cast<uint32_t *>(o + KC) = ih;
        *reinterpret_cast<uint32_t *>(o + 2 * KC) = rl;
        *reinterpret_cast<uint32_t *>(o + 3 * KC) = il;
    }
}

// Persistent, warp-specialised form.  CTA c takes tiles c, c + grid,
// c + 2 grid, ...; its warps split the work of every tile:
//   warps 5-8 (producers): load stage g of the CTA into ring buffer g % ST:
//       the operator panels of the tile's row tiles by one bulk copy each,
//       the tile's density columns (256 contiguous bytes each) by 16-byte
//       cp.async copies (zero fill for columns with no pair); full[b]
//       completes when all of them have landed (arrival count = 128 producer
//       threads + 1 for the byte count);
//   warp 4 (MMA): one thread issues the stage's MMAs into the tile's
//       accumulator slot (R row tiles x [D1 D2]) and commits them to
//       empty[b] (frees the buffer) and, after the tile's last stage, to
//       accf[slot];
//   warps 0-3 (epilogue, one warp per TMEM lane quarter): read the slot,
//       combine real and imaginary parts and add the result to the targets,
//       then arrive on acce[slot] (count 128) so the slot can be reused.
// Where tensor memory holds two accumulator slots (2 R NC TMEM columns each,
// 4 R NC <= 512) they let the epilogue of tile j
// overlap the MMAs of tile j + 1.  Every wait is bounded and also gives up
// once another role has recorded an error; the CTA then waits (bounded) for
// its copies and MMAs in flight, frees its tensor memory and returns.
constexpr int EPC = 16;          // epilogue chunk: accumulator columns read from tensor memory per pass
constexpr int WS_THREADS = 288;  // 9 warps
constexpr int NPROD = 128;       // producer threads (warps 5-8)

template <int NC, int R, int ST>
__global__ void __launch_bounds__(WS_THREADS, 1) k_btr_tc(const tc_tile *tiles, int ntiles, const int2 *pairs,
                                                        const uint8_t *opsA, int64_t op_bytes, int nkc, int nrt,
                                                        int Tout, int Tin, const __nv_bfloat16 *qb, c32f *dst, int mr,
                                                        int64_t svstride, int64_t dstride, int *err)
{
    extern __shared__ __align__(128) uint8_t smem_raw[];
    // 128-byte aligned base inside the dynamic allocation (launched with 128 extra)
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
    constexpr int BB = NC * KC * 2;                // bytes of one B panel (Br or Bi, hi or lo)
    constexpr int AR = R * 2 * ABYTES;             // A hi, A lo of each of the R row tiles
    constexpr int STAGE = AR + 4 * BB;             // then Br hi, Bi hi, Br lo, Bi lo
    constexpr int SLOT = R * 2 * NC;               // TMEM columns of one accumulator slot
    constexpr int NSLOT = 2 * SLOT <= 512 ? 2 : 1; // one slot for the widest tiles (no epilogue overlap)
    constexpr int TALLOC = NSLOT * SLOT <= 128 ? 128 : (NSLOT * SLOT <= 256 ? 256 : 512);  // power of two
    static_assert(NSLOT * SLOT <= 512, "accumulators exceed tensor memory");
    static_assert(NC <= NPROD, "one tile column per producer thread");
    __shared__ long long srcv[NC];             // producers: source vector per column of the current tile
    __shared__ int stage_nr[ST];               // row tiles present in the tile of each stage
    __shared__ long long tgt[NC];              // epilogue: target offset per column of the current tile
    __shared__ uint32_t tmem_base;
    __shared__ __align__(8) uint64_t full[ST], empty[ST], accf[2], acce[2];
    __shared__ int abort_flag, n_issued, n_consumed, n_commit;
    volatile int *abort_v = &abort_flag;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int my_tiles = (int)blockIdx.x < ntiles ? (ntiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    const int Tp = nkc * KC;                   // split vector length of the source level

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "r"(TALLOC));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        for (int b = 0; b < ST; ++b) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&full[b])), "r"(NPROD + 1));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&empty[b])));
        }
        for (int b = 0; b < 2; ++b) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&accf[b])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&acce[b])), "r"(128));
        }
        asm volatile("fence.mbarrier_init.release.cluster;");
        abort_flag = 0;
        n_issued = n_consumed = n_commit = 0;
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = tmem_base;

    if (warp >= 5) {
        // ---------------- producers
        // Tile descriptors are fetched two tiles ahead and the column's pair
        // one tile ahead, so the global-memory latency of both is hidden
        // behind the previous tile's stages (NC <= NPROD: one column per
        // thread).
        const int tp = tid - 160;
        auto tile_at = [&](int j) {
            return j < my_tiles ? tiles[blockIdx.x + (int64_t)j * gridDim.x] : tc_tile{0, 0, 0, 0};
        };
        auto col_src = [&](const tc_tile &t, int2 q) -> long long {
            if (tp >= t.npair) return -1;
            const int vi = t.pair0 + tp;
            const int m = vi - (vi / mr) * mr;
            return q.x / Tin + m * svstride;
        };
        auto pair_of = [&](const tc_tile &t) {
            if (tp >= t.npair) return make_int2(0, 0);
            return pairs[(t.pair0 + tp) / mr];
        };
        tc_tile t_next = tile_at(1), t_cur = tile_at(0);
        long long v_cur = col_src(t_cur, pair_of(t_cur));
        int g = 0;
        bool ok = true;
        for (int j = 0; j < my_tiles && ok; ++j) {
            const tc_tile t = t_cur;
            const tc_tile t_after = tile_at(j + 2);     // used two tiles from now
            const int2 q_next = pair_of(t_next);        // used at the next tile
            asm volatile("bar.sync 1, %0;" ::"r"(NPROD));  // everyone is done with the previous srcv
            if (tp < NC) srcv[tp] = v_cur;
            asm volatile("bar.sync 1, %0;" ::"r"(NPROD));
            const int nr = min(R, nrt - t.rt);  // row tiles of this tile
            const uint8_t *gA = opsA + (int64_t)t.op * op_bytes + (int64_t)t.rt * nkc * 2 * ABYTES;
            for (int s = 0; s < nkc; ++s, ++g) {
                const int b = g % ST;
                const bool fail = g >= ST && !mbar_wait_ab(smem_u32(&empty[b]), ((g - ST) / ST) & 1, abort_v);
                if (bar_any(1, NPROD, fail)) {
                    if (fail && !*abort_v) atomicExch(err, 2);
                    *abort_v = 1;
                    ok = false;
                    break;
                }
                uint8_t *st = smem + b * STAGE;
                const uint32_t fb = smem_u32(&full[b]);
                if (tp == 0) {
                    stage_nr[b] = nr;
                    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(fb),
                                 "r"(nr * 2 * ABYTES));
                    for (int r = 0; r < nr; ++r)
                        asm volatile(
                            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                                smem_u32(st + r * 2 * ABYTES)),
                            "l"(gA + ((int64_t)r * nkc + s) * 2 * ABYTES), "r"(2 * ABYTES), "r"(fb)
                            : "memory");
                    n_issued = g + 1;
                }
                // 16 copies of 16 bytes per column: panel part = c16 / 4 (Re hi, Im hi,
                // Re lo, Im lo), K group gq = c16 % 4; one column's stage is 256
                // contiguous bytes, so a warp instruction reads two whole columns
                for (int e = tp; e < NC * 16; e += NPROD) {
                    const int n = e >> 4, c16 = e & 15, part = c16 >> 2, gq = c16 & 3;
                    const long long v = srcv[n];
                    const __nv_bfloat16 *srcp = qb;
                    uint32_t bytes = 0;
                    if (v >= 0) {
                        srcp = qb + v * 4 * Tp + s * 4 * KC + c16 * 8;
                        bytes = 16;
                    }
                    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(
                                     smem_u32(st + AR + part * BB + core_off(n, gq * 8))),
                                 "l"(srcp), "r"(bytes)
                                 : "memory");
                }
                asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(fb));
            }
            v_cur = col_src(t_next, q_next);
            t_cur = t_next;
            t_next = t_after;
        }
        asm volatile("cp.async.wait_all;" ::: "memory");
    } else if (warp == 4) {
        // ---------------- MMA issue (one thread)
        if (lane == 0) {
            // bf16 x bf16 -> f32, K-major A and B, M = 128, N = 2 NC
            const uint32_t idesc =
                (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)((2 * NC) >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
            int g = 0;
            bool ok = true;
            for (int j = 0; j < my_tiles && ok; ++j) {
                const int slot = j % NSLOT;
                if (j >= NSLOT && !mbar_wait_ab(smem_u32(&acce[slot]), ((j - NSLOT) / NSLOT) & 1, abort_v)) {
                    if (!*abort_v) atomicExch(err, 3);
                    *abort_v = 1;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;");
                const uint32_t dslot = tmem + slot * SLOT;
                for (int s = 0; s < nkc; ++s, ++g) {
                    const int b = g % ST;
                    if (!mbar_wait_ab(smem_u32(&full[b]), (g / ST) & 1, abort_v)) {
                        if (!*abort_v) atomicExch(err, 1);
                        *abort_v = 1;
                        ok = false;
                        break;
                    }
                    asm volatile("fence.proxy.async.shared::cta;");
                    asm volatile("tcgen05.fence::after_thread_sync;");
                    const int nr = stage_nr[b];
                    const uint32_t base = smem_u32(smem + b * STAGE);
                    const uint32_t bHi = base + AR, bLo = bHi + 2 * BB;
                    for (int r = 0; r < nr; ++r) {
                        const uint32_t aHi = base + r * 2 * ABYTES, aLo = aHi + ABYTES, d = dslot + r * 2 * NC;
                        for (int k = 0; k < KC / 16; ++k) {
                            const uint32_t so = k * 256;  // two core matrices along K per k-step
                            const uint32_t en = (s > 0 || k > 0) ? 1u : 0u;
                            asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                                         "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
                                         "l"(smem_desc(aHi + so)), "l"(smem_desc(bHi + so)), "r"(idesc), "r"(en));
                            asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                                         "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
                                         "l"(smem_desc(aHi + so)), "l"(smem_desc(bLo + so)), "r"(idesc), "r"(1u));
                            asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                                         "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
                                         "l"(smem_desc(aLo + so)), "l"(smem_desc(bHi + so)), "r"(idesc), "r"(1u));
                        }
                    }
                    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                        smem_u32(&empty[b])));
                    n_consumed = g + 1;
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
        // The panels interleave the real and imaginary rows: lane 2i holds
        // Ar_i (D1 = Ar xr, D2 = Ar xi), lane 2i + 1 holds Ai_i (D1 = Ai xr,
        // D2 = Ai xi), so the two lanes of complex row i are neighbours in one
        // warp.  Of each pair of columns the even lane finishes the first and
        // the odd lane the second after one exchange of two values
        // (Re = Ar xr - Ai xi, Im = Ar xi + Ai xr), and adds it to the target.
        const int odd = lane & 1, row = warp * 16 + (lane >> 1);
        for (int j = 0; j < my_tiles; ++j) {
            const int slot = j % NSLOT;
            const tc_tile t = tiles[blockIdx.x + (int64_t)j * gridDim.x];
            asm volatile("bar.sync 2, 128;");  // everyone is done with the previous tgt
            for (int c = tid; c < NC; c += 128) {
                long long v = -1;
                if (c < t.npair) {
                    int vi = t.pair0 + c;
                    int pi = vi / mr, m = vi - pi * mr;
                    v = pairs[pi].y + m * dstride;
                }
                tgt[c] = v;
            }
            const bool have = mbar_wait_ab(smem_u32(&accf[slot]), (j / NSLOT) & 1, abort_v);
            if (bar_any(2, 128, !have)) {
                if (!have && !*abort_v) atomicExch(err, 4);
                *abort_v = 1;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;");
            // row tile r of the slot: columns [2 r NC, 2 r NC + NC) hold D1, the next NC D2
            const int nr = min(R, nrt - t.rt);
            for (int r = 0; r < nr; ++r) {
                const uint32_t d1 = tmem + slot * SLOT + r * 2 * NC + ((uint32_t)(warp * 32) << 16), d2 = d1 + NC;
                const int rowg = (t.rt + r) * 64 + row;
                for (int c0 = 0; c0 < NC; c0 += EPC) {
                    uint32_t v1[16], v2[16];
                    tmem_ld16x2(d1 + c0, d2 + c0, v1, v2);
#pragma unroll
                    for (int jj = 0; jj < EPC; jj += 2) {
                        // the even lane needs the odd lane's column jj, the odd lane the even lane's jj + 1
                        const float s1 = __uint_as_float(odd ? v1[jj] : v1[jj + 1]);
                        const float s2 = __uint_as_float(odd ? v2[jj] : v2[jj + 1]);
                        const float p1 = __shfl_xor_sync(0xffffffffu, s1, 1);
                        const float p2 = __shfl_xor_sync(0xffffffffu, s2, 1);
                        const int n = c0 + jj + odd;
                        if (rowg < Tout && n < t.npair) {
                            const float2 v = odd ? make_float2(p1 - __uint_as_float(v2[jj + 1]),
                                                               p2 + __uint_as_float(v1[jj + 1]))
                                                 : make_float2(__uint_as_float(v1[jj]) - p2,
                                                               __uint_as_float(v2[jj]) + p1);
                            atomicAdd(reinterpret_cast<float2 *>(dst + tgt[n] + rowg), v);
                        }
                    }
                }
            }
            // this slot is read: the MMAs of tile j + NSLOT may overwrite it
            asm volatile("tcgen05.fence::before_thread_sync;");
            asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&acce[slot])));
        }
    }
    __syncthreads();
    // drain after an error: copies issued but not consumed, then the last MMA
    // commit (it covers every MMA issued before it)
    if (*abort_v && tid == 0)
        for (int s2 = n_consumed; s2 < n_issued; ++s2) mbar_wait(smem_u32(&full[s2 % ST]), (s2 / ST) & 1);
    const int nc = n_commit;
    if (*abort_v && nc > 0 && tid == 0) mbar_wait(smem_u32(&empty[(nc - 1) % ST]), ((nc - 1) / ST) & 1);
    asm volatile("tcgen05.fence::after_thread_sync;");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TALLOC));
}

// operator panels: per operator, per row tile (64 complex rows), per stage
// (32 real K): [hi 128 x 32][lo 128 x 32] bf16 in the core-matrix layout
__global__ void k_pack_tc(const c64d *ops, int nops, int Tout, int Tin, int nrt, int nkc, uint8_t *out)
{
    const int64_t per_op = (int64_t)nrt * nkc * 2 * ABYTES;
    const int64_t total_vals = (int64_t)nops * nrt * nkc * 128 * KC;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total_vals;
         e += (int64_t)gridDim.x * blockDim.x) {
        int k = (int)(e % KC);
        int64_t r1 = e / KC;
        int r = (int)(r1 % 128);
        int64_t r2 = r1 / 128;
        int kc = (int)(r2 % nkc);
        int64_t r3 = r2 / nkc;
        int rt = (int)(r3 % nrt);
        int op = (int)(r3 / nrt);
        int part = r & 1;                   // even rows Re(A), odd rows Im(A) of the same complex row
        int i = rt * 64 + (r >> 1);         // complex row
        int j = kc * KC + k;                // complex column
        double v = 0.0;
        if (i < Tout && j < Tin) {
            c64d a = ops[(int64_t)op * Tout * Tin + (int64_t)j * Tout + i];
            v = part == 0 ? a.re : a.im;
        }
        float f = (float)v;
        __nv_bfloat16 hi = __float2bfloat16_rn(f);
        __nv_bfloat16 lo = __float2bfloat16_rn(f - __bfloat162float(hi));
        uint8_t *base = out + (int64_t)op * per_op + ((int64_t)rt * nkc + kc) * 2 * ABYTES;
        int o = core_off(r, k);
        *reinterpret_cast<__nv_bfloat16 *>(base + o) = hi;
        *reinterpret_cast<__nv_bfloat16 *>(base + ABYTES + o) = lo;
    }
}

struct tc_args {
    const tc_tile *tiles;
    const int2 *pairs;
    const uint8_t *A;
    int64_t op_bytes;
    int nkc, nrt, Tout, Tin;
    const __nv_bfloat16 *qb;
    c32f *dst;
    int mr;
    int64_t svstride, dstride;
    int *err;
};

template <int NC, int R, int ST>
void launch_tc(const tc_args &a, int ntiles, cudaStream_t s)
{
    const size_t stage = (size_t)R * 2 * ABYTES + 4 * (size_t)NC * KC * 2;
    const size_t smem = 128 + ST * stage;
    static int per_sm = 0, nsm = 0;  // resident CTAs per SM for this instantiation
    if (!per_sm) {
        int dev = 0;
        FDA_CUDA(cudaGetDevice(&dev));
        FDA_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
        FDA_CUDA(cudaFuncSetAttribute(k_btr_tc<NC, R, ST>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        FDA_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_btr_tc<NC, R, ST>, WS_THREADS, smem));
        const int cols = (4 * R * NC <= 512 ? 2 : 1) * 2 * R * NC;  // accumulator slots x slot columns
        const int talloc = cols <= 128 ? 128 : (cols <= 256 ? 256 : 512);
        per_sm = std::min(per_sm, 512 / talloc);  // tensor memory per CTA
        if (per_sm < 1) fda_fail(FDA_ERR_CUDA, "tensor-core translation kernel does not fit on an SM");
    }
    const int grid = std::min(ntiles, per_sm * nsm);
    k_btr_tc<NC, R, ST><<<grid, WS_THREADS, smem, s>>>(a.tiles, ntiles, a.pairs, a.A, a.op_bytes, a.nkc, a.nrt,
                                                       a.Tout, a.Tin, a.qb, a.dst, a.mr, a.svstride, a.dstride,
                                                       a.err);
}

void pack_one(fda_handle *h, tc_ops &P, const tr_batch &B, const dbuf &ops64, int nops, int Tout, int Tin)
{
    if (B.npairs == 0 || nops == 0 || Tout == 0 || Tin == 0) return;
    P.Tout = Tout;
    P.Tin = Tin;
    P.nrt = (Tout + 63) / 64;
    P.nkc = (Tin + KC - 1) / KC;
    P.op_bytes = (int64_t)P.nrt * P.nkc * 2 * ABYTES;
    P.A.alloc((size_t)P.op_bytes * nops);
    k_pack_tc<<<2048, 256, 0, h->stream>>>(ops64.as<c64d>(), nops, Tout, Tin, P.nrt, P.nkc, P.A.as<uint8_t>());
    FDA_CHECK_LAUNCH();
}

}  // namespace

// pack the M2L, M2M and L2L operators of every level for the tensor-core
// kernel and size the split density buffers
void fda_pack_tc(fda_handle *h)
{
    const int mrmax = std::max(1, h->cfg.max_rhs);
    for (int l = h->lev_lo; l >= 0 && l < h->nlev; ++l) {
        const level_info &L = h->lev[l];
        if (L.T == 0) continue;
        // every operator in full form (the batch of all pairs where the level
        // has low-rank buckets)
        pack_one(h, h->tc_m2l[l], h->lr[l].empty() ? h->b_m2l[l] : h->b_m2l_all[l], h->op64.Kt[l], L.n_ops, L.T,
                 L.T);
        if (l + 1 < h->nlev && h->lev[l + 1].T > 0) {
            const int Tc = h->lev[l + 1].T;
            pack_one(h, h->tc_m2m[l], h->b_m2m[l], h->op64.Mt[l], 8 * L.ncones, L.T, Tc);
            pack_one(h, h->tc_l2l[l], h->b_l2l[l], h->op64.Lt[l], 8 * L.ncones, Tc, L.T);
        }
        // low-rank M2L buckets (Sec. 4.2): V^ (rpad x T) and U^ (T x rpad) panels
        for (lr_bucket &B : h->lr[l]) {
            pack_one(h, B.tc1, B.b1, B.V64, (int)B.ops.size(), B.rpad, L.T);
            pack_one(h, B.tc2, B.b2, B.U64, (int)B.ops.size(), L.T, B.rpad);
        }
        const size_t nvec = (size_t)L.nbox * L.ncones * mrmax;
        const size_t Tp = (size_t)((L.T + KC - 1) / KC) * KC;
        h->qs[l].alloc(sizeof(__nv_bfloat16) * nvec * 4 * Tp);
        h->ps[l].alloc(sizeof(__nv_bfloat16) * nvec * 4 * Tp);
        FDA_CUDA(cudaMemsetAsync(h->qs[l].p, 0, h->qs[l].bytes, h->stream));
        FDA_CUDA(cudaMemsetAsync(h->ps[l].p, 0, h->ps[l].bytes, h->stream));
    }
    h->tc_err.alloc(sizeof(int));
    FDA_CUDA(cudaMemsetAsync(h->tc_err.p, 0, sizeof(int), h->stream));
    FDA_CUDA(cudaStreamSynchronize(h->stream));
    h->have_tc = 1;
}

void fda_split_tc(fda_handle *h, int l, const c32f *src, dbuf &out, int mr)
{
    const level_info &L = h->lev[l];
    if (L.T == 0 || !out.p) return;
    const int Tp = (L.T + KC - 1) / KC * KC;
    const int64_t nvec = (int64_t)L.nbox * L.ncones * mr;
    if (out.bytes < sizeof(__nv_bfloat16) * (size_t)nvec * 4 * Tp) fda_fail(FDA_ERR_STATE, "split buffer too small");
    k_split_density<<<1024, 256, 0, h->stream>>>(src, nvec, L.T, Tp, out.as<__nv_bfloat16>());
    FDA_CHECK_LAUNCH();
}

void fda_split_vectors(fda_handle *h, const c32f *src, int64_t nvec, int T, dbuf &out)
{
    const int Tp = (T + KC - 1) / KC * KC;
    const size_t need = sizeof(__nv_bfloat16) * (size_t)nvec * 4 * Tp;
    if (out.bytes < need) fda_fail(FDA_ERR_STATE, "split buffer too small");
    k_split_density<<<1024, 256, 0, h->stream>>>(src, nvec, T, Tp, out.as<__nv_bfloat16>());
    FDA_CHECK_LAUNCH();
}

void fda_run_tc(fda_handle *h, tr_batch &B, tc_ops &P, const dbuf &src, int64_t svstride, c32f *dst, int mr,
                int64_t dstride, int nc, int rows, int st)
{
    if (B.npairs == 0) return;
    if (!P.A.p) fda_fail(FDA_ERR_STATE, "tensor-core operators missing for a nonempty translation batch");
    const int nops = (int)B.op_start.size() - 1;
    const double avg_cols = (double)B.npairs * mr / std::max(1, nops);
    // tile shape (columns, row tiles, ring stages): the caller's, else the
    // tuned one (at one or at max_rhs right-hand sides), else narrow tiles
    // where an operator has few columns, one row tile, four stages
    int NC = avg_cols < 48.0 ? 32 : (avg_cols < 256.0 ? 64 : 128), R = 1, ST = NC == 128 ? 3 : 4;
    if (mr == 1 && B.nc_tuned) {
        NC = B.nc_tuned;
        R = B.r_tuned;
        ST = B.st_tuned;
    } else if (mr > 1 && B.nc_tm) {
        NC = B.nc_tm;
        R = B.r_tm;
        ST = B.st_tm;
    }
    if (!nc && !rows && !st && h->tc_force[0]) {
        nc = h->tc_force[0];
        rows = h->tc_force[1];
        st = h->tc_force[2];
    }
    if (nc) NC = nc;
    if (rows) R = rows;
    if (st) ST = st;
    // the instantiated shapes (columns, row tiles, stages):
    // (32,1,2) (32,1,4) (64,1,2) (64,1,4) (128,1,3) (128,1,4) (32,2,4) (64,2,3) (64,2,4) (128,2,2)
    // (128,2,3) (32,3,3) (32,3,4) (64,3,3) (64,4,2)
    if (R > P.nrt) R = 1;
    if (R == 3) {
        if (NC == 64) ST = 3;
        else NC = 32, ST = ST == 4 ? 4 : 3;
    }
    if (R == 4) NC = 64, ST = 2;
    if (R == 2) ST = NC == 32 ? 4 : (NC == 64 ? (ST == 4 ? 4 : 3) : (ST == 3 ? 3 : 2));
    if (R == 1) ST = NC == 128 ? (ST == 4 ? 4 : 3) : (ST == 2 ? 2 : 4);
    const tile_set *ts = nullptr;
    for (const auto &t : B.tc_tilesets)
        if (t.mr == mr && t.nc == NC && t.rows == R) ts = &t;
    if (!ts) {
        std::vector<tc_tile> tiles;
        for (int o = 0; o < nops; ++o) {
            int a = B.op_start[o] * mr, b = B.op_start[o + 1] * mr;
            if (a == b) continue;
            for (int p0 = a; p0 < b; p0 += NC)
                for (int rt = 0; rt < P.nrt; rt += R) tiles.push_back(tc_tile{o, p0, std::min(NC, b - p0), rt});
        }
        B.tc_tilesets.emplace_back();
        tile_set &t = B.tc_tilesets.back();
        t.mr = mr;
        t.nc = NC;
        t.rows = R;
        t.n = (int)tiles.size();
        t.buf.alloc(sizeof(tc_tile) * std::max<size_t>(tiles.size(), 1));
        if (!tiles.empty())
            FDA_CUDA(cudaMemcpy(t.buf.p, tiles.data(), sizeof(tc_tile) * tiles.size(), cudaMemcpyHostToDevice));
        ts = &t;
    }
    if (ts->n == 0) return;
    tc_args a{ts->buf.as<tc_tile>(), B.pairs.as<int2>(), P.A.as<uint8_t>(), P.op_bytes, P.nkc, P.nrt, P.Tout, P.Tin,
              src.as<__nv_bfloat16>(), dst, mr, svstride, dstride, h->tc_err.as<int>()};
    if (R == 4) {
        launch_tc<64, 4, 2>(a, ts->n, h->stream);
    } else if (R == 3) {
        if (NC == 64) launch_tc<64, 3, 3>(a, ts->n, h->stream);
        else if (ST == 4) launch_tc<32, 3, 4>(a, ts->n, h->stream);
        else launch_tc<32, 3, 3>(a, ts->n, h->stream);
    } else if (R == 2) {
        if (NC == 32) launch_tc<32, 2, 4>(a, ts->n, h->stream);
        else if (NC == 64 && ST == 4) launch_tc<64, 2, 4>(a, ts->n, h->stream);
        else if (NC == 64) launch_tc<64, 2, 3>(a, ts->n, h->stream);
        else if (ST == 3) launch_tc<128, 2, 3>(a, ts->n, h->stream);
        else launch_tc<128, 2, 2>(a, ts->n, h->stream);
    } else if (NC == 128) {
        if (ST == 4) launch_tc<128, 1, 4>(a, ts->n, h->stream);
        else launch_tc<128, 1, 3>(a, ts->n, h->stream);
    } else if (NC == 32) {
        if (ST == 2) launch_tc<32, 1, 2>(a, ts->n, h->stream);
        else launch_tc<32, 1, 4>(a, ts->n, h->stream);
    } else {
        if (ST == 2) launch_tc<64, 1, 2>(a, ts->n, h->stream);
        else launch_tc<64, 1, 4>(a, ts->n, h->stream);
    }
    FDA_CHECK_LAUNCH();
}

// error flag of the tensor-core kernel (bounded waits that gave up)
int fda_tc_error(fda_handle *h)
{
    if (!h->tc_err.p) return 0;
    int e = 0;
    FDA_CUDA(cudaMemcpyAsync(&e, h->tc_err.p, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    FDA_CUDA(cudaStreamSynchronize(h->stream));
    return e;
}
