// Tensor-core (tcgen05) form of the batched translations for the chosen
// precision: the M2L tiles of translate.cu as bf16 tensor-core GEMMs.
//
// A complex tile C (64 rows x NC columns) += A (64 x Tin) B (Tin x NC) is
// computed from two real GEMMs with the stacked operator [Ar; Ai] (128 rows,
// M = 128 per tcgen05.mma, each operator element stored once):
//     D1 = [Ar; Ai] Br,  D2 = [Ar; Ai] Bi,
//     Cr = D1_top - D2_bottom,  Ci = D2_top + D1_bottom,
// with D1 and D2 in two tensor-memory accumulators.  Each FP32 value is split
// into two bf16 numbers, x = x_hi + x_lo, and every product is taken as
// A_hi B_hi + A_hi B_lo + A_lo B_hi with FP32 accumulation in tensor memory,
// which keeps about 16 significant bits per operand.
//
// Operands in shared memory use the tcgen05 K-major layout without swizzle:
// 8-row x 16-byte core matrices, LBO = 128 B between core matrices along K,
// SBO = 512 B between 8-row groups (32 complex columns of K per stage).  The operator
// panels are stored in HBM already in that layout (built once in setup) and
// copied to shared memory with cp.async.bulk on an mbarrier; the densities,
// split into bf16 once per level, are gathered column by column with 16-byte
// cp.async copies that arrive on the same mbarrier.  Every mbarrier wait
// is bounded: on timeout the kernel records an error, waits (bounded) for its
// own copies and MMAs, frees its tensor memory and returns.
#include <cuda_bf16.h>

#include <algorithm>
#include <vector>

#include "fda_internal.cuh"

namespace {

constexpr int KC = 32;            // real K per stage (two MMA k-steps of 16)
constexpr int ABYTES = 128 * KC * 2;  // one bf16 operand panel stage (hi or lo): 8 KB
constexpr int TCT = 128;          // threads (4 warps = the 128 TMEM lanes)
constexpr long long SPIN = 20000000;  // bounded mbarrier polls

struct tc_tile {
    int op, pair0, npair, rt;     // operator, first column, columns, row tile (64 complex rows)
};

__device__ inline uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ inline uint64_t smem_desc(uint32_t saddr)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFF);
    d |= (uint64_t)((128u >> 4) & 0x3FFF) << 16;   // LBO: next core matrix along K
    d |= (uint64_t)((512u >> 4) & 0x3FFF) << 32;   // SBO: next 8-row group
    d |= (uint64_t)1 << 46;                        // descriptor version
    return d;
}

__device__ inline bool mbar_wait(uint32_t bar, uint32_t parity)
{
    uint32_t done = 0;
    for (long long it = 0; it < SPIN && !done; ++it)
        asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}"
                     : "=r"(done)
                     : "r"(bar), "r"(parity));
    return done != 0;
}

// byte offset of element (row, k) inside a [rows x 32] K-major bf16 stage
__device__ inline int core_off(int row, int k) { return (row >> 3) * 512 + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2; }

// Densities of one level split once per apply into bf16 hi/lo: vector v
// (box, cone, right-hand side) -> [hi: Re(0..Tp) Im(0..Tp)][lo: same],
// 4 Tp bf16 per vector, Tp = T rounded up to 32, zero beyond T.
__global__ void k_split_density(const c32f *q, int64_t nvec, int T, int Tp, __nv_bfloat16 *out)
{
    const int64_t total = nvec * 2 * Tp;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        int64_t v = e / (2 * Tp);
        int r = (int)(e % (2 * Tp));
        int j = r < Tp ? r : r - Tp;
        float x = 0.0f;
        if (j < T) {
            c32f c = q[v * T + j];
            x = r < Tp ? c.re : c.im;
        }
        __nv_bfloat16 hi = __float2bfloat16_rn(x);
        __nv_bfloat16 lo = __float2bfloat16_rn(x - __bfloat162float(hi));
        out[v * 4 * Tp + r] = hi;
        out[v * 4 * Tp + 2 * Tp + r] = lo;
    }
}

// NC = columns per tile (pairs x right-hand sides): 32, 64 or 128.  ST stage
// buffers: while the MMAs of stage s run, stages s+1 .. s+ST-1 are in flight.
// Each stage's full barrier completes when the operator panel's bulk copy has
// landed and every thread's cp.async copies of the density panels are done
// (arrival count = threads + 1); its empty barrier completes when the MMAs
// that read it are done (tcgen05.commit).
template <int NC, int ST>
__global__ void __launch_bounds__(TCT) k_btr_tc(const tc_tile *tiles, const int2 *pairs, const uint8_t *opsA,
                                                 int64_t op_bytes, int nkc, int Tout, int Tin,
                                                 const __nv_bfloat16 *qb, c32f *dst, int mr, int64_t svstride,
                                                 int64_t dstride, int *err)
{
    extern __shared__ __align__(128) uint8_t smem_raw[];
    // 128-byte aligned base inside the dynamic allocation (launched with 128 extra)
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
    constexpr int BB = NC * KC * 2;            // bytes of one B panel (Br or Bi, hi or lo)
    constexpr int STAGE = 2 * ABYTES + 4 * BB; // A hi, A lo, Br hi, Br lo, Bi hi, Bi lo
    float2 *sD = reinterpret_cast<float2 *>(smem);  // epilogue staging, 64 x NC (reuses the stages)
    __shared__ longlong2 pp[NC];               // (source vector, target offset)
    __shared__ uint32_t tmem_base;
    __shared__ __align__(8) uint64_t full[ST], empty[ST];
    __shared__ int abort_flag, ncommit;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const tc_tile t = tiles[blockIdx.x];

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "r"(2 * NC));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        for (int b = 0; b < ST; ++b) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&full[b])), "r"(TCT + 1));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&empty[b])));
        }
        asm volatile("fence.mbarrier_init.release.cluster;");
        abort_flag = 0;
        ncommit = 0;
    }
    for (int c = tid; c < NC; c += TCT) {
        longlong2 v = make_longlong2(-1, -1);
        if (c < t.npair) {
            int vi = t.pair0 + c;
            int pi = vi / mr, m = vi - pi * mr;
            int2 q = pairs[pi];
            v = make_longlong2(q.x / Tin + m * svstride, q.y + m * dstride);
        }
        pp[c] = v;
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = tmem_base;                    // D1 columns [0, NC)
    const uint32_t tmem2 = tmem_base + NC;              // D2 columns [NC, 2 NC)
    const int Tp = nkc * KC;  // split vector length of the source level
    const uint8_t *gA = opsA + (int64_t)t.op * op_bytes + (int64_t)t.rt * nkc * 2 * ABYTES;
    const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(NC >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);

    // stage s into buffer b, fully asynchronous: operator panel by bulk copy,
    // density panels by 16-byte cp.async (zero fill for empty columns)
    auto produce = [&](int s, int b) {
        uint8_t *st = smem + b * STAGE;
        const uint32_t fb = smem_u32(&full[b]);
        if (tid == 0) {
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(fb), "r"(2 * ABYTES));
            asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                             smem_u32(st)),
                         "l"(gA + (int64_t)s * 2 * ABYTES), "r"(2 * ABYTES), "r"(fb));
        }
        // 16 copies per column: {Br, Bi} x {hi, lo} x 4 groups of 8 columns of K
        for (int e = tid; e < NC * 16; e += TCT) {
            int n = e >> 4, g = (e >> 2) & 3, part = e & 3;  // part: 0 Br hi, 1 Br lo, 2 Bi hi, 3 Bi lo
            long long v = pp[n].x;
            const __nv_bfloat16 *srcp = qb;
            uint32_t bytes = 0;
            if (v >= 0) {
                srcp = qb + v * 4 * Tp + (part & 1) * 2 * Tp + (part >> 1) * Tp + s * KC + g * 8;
                bytes = 16;
            }
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(
                             smem_u32(st + 2 * ABYTES + part * BB + core_off(n, g * 8))),
                         "l"(srcp), "r"(bytes));
        }
        asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(fb));
    };

    bool ok = true;
    int nprod = 0;  // stages whose copies have been issued
    for (; nprod < ST - 1 && nprod < nkc; ++nprod) produce(nprod, nprod);
    int s = 0;
    for (; s < nkc; ++s) {
        const int b = s % ST, u = s / ST;
        if (tid == 0) {
            if (!mbar_wait(smem_u32(&full[b]), u & 1)) {
                atomicExch(err, 1);
                abort_flag = 1;
            } else {
                asm volatile("fence.proxy.async.shared::cta;");
                asm volatile("tcgen05.fence::after_thread_sync;");
                const uint32_t aHi = smem_u32(smem + b * STAGE), aLo = aHi + ABYTES;
                const uint32_t rHi = aHi + 2 * ABYTES, rLo = rHi + BB, iHi = rLo + BB, iLo = iHi + BB;
                for (int k = 0; k < KC / 16; ++k) {
                    const uint32_t so = k * 256;  // two core matrices along K per k-step
                    const uint64_t da[3] = {smem_desc(aHi + so), smem_desc(aHi + so), smem_desc(aLo + so)};
                    const uint64_t dr[3] = {smem_desc(rHi + so), smem_desc(rLo + so), smem_desc(rHi + so)};
                    const uint64_t di[3] = {smem_desc(iHi + so), smem_desc(iLo + so), smem_desc(iHi + so)};
                    for (int q = 0; q < 3; ++q) {
                        uint32_t en = (s > 0 || k > 0 || q > 0) ? 1u : 0u;
                        asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                                     "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
                                     "l"(da[q]), "l"(dr[q]), "r"(idesc), "r"(en));
                        asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                                     "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem2),
                                     "l"(da[q]), "l"(di[q]), "r"(idesc), "r"(en));
                    }
                }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                    smem_u32(&empty[b])));
                ncommit = s + 1;
            }
        }
        // the next stage to load reuses the buffer of stage s - 1
        if (nprod < nkc && s >= 1 && !mbar_wait(smem_u32(&empty[nprod % ST]), ((s - 1) / ST) & 1)) {
            if (tid == 0) atomicExch(err, 2);
            abort_flag = 1;
        }
        __syncthreads();
        if (abort_flag) {
            ok = false;
            break;
        }
        if (nprod < nkc) {
            produce(nprod, nprod % ST);
            ++nprod;
        }
    }
    // drain: this thread's density copies; on abort, the operator copies of
    // stages issued but not consumed; then the last commit (it covers every
    // MMA issued before it)
    asm volatile("cp.async.wait_all;");
    if (!ok && tid == 0)
        for (int s2 = s; s2 < nprod; ++s2) mbar_wait(smem_u32(&full[s2 % ST]), (s2 / ST) & 1);
    __syncthreads();
    const int nc = ncommit;
    if (nc > 0 && !mbar_wait(smem_u32(&empty[(nc - 1) % ST]), ((nc - 1) / ST) & 1)) {
        if (tid == 0) atomicExch(err, 2);
        abort_flag = 1;
    }
    asm volatile("tcgen05.fence::after_thread_sync;");
    __syncthreads();
    ok = ok && !abort_flag;
    // epilogue: lane r < 64 holds Ar rows (D1 -> Re, D2 -> Im); lane r >= 64
    // holds Ai rows (D1 -> Im, D2 -> -Re).  Warps 0-1 write, then warps 2-3 add.
    const int r = warp * 32 + lane;
    for (int pass = 0; pass < 2 && ok; ++pass) {
        if ((warp >> 1) == pass) {
            float2 *row = sD + (r & 63) * NC;
            for (int c0 = 0; c0 < NC; c0 += 16) {
                uint32_t v1[16], v2[16];
                uint32_t a1 = tmem + ((uint32_t)(warp * 32) << 16) + c0;
                uint32_t a2 = tmem2 + ((uint32_t)(warp * 32) << 16) + c0;
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                    : "=r"(v1[0]), "=r"(v1[1]), "=r"(v1[2]), "=r"(v1[3]), "=r"(v1[4]), "=r"(v1[5]), "=r"(v1[6]),
                      "=r"(v1[7]), "=r"(v1[8]), "=r"(v1[9]), "=r"(v1[10]), "=r"(v1[11]), "=r"(v1[12]), "=r"(v1[13]),
                      "=r"(v1[14]), "=r"(v1[15])
                    : "r"(a1));
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                    : "=r"(v2[0]), "=r"(v2[1]), "=r"(v2[2]), "=r"(v2[3]), "=r"(v2[4]), "=r"(v2[5]), "=r"(v2[6]),
                      "=r"(v2[7]), "=r"(v2[8]), "=r"(v2[9]), "=r"(v2[10]), "=r"(v2[11]), "=r"(v2[12]), "=r"(v2[13]),
                      "=r"(v2[14]), "=r"(v2[15])
                    : "r"(a2));
                asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    float d1 = __uint_as_float(v1[j]), d2 = __uint_as_float(v2[j]);
                    if (pass == 0) {
                        row[c0 + j] = make_float2(d1, d2);
                    } else {
                        float2 o = row[c0 + j];
                        row[c0 + j] = make_float2(o.x - d2, o.y + d1);
                    }
                }
            }
        }
        __syncthreads();
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (ok) {
        const int row0 = t.rt * 64;
        for (int e = tid; e < 64 * NC; e += TCT) {
            int rr = e & 63, n = e >> 6;
            int rowg = row0 + rr;
            if (n < t.npair && rowg < Tout) {
                float2 v = sD[rr * NC + n];
                atomicAdd(reinterpret_cast<float2 *>(dst + pp[n].y + rowg), v);
            }
        }
    }
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * NC));
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
        int part = r >> 6;                  // rows 0-63: Re(A), rows 64-127: Im(A)
        int i = rt * 64 + (r & 63);         // complex row
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
    int nkc, Tout, Tin;
    const __nv_bfloat16 *qb;
    c32f *dst;
    int mr;
    int64_t svstride, dstride;
    int *err;
};

template <int NC, int ST>
void launch_tc(const tc_args &a, int ntiles, cudaStream_t s)
{
    const size_t stage = 2 * (size_t)ABYTES + 4 * (size_t)NC * KC * 2;
    const size_t smem = 128 + std::max<size_t>(ST * stage, (size_t)64 * NC * sizeof(float2));
    FDA_CUDA(cudaFuncSetAttribute(k_btr_tc<NC, ST>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_btr_tc<NC, ST><<<ntiles, TCT, smem, s>>>(a.tiles, a.pairs, a.A, a.op_bytes, a.nkc, a.Tout, a.Tin, a.qb, a.dst,
                                               a.mr, a.svstride, a.dstride, a.err);
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
        pack_one(h, h->tc_m2l[l], h->b_m2l[l], h->op64.Kt[l], L.n_ops, L.T, L.T);
        if (l + 1 < h->nlev && h->lev[l + 1].T > 0) {
            const int Tc = h->lev[l + 1].T;
            pack_one(h, h->tc_m2m[l], h->b_m2m[l], h->op64.Mt[l], 8 * L.ncones, L.T, Tc);
            pack_one(h, h->tc_l2l[l], h->b_l2l[l], h->op64.Lt[l], 8 * L.ncones, Tc, L.T);
        }
        const size_t nvec = (size_t)L.nbox * L.ncones * mrmax;
        const size_t Tp = (size_t)((L.T + KC - 1) / KC) * KC;
        h->qs[l].alloc(sizeof(__nv_bfloat16) * nvec * 4 * Tp);
        h->ps[l].alloc(sizeof(__nv_bfloat16) * nvec * 4 * Tp);
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

void fda_run_tc(fda_handle *h, tr_batch &B, tc_ops &P, const dbuf &src, int64_t svstride, c32f *dst, int mr,
                int64_t dstride)
{
    if (B.npairs == 0) return;
    if (!P.A.p) fda_fail(FDA_ERR_STATE, "tensor-core operators missing for a nonempty translation batch");
    const int nops = (int)B.op_start.size() - 1;
    const double avg_cols = (double)B.npairs * mr / std::max(1, nops);
    // narrow tiles where an operator has few pairs (less padding, more CTAs per SM)
    const int NC = avg_cols < 48.0 ? 32 : 64;
    if (P.tiles_nc != NC || P.tiles_mr != mr) {
        std::vector<tc_tile> tiles;
        for (int o = 0; o < nops; ++o) {
            int a = B.op_start[o] * mr, b = B.op_start[o + 1] * mr;
            for (int p0 = a; p0 < b; p0 += NC)
                for (int rt = 0; rt < P.nrt; ++rt) tiles.push_back(tc_tile{o, p0, std::min(NC, b - p0), rt});
        }
        P.ntiles = (int)tiles.size();
        P.tiles.alloc(sizeof(tc_tile) * std::max<size_t>(tiles.size(), 1));
        if (!tiles.empty())
            FDA_CUDA(cudaMemcpy(P.tiles.p, tiles.data(), sizeof(tc_tile) * tiles.size(), cudaMemcpyHostToDevice));
        P.tiles_mr = mr;
        P.tiles_nc = NC;
    }
    if (P.ntiles == 0) return;
    tc_args a{P.tiles.as<tc_tile>(), B.pairs.as<int2>(), P.A.as<uint8_t>(), P.op_bytes, P.nkc, P.Tout, P.Tin,
              src.as<__nv_bfloat16>(), dst, mr, svstride, dstride, h->tc_err.as<int>()};
    if (NC == 32) launch_tc<32, 2>(a, P.ntiles, h->stream);
    else launch_tc<64, 2>(a, P.ntiles, h->stream);
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
