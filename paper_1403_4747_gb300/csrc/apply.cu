// One FDA matrix-vector product (Sec. 3.3 Steps 2-4) on the device:
//   near field (S2T, Step 4) -> y
//   upward pass (Step 2): S2M at leaves, M2M bottom-up (per cone at
//       high-frequency levels; a high-frequency parent takes each child's
//       cone that contains its own cone, or the child's non-directional
//       densities if the child is low-frequency)
//   downward pass (Step 3): M2L at every level, then L2L top-down (a
//       low-frequency child sums all of its high-frequency parent's cones)
//   L2T at leaves -> y += ...
// Densities are kept in the compressed coordinates of Sec. 4 (q~ of rank T
// per box and cone; p~ = U_dn^H p).  Every pass is templated on the real
// type: double (plain FP64 form) or float (chosen form: FP32 operators and
// densities, FP32 accumulation, the result added into the FP64 output).
#include <cuda_bf16.h>
#include <stdio.h>

#include <algorithm>
#include <array>
#include <map>
#include <string>

#include "fda_internal.cuh"

namespace {

constexpr int AT = 256;    // threads per CTA
constexpr int MAXR = 4;    // rows per thread (rank <= 1024)
constexpr int MAXT = AT * MAXR;

template <typename R>
struct lvl_ptrs {
    int box0[FDA_MAX_LEVELS], nbox[FDA_MAX_LEVELS], T[FDA_MAX_LEVELS], ncones[FDA_MAX_LEVELS];
    int nc[FDA_MAX_LEVELS], hf[FDA_MAX_LEVELS];
    int64_t stride[FDA_MAX_LEVELS];  // per right-hand side: nbox * ncones * T
    cx<R> *q[FDA_MAX_LEVELS];
    cx<R> *p[FDA_MAX_LEVELS];
    const cx<R> *Kt[FDA_MAX_LEVELS];
    const cx<R> *Mt[FDA_MAX_LEVELS];
    const cx<R> *Lt[FDA_MAX_LEVELS];
};

template <typename R>
__device__ inline cx<R> ldx(const void *x, int64_t i, int x64)
{
    if (x64) {
        c64d v = ((const c64d *)x)[i];
        return cx<R>((R)v.re, (R)v.im);
    }
    c32f v = ((const c32f *)x)[i];
    return cx<R>((R)v.re, (R)v.im);
}

// ---- Step 4: near field, y = A_near x (overwrites y)
// Right-hand sides are processed in groups of NR per CTA (blockIdx.z), so
// every matrix entry read from HBM serves NR products (NR = 1 for a single
// right-hand side).
constexpr int NRG = 8;

constexpr int NRW = 2;  // rows per warp in the near-field product

// one thread's L2 prefetch of entries [b, e) of an array that ends at lim
// (16-byte aligned start, size a multiple of 16, never past lim)
template <typename T>
__device__ __forceinline__ void prefetch_l2(const T *b, const T *e, const T *lim)
{
    const uintptr_t pb = reinterpret_cast<uintptr_t>(b) & ~uintptr_t(15);
    uintptr_t pe = (reinterpret_cast<uintptr_t>(e) + 15) & ~uintptr_t(15);
    const uintptr_t pl = reinterpret_cast<uintptr_t>(lim) & ~uintptr_t(15);
    if (pe > pl) pe = pl;
    if (pe > pb) asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(pb), "r"((uint32_t)(pe - pb)) : "memory");
}

// NW rows r0, r0 + AT / 32, ... of a leaf block (row-major, nc columns)
// times x, written to y
template <typename R, int NR, bool XS, int NW>
__device__ __forceinline__ void near_rows(int r0, int nB, int lane, const cx<R> *A, int nc, const int32_t *cl,
                                          const cx<R> *xsm, const void *x, int x64, int64_t xstr, int m0, int nm,
                                          c64d *y, int64_t ldy, int i0)
{
    if (r0 >= nB) return;
    const cx<R> *rowp[NW];
    bool rv[NW];
#pragma unroll
    for (int w = 0; w < NW; ++w) {
        const int r = r0 + w * (AT / 32);
        rv[w] = r < nB;
        rowp[w] = A + (int64_t)(rv[w] ? r : r0) * nc;
    }
    cx<R> acc[NW][NR];
    for (int cb = 0; cb < nc; cb += 128) {
        cx<R> a[NW][4];
        int j[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int cc = cb + 32 * u + lane;
            j[u] = 0;
            if (cc < nc) {
                j[u] = XS ? cc : __ldg(cl + cc);
#pragma unroll
                for (int w = 0; w < NW; ++w)
                    if (rv[w]) a[w][u] = rowp[w][cc];
            }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int mm = 0; mm < NR; ++mm)
                if (mm < nm) {
                    const cx<R> xv = XS ? (cb + 32 * u + lane < nc ? xsm[j[u]] : cx<R>())
                                        : ldx<R>(x, (int64_t)(m0 + mm) * xstr + j[u], x64);
#pragma unroll
                    for (int w = 0; w < NW; ++w) cfma(acc[w][mm], a[w][u], xv);
                }
    }
#pragma unroll
    for (int w = 0; w < NW; ++w) {
        if (!rv[w]) break;  // uniform across the warp
        const int r = r0 + w * (AT / 32);
#pragma unroll
        for (int mm = 0; mm < NR; ++mm) {
            if (mm >= nm) break;  // uniform across the warp
            cx<R> v = acc[w][mm];
            for (int o = 16; o > 0; o >>= 1) {
                v.re += __shfl_xor_sync(0xffffffffu, v.re, o);
                v.im += __shfl_xor_sync(0xffffffffu, v.im, o);
            }
            if (lane == 0) y[(int64_t)(m0 + mm) * ldy + i0 + r] = c64d((double)v.re, (double)v.im);
        }
    }
}

template <typename R, int NR, bool XS, int NW = NRW>
__global__ void __launch_bounds__(AT) k_near_apply(const int32_t *leaf_box, const int32_t *bbeg,
                                                   const int32_t *bend, const int64_t *colptr, const int32_t *cols,
                                                   const int64_t *off, const cx<R> *A, const void *x, int x64,
                                                   int64_t xstr, int mr, c64d *y, int64_t ldy, int64_t nnz)
{
    // Each warp takes NW rows of a leaf (rows r, r + 8, ... of its group of
    // 8 NW); the leaf's columns (its flattened near ranges, shared by all
    // its rows) are streamed four 32-wide slices at a time, the last ones
    // predicated, so every lane keeps 4 NW independent matrix loads in
    // flight and each x value serves NW rows.  With XS (one right-hand
    // side) the CTA first gathers x over the leaf's columns into shared
    // memory, so the warps read it from there instead of through the column
    // list.
    extern __shared__ unsigned char xs_raw[];
    cx<R> *xsm = reinterpret_cast<cx<R> *>(xs_raw);
    int li = blockIdx.x;
    int B = leaf_box[li];
    int i0 = bbeg[B], nB = bend[B] - i0;
    int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (blockIdx.y * (AT / 32) * NW >= nB) return;  // whole CTA
    const int m0 = blockIdx.z * NR;
    const int nm = min(NR, mr - m0);
    const int64_t c0 = colptr[li];
    const int nc = (int)(colptr[li + 1] - c0);
    const int32_t *cl = cols + c0;
    // the leaf's whole block (contiguous) into L2 while x is gathered
    if (XS && gridDim.y == 1 && threadIdx.x == 0) prefetch_l2(A + off[li], A + off[li + 1], A + nnz);
    if (XS) {
        for (int c = threadIdx.x; c < nc; c += AT) xsm[c] = ldx<R>(x, __ldg(cl + c), x64);
        __syncthreads();
    }
    // groups of (AT / 32) x NRW rows: one group per CTA row, or all of the
    // leaf's groups in one CTA when gridDim.y == 1 (x gathered once)
    for (int g0 = blockIdx.y * (AT / 32) * NW; g0 < nB; g0 += gridDim.y * (AT / 32) * NW)
        near_rows<R, NR, XS, NW>(g0 + warp, nB, lane, A + off[li], nc, cl, xsm, x, x64, xstr, m0, nm, y, ldy, i0);
}


// q~ and p~ of level lev_lo + blockIdx.y / 2 (even: q~, odd: p~) set to zero
// for mr right-hand sides
template <typename R>
__global__ void k_zero_levels(lvl_ptrs<R> P, int lev_lo, int mr)
{
    const int l = lev_lo + (int)blockIdx.y / 2;
    cx<R> *v = (blockIdx.y & 1) ? P.p[l] : P.q[l];
    const int64_t n = P.stride[l] * mr;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
        v[e] = cx<R>();
}

// ---- Step 2: S2M at leaves, q~ = S~ x_B
// One CTA per leaf.  With T < blockDim the CTA splits the sum over the
// leaf's elements into blockDim / T interleaved groups (every thread has a
// share of the loads) and adds the groups' partial sums in shared memory.
template <typename R>
__global__ void k_s2m(lvl_ptrs<R> P, const int32_t *leaf_box, const int32_t *blev, const int32_t *bbeg,
                      const int32_t *bend, const int64_t *loff, const cx<R> *St, const void *x, int x64,
                      int64_t xstr, int mr)
{
    __shared__ cx<R> xs[64];
    __shared__ cx<R> part[AT];
    int li = blockIdx.x;
    int B = leaf_box[li];
    int l = blev[B];
    int T = P.T[l];
    if (T == 0) return;
    int j0 = bbeg[B], nB = bend[B] - j0;
    const cx<R> *S = St + loff[li];
    const int G = T < (int)blockDim.x ? (int)blockDim.x / T : 1;
    for (int m = 0; m < mr; ++m) {
        __syncthreads();
        for (int j = threadIdx.x; j < nB; j += blockDim.x) xs[j] = ldx<R>(x, (int64_t)m * xstr + j0 + j, x64);
        __syncthreads();
        cx<R> *q = P.q[l] + m * P.stride[l] + (int64_t)(B - P.box0[l]) * T;
        if (G == 1) {
            for (int t = threadIdx.x; t < T; t += blockDim.x) {
                cx<R> acc;
#pragma unroll 4
                for (int j = 0; j < nB; ++j) cfma(acc, S[(int64_t)j * T + t], xs[j]);
                q[t] = acc;
            }
        } else {
            const int g = threadIdx.x / T, t = threadIdx.x - g * T;
            cx<R> acc;
            if (g < G) {
#pragma unroll 4
                for (int j = g; j < nB; j += G) cfma(acc, S[(int64_t)j * T + t], xs[j]);
            }
            part[threadIdx.x] = acc;
            __syncthreads();
            if ((int)threadIdx.x < T) {
                cx<R> sum = part[threadIdx.x];
                for (int gg = 1; gg < G; ++gg) {
                    const cx<R> v = part[gg * T + threadIdx.x];
                    sum.re += v.re;
                    sum.im += v.im;
                }
                q[threadIdx.x] = sum;
            }
        }
    }
}

// ---- Step 3: L2T at leaves, y += T~ p~
template <typename R>
__global__ void k_l2t(lvl_ptrs<R> P, const int32_t *leaf_box, const int32_t *blev, const int32_t *bbeg,
                      const int32_t *bend, const int64_t *loff, const cx<R> *Tt, c64d *y, int64_t ldy, int mr)
{
    __shared__ cx<R> pp[MAXT];
    int li = blockIdx.x;
    int B = leaf_box[li];
    int l = blev[B];
    int T = P.T[l];
    if (T == 0) return;
    int i0 = bbeg[B], nB = bend[B] - i0;
    const cx<R> *Tm = Tt + loff[li];
    for (int m = 0; m < mr; ++m) {
        const cx<R> *src = P.p[l] + m * P.stride[l] + (int64_t)(B - P.box0[l]) * T;
        __syncthreads();
        for (int j = threadIdx.x; j < T; j += blockDim.x) pp[j] = src[j];
        __syncthreads();
        for (int i = threadIdx.x; i < nB; i += blockDim.x) {
            cx<R> acc;
            for (int t = 0; t < T; ++t) cfma(acc, Tm[(int64_t)t * 64 + i], pp[t]);
            c64d *yp = y + (int64_t)m * ldy + i0 + i;
            c64d v = *yp;
            *yp = c64d(v.re + (double)acc.re, v.im + (double)acc.im);
        }
    }
}

// ---- one right-hand side: S2M and L2T with a warp per leaf (LPB leaves per
// CTA), so that many leaves are in flight per SM
constexpr int LPB = 8;

// q~_B = S~_B x_B: lane t < T (rows lane, lane + 32, ...) sums over the
// leaf's elements eight at a time; x_B (n_B <= 64) sits in two registers per
// lane and is broadcast by shuffles
template <typename R, bool ADD = false>  // ADD: q~ += S~ x (a second layer of sources)
__global__ void __launch_bounds__(32 * LPB) k_s2m_w(lvl_ptrs<R> P, int nleaf, const int32_t *leaf_box,
                                                     const int32_t *blev, const int32_t *bbeg, const int32_t *bend,
                                                     const int64_t *loff, const cx<R> *St, const void *x, int x64)
{
    const int li = blockIdx.x * LPB + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (li >= nleaf) return;
    const int B = leaf_box[li], l = blev[B], T = P.T[l];
    if (T == 0) return;
    const int j0 = bbeg[B], nB = bend[B] - j0;
    const cx<R> *S = St + loff[li];
    const cx<R> x0 = lane < nB ? ldx<R>(x, j0 + lane, x64) : cx<R>();
    const cx<R> x1 = lane + 32 < nB ? ldx<R>(x, j0 + lane + 32, x64) : cx<R>();
    cx<R> *q = P.q[l] + (int64_t)(B - P.box0[l]) * T;
    constexpr int JU = 8;  // elements per step: their operator loads are issued before the products
    for (int t0 = 0; t0 < T; t0 += 32) {  // every lane stays in the loop (the shuffles need all 32)
        const int t = t0 + lane;
        const bool on = t < T;
        cx<R> acc;
        for (int jb = 0; jb < nB; jb += JU) {
            cx<R> sv[JU];
#pragma unroll
            for (int u = 0; u < JU; ++u) sv[u] = on && jb + u < nB ? S[(int64_t)(jb + u) * T + t] : cx<R>();
#pragma unroll
            for (int u = 0; u < JU; ++u) {
                const int j = jb + u;  // past nB the operator values are 0
                const cx<R> src = j < 32 ? x0 : x1;
                const cx<R> xj(__shfl_sync(0xffffffffu, src.re, j & 31), __shfl_sync(0xffffffffu, src.im, j & 31));
                cfma(acc, sv[u], xj);
            }
        }
        if (on) q[t] = ADD ? q[t] + acc : acc;
    }
}

// y_B += T~_B p~_B: lane owns rows lane and lane + 32 of the leaf (n_B <= 64)
// and sums over the T densities, read 32 at a time into registers and
// broadcast by shuffles; the operator columns are loaded eight at a time
template <typename R>
__global__ void __launch_bounds__(32 * LPB) k_l2t_w(lvl_ptrs<R> P, int nleaf, const int32_t *leaf_box,
                                                     const int32_t *blev, const int32_t *bbeg, const int32_t *bend,
                                                     const int64_t *loff, const cx<R> *Tt, c64d *y, int compact)
{
    const int li = blockIdx.x * LPB + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (li >= nleaf) return;
    const int B = leaf_box[li], l = blev[B], T = P.T[l];
    if (T == 0) return;
    const int i0 = bbeg[B], nB = bend[B] - i0;
    const int ld = compact ? nB : 64;  // column stride of the leaf's operator
    const cx<R> *Tm = Tt + loff[li];
    if (compact && lane == 0) prefetch_l2(Tm, Tm + (int64_t)T * nB, Tt + loff[nleaf]);  // the leaf's block
    const cx<R> *src = P.p[l] + (int64_t)(B - P.box0[l]) * T;
    const bool r0 = lane < nB, r1 = lane + 32 < nB;
    cx<R> a0, a1;
    if (nB <= 32) {
        // one row per lane: sixteen operator loads in flight per step
        constexpr int UV = 16;
        for (int tb = 0; tb < T; tb += 32) {
            const cx<R> pv = tb + lane < T ? src[tb + lane] : cx<R>();
            const int nt = min(32, T - tb);
            for (int ub = 0; ub < nt; ub += UV) {
                cx<R> c0[UV];
#pragma unroll
                for (int u = 0; u < UV; ++u)
                    c0[u] = ub + u < nt && r0 ? Tm[(int64_t)(tb + ub + u) * ld + lane] : cx<R>();
#pragma unroll
                for (int u = 0; u < UV; ++u) {
                    const cx<R> pt(__shfl_sync(0xffffffffu, pv.re, (ub + u) & 31),
                                   __shfl_sync(0xffffffffu, pv.im, (ub + u) & 31));
                    cfma(a0, c0[u], pt);
                }
            }
        }
        if (r0) {
            c64d v = y[i0 + lane];
            y[i0 + lane] = c64d(v.re + (double)a0.re, v.im + (double)a0.im);
        }
        return;
    }
    constexpr int UU = 8;  // densities per step: their operator loads are issued before the products
    for (int tb = 0; tb < T; tb += 32) {
        const cx<R> pv = tb + lane < T ? src[tb + lane] : cx<R>();
        const int nt = min(32, T - tb);
        for (int ub = 0; ub < nt; ub += UU) {
            cx<R> c0[UU], c1[UU];
#pragma unroll
            for (int u = 0; u < UU; ++u) {
                const cx<R> *col = Tm + (int64_t)(tb + ub + u) * ld;
                const bool in = ub + u < nt;
                c0[u] = in && r0 ? col[lane] : cx<R>();
                c1[u] = in && r1 ? col[lane + 32] : cx<R>();
            }
#pragma unroll
            for (int u = 0; u < UU; ++u) {
                // past nt the operator values are 0 (pv of lanes past T is 0 too)
                const cx<R> pt(__shfl_sync(0xffffffffu, pv.re, (ub + u) & 31),
                               __shfl_sync(0xffffffffu, pv.im, (ub + u) & 31));
                cfma(a0, c0[u], pt);
                cfma(a1, c1[u], pt);
            }
        }
    }
    if (r0) {
        c64d v = y[i0 + lane];
        y[i0 + lane] = c64d(v.re + (double)a0.re, v.im + (double)a0.im);
    }
    if (r1) {
        c64d v = y[i0 + lane + 32];
        y[i0 + lane + 32] = c64d(v.re + (double)a1.re, v.im + (double)a1.im);
    }
}

__global__ void k_add_c64(c64d *a, const c64d *b, int64_t n)
{
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t < n) a[t] = a[t] + b[t];
}

__global__ void k_c64_to_c32(const c64d *a, c32f *b, int64_t n)
{
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t < n) b[t] = c32f((float)a[t].re, (float)a[t].im);
}

template <typename R>
lvl_ptrs<R> make_ptrs(fda_handle *h, far_ops<R> &ops, dbuf *q, dbuf *p)
{
    lvl_ptrs<R> P;
    for (int l = 0; l < FDA_MAX_LEVELS; ++l) {
        P.box0[l] = l < h->nlev ? h->lev[l].box0 : 0;
        P.nbox[l] = l < h->nlev ? h->lev[l].nbox : 0;
        P.T[l] = (l < h->nlev && h->lev[l].active) ? h->lev[l].T : 0;
        P.ncones[l] = l < h->nlev ? h->lev[l].ncones : 1;
        P.nc[l] = l < h->nlev ? h->lev[l].nc : 0;
        P.hf[l] = l < h->nlev ? h->lev[l].hf : 0;
        P.stride[l] = l < h->nlev ? (int64_t)h->lev[l].nbox * h->lev[l].ncones * h->lev[l].T : 0;
        P.q[l] = q[l].as<cx<R>>();
        P.p[l] = p[l].as<cx<R>>();
        P.Kt[l] = ops.Kt[l].template as<cx<R>>();
        P.Mt[l] = ops.Mt[l].template as<cx<R>>();
        P.Lt[l] = ops.Lt[l].template as<cx<R>>();
    }
    return P;
}

// M2L of the low-rank operators of one rank bucket at level l (Sec. 4.2):
// t_p = V^ q~_C for every pair p, then p~_D += U^ t_p.  The intermediates
// were allocated for max_rhs right-hand sides at setup (never reallocated:
// captured graphs hold their addresses).
template <typename R>
void lowrank_m2l(fda_handle *h, lr_bucket &B, int l, const lvl_ptrs<R> &P, int mr, bool tc)
{
    if (B.npairs == 0) return;
    cudaStream_t s = h->stream;
    const int T = h->lev[l].T;
    const int64_t per = B.npairs * B.rpad;  // intermediate values per right-hand side
    dbuf &t = sizeof(R) == 8 ? B.t64 : B.t32;
    const size_t need = sizeof(cx<R>) * (size_t)per * mr;
    if (t.bytes < need) fda_fail(FDA_ERR_STATE, "low-rank intermediate smaller than max_rhs columns");
    FDA_CUDA(cudaMemsetAsync(t.p, 0, need, s));
    if (tc) {
        const size_t sneed = sizeof(__nv_bfloat16) * (size_t)B.npairs * mr * 4 * ((B.rpad + 31) / 32 * 32);
        if (B.ts.bytes < sneed) fda_fail(FDA_ERR_STATE, "low-rank split buffer smaller than max_rhs columns");
        fda_run_tc(h, B.b1, B.tc1, h->qs[l], P.stride[l] / std::max(1, T), t.as<c32f>(), mr, per);
        fda_split_vectors(h, t.as<c32f>(), B.npairs * mr, B.rpad, B.ts);
        fda_run_tc(h, B.b2, B.tc2, B.ts, B.npairs, reinterpret_cast<c32f *>(P.p[l]), mr, P.stride[l]);
    } else {
        const dbuf &V = sizeof(R) == 8 ? B.V64 : B.V32;
        const dbuf &U = sizeof(R) == 8 ? B.U64 : B.U32;
        fda_run_batch<R>(B.b1, V.as<cx<R>>(), B.rpad, T, P.q[l], t.as<cx<R>>(), mr, P.stride[l], per, s);
        fda_run_batch<R>(B.b2, U.as<cx<R>>(), T, B.rpad, t.as<cx<R>>(), P.p[l], mr, per, P.stride[l], s);
    }
}

// M2M, M2L and L2L of one apply (Sec. 3.3 Steps 2-3) on the densities of P,
// the leaves' q~ already in place; mark(i) records the pass boundaries 3-5.
// With tc (FP32): every translation reads bf16 hi/lo splits of its source
// level, made once that level is complete.
template <typename R, typename Mark>
void translate_passes(fda_handle *h, const lvl_ptrs<R> &P, int mr, bool tc, Mark mark)
{
    cudaStream_t s = h->stream;
    auto c32 = [](auto *v) { return reinterpret_cast<c32f *>(v); };
    // M2M bottom-up: q~_parent += M~ q~_child
    for (int l = h->nlev - 2; l >= h->lev_lo; --l) {
        if (tc) {
            fda_split_tc(h, l + 1, c32(P.q[l + 1]), h->qs[l + 1], mr);
            fda_run_tc(h, h->b_m2m[l], h->tc_m2m[l], h->qs[l + 1], P.stride[l + 1] / std::max(1, h->lev[l + 1].T),
                       c32(P.q[l]), mr, P.stride[l]);
        } else {
            fda_run_batch<R>(h->b_m2m[l], P.Mt[l], h->lev[l].T, h->lev[l + 1].T, P.q[l + 1], P.q[l], mr,
                             P.stride[l + 1], P.stride[l], s);
        }
    }
    if (tc) fda_split_tc(h, h->lev_lo, c32(P.q[h->lev_lo]), h->qs[h->lev_lo], mr);
    mark(3);
    // M2L at every level: p~_target += K~ q~_source
    // (the CUDA-core forms always apply the low-rank operators of Sec. 4.2
    // in two stages; the tensor-core form does so where the autotuner found
    // it faster, else it applies every operator in full)
    for (int l = h->lev_lo; l < h->nlev; ++l) {
        const bool lr = !h->lr[l].empty() && (!tc || (mr == 1 ? h->lr_tc[l] : h->lr_tc_many[l]));
        if (tc) {
            tr_batch &F = lr || h->lr[l].empty() ? h->b_m2l[l] : h->b_m2l_all[l];
            fda_run_tc(h, F, h->tc_m2l[l], h->qs[l], P.stride[l] / std::max(1, h->lev[l].T), c32(P.p[l]), mr,
                       P.stride[l]);
        } else {
            fda_run_batch<R>(h->b_m2l[l], P.Kt[l], h->lev[l].T, h->lev[l].T, P.q[l], P.p[l], mr, P.stride[l],
                             P.stride[l], s);
        }
        if (lr)
            for (lr_bucket &B : h->lr[l]) lowrank_m2l<R>(h, B, l, P, mr, tc);
    }
    mark(4);
    // L2L top-down: p~_child += L~ p~_parent
    for (int l = h->lev_lo; l + 1 < h->nlev; ++l) {
        if (tc) {
            fda_split_tc(h, l, c32(P.p[l]), h->ps[l], mr);
            fda_run_tc(h, h->b_l2l[l], h->tc_l2l[l], h->ps[l], P.stride[l] / std::max(1, h->lev[l].T),
                       c32(P.p[l + 1]), mr, P.stride[l + 1]);
        } else {
            fda_run_batch<R>(h->b_l2l[l], P.Lt[l], h->lev[l + 1].T, h->lev[l].T, P.p[l], P.p[l + 1], mr,
                             P.stride[l], P.stride[l + 1], s);
        }
    }
    mark(5);
}

// side 0: the Burton-Miller operator of Eq. eq_sum applied to u; side 1: the
// right-hand side's layers of Eq. eq_bm applied to q = du/dn (its own near
// field and single-layer S2M; every translation and the L2T are shared)
template <typename R>
void apply_impl(fda_handle *h, far_ops<R> &ops, dbuf *q, dbuf *p, const void *x, int x64, c64d *y, int mr,
                int side)
{
    const dbuf &near = side ? ops.near1 : ops.near;
    const dbuf &St = side ? ops.St1 : ops.St;
    const int64_t N = h->N;
    cudaStream_t s = h->stream;
    const int NL = h->nleaf;
    auto mark = [&](int i) {
        if (h->timing) FDA_CUDA(cudaEventRecord(h->ev[i], s));
    };
    mark(0);
    const int max_rows = h->max_leaf_rows;
    const size_t xs_bytes = sizeof(cx<R>) * (size_t)h->max_near_cols;
    // several right-hand sides in the chosen precision: the leaf products
    // (near field, S2M, L2T) as tensor-core GEMMs with the right-hand sides as
    // columns; one right-hand side stays on the CUDA cores (bandwidth-bound)
    const bool leaf_tc = sizeof(R) == 4 && h->have_tc && h->cfg.tensor_cores && mr > 1 && !x64;
    if (leaf_tc) {
        fda_leaf_tc(h, 0, near, reinterpret_cast<const c32f *>(x), y, mr);
    } else if (mr == 1 && xs_bytes <= 160 * 1024) {
        dim3 gn(NL, 1, 1);  // one CTA per leaf: x gathered once, the CTA loops over the row groups
        static bool attr = false;
        if (!attr) {
            FDA_CUDA(cudaFuncSetAttribute(k_near_apply<R, 1, true, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          160 * 1024));
            attr = true;
        }
        k_near_apply<R, 1, true, 3><<<gn, AT, xs_bytes, s>>>(h->leaf_box.as<int32_t>(), h->box_begin.as<int32_t>(),
                                                          h->box_end.as<int32_t>(), h->nf_colptr.as<int64_t>(),
                                                          h->nf_cols.as<int32_t>(), h->nf_off.as<int64_t>(),
                                                          near.template as<cx<R>>(), x, x64, N, mr, y, N, h->nnz_near);
    } else if (mr == 1) {
        dim3 gn(NL, (max_rows + NRW * AT / 32 - 1) / (NRW * AT / 32), 1);
        k_near_apply<R, 1, false><<<gn, AT, 0, s>>>(h->leaf_box.as<int32_t>(), h->box_begin.as<int32_t>(),
                                                    h->box_end.as<int32_t>(), h->nf_colptr.as<int64_t>(),
                                                    h->nf_cols.as<int32_t>(), h->nf_off.as<int64_t>(),
                                                    near.template as<cx<R>>(), x, x64, N, mr, y, N, h->nnz_near);
    } else {
        dim3 gn(NL, (max_rows + NRW * AT / 32 - 1) / (NRW * AT / 32), (mr + NRG - 1) / NRG);
        k_near_apply<R, NRG, false><<<gn, AT, 0, s>>>(h->leaf_box.as<int32_t>(), h->box_begin.as<int32_t>(),
                                                      h->box_end.as<int32_t>(), h->nf_colptr.as<int64_t>(),
                                                      h->nf_cols.as<int32_t>(), h->nf_off.as<int64_t>(),
                                                      near.template as<cx<R>>(), x, x64, N, mr, y, N, h->nnz_near);
    }
    FDA_CHECK_LAUNCH();
    mark(1);
    if (h->lev_lo < 0) {
        for (int i = 2; i <= 6; ++i) mark(i);
        return;
    }
    lvl_ptrs<R> P = make_ptrs<R>(h, ops, q, p);
    {
        // every level's multipole and local densities to zero, one launch
        // (blocks per array from the largest one, about 2,048 elements each)
        const int nl = h->nlev - h->lev_lo;
        int64_t maxn = 0;
        for (int l = h->lev_lo; l < h->nlev; ++l) maxn = std::max(maxn, P.stride[l] * mr);
        const int gx = (int)std::min<int64_t>(2048, std::max<int64_t>(16, maxn / 2048));
        k_zero_levels<R><<<dim3(gx, 2 * nl), 256, 0, s>>>(P, h->lev_lo, mr);
        FDA_CHECK_LAUNCH();
    }
    if (leaf_tc) {
        fda_leaf_tc(h, 1, St, reinterpret_cast<const c32f *>(x), y, mr);
    } else if (mr == 1) {
        k_s2m_w<R><<<(NL + LPB - 1) / LPB, 32 * LPB, 0, s>>>(P, NL, h->leaf_box.as<int32_t>(),
                                                              h->box_level.as<int32_t>(), h->box_begin.as<int32_t>(),
                                                              h->box_end.as<int32_t>(), h->leaf_op_off.as<int64_t>(),
                                                              St.template as<cx<R>>(), x, x64);
        FDA_CHECK_LAUNCH();
    } else {
        k_s2m<R><<<NL, AT, 0, s>>>(P, h->leaf_box.as<int32_t>(), h->box_level.as<int32_t>(),
                                   h->box_begin.as<int32_t>(), h->box_end.as<int32_t>(),
                                   h->leaf_op_off.as<int64_t>(), St.template as<cx<R>>(), x, x64, N, mr);
        FDA_CHECK_LAUNCH();
    }
    mark(2);
    const bool tc = sizeof(R) == 4 && h->have_tc && h->cfg.tensor_cores;
    translate_passes<R>(h, P, mr, tc, mark);
    if (leaf_tc) {
        fda_leaf_tc(h, 2, ops.Tt, nullptr, y, mr);
    } else if (mr == 1) {
        // FP32: the operators without the 64-row padding (fewer DRAM bytes)
        const bool cpt = sizeof(R) == 4 && h->tt32c.p;
        const int64_t *lo = cpt ? h->tt_c_off.as<int64_t>() : h->leaf_op_off.as<int64_t>();
        const cx<R> *tt = cpt ? reinterpret_cast<const cx<R> *>(h->tt32c.p) : ops.Tt.template as<cx<R>>();
        k_l2t_w<R><<<(NL + LPB - 1) / LPB, 32 * LPB, 0, s>>>(P, NL, h->leaf_box.as<int32_t>(),
                                                              h->box_level.as<int32_t>(), h->box_begin.as<int32_t>(),
                                                              h->box_end.as<int32_t>(), lo, tt, y, cpt ? 1 : 0);
        FDA_CHECK_LAUNCH();
    } else {
        k_l2t<R><<<NL, AT, 0, s>>>(P, h->leaf_box.as<int32_t>(), h->box_level.as<int32_t>(),
                                   h->box_begin.as<int32_t>(), h->box_end.as<int32_t>(),
                                   h->leaf_op_off.as<int64_t>(), ops.Tt.template as<cx<R>>(), y, N, mr);
        FDA_CHECK_LAUNCH();
    }
    mark(6);
}

}  // namespace

void fda_near_product_f32(fda_handle *h, const c32f *A, const c64d *x, c64d *z)
{
    const size_t xs_bytes = sizeof(c32f) * (size_t)h->max_near_cols;
    dim3 gn(h->nleaf, (h->max_leaf_rows + NRW * AT / 32 - 1) / (NRW * AT / 32), 1);
    if (xs_bytes <= 160 * 1024) {
        gn.y = 1;  // one CTA per leaf (x gathered once)
        static bool attr = false;
        if (!attr) {
            FDA_CUDA(cudaFuncSetAttribute(k_near_apply<float, 1, true, 3>,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024));
            attr = true;
        }
        k_near_apply<float, 1, true, 3><<<gn, AT, xs_bytes, h->stream>>>(
            h->leaf_box.as<int32_t>(), h->box_begin.as<int32_t>(), h->box_end.as<int32_t>(),
            h->nf_colptr.as<int64_t>(), h->nf_cols.as<int32_t>(), h->nf_off.as<int64_t>(), A, x, 1, h->N, 1, z, h->N, h->nnz_near);
    } else {
        k_near_apply<float, 1, false><<<gn, AT, 0, h->stream>>>(
            h->leaf_box.as<int32_t>(), h->box_begin.as<int32_t>(), h->box_end.as<int32_t>(),
            h->nf_colptr.as<int64_t>(), h->nf_cols.as<int32_t>(), h->nf_off.as<int64_t>(), A, x, 1, h->N, 1, z, h->N, h->nnz_near);
    }
    FDA_CHECK_LAUNCH();
}

// Upward pass only, FP64 (Sec. 3.3 Step 2), for the far-field pattern: the
// outgoing densities q~ of every box from S2M at the leaves (side 0: the
// double layer of xs; side 1: the single layer, added to what is there) and
// M2M up to the coarsest level with interaction lists.  xs: Morton order.
void fda_upward_fp64(fda_handle *h, const c64d *xs, int side, int add)
{
    if (h->lev_lo < 0) return;
    cudaStream_t s = h->stream;
    lvl_ptrs<double> Q = make_ptrs<double>(h, h->op64, h->q64, h->p64);
    const dbuf &St = side ? h->op64.St1 : h->op64.St;
    if (!St.p) fda_fail(FDA_ERR_STATE, "S2M operators of this side were not built");
    // S2M writes the leaves' q~ into p64 (scratch) when adding, else into q64
    lvl_ptrs<double> D = Q;
    if (add)
        for (int l = 0; l < FDA_MAX_LEVELS; ++l) D.q[l] = Q.p[l];
    for (int l = h->lev_lo; l < h->nlev; ++l) {
        const level_info &L = h->lev[l];
        if (!L.active || L.T == 0) continue;
        const size_t bytes = sizeof(c64d) * (size_t)L.nbox * L.ncones * L.T;
        FDA_CUDA(cudaMemsetAsync(D.q[l], 0, bytes, s));
    }
    k_s2m<double><<<h->nleaf, AT, 0, s>>>(D, h->leaf_box.as<int32_t>(), h->box_level.as<int32_t>(),
                                          h->box_begin.as<int32_t>(), h->box_end.as<int32_t>(),
                                          h->leaf_op_off.as<int64_t>(), St.as<c64d>(), xs, 1, h->N, 1);
    FDA_CHECK_LAUNCH();
    if (add)
        for (int l = h->lev_lo; l < h->nlev; ++l) {
            const level_info &L = h->lev[l];
            if (!L.active || L.T == 0) continue;
            const int64_t n = (int64_t)L.nbox * L.ncones * L.T;
            k_add_c64<<<fda_blocks(n, 256), 256, 0, s>>>(Q.q[l], D.q[l], n);
            FDA_CHECK_LAUNCH();
        }
}

// M2M bottom-up in FP64 on q64 (after fda_upward_fp64)
void fda_m2m_fp64(fda_handle *h)
{
    if (h->lev_lo < 0) return;
    lvl_ptrs<double> Q = make_ptrs<double>(h, h->op64, h->q64, h->p64);
    for (int l = h->nlev - 2; l >= h->lev_lo; --l)
        fda_run_batch<double>(h->b_m2m[l], Q.Mt[l], h->lev[l].T, h->lev[l + 1].T, Q.q[l + 1], Q.q[l], 1,
                              Q.stride[l + 1], Q.stride[l], h->stream);
}

// Downward pass only, FP64 (Sec. 3.3 Step 3 without L2T), on the outgoing
// densities in q64 (after fda_upward_fp64 and fda_m2m_fp64): M2L at every
// level (the low-rank operators of Sec. 4.2 in two stages) and L2L top-down,
// leaving every box's complete local density in p64.
void fda_downward_fp64(fda_handle *h)
{
    if (h->lev_lo < 0) return;
    cudaStream_t s = h->stream;
    lvl_ptrs<double> P = make_ptrs<double>(h, h->op64, h->q64, h->p64);
    for (int l = h->lev_lo; l < h->nlev; ++l)
        if (P.stride[l] > 0 && P.T[l] > 0) FDA_CUDA(cudaMemsetAsync(P.p[l], 0, sizeof(c64d) * P.stride[l], s));
    for (int l = h->lev_lo; l < h->nlev; ++l) {
        fda_run_batch<double>(h->b_m2l[l], P.Kt[l], h->lev[l].T, h->lev[l].T, P.q[l], P.p[l], 1, P.stride[l],
                              P.stride[l], s);
        for (lr_bucket &B : h->lr[l]) lowrank_m2l<double>(h, B, l, P, 1, false);
    }
    for (int l = h->lev_lo; l + 1 < h->nlev; ++l)
        fda_run_batch<double>(h->b_l2l[l], P.Lt[l], h->lev[l + 1].T, h->lev[l].T, P.p[l], P.p[l + 1], 1,
                              P.stride[l], P.stride[l + 1], s);
}

__global__ void k_c32_to_c64(const c32f *a, c64d *b, int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        b[i] = c64d(a[i].re, a[i].im);
}

// Upward and downward passes in the chosen precision for the sources
// -D[u] + S[q] (xs = -u, qs = q or null; FP64, Morton order): S2M of xs by
// the operator's FP32 S2M and of qs by the right-hand side's (added), then
// M2M, M2L and L2L exactly as in an apply (the tensor cores where the
// handle uses them); the complete outgoing and local densities are then
// copied into q64 and p64.
void fda_translate_chosen(fda_handle *h, const c64d *xs, const c64d *qs)
{
    if (h->lev_lo < 0) return;
    if (!h->have32) fda_fail(FDA_ERR_STATE, "FP32 operators were not built (precision = plain)");
    if (qs && !h->op32.St1.p) fda_fail(FDA_ERR_STATE, "FP32 S2M operators of the right-hand side's layers missing");
    cudaStream_t s = h->stream;
    const int NL = h->nleaf;
    const int64_t N = h->N;
    if (!h->xs32.p) h->xs32.alloc(sizeof(c32f) * N * std::max(1, h->cfg.max_rhs));
    dbuf q32;
    lvl_ptrs<float> P = make_ptrs<float>(h, h->op32, h->q32, h->p32);
    const int nl = h->nlev - h->lev_lo;
    int64_t maxn = 0;
    for (int l = h->lev_lo; l < h->nlev; ++l) maxn = std::max(maxn, P.stride[l]);
    const int gx = (int)std::min<int64_t>(2048, std::max<int64_t>(16, maxn / 2048));
    k_zero_levels<float><<<dim3(gx, 2 * nl), 256, 0, s>>>(P, h->lev_lo, 1);
    FDA_CHECK_LAUNCH();
    k_c64_to_c32<<<fda_blocks(N, 256), 256, 0, s>>>(xs, h->xs32.as<c32f>(), N);
    FDA_CHECK_LAUNCH();
    k_s2m_w<float><<<(NL + LPB - 1) / LPB, 32 * LPB, 0, s>>>(
        P, NL, h->leaf_box.as<int32_t>(), h->box_level.as<int32_t>(), h->box_begin.as<int32_t>(),
        h->box_end.as<int32_t>(), h->leaf_op_off.as<int64_t>(), h->op32.St.as<c32f>(), h->xs32.p, 0);
    FDA_CHECK_LAUNCH();
    if (qs) {
        q32.alloc(sizeof(c32f) * N);
        k_c64_to_c32<<<fda_blocks(N, 256), 256, 0, s>>>(qs, q32.as<c32f>(), N);
        FDA_CHECK_LAUNCH();
        k_s2m_w<float, true><<<(NL + LPB - 1) / LPB, 32 * LPB, 0, s>>>(
            P, NL, h->leaf_box.as<int32_t>(), h->box_level.as<int32_t>(), h->box_begin.as<int32_t>(),
            h->box_end.as<int32_t>(), h->leaf_op_off.as<int64_t>(), h->op32.St1.as<c32f>(), q32.p, 0);
        FDA_CHECK_LAUNCH();
    }
    translate_passes<float>(h, P, 1, h->have_tc && h->cfg.tensor_cores, [](int) {});
    for (int l = h->lev_lo; l < h->nlev; ++l) {
        if (P.T[l] == 0 || !h->q64[l].p || !h->p64[l].p) continue;
        const int64_t n = P.stride[l];
        k_c32_to_c64<<<(unsigned)std::min<int64_t>(2048, std::max<int64_t>(1, n / 256)), 256, 0, s>>>(
            h->q32[l].as<c32f>(), h->q64[l].as<c64d>(), n);
        k_c32_to_c64<<<(unsigned)std::min<int64_t>(2048, std::max<int64_t>(1, n / 256)), 256, 0, s>>>(
            h->p32[l].as<c32f>(), h->p64[l].as<c64d>(), n);
        FDA_CHECK_LAUNCH();
    }
    FDA_CUDA(cudaStreamSynchronize(s));  // q32 (scratch) is freed on return
}

void fda_alloc_densities(fda_handle *h, int want32)
{
    for (int l = 0; l < h->nlev; ++l) {
        const level_info &L = h->lev[l];
        if (!L.active || L.T == 0) continue;
        size_t n = (size_t)L.nbox * L.ncones * L.T * std::max(1, h->cfg.max_rhs);
        h->q64[l].alloc(sizeof(c64d) * n);
        h->p64[l].alloc(sizeof(c64d) * n);
        if (want32) {
            h->q32[l].alloc(sizeof(c32f) * n);
            h->p32[l].alloc(sizeof(c32f) * n);
        }
    }
}

// ys = A xs, both complex double in Morton order
void fda_apply_sorted(fda_handle *h, const c64d *xs, c64d *ys, int precision, int mr, int side)
{
    if (mr < 1 || mr > std::max(1, h->cfg.max_rhs)) fda_fail(FDA_ERR_ARG, "more right-hand sides than max_rhs");
    if (precision == FDA_CHOSEN_FP32) {
        if (!h->have32) fda_fail(FDA_ERR_STATE, "FP32 operators were not built (precision = plain)");
        if (!h->xs32.p) h->xs32.alloc(sizeof(c32f) * h->N * std::max(1, h->cfg.max_rhs));
        k_c64_to_c32<<<fda_blocks(h->N * mr, 256), 256, 0, h->stream>>>(xs, h->xs32.as<c32f>(), h->N * mr);
        FDA_CHECK_LAUNCH();
        apply_impl<float>(h, h->op32, h->q32, h->p32, h->xs32.p, 0, ys, mr, side);
    } else {
        apply_impl<double>(h, h->op64, h->q64, h->p64, xs, 1, ys, mr, side);
    }
    if (h->timing) {
        FDA_CUDA(cudaEventSynchronize(h->ev[6]));
        float t[6];
        for (int i = 0; i < 6; ++i) FDA_CUDA(cudaEventElapsedTime(&t[i], h->ev[i], h->ev[i + 1]));
        // events: near | S2M | M2M | M2L | L2L | L2T
        h->pass_ms[5] = t[0];
        h->pass_ms[0] = t[1];
        h->pass_ms[1] = t[2];
        h->pass_ms[2] = t[3];
        h->pass_ms[3] = t[4];
        h->pass_ms[4] = t[5];
    }
}

// ---- tile-shape autotuner for the tensor-core batches
// For every M2M, M2L and L2L batch, each candidate (columns per tile, row
// tiles per tile, ring stages) is run twice on the FP32 densities of one right-hand side (their
// values do not change the work) and timed with CUDA events on the library
// stream; the faster candidate of the second runs is kept for one right-hand
// side.  Runs once, at the end of fda_precompute_translations.
// With an autotune cache file, batches found there (same GPU model, pass,
// level, ranks, operator and pair counts) take the stored shape untimed;
// the shapes of the batches timed here are appended to it.
void fda_autotune_tc(fda_handle *h)
{
    if (!h->have_tc || h->lev_lo < 0) return;
    cudaStream_t s = h->stream;
    cudaEvent_t e0, e1;
    FDA_CUDA(cudaEventCreate(&e0));
    FDA_CUDA(cudaEventCreate(&e1));
    lvl_ptrs<float> P = make_ptrs<float>(h, h->op32, h->q32, h->p32);
    // (columns, row tiles, stages)
    static const int cand[15][3] = {{32, 1, 2}, {32, 1, 4}, {64, 1, 2}, {64, 1, 4}, {32, 2, 4},
                                    {64, 2, 3}, {64, 2, 4}, {32, 3, 3}, {32, 3, 4}, {128, 1, 3},
                                    {128, 1, 4}, {128, 2, 2}, {128, 2, 3}, {64, 3, 3}, {64, 4, 2}};
    // launches are timed from a cold L2, as in an apply, where the other
    // passes evict the operators between two launches of one batch
    dbuf flush;
    flush.alloc((size_t)256 << 20);
    int nflush = 0;
    auto timed = [&](auto &&launch) {
        FDA_CUDA(cudaMemsetAsync(flush.p, ++nflush & 0xff, flush.bytes, s));
        FDA_CUDA(cudaEventRecord(e0, s));
        launch();
        FDA_CUDA(cudaEventRecord(e1, s));
        FDA_CUDA(cudaEventSynchronize(e1));
        float ms = 0.0f;
        FDA_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        return ms;
    };
    std::map<std::string, std::array<int, 3>> cache;
    std::string added;
    std::string gpu;
    if (!h->autotune_cache.empty()) {
        int dev = 0;
        cudaDeviceProp prop;
        FDA_CUDA(cudaGetDevice(&dev));
        FDA_CUDA(cudaGetDeviceProperties(&prop, dev));
        for (const char *c = prop.name; *c; ++c) gpu += (*c == ' ' || *c == '|') ? '_' : *c;
        gpu += "|" + std::to_string(prop.multiProcessorCount);
        if (FILE *f = fopen(h->autotune_cache.c_str(), "r")) {
            char key[512];
            int a, b, c;
            while (fscanf(f, "%511s %d %d %d", key, &a, &b, &c) == 4) cache[key] = {a, b, c};
            fclose(f);
        }
    }
    const int mmax = std::max(1, h->cfg.max_rhs);
    // one batch at mr right-hand sides (1 or max_rhs); at max_rhs only the
    // shapes of 64 or more columns are timed, each launch then being long
    auto tune1 = [&](const char *pass, int l, tr_batch &B, tc_ops &T, const dbuf &src, int64_t sv, float *dst,
                     int64_t ds, int mr) {
        if (B.npairs == 0 || !T.A.p) return;
        int &tnc = mr == 1 ? B.nc_tuned : B.nc_tm, &tr = mr == 1 ? B.r_tuned : B.r_tm,
            &tst = mr == 1 ? B.st_tuned : B.st_tm;
        std::string key;
        if (!gpu.empty()) {
            key = gpu + "|" + pass + "|" + std::to_string(l) + "|" + std::to_string(T.Tout) + "|" +
                  std::to_string(T.Tin) + "|" + std::to_string(B.op_start.empty() ? 0 : B.op_start.size() - 1) +
                  "|" + std::to_string(B.npairs) + (mr > 1 ? "|rhs" + std::to_string(mr) : std::string());
            auto it = cache.find(key);
            if (it != cache.end()) {
                const auto &c = it->second;
                bool known = false;
                for (const auto &k : cand) known |= k[0] == c[0] && k[1] == c[1] && k[2] == c[2];
                if (known && c[1] <= T.nrt) {
                    tnc = c[0];
                    tr = c[1];
                    tst = c[2];
                    ++h->autotune_cached;
                    return;
                }
            }
        }
        ++h->autotune_timed;
        float best = 1e30f;
        for (const auto &c : cand) {
            if (c[1] > T.nrt || (mr > 1 && c[0] < 64)) continue;
            // an untimed launch builds the shape's tile list; then the
            // fastest of three launches (two at max_rhs), each after L2 is flushed
            fda_run_tc(h, B, T, src, sv, reinterpret_cast<c32f *>(dst), mr, ds, c[0], c[1], c[2]);
            float ms = 1e30f;
            for (int rep = 0; rep < (mr == 1 ? 3 : 2); ++rep) ms = std::min(ms, timed([&] {
                fda_run_tc(h, B, T, src, sv, reinterpret_cast<c32f *>(dst), mr, ds, c[0], c[1], c[2]);
            }));
            if (ms < best) {
                best = ms;
                tnc = c[0];
                tr = c[1];
                tst = c[2];
            }
        }
        if (!key.empty())
            added += key + " " + std::to_string(tnc) + " " + std::to_string(tr) + " " + std::to_string(tst) + "\n";
    };
    auto tune = [&](const char *pass, int l, tr_batch &B, tc_ops &T, const dbuf &src, int64_t sv, float *dst,
                    int64_t ds) {
        tune1(pass, l, B, T, src, sv, dst, ds, 1);
        if (mmax > 1) tune1(pass, l, B, T, src, sv, dst, ds, mmax);
    };
    auto sv = [&](int l) { return P.stride[l] / std::max(1, h->lev[l].T); };
    for (int l = h->lev_lo; l < h->nlev; ++l) {
        if (h->lev[l].T == 0) continue;
        tune("m2l", l, h->b_m2l[l], h->tc_m2l[l], h->qs[l], sv(l), reinterpret_cast<float *>(P.p[l]), P.stride[l]);
        if (!h->lr[l].empty()) {
            tune("m2l_all", l, h->b_m2l_all[l], h->tc_m2l[l], h->qs[l], sv(l), reinterpret_cast<float *>(P.p[l]),
                 P.stride[l]);
            for (lr_bucket &B : h->lr[l]) {
                if (B.npairs == 0) continue;
                const int64_t per = B.npairs * B.rpad;
                if (B.t32.bytes < sizeof(c32f) * (size_t)per || B.ts.bytes < 8 * (size_t)per)
                    fda_fail(FDA_ERR_STATE, "low-rank intermediates missing at autotune");
                tune("lr1", l, B.b1, B.tc1, h->qs[l], sv(l), reinterpret_cast<float *>(B.t32.p), per);
                tune("lr2", l, B.b2, B.tc2, B.ts, B.npairs, reinterpret_cast<float *>(P.p[l]), P.stride[l]);
            }
            // the level's M2L in full form against the low-rank form (Sec. 4.2),
            // tuned shapes, for one right-hand side and for max_rhs; the faster
            // form is kept for each
            for (int mr = 1; mr <= mmax; mr = mr == mmax ? mmax + 1 : mmax) {
                auto full = [&] {
                    fda_run_tc(h, h->b_m2l_all[l], h->tc_m2l[l], h->qs[l], sv(l), reinterpret_cast<c32f *>(P.p[l]),
                               mr, P.stride[l]);
                };
                auto lowrank = [&] {
                    fda_run_tc(h, h->b_m2l[l], h->tc_m2l[l], h->qs[l], sv(l), reinterpret_cast<c32f *>(P.p[l]), mr,
                               P.stride[l]);
                    for (lr_bucket &B : h->lr[l]) lowrank_m2l<float>(h, B, l, P, mr, true);
                };
                full();
                lowrank();
                float t_full = 1e30f, t_lr = 1e30f;
                for (int rep = 0; rep < 3; ++rep) {
                    t_full = std::min(t_full, timed(full));
                    t_lr = std::min(t_lr, timed(lowrank));
                }
                (mr == 1 ? h->lr_tc[l] : h->lr_tc_many[l]) = t_lr < t_full ? 1 : 0;
                if (mmax == 1) h->lr_tc_many[l] = h->lr_tc[l];
            }
        }
        if (l + 1 < h->nlev && h->lev[l + 1].T > 0) {
            tune("m2m", l, h->b_m2m[l], h->tc_m2m[l], h->qs[l + 1], sv(l + 1), reinterpret_cast<float *>(P.q[l]),
                 P.stride[l]);
            tune("l2l", l, h->b_l2l[l], h->tc_l2l[l], h->ps[l], sv(l), reinterpret_cast<float *>(P.p[l + 1]),
                 P.stride[l + 1]);
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (!added.empty()) {
        if (FILE *f = fopen(h->autotune_cache.c_str(), "a")) {
            fputs(added.c_str(), f);
            fclose(f);
        }
    }
    if (fda_tc_error(h)) fda_fail(FDA_ERR_TIMEOUT, "a tensor-core translation gave up waiting on its copies");
}

// ---- one CUDA graph per operator application
// The first apply with a given (precision, right-hand sides, tensor-core
// switch) runs eagerly, which also cuts the tiles and sizes every buffer the
// apply touches; the second captures the same launch sequence on the
// handle's private stream; later ones replay it.  The graph reads h->xs and
// writes h->ys.  A capture that fails falls back to eager launches for good.
void fda_apply_staged(fda_handle *h, int precision, int mr)
{
    const c64d *xs = h->xs.as<c64d>();
    c64d *ys = h->ys.as<c64d>();
    if (h->timing || !h->cfg.graphs || h->graphs_broken) {
        fda_apply_sorted(h, xs, ys, precision, mr);
        return;
    }
    const int key = precision | (h->cfg.tensor_cores << 1) | (mr << 2);
    fda_handle::apply_graph *g = nullptr;
    for (auto &e : h->graphs)
        if (e.key == key) g = &e;
    if (!g) {
        fda_apply_sorted(h, xs, ys, precision, mr);
        h->graphs.push_back(fda_handle::apply_graph{key, nullptr, 0});
        return;
    }
    if (!h->gstream) {
        FDA_CUDA(cudaStreamCreateWithFlags(&h->gstream, cudaStreamNonBlocking));
        FDA_CUDA(cudaEventCreateWithFlags(&h->gev[0], cudaEventDisableTiming));
        FDA_CUDA(cudaEventCreateWithFlags(&h->gev[1], cudaEventDisableTiming));
    }
    if (!g->exec) {
        cudaStream_t user = h->stream;
        cudaGraph_t graph = nullptr;
        FDA_CUDA(cudaStreamSynchronize(user));
        h->stream = h->gstream;
        bool ok = cudaStreamBeginCapture(h->gstream, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
        const long long n0 = fda_launches_so_far();
        if (ok) {
            try {
                fda_apply_sorted(h, xs, ys, precision, mr);
            } catch (...) {
                ok = false;
            }
            // the captured launches were counted but did not run
            g->kernels = fda_launches_so_far() - n0;
            fda_count_launches(-g->kernels);
            ok = (cudaStreamEndCapture(h->gstream, &graph) == cudaSuccess) && ok && graph;
        }
        h->stream = user;
        if (ok) ok = cudaGraphInstantiate(&g->exec, graph, 0) == cudaSuccess;
        if (graph) cudaGraphDestroy(graph);
        if (!ok) {
            (void)cudaGetLastError();
            g->exec = nullptr;
            h->graphs_broken = 1;
            fda_apply_sorted(h, xs, ys, precision, mr);
            return;
        }
    }
    FDA_CUDA(cudaEventRecord(h->gev[0], h->stream));
    FDA_CUDA(cudaStreamWaitEvent(h->gstream, h->gev[0], 0));
    FDA_CUDA(cudaGraphLaunch(g->exec, h->gstream));
    ++h->graph_replays;
    fda_count_launches(g->kernels);
    FDA_CUDA(cudaEventRecord(h->gev[1], h->gstream));
    FDA_CUDA(cudaStreamWaitEvent(h->stream, h->gev[1], 0));
}

void fda_graphs_release(fda_handle *h)
{
    if (h->gstream) cudaStreamSynchronize(h->gstream);
    for (auto &e : h->graphs)
        if (e.exec) cudaGraphExecDestroy(e.exec);
    h->graphs.clear();
    for (int i = 0; i < 2; ++i)
        if (h->gev[i]) cudaEventDestroy(h->gev[i]);
    if (h->gstream) cudaStreamDestroy(h->gstream);
    h->gstream = nullptr;
}
