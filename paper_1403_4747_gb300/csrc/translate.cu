// Batched translations (M2L, M2M, L2L of Sec. 3.3 Steps 2-3, in the
// compressed coordinates of Sec. 4).
//
// Every translation of one pass and level is y_dst += A_op x_src with one of
// a few distinct operators A_op (an M2L offset; an octant and cone for M2M
// and L2L).  The (src, dst) pairs are grouped by operator into tiles of up to
// NP pairs and TM output rows; one CTA streams the operator's TM-row panel
// through shared memory once and multiplies it against the NP gathered source
// vectors, a complex GEMM of TM x Tin x NP with (TM/16) x (NP/16) register blocking,
// then adds its results into the targets with atomics (targets of one tile are
// distinct; different operators reach the same target from other CTAs).
// This replaces one operator read per (target, source) pair by one per tile.
#include <algorithm>
#include <vector>

#include "fda_internal.cuh"

int fda_child_cone(const fda_handle *h, int l, int u);

namespace {

constexpr int TK = 16;   // inner dimension per shared-memory stage
constexpr int BT = 256;  // threads

struct tr_tile {
    int op, pair0, npair, row0;
};

template <typename R>
__device__ inline void atomic_add_cx(cx<R> *p, cx<R> v);

template <>
__device__ inline void atomic_add_cx<float>(cx<float> *p, cx<float> v)
{
    atomicAdd(reinterpret_cast<float2 *>(p), make_float2(v.re, v.im));
}

template <>
__device__ inline void atomic_add_cx<double>(cx<double> *p, cx<double> v)
{
    atomicAdd(&p->re, v.re);
    atomicAdd(&p->im, v.im);
}

// One tile: TM output rows x NP (source, target) pairs.  Thread (tx, ty)
// owns rows row0 + tx + 16 i (i < TM/16; a warp reads consecutive rows of the
// operator panel, so shared-memory reads are conflict-free) and pairs
// ty * PT + j (j < PT = NP/16).
//
// With several right-hand sides the source densities of right-hand side m
// sit at offset m * sstride and the targets at m * dstride (M2M and L2L read
// one level and write another), and a tile's columns run over (pair,
// right-hand side) combinations: column v of an operator's range is pair
// v / mr, side v % mr.
template <typename R, int TM, int NP>
__global__ void __launch_bounds__(BT) k_btr(const tr_tile *tiles, const int2 *pairs, const cx<R> *ops, int Tout,
                                            int Tin, const cx<R> *src, cx<R> *dst, int mr, int64_t sstride,
                                            int64_t dstride)
{
    constexpr int PT = NP / 16;  // pairs per thread
    constexpr int RT = TM / 16;  // rows per thread
    __shared__ cx<R> As[TK][TM];
    __shared__ cx<R> Bs[TK][NP + 1];
    __shared__ longlong2 pp[NP];
    const tr_tile t = tiles[blockIdx.x];
    const cx<R> *A = ops + (int64_t)t.op * Tout * Tin;
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    if (tid < NP) {
        longlong2 v = make_longlong2(-1, -1);
        if (tid < t.npair) {
            int vi = t.pair0 + tid;
            int pi = vi / mr, m = vi - pi * mr;
            int2 q = pairs[pi];
            v = make_longlong2(q.x + m * sstride, q.y + m * dstride);
        }
        pp[tid] = v;
    }
    cx<R> acc[RT][PT];
    __syncthreads();
    for (int k0 = 0; k0 < Tin; k0 += TK) {
        for (int e = tid; e < TK * TM; e += BT) {
            int kk = e / TM, rr = e % TM;
            int c = k0 + kk, r = t.row0 + rr;
            As[kk][rr] = (c < Tin && r < Tout) ? A[(int64_t)c * Tout + r] : cx<R>();
        }
        for (int e = tid; e < TK * NP; e += BT) {
            int p = e / TK, kk = e % TK;  // 16 consecutive entries of one source vector per half-warp
            int c = k0 + kk;
            long long so = pp[p].x;
            Bs[kk][p] = (so >= 0 && c < Tin) ? src[so + c] : cx<R>();
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < TK; ++kk) {
            cx<R> a[RT], b[PT];
#pragma unroll
            for (int i = 0; i < RT; ++i) a[i] = As[kk][tx + 16 * i];
#pragma unroll
            for (int j = 0; j < PT; ++j) b[j] = Bs[kk][ty * PT + j];
#pragma unroll
            for (int i = 0; i < RT; ++i)
#pragma unroll
                for (int j = 0; j < PT; ++j) cfma(acc[i][j], a[i], b[j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int j = 0; j < PT; ++j) {
        int p = ty * PT + j;
        if (p >= t.npair) continue;
        long long dof = pp[p].y;
#pragma unroll
        for (int i = 0; i < RT; ++i) {
            int r = t.row0 + tx + 16 * i;
            if (r < Tout) atomic_add_cx<R>(dst + dof + r, acc[i][j]);
        }
    }
}

struct pair_rec {
    int op, src, dst;
};

// group pairs by operator (stable) and cut them into tiles
void make_batch(std::vector<pair_rec> &pr, int nops, int Tout, tr_batch &B)
{
    std::vector<int> cnt(nops + 1, 0);
    for (auto &p : pr) cnt[p.op + 1]++;
    for (int o = 0; o < nops; ++o) cnt[o + 1] += cnt[o];
    std::vector<int2> pairs(pr.size());
    std::vector<int> pos(cnt.begin(), cnt.end() - 1);
    for (auto &p : pr) pairs[pos[p.op]++] = make_int2(p.src, p.dst);
    // row-tile height: the one that pads Tout the least (ties: 64)
    int pad64 = (Tout + 63) / 64 * 64 - Tout, pad32 = (Tout + 31) / 32 * 32 - Tout;
    B.tm = pad64 <= pad32 ? 64 : 32;
    B.tout = Tout;
    B.op_start.assign(cnt.begin(), cnt.end());
    B.npairs = (int64_t)pairs.size();
    B.pairs.alloc(sizeof(int2) * std::max<size_t>(pairs.size(), 1));
    if (!pairs.empty()) FDA_CUDA(cudaMemcpy(B.pairs.p, pairs.data(), sizeof(int2) * pairs.size(), cudaMemcpyHostToDevice));
    B.tilesets.clear();
}

// tiles for mr right-hand sides: each operator's pairs x mr columns, cut
// into NP-column, TM-row tiles
const tile_set &ensure_tiles(tr_batch &B, int mr)
{
    for (const auto &t : B.tilesets)
        if (t.mr == mr) return t;
    const int nops = (int)B.op_start.size() - 1;
    double avg = B.npairs == 0 ? 0.0 : (double)B.npairs * mr / std::max(1, nops);
    const int np = avg >= 48.0 ? 64 : 32;
    std::vector<tr_tile> tiles;
    for (int o = 0; o < nops; ++o) {
        int a = B.op_start[o] * mr, b = B.op_start[o + 1] * mr;
        for (int p0 = a; p0 < b; p0 += np)
            for (int r0 = 0; r0 < B.tout; r0 += B.tm) tiles.push_back(tr_tile{o, p0, std::min(np, b - p0), r0});
    }
    B.tilesets.emplace_back();
    tile_set &t = B.tilesets.back();
    t.mr = mr;
    t.nc = np;
    t.n = (int)tiles.size();
    t.buf.alloc(sizeof(tr_tile) * std::max<size_t>(tiles.size(), 1));
    if (!tiles.empty())
        FDA_CUDA(cudaMemcpy(t.buf.p, tiles.data(), sizeof(tr_tile) * tiles.size(), cudaMemcpyHostToDevice));
    return t;
}

}  // namespace

// Build the M2L, M2M and L2L batches from the interaction lists and the tree.
void fda_build_batches(fda_handle *h)
{
    const int NB = h->nbox_total;
    std::vector<int32_t> par(NB), coord(3 * (size_t)NB), leaf(NB);
    FDA_CUDA(cudaMemcpy(par.data(), h->box_parent.p, 4 * (size_t)NB, cudaMemcpyDeviceToHost));
    FDA_CUDA(cudaMemcpy(coord.data(), h->box_coord.p, 12 * (size_t)NB, cudaMemcpyDeviceToHost));
    FDA_CUDA(cudaMemcpy(leaf.data(), h->box_leaf.p, 4 * (size_t)NB, cudaMemcpyDeviceToHost));
    std::vector<int64_t> ilp(NB + 1);
    FDA_CUDA(cudaMemcpy(ilp.data(), h->il_ptr.p, 8 * (size_t)(NB + 1), cudaMemcpyDeviceToHost));
    const int64_t nil = h->n_il_total;
    std::vector<int32_t> ils(nil), ilo(nil), ilc(nil);
    if (nil) {
        FDA_CUDA(cudaMemcpy(ils.data(), h->il_src.p, 4 * (size_t)nil, cudaMemcpyDeviceToHost));
        FDA_CUDA(cudaMemcpy(ilo.data(), h->il_op.p, 4 * (size_t)nil, cudaMemcpyDeviceToHost));
        FDA_CUDA(cudaMemcpy(ilc.data(), h->il_cone.p, 4 * (size_t)nil, cudaMemcpyDeviceToHost));
    }
    auto octant = [&](int b) {
        return ((coord[3 * b] & 1) << 2) | ((coord[3 * b + 1] & 1) << 1) | (coord[3 * b + 2] & 1);
    };
    for (int l = h->lev_lo; l >= 0 && l < h->nlev; ++l) {
        const level_info &L = h->lev[l];
        std::vector<pair_rec> pr;
        for (int b = L.box0; b < L.box0 + L.nbox; ++b)
            for (int64_t e = ilp[b]; e < ilp[b + 1]; ++e) {
                int u = ilc[e] & 0xffff, su = ilc[e] >> 16;
                pr.push_back(pair_rec{ilo[e], ((ils[e] - L.box0) * L.ncones + su) * L.T,
                                      ((b - L.box0) * L.ncones + u) * L.T});
            }
        // low-rank operators (Sec. 4.2): their pairs go to the rank buckets,
        // stage 1 writing pair p's intermediate at p rpad, stage 2 reading it
        const std::vector<int> &bk = h->op_bucket[l];
        if (!h->lr[l].empty()) {
            std::vector<pair_rec> all(pr);
            make_batch(all, std::max(1, L.n_ops), L.T, h->b_m2l_all[l]);
            std::vector<pair_rec> full;
            std::vector<std::vector<pair_rec>> per(h->lr[l].size());
            std::vector<int> local(L.n_ops, -1);  // operator index inside its bucket
            for (size_t b = 0; b < h->lr[l].size(); ++b)
                for (size_t i = 0; i < h->lr[l][b].ops.size(); ++i) local[h->lr[l][b].ops[i]] = (int)i;
            for (const pair_rec &p : pr) {
                const int b = p.op < (int)bk.size() ? bk[p.op] : -1;
                if (b < 0) full.push_back(p);
                else per[b].push_back(pair_rec{local[p.op], p.src, p.dst});
            }
            for (size_t b = 0; b < per.size(); ++b) {
                lr_bucket &B = h->lr[l][b];
                std::vector<pair_rec> &q = per[b];
                // group by bucket operator (stable), so both stages see the same order
                std::stable_sort(q.begin(), q.end(), [](const pair_rec &x, const pair_rec &y) { return x.op < y.op; });
                std::vector<pair_rec> s1(q.size()), s2(q.size());
                for (size_t i = 0; i < q.size(); ++i) {
                    s1[i] = pair_rec{q[i].op, q[i].src, (int)i * B.rpad};
                    s2[i] = pair_rec{q[i].op, (int)i * B.rpad, q[i].dst};
                }
                const int nb = std::max(1, (int)B.ops.size());
                make_batch(s1, nb, B.rpad, B.b1);
                make_batch(s2, nb, L.T, B.b2);
                B.npairs = (int64_t)q.size();
                // intermediates for max_rhs right-hand sides, allocated once:
                // captured graphs keep their addresses
                const size_t vals = (size_t)B.npairs * B.rpad * std::max(1, h->cfg.max_rhs);
                B.t64.alloc(sizeof(c64d) * vals);
                if (h->cfg.precision == FDA_CHOSEN_FP32) {
                    B.t32.alloc(sizeof(c32f) * vals);
                    if (h->cfg.tensor_cores) {
                        // bf16 hi/lo of Re and Im: 8 bytes per value (rpad is a multiple of 32)
                        B.ts.alloc(8 * vals);
                        FDA_CUDA(cudaMemsetAsync(B.ts.p, 0, B.ts.bytes, h->stream));
                    }
                }
            }
            pr.swap(full);
        }
        make_batch(pr, std::max(1, L.n_ops), L.T, h->b_m2l[l]);
        if (l + 1 >= h->nlev) continue;
        const level_info &C = h->lev[l + 1];
        std::vector<pair_rec> up, dn;
        for (int c = C.box0; c < C.box0 + C.nbox; ++c) {
            int P = par[c];
            int o = octant(c);
            for (int u = 0; u < L.ncones; ++u) {
                int uc = C.hf ? fda_child_cone(h, l, u) : 0;
                int op = o * L.ncones + u;
                int qc = ((c - C.box0) * C.ncones + uc) * C.T;
                int qp = ((P - L.box0) * L.ncones + u) * L.T;
                up.push_back(pair_rec{op, qc, qp});
                dn.push_back(pair_rec{op, qp, qc});
            }
        }
        make_batch(up, 8 * L.ncones, L.T, h->b_m2m[l]);
        make_batch(dn, 8 * L.ncones, C.T, h->b_l2l[l]);
    }
}

template <typename R>
void fda_run_batch(tr_batch &B, const cx<R> *ops, int Tout, int Tin, const cx<R> *src, cx<R> *dst, int mr,
                   int64_t sstride, int64_t dstride, cudaStream_t s)
{
    if (B.npairs == 0) return;
    const tile_set &ts = ensure_tiles(B, mr);
    const tr_tile *t = ts.buf.as<tr_tile>();
    const int2 *pr = B.pairs.as<int2>();
    if (B.tm == 64 && ts.nc == 64)
        k_btr<R, 64, 64><<<ts.n, BT, 0, s>>>(t, pr, ops, Tout, Tin, src, dst, mr, sstride, dstride);
    else if (B.tm == 64)
        k_btr<R, 64, 32><<<ts.n, BT, 0, s>>>(t, pr, ops, Tout, Tin, src, dst, mr, sstride, dstride);
    else if (ts.nc == 64)
        k_btr<R, 32, 64><<<ts.n, BT, 0, s>>>(t, pr, ops, Tout, Tin, src, dst, mr, sstride, dstride);
    else
        k_btr<R, 32, 32><<<ts.n, BT, 0, s>>>(t, pr, ops, Tout, Tin, src, dst, mr, sstride, dstride);
    FDA_CHECK_LAUNCH();
}

template void fda_run_batch<float>(tr_batch &, const cx<float> *, int, int, const cx<float> *, cx<float> *, int,
                                   int64_t, int64_t, cudaStream_t);
template void fda_run_batch<double>(tr_batch &, const cx<double> *, int, int, const cx<double> *, cx<double> *,
                                    int, int64_t, int64_t, cudaStream_t);
