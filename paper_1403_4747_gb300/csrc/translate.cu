// Batched translations (M2L, M2M, L2L of Sec. 3.3 Steps 2-3, in the
// compressed coordinates of Sec. 4).
//
// Every translation of one pass and level is y_dst += A_op x_src with one of
// a few distinct operators A_op (an M2L offset; an octant and cone for M2M
// and L2L).  The (src, dst) pairs are grouped by operator into tiles of up to
// NP pairs and TM output rows; one CTA streams the operator's TM-row panel
// through shared memory once and multiplies it against the NP gathered source
// vectors, a complex GEMM of TM x Tin x NP with 4 x (NP/16) register blocking,
// then adds its results into the targets with atomics (targets of one tile are
// distinct; different operators reach the same target from other CTAs).
// This replaces one operator read per (target, source) pair by one per tile.
#include <algorithm>
#include <vector>

#include "fda_internal.cuh"

int fda_child_cone(const fda_handle *h, int l, int u);

namespace {

constexpr int TM = 64;   // output rows per tile
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

template <typename R, int NP>
__global__ void __launch_bounds__(BT) k_btr(const tr_tile *tiles, const int2 *pairs, const cx<R> *ops, int Tout,
                                            int Tin, const cx<R> *src, cx<R> *dst)
{
    constexpr int PT = NP / 16;  // pairs per thread
    __shared__ cx<R> As[TK][TM];
    __shared__ cx<R> Bs[TK][NP];
    __shared__ int2 pp[NP];
    const tr_tile t = tiles[blockIdx.x];
    const cx<R> *A = ops + (int64_t)t.op * Tout * Tin;
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    if (tid < NP) pp[tid] = tid < t.npair ? pairs[t.pair0 + tid] : make_int2(-1, -1);
    cx<R> acc[4][PT];
    __syncthreads();
    for (int k0 = 0; k0 < Tin; k0 += TK) {
        for (int e = tid; e < TK * TM; e += BT) {
            int kk = e / TM, rr = e % TM;
            int c = k0 + kk, r = t.row0 + rr;
            As[kk][rr] = (c < Tin && r < Tout) ? A[(int64_t)c * Tout + r] : cx<R>();
        }
        for (int e = tid; e < TK * NP; e += BT) {
            int p = e / TK, kk = e % TK;
            int c = k0 + kk;
            int so = pp[p].x;
            Bs[kk][p] = (so >= 0 && c < Tin) ? src[so + c] : cx<R>();
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < TK; ++kk) {
            cx<R> a[4], b[PT];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][tx * 4 + i];
#pragma unroll
            for (int j = 0; j < PT; ++j) b[j] = Bs[kk][ty * PT + j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < PT; ++j) cfma(acc[i][j], a[i], b[j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int j = 0; j < PT; ++j) {
        int p = ty * PT + j;
        if (p >= t.npair) continue;
        int dof = pp[p].y;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            int r = t.row0 + tx * 4 + i;
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
    double avg = pr.empty() ? 0.0 : (double)pr.size() / std::max(1, nops);
    B.np = avg >= 48.0 ? 64 : 32;
    std::vector<tr_tile> tiles;
    for (int o = 0; o < nops; ++o) {
        int a = cnt[o], b = cnt[o + 1];
        for (int p0 = a; p0 < b; p0 += B.np)
            for (int r0 = 0; r0 < Tout; r0 += TM) tiles.push_back(tr_tile{o, p0, std::min(B.np, b - p0), r0});
    }
    B.ntiles = (int)tiles.size();
    B.npairs = (int64_t)pairs.size();
    B.tiles.alloc(sizeof(tr_tile) * std::max<size_t>(tiles.size(), 1));
    B.pairs.alloc(sizeof(int2) * std::max<size_t>(pairs.size(), 1));
    if (!tiles.empty()) FDA_CUDA(cudaMemcpy(B.tiles.p, tiles.data(), sizeof(tr_tile) * tiles.size(), cudaMemcpyHostToDevice));
    if (!pairs.empty()) FDA_CUDA(cudaMemcpy(B.pairs.p, pairs.data(), sizeof(int2) * pairs.size(), cudaMemcpyHostToDevice));
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
void fda_run_batch(const tr_batch &B, const cx<R> *ops, int Tout, int Tin, const cx<R> *src, cx<R> *dst,
                   cudaStream_t s)
{
    if (B.ntiles == 0) return;
    if (B.np == 64)
        k_btr<R, 64><<<B.ntiles, BT, 0, s>>>(B.tiles.as<tr_tile>(), B.pairs.as<int2>(), ops, Tout, Tin, src, dst);
    else
        k_btr<R, 32><<<B.ntiles, BT, 0, s>>>(B.tiles.as<tr_tile>(), B.pairs.as<int2>(), ops, Tout, Tin, src, dst);
    FDA_CHECK_LAUNCH();
}

template void fda_run_batch<float>(const tr_batch &, const cx<float> *, int, int, const cx<float> *, cx<float> *,
                                   cudaStream_t);
template void fda_run_batch<double>(const tr_batch &, const cx<double> *, int, int, const cx<double> *,
                                    cx<double> *, cudaStream_t);
