// Sec. 3.3 Step 1 on the device: adaptive octree (built as in FMM and
// kernel-independent FMM, Sec. 3.2), far fields per level, the split into
// low- and high-frequency regimes, directional cones of the high-frequency
// far fields, interaction lists and near-field lists.
//
// Readings of what the paper leaves to its references (each listed in the
// design notes):
//   * a cube is high-frequency iff its width w >= hf_wavelengths * lambda;
//     high-frequency cubes are always split, so leaves are low-frequency;
//   * "near" at level l for an integer offset D (in box widths) between two
//     cubes: max|D_i| <= 1 (adjacent), or, at a high-frequency level,
//     |D| < rho_l = max(rho_min, w/lambda) (the directional far field starts
//     at distance w^2/lambda, the parabolic separation of Sec. 3.1);
//   * the interaction list of a cube: cubes of its level that are not near
//     it but whose parents are near its parent (and have children);
//   * high-frequency cones: each of the 6 cube faces is split into nc x nc
//     cells, nc = 2^floor(log2(w/lambda)); a cone is the set of directions
//     through one cell;
//   * near field of a leaf B: every leaf X at a level l <= level(B) that is
//     near B's ancestor at level l, and every non-leaf cube near B at B's own
//     level (its whole element range).  These are exactly the element pairs
//     that no translation covers, so the far field and the near field
//     partition all pairs.
#include <math.h>

#include <algorithm>
#include <array>
#include <map>
#include <vector>

#include "fda_internal.cuh"
#include "tree_util.cuh"

namespace {

constexpr int MAXD = 20;  // Morton depth

__device__ __host__ inline uint64_t compact3(uint64_t v)
{
    v &= 0x1249249249249249ull;
    v = (v ^ (v >> 2)) & 0x10c30c30c30c30c3ull;
    v = (v ^ (v >> 4)) & 0x100f00f00f00f00full;
    v = (v ^ (v >> 8)) & 0x1f0000ff0000ffull;
    v = (v ^ (v >> 16)) & 0x1f00000000ffffull;
    v = (v ^ (v >> 32)) & 0x1fffffull;
    return v;
}

__global__ void k_heads(const uint64_t *key, const int32_t *active, int64_t n, int shift, int32_t *head)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    int h = 0;
    if (active[i]) {
        if (i == 0 || !active[i - 1] || (key[i] >> shift) != (key[i - 1] >> shift)) h = 1;
    }
    head[i] = h;
}

__global__ void k_boxes(const uint64_t *key, const int32_t *active, const int32_t *head, const int32_t *scan,
                        int64_t n, int shift, int level, int parent_box0, const int32_t *ebox_prev, int32_t *ebox,
                        int32_t *bbeg, int32_t *bend, uint64_t *bkey, int32_t *bcoord, int32_t *bpar)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (!active[i]) {
        ebox[i] = -1;
        return;
    }
    int b = scan[i] + head[i] - 1;
    ebox[i] = b;
    uint64_t pre = key[i] >> shift;
    if (head[i]) {
        bbeg[b] = (int32_t)i;
        bkey[b] = pre;
        bcoord[3 * b + 0] = (int32_t)compact3(pre >> 2);
        bcoord[3 * b + 1] = (int32_t)compact3(pre >> 1);
        bcoord[3 * b + 2] = (int32_t)compact3(pre);
        bpar[b] = level == 0 ? -1 : parent_box0 + ebox_prev[i];
    }
    if (i == n - 1 || !active[i + 1] || (key[i + 1] >> shift) != pre) bend[b] = (int32_t)(i + 1);
}

__global__ void k_leaf_flags(const int32_t *bbeg, const int32_t *bend, int nbox, int can_leaf, int leaf_max,
                             int force, int32_t *leaf)
{
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nbox) return;
    int cnt = bend[b] - bbeg[b];
    leaf[b] = force || (can_leaf && cnt <= leaf_max);
}

__global__ void k_deactivate(int32_t *active, const int32_t *ebox, const int32_t *leaf, int64_t n)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (active[i] && leaf[ebox[i]]) active[i] = 0;
}

__global__ void k_children(const int32_t *par, int nbox, int box0, int32_t *c0, int32_t *c1)
{
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nbox) return;
    int p = par[box0 + b];
    if (p < 0) return;
    if (b == 0 || par[box0 + b - 1] != p) c0[p] = box0 + b;
    if (b == nbox - 1 || par[box0 + b + 1] != p) c1[p] = box0 + b + 1;
}

struct dev_levels {
    int box0[FDA_MAX_LEVELS];
    int nbox[FDA_MAX_LEVELS];
    int hf[FDA_MAX_LEVELS];
    double rho2[FDA_MAX_LEVELS];
    int Roff[FDA_MAX_LEVELS];
    int nc[FDA_MAX_LEVELS];
    int noff[FDA_MAX_LEVELS];   // near offsets per level
    int off0[FDA_MAX_LEVELS];   // start in the near-offset table
};

__device__ int find_box(const dev_levels &L, const uint64_t *bkey, int level, int x, int y, int z)
{
    return find_box_at(bkey, L.box0[level], L.nbox[level], level, x, y, z);
}

__device__ inline bool is_near(const dev_levels &L, int level, int dx, int dy, int dz)
{
    int m = max(abs(dx), max(abs(dy), abs(dz)));
    if (m <= 1) return true;
    if (L.hf[level]) return (double)(dx * dx + dy * dy + dz * dz) < L.rho2[level];
    return false;
}

// interaction lists: pass 0 counts, pass 1 fills (cnt holds CSR offsets then)
// Every index is checked against its array before use; a violation is
// recorded in err[0..3] (code, box, value, level) and the access skipped.
__device__ inline bool il_bad(int *err, int code, int b, long long v, int level)
{
    if (atomicCAS(err, 0, code) == 0) {
        err[1] = b;
        err[2] = (int)v;
        err[3] = level;
    }
    return true;
}

__global__ void k_il(dev_levels L, int level, const int3 *offs, int noffs, const uint64_t *bkey,
                     const int32_t *bcoord, const int32_t *bpar, const int32_t *bleaf, const int32_t *c0,
                     const int32_t *c1, int NB, int pass, int64_t *cnt, int32_t *src, int32_t *opi, int32_t *cone,
                     int64_t ncap, int *err)
{
    int lb = blockIdx.x * blockDim.x + threadIdx.x;
    if (lb >= L.nbox[level]) return;
    int b = L.box0[level] + lb;
    if (b < 0 || b >= NB) { il_bad(err, 1, b, b, level); return; }
    int P = bpar[b];
    if (P < 0 || P >= NB) { il_bad(err, 2, b, P, level); return; }
    int px = bcoord[3 * P], py = bcoord[3 * P + 1], pz = bcoord[3 * P + 2];
    int bx = bcoord[3 * b], by = bcoord[3 * b + 1], bz = bcoord[3 * b + 2];
    int pl = level - 1;
    int64_t k = pass ? cnt[b] : 0;
    int R = L.Roff[level], S = 2 * R + 1;
    for (int o = 0; o < L.noff[pl]; ++o) {
        int oi = L.off0[pl] + o;
        if (oi < 0 || oi >= noffs) { il_bad(err, 3, b, oi, level); return; }
        int3 d = offs[oi];
        int nb = find_box(L, bkey, pl, px + d.x, py + d.y, pz + d.z);
        if (nb >= NB) { il_bad(err, 4, b, nb, level); return; }
        if (nb < 0 || bleaf[nb]) continue;
        int cb = c0[nb], ce = c1[nb];
        if (cb < 0 || ce > NB || cb > ce) { il_bad(err, 5, b, ((long long)cb << 16) ^ ce, level); return; }
        for (int c = cb; c < ce; ++c) {
            int dx = bcoord[3 * c] - bx, dy = bcoord[3 * c + 1] - by, dz = bcoord[3 * c + 2] - bz;
            if (is_near(L, level, dx, dy, dz)) continue;
            if (pass) {
                if (k >= ncap) { il_bad(err, 6, b, k, level); return; }
                src[k] = c;
                opi[k] = ((dx + R) * S + (dy + R)) * S + (dz + R);
                // target cone (direction D -> C) in the low 16 bits, source cone (C -> D) above
                cone[k] = L.hf[level] ? (cone_index(dx, dy, dz, L.nc[level]) |
                                         (cone_index(-dx, -dy, -dz, L.nc[level]) << 16))
                                      : 0;
            }
            ++k;
        }
    }
    if (!pass) cnt[b] = k;
}

__global__ void k_mark_ops(const int32_t *opi, int64_t n, int32_t *used)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) used[opi[i]] = 1;
}

__global__ void k_remap_ops(int32_t *opi, int64_t n, const int32_t *map)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) opi[i] = map[opi[i]];
}

// near-field source ranges of each leaf (pass 0 count, pass 1 fill)
__global__ void k_near(dev_levels L, int nlev, const int3 *offs, int noffs, const uint64_t *bkey,
                       const int32_t *bcoord, const int32_t *bpar, const int32_t *bleaf, const int32_t *blev,
                       const int32_t *bbeg, const int32_t *bend, const int32_t *leaf_box, int nleaf, int NB,
                       int pass, int64_t *cnt, int32_t *rb, int32_t *re, int64_t *ncols, int64_t ncap, int *err)
{
    int li = blockIdx.x * blockDim.x + threadIdx.x;
    if (li >= nleaf) return;
    int B = leaf_box[li];
    if (B < 0 || B >= NB) { il_bad(err, 11, li, B, -1); return; }
    int lB = blev[B];
    if (lB < 0 || lB >= nlev || lB >= 32) { il_bad(err, 12, B, lB, -1); return; }
    int anc[32];
    int a = B;
    for (int l = lB; l >= 0; --l) {
        if (a < 0 || a >= NB) { il_bad(err, 13, B, a, l); return; }
        anc[l] = a;
        a = bpar[a];
    }
    int64_t k = pass ? cnt[li] : 0;
    int64_t cols = 0;
    for (int l = 0; l <= lB; ++l) {
        if (L.hf[l] && l != lB) continue;  // no leaves at high-frequency levels
        int A = anc[l];
        int ax = bcoord[3 * A], ay = bcoord[3 * A + 1], az = bcoord[3 * A + 2];
        for (int o = 0; o < L.noff[l]; ++o) {
            int oi = L.off0[l] + o;
            if (oi < 0 || oi >= noffs) { il_bad(err, 14, B, oi, l); return; }
            int3 d = offs[oi];
            int X = find_box(L, bkey, l, ax + d.x, ay + d.y, az + d.z);
            if (X >= NB) { il_bad(err, 15, B, X, l); return; }
            if (X < 0) continue;
            if (bleaf[X] || l == lB) {
                if (pass) {
                    if (k >= ncap) { il_bad(err, 16, B, k, l); return; }
                    rb[k] = bbeg[X];
                    re[k] = bend[X];
                }
                cols += bend[X] - bbeg[X];
                ++k;
            }
        }
    }
    if (!pass) {
        cnt[li] = k;
        ncols[li] = cols;
    }
}

__global__ void k_near_cols(const int64_t *rptr, const int32_t *rb, const int32_t *re, const int64_t *colptr,
                            int nleaf, int32_t *cols)
{
    int li = blockIdx.x;
    if (li >= nleaf) return;
    int64_t c = colptr[li];
    for (int64_t r = rptr[li]; r < rptr[li + 1]; ++r) {
        int len = re[r] - rb[r];
        for (int t = threadIdx.x; t < len; t += blockDim.x) cols[c + t] = rb[r] + t;
        c += len;
    }
}

__global__ void k_block_sizes(const int32_t *leaf_box, const int32_t *bbeg, const int32_t *bend,
                              const int64_t *ncols, int nleaf, int64_t *sz)
{
    int li = blockIdx.x * blockDim.x + threadIdx.x;
    if (li >= nleaf) return;
    int B = leaf_box[li];
    sz[li] = (int64_t)(bend[B] - bbeg[B]) * ncols[li];
}

}  // namespace

// host helpers shared with precompute.cu
int fda_cone_index_host(double dx, double dy, double dz, int nc) { return cone_index(dx, dy, dz, nc); }

// Symmetry of the cone partition (the rotation invariance of Sec. 4.1.1).
// The 6 nc^2 cones of a level are the images of a few representative cones
// on the +z face (cells whose centre (A, B, nc) has 0 <= A <= B) under the 48
// signed permutations of the axes.  Cone u gets the frame R_u = g_u R_rep(u)
// with g_u mapping the representative's centre to u's centre, and the
// opposite cone gets g = -g_u.  Since the kernel depends on distances only,
// the M2L matrix of offset d, G(R_u eq, d w + R_ub eq) (u, ub the cones of d
// and -d), equals G(R_rep eq, (g_u^T d) w + g_u^T R_ub eq): offsets with the
// same representative, rotated offset and relative source frame share one
// operator.  g is row-major, 9 integers per cone.
void fda_cone_symmetry(int nc, std::vector<int> &rep, std::vector<int> &g)
{
    const int nco = 6 * nc * nc;
    rep.assign(nco, -1);
    g.assign(9 * (size_t)nco, 0);
    auto center = [&](int u, int c[3]) {
        int face = u / (nc * nc), rem = u % (nc * nc);
        int a = rem / nc, b = rem % nc;
        int ax = face / 2, sg = face % 2;
        int o0 = ax == 0 ? 1 : 0, o1 = ax == 2 ? 1 : 2;
        c[ax] = sg ? nc : -nc;
        c[o0] = 2 * a + 1 - nc;
        c[o1] = 2 * b + 1 - nc;
    };
    auto opposite = [&](int u) {
        int face = u / (nc * nc), rem = u % (nc * nc);
        int a = rem / nc, b = rem % nc;
        return (face ^ 1) * nc * nc + (nc - 1 - a) * nc + (nc - 1 - b);
    };
    static const int perms[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
    std::vector<std::array<int, 9>> grp;
    for (const auto &pm : perms)
        for (int sg = 0; sg < 8; ++sg) {
            std::array<int, 9> m{};
            for (int i = 0; i < 3; ++i) m[3 * i + pm[i]] = ((sg >> i) & 1) ? -1 : 1;
            grp.push_back(m);
        }
    std::vector<int> reps;
    for (int u = 0; u < nco; ++u) {
        int c[3];
        center(u, c);
        if (c[2] == nc && c[0] >= 0 && c[1] >= c[0]) reps.push_back(u);
    }
    for (int u = 0; u < nco; ++u) {
        const int v = opposite(u);
        if (rep[v] >= 0) {
            rep[u] = rep[v];
            for (int k = 0; k < 9; ++k) g[9 * (size_t)u + k] = -g[9 * (size_t)v + k];
            continue;
        }
        int cu[3];
        center(u, cu);
        for (size_t r = 0; r < reps.size() && rep[u] < 0; ++r) {
            int cr[3];
            center(reps[r], cr);
            for (const auto &m : grp) {
                bool hit = true;
                for (int i = 0; i < 3 && hit; ++i) hit = m[3 * i] * cr[0] + m[3 * i + 1] * cr[1] + m[3 * i + 2] * cr[2] == cu[i];
                if (hit) {
                    rep[u] = reps[r];
                    for (int k = 0; k < 9; ++k) g[9 * (size_t)u + k] = m[k];
                    break;
                }
            }
        }
        if (rep[u] < 0) fda_fail(FDA_ERR_NUMERIC, "cone without a representative under the cube group");
    }
}

void fda_tree_build(fda_handle *h)
{
    cudaStream_t s = h->stream;
    const int64_t N = h->N;
    const fda_config &cfg = h->cfg;
    h->lambda = 2.0 * FDA_PI / h->k;

    dbuf active, head, scan, ebox, ebox_prev;
    active.alloc(sizeof(int32_t) * N);
    head.alloc(sizeof(int32_t) * N);
    scan.alloc(sizeof(int32_t) * N);
    ebox.alloc(sizeof(int32_t) * N);
    ebox_prev.alloc(sizeof(int32_t) * N);
    {
        std::vector<int32_t> ones(N, 1);
        FDA_CUDA(cudaMemcpy(active.p, ones.data(), sizeof(int32_t) * N, cudaMemcpyHostToDevice));
    }
    // per-level temporaries
    std::vector<dbuf *> lb_beg, lb_end, lb_key, lb_coord, lb_par, lb_leaf;
    int nlev = 0, box0 = 0;
    unsigned g = fda_blocks(N, 256);
    for (int l = 0; l <= MAXD; ++l) {
        int shift = 3 * (MAXD - l);
        k_heads<<<g, 256, 0, s>>>(h->keys.as<uint64_t>(), active.as<int32_t>(), N, shift, head.as<int32_t>());
        FDA_CHECK_LAUNCH();
        int32_t nbox = 0;
        fda_exclusive_scan_i32(head.as<int32_t>(), scan.as<int32_t>(), N, s, &nbox);
        if (nbox == 0) break;
        if (l >= FDA_MAX_LEVELS - 1) fda_fail(FDA_ERR_ARG, "octree deeper than supported (coincident centroids?)");
        level_info &L = h->lev[l];
        L = level_info();
        L.nbox = nbox;
        L.box0 = box0;
        L.w = h->W / (double)(1 << l);
        L.hf = L.w >= cfg.hf_wavelengths * h->lambda ? 1 : 0;
        if (cfg.mode == FDA_MODE_DENSE) L.hf = 0;
        L.nc = L.hf ? std::max(1, 1 << (int)floor(log2(L.w / h->lambda))) : 0;
        L.ncones = L.hf ? 6 * L.nc * L.nc : 1;
        L.rho = L.hf ? std::max(cfg.rho_min, L.w / h->lambda) : 0.0;
        auto mk = [&](size_t bytes) {
            dbuf *b = new dbuf();
            b->alloc(bytes);
            return b;
        };
        lb_beg.push_back(mk(sizeof(int32_t) * nbox));
        lb_end.push_back(mk(sizeof(int32_t) * nbox));
        lb_key.push_back(mk(sizeof(uint64_t) * nbox));
        lb_coord.push_back(mk(sizeof(int32_t) * 3 * nbox));
        lb_par.push_back(mk(sizeof(int32_t) * nbox));
        lb_leaf.push_back(mk(sizeof(int32_t) * nbox));
        int parent_box0 = l > 0 ? h->lev[l - 1].box0 : 0;
        k_boxes<<<g, 256, 0, s>>>(h->keys.as<uint64_t>(), active.as<int32_t>(), head.as<int32_t>(),
                                  scan.as<int32_t>(), N, shift, l, parent_box0, ebox_prev.as<int32_t>(),
                                  ebox.as<int32_t>(), lb_beg[l]->as<int32_t>(), lb_end[l]->as<int32_t>(),
                                  lb_key[l]->as<uint64_t>(), lb_coord[l]->as<int32_t>(), lb_par[l]->as<int32_t>());
        FDA_CHECK_LAUNCH();
        int can_leaf = (!L.hf) || cfg.mode == FDA_MODE_DENSE;
        int force = l == MAXD;
        if (cfg.mode == FDA_MODE_DENSE) force = 1;  // dense mode: the root is the only leaf
        k_leaf_flags<<<fda_blocks(nbox, 256), 256, 0, s>>>(lb_beg[l]->as<int32_t>(), lb_end[l]->as<int32_t>(), nbox,
                                                           can_leaf, cfg.leaf_max, force, lb_leaf[l]->as<int32_t>());
        FDA_CHECK_LAUNCH();
        k_deactivate<<<g, 256, 0, s>>>(active.as<int32_t>(), ebox.as<int32_t>(), lb_leaf[l]->as<int32_t>(), N);
        FDA_CHECK_LAUNCH();
        std::swap(ebox.p, ebox_prev.p);
        box0 += nbox;
        nlev = l + 1;
    }
    h->nlev = nlev;
    h->nbox_total = box0;
    const int NB = box0;
    h->box_begin.alloc(sizeof(int32_t) * NB);
    h->box_end.alloc(sizeof(int32_t) * NB);
    h->box_key.alloc(sizeof(uint64_t) * NB);
    h->box_coord.alloc(sizeof(int32_t) * 3 * NB);
    h->box_parent.alloc(sizeof(int32_t) * NB);
    h->box_leaf.alloc(sizeof(int32_t) * NB);
    h->box_level.alloc(sizeof(int32_t) * NB);
    h->box_child0.alloc(sizeof(int32_t) * NB);
    h->box_child1.alloc(sizeof(int32_t) * NB);
    FDA_CUDA(cudaMemsetAsync(h->box_child0.p, 0, sizeof(int32_t) * NB, s));
    FDA_CUDA(cudaMemsetAsync(h->box_child1.p, 0, sizeof(int32_t) * NB, s));
    std::vector<int32_t> hlev(NB);
    for (int l = 0; l < nlev; ++l) {
        const level_info &L = h->lev[l];
        size_t o = L.box0, n = L.nbox;
        FDA_CUDA(cudaMemcpyAsync(h->box_begin.as<int32_t>() + o, lb_beg[l]->p, 4 * n, cudaMemcpyDeviceToDevice, s));
        FDA_CUDA(cudaMemcpyAsync(h->box_end.as<int32_t>() + o, lb_end[l]->p, 4 * n, cudaMemcpyDeviceToDevice, s));
        FDA_CUDA(cudaMemcpyAsync(h->box_key.as<uint64_t>() + o, lb_key[l]->p, 8 * n, cudaMemcpyDeviceToDevice, s));
        FDA_CUDA(cudaMemcpyAsync(h->box_coord.as<int32_t>() + 3 * o, lb_coord[l]->p, 12 * n,
                                 cudaMemcpyDeviceToDevice, s));
        FDA_CUDA(cudaMemcpyAsync(h->box_parent.as<int32_t>() + o, lb_par[l]->p, 4 * n, cudaMemcpyDeviceToDevice, s));
        FDA_CUDA(cudaMemcpyAsync(h->box_leaf.as<int32_t>() + o, lb_leaf[l]->p, 4 * n, cudaMemcpyDeviceToDevice, s));
        for (size_t b = 0; b < n; ++b) hlev[o + b] = l;
    }
    FDA_CUDA(cudaMemcpyAsync(h->box_level.p, hlev.data(), 4 * (size_t)NB, cudaMemcpyHostToDevice, s));
    for (int l = 1; l < nlev; ++l) {
        k_children<<<fda_blocks(h->lev[l].nbox, 256), 256, 0, s>>>(h->box_parent.as<int32_t>(), h->lev[l].nbox,
                                                                     h->lev[l].box0, h->box_child0.as<int32_t>(),
                                                                     h->box_child1.as<int32_t>());
        FDA_CHECK_LAUNCH();
    }
    FDA_CUDA(cudaStreamSynchronize(s));
    for (auto *v : {&lb_beg, &lb_end, &lb_key, &lb_coord, &lb_par, &lb_leaf})
        for (dbuf *b : *v) delete b;

    // leaves
    std::vector<int32_t> hleaf(NB);
    FDA_CUDA(cudaMemcpy(hleaf.data(), h->box_leaf.p, 4 * (size_t)NB, cudaMemcpyDeviceToHost));
    std::vector<int32_t> leaf_box, leaf_of_box(NB, -1);
    h->h_leaf_level.clear();
    for (int b = 0; b < NB; ++b)
        if (hleaf[b]) {
            leaf_of_box[b] = (int32_t)leaf_box.size();
            leaf_box.push_back(b);
            h->h_leaf_level.push_back(hlev[b]);
            h->lev[hlev[b]].nleaf++;
        }
    h->nleaf = (int)leaf_box.size();
    {
        std::vector<int32_t> hb(NB), he(NB);
        FDA_CUDA(cudaMemcpy(hb.data(), h->box_begin.p, 4 * (size_t)NB, cudaMemcpyDeviceToHost));
        FDA_CUDA(cudaMemcpy(he.data(), h->box_end.p, 4 * (size_t)NB, cudaMemcpyDeviceToHost));
        int mx = 0;
        for (int b : leaf_box) mx = std::max(mx, he[b] - hb[b]);
        h->max_leaf_rows = mx;
        if (cfg.mode != FDA_MODE_DENSE && mx > 64)
            fda_fail(FDA_ERR_ARG, "a leaf holds more than 64 elements (coincident centroids)");
    }
    h->leaf_box.alloc(4 * leaf_box.size());
    FDA_CUDA(cudaMemcpy(h->leaf_box.p, leaf_box.data(), 4 * leaf_box.size(), cudaMemcpyHostToDevice));
    h->leaf_of_box.alloc(4 * (size_t)NB);
    FDA_CUDA(cudaMemcpy(h->leaf_of_box.p, leaf_of_box.data(), 4 * (size_t)NB, cudaMemcpyHostToDevice));

    // near-offset tables per level
    dev_levels DL;
    std::vector<int3> offs;
    for (int l = 0; l < nlev; ++l) {
        level_info &L = h->lev[l];
        DL.box0[l] = L.box0;
        DL.nbox[l] = L.nbox;
        DL.hf[l] = L.hf;
        DL.rho2[l] = L.rho * L.rho;
        DL.nc[l] = L.nc;
        DL.off0[l] = (int)offs.size();
        int R = L.hf ? (int)ceil(L.rho) + 1 : 1;
        for (int dx = -R; dx <= R; ++dx)
            for (int dy = -R; dy <= R; ++dy)
                for (int dz = -R; dz <= R; ++dz) {
                    int m = std::max(abs(dx), std::max(abs(dy), abs(dz)));
                    bool nr = m <= 1 || (L.hf && (double)(dx * dx + dy * dy + dz * dz) < L.rho * L.rho);
                    if (nr) offs.push_back(make_int3(dx, dy, dz));
                }
        DL.noff[l] = (int)offs.size() - DL.off0[l];
        int Rp = 1;
        if (l > 0 && h->lev[l - 1].hf) Rp = (int)ceil(h->lev[l - 1].rho) + 1;
        L.R_off = 2 * Rp + 1;
        DL.Roff[l] = L.R_off;
    }
    dbuf doffs;
    doffs.alloc(sizeof(int3) * offs.size());
    FDA_CUDA(cudaMemcpy(doffs.p, offs.data(), sizeof(int3) * offs.size(), cudaMemcpyHostToDevice));

    // interaction lists (CSR over all boxes)
    dbuf cnt, ilerr;
    cnt.alloc(sizeof(int64_t) * (NB + 1));
    ilerr.alloc(sizeof(int) * 4);
    FDA_CUDA(cudaMemsetAsync(cnt.p, 0, sizeof(int64_t) * (NB + 1), s));
    FDA_CUDA(cudaMemsetAsync(ilerr.p, 0, sizeof(int) * 4, s));
    const int noffs = (int)offs.size();
    auto check_il = [&](const char *what) {
        int e[4];
        FDA_CUDA(cudaMemcpy(e, ilerr.p, sizeof(e), cudaMemcpyDeviceToHost));
        if (e[0])
            fda_fail(FDA_ERR_NUMERIC, std::string("internal list error in ") + what + ": code " + std::to_string(e[0]) +
                                          " box " + std::to_string(e[1]) + " value " + std::to_string(e[2]) +
                                          " level " + std::to_string(e[3]));
    };
    if (cfg.mode != FDA_MODE_DENSE)
        for (int l = 1; l < nlev; ++l)
            k_il<<<fda_blocks(h->lev[l].nbox, 128), 128, 0, s>>>(
                DL, l, doffs.as<int3>(), noffs, h->box_key.as<uint64_t>(), h->box_coord.as<int32_t>(),
                h->box_parent.as<int32_t>(), h->box_leaf.as<int32_t>(), h->box_child0.as<int32_t>(),
                h->box_child1.as<int32_t>(), NB, 0, cnt.as<int64_t>(), nullptr, nullptr, nullptr, 0,
                ilerr.as<int>());
    FDA_CHECK_LAUNCH();
    check_il("interaction-list count");
    h->il_ptr.alloc(sizeof(int64_t) * (NB + 1));
    int64_t nil = 0;
    fda_exclusive_scan_i64(cnt.as<int64_t>(), h->il_ptr.as<int64_t>(), NB + 1, s, &nil);
    h->n_il_total = nil;
    h->il_src.alloc(sizeof(int32_t) * std::max<int64_t>(nil, 1));
    h->il_op.alloc(sizeof(int32_t) * std::max<int64_t>(nil, 1));
    h->il_cone.alloc(sizeof(int32_t) * std::max<int64_t>(nil, 1));
    if (cfg.mode != FDA_MODE_DENSE)
        for (int l = 1; l < nlev; ++l)
            k_il<<<fda_blocks(h->lev[l].nbox, 128), 128, 0, s>>>(
                DL, l, doffs.as<int3>(), noffs, h->box_key.as<uint64_t>(), h->box_coord.as<int32_t>(),
                h->box_parent.as<int32_t>(), h->box_leaf.as<int32_t>(), h->box_child0.as<int32_t>(),
                h->box_child1.as<int32_t>(), NB, 1, h->il_ptr.as<int64_t>(), h->il_src.as<int32_t>(),
                h->il_op.as<int32_t>(), h->il_cone.as<int32_t>(), nil, ilerr.as<int>());
    FDA_CHECK_LAUNCH();
    check_il("interaction-list fill");
    // distinct operators per level: mark the dense offset table, compact on the host
    std::vector<int64_t> hptr(NB + 1);
    FDA_CUDA(cudaMemcpyAsync(hptr.data(), h->il_ptr.p, 8 * (size_t)(NB + 1), cudaMemcpyDeviceToHost, s));
    FDA_CUDA(cudaStreamSynchronize(s));
    h->lev_lo = -1;
    for (int l = 1; l < nlev; ++l) {
        level_info &L = h->lev[l];
        int64_t a = hptr[L.box0], b = hptr[L.box0 + L.nbox];
        L.n_il = (int)(b - a);
        if (L.n_il == 0) continue;
        if (h->lev_lo < 0) h->lev_lo = l;
        int S = 2 * L.R_off + 1;
        dbuf used;
        used.alloc(sizeof(int32_t) * S * S * S);
        FDA_CUDA(cudaMemsetAsync(used.p, 0, sizeof(int32_t) * S * S * S, s));
        k_mark_ops<<<fda_blocks(b - a, 256), 256, 0, s>>>(h->il_op.as<int32_t>() + a, b - a, used.as<int32_t>());
        FDA_CHECK_LAUNCH();
        std::vector<int32_t> hu(S * S * S);
        FDA_CUDA(cudaMemcpyAsync(hu.data(), used.p, 4 * hu.size(), cudaMemcpyDeviceToHost, s));
        FDA_CUDA(cudaStreamSynchronize(s));
        int nops = 0;
        h->h_ops[l].clear();
        // high frequency: offsets equal under the cone symmetry share an operator
        std::vector<int> crep, cg;
        std::map<std::array<int, 6>, int> key_op;
        if (L.hf) fda_cone_symmetry(L.nc, crep, cg);
        for (size_t t = 0; t < hu.size(); ++t) {
            if (!hu[t]) {
                hu[t] = -1;
                continue;
            }
            int dz = (int)(t % S) - L.R_off, dy = (int)((t / S) % S) - L.R_off, dx = (int)(t / S / S) - L.R_off;
            if (L.hf) {
                const int d[3] = {dx, dy, dz};
                const int u = cone_index(dx, dy, dz, L.nc), ub = cone_index(-dx, -dy, -dz, L.nc);
                const int *gu = &cg[9 * (size_t)u], *gb = &cg[9 * (size_t)ub];
                std::array<int, 6> key{crep[u], 0, 0, 0, 0, crep[ub]};
                for (int i = 0; i < 3; ++i) key[1 + i] = gu[i] * d[0] + gu[3 + i] * d[1] + gu[6 + i] * d[2];
                int enc = 0;  // g_u^T g_ub, entries in {-1, 0, 1}, base 3
                for (int i = 0; i < 3; ++i)
                    for (int j = 0; j < 3; ++j)
                        enc = 3 * enc + 1 + gu[i] * gb[j] + gu[3 + i] * gb[3 + j] + gu[6 + i] * gb[6 + j];
                key[4] = enc;
                auto it = key_op.find(key);
                if (it != key_op.end()) {
                    hu[t] = it->second;
                    continue;
                }
                key_op.emplace(key, nops);
            }
            hu[t] = nops++;
            h->h_ops[l].push_back(make_int3(dx, dy, dz));
        }
        L.n_ops = nops;
        FDA_CUDA(cudaMemcpy(used.p, hu.data(), 4 * hu.size(), cudaMemcpyHostToDevice));
        k_remap_ops<<<fda_blocks(b - a, 256), 256, 0, s>>>(h->il_op.as<int32_t>() + a, b - a, used.as<int32_t>());
        FDA_CHECK_LAUNCH();
        FDA_CUDA(cudaStreamSynchronize(s));
    }
    // densities are needed from lev_lo down to the deepest level
    for (int l = 0; l < nlev; ++l) h->lev[l].active = (h->lev_lo >= 0 && l >= h->lev_lo) ? 1 : 0;

    // near-field lists
    const int NL = h->nleaf;
    dbuf ncnt, ncols;
    ncnt.alloc(sizeof(int64_t) * (NL + 1));
    ncols.alloc(sizeof(int64_t) * (NL + 1));
    FDA_CUDA(cudaMemsetAsync(ncnt.p, 0, sizeof(int64_t) * (NL + 1), s));
    FDA_CUDA(cudaMemsetAsync(ncols.p, 0, sizeof(int64_t) * (NL + 1), s));
    if (cfg.mode == FDA_MODE_DENSE) {
        // single leaf (the root) with the whole element range as its near field
        int64_t one = 1;
        FDA_CUDA(cudaMemcpy(ncnt.p, &one, 8, cudaMemcpyHostToDevice));
        FDA_CUDA(cudaMemcpy(ncols.p, &N, 8, cudaMemcpyHostToDevice));
    } else {
        k_near<<<fda_blocks(NL, 128), 128, 0, s>>>(DL, nlev, doffs.as<int3>(), noffs, h->box_key.as<uint64_t>(),
                                                   h->box_coord.as<int32_t>(), h->box_parent.as<int32_t>(),
                                                   h->box_leaf.as<int32_t>(), h->box_level.as<int32_t>(),
                                                   h->box_begin.as<int32_t>(), h->box_end.as<int32_t>(),
                                                   h->leaf_box.as<int32_t>(), NL, NB, 0, ncnt.as<int64_t>(), nullptr,
                                                   nullptr, ncols.as<int64_t>(), 0, ilerr.as<int>());
        FDA_CHECK_LAUNCH();
        check_il("near-field count");
    }
    h->nr_ptr.alloc(sizeof(int64_t) * (NL + 1));
    int64_t nranges = 0;
    fda_exclusive_scan_i64(ncnt.as<int64_t>(), h->nr_ptr.as<int64_t>(), NL + 1, s, &nranges);
    h->nr_begin.alloc(sizeof(int32_t) * std::max<int64_t>(nranges, 1));
    h->nr_end.alloc(sizeof(int32_t) * std::max<int64_t>(nranges, 1));
    if (cfg.mode == FDA_MODE_DENSE) {
        int32_t zb = 0, ze = (int32_t)N;
        FDA_CUDA(cudaMemcpy(h->nr_begin.p, &zb, 4, cudaMemcpyHostToDevice));
        FDA_CUDA(cudaMemcpy(h->nr_end.p, &ze, 4, cudaMemcpyHostToDevice));
    } else {
        k_near<<<fda_blocks(NL, 128), 128, 0, s>>>(DL, nlev, doffs.as<int3>(), noffs, h->box_key.as<uint64_t>(),
                                                   h->box_coord.as<int32_t>(), h->box_parent.as<int32_t>(),
                                                   h->box_leaf.as<int32_t>(), h->box_level.as<int32_t>(),
                                                   h->box_begin.as<int32_t>(), h->box_end.as<int32_t>(),
                                                   h->leaf_box.as<int32_t>(), NL, NB, 1, h->nr_ptr.as<int64_t>(),
                                                   h->nr_begin.as<int32_t>(), h->nr_end.as<int32_t>(), nullptr,
                                                   nranges, ilerr.as<int>());
        FDA_CHECK_LAUNCH();
        check_il("near-field fill");
    }
    h->nf_colptr.alloc(sizeof(int64_t) * (NL + 1));
    fda_exclusive_scan_i64(ncols.as<int64_t>(), h->nf_colptr.as<int64_t>(), NL + 1, s, &h->ncols_total);
    {
        // widest leaf row (columns), for the near-field kernel's shared-memory staging
        std::vector<int64_t> cp(NL + 1);
        FDA_CUDA(cudaMemcpyAsync(cp.data(), h->nf_colptr.p, 8 * (size_t)(NL + 1), cudaMemcpyDeviceToHost, s));
        FDA_CUDA(cudaStreamSynchronize(s));
        int64_t mx = 0;
        for (int li = 0; li < NL; ++li) mx = std::max(mx, cp[li + 1] - cp[li]);
        h->max_near_cols = mx;
    }
    h->nf_cols.alloc(sizeof(int32_t) * std::max<int64_t>(h->ncols_total, 1));
    k_near_cols<<<NL, 128, 0, s>>>(h->nr_ptr.as<int64_t>(), h->nr_begin.as<int32_t>(), h->nr_end.as<int32_t>(),
                                   h->nf_colptr.as<int64_t>(), NL, h->nf_cols.as<int32_t>());
    FDA_CHECK_LAUNCH();
    dbuf bsz;
    bsz.alloc(sizeof(int64_t) * (NL + 1));
    FDA_CUDA(cudaMemsetAsync(bsz.p, 0, sizeof(int64_t) * (NL + 1), s));
    k_block_sizes<<<fda_blocks(NL, 128), 128, 0, s>>>(h->leaf_box.as<int32_t>(), h->box_begin.as<int32_t>(),
                                                      h->box_end.as<int32_t>(), ncols.as<int64_t>(), NL,
                                                      bsz.as<int64_t>());
    FDA_CHECK_LAUNCH();
    h->nf_off.alloc(sizeof(int64_t) * (NL + 1));
    fda_exclusive_scan_i64(bsz.as<int64_t>(), h->nf_off.as<int64_t>(), NL + 1, s, &h->nnz_near);
    FDA_CUDA(cudaStreamSynchronize(s));
}
