// Fields off the surface from the boundary solution: Green's representation
// of Eq. cbie in the acoustic domain (c = 1, n into the body),
//   u(x) = u_inc(x) + int G(x, y) q(y) dy - int dG/dn_y(x, y) u(y) dy,
// and its large-|x| limit, the far-field pattern F of u_sc ~ e^{ik|x|}/|x| F,
//   F(xh) = (1/(4 pi)) int [ q(y) + ik (xh . n_y) u(y) ] e^{-ik xh . y} dy,
// each element integral by the six-point rule of the regular near field.
// Direct summation over all elements for every target (no fast algorithm):
// N x M x 6 FP64 kernel evaluations, sincos-bound.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <utility>
#include <vector>

#include "fda_internal.cuh"
#include "tree_util.cuh"

namespace {

constexpr int FT = 256;  // threads per block
constexpr int FD = 4;    // targets per block (element data loaded once for all of them)

// One block: FD targets x one slice of the elements; partial sums reduced in
// the block and added to out[target] with FP64 atomics.  far = 1: targets
// are unit directions (pattern); far = 0: points (scattered field).
__global__ void __launch_bounds__(FT) k_field(const double *qpt, const double *qw, const double *nrm,
                                              const c64d *u, const c64d *q, int64_t n, const double *tgt,
                                              int64_t ntgt, double k, int far, int64_t per_block, c64d *out)
{
    const int64_t t0 = (int64_t)blockIdx.x * FD;
    const int64_t e0 = (int64_t)blockIdx.y * per_block;
    const int64_t e1 = e0 + per_block < n ? e0 + per_block : n;
    double x[FD][3];
    for (int d = 0; d < FD; ++d)
        for (int c = 0; c < 3; ++c) x[d][c] = t0 + d < ntgt ? tgt[3 * (t0 + d) + c] : 0.0;
    double are[FD], aim[FD];
    for (int d = 0; d < FD; ++d) are[d] = aim[d] = 0.0;
    for (int64_t j = e0 + threadIdx.x; j < e1; j += FT) {
        const double *ny = nrm + 3 * j;
        const c64d uj = u[j];
        const c64d qj = q ? q[j] : c64d(0.0, 0.0);
        for (int g = 0; g < 6; ++g) {
            const double *y = qpt + 18 * j + 3 * g;
            const double w = qw[6 * j + g];
            for (int d = 0; d < FD; ++d) {
                double sn, cs;
                if (far) {
                    // w e^{-ik xh.y} (q + ik (xh.n) u)
                    double xn = x[d][0] * ny[0] + x[d][1] * ny[1] + x[d][2] * ny[2];
                    double xy = x[d][0] * y[0] + x[d][1] * y[1] + x[d][2] * y[2];
                    sincos(k * xy, &sn, &cs);
                    double fre = qj.re - k * xn * uj.im, fim = qj.im + k * xn * uj.re;
                    are[d] += w * (cs * fre + sn * fim);
                    aim[d] += w * (cs * fim - sn * fre);
                } else {
                    // w [G q - dG/dn_y u], r = x - y
                    double r0 = x[d][0] - y[0], r1 = x[d][1] - y[1], r2 = x[d][2] - y[2];
                    double R2 = r0 * r0 + r1 * r1 + r2 * r2, R = sqrt(R2);
                    sincos(k * R, &sn, &cs);
                    double g = w / (4.0 * FDA_PI * R);
                    // dG/dn_y = e^{ikR}(1 - ikR)(r.n_y)/(4 pi R^3)
                    double f = g * (r0 * ny[0] + r1 * ny[1] + r2 * ny[2]) / R2;
                    double dre = f * (cs + k * R * sn), dim = f * (sn - k * R * cs);
                    double gre = g * cs, gim = g * sn;
                    are[d] += gre * qj.re - gim * qj.im - (dre * uj.re - dim * uj.im);
                    aim[d] += gre * qj.im + gim * qj.re - (dre * uj.im + dim * uj.re);
                }
            }
        }
    }
    __shared__ double red[FT / 32][FD][2];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int d = 0; d < FD; ++d) {
        double a = are[d], b = aim[d];
        for (int o = 16; o > 0; o >>= 1) {
            a += __shfl_xor_sync(0xffffffffu, a, o);
            b += __shfl_xor_sync(0xffffffffu, b, o);
        }
        if (lane == 0) {
            red[wid][d][0] = a;
            red[wid][d][1] = b;
        }
    }
    __syncthreads();
    if (threadIdx.x < FD && t0 + threadIdx.x < ntgt) {
        double a = 0.0, b = 0.0;
        for (int w = 0; w < FT / 32; ++w) {
            a += red[w][threadIdx.x][0];
            b += red[w][threadIdx.x][1];
        }
        const double s = far ? 1.0 / (4.0 * FDA_PI) : 1.0;
        atomicAdd(&out[t0 + threadIdx.x].re, s * a);
        atomicAdd(&out[t0 + threadIdx.x].im, s * b);
    }
}

// Far-field pattern from the outgoing densities of the boxes of one level
// (the level's equivalent sources phi = V q~ reproduce each box's field
// outside its check region, so also its limit at infinity):
//   F(xh) += (1/(4 pi)) sum_B e^{-ik xh.c_B} sum_t w_t(xh) q~_{B,u,t},
//   w_t(xh) = sum_e e^{-ik (R_u^T xh).y_e} V_{e,t},
// with u the cone of direction xh at a high-frequency level (equivalent
// points y_e in the cone's frame R_u), u = 0 at a low-frequency level.  One
// block per direction; w in shared memory; a warp per box.
__global__ void __launch_bounds__(FT) k_pattern_boxes(const double *dirs, int ndir, const c64d *qd, int box0,
                                                      int nbox, int ncones, int nc, int hf, int T, const double *eq,
                                                      int neq, const double *rot, const c64d *V,
                                                      const int32_t *coord, double lo0, double lo1, double lo2,
                                                      double w, double k, double sign, c64d *out)
{
    extern __shared__ c64d wsm[];  // [T]
    __shared__ double red[FT / 32][2];
    const int d = blockIdx.x;
    if (d >= ndir) return;
    const double x0 = dirs[3 * d], x1 = dirs[3 * d + 1], x2 = dirs[3 * d + 2];
    int u = 0;
    double r0 = x0, r1 = x1, r2 = x2;  // R_u^T xh
    if (hf) {
        // cone of the direction: face of the largest component, cell of the other two
        const double xd[3] = {x0, x1, x2}, ad[3] = {fabs(x0), fabs(x1), fabs(x2)};
        int ax = 0;
        if (ad[1] > ad[ax]) ax = 1;
        if (ad[2] > ad[ax]) ax = 2;
        const int sg = xd[ax] > 0 ? 1 : 0;
        const int o0 = ax == 0 ? 1 : 0, o1 = ax == 2 ? 1 : 2;
        const double am = ad[ax];
        int ca = (int)floor((xd[o0] / am + 1.0) * 0.5 * nc), cb = (int)floor((xd[o1] / am + 1.0) * 0.5 * nc);
        ca = ca < 0 ? 0 : (ca > nc - 1 ? nc - 1 : ca);
        cb = cb < 0 ? 0 : (cb > nc - 1 ? nc - 1 : cb);
        u = (2 * ax + sg) * nc * nc + ca * nc + cb;
        const double *R = rot + 9 * u;  // row-major, world = R * frame
        r0 = R[0] * x0 + R[3] * x1 + R[6] * x2;
        r1 = R[1] * x0 + R[4] * x1 + R[7] * x2;
        r2 = R[2] * x0 + R[5] * x1 + R[8] * x2;
    }
    for (int t = threadIdx.x; t < T; t += FT) {
        c64d acc;
        for (int e = 0; e < neq; ++e) {
            double sn, cs;
            sincos(-k * (r0 * eq[3 * e] + r1 * eq[3 * e + 1] + r2 * eq[3 * e + 2]), &sn, &cs);
            cfma(acc, c64d(cs, sn), V[e + (int64_t)t * neq]);
        }
        wsm[t] = acc;
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    double are = 0.0, aim = 0.0;
    for (int b = warp; b < nbox; b += FT / 32) {
        const c64d *qb = qd + ((int64_t)b * ncones + u) * T;
        c64d acc;
        for (int t = lane; t < T; t += 32) cfma(acc, wsm[t], qb[t]);
        const int32_t *c = coord + 3 * (int64_t)(box0 + b);
        const double cx = lo0 + (c[0] + 0.5) * w, cy = lo1 + (c[1] + 0.5) * w, cz = lo2 + (c[2] + 0.5) * w;
        double sn, cs;
        sincos(-k * (x0 * cx + x1 * cy + x2 * cz), &sn, &cs);
        are += cs * acc.re - sn * acc.im;
        aim += cs * acc.im + sn * acc.re;
    }
    for (int o = 16; o > 0; o >>= 1) {
        are += __shfl_xor_sync(0xffffffffu, are, o);
        aim += __shfl_xor_sync(0xffffffffu, aim, o);
    }
    if (lane == 0) {
        red[warp][0] = are;
        red[warp][1] = aim;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int i = 0; i < FT / 32; ++i) {
            a += red[i][0];
            b += red[i][1];
        }
        const double f = sign / (4.0 * FDA_PI);
        out[d].re += f * a;
        out[d].im += f * b;
    }
}

__global__ void k_negate(c64d *x, int64_t n)
{
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t < n) x[t] = c64d(-x[t].re, -x[t].im);
}

// ---- scattered field at points through the fast algorithm
//
// A target x is placed in the deepest box A of the tree whose cube contains
// it.  If A is a low-frequency box with local densities, x is treated as one
// more collocation point of A: its field from the sources that A's local
// density covers (the interaction lists of A and its ancestors) is the L2T
// of A's density at x, sum_m G(x, y_m) psi_m with psi = conj(U) S^-1 p~_A on
// A's equivalent points y_m (as the L2T operators of the leaves, Eq. l2t,
// with the value of G in place of the Burton-Miller kernel); what remains is
// A's near field as if A were a leaf (leaves near A's ancestors and every
// box near A).  Otherwise (x outside every low-frequency box) nothing is
// covered by local densities and the whole tree is what remains.  What
// remains is walked top-down: a box whose cube is not near x's cube of its
// level (the interaction-list test of the tree, directional at a
// high-frequency level) contributes through its equivalent sources,
// sum_e G(x, c + R_u y_e) phi_e with phi = V q~ of the cone u containing the
// direction towards x (the evaluation behind M2L); a near leaf is summed
// directly by the six-point rule; a near box with children is opened.
constexpr int FF = 128;         // threads per target
constexpr int FSET = 2048;      // boxes of one level near a target (capacity)
constexpr int FCH = 128;        // near boxes opened per round
constexpr int FLIST = 8 * FCH;  // equivalent-source and direct lists of a round

struct ff_level {
    int box0, nbox, T, ncones, nc, hf, n_eq, n_chk, far;  // far: outgoing densities at this level
    double w, rho2;
    const void *phi;    // [nbox][ncones][n_eq] equivalent sources V q~ (in the arithmetic type)
    const c64d *p;      // [nbox][T] local densities (low frequency; null elsewhere)
    const double *eq;   // [n_eq][3] equivalent points, box-relative (cone frame at high frequency)
    const double *chk;  // [n_chk][3] the L2T's equivalent points (the upward check points)
    const double *rot;  // [ncones][9] row-major cone rotations (high frequency)
    const c64d *U;      // [T][n_chk] left singular vectors of the level
    const double *sig;  // [T]
};

struct ff_tree {
    ff_level L[FDA_MAX_LEVELS];
    int nlev, lev_lo, max_chk;
    double lo[3];
    const uint64_t *key;
    const int32_t *coord, *leaf, *c0, *c1, *bbeg, *bend;
};

__device__ inline int ff_cell(double x, double lo, double w)
{
    double c = floor((x - lo) / w);
    c = c < -268435456.0 ? -268435456.0 : (c > 268435456.0 ? 268435456.0 : c);
    return (int)c;
}

__device__ inline bool ff_near(const ff_level &L, int dx, int dy, int dz)
{
    const int m = max(abs(dx), max(abs(dy), abs(dz)));
    if (m <= 1) return true;
    if (L.hf) return (double)dx * dx + (double)dy * dy + (double)dz * dz < L.rho2;
    return false;
}

__device__ inline void ff_sincos(double a, double *sn, double *cs) { sincos(a, sn, cs); }
__device__ inline void ff_sincos(float a, float *sn, float *cs) { sincosf(a, sn, cs); }

// a += G(x, y) b, G = e^{ikR}/(4 pi R), in the arithmetic type F (the
// difference x - y in FP64)
template <typename F>
__device__ inline void ff_acc_g(F &are, F &aim, const double *x, double y0, double y1, double y2, F k, cx<F> b)
{
    const F r0 = (F)(x[0] - y0), r1 = (F)(x[1] - y1), r2 = (F)(x[2] - y2);
    const F R = sqrt(r0 * r0 + r1 * r1 + r2 * r2);
    F sn, cs;
    ff_sincos(k * R, &sn, &cs);
    const F g = (F)1 / ((F)(4.0 * FDA_PI) * R);
    const F gre = g * cs, gim = g * sn;
    are += gre * b.re - gim * b.im;
    aim += gre * b.im + gim * b.re;
}

// one warp: the six-point sums of the elements [j0, j1) of a leaf,
// w [G q + dG/dn_y un] with un = -u
template <typename F>
__device__ inline void ff_direct(int j0, int j1, const double *qpt, const double *qw, const double *nrm,
                                 const c64d *un, const c64d *q, const double *x, F k, int lane, F &are, F &aim)
{
    for (int t = j0 * 6 + lane; t < j1 * 6; t += 32) {
        const int j = t / 6, g = t - 6 * (t / 6);
        const double *y = qpt + 18 * (int64_t)j + 3 * g, *ny = nrm + 3 * (int64_t)j;
        const F w = (F)qw[6 * (int64_t)j + g];
        const F r0 = (F)(x[0] - y[0]), r1 = (F)(x[1] - y[1]), r2 = (F)(x[2] - y[2]);
        const F R2 = r0 * r0 + r1 * r1 + r2 * r2, R = sqrt(R2);
        F sn, cs;
        ff_sincos(k * R, &sn, &cs);
        const F gw = w / ((F)(4.0 * FDA_PI) * R);
        // dG/dn_y = e^{ikR}(1 - ikR)(r.n_y)/(4 pi R^3)
        const F f = gw * (r0 * (F)ny[0] + r1 * (F)ny[1] + r2 * (F)ny[2]) / R2;
        const F dre = f * (cs + k * R * sn), dim = f * (sn - k * R * cs);
        const F gre = gw * cs, gim = gw * sn;
        const c64d u64 = un[j], q64 = q ? q[j] : c64d(0.0, 0.0);
        const cx<F> uj((F)u64.re, (F)u64.im), qj((F)q64.re, (F)q64.im);
        are += gre * qj.re - gim * qj.im + dre * uj.re - dim * uj.im;
        aim += gre * qj.im + gim * qj.re + dre * uj.im + dim * uj.re;
    }
}

// one warp: box b of level l through its equivalent sources of cone u
template <typename F>
__device__ inline void ff_m2t(const ff_tree &t, int l, int b, int u, const double *x, F k, int lane, F &are, F &aim)
{
    const ff_level &L = t.L[l];
    const cx<F> *phi = reinterpret_cast<const cx<F> *>(L.phi) + ((int64_t)(b - L.box0) * L.ncones + u) * L.n_eq;
    const int32_t *cb = t.coord + 3 * (int64_t)b;
    const double c0 = t.lo[0] + (cb[0] + 0.5) * L.w, c1 = t.lo[1] + (cb[1] + 0.5) * L.w,
                 c2 = t.lo[2] + (cb[2] + 0.5) * L.w;
    const double *R = L.hf ? L.rot + 9 * u : nullptr;
    for (int e = lane; e < L.n_eq; e += 32) {
        const double *f = L.eq + 3 * e;
        double y0 = f[0], y1 = f[1], y2 = f[2];
        if (R) {
            y0 = R[0] * f[0] + R[1] * f[1] + R[2] * f[2];
            y1 = R[3] * f[0] + R[4] * f[1] + R[5] * f[2];
            y2 = R[6] * f[0] + R[7] * f[1] + R[8] * f[2];
        }
        ff_acc_g<F>(are, aim, x, c0 + y0, c1 + y1, c2 + y2, k, phi[e]);
    }
}

// One CTA per target.  err[0] records a near set above its capacity (the
// target's value is then left at NaN and the host reports the error).
template <typename F>
__global__ void __launch_bounds__(FF) k_field_fast(ff_tree t, const double *qpt, const double *qw,
                                                   const double *nrm, const c64d *un, const c64d *q,
                                                   const double *tgt, int64_t ntgt, double kd, int *err, c64d *out)
{
    extern __shared__ __align__(16) uint8_t psi_raw[];
    cx<F> *psi = reinterpret_cast<cx<F> *>(psi_raw);  // [max_chk]
    const F k = (F)kd;
    __shared__ int sset[2][FSET];
    __shared__ int mlist[FLIST], mcone[FLIST], dlist[FLIST];
    __shared__ int ns, nn, nm, nd, overflow, lA, A;
    __shared__ int anc[FDA_MAX_LEVELS];
    __shared__ double red[FF / 32][2];
    const int64_t ti = blockIdx.x;
    if (ti >= ntgt) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const double x[3] = {tgt[3 * ti], tgt[3 * ti + 1], tgt[3 * ti + 2]};
    F are = 0, aim = 0;
    // the chain of boxes containing x, down to a leaf or an empty cube
    if (threadIdx.x == 0) {
        A = -1;
        lA = -1;
        overflow = 0;
        for (int l = 0; l < t.nlev; ++l) {
            const ff_level &L = t.L[l];
            const int b = find_box_at(t.key, L.box0, L.nbox, l, ff_cell(x[0], t.lo[0], L.w),
                                      ff_cell(x[1], t.lo[1], L.w), ff_cell(x[2], t.lo[2], L.w));
            if (b < 0) break;
            anc[l] = b;
            A = b;
            lA = l;
            if (t.leaf[b]) break;
        }
        ns = 0;
        nd = 0;
    }
    __syncthreads();
    int l0 = 0;  // level of the first near set
    const bool l2t = A >= 0 && !t.L[lA].hf && t.L[lA].far && t.L[lA].p && lA >= t.lev_lo;
    if (l2t) {
        // L2T at x from A's local density
        const ff_level &L = t.L[lA];
        const c64d *pA = L.p + (int64_t)(A - L.box0) * L.T;
        for (int m = threadIdx.x; m < L.n_chk; m += FF) {
            cx<F> a;
            for (int s = 0; s < L.T; ++s) {
                const c64d uv = L.U[m + (int64_t)s * L.n_chk];
                const double f = 1.0 / L.sig[s];
                cfma_conj(a, cx<F>((F)uv.re, (F)uv.im), cx<F>((F)(f * pA[s].re), (F)(f * pA[s].im)));
            }
            psi[m] = a;
        }
        __syncthreads();
        const int32_t *cA = t.coord + 3 * (int64_t)A;
        const double a0 = t.lo[0] + (cA[0] + 0.5) * L.w, a1 = t.lo[1] + (cA[1] + 0.5) * L.w,
                     a2 = t.lo[2] + (cA[2] + 0.5) * L.w;
        for (int m = threadIdx.x; m < L.n_chk; m += FF)
            ff_acc_g<F>(are, aim, x, a0 + L.chk[3 * m], a1 + L.chk[3 * m + 1], a2 + L.chk[3 * m + 2], k, psi[m]);
        // A's near field as if A were a leaf: leaves near A's ancestors at
        // coarser low-frequency levels, and every box near A (opened below)
        for (int l = 0; l <= lA; ++l) {
            if (t.L[l].hf && l != lA) continue;
            const ff_level &Ll = t.L[l];
            const int32_t *ca = t.coord + 3 * (int64_t)anc[l];
            for (int o = threadIdx.x; o < 27; o += FF) {
                const int X = find_box_at(t.key, Ll.box0, Ll.nbox, l, ca[0] + o % 3 - 1, ca[1] + (o / 3) % 3 - 1,
                                          ca[2] + o / 9 - 1);
                if (X < 0) continue;
                if (t.leaf[X]) {
                    const int i = atomicAdd(&nd, 1);
                    if (i < FLIST) dlist[i] = X; else overflow = 1;
                } else if (l == lA) {
                    const int i = atomicAdd(&ns, 1);
                    if (i < FSET) sset[0][i] = X; else overflow = 1;
                }
            }
        }
        l0 = lA;
    } else if (threadIdx.x == 0 && t.L[0].nbox > 0) {
        sset[0][0] = t.L[0].box0;  // the whole tree from the root
        ns = 1;
    }
    __syncthreads();
    // direct sums of the leaves found so far
    for (int i = warp; i < min(nd, FLIST); i += FF / 32) {
        const int X = dlist[i];
        ff_direct<F>(t.bbeg[X], t.bend[X], qpt, qw, nrm, un, q, x, k, lane, are, aim);
    }
    int cur = 0;
    for (int l = l0; l < t.nlev; ++l) {
        __syncthreads();
        const int nset = min(ns, FSET);
        if (nset == 0 || overflow) break;
        if (threadIdx.x == 0) nn = 0;
        const bool child_far = l + 1 < t.nlev && t.L[l + 1].far && l + 1 >= t.lev_lo;
        int cx = 0, cy = 0, cz = 0;
        if (l + 1 < t.nlev) {
            const double w1 = t.L[l + 1].w;
            cx = ff_cell(x[0], t.lo[0], w1);
            cy = ff_cell(x[1], t.lo[1], w1);
            cz = ff_cell(x[2], t.lo[2], w1);
        }
        for (int r0 = 0; r0 < nset; r0 += FCH) {
            __syncthreads();
            if (threadIdx.x == 0) {
                nm = 0;
                nd = 0;
            }
            __syncthreads();
            for (int i = r0 + threadIdx.x; i < min(nset, r0 + FCH); i += FF) {
                const int B = sset[cur][i];
                if (t.leaf[B]) {
                    const int j = atomicAdd(&nd, 1);
                    if (j < FLIST) dlist[j] = B; else overflow = 1;
                    continue;
                }
                for (int C = t.c0[B]; C < t.c1[B]; ++C) {
                    const int32_t *cc = t.coord + 3 * (int64_t)C;
                    const int dx = cx - cc[0], dy = cy - cc[1], dz = cz - cc[2];
                    if (child_far && !ff_near(t.L[l + 1], dx, dy, dz)) {
                        const int j = atomicAdd(&nm, 1);
                        if (j < FLIST) {
                            mlist[j] = C;
                            mcone[j] = t.L[l + 1].hf ? cone_index(dx, dy, dz, t.L[l + 1].nc) : 0;
                        } else {
                            overflow = 1;
                        }
                    } else {
                        const int j = atomicAdd(&nn, 1);
                        if (j < FSET) sset[cur ^ 1][j] = C; else overflow = 1;
                    }
                }
            }
            __syncthreads();
            for (int i = warp; i < min(nm, FLIST); i += FF / 32) ff_m2t<F>(t, l + 1, mlist[i], mcone[i], x, k, lane, are, aim);
            for (int i = warp; i < min(nd, FLIST); i += FF / 32) {
                const int X = dlist[i];
                ff_direct<F>(t.bbeg[X], t.bend[X], qpt, qw, nrm, un, q, x, k, lane, are, aim);
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) ns = nn;
        cur ^= 1;
    }
    __syncthreads();
    double dre = are, dim = aim;  // partial sums added in FP64
    for (int o = 16; o > 0; o >>= 1) {
        dre += __shfl_xor_sync(0xffffffffu, dre, o);
        dim += __shfl_xor_sync(0xffffffffu, dim, o);
    }
    if (lane == 0) {
        red[warp][0] = dre;
        red[warp][1] = dim;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int i = 0; i < FF / 32; ++i) {
            a += red[i][0];
            b += red[i][1];
        }
        if (overflow) {
            atomicExch(err, 1);
            a = b = nan("");
        }
        out[ti] = c64d(a, b);
    }
}

// equivalent sources phi = V q~ of every box and cone of one level
// (one block per box and cone)
template <typename F>
__global__ void k_equiv_sources(const c64d *qd, const c64d *V, int T, int n_eq, int64_t nvec, cx<F> *phi)
{
    extern __shared__ __align__(16) uint8_t qsm_raw[];
    cx<F> *qsm = reinterpret_cast<cx<F> *>(qsm_raw);  // [T]
    for (int64_t v = blockIdx.x; v < nvec; v += gridDim.x) {
        __syncthreads();
        for (int s = threadIdx.x; s < T; s += blockDim.x) qsm[s] = cx<F>((F)qd[v * T + s].re, (F)qd[v * T + s].im);
        __syncthreads();
        for (int e = threadIdx.x; e < n_eq; e += blockDim.x) {
            cx<F> a;
            for (int s = 0; s < T; ++s) {
                const c64d vv = V[e + (int64_t)s * n_eq];
                cfma(a, cx<F>((F)vv.re, (F)vv.im), qsm[s]);
            }
            phi[v * n_eq + e] = a;
        }
    }
}

}  // namespace

// u, q: caller order (device, q may be null); tgt: device [ntgt][3]; out:
// device [ntgt], overwritten.
void fda_field(fda_handle *h, const c64d *u, const c64d *q, const double *tgt_dev, int64_t ntgt, int far, c64d *out)
{
    cudaStream_t s = h->stream;
    FDA_CUDA(cudaMemsetAsync(out, 0, sizeof(c64d) * ntgt, s));
    if (ntgt == 0 || h->N == 0) return;
    // u, q into Morton order (the element data's order)
    c64d *us = h->xs.as<c64d>(), *qs = q ? h->ys.as<c64d>() : nullptr;
    fda_gather_cols(h, u, h->N, us, 1, s);
    if (q) fda_gather_cols(h, q, h->N, qs, 1, s);
    int dev = 0, nsm = 0;
    FDA_CUDA(cudaGetDevice(&dev));
    FDA_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    const int64_t tb = (ntgt + FD - 1) / FD;
    // about eight blocks per SM over the element slices, at least 1,024 elements a slice
    int64_t slices = std::max<int64_t>(1, std::min<int64_t>((8ll * nsm + tb - 1) / tb, (h->N + 1023) / 1024));
    slices = std::min<int64_t>(slices, 65535);
    const int64_t per_block = (h->N + slices - 1) / slices;
    for (int64_t b0 = 0; b0 < tb; b0 += 65535) {
        const int64_t nb = std::min<int64_t>(65535, tb - b0);
        dim3 g((unsigned)nb, (unsigned)slices);
        k_field<<<g, FT, 0, s>>>(h->qpt.as<double>(), h->qw.as<double>(), h->nrm.as<double>(), us, qs, h->N,
                                 tgt_dev + 3 * b0 * FD, ntgt - b0 * FD, h->k, far, per_block, out + b0 * FD);
        FDA_CHECK_LAUNCH();
    }
}

// Far-field pattern through the fast algorithm: the outgoing densities of
// -D[u] + S[q] (the double layer of u by the operator's S2M, the single layer
// of q by the right-hand side's S2M) carried by M2M to the coarsest level
// with interaction lists, and summed there box by box (k_pattern_boxes).
// Elements of leaves above that level (none on a sphere) are summed directly.
// u, q: caller order (device, q may be null); dirs: device [ndir][3] unit
// vectors; out: device [ndir], overwritten.
void fda_far_field_upward(fda_handle *h, const c64d *u, const c64d *q, const double *dirs_dev, int ndir, c64d *out)
{
    cudaStream_t s = h->stream;
    FDA_CUDA(cudaMemsetAsync(out, 0, sizeof(c64d) * ndir, s));
    if (ndir == 0 || h->N == 0) return;
    c64d *us = h->xs.as<c64d>(), *qs = q ? h->ys.as<c64d>() : nullptr;
    fda_gather_cols(h, u, h->N, us, 1, s);
    if (q) fda_gather_cols(h, q, h->N, qs, 1, s);
    const int L = h->lev_lo;
    // element ranges (Morton order) not below a box of level L
    std::vector<std::pair<int64_t, int64_t>> direct;
    if (L < 0) {
        direct.push_back({0, h->N});
    } else {
        std::vector<int32_t> lb(h->nleaf), bb(h->nbox_total), be(h->nbox_total);
        FDA_CUDA(cudaMemcpy(lb.data(), h->leaf_box.p, 4 * (size_t)h->nleaf, cudaMemcpyDeviceToHost));
        FDA_CUDA(cudaMemcpy(bb.data(), h->box_begin.p, 4 * (size_t)h->nbox_total, cudaMemcpyDeviceToHost));
        FDA_CUDA(cudaMemcpy(be.data(), h->box_end.p, 4 * (size_t)h->nbox_total, cudaMemcpyDeviceToHost));
        for (int li = 0; li < h->nleaf; ++li)
            if (h->h_leaf_level[li] < L) direct.push_back({bb[lb[li]], be[lb[li]]});
    }
    for (const auto &r : direct) {
        const int64_t n = r.second - r.first, j0 = r.first;
        if (n <= 0) continue;
        const int64_t tb = (ndir + FD - 1) / FD;
        const int64_t slices = std::max<int64_t>(1, std::min<int64_t>((n + 1023) / 1024, 65535));
        const int64_t per_block = (n + slices - 1) / slices;
        for (int64_t b0 = 0; b0 < tb; b0 += 65535) {
            const int64_t nb = std::min<int64_t>(65535, tb - b0);
            k_field<<<dim3((unsigned)nb, (unsigned)slices), FT, 0, s>>>(
                h->qpt.as<double>() + 18 * j0, h->qw.as<double>() + 6 * j0, h->nrm.as<double>() + 3 * j0, us + j0,
                qs ? qs + j0 : nullptr, n, dirs_dev + 3 * b0 * FD, ndir - b0 * FD, h->k, 1, per_block, out + b0 * FD);
            FDA_CHECK_LAUNCH();
        }
    }
    if (L < 0) return;
    // -D[u] + S[q]: negate the (scratch) copy of u, S2M of both sides, M2M
    k_negate<<<fda_blocks(h->N, 256), 256, 0, s>>>(us, h->N);
    FDA_CHECK_LAUNCH();
    fda_upward_fp64(h, us, 0, 0);
    if (q) {
        fda_rhs_layers_prepare(h);
        fda_upward_fp64(h, qs, 1, 1);
    }
    fda_m2m_fp64(h);
    const level_info &V = h->lev[L];
    const size_t wbytes = sizeof(c64d) * (size_t)V.T;
    if (V.T > 1024) fda_fail(FDA_ERR_STATE, "far-field pattern: rank above 1024");
    k_pattern_boxes<<<ndir, FT, wbytes, s>>>(dirs_dev, ndir, h->q64[L].as<c64d>(), V.box0, V.nbox, V.ncones, V.nc,
                                             V.hf, V.T, h->eq_up[L].as<double>(), V.n_eq,
                                             V.hf ? h->rot[L].as<double>() : nullptr, h->Vup[L].as<c64d>(),
                                             h->box_coord.as<int32_t>(), h->root_lo[0], h->root_lo[1], h->root_lo[2],
                                             V.w, h->k, 1.0, out);
    FDA_CHECK_LAUNCH();
}

namespace {

// equivalent sources of every level and the point kernel, arithmetic type F
// (the densities in q64 / p64 are complete; us = -u, qs = q, Morton order)
template <typename F>
void field_points(fda_handle *h, const c64d *us, const c64d *qs, const double *tgt_dev, int64_t ntgt, c64d *out)
{
    cudaStream_t s = h->stream;
    ff_tree t;
    memset(&t, 0, sizeof(t));
    t.nlev = h->nlev;
    t.lev_lo = h->lev_lo;
    for (int d = 0; d < 3; ++d) t.lo[d] = h->root_lo[d];
    t.key = h->box_key.as<uint64_t>();
    t.coord = h->box_coord.as<int32_t>();
    t.leaf = h->box_leaf.as<int32_t>();
    t.c0 = h->box_child0.as<int32_t>();
    t.c1 = h->box_child1.as<int32_t>();
    t.bbeg = h->box_begin.as<int32_t>();
    t.bend = h->box_end.as<int32_t>();
    // equivalent sources of every level with outgoing densities, in one buffer
    std::vector<int64_t> phi_off(h->nlev + 1, 0);
    for (int l = 0; l < h->nlev; ++l) {
        const level_info &L = h->lev[l];
        const bool far = l >= h->lev_lo && L.active && L.T > 0 && h->q64[l].p;
        phi_off[l + 1] = phi_off[l] + (far ? (int64_t)L.nbox * L.ncones * L.n_eq : 0);
    }
    dbuf phi, derr;
    phi.alloc(sizeof(cx<F>) * (size_t)std::max<int64_t>(1, phi_off[h->nlev]));
    derr.alloc(sizeof(int));
    FDA_CUDA(cudaMemsetAsync(derr.p, 0, sizeof(int), s));
    for (int l = 0; l < h->nlev; ++l) {
        const level_info &L = h->lev[l];
        ff_level &V = t.L[l];
        V.box0 = L.box0;
        V.nbox = L.nbox;
        V.T = L.T;
        V.ncones = L.ncones;
        V.nc = L.nc;
        V.hf = L.hf;
        V.n_eq = L.n_eq;
        V.n_chk = L.n_chk;
        V.w = L.w;
        V.rho2 = L.rho * L.rho;
        V.far = phi_off[l + 1] > phi_off[l] ? 1 : 0;
        if (!V.far) continue;
        V.phi = phi.as<cx<F>>() + phi_off[l];
        V.eq = h->eq_up[l].as<double>();
        V.chk = h->chk_up[l].as<double>();
        V.rot = L.hf ? h->rot[l].as<double>() : nullptr;
        V.U = h->Uup[l].as<c64d>();
        V.sig = h->sig[l].as<double>();
        V.p = L.hf ? nullptr : h->p64[l].as<c64d>();
        if (!L.hf) t.max_chk = std::max(t.max_chk, L.n_chk);
        const int64_t nvec = (int64_t)L.nbox * L.ncones;
        k_equiv_sources<F><<<(unsigned)std::min<int64_t>(nvec, 65535), 128, sizeof(cx<F>) * L.T, s>>>(
            h->q64[l].as<c64d>(), h->Vup[l].as<c64d>(), L.T, L.n_eq, nvec, phi.as<cx<F>>() + phi_off[l]);
        FDA_CHECK_LAUNCH();
    }
    const size_t dyn = sizeof(cx<F>) * (size_t)std::max(1, t.max_chk);
    if (dyn > 96 * 1024) fda_fail(FDA_ERR_STATE, "fast field: more than 6,144 equivalent points at a level");
    FDA_CUDA(cudaFuncSetAttribute(k_field_fast<F>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn));
    for (int64_t t0 = 0; t0 < ntgt; t0 += (1ll << 30)) {
        const int64_t nb = std::min<int64_t>(1ll << 30, ntgt - t0);
        k_field_fast<F><<<(unsigned)nb, FF, dyn, s>>>(t, h->qpt.as<double>(), h->qw.as<double>(),
                                                      h->nrm.as<double>(), us, qs, tgt_dev + 3 * t0, nb, h->k,
                                                      derr.as<int>(), out + t0);
        FDA_CHECK_LAUNCH();
    }
    int herr = 0;
    FDA_CUDA(cudaMemcpyAsync(&herr, derr.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    FDA_CUDA(cudaStreamSynchronize(s));
    if (herr) fda_fail(FDA_ERR_STATE, "fast field: more than 2,048 boxes of one level near a point");
}

}  // namespace

// Scattered field at points through the fast algorithm (see k_field_fast):
// the outgoing densities of -D[u] + S[q] by S2M and M2M, the local densities
// by M2L and L2L (in FP64, or as in the chosen form's apply when the handle
// is in the chosen precision), the equivalent sources of every box, then one
// CTA per point (FP64 arithmetic; FP32 in the chosen precision, the
// differences x - y in FP64 and each CTA's partial sums added in FP64).  u, q: caller order (device, q may be null); tgt:
// device [ntgt][3]; out: device [ntgt], overwritten.
void fda_field_fast(fda_handle *h, const c64d *u, const c64d *q, const double *tgt_dev, int64_t ntgt, c64d *out)
{
    cudaStream_t s = h->stream;
    if (ntgt == 0 || h->N == 0) {
        FDA_CUDA(cudaMemsetAsync(out, 0, sizeof(c64d) * ntgt, s));
        return;
    }
    // no level with interaction lists: every pair is near and the direct sum is the method
    if (h->lev_lo < 0) {
        fda_field(h, u, q, tgt_dev, ntgt, 0, out);
        return;
    }
    c64d *us = h->xs.as<c64d>(), *qs = q ? h->ys.as<c64d>() : nullptr;
    fda_gather_cols(h, u, h->N, us, 1, s);
    if (q) fda_gather_cols(h, q, h->N, qs, 1, s);
    k_negate<<<fda_blocks(h->N, 256), 256, 0, s>>>(us, h->N);
    FDA_CHECK_LAUNCH();
    if (q) fda_rhs_layers_prepare(h);
    const bool chosen = h->cfg.precision == FDA_CHOSEN_FP32 && h->have32;
    if (chosen) {
        // the translations as in the chosen form's apply, densities then in FP64
        fda_translate_chosen(h, us, qs);
    } else {
        fda_upward_fp64(h, us, 0, 0);
        if (q) fda_upward_fp64(h, qs, 1, 1);
        fda_m2m_fp64(h);
        fda_downward_fp64(h);
    }
    // point evaluation in FP32 in the chosen precision, else in FP64
    if (chosen) field_points<float>(h, us, qs, tgt_dev, ntgt, out);
    else field_points<double>(h, us, qs, tgt_dev, ntgt, out);
}
