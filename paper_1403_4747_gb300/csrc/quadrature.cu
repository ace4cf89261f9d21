// Near-field matrix of Sec. 3.3 Step 4 (S2T): for every target element i of a
// leaf and every source element j of its near field,
//   A_ij = int_{tri_j} [ dG/dn_y + alpha d2G/dn_x dn_y ](x_i, y) dy      (Eq. eq_sum)
//   A_ii = 1/2 + alpha * FP int_{tri_i} d2G/dn_x dn_y (x_i, y) dy
// with collocation at centroids and constant elements (Sec. 5), alpha = i/k,
// c(x) = 1/2.  The paper names no element quadrature; the rules used here
// (also the operator's definition in the tests) are:
//   * regular pairs: Dunavant's six-point degree-4 rule;
//   * near pairs (j != i, |x_i - c_j| < 2 h_j, h_j = longest edge): the same
//     rule on the 64 sub-triangles of three rounds of midpoint subdivision;
//   * the self pair: the double layer vanishes on a flat triangle; the
//     hypersingular part is the Hadamard finite part with circular exclusion,
//       ik/2 - (1/4pi) sum_edges int e^{ik rho(phi)}/rho(phi) dphi,
//     per edge a closed-form static part plus a 16-point Gauss-Legendre rule
//     for the smooth remainder (e^{ik rho} - 1)/rho.
// All of it in FP64: these are the singular and near-singular integrals the
// method keeps in double precision.
//
// The same rules also build the near field of the right-hand side's layers
// of Eq. eq_bm for given Neumann data q = du/dn (side 1):
//   B_ij = int_{tri_j} [ G + alpha dG/dn_x ](x_i, y) dy,
//   B_ii = -alpha/2 + int_{tri_i} G(x_i, y) dy   (dG/dn_x vanishes in the plane),
// the weakly singular self integral in polar coordinates about x_i, whose
// radial part is closed: per edge int (e^{ik rho} - 1)/(4 pi ik) dphi,
// written as rho e^{ik rho/2} sin(k rho/2)/(k rho/2) (no cancellation at
// small k rho), by the 16-point Gauss-Legendre rule.
#include <math.h>

#include <vector>

#include "fda_internal.cuh"

namespace {

constexpr double NEAR_ETA2 = 4.0;  // (eta = 2)^2
constexpr int GL_N = 16;

__constant__ double c_gl_x[GL_N], c_gl_w[GL_N];
__constant__ double c_q6a[2] = {0.44594849091596488632, 0.09157621350977074346};
__constant__ double c_q6w[2] = {0.22338158967801146570, 0.10995174365532186764};

// Burton-Miller layer kernel: dG/dn_y + alpha d2G/dn_x dn_y, r = x - y
__device__ inline c64d bm_kernel(const double *x, const double *nx, const double *y, const double *ny, double k,
                                 double as)
{
    double r0 = x[0] - y[0], r1 = x[1] - y[1], r2 = x[2] - y[2];
    double R2 = r0 * r0 + r1 * r1 + r2 * r2;
    double R = sqrt(R2);
    double sn, cs;
    sincos(k * R, &sn, &cs);
    double inv4pR3 = 1.0 / (4.0 * FDA_PI * R2 * R);
    double rny = r0 * ny[0] + r1 * ny[1] + r2 * ny[2];
    double rnx = r0 * nx[0] + r1 * nx[1] + r2 * nx[2];
    double nn = nx[0] * ny[0] + nx[1] * ny[1] + nx[2] * ny[2];
    double kR = k * R;
    // a = (1 - ikR), b = (k^2R^2 - 3) + 3ikR
    c64d a(1.0, -kR);
    c64d e(cs, sn);
    double t = rnx * rny / R2;
    c64d bracket(nn + (kR * kR - 3.0) * t, -kR * nn + 3.0 * kR * t);
    c64d dl = (rny * inv4pR3) * (e * a);        // dG/dn_y
    c64d hs = inv4pR3 * (e * bracket);          // d2G/dn_x dn_y
    // alpha * hs with alpha = as i/k: as (i/k)(re + i im) = as (-im/k, re/k)
    return c64d(dl.re - as * hs.im / k, dl.im + as * hs.re / k);
}

// right-hand side's layer kernel: G + alpha dG/dn_x, r = x - y
__device__ inline c64d rhs_kernel(const double *x, const double *nx, const double *y, double k, double as)
{
    double r0 = x[0] - y[0], r1 = x[1] - y[1], r2 = x[2] - y[2];
    double R2 = r0 * r0 + r1 * r1 + r2 * r2;
    double R = sqrt(R2);
    double sn, cs;
    sincos(k * R, &sn, &cs);
    double g = 1.0 / (4.0 * FDA_PI * R);
    double rnx = r0 * nx[0] + r1 * nx[1] + r2 * nx[2];
    // dG/dn_x = -e^{ikR}(1 - ikR) rnx/(4 pi R^3)
    double f = -rnx * g / R2;
    double dre = f * (cs + k * R * sn), dim = f * (sn - k * R * cs);
    // G + as (i/k) dG/dn_x
    return c64d(cs * g - as * dim / k, sn * g + as * dre / k);
}

template <int SIDE>
__device__ inline c64d layer_kernel(const double *x, const double *nx, const double *y, const double *ny, double k,
                                    double as)
{
    if (SIDE == 1) return rhs_kernel(x, nx, y, k, as);
    return bm_kernel(x, nx, y, ny, k, as);
}

template <int SIDE>
__device__ inline c64d rule6(const double *x, const double *nx, const double *p0, const double *p1,
                             const double *p2, const double *ny, double area, double k, double as)
{
    c64d s;
    for (int g = 0; g < 2; ++g) {
        double a = c_q6a[g], b = 1.0 - 2.0 * c_q6a[g];
        double wa = c_q6w[g] * area;
        double bc[3][3] = {{b, a, a}, {a, b, a}, {a, a, b}};
        for (int r = 0; r < 3; ++r) {
            double y[3];
            for (int d = 0; d < 3; ++d) y[d] = bc[r][0] * p0[d] + bc[r][1] * p1[d] + bc[r][2] * p2[d];
            c64d v = layer_kernel<SIDE>(x, nx, y, ny, k, as);
            s.re += wa * v.re;
            s.im += wa * v.im;
        }
    }
    return s;
}

__device__ inline bool near_pair(const double *ci, const double *cj, double h2j)
{
    double d0 = ci[0] - cj[0], d1 = ci[1] - cj[1], d2 = ci[2] - cj[2];
    return d0 * d0 + d1 * d1 + d2 * d2 < NEAR_ETA2 * h2j;
}

// regular entries; near and self entries are left for the special kernels
template <int SIDE>
__global__ void k_near_regular(const int32_t *leaf_box, const int32_t *bbeg, const int32_t *bend,
                               const int64_t *colptr, const int32_t *cols, const int64_t *off, const double *cent,
                               const double *nrm, const double *v9, const double *area, const double *h2, double k,
                               double as, c64d *A)
{
    int li = blockIdx.x, r = blockIdx.y;
    int B = leaf_box[li];
    int i = bbeg[B] + r;
    if (i >= bend[B]) return;
    int64_t nc = colptr[li + 1] - colptr[li];
    const int32_t *cl = cols + colptr[li];
    c64d *row = A + off[li] + (int64_t)r * nc;
    const double *x = cent + 3 * i, *nx = nrm + 3 * i;
    for (int64_t c = threadIdx.x; c < nc; c += blockDim.x) {
        int j = cl[c];
        if (j == i || near_pair(x, cent + 3 * j, h2[j])) continue;
        const double *p = v9 + 9 * (int64_t)j;
        row[c] = rule6<SIDE>(x, nx, p, p + 3, p + 6, nrm + 3 * j, area[j], k, as);
    }
}

struct special_entry {
    int64_t idx;
    int32_t i, j;
};

// pass 0: count near/self entries per leaf row; pass 1: list them
__global__ void k_near_special_list(const int32_t *leaf_box, const int32_t *bbeg, const int32_t *bend,
                                    const int64_t *colptr, const int32_t *cols, const int64_t *off,
                                    const double *cent, const double *h2, int pass, unsigned long long *counter,
                                    special_entry *out)
{
    int li = blockIdx.x, r = blockIdx.y;
    int B = leaf_box[li];
    int i = bbeg[B] + r;
    if (i >= bend[B]) return;
    int64_t nc = colptr[li + 1] - colptr[li];
    const int32_t *cl = cols + colptr[li];
    const double *x = cent + 3 * i;
    for (int64_t c = threadIdx.x; c < nc; c += blockDim.x) {
        int j = cl[c];
        if (j == i || near_pair(x, cent + 3 * j, h2[j])) {
            unsigned long long slot = atomicAdd(counter, 1ull);
            if (pass) out[slot] = special_entry{off[li] + (int64_t)r * nc + c, i, j};
        }
    }
}

// one warp per near entry: 64 sub-triangles, two per lane
template <int SIDE>
__global__ void k_near_subdiv(const special_entry *list, int64_t n, const double *cent, const double *nrm,
                              const double *v9, const double *area, double k, double as, c64d *A)
{
    int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (w >= n) return;
    special_entry e = list[w];
    if (e.i == e.j) return;
    const double *x = cent + 3 * (int64_t)e.i, *nx = nrm + 3 * (int64_t)e.i;
    const double *ny = nrm + 3 * (int64_t)e.j;
    const double *P = v9 + 9 * (int64_t)e.j;
    double sub_area = area[e.j] / 64.0;
    c64d acc;
    for (int s = 2 * lane; s < 2 * lane + 2; ++s) {
        double a[3], b[3], c[3];
        for (int d = 0; d < 3; ++d) {
            a[d] = P[d];
            b[d] = P[3 + d];
            c[d] = P[6 + d];
        }
        for (int level = 2; level >= 0; --level) {
            int digit = (s >> (2 * level)) & 3;
            double m01[3], m12[3], m20[3];
            for (int d = 0; d < 3; ++d) {
                m01[d] = 0.5 * (a[d] + b[d]);
                m12[d] = 0.5 * (b[d] + c[d]);
                m20[d] = 0.5 * (c[d] + a[d]);
            }
            for (int d = 0; d < 3; ++d) {
                double na, nb, ncc;
                if (digit == 0) { na = a[d]; nb = m01[d]; ncc = m20[d]; }
                else if (digit == 1) { na = m01[d]; nb = b[d]; ncc = m12[d]; }
                else if (digit == 2) { na = m20[d]; nb = m12[d]; ncc = c[d]; }
                else { na = m01[d]; nb = m12[d]; ncc = m20[d]; }
                a[d] = na; b[d] = nb; c[d] = ncc;
            }
        }
        c64d v = rule6<SIDE>(x, nx, a, b, c, ny, sub_area, k, as);
        acc.re += v.re;
        acc.im += v.im;
    }
    for (int o = 16; o > 0; o >>= 1) {
        acc.re += __shfl_xor_sync(0xffffffffu, acc.re, o);
        acc.im += __shfl_xor_sync(0xffffffffu, acc.im, o);
    }
    if (lane == 0) A[e.idx] = acc;
}

// self entries: 1/2 + alpha * finite part (one thread each)
__global__ void k_near_self(const special_entry *list, int64_t n, const double *cent, const double *v9, double k,
                            double as, c64d *A)
{
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= n) return;
    special_entry e = list[t];
    if (e.i != e.j) return;
    const double *x = cent + 3 * (int64_t)e.i;
    const double *P = v9 + 9 * (int64_t)e.i;
    double st = 0.0, dre = 0.0, dim = 0.0;
    for (int ed = 0; ed < 3; ++ed) {
        const double *a = P + 3 * ed, *b = P + 3 * ((ed + 1) % 3);
        double tv[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
        double L = sqrt(tv[0] * tv[0] + tv[1] * tv[1] + tv[2] * tv[2]);
        for (int d = 0; d < 3; ++d) tv[d] /= L;
        double s = (x[0] - a[0]) * tv[0] + (x[1] - a[1]) * tv[1] + (x[2] - a[2]) * tv[2];
        double f[3] = {x[0] - (a[0] + s * tv[0]), x[1] - (a[1] + s * tv[1]), x[2] - (a[2] + s * tv[2])};
        double dist = sqrt(f[0] * f[0] + f[1] * f[1] + f[2] * f[2]);
        double pa = atan2(-s, dist), pb = atan2(L - s, dist);
        st += (sin(pb) - sin(pa)) / dist;
        double half = 0.5 * (pb - pa), mid = 0.5 * (pb + pa);
        for (int g = 0; g < GL_N; ++g) {
            double phi = mid + half * c_gl_x[g];
            double rho = dist / cos(phi);
            double sn, cs;
            sincos(k * rho, &sn, &cs);
            dre += half * c_gl_w[g] * (cs - 1.0) / rho;
            dim += half * c_gl_w[g] * sn / rho;
        }
    }
    // H = ik/2 - (st + D)/(4 pi);  A_ii = 1/2 + as (i/k) H
    double Hre = -(st + dre) / (4.0 * FDA_PI);
    double Him = 0.5 * k - dim / (4.0 * FDA_PI);
    A[e.idx] = c64d(0.5 - as * Him / k, as * Hre / k);
}

// right-hand side's self entries: -alpha/2 + int G (one thread each)
__global__ void k_near_self_rhs(const special_entry *list, int64_t n, const double *cent, const double *v9, double k,
                                double as, c64d *A)
{
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= n) return;
    special_entry e = list[t];
    if (e.i != e.j) return;
    const double *x = cent + 3 * (int64_t)e.i;
    const double *P = v9 + 9 * (int64_t)e.i;
    double sre = 0.0, sim = 0.0;
    for (int ed = 0; ed < 3; ++ed) {
        const double *a = P + 3 * ed, *b = P + 3 * ((ed + 1) % 3);
        double tv[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
        double L = sqrt(tv[0] * tv[0] + tv[1] * tv[1] + tv[2] * tv[2]);
        for (int d = 0; d < 3; ++d) tv[d] /= L;
        double s = (x[0] - a[0]) * tv[0] + (x[1] - a[1]) * tv[1] + (x[2] - a[2]) * tv[2];
        double f[3] = {x[0] - (a[0] + s * tv[0]), x[1] - (a[1] + s * tv[1]), x[2] - (a[2] + s * tv[2])};
        double dist = sqrt(f[0] * f[0] + f[1] * f[1] + f[2] * f[2]);
        double pa = atan2(-s, dist), pb = atan2(L - s, dist);
        double half = 0.5 * (pb - pa), mid = 0.5 * (pb + pa);
        for (int g = 0; g < GL_N; ++g) {
            double rho = dist / cos(mid + half * c_gl_x[g]);
            double th = 0.5 * k * rho;
            double sn, cs;
            sincos(th, &sn, &cs);
            double m = rho * (sn / th);  // (e^{ik rho} - 1)/(ik) = rho e^{i th} sin(th)/th
            sre += half * c_gl_w[g] * m * cs;
            sim += half * c_gl_w[g] * m * sn;
        }
    }
    // -as (i/k)/2 + (sre + i sim)/(4 pi)
    A[e.idx] = c64d(sre / (4.0 * FDA_PI), sim / (4.0 * FDA_PI) - 0.5 * as / k);
}

__global__ void k_to_f32(const c64d *a, c32f *b, int64_t n)
{
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t < n) b[t] = c32f((float)a[t].re, (float)a[t].im);
}

// Gauss-Legendre nodes by Newton iteration on the three-term recurrence
void gauss_legendre_host(int n, double *x, double *w)
{
    for (int i = 0; i < n; ++i) {
        double z = cos(FDA_PI * (i + 0.75) / (n + 0.5));
        double dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p1 = 1.0, p0 = 0.0;
            for (int j = 1; j <= n; ++j) {
                double p2 = p0;
                p0 = p1;
                p1 = ((2.0 * j - 1.0) * z * p0 - (j - 1.0) * p2) / j;
            }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
            double dz = p1 / dp;
            z -= dz;
            if (fabs(dz) < 1e-16) break;
        }
        double p1 = 1.0, p0 = 0.0;
        for (int j = 1; j <= n; ++j) {
            double p2 = p0;
            p0 = p1;
            p1 = ((2.0 * j - 1.0) * z * p0 - (j - 1.0) * p2) / j;
        }
        dp = n * (z * p1 - p0) / (z * z - 1.0);
        x[i] = -z;
        w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

}  // namespace

void fda_near_convert_f32(fda_handle *h, int side)
{
    dbuf &src = side ? h->op64.near1 : h->op64.near, &dst = side ? h->op32.near1 : h->op32.near;
    dst.alloc(sizeof(c32f) * std::max<int64_t>(h->nnz_near, 1));
    k_to_f32<<<fda_blocks(h->nnz_near, 256), 256, 0, h->stream>>>(src.as<c64d>(), dst.as<c32f>(), h->nnz_near);
    FDA_CHECK_LAUNCH();
}

// side 0: the Burton-Miller operator's near field; side 1: the right-hand
// side's layers (same pattern)
void fda_near_build(fda_handle *h, int side)
{
    cudaStream_t s = h->stream;
    double gx[GL_N], gw[GL_N];
    gauss_legendre_host(GL_N, gx, gw);
    FDA_CUDA(cudaMemcpyToSymbolAsync(c_gl_x, gx, sizeof(gx), 0, cudaMemcpyHostToDevice, s));
    FDA_CUDA(cudaMemcpyToSymbolAsync(c_gl_w, gw, sizeof(gw), 0, cudaMemcpyHostToDevice, s));
    const int NL = h->nleaf;
    dbuf &dst = side ? h->op64.near1 : h->op64.near;
    dst.alloc(sizeof(c64d) * std::max<int64_t>(h->nnz_near, 1));
    dim3 g(NL, h->max_leaf_rows);
    // near/self entries first (cheap geometry test), then the regular rule
    dbuf counter;
    counter.alloc(sizeof(unsigned long long));
    FDA_CUDA(cudaMemsetAsync(counter.p, 0, 8, s));
    k_near_special_list<<<g, 128, 0, s>>>(h->leaf_box.as<int32_t>(), h->box_begin.as<int32_t>(),
                                          h->box_end.as<int32_t>(), h->nf_colptr.as<int64_t>(),
                                          h->nf_cols.as<int32_t>(), h->nf_off.as<int64_t>(), h->cent.as<double>(),
                                          h->h2.as<double>(), 0, counter.as<unsigned long long>(), nullptr);
    FDA_CHECK_LAUNCH();
    unsigned long long nspec = 0;
    FDA_CUDA(cudaMemcpyAsync(&nspec, counter.p, 8, cudaMemcpyDeviceToHost, s));
    FDA_CUDA(cudaStreamSynchronize(s));
    dbuf list;
    list.alloc(sizeof(special_entry) * (nspec + 1));
    FDA_CUDA(cudaMemsetAsync(counter.p, 0, 8, s));
    k_near_special_list<<<g, 128, 0, s>>>(h->leaf_box.as<int32_t>(), h->box_begin.as<int32_t>(),
                                          h->box_end.as<int32_t>(), h->nf_colptr.as<int64_t>(),
                                          h->nf_cols.as<int32_t>(), h->nf_off.as<int64_t>(), h->cent.as<double>(),
                                          h->h2.as<double>(), 1, counter.as<unsigned long long>(),
                                          list.as<special_entry>());
    FDA_CHECK_LAUNCH();
    auto regular = side ? k_near_regular<1> : k_near_regular<0>;
    regular<<<g, 128, 0, s>>>(h->leaf_box.as<int32_t>(), h->box_begin.as<int32_t>(), h->box_end.as<int32_t>(),
                              h->nf_colptr.as<int64_t>(), h->nf_cols.as<int32_t>(), h->nf_off.as<int64_t>(),
                              h->cent.as<double>(), h->nrm.as<double>(), h->verts9.as<double>(), h->area.as<double>(),
                              h->h2.as<double>(), h->k, h->cfg.alpha_sign, dst.as<c64d>());
    FDA_CHECK_LAUNCH();
    if (nspec > 0) {
        auto subdiv = side ? k_near_subdiv<1> : k_near_subdiv<0>;
        subdiv<<<fda_blocks((int64_t)nspec * 32, 256), 256, 0, s>>>(
            list.as<special_entry>(), (int64_t)nspec, h->cent.as<double>(), h->nrm.as<double>(),
            h->verts9.as<double>(), h->area.as<double>(), h->k, h->cfg.alpha_sign, dst.as<c64d>());
        FDA_CHECK_LAUNCH();
        auto self = side ? k_near_self_rhs : k_near_self;
        self<<<fda_blocks((int64_t)nspec, 128), 128, 0, s>>>(list.as<special_entry>(), (int64_t)nspec,
                                                              h->cent.as<double>(), h->verts9.as<double>(), h->k,
                                                              h->cfg.alpha_sign, dst.as<c64d>());
        FDA_CHECK_LAUNCH();
    }
    FDA_CUDA(cudaStreamSynchronize(s));
}
