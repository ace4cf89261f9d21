/*
 * Plain FP64 CPU oracle for the collocation Burton-Miller operator.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library calls, links or
 * loads this file; only tests/, the smoke check and the benchmark's CPU
 * baseline leg do.  It shares no code with the CUDA path.
 *
 * What it computes (all in double / double complex, no blocking, no reuse):
 *
 *   (A x)_i = sum_j A_ij x_j,
 *   A_ij    = int_{tri_j} [ dG/dn_y + alpha d2G/dn_x dn_y ](x_i, y) dy   (i != j)
 *   A_ii    = 1/2 + alpha * FP int_{tri_i} d2G/dn_x dn_y (x_i, y) dy
 *
 * which is the left-hand side of the Burton-Miller equation (Sec. 2, Eq.
 * eq_bm) discretised as in Eq. eq_sum with collocation at centroids and
 * piecewise-constant elements (Sec. 5): w_i = delta(x_i), chi_j = 1 on
 * triangle j, c(x) = 1/2 at a centroid of a flat triangle, alpha = i/k.
 *
 * Readings of what the paper leaves open (each listed in the design notes):
 *   - normal n = unit normal pointing out of the acoustic domain, i.e. into
 *     the body: n = -(v1 - v0) x (v2 - v0)/|.|, for triangles oriented with
 *     (v1 - v0) x (v2 - v0) pointing into the acoustic domain.  This is the
 *     orientation under which Eq. cbie, with G = e^{ikr}/(4 pi r), is Green's
 *     representation for the exterior problem.
 *   - element quadrature (the paper names none):
 *       regular pairs: 6-point degree-4 symmetric triangle rule (Dunavant);
 *       near pairs, j != i and |x_i - c_j| < ETA * h_j (h_j = longest edge):
 *         the same rule on each of the 4^SUBDIV sub-triangles of a uniform
 *         midpoint subdivision;
 *       self pair: the double-layer part vanishes (x_i lies in the plane of
 *         the triangle); the hypersingular part is the Hadamard finite part
 *         with circular exclusion,
 *           FP int e^{ikR}(1 - ikR)/(4 pi R^3) dA
 *             = ik/2 - (1/(4 pi)) int_0^{2 pi} e^{ik rho(t)}/rho(t) dt,
 *         rho(t) = distance from x_i to the boundary along direction t; the
 *         angular integral is split per edge into its closed-form static
 *         part and a smooth remainder integrated by Gauss-Legendre.
 *
 * The right-hand side's layers of Eq. eq_bm, acting on given Neumann data
 * q = du/dn (a radiating body, u_inc = 0), discretised the same way:
 *
 *   (B q)_i = -alpha c q_i + sum_j B_ij q_j,
 *   B_ij    = int_{tri_j} [ G + alpha dG/dn_x ](x_i, y) dy                 (i != j)
 *   B_ii    = int_{tri_i} G(x_i, y) dy       (dG/dn_x vanishes: r.n_x = 0 on a flat triangle)
 *
 * with the same element rules; the weakly singular self integral is taken in
 * polar coordinates about x_i, where the radial integral is closed:
 *   int_tri G dA = (1/(4 pi)) int_0^{2 pi} (e^{ik rho(t)} - 1)/(ik) dt.
 *
 * Kernels (r = x - y, R = |r|, derived from G; pinned by finite differences):
 *   G           = e^{ikR}/(4 pi R)
 *   dG/dn_y     = e^{ikR}(1 - ikR)(r.n_y)/(4 pi R^3)
 *   dG/dn_x     = -e^{ikR}(1 - ikR)(r.n_x)/(4 pi R^3)
 *   d2G/dnx dny = e^{ikR}/(4 pi R^3) [ (1 - ikR)(n_x.n_y)
 *                  + (k^2 R^2 + 3ikR - 3)(r.n_x)(r.n_y)/R^2 ]
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

#define ORC_PI 3.14159265358979323846
#define ETA 2.0
#define SUBDIV 3
#define GL_SELF 16

/* Dunavant degree-4 six-point rule on a triangle: barycentric points
 * (a, a, 1-2a) and permutations, weights relative to the area. */
static const double R6_A[2] = {0.44594849091596488632, 0.09157621350977074346};
static const double R6_W[2] = {0.22338158967801146570, 0.10995174365532186764};

/* ------------------------------------------------------------------ */
/* small vector helpers                                                */
/* ------------------------------------------------------------------ */
static double dot3(const double *a, const double *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static void sub3(const double *a, const double *b, double *o) { o[0] = a[0] - b[0]; o[1] = a[1] - b[1]; o[2] = a[2] - b[2]; }
static void cross3(const double *a, const double *b, double *o)
{
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}

/* ------------------------------------------------------------------ */
/* geometry of one triangle                                            */
/* ------------------------------------------------------------------ */
typedef struct {
    double v[3][3];   /* vertices */
    double c[3];      /* centroid */
    double n[3];      /* unit normal into the body (see header) */
    double area;
    double h2;        /* squared longest edge */
} tri_t;

static void make_tri(const double *verts, const int32_t *tris, int64_t t, tri_t *T)
{
    for (int a = 0; a < 3; ++a)
        for (int d = 0; d < 3; ++d) T->v[a][d] = verts[3 * (int64_t)tris[3 * t + a] + d];
    for (int d = 0; d < 3; ++d) T->c[d] = (T->v[0][d] + T->v[1][d] + T->v[2][d]) / 3.0;
    double e1[3], e2[3], e3[3], nu[3];
    sub3(T->v[1], T->v[0], e1);
    sub3(T->v[2], T->v[0], e2);
    sub3(T->v[2], T->v[1], e3);
    cross3(e1, e2, nu);
    double len = sqrt(dot3(nu, nu));
    T->area = 0.5 * len;
    for (int d = 0; d < 3; ++d) T->n[d] = -nu[d] / len;
    double l1 = dot3(e1, e1), l2 = dot3(e2, e2), l3 = dot3(e3, e3);
    T->h2 = fmax(l1, fmax(l2, l3));
}

/* ------------------------------------------------------------------ */
/* kernels                                                             */
/* ------------------------------------------------------------------ */
/* out[0] = G, out[1] = dG/dn_y, out[2] = dG/dn_x, out[3] = d2G/dn_x dn_y */
static void kernels_all(const double *x, const double *nx, const double *y, const double *ny,
                        double k, cplx out[4])
{
    double r[3];
    sub3(x, y, r);
    double R2 = dot3(r, r), R = sqrt(R2);
    cplx e = cexp(I * k * R);
    double rny = dot3(r, ny), rnx = dot3(r, nx), nxny = dot3(nx, ny);
    double f4 = 4.0 * ORC_PI;
    out[0] = e / (f4 * R);
    out[1] = e * (1.0 - I * k * R) * rny / (f4 * R2 * R);
    out[2] = -e * (1.0 - I * k * R) * rnx / (f4 * R2 * R);
    out[3] = e / (f4 * R2 * R) *
             ((1.0 - I * k * R) * nxny + (k * k * R2 + 3.0 * I * k * R - 3.0) * rnx * rny / R2);
}

/* Sign s of the coupling alpha = s i/k (s = +1: the paper's alpha = i/k as
 * written; s = -1: the conjugate coupling).  Set per exported call. */
static double g_alpha_sign = 1.0;

void orc_set_alpha_sign(double s) { g_alpha_sign = s; }

/* Which layer an integral takes: the Burton-Miller combination of Eq.
 * eq_sum, or (for the pin tests) the double layer or hypersingular layer
 * alone.  Set once per exported call, before any parallel region. */
static int g_part = 0;

/* Which side of Eq. eq_bm the integrals take: 0 the left-hand side (acting
 * on u), 1 the right-hand side's layers (acting on q = du/dn).  Set once per
 * exported call, before any parallel region. */
static int g_side = 0;

void orc_set_side(int side) { g_side = side; }

/* Layer kernel: left-hand side of Eq. eq_sum, dG/dn_y + alpha d2G/dn_x dn_y;
 * right-hand side, G + alpha dG/dn_x */
static cplx kernel_bm(const double *x, const double *nx, const double *y, const double *ny, double k)
{
    cplx o[4];
    kernels_all(x, nx, y, ny, k, o);
    cplx alpha = g_alpha_sign * I / k;
    if (g_side == 1) return o[0] + alpha * o[2];
    if (g_part == 1) return o[1];
    if (g_part == 2) return o[3];
    return o[1] + alpha * o[3];
}

/* ------------------------------------------------------------------ */
/* element quadrature                                                  */
/* ------------------------------------------------------------------ */
/* six-point rule on the triangle (p0, p1, p2) of area `area` */
static cplx integrate_r6(const double *x, const double *nx, const double p[3][3], const double *ny,
                         double area, double k)
{
    cplx s = 0.0;
    for (int g = 0; g < 2; ++g) {
        double a = R6_A[g], b = 1.0 - 2.0 * R6_A[g];
        double bary[3][3] = {{b, a, a}, {a, b, a}, {a, a, b}};
        for (int q = 0; q < 3; ++q) {
            double y[3];
            for (int d = 0; d < 3; ++d)
                y[d] = bary[q][0] * p[0][d] + bary[q][1] * p[1][d] + bary[q][2] * p[2][d];
            s += R6_W[g] * area * kernel_bm(x, nx, y, ny, k);
        }
    }
    return s;
}

/* same rule on every sub-triangle of `levels` rounds of midpoint subdivision */
static cplx integrate_subdiv(const double *x, const double *nx, const double p[3][3], const double *ny,
                             double area, double k, int levels)
{
    if (levels == 0) return integrate_r6(x, nx, p, ny, area, k);
    double m01[3], m12[3], m20[3];
    for (int d = 0; d < 3; ++d) {
        m01[d] = 0.5 * (p[0][d] + p[1][d]);
        m12[d] = 0.5 * (p[1][d] + p[2][d]);
        m20[d] = 0.5 * (p[2][d] + p[0][d]);
    }
    double s0[3][3], s1[3][3], s2[3][3], s3[3][3];
    memcpy(s0[0], p[0], sizeof m01); memcpy(s0[1], m01, sizeof m01); memcpy(s0[2], m20, sizeof m01);
    memcpy(s1[0], m01, sizeof m01); memcpy(s1[1], p[1], sizeof m01); memcpy(s1[2], m12, sizeof m01);
    memcpy(s2[0], m20, sizeof m01); memcpy(s2[1], m12, sizeof m01); memcpy(s2[2], p[2], sizeof m01);
    memcpy(s3[0], m01, sizeof m01); memcpy(s3[1], m12, sizeof m01); memcpy(s3[2], m20, sizeof m01);
    double a4 = 0.25 * area;
    return integrate_subdiv(x, nx, s0, ny, a4, k, levels - 1) + integrate_subdiv(x, nx, s1, ny, a4, k, levels - 1) +
           integrate_subdiv(x, nx, s2, ny, a4, k, levels - 1) + integrate_subdiv(x, nx, s3, ny, a4, k, levels - 1);
}

/* Gauss-Legendre nodes/weights on [-1, 1] by Newton iteration on P_n */
static void gauss_legendre(int n, double *xs, double *ws)
{
    for (int i = 0; i < n; ++i) {
        double z = cos(ORC_PI * (i + 0.75) / (n + 0.5)), pp = 0.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = 0.0;
            for (int j = 1; j <= n; ++j) {
                double p2 = p1;
                p1 = p0;
                p0 = ((2.0 * j - 1.0) * z * p1 - (j - 1.0) * p2) / j;
            }
            pp = n * (z * p0 - p1) / (z * z - 1.0);
            double dz = p0 / pp;
            z -= dz;
            if (fabs(dz) < 1e-16) break;
        }
        {
            double p0 = 1.0, p1 = 0.0;
            for (int j = 1; j <= n; ++j) {
                double p2 = p1;
                p1 = p0;
                p0 = ((2.0 * j - 1.0) * z * p1 - (j - 1.0) * p2) / j;
            }
            pp = n * (z * p0 - p1) / (z * z - 1.0);
        }
        xs[i] = -z;
        ws[i] = 2.0 / ((1.0 - z * z) * pp * pp);
    }
}

/* Hadamard finite part of int_tri e^{ikR}(1 - ikR)/(4 pi R^3) dA about the
 * interior point x (the centroid), in polar coordinates about x:
 *   = ik/2 - (1/(4 pi)) sum_edges int_{phi_a}^{phi_b} e^{ik d/cos(phi)} cos(phi)/d dphi
 * with d the distance from x to the edge line and phi the angle from the
 * perpendicular.  Per edge: static part (sin phi_b - sin phi_a)/d exactly, and
 * the smooth remainder (e^{ik rho} - 1)/rho by Gauss-Legendre. */
static cplx self_hypersingular(const tri_t *T, double k)
{
    double gx[GL_SELF], gw[GL_SELF];
    gauss_legendre(GL_SELF, gx, gw);
    cplx acc = 0.0;
    for (int e = 0; e < 3; ++e) {
        const double *a = T->v[e], *b = T->v[(e + 1) % 3];
        double t[3], xa[3];
        sub3(b, a, t);
        double L = sqrt(dot3(t, t));
        for (int d = 0; d < 3; ++d) t[d] /= L;
        sub3(T->c, a, xa);
        double s = dot3(xa, t);
        double foot[3], dv[3];
        for (int d = 0; d < 3; ++d) foot[d] = a[d] + s * t[d];
        sub3(T->c, foot, dv);
        double dist = sqrt(dot3(dv, dv));
        double sa = -s, sb = L - s; /* tangential coordinates of a and b from the foot */
        double pa = atan2(sa, dist), pb = atan2(sb, dist);
        acc += (sin(pb) - sin(pa)) / dist;
        double half = 0.5 * (pb - pa), mid = 0.5 * (pb + pa);
        for (int g = 0; g < GL_SELF; ++g) {
            double phi = mid + half * gx[g];
            double rho = dist / cos(phi);
            acc += half * gw[g] * (cexp(I * k * rho) - 1.0) / rho;
        }
    }
    return I * k / 2.0 - acc / (4.0 * ORC_PI);
}

/* int_tri G(x, y) dA about the interior point x (the centroid), in polar
 * coordinates about x: per edge, with d the distance from x to the edge line
 * and phi the angle from the perpendicular, rho(phi) = d/cos(phi) and
 *   int_0^rho e^{ikr}/(4 pi r) r dr = (e^{ik rho} - 1)/(4 pi ik),
 * integrated over phi by Gauss-Legendre. */
static cplx self_single(const tri_t *T, double k)
{
    double gx[GL_SELF], gw[GL_SELF];
    gauss_legendre(GL_SELF, gx, gw);
    cplx acc = 0.0;
    for (int e = 0; e < 3; ++e) {
        const double *a = T->v[e], *b = T->v[(e + 1) % 3];
        double t[3], xa[3];
        sub3(b, a, t);
        double L = sqrt(dot3(t, t));
        for (int d = 0; d < 3; ++d) t[d] /= L;
        sub3(T->c, a, xa);
        double s = dot3(xa, t);
        double foot[3], dv[3];
        for (int d = 0; d < 3; ++d) foot[d] = a[d] + s * t[d];
        sub3(T->c, foot, dv);
        double dist = sqrt(dot3(dv, dv));
        double pa = atan2(-s, dist), pb = atan2(L - s, dist);
        double half = 0.5 * (pb - pa), mid = 0.5 * (pb + pa);
        for (int g = 0; g < GL_SELF; ++g) {
            double rho = dist / cos(mid + half * gx[g]);
            acc += half * gw[g] * (cexp(I * k * rho) - 1.0) / (I * k);
        }
    }
    return acc / (4.0 * ORC_PI);
}

/* one matrix entry A_ij (left-hand side) or B_ij (right-hand side) */
static cplx entry(const tri_t *Ti, const tri_t *Tj, int same, double k)
{
    if (same && g_side == 1) return -0.5 * (g_alpha_sign * I / k) + self_single(Ti, k);
    if (same) {
        if (g_part == 1) return 0.5;
        if (g_part == 2) return self_hypersingular(Ti, k);
        return 0.5 + (g_alpha_sign * I / k) * self_hypersingular(Ti, k);
    }
    double dv[3];
    sub3(Ti->c, Tj->c, dv);
    double d2 = dot3(dv, dv);
    if (d2 < ETA * ETA * Tj->h2)
        return integrate_subdiv(Ti->c, Ti->n, Tj->v, Tj->n, Tj->area, k, SUBDIV);
    return integrate_r6(Ti->c, Ti->n, Tj->v, Tj->n, Tj->area, k);
}

/* ------------------------------------------------------------------ */
/* exported API (ctypes)                                               */
/* ------------------------------------------------------------------ */
static tri_t *build_all(const double *verts, const int32_t *tris, int64_t nt)
{
    tri_t *T = (tri_t *)malloc(sizeof(tri_t) * (size_t)(nt > 0 ? nt : 1));
    for (int64_t t = 0; t < nt; ++t) make_tri(verts, tris, t, &T[t]);
    return T;
}

static void set_threads(int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* centroids [nt,3], normals n (into the body) [nt,3], areas [nt], h^2 [nt] */
void orc_geometry(const double *verts, const int32_t *tris, int64_t nt, double *cent, double *nrm,
                  double *area, double *h2)
{
    for (int64_t t = 0; t < nt; ++t) {
        tri_t T;
        make_tri(verts, tris, t, &T);
        for (int d = 0; d < 3; ++d) {
            cent[3 * t + d] = T.c[d];
            nrm[3 * t + d] = T.n[d];
        }
        area[t] = T.area;
        h2[t] = T.h2;
    }
}

/* the four kernels at one point pair: out = [G, dG/dny, dG/dnx, d2G] interleaved */
void orc_kernels(const double *x, const double *nx, const double *y, const double *ny, double k, double *out)
{
    cplx o[4];
    kernels_all(x, nx, y, ny, k, o);
    for (int a = 0; a < 4; ++a) {
        out[2 * a] = creal(o[a]);
        out[2 * a + 1] = cimag(o[a]);
    }
}

/* int over triangle p (vertices row-major [3,3], normal ny, area) of the
 * Burton-Miller kernel at (x, nx), with `levels` rounds of subdivision */
void orc_integrate_triangle(const double *x, const double *nx, const double *p, const double *ny,
                            double area, double k, int levels, double *out)
{
    double P[3][3];
    memcpy(P, p, sizeof P);
    g_part = 0;
    cplx v = integrate_subdiv(x, nx, P, ny, area, k, levels);
    out[0] = creal(v);
    out[1] = cimag(v);
}

/* FP integral of the hypersingular kernel over triangle t about its centroid */
void orc_self_hypersingular(const double *verts, const int32_t *tris, int64_t t, double k, double *out)
{
    tri_t T;
    make_tri(verts, tris, t, &T);
    cplx v = self_hypersingular(&T, k);
    out[0] = creal(v);
    out[1] = cimag(v);
}

void orc_gauss_legendre(int n, double *xs, double *ws) { gauss_legendre(n, xs, ws); }

/* the six-point rule on the reference triangle (0,0),(1,0),(0,1):
 * pts [6,2], weights [6] summing to 1 (relative to the area) */
void orc_rule6(double *pts, double *w)
{
    int q = 0;
    for (int g = 0; g < 2; ++g) {
        double a = R6_A[g], b = 1.0 - 2.0 * R6_A[g];
        double bary[3][3] = {{b, a, a}, {a, b, a}, {a, a, b}};
        for (int p = 0; p < 3; ++p, ++q) {
            pts[2 * q] = bary[p][1];
            pts[2 * q + 1] = bary[p][2];
            w[q] = R6_W[g];
        }
    }
}

/* row sums of one layer: part 1 -> 1/2 + sum_j D_ij, part 2 -> sum_j H_ij
 * (the hypersingular integrals without alpha), for all rows */
void orc_layer_rowsum(const double *verts, const int32_t *tris, int64_t nt, double k, int part, double *out,
                      int nthreads)
{
    tri_t *T = (tri_t *)malloc(sizeof(tri_t) * (size_t)(nt > 0 ? nt : 1));
    for (int64_t t = 0; t < nt; ++t) make_tri(verts, tris, t, &T[t]);
    g_part = part;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t i = 0; i < nt; ++i) {
        cplx acc = 0.0;
        for (int64_t j = 0; j < nt; ++j) acc += entry(&T[i], &T[j], i == j, k);
        out[2 * i] = creal(acc);
        out[2 * i + 1] = cimag(acc);
    }
    g_part = 0;
    free(T);
}

/* int_tri G(x_t, y) dy over triangle t from its own centroid (interleaved complex) */
void orc_self_single(const double *verts, const int32_t *tris, int64_t t, double k, double *out)
{
    tri_t T;
    make_tri(verts, tris, t, &T);
    cplx v = self_single(&T, k);
    out[0] = creal(v);
    out[1] = cimag(v);
}

/* single entry A_ij (interleaved complex) */
void orc_entry(const double *verts, const int32_t *tris, int64_t nt, double k, int64_t i, int64_t j, double *out)
{
    (void)nt;
    tri_t Ti, Tj;
    make_tri(verts, tris, i, &Ti);
    make_tri(verts, tris, j, &Tj);
    g_part = 0;
    cplx v = entry(&Ti, &Tj, i == j, k);
    out[0] = creal(v);
    out[1] = cimag(v);
}

/* 1 if the pair (i, j), i != j, takes the subdivided near rule */
int orc_is_near_pair(const double *verts, const int32_t *tris, int64_t i, int64_t j)
{
    tri_t Ti, Tj;
    make_tri(verts, tris, i, &Ti);
    make_tri(verts, tris, j, &Tj);
    double dv[3];
    sub3(Ti.c, Tj.c, dv);
    return (i != j) && (dot3(dv, dv) < ETA * ETA * Tj.h2);
}

/* y[r] = sum_j A_{rows[r], j} x_j for nrows rows (rows == NULL: all rows, in
 * order); x and y interleaved complex; x may hold nrhs columns of length nt
 * (column-major), y then holds nrhs columns of length nrows. */
void orc_matvec(const double *verts, const int32_t *tris, int64_t nt, double k, const double *x, int nrhs,
                const int64_t *rows, int64_t nrows, double *y, int nthreads)
{
    g_part = 0;
    tri_t *T = build_all(verts, tris, nt);
    set_threads(nthreads);
    const cplx *xc = (const cplx *)x;
    cplx *yc = (cplx *)y;
    int64_t nr = rows ? nrows : nt;
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t r = 0; r < nr; ++r) {
        int64_t i = rows ? rows[r] : r;
        cplx acc[64];
        int nb = nrhs < 64 ? nrhs : 64;
        for (int c0 = 0; c0 < nrhs; c0 += nb) {
            int cn = (nrhs - c0) < nb ? (nrhs - c0) : nb;
            for (int c = 0; c < cn; ++c) acc[c] = 0.0;
            for (int64_t j = 0; j < nt; ++j) {
                cplx a = entry(&T[i], &T[j], i == j, k);
                for (int c = 0; c < cn; ++c) acc[c] += a * xc[(int64_t)(c0 + c) * nt + j];
            }
            for (int c = 0; c < cn; ++c) yc[(int64_t)(c0 + c) * nr + r] = acc[c];
        }
    }
    free(T);
}

/* dense A, row-major [nt, nt] interleaved complex (small meshes only) */
void orc_assemble(const double *verts, const int32_t *tris, int64_t nt, double k, double *A, int nthreads)
{
    g_part = 0;
    tri_t *T = build_all(verts, tris, nt);
    set_threads(nthreads);
    cplx *Ac = (cplx *)A;
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t i = 0; i < nt; ++i)
        for (int64_t j = 0; j < nt; ++j) Ac[i * nt + j] = entry(&T[i], &T[j], i == j, k);
    free(T);
}

/* plane-wave right-hand side of Eq. eq_bm for a sound-hard body
 * (du/dn = 0): b_i = u_inc(x_i) + alpha du_inc/dn(x_i), u_inc = e^{ik d.x},
 * for nrhs directions dirs[nrhs, 3]; b column-major [nrhs][nt] */
void orc_rhs_plane_wave(const double *verts, const int32_t *tris, int64_t nt, double k, const double *dirs,
                        int nrhs, double *b)
{
    cplx *bc = (cplx *)b;
    cplx alpha = g_alpha_sign * I / k;
    for (int m = 0; m < nrhs; ++m)
        for (int64_t t = 0; t < nt; ++t) {
            tri_t T;
            make_tri(verts, tris, t, &T);
            const double *d = dirs + 3 * m;
            cplx uinc = cexp(I * k * dot3(d, T.c));
            cplx dudn = I * k * dot3(d, T.n) * uinc;
            bc[(int64_t)m * nt + t] = uinc + alpha * dudn;
        }
}

/* point-source right-hand side of Eq. eq_bm for a sound-hard body
 * (du/dn = 0) and u_inc = G(x, x_s): b_i = G(x_i, x_s) + alpha dG/dn_x(x_i, x_s)
 * for nrhs sources src[nrhs, 3] off the surface; b column-major [nrhs][nt] */
void orc_rhs_point_source(const double *verts, const int32_t *tris, int64_t nt, double k, const double *src,
                          int nrhs, double *b)
{
    cplx *bc = (cplx *)b;
    cplx alpha = g_alpha_sign * I / k;
    for (int m = 0; m < nrhs; ++m)
        for (int64_t t = 0; t < nt; ++t) {
            tri_t T;
            make_tri(verts, tris, t, &T);
            cplx o[4];
            kernels_all(T.c, T.n, src + 3 * m, T.n, k, o);
            bc[(int64_t)m * nt + t] = o[0] + alpha * o[2];
        }
}

/* ------------------------------------------------------------------ */
/* fields off the surface                                              */
/* ------------------------------------------------------------------ */
/* Green's representation in the acoustic domain (Eq. cbie with c = 1, n
 * into the body): u(x) = u_inc(x) + int G(x, y) q(y) dy - int dG/dn_y(x, y) u(y) dy.
 * Scattered part at npts points pts[npts, 3] (off the surface) from the
 * element values u (and q, NULL = 0), six-point rule per element. */
void orc_scattered_field(const double *verts, const int32_t *tris, int64_t nt, double k, const double *u,
                         const double *q, const double *pts, int64_t npts, double *out, int nthreads)
{
    tri_t *T = build_all(verts, tris, nt);
    set_threads(nthreads);
    const cplx *uc = (const cplx *)u, *qc = (const cplx *)q;
    cplx *oc = (cplx *)out;
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t p = 0; p < npts; ++p) {
        const double *x = pts + 3 * p;
        cplx acc = 0.0;
        for (int64_t j = 0; j < nt; ++j) {
            cplx sg = 0.0, sd = 0.0;
            for (int g = 0; g < 2; ++g) {
                double a = R6_A[g], b = 1.0 - 2.0 * R6_A[g];
                double bary[3][3] = {{b, a, a}, {a, b, a}, {a, a, b}};
                for (int r = 0; r < 3; ++r) {
                    double y[3];
                    for (int d = 0; d < 3; ++d)
                        y[d] = bary[r][0] * T[j].v[0][d] + bary[r][1] * T[j].v[1][d] + bary[r][2] * T[j].v[2][d];
                    cplx o[4];
                    kernels_all(x, T[j].n, y, T[j].n, k, o);
                    sg += R6_W[g] * T[j].area * o[0];
                    sd += R6_W[g] * T[j].area * o[1];
                }
            }
            acc += (qc ? sg * qc[j] : 0.0) - sd * uc[j];
        }
        oc[p] = acc;
    }
    free(T);
}

/* Far-field pattern F of the scattered field, u_sc ~ e^{ik|x|}/|x| F(xh):
 *   F(xh) = (1/(4 pi)) int [ q(y) + ik (xh . n_y) u(y) ] e^{-ik xh . y} dy
 * (the large-|x| limit of the representation above), for ndir unit
 * directions dirs[ndir, 3]; six-point rule per element. */
void orc_far_field(const double *verts, const int32_t *tris, int64_t nt, double k, const double *u,
                   const double *q, const double *dirs, int64_t ndir, double *out, int nthreads)
{
    tri_t *T = build_all(verts, tris, nt);
    set_threads(nthreads);
    const cplx *uc = (const cplx *)u, *qc = (const cplx *)q;
    cplx *oc = (cplx *)out;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t m = 0; m < ndir; ++m) {
        const double *xh = dirs + 3 * m;
        cplx acc = 0.0;
        for (int64_t j = 0; j < nt; ++j) {
            cplx se = 0.0;
            for (int g = 0; g < 2; ++g) {
                double a = R6_A[g], b = 1.0 - 2.0 * R6_A[g];
                double bary[3][3] = {{b, a, a}, {a, b, a}, {a, a, b}};
                for (int r = 0; r < 3; ++r) {
                    double y[3];
                    for (int d = 0; d < 3; ++d)
                        y[d] = bary[r][0] * T[j].v[0][d] + bary[r][1] * T[j].v[1][d] + bary[r][2] * T[j].v[2][d];
                    se += R6_W[g] * T[j].area * cexp(-I * k * dot3(xh, y));
                }
            }
            acc += se * ((qc ? qc[j] : 0.0) + I * k * dot3(xh, T[j].n) * uc[j]);
        }
        oc[m] = acc / (4.0 * ORC_PI);
    }
    free(T);
}
