// Sec. 3.1 / 3.3 Step 1 (equivalent and check points) and Sec. 4
// (compressed translations), in FP64 on the device.
//
// Per active level l (box width w):
//   low frequency  (kernel-independent FMM surfaces): upward equivalent points
//       on the cube surface of half-width 1.05 w/2, upward check points on the
//       cube of half-width 2.95 w/2, p_lf points per edge;
//   high frequency (directional, Sec. 3.1): upward equivalent points on the
//       sphere of radius 1.05 (sqrt 3/2) w (the cube-surface grid projected
//       radially, p_hf per edge), which encloses the box in every rotated
//       frame; upward check points in the cone of half-angle Theta around +z
//       from r_min = (rho - sqrt 3/2) w out to the size of the boundary
//       (diameter + 2w), on hf_nr shells uniform in 1/r (dense at the small
//       end) with hf_na directions each (Fibonacci points on the cap).  Theta
//       = the largest angle between a face cell's centre direction and its
//       corners plus 1.3 asin((sqrt 3/2)/rho) for the extent of the target
//       boxes.  Cone u uses the same points transformed by the orthogonal
//       R_u (+z -> centre direction of u; R_u = g_u R_rep, a signed axis
//       permutation of a representative cone's frame), so one SVD serves
//       every cone of a level (the rotation invariance of Sec. 4.1.1), and
//       M2L offsets related by the g_u share one operator.
//   The downward sets are the upward sets with roles swapped (check on the
//   equivalent set, equivalent on the check set), so G_dn = G_up^T and one
//   truncated SVD G_up ~ U S V^H (Eq. svdg, epsg: sigma_i >= eps sigma_0)
//   gives U_dn = conj(V), V_dn = conj(U).
// Compressed operators (Sec. 4.1.2 and 4.3), with E the kernel matrices
// between the point sets involved:
//   S~ = S^-1 U^H E_up(sources)           (per leaf)
//   M~ = S_l^-1 U_l^H E_up V_{l+1}        (per octant and cone)
//   K~ = U_dn^H K V_up = V^T K V          (per distinct M2L offset, Eq. cmpm2l)
//   L~ = U_dn,l+1^H E_dn V_dn,l S_l^-1 = V_{l+1}^T E conj(U_l) S_l^-1
//   T~ = E_t V_dn S^-1 = E_t conj(U) S^-1 (per leaf)
// The SVD is taken as the Hermitian eigen-decomposition of G^H G by a
// cyclic Jacobi method (all singular values kept are >= eps sigma_0, so the
// squared spectrum stays far above FP64 round-off).
#include <cooperative_groups.h>
#include <math.h>

#include <algorithm>
#include <numeric>
#include <vector>

#include "fda_internal.cuh"

namespace cg = cooperative_groups;

int fda_cone_index_host(double dx, double dy, double dz, int nc);
void fda_cone_symmetry(int nc, std::vector<int> &rep, std::vector<int> &g);

namespace {

// ---------------------------------------------------------------------------
// host point sets
// ---------------------------------------------------------------------------
std::vector<double> cube_surface(int p)
{
    std::vector<double> v;
    for (int i = 0; i < p; ++i)
        for (int j = 0; j < p; ++j)
            for (int l = 0; l < p; ++l) {
                if (!(i == 0 || i == p - 1 || j == 0 || j == p - 1 || l == 0 || l == p - 1)) continue;
                v.push_back(-1.0 + 2.0 * i / (p - 1));
                v.push_back(-1.0 + 2.0 * j / (p - 1));
                v.push_back(-1.0 + 2.0 * l / (p - 1));
            }
    return v;
}

void cone_dir_host(int ci, int nc, double d[3])
{
    int face = ci / (nc * nc), rem = ci % (nc * nc);
    int a = rem / nc, b = rem % nc;
    int ax = face / 2, s = face % 2;
    int o0 = ax == 0 ? 1 : 0, o1 = ax == 2 ? 1 : 2;
    d[ax] = s ? 1.0 : -1.0;
    d[o0] = -1.0 + (2.0 * a + 1.0) / nc;
    d[o1] = -1.0 + (2.0 * b + 1.0) / nc;
    double n = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    for (int t = 0; t < 3; ++t) d[t] /= n;
}

// rotation (row-major) taking +z to d
void rot_to_host(const double d[3], double R[9])
{
    double a[3] = {fabs(d[0]) < 0.9 ? 1.0 : 0.0, fabs(d[0]) < 0.9 ? 0.0 : 1.0, 0.0};
    double e1[3] = {a[1] * d[2] - a[2] * d[1], a[2] * d[0] - a[0] * d[2], a[0] * d[1] - a[1] * d[0]};
    double n = sqrt(e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2]);
    for (int t = 0; t < 3; ++t) e1[t] /= n;
    double e2[3] = {d[1] * e1[2] - d[2] * e1[1], d[2] * e1[0] - d[0] * e1[2], d[0] * e1[1] - d[1] * e1[0]};
    for (int r = 0; r < 3; ++r) {
        R[3 * r + 0] = e1[r];
        R[3 * r + 1] = e2[r];
        R[3 * r + 2] = d[r];
    }
}

double cone_halfangle_host(int nc)
{
    double best = 0;
    for (int a = 0; a < nc; ++a)
        for (int b = 0; b < nc; ++b) {
            double c[3] = {-1.0 + (2.0 * a + 1.0) / nc, -1.0 + (2.0 * b + 1.0) / nc, 1.0};
            double cn = sqrt(c[0] * c[0] + c[1] * c[1] + 1.0);
            for (int ca = a; ca <= a + 1; ++ca)
                for (int cb = b; cb <= b + 1; ++cb) {
                    double r[3] = {-1.0 + 2.0 * ca / nc, -1.0 + 2.0 * cb / nc, 1.0};
                    double rn = sqrt(r[0] * r[0] + r[1] * r[1] + 1.0);
                    double cosv = (c[0] * r[0] + c[1] * r[1] + 1.0) / (cn * rn);
                    best = std::max(best, acos(std::min(1.0, cosv)));
                }
        }
    return best;
}

std::vector<double> cone_points(double theta, double rmin, double rmax, int nr, int na)
{
    std::vector<double> v;
    const double ga = FDA_PI * (3.0 - sqrt(5.0));
    for (int i = 0; i < nr; ++i) {
        double u = cos(FDA_PI * (i + 0.5) / nr);
        double inv = 0.5 * (1.0 / rmin + 1.0 / rmax) + 0.5 * (1.0 / rmin - 1.0 / rmax) * u;
        double r = 1.0 / inv;
        double rot = i * 2.39996;
        for (int j = 0; j < na; ++j) {
            double jj = j + 0.5;
            double z = 1.0 - (1.0 - cos(theta)) * jj / na;
            double rr = sqrt(std::max(0.0, 1.0 - z * z));
            double ph = jj * ga + rot;
            v.push_back(r * rr * cos(ph));
            v.push_back(r * rr * sin(ph));
            v.push_back(r * z);
        }
    }
    return v;
}

// ---------------------------------------------------------------------------
// device kernels
// ---------------------------------------------------------------------------
struct pts_desc {
    const double *base;  // [n][3]
    int n;
    double R[9];         // row-major rotation
    double t[3];         // translation
};

struct kmat_job {
    pts_desc X, Y;       // rows: X, columns: Y
    c64d *out;           // column-major, ld = X.n
};

__device__ inline void apply_pt(const pts_desc &d, int i, double p[3])
{
    const double *b = d.base + 3 * i;
    for (int r = 0; r < 3; ++r) p[r] = d.R[3 * r] * b[0] + d.R[3 * r + 1] * b[1] + d.R[3 * r + 2] * b[2] + d.t[r];
}

// G(x, y) = e^{ikr}/(4 pi r) between two point sets
__global__ void k_kmat(const kmat_job *jobs, double k)
{
    const kmat_job &J = jobs[blockIdx.y];
    int64_t n = (int64_t)J.X.n * J.Y.n;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        int i = (int)(e % J.X.n), j = (int)(e / J.X.n);
        double x[3], y[3];
        apply_pt(J.X, i, x);
        apply_pt(J.Y, j, y);
        double r = sqrt((x[0] - y[0]) * (x[0] - y[0]) + (x[1] - y[1]) * (x[1] - y[1]) + (x[2] - y[2]) * (x[2] - y[2]));
        double s, c;
        sincos(k * r, &s, &c);
        double f = 1.0 / (4.0 * FDA_PI * r);
        J.out[e] = c64d(c * f, s * f);
    }
}

// S2M sources: E[c][j] = sum_q w_jq dG/dn_y(x_c, y_jq) (SIDE 0, the double
// layer of the unknown u) or sum_q w_jq G(x_c, y_jq) (SIDE 1, the single
// layer of given Neumann data), x_c = check points of the leaf, j < n_B
// (padded to 64 columns)
template <int SIDE>
__global__ void k_emat_s2m(const double *chk, int nchk, const double *centers, const int32_t *leaf_list,
                           const int32_t *leaf_box, const int32_t *bbeg, const int32_t *bend, const double *qpt,
                           const double *qw, const double *nrm, double k, c64d *out)
{
    int b = blockIdx.y;
    int li = leaf_list[b];
    int B = leaf_box[li];
    int j0 = bbeg[B], nB = bend[B] - j0;
    const double *ctr = centers + 3 * (int64_t)b;
    c64d *E = out + (int64_t)b * nchk * 64;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nchk * 64; e += gridDim.x * blockDim.x) {
        int c = e % nchk, jl = e / nchk;
        c64d acc;
        if (jl < nB) {
            int j = j0 + jl;
            double x[3] = {chk[3 * c] + ctr[0], chk[3 * c + 1] + ctr[1], chk[3 * c + 2] + ctr[2]};
            const double *ny = nrm + 3 * (int64_t)j;
            for (int q = 0; q < 6; ++q) {
                const double *y = qpt + 18 * (int64_t)j + 3 * q;
                double r0 = x[0] - y[0], r1 = x[1] - y[1], r2 = x[2] - y[2];
                double R2 = r0 * r0 + r1 * r1 + r2 * r2, R = sqrt(R2);
                double s, cc;
                sincos(k * R, &s, &cc);
                if (SIDE == 1) {
                    double g = qw[6 * (int64_t)j + q] / (4.0 * FDA_PI * R);
                    acc.re += g * cc;
                    acc.im += g * s;
                    continue;
                }
                double f = qw[6 * (int64_t)j + q] * (r0 * ny[0] + r1 * ny[1] + r2 * ny[2]) / (4.0 * FDA_PI * R2 * R);
                // e^{ikR}(1 - ikR) f
                acc.re += f * (cc + k * R * s);
                acc.im += f * (s - k * R * cc);
            }
        }
        E[e] = acc;
    }
}

// L2T: E[i][m] = G(x_i, y_m) + alpha dG/dn_x(x_i, y_m), i < n_B (64 rows),
// y_m = downward equivalent points of the leaf
__global__ void k_emat_l2t(const double *eq, int neq, const double *centers, const int32_t *leaf_list,
                           const int32_t *leaf_box, const int32_t *bbeg, const int32_t *bend, const double *cent,
                           const double *nrm, double k, double as, c64d *out)
{
    int b = blockIdx.y;
    int li = leaf_list[b];
    int B = leaf_box[li];
    int i0 = bbeg[B], nB = bend[B] - i0;
    const double *ctr = centers + 3 * (int64_t)b;
    c64d *E = out + (int64_t)b * 64 * neq;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < 64 * neq; e += gridDim.x * blockDim.x) {
        int il = e % 64, m = e / 64;
        c64d v;
        if (il < nB) {
            int i = i0 + il;
            const double *x = cent + 3 * (int64_t)i, *nx = nrm + 3 * (int64_t)i;
            double y[3] = {eq[3 * m] + ctr[0], eq[3 * m + 1] + ctr[1], eq[3 * m + 2] + ctr[2]};
            double r0 = x[0] - y[0], r1 = x[1] - y[1], r2 = x[2] - y[2];
            double R2 = r0 * r0 + r1 * r1 + r2 * r2, R = sqrt(R2);
            double s, cc;
            sincos(k * R, &s, &cc);
            double g = 1.0 / (4.0 * FDA_PI * R);
            double rnx = r0 * nx[0] + r1 * nx[1] + r2 * nx[2];
            // dG/dn_x = -e^{ikR}(1 - ikR) rnx/(4 pi R^3); alpha = as i/k
            double f = -rnx / (4.0 * FDA_PI * R2 * R);
            double dre = f * (cc + k * R * s), dim = f * (s - k * R * cc);
            v = c64d(cc * g - as * dim / k, s * g + as * dre / k);
        }
        E[e] = v;  // column-major 64 x neq
    }
}

// batched complex FP64 GEMM, column-major: C = op(A) op(B)
// opA: 0 N (M x K, lda), 1 T, 2 H (A stored K x M);  opB: 0 N, 1 conj (K x N)
struct gemm_job {
    const c64d *A, *B;
    c64d *C;
};

constexpr int GT = 32, GK = 16;

__global__ void k_zgemm(const gemm_job *jobs, int M, int N, int K, int lda, int ldb, int ldc, int opA, int opB)
{
    __shared__ c64d As[GK][GT + 1], Bs[GK][GT + 1];
    const gemm_job J = jobs[blockIdx.z];
    int tx = threadIdx.x % 16, ty = threadIdx.x / 16;  // 256 threads
    int i0 = blockIdx.x * GT, j0 = blockIdx.y * GT;
    c64d acc[2][2];
    for (int k0 = 0; k0 < K; k0 += GK) {
        for (int e = threadIdx.x; e < GK * GT; e += 256) {
            int kk = e / GT, ii = e % GT;
            int gi = i0 + ii, gk = k0 + kk;
            c64d a;
            if (gi < M && gk < K) {
                if (opA == 0) a = J.A[gi + (int64_t)gk * lda];
                else {
                    a = J.A[gk + (int64_t)gi * lda];
                    if (opA == 2) a.im = -a.im;
                }
            }
            As[kk][ii] = a;
            int gj = j0 + ii;
            c64d b;
            if (gj < N && gk < K) {
                b = J.B[gk + (int64_t)gj * ldb];
                if (opB == 1) b.im = -b.im;
            }
            Bs[kk][ii] = b;
        }
        __syncthreads();
        for (int kk = 0; kk < GK; ++kk) {
            c64d a0 = As[kk][tx], a1 = As[kk][tx + 16];
            c64d b0 = Bs[kk][ty], b1 = Bs[kk][ty + 16];
            cfma(acc[0][0], a0, b0);
            cfma(acc[1][0], a1, b0);
            cfma(acc[0][1], a0, b1);
            cfma(acc[1][1], a1, b1);
        }
        __syncthreads();
    }
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) {
            int gi = i0 + tx + 16 * a, gj = j0 + ty + 16 * b;
            if (gi < M && gj < N) J.C[gi + (int64_t)gj * ldc] = acc[a][b];
        }
}

// C[:, j] *= s[j] (col) or C[i, :] *= s[i] (row), inverse of sigma
__global__ void k_scale_inv(c64d *C, int M, int N, int ldc, int64_t stride, const double *sig, int by_row)
{
    c64d *c = C + blockIdx.y * stride;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)M * N;
         e += (int64_t)gridDim.x * blockDim.x) {
        int i = (int)(e % M), j = (int)(e / M);
        double f = 1.0 / sig[by_row ? i : j];
        c64d &v = c[i + (int64_t)j * ldc];
        v.re *= f;
        v.im *= f;
    }
}

// cyclic Jacobi for a Hermitian n x n matrix (column-major, in place), with
// eigenvectors accumulated in V; round-robin pairing, cooperative grid
__global__ void k_jacobi(c64d *A, c64d *V, int n, int npad, int max_sweeps, double *scratch, int *sweeps_done)
{
    cg::grid_group grid = cg::this_grid();
    int nthreads = gridDim.x * blockDim.x;
    int tid = blockIdx.x * blockDim.x + threadIdx.x;
    double *rot = scratch;       // per pair: cs, sn, cos(phi), sin(phi)
    double *off = scratch + 4 * (npad / 2);
    int *pairs = (int *)(scratch + 4 * (npad / 2) + 2);
    int half = npad / 2;
    for (int e = tid; e < n * n; e += nthreads) V[e] = c64d((e % n) == (e / n) ? 1.0 : 0.0, 0.0);
    grid.sync();
    int sweep = 0;
    double hist[3] = {0.0, 0.0, 0.0};  // off-diagonal mass of the last three sweeps
    // accepted floor of the off-diagonal mass once it stalls (large n): an
    // off-diagonal norm of 1e-10 of the diagonal's perturbs the kept singular
    // vectors (sigma >= eps sigma_0, eps >= 1e-6) far below eps
    const double floor_rel = 1e-20;
    for (; sweep < max_sweeps; ++sweep) {
        // convergence measure
        if (tid == 0) {
            off[0] = 0.0;
            off[1] = 0.0;
        }
        grid.sync();
        double so = 0.0, sd = 0.0;
        for (int e = tid; e < n * n; e += nthreads) {
            int i = e % n, j = e / n;
            double m2 = A[e].re * A[e].re + A[e].im * A[e].im;
            if (i == j) sd += m2; else so += m2;
        }
        for (int o = 16; o > 0; o >>= 1) {
            so += __shfl_xor_sync(0xffffffffu, so, o);
            sd += __shfl_xor_sync(0xffffffffu, sd, o);
        }
        if ((threadIdx.x & 31) == 0) {
            atomicAdd(&off[0], so);
            atomicAdd(&off[1], sd);
        }
        grid.sync();
        // stop when the off-diagonal part is at FP64 round-off of the diagonal,
        // or when it has stalled for three sweeps below the accepted floor
        // (rounding in the rotations of a large matrix)
        const double o0 = off[0], d0 = off[1];
        if (o0 <= 1e-26 * d0) break;
        if (sweep >= 3 && o0 > 0.5 * hist[0] && o0 <= floor_rel * d0) break;
        hist[0] = hist[1];
        hist[1] = hist[2];
        hist[2] = o0;
        for (int r = 0; r < npad - 1; ++r) {
            // pairs of this round and their rotations
            for (int q = tid; q < half; q += nthreads) {
                int a = q == 0 ? 0 : ((q - 1 + r) % (npad - 1)) + 1;
                int b = ((npad - 1 - q - 1 + r) % (npad - 1)) + 1;
                int p = min(a, b), s = max(a, b);
                pairs[2 * q] = p;
                pairs[2 * q + 1] = s;
                double cs = 1.0, sn = 0.0, cph = 1.0, sph = 0.0;
                if (s < n) {
                    c64d apq = A[p + (int64_t)s * n];
                    double mag = sqrt(apq.re * apq.re + apq.im * apq.im);
                    double app = A[p + (int64_t)p * n].re, aqq = A[s + (int64_t)s * n].re;
                    if (mag > 1e-300 && mag > 1e-18 * sqrt(fabs(app * aqq))) {
                        cph = apq.re / mag;
                        sph = apq.im / mag;
                        double zeta = (aqq - app) / (2.0 * mag);
                        double t = (zeta >= 0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
                        cs = 1.0 / sqrt(1.0 + t * t);
                        sn = t * cs;
                    }
                }
                rot[4 * q] = cs;
                rot[4 * q + 1] = sn;
                rot[4 * q + 2] = cph;
                rot[4 * q + 3] = sph;
            }
            grid.sync();
            // columns of A and V: A J, J = [[cs, sn], [-sn e^{-i phi}, cs e^{-i phi}]]
            for (int e = tid; e < 2 * half * n; e += nthreads) {
                int which = e / (half * n);
                int rem = e % (half * n);
                int q = rem / n, i = rem % n;
                int p = pairs[2 * q], s = pairs[2 * q + 1];
                if (s >= n) continue;
                double cs = rot[4 * q], sn = rot[4 * q + 1];
                c64d em(rot[4 * q + 2], -rot[4 * q + 3]);  // e^{-i phi}
                c64d *M = which ? V : A;
                c64d xp = M[i + (int64_t)p * n], xq = M[i + (int64_t)s * n];
                c64d xqe = xq * em;
                M[i + (int64_t)p * n] = c64d(cs * xp.re - sn * xqe.re, cs * xp.im - sn * xqe.im);
                M[i + (int64_t)s * n] = c64d(sn * xp.re + cs * xqe.re, sn * xp.im + cs * xqe.im);
            }
            grid.sync();
            // rows of A: J^H A
            for (int e = tid; e < half * n; e += nthreads) {
                int q = e / n, j = e % n;
                int p = pairs[2 * q], s = pairs[2 * q + 1];
                if (s >= n) continue;
                double cs = rot[4 * q], sn = rot[4 * q + 1];
                c64d ep(rot[4 * q + 2], rot[4 * q + 3]);  // e^{+i phi}
                c64d xp = A[p + (int64_t)j * n], xq = A[s + (int64_t)j * n];
                c64d xqe = xq * ep;
                A[p + (int64_t)j * n] = c64d(cs * xp.re - sn * xqe.re, cs * xp.im - sn * xqe.im);
                A[s + (int64_t)j * n] = c64d(sn * xp.re + cs * xqe.re, sn * xp.im + cs * xqe.im);
            }
            grid.sync();
        }
    }
    if (tid == 0) *sweeps_done = sweep;
}

__global__ void k_gather_cols(const c64d *V, int n, const int *order, int T, c64d *out)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)n * T;
         e += (int64_t)gridDim.x * blockDim.x) {
        int i = (int)(e % n), t = (int)(e / n);
        out[e] = V[i + (int64_t)order[t] * n];
    }
}

__global__ void k_diag(const c64d *A, int n, double *d)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) d[i] = A[i + (int64_t)i * n].re;
}

// ---- low-rank reduced M2L operators (Sec. 4.2, Eq. epsk)
// Column-pivoted modified Gram-Schmidt of one m x n column-major matrix per
// CTA, in place (A becomes the residual of the retained columns): at each
// step the remaining column of largest norm is orthogonalised once more
// against the chosen ones, normalised and stored as the next column of Q,
// and projected out of every remaining column.  It stops when the squared
// Frobenius norm of the remaining columns is at most (tol_rel x the largest
// initial column norm)^2, or after kmax columns (rank[] = kmax + 1 then:
// not converged).  Q (m x kmax) is zero beyond the rank.  m <= 1024.
constexpr int QRT = 256;

__global__ void __launch_bounds__(QRT) k_cpqr(c64d *A, int m, int n, int64_t sA, c64d *Q, int64_t sQ, int kmax,
                                              double tol_rel, int *rank, double *colmax2)
{
    extern __shared__ double qr_smem[];
    double *nrm = qr_smem;                                   // [n]
    c64d *q = reinterpret_cast<c64d *>(qr_smem + n + (n & 1));  // [m]
    __shared__ double red_v[QRT / 32];
    __shared__ int red_i[QRT / 32];
    __shared__ c64d coef[1024];
    __shared__ double s_tol2, s_tot;
    __shared__ int s_piv;
    c64d *a = A + (int64_t)blockIdx.x * sA;
    c64d *Qm = Q + (int64_t)blockIdx.x * sQ;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, nw = QRT / 32;
    for (int j = warp; j < n; j += nw) {
        double s = 0.0;
        for (int r = lane; r < m; r += 32) s += a[r + (int64_t)j * m].re * a[r + (int64_t)j * m].re + a[r + (int64_t)j * m].im * a[r + (int64_t)j * m].im;
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) nrm[j] = s;
    }
    for (int e = tid; e < m * kmax; e += QRT) Qm[e] = c64d();
    __syncthreads();
    int k = 0;
    bool done = false;
    for (; k <= kmax; ++k) {
        // remaining mass and pivot
        double tot = 0.0, best = -1.0;
        int bi = -1;
        for (int j = tid; j < n; j += QRT) {
            const double v = nrm[j];
            if (v >= 0.0) {
                tot += v;
                if (v > best) { best = v; bi = j; }
            }
        }
        for (int o = 16; o > 0; o >>= 1) {
            tot += __shfl_xor_sync(0xffffffffu, tot, o);
            const double ob = __shfl_xor_sync(0xffffffffu, best, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (ob > best || (ob == best && oi >= 0 && (bi < 0 || oi < bi))) { best = ob; bi = oi; }
        }
        if (lane == 0) { red_v[warp] = best; red_i[warp] = bi; coef[warp] = c64d(tot, 0.0); }
        __syncthreads();
        if (tid == 0) {
            double b2 = -1.0, t2 = 0.0;
            int i2 = -1;
            for (int w = 0; w < nw; ++w) {
                t2 += coef[w].re;
                if (red_v[w] > b2 || (red_v[w] == b2 && red_i[w] >= 0 && (i2 < 0 || red_i[w] < i2))) { b2 = red_v[w]; i2 = red_i[w]; }
            }
            if (k == 0) {
                s_tol2 = tol_rel * tol_rel * fmax(b2, 0.0);
                if (colmax2) colmax2[blockIdx.x] = fmax(b2, 0.0);
            }
            s_tot = t2;
            s_piv = i2;
        }
        __syncthreads();
        if (s_tot <= s_tol2 || s_piv < 0) { done = true; break; }
        if (k == kmax) break;
        const int p = s_piv;
        for (int r = tid; r < m; r += QRT) q[r] = a[r + (int64_t)p * m];
        __syncthreads();
        // one more orthogonalisation against the chosen columns
        for (int i = warp; i < k; i += nw) {
            c64d c;
            for (int r = lane; r < m; r += 32) cfma_conj(c, Qm[r + (int64_t)i * m], q[r]);
            for (int o = 16; o > 0; o >>= 1) {
                c.re += __shfl_xor_sync(0xffffffffu, c.re, o);
                c.im += __shfl_xor_sync(0xffffffffu, c.im, o);
            }
            if (lane == 0) coef[i] = c;
        }
        __syncthreads();
        for (int r = tid; r < m; r += QRT) {
            c64d v = q[r];
            for (int i = 0; i < k; ++i) {
                const c64d t = coef[i] * Qm[r + (int64_t)i * m];
                v.re -= t.re;
                v.im -= t.im;
            }
            q[r] = v;
        }
        __syncthreads();
        if (warp == 0) {
            double s = 0.0;
            for (int r = lane; r < m; r += 32) s += q[r].re * q[r].re + q[r].im * q[r].im;
            for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            if (lane == 0) red_v[0] = s > 0.0 ? 1.0 / sqrt(s) : 0.0;
        }
        __syncthreads();
        const double inv = red_v[0];
        for (int r = tid; r < m; r += QRT) {
            const c64d v(q[r].re * inv, q[r].im * inv);
            q[r] = v;
            Qm[r + (int64_t)k * m] = v;
        }
        if (tid == 0) nrm[p] = -1.0;
        __syncthreads();
        // project q out of the remaining columns, fresh norms
        for (int j = warp; j < n; j += nw) {
            if (nrm[j] < 0.0) continue;
            c64d c;
            for (int r = lane; r < m; r += 32) cfma_conj(c, q[r], a[r + (int64_t)j * m]);
            for (int o = 16; o > 0; o >>= 1) {
                c.re += __shfl_xor_sync(0xffffffffu, c.re, o);
                c.im += __shfl_xor_sync(0xffffffffu, c.im, o);
            }
            double s = 0.0;
            for (int r = lane; r < m; r += 32) {
                c64d v = a[r + (int64_t)j * m];
                const c64d t = c * q[r];
                v.re -= t.re;
                v.im -= t.im;
                a[r + (int64_t)j * m] = v;
                s += v.re * v.re + v.im * v.im;
            }
            for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            if (lane == 0) nrm[j] = s;
        }
        __syncthreads();
    }
    if (tid == 0) rank[blockIdx.x] = done ? k : kmax + 1;
}

// err2[b] = || K_b - U_b Q_b^H ||_F^2 and ref2[b] = (largest column norm of
// K_b)^2 for T x T operators K, U and Q of T x r columns (column-major).
__global__ void k_lr_check(const c64d *K, const c64d *U, const c64d *Qm, int T, int r, double *err2, double *ref2)
{
    __shared__ double se[QRT / 32], sr[QRT / 32];
    const int b = blockIdx.x, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const c64d *Kb = K + (int64_t)b * T * T, *Ub = U + (int64_t)b * T * r, *Qb = Qm + (int64_t)b * T * r;
    double e = 0.0, mx = 0.0;
    for (int j = warp; j < T; j += QRT / 32) {
        double cn = 0.0;
        for (int i = lane; i < T; i += 32) {
            c64d v = Kb[i + (int64_t)j * T];
            cn += v.re * v.re + v.im * v.im;
            for (int t = 0; t < r; ++t) {
                const c64d u = Ub[i + (int64_t)t * T], qq = Qb[j + (int64_t)t * T];
                // v -= u conj(qq)
                v.re -= u.re * qq.re + u.im * qq.im;
                v.im -= u.im * qq.re - u.re * qq.im;
            }
            e += v.re * v.re + v.im * v.im;
        }
        for (int o = 16; o > 0; o >>= 1) cn += __shfl_xor_sync(0xffffffffu, cn, o);
        mx = fmax(mx, cn);
    }
    for (int o = 16; o > 0; o >>= 1) e += __shfl_xor_sync(0xffffffffu, e, o);
    if (lane == 0) {
        se[warp] = e;
        sr[warp] = mx;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, m = 0.0;
        for (int w = 0; w < QRT / 32; ++w) {
            a += se[w];
            m = fmax(m, sr[w]);
        }
        err2[b] = a;
        ref2[b] = m;
    }
}

// bucket factors: U^ (T x rpad) from U (T x rcap) and V^ = Q^H (rpad x T)
// from Q (T x rcap), for the bucket's operators ops[b]
__global__ void k_lr_gather(const c64d *U, const c64d *Qm, int T, int rcap, const int32_t *ops, int rpad, c64d *Ub,
                            c64d *Vb)
{
    const int b = blockIdx.y, o = ops[b];
    const c64d *Uo = U + (int64_t)o * T * rcap, *Qo = Qm + (int64_t)o * T * rcap;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)T * rpad;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(e % T), j = (int)(e / T);  // U^(i, j)
        Ub[(int64_t)b * T * rpad + e] = j < rcap ? Uo[i + (int64_t)j * T] : c64d();
        // V^(j, i) = conj(Q(i, j)), column-major rpad x T
        const c64d q = j < rcap ? Qo[i + (int64_t)j * T] : c64d();
        Vb[(int64_t)b * T * rpad + j + (int64_t)i * rpad] = c64d(q.re, -q.im);
    }
}

__global__ void k_f64_to_f32(const c64d *a, c32f *b, int64_t n)
{
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
        b[t] = c32f((float)a[t].re, (float)a[t].im);
}

// ---------------------------------------------------------------------------
// host orchestration helpers
// ---------------------------------------------------------------------------
struct level_pts {
    std::vector<double> eq, chk;  // box-relative, scaled
    std::vector<double> rot;      // [ncones][9]
};

void run_kmat(fda_handle *h, const std::vector<kmat_job> &jobs)
{
    if (jobs.empty()) return;
    dbuf dj;
    dj.alloc(sizeof(kmat_job) * jobs.size());
    FDA_CUDA(cudaMemcpyAsync(dj.p, jobs.data(), sizeof(kmat_job) * jobs.size(), cudaMemcpyHostToDevice, h->stream));
    int64_t n = (int64_t)jobs[0].X.n * jobs[0].Y.n;
    unsigned gx = (unsigned)std::min<int64_t>((n + 255) / 256, 1024);
    for (size_t b0 = 0; b0 < jobs.size(); b0 += 65535) {
        unsigned nb = (unsigned)std::min<size_t>(65535, jobs.size() - b0);
        k_kmat<<<dim3(gx, nb), 256, 0, h->stream>>>(dj.as<kmat_job>() + b0, h->k);
        FDA_CHECK_LAUNCH();
    }
    FDA_CUDA(cudaStreamSynchronize(h->stream));
}

void run_gemm(fda_handle *h, const std::vector<gemm_job> &jobs, int M, int N, int K, int lda, int ldb, int ldc,
              int opA, int opB)
{
    if (jobs.empty()) return;
    dbuf dj;
    dj.alloc(sizeof(gemm_job) * jobs.size());
    FDA_CUDA(cudaMemcpyAsync(dj.p, jobs.data(), sizeof(gemm_job) * jobs.size(), cudaMemcpyHostToDevice, h->stream));
    for (size_t b0 = 0; b0 < jobs.size(); b0 += 65535) {
        unsigned nb = (unsigned)std::min<size_t>(65535, jobs.size() - b0);
        dim3 g((M + GT - 1) / GT, (N + GT - 1) / GT, nb);
        k_zgemm<<<g, 256, 0, h->stream>>>(dj.as<gemm_job>() + b0, M, N, K, lda, ldb, ldc, opA, opB);
        FDA_CHECK_LAUNCH();
    }
    FDA_CUDA(cudaStreamSynchronize(h->stream));
}

pts_desc make_desc(const double *base, int n, const double *R, double tx, double ty, double tz)
{
    pts_desc d;
    d.base = base;
    d.n = n;
    static const double I[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
    for (int t = 0; t < 9; ++t) d.R[t] = R ? R[t] : I[t];
    d.t[0] = tx;
    d.t[1] = ty;
    d.t[2] = tz;
    return d;
}

// truncated SVD of G (m x n, column-major device) -> U (m x T), V (n x T), sig
int truncated_svd(fda_handle *h, const c64d *G, int m, int n, double eps, dbuf &U, dbuf &V, dbuf &sig)
{
    cudaStream_t s = h->stream;
    dbuf gram, vecs, scratch, sweeps;
    gram.alloc(sizeof(c64d) * n * n);
    vecs.alloc(sizeof(c64d) * n * n);
    int npad = n + (n & 1);
    scratch.alloc(sizeof(double) * (4 * (npad / 2) + 2) + sizeof(int) * npad + 64);
    sweeps.alloc(sizeof(int));
    run_gemm(h, {gemm_job{G, G, gram.as<c64d>()}}, n, n, m, m, m, n, 2, 0);
    int dev = 0, nsm = 0, per_sm = 0;
    FDA_CUDA(cudaGetDevice(&dev));
    FDA_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    FDA_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_jacobi, 256, 0));
    int grid = std::max(1, std::min(nsm * std::max(per_sm, 1), std::max(1, (n * n) / 2048)));
    c64d *Ap = gram.as<c64d>(), *Vp = vecs.as<c64d>();
    double *scp = scratch.as<double>();
    int *swp = sweeps.as<int>();
    int max_sweeps = 60;
    void *args[] = {&Ap, &Vp, &n, &npad, &max_sweeps, &scp, &swp};
    FDA_CUDA(cudaLaunchCooperativeKernel((void *)k_jacobi, grid, 256, args, 0, s));
    FDA_CHECK_LAUNCH();
    dbuf dg;
    dg.alloc(sizeof(double) * n);
    k_diag<<<fda_blocks(n, 128), 128, 0, s>>>(gram.as<c64d>(), n, dg.as<double>());
    FDA_CHECK_LAUNCH();
    std::vector<double> lam(n);
    int hsw = 0;
    FDA_CUDA(cudaMemcpyAsync(lam.data(), dg.p, sizeof(double) * n, cudaMemcpyDeviceToHost, s));
    FDA_CUDA(cudaMemcpyAsync(&hsw, swp, sizeof(int), cudaMemcpyDeviceToHost, s));
    FDA_CUDA(cudaStreamSynchronize(s));
    if (hsw >= max_sweeps) fda_fail(FDA_ERR_NUMERIC, "Jacobi eigen-solver did not converge");
    std::vector<int> order(n);
    std::iota(order.begin(), order.end(), 0);
    std::sort(order.begin(), order.end(), [&](int a, int b) { return lam[a] > lam[b]; });
    double s0 = sqrt(std::max(lam[order[0]], 0.0));
    if (!(s0 > 0)) fda_fail(FDA_ERR_NUMERIC, "zero operator in truncated SVD");
    int T = 0;
    std::vector<double> hs;
    for (int t = 0; t < n; ++t) {
        double sv = sqrt(std::max(lam[order[t]], 0.0));
        if (sv < eps * s0) break;
        hs.push_back(sv);
        ++T;
    }
    dbuf dord;
    dord.alloc(sizeof(int) * T);
    FDA_CUDA(cudaMemcpyAsync(dord.p, order.data(), sizeof(int) * T, cudaMemcpyHostToDevice, s));
    V.alloc(sizeof(c64d) * n * T);
    k_gather_cols<<<256, 256, 0, s>>>(vecs.as<c64d>(), n, dord.as<int>(), T, V.as<c64d>());
    FDA_CHECK_LAUNCH();
    sig.alloc(sizeof(double) * T);
    FDA_CUDA(cudaMemcpyAsync(sig.p, hs.data(), sizeof(double) * T, cudaMemcpyHostToDevice, s));
    U.alloc(sizeof(c64d) * m * T);
    run_gemm(h, {gemm_job{G, V.as<c64d>(), U.as<c64d>()}}, m, T, n, m, n, m, 0, 0);
    k_scale_inv<<<dim3(256, 1), 256, 0, s>>>(U.as<c64d>(), m, T, m, 0, sig.as<double>(), 0);
    FDA_CHECK_LAUNCH();
    FDA_CUDA(cudaStreamSynchronize(s));
    return T;
}

void box_center_host(const fda_handle *h, const int32_t *coord, int level, double c[3])
{
    double w = h->lev[level].w;
    for (int d = 0; d < 3; ++d) c[d] = h->root_lo[d] + (coord[d] + 0.5) * w;
}

}  // namespace

// cone at level l+1 containing cone u of level l (both high frequency)
int fda_child_cone(const fda_handle *h, int l, int u)
{
    int ncp = h->lev[l].nc, ncc = h->lev[l + 1].nc;
    int face = u / (ncp * ncp), rem = u % (ncp * ncp);
    int a = rem / ncp, b = rem % ncp;
    int f = ncp / ncc;
    return face * ncc * ncc + (a / f) * ncc + (b / f);
}

// Per-leaf S~ (and, for side 0, T~) at the active levels (leaves are low
// frequency).  side 0: S~ of the double-layer sources and T~; side 1: S~ of
// the single-layer sources of the right-hand side's layers (same check
// points, pseudo-inverse and layout).
static void leaf_operators(fda_handle *h, int side)
{
    cudaStream_t s = h->stream;
    const int nlev = h->nlev;
    std::vector<int32_t> hbox_coord(3 * (size_t)h->nbox_total), hleaf_box(h->nleaf);
    std::vector<int32_t> hbeg(h->nbox_total), hend(h->nbox_total);
    FDA_CUDA(cudaMemcpy(hbox_coord.data(), h->box_coord.p, 12 * (size_t)h->nbox_total, cudaMemcpyDeviceToHost));
    FDA_CUDA(cudaMemcpy(hleaf_box.data(), h->leaf_box.p, 4 * (size_t)h->nleaf, cudaMemcpyDeviceToHost));
    FDA_CUDA(cudaMemcpy(hbeg.data(), h->box_begin.p, 4 * (size_t)h->nbox_total, cudaMemcpyDeviceToHost));
    FDA_CUDA(cudaMemcpy(hend.data(), h->box_end.p, 4 * (size_t)h->nbox_total, cudaMemcpyDeviceToHost));
    std::vector<int64_t> off(h->nleaf + 1, 0);
    for (int li = 0; li < h->nleaf; ++li) {
        int l = h->h_leaf_level[li];
        int T = h->lev[l].active ? h->lev[l].T : 0;
        off[li + 1] = off[li] + (int64_t)64 * T;
    }
    dbuf &St = side ? h->op64.St1 : h->op64.St;
    if (side == 0) {
        h->leaf_T_off.assign(off.begin(), off.end() - 1);
        h->leaf_op_off.alloc(sizeof(int64_t) * (h->nleaf + 1));
        FDA_CUDA(cudaMemcpy(h->leaf_op_off.p, off.data(), sizeof(int64_t) * (h->nleaf + 1), cudaMemcpyHostToDevice));
        h->op64.Tt.alloc(sizeof(c64d) * std::max<int64_t>(off[h->nleaf], 1));
        FDA_CUDA(cudaMemset(h->op64.Tt.p, 0, sizeof(c64d) * std::max<int64_t>(off[h->nleaf], 1)));
    }
    St.alloc(sizeof(c64d) * std::max<int64_t>(off[h->nleaf], 1));
    FDA_CUDA(cudaMemset(St.p, 0, sizeof(c64d) * std::max<int64_t>(off[h->nleaf], 1)));
    for (int l = h->lev_lo; l < nlev; ++l) {
        level_info &L = h->lev[l];
        std::vector<int32_t> lv;
        for (int li = 0; li < h->nleaf; ++li)
            if (h->h_leaf_level[li] == l) lv.push_back(li);
        if (lv.empty()) continue;
        const int T = L.T, nchk = L.n_chk, neq = L.n_eq;
        const int chunk = std::max(1, (int)std::min<int64_t>(4096, (int64_t)(768ll << 20) / (16ll * 64 * nchk)));
        dbuf dlist, dctr, E, R;
        dlist.alloc(sizeof(int32_t) * chunk);
        dctr.alloc(sizeof(double) * 3 * chunk);
        E.alloc(sizeof(c64d) * (size_t)chunk * 64 * std::max(nchk, neq));
        R.alloc(sizeof(c64d) * (size_t)chunk * 64 * T);
        for (size_t c0 = 0; c0 < lv.size(); c0 += chunk) {
            int nb = (int)std::min<size_t>(chunk, lv.size() - c0);
            std::vector<double> ctr(3 * nb);
            for (int b = 0; b < nb; ++b) box_center_host(h, &hbox_coord[3 * (size_t)hleaf_box[lv[c0 + b]]], l, &ctr[3 * b]);
            FDA_CUDA(cudaMemcpy(dlist.p, &lv[c0], 4 * nb, cudaMemcpyHostToDevice));
            FDA_CUDA(cudaMemcpy(dctr.p, ctr.data(), 8 * 3 * nb, cudaMemcpyHostToDevice));
            // S2M: E_s (nchk x 64) then S~ = S^-1 U^H E_s  (T x 64), stored as [64][T]
            auto emat = side ? k_emat_s2m<1> : k_emat_s2m<0>;
            emat<<<dim3(32, nb), 256, 0, s>>>(h->chk_up[l].as<double>(), nchk, dctr.as<double>(),
                                                   dlist.as<int32_t>(), h->leaf_box.as<int32_t>(),
                                                   h->box_begin.as<int32_t>(), h->box_end.as<int32_t>(),
                                                   h->qpt.as<double>(), h->qw.as<double>(), h->nrm.as<double>(),
                                                   h->k, E.as<c64d>());
            FDA_CHECK_LAUNCH();
            std::vector<gemm_job> gj(nb);
            for (int b = 0; b < nb; ++b)
                gj[b] = gemm_job{h->Uup[l].as<c64d>(), E.as<c64d>() + (size_t)b * nchk * 64,
                                 St.as<c64d>() + off[lv[c0 + b]]};
            run_gemm(h, gj, T, 64, nchk, nchk, nchk, T, 2, 0);
            for (int b = 0; b < nb; ++b) {
                k_scale_inv<<<dim3(16, 1), 256, 0, s>>>(St.as<c64d>() + off[lv[c0 + b]], T, 64, T, 0,
                                                        h->sig[l].as<double>(), 1);
            }
            FDA_CHECK_LAUNCH();
            if (side) continue;
            // L2T: E_t (64 x n_eq_dn = nchk) then T~ = E_t conj(U) S^-1 (64 x T)
            k_emat_l2t<<<dim3(32, nb), 256, 0, s>>>(h->chk_up[l].as<double>(), nchk, dctr.as<double>(),
                                                   dlist.as<int32_t>(), h->leaf_box.as<int32_t>(),
                                                   h->box_begin.as<int32_t>(), h->box_end.as<int32_t>(),
                                                   h->cent.as<double>(), h->nrm.as<double>(), h->k,
                                                   h->cfg.alpha_sign, E.as<c64d>());
            FDA_CHECK_LAUNCH();
            for (int b = 0; b < nb; ++b)
                gj[b] = gemm_job{E.as<c64d>() + (size_t)b * 64 * nchk, h->Uup[l].as<c64d>(),
                                 h->op64.Tt.as<c64d>() + off[lv[c0 + b]]};
            run_gemm(h, gj, 64, T, nchk, 64, nchk, 64, 0, 1);
            for (int b = 0; b < nb; ++b) {
                k_scale_inv<<<dim3(16, 1), 256, 0, s>>>(h->op64.Tt.as<c64d>() + off[lv[c0 + b]], 64, T, 64, 0,
                                                        h->sig[l].as<double>(), 0);
            }
            FDA_CHECK_LAUNCH();
        }
    }
}

// Sec. 4.2: truncated low-rank factorisation of every reduced M2L operator
// K~_o of level l in FP64, K~_o ~= (K~_o Q) Q^H with Q (T x r) orthonormal.
// A randomized range sketch (Y = K~ Omega, s columns, Omega Gaussian) and a
// pivoted Gram-Schmidt of Y give a basis Q1 of K~'s range; a pivoted
// Gram-Schmidt of C = K~^H Q1 = (Q1^H K~)^H, stopped when the Frobenius norm
// of what remains is at most eps times its largest column norm, gives the
// row-space basis Q of rank r (Eq. epsk, in the Frobenius norm).  Every
// factorisation is checked explicitly: ||K~ - U^ V^||_F <= eps times the
// larger of the largest column norms of K~ and of C (both lower bounds of
// sigma_0); an operator that fails the check or needs r >= T/2 stays in full
// form.  Operators whose
// two-stage application (rank padded to 32) is cheaper than the full one,
// both in flops (2 r T < T^2) and in tensor-core tiles (64 rows, 32 of K),
// are grouped by padded rank.
static void lowrank_level(fda_handle *h, int l)
{
    level_info &L = h->lev[l];
    const int T = L.T, nops = L.n_ops;
    h->op_rank[l].assign(std::max(nops, 0), -1);
    h->op_bucket[l].assign(std::max(nops, 0), -1);
    h->lr[l].clear();
    const int rcap = (T - 1) / 2;  // r < T/2
    if (!h->cfg.lowrank || nops == 0 || T > 1024 || 2 * 32 >= T) return;
    const int sk = std::min(T, rcap + 16);
    const double eps = h->cfg.eps;
    cudaStream_t st = h->stream;
    // Gaussian test matrix (splitmix64 and the Box-Muller transform), T x sk
    std::vector<c64d> om((size_t)T * sk);
    uint64_t z = 0x2545f4914f6cdd1dull + 0x9e3779b97f4a7c15ull * (uint64_t)(l + 1);
    auto next = [&]() {
        z += 0x9e3779b97f4a7c15ull;
        uint64_t x = z;
        x = (x ^ (x >> 30)) * 0xbf58476d1ce4e5b9ull;
        x = (x ^ (x >> 27)) * 0x94d049bb133111ebull;
        return x ^ (x >> 31);
    };
    for (auto &v : om) {
        const double u1 = ((double)(next() >> 11) + 0.5) / 9007199254740992.0;
        const double u2 = ((double)(next() >> 11) + 0.5) / 9007199254740992.0;
        const double rr = sqrt(-2.0 * log(u1));
        v = c64d(rr * cos(2.0 * FDA_PI * u2), rr * sin(2.0 * FDA_PI * u2));
    }
    dbuf Om, Uall, Qall;
    Om.alloc(sizeof(c64d) * om.size());
    FDA_CUDA(cudaMemcpy(Om.p, om.data(), sizeof(c64d) * om.size(), cudaMemcpyHostToDevice));
    Uall.alloc(sizeof(c64d) * (size_t)nops * T * rcap);
    Qall.alloc(sizeof(c64d) * (size_t)nops * T * rcap);
    const int chunk = std::max(1, std::min(nops, (int)((512ll << 20) / (16ll * T * (2 * sk)))));
    dbuf Y, Q1, C, rk1, rk2, e2, r2, c2;
    Y.alloc(sizeof(c64d) * (size_t)chunk * T * sk);
    Q1.alloc(sizeof(c64d) * (size_t)chunk * T * sk);
    C.alloc(sizeof(c64d) * (size_t)chunk * T * sk);
    rk1.alloc(sizeof(int) * chunk);
    rk2.alloc(sizeof(int) * chunk);
    e2.alloc(sizeof(double) * chunk);
    r2.alloc(sizeof(double) * chunk);
    c2.alloc(sizeof(double) * chunk);
    const size_t qsm = sizeof(double) * (sk + (sk & 1)) + sizeof(c64d) * T;
    const c64d *K = h->op64.Kt[l].as<c64d>();
    std::vector<int> hr(chunk);
    std::vector<double> he(chunk), hq(chunk), hc(chunk);
    for (int o0 = 0; o0 < nops; o0 += chunk) {
        const int nb = std::min(chunk, nops - o0);
        std::vector<gemm_job> g1(nb), g2(nb), g3(nb);
        for (int b = 0; b < nb; ++b) {
            const c64d *Ko = K + (size_t)(o0 + b) * T * T;
            g1[b] = gemm_job{Ko, Om.as<c64d>(), Y.as<c64d>() + (size_t)b * T * sk};
            g2[b] = gemm_job{Ko, Q1.as<c64d>() + (size_t)b * T * sk, C.as<c64d>() + (size_t)b * T * sk};
            g3[b] = gemm_job{Ko, Qall.as<c64d>() + (size_t)(o0 + b) * T * rcap,
                             Uall.as<c64d>() + (size_t)(o0 + b) * T * rcap};
        }
        run_gemm(h, g1, T, sk, T, T, T, T, 0, 0);  // Y = K~ Omega
        k_cpqr<<<nb, QRT, qsm, st>>>(Y.as<c64d>(), T, sk, (int64_t)T * sk, Q1.as<c64d>(), (int64_t)T * sk, sk,
                                     0.01 * eps, rk1.as<int>(), nullptr);
        FDA_CHECK_LAUNCH();
        run_gemm(h, g2, T, sk, T, T, T, T, 2, 0);  // C = K~^H Q1
        k_cpqr<<<nb, QRT, qsm, st>>>(C.as<c64d>(), T, sk, (int64_t)T * sk,
                                     Qall.as<c64d>() + (size_t)o0 * T * rcap, (int64_t)T * rcap, rcap, eps,
                                     rk2.as<int>(), c2.as<double>());
        FDA_CHECK_LAUNCH();
        run_gemm(h, g3, T, rcap, T, T, T, T, 0, 0);  // U^ = K~ Q
        k_lr_check<<<nb, QRT, 0, st>>>(K + (size_t)o0 * T * T, Uall.as<c64d>() + (size_t)o0 * T * rcap,
                                       Qall.as<c64d>() + (size_t)o0 * T * rcap, T, rcap, e2.as<double>(),
                                       r2.as<double>());
        FDA_CHECK_LAUNCH();
        FDA_CUDA(cudaMemcpyAsync(hr.data(), rk2.p, sizeof(int) * nb, cudaMemcpyDeviceToHost, st));
        FDA_CUDA(cudaMemcpyAsync(he.data(), e2.p, sizeof(double) * nb, cudaMemcpyDeviceToHost, st));
        FDA_CUDA(cudaMemcpyAsync(hq.data(), r2.p, sizeof(double) * nb, cudaMemcpyDeviceToHost, st));
        FDA_CUDA(cudaMemcpyAsync(hc.data(), c2.p, sizeof(double) * nb, cudaMemcpyDeviceToHost, st));
        FDA_CUDA(cudaStreamSynchronize(st));
        for (int b = 0; b < nb; ++b) {
            // both column maxima (of K~ and of C = K~^H Q1) are lower bounds of sigma_0^2
            const bool ok = hr[b] >= 1 && hr[b] <= rcap && std::isfinite(he[b]) &&
                            he[b] <= eps * eps * std::max(hq[b], hc[b]);
            h->op_rank[l][o0 + b] = ok ? hr[b] : -1;
        }
    }
    // buckets of padded rank where the two stages are cheaper
    auto nrt = [](int x) { return (x + 63) / 64; };
    auto nkc = [](int x) { return (x + 31) / 32; };
    std::vector<int> bucket_of_rpad(T + 1, -1);
    for (int o = 0; o < nops; ++o) {
        const int r = h->op_rank[l][o];
        if (r < 1) continue;
        const int rpad = (r + 31) / 32 * 32;
        const int cost_full = nrt(T) * nkc(T), cost_lr = nrt(rpad) * nkc(T) + nrt(T) * nkc(rpad);
        if (2 * rpad >= T || cost_lr >= cost_full) continue;
        if (bucket_of_rpad[rpad] < 0) {
            bucket_of_rpad[rpad] = (int)h->lr[l].size();
            h->lr[l].emplace_back();
            h->lr[l].back().rpad = rpad;
        }
        const int b = bucket_of_rpad[rpad];
        h->op_bucket[l][o] = b;
        h->lr[l][b].ops.push_back(o);
    }
    for (lr_bucket &B : h->lr[l]) {
        const int nb = (int)B.ops.size();
        dbuf dops;
        dops.alloc(sizeof(int32_t) * nb);
        FDA_CUDA(cudaMemcpy(dops.p, B.ops.data(), sizeof(int32_t) * nb, cudaMemcpyHostToDevice));
        B.U64.alloc(sizeof(c64d) * (size_t)nb * T * B.rpad);
        B.V64.alloc(sizeof(c64d) * (size_t)nb * T * B.rpad);
        k_lr_gather<<<dim3(64, nb), 256, 0, st>>>(Uall.as<c64d>(), Qall.as<c64d>(), T, rcap, dops.as<int32_t>(),
                                                  B.rpad, B.U64.as<c64d>(), B.V64.as<c64d>());
        FDA_CHECK_LAUNCH();
    }
    FDA_CUDA(cudaStreamSynchronize(st));
}

void fda_far_precompute(fda_handle *h)
{
    cudaStream_t s = h->stream;
    const fda_config &cfg = h->cfg;
    if (h->lev_lo < 0) return;  // no far field at all
    const int nlev = h->nlev;
    std::vector<level_pts> P(nlev);
    // ---- point sets and truncated SVDs
    for (int l = h->lev_lo; l < nlev; ++l) {
        level_info &L = h->lev[l];
        double w = L.w;
        if (!L.hf) {
            std::vector<double> c = cube_surface(cfg.p_lf);
            for (double v : c) {
                P[l].eq.push_back(v * 1.05 * w / 2);
                P[l].chk.push_back(v * 2.95 * w / 2);
            }
        } else {
            std::vector<double> c = cube_surface(cfg.p_hf);
            double rad = 1.05 * sqrt(3.0) / 2.0 * w;
            for (size_t i = 0; i < c.size(); i += 3) {
                double n = sqrt(c[i] * c[i] + c[i + 1] * c[i + 1] + c[i + 2] * c[i + 2]);
                for (int d = 0; d < 3; ++d) P[l].eq.push_back(c[i + d] / n * rad);
            }
            double rmin = (L.rho - sqrt(3.0) / 2.0) * w;
            double rmax = h->diam + 2.0 * w;
            if (rmax < 1.5 * rmin) rmax = 1.5 * rmin;
            double delta = 1.3 * asin(std::min(1.0, (sqrt(3.0) / 2.0) / L.rho));
            double theta = std::min(0.999 * FDA_PI / 2.0, cone_halfangle_host(L.nc) + delta);
            P[l].chk = cone_points(theta, rmin, rmax, cfg.hf_nr, cfg.hf_na);
            // R_u = g_u R_rep(u): a rotation taking +z to the representative
            // cone's centre, mapped to cone u by a signed axis permutation
            std::vector<int> crep, cg;
            fda_cone_symmetry(L.nc, crep, cg);
            for (int u = 0; u < L.ncones; ++u) {
                double d[3], R0[9], R[9];
                cone_dir_host(crep[u], L.nc, d);
                rot_to_host(d, R0);
                const int *g = &cg[9 * (size_t)u];
                for (int i = 0; i < 3; ++i)
                    for (int j = 0; j < 3; ++j)
                        R[3 * i + j] = g[3 * i] * R0[j] + g[3 * i + 1] * R0[3 + j] + g[3 * i + 2] * R0[6 + j];
                P[l].rot.insert(P[l].rot.end(), R, R + 9);
            }
            h->rot[l].alloc(sizeof(double) * P[l].rot.size());
            FDA_CUDA(cudaMemcpy(h->rot[l].p, P[l].rot.data(), sizeof(double) * P[l].rot.size(),
                                cudaMemcpyHostToDevice));
        }
        L.n_eq = (int)P[l].eq.size() / 3;
        L.n_chk = (int)P[l].chk.size() / 3;
        h->eq_up[l].alloc(sizeof(double) * P[l].eq.size());
        h->chk_up[l].alloc(sizeof(double) * P[l].chk.size());
        FDA_CUDA(cudaMemcpy(h->eq_up[l].p, P[l].eq.data(), sizeof(double) * P[l].eq.size(), cudaMemcpyHostToDevice));
        FDA_CUDA(cudaMemcpy(h->chk_up[l].p, P[l].chk.data(), sizeof(double) * P[l].chk.size(),
                            cudaMemcpyHostToDevice));
        dbuf G;
        G.alloc(sizeof(c64d) * (size_t)L.n_chk * L.n_eq);
        kmat_job j;
        j.X = make_desc(h->chk_up[l].as<double>(), L.n_chk, nullptr, 0, 0, 0);
        j.Y = make_desc(h->eq_up[l].as<double>(), L.n_eq, nullptr, 0, 0, 0);
        j.out = G.as<c64d>();
        run_kmat(h, {j});
        L.T = truncated_svd(h, G.as<c64d>(), L.n_chk, L.n_eq, cfg.eps, h->Uup[l], h->Vup[l], h->sig[l]);
    }

    // ---- M2L operators: K~ = V^T K V, K = G(R_u eq (at 0), D w + R_ubar eq)
    for (int l = h->lev_lo; l < nlev; ++l) {
        level_info &L = h->lev[l];
        if (L.n_ops == 0) continue;
        const int n = L.n_eq, T = L.T;
        h->op64.Kt[l].alloc(sizeof(c64d) * (size_t)L.n_ops * T * T);
        const int chunk = std::max(1, (int)std::min<int64_t>(256, (int64_t)(512ll << 20) / (16ll * n * n)));
        dbuf Kbuf, KV;
        Kbuf.alloc(sizeof(c64d) * (size_t)chunk * n * n);
        KV.alloc(sizeof(c64d) * (size_t)chunk * n * T);
        for (int o0 = 0; o0 < L.n_ops; o0 += chunk) {
            int nb = std::min(chunk, L.n_ops - o0);
            std::vector<kmat_job> kj(nb);
            std::vector<gemm_job> g1(nb), g2(nb);
            for (int b = 0; b < nb; ++b) {
                int3 d = h->h_ops[l][o0 + b];
                const double *Ru = nullptr, *Rs = nullptr;
                if (L.hf) {
                    int u = fda_cone_index_host(d.x, d.y, d.z, L.nc);
                    int ub = fda_cone_index_host(-d.x, -d.y, -d.z, L.nc);
                    Ru = &P[l].rot[9 * u];
                    Rs = &P[l].rot[9 * ub];
                }
                kj[b].X = make_desc(h->eq_up[l].as<double>(), n, Ru, 0, 0, 0);
                kj[b].Y = make_desc(h->eq_up[l].as<double>(), n, Rs, d.x * L.w, d.y * L.w, d.z * L.w);
                kj[b].out = Kbuf.as<c64d>() + (size_t)b * n * n;
                g1[b] = gemm_job{kj[b].out, h->Vup[l].as<c64d>(), KV.as<c64d>() + (size_t)b * n * T};
                g2[b] = gemm_job{h->Vup[l].as<c64d>(), g1[b].C, h->op64.Kt[l].as<c64d>() + (size_t)(o0 + b) * T * T};
            }
            run_kmat(h, kj);
            run_gemm(h, g1, n, T, n, n, n, n, 0, 0);
            run_gemm(h, g2, T, T, n, n, n, T, 1, 0);
        }
        lowrank_level(h, l);
    }

    // ---- M2M and L2L operators (parent level l, child level l+1)
    for (int l = h->lev_lo; l + 1 < nlev; ++l) {
        level_info &L = h->lev[l], &C = h->lev[l + 1];
        const int nj = 8 * L.ncones;
        const int Tp = L.T, Tc = C.T;
        h->op64.Mt[l].alloc(sizeof(c64d) * (size_t)nj * Tp * Tc);
        h->op64.Lt[l].alloc(sizeof(c64d) * (size_t)nj * Tp * Tc);
        double wc = C.w;
        // M2M: E = G(R_u chk_P, c_o + R_uc eq_C): n_chk,P x n_eq,C
        {
            dbuf E, EV;
            E.alloc(sizeof(c64d) * (size_t)nj * L.n_chk * C.n_eq);
            EV.alloc(sizeof(c64d) * (size_t)nj * L.n_chk * Tc);
            std::vector<kmat_job> kj(nj);
            std::vector<gemm_job> g1(nj), g2(nj);
            for (int o = 0; o < 8; ++o)
                for (int u = 0; u < L.ncones; ++u) {
                    int b = o * L.ncones + u;
                    double cx = ((o >> 2) & 1 ? 0.5 : -0.5) * wc, cy = ((o >> 1) & 1 ? 0.5 : -0.5) * wc,
                           cz = (o & 1 ? 0.5 : -0.5) * wc;
                    const double *Ru = L.hf ? &P[l].rot[9 * u] : nullptr;
                    const double *Rc = C.hf ? &P[l + 1].rot[9 * fda_child_cone(h, l, u)] : nullptr;
                    kj[b].X = make_desc(h->chk_up[l].as<double>(), L.n_chk, Ru, 0, 0, 0);
                    kj[b].Y = make_desc(h->eq_up[l + 1].as<double>(), C.n_eq, Rc, cx, cy, cz);
                    kj[b].out = E.as<c64d>() + (size_t)b * L.n_chk * C.n_eq;
                    g1[b] = gemm_job{kj[b].out, h->Vup[l + 1].as<c64d>(), EV.as<c64d>() + (size_t)b * L.n_chk * Tc};
                    g2[b] = gemm_job{h->Uup[l].as<c64d>(), g1[b].C, h->op64.Mt[l].as<c64d>() + (size_t)b * Tp * Tc};
                }
            run_kmat(h, kj);
            run_gemm(h, g1, L.n_chk, Tc, C.n_eq, L.n_chk, C.n_eq, L.n_chk, 0, 0);
            run_gemm(h, g2, Tp, Tc, L.n_chk, L.n_chk, L.n_chk, Tp, 2, 0);
            k_scale_inv<<<dim3(64, nj), 256, 0, s>>>(h->op64.Mt[l].as<c64d>(), Tp, Tc, Tp, (int64_t)Tp * Tc,
                                                     h->sig[l].as<double>(), 1);
            FDA_CHECK_LAUNCH();
        }
        // L2L: E = G(c_o + R_uc eq_C (child's downward check set), R_u chk_P (parent's downward equivalent set))
        {
            dbuf E, EU;
            E.alloc(sizeof(c64d) * (size_t)nj * C.n_eq * L.n_chk);
            EU.alloc(sizeof(c64d) * (size_t)nj * C.n_eq * Tp);
            std::vector<kmat_job> kj(nj);
            std::vector<gemm_job> g1(nj), g2(nj);
            for (int o = 0; o < 8; ++o)
                for (int u = 0; u < L.ncones; ++u) {
                    int b = o * L.ncones + u;
                    double cx = ((o >> 2) & 1 ? 0.5 : -0.5) * wc, cy = ((o >> 1) & 1 ? 0.5 : -0.5) * wc,
                           cz = (o & 1 ? 0.5 : -0.5) * wc;
                    const double *Ru = L.hf ? &P[l].rot[9 * u] : nullptr;
                    const double *Rc = C.hf ? &P[l + 1].rot[9 * fda_child_cone(h, l, u)] : nullptr;
                    kj[b].X = make_desc(h->eq_up[l + 1].as<double>(), C.n_eq, Rc, cx, cy, cz);
                    kj[b].Y = make_desc(h->chk_up[l].as<double>(), L.n_chk, Ru, 0, 0, 0);
                    kj[b].out = E.as<c64d>() + (size_t)b * C.n_eq * L.n_chk;
                    g1[b] = gemm_job{kj[b].out, h->Uup[l].as<c64d>(), EU.as<c64d>() + (size_t)b * C.n_eq * Tp};
                    g2[b] = gemm_job{h->Vup[l + 1].as<c64d>(), g1[b].C, h->op64.Lt[l].as<c64d>() + (size_t)b * Tc * Tp};
                }
            run_kmat(h, kj);
            run_gemm(h, g1, C.n_eq, Tp, L.n_chk, C.n_eq, L.n_chk, C.n_eq, 0, 1);
            run_gemm(h, g2, Tc, Tp, C.n_eq, C.n_eq, C.n_eq, Tc, 1, 0);
            k_scale_inv<<<dim3(64, nj), 256, 0, s>>>(h->op64.Lt[l].as<c64d>(), Tc, Tp, Tc, (int64_t)Tc * Tp,
                                                     h->sig[l].as<double>(), 0);
            FDA_CHECK_LAUNCH();
        }
    }

    leaf_operators(h, 0);
    FDA_CUDA(cudaStreamSynchronize(s));
}

void fda_far_rhs_s2m(fda_handle *h)
{
    if (h->lev_lo < 0) return;
    leaf_operators(h, 1);
    FDA_CUDA(cudaStreamSynchronize(h->stream));
}

void fda_far_rhs_convert_f32(fda_handle *h)
{
    if (!h->op64.St1.p) return;
    int64_t n = (int64_t)(h->op64.St1.bytes / sizeof(c64d));
    h->op32.St1.alloc(sizeof(c32f) * n);
    k_f64_to_f32<<<1024, 256, 0, h->stream>>>(h->op64.St1.as<c64d>(), h->op32.St1.as<c32f>(), n);
    FDA_CHECK_LAUNCH();
    FDA_CUDA(cudaStreamSynchronize(h->stream));
}

// near field and single-layer S2M of the right-hand side's layers, once
void fda_rhs_layers_prepare(fda_handle *h)
{
    if (h->rhs_layers) return;
    fda_near_build(h, 1);
    fda_far_rhs_s2m(h);
    if (h->have32) {
        fda_near_convert_f32(h, 1);
        fda_far_rhs_convert_f32(h);
    }
    FDA_CUDA(cudaStreamSynchronize(h->stream));
    h->rhs_layers = 1;
}

// the FP32 L2T operators without the 64-row padding: leaf li's T columns of
// n_B rows, one after another from coff[li]
__global__ void k_compact_l2t(const c32f *Tt, const int64_t *off, const int64_t *coff, const int32_t *leaf_box,
                              const int32_t *bbeg, const int32_t *bend, int nleaf, c32f *out)
{
    const int li = blockIdx.x;
    if (li >= nleaf) return;
    const int B = leaf_box[li], nB = bend[B] - bbeg[B];
    const int T = (int)((off[li + 1] - off[li]) / 64);
    for (int e = threadIdx.x; e < T * nB; e += blockDim.x) {
        const int t = e / nB, i = e - t * nB;
        out[coff[li] + e] = Tt[off[li] + (int64_t)t * 64 + i];
    }
}

// FP32 copies of every far-field operator (chosen precision)
void fda_far_convert_f32(fda_handle *h)
{
    cudaStream_t s = h->stream;
    auto conv = [&](dbuf &src, dbuf &dst) {
        if (!src.p) return;
        int64_t n = (int64_t)(src.bytes / sizeof(c64d));
        dst.alloc(sizeof(c32f) * n);
        k_f64_to_f32<<<1024, 256, 0, s>>>(src.as<c64d>(), dst.as<c32f>(), n);
        FDA_CHECK_LAUNCH();
    };
    for (int l = 0; l < h->nlev; ++l) {
        conv(h->op64.Kt[l], h->op32.Kt[l]);
        conv(h->op64.Mt[l], h->op32.Mt[l]);
        conv(h->op64.Lt[l], h->op32.Lt[l]);
        for (lr_bucket &B : h->lr[l]) {
            conv(B.U64, B.U32);
            conv(B.V64, B.V32);
        }
    }
    conv(h->op64.St, h->op32.St);
    conv(h->op64.Tt, h->op32.Tt);
    if (h->op32.Tt.p && h->nleaf > 0) {
        const int NL = h->nleaf;
        std::vector<int32_t> lb(NL), bb(h->nbox_total), be(h->nbox_total);
        std::vector<int64_t> off(NL + 1), coff(NL + 1, 0);
        FDA_CUDA(cudaMemcpy(lb.data(), h->leaf_box.p, 4 * (size_t)NL, cudaMemcpyDeviceToHost));
        FDA_CUDA(cudaMemcpy(bb.data(), h->box_begin.p, 4 * bb.size(), cudaMemcpyDeviceToHost));
        FDA_CUDA(cudaMemcpy(be.data(), h->box_end.p, 4 * be.size(), cudaMemcpyDeviceToHost));
        FDA_CUDA(cudaMemcpy(off.data(), h->leaf_op_off.p, 8 * off.size(), cudaMemcpyDeviceToHost));
        for (int li = 0; li < NL; ++li)
            coff[li + 1] = coff[li] + (off[li + 1] - off[li]) / 64 * (be[lb[li]] - bb[lb[li]]);
        h->tt_c_off.alloc(8 * coff.size());
        FDA_CUDA(cudaMemcpy(h->tt_c_off.p, coff.data(), 8 * coff.size(), cudaMemcpyHostToDevice));
        h->tt32c.alloc(sizeof(c32f) * std::max<int64_t>(coff[NL], 1));
        k_compact_l2t<<<NL, 256, 0, s>>>(h->op32.Tt.as<c32f>(), h->leaf_op_off.as<int64_t>(),
                                         h->tt_c_off.as<int64_t>(), h->leaf_box.as<int32_t>(),
                                         h->box_begin.as<int32_t>(), h->box_end.as<int32_t>(), NL,
                                         h->tt32c.as<c32f>());
        FDA_CHECK_LAUNCH();
    }
    FDA_CUDA(cudaStreamSynchronize(s));
}
