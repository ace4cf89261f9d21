// Element geometry (Sec. 5: flat triangles, collocation at centroids,
// piecewise-constant basis), Morton ordering for the octree of Sec. 3.3
// Step 1, and the plane-wave right-hand side of Eq. eq_bm.
#include <math.h>

#include <algorithm>
#include <mutex>

#include "fda_internal.cuh"

namespace {

// Dunavant degree-4 six-point rule: barycentric (a, a, 1 - 2a) and
// permutations, weights relative to the triangle area.
__constant__ double c_r6a[2] = {0.44594849091596488632, 0.09157621350977074346};
__constant__ double c_r6w[2] = {0.22338158967801146570, 0.10995174365532186764};

__global__ void k_geometry(const double *verts, const int32_t *tris, int64_t nt, double *v9, double *cent,
                           double *nrm, double *area, double *h2, int *bad)
{
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= nt) return;
    double p[3][3];
    for (int a = 0; a < 3; ++a) {
        int64_t vi = tris[3 * t + a];
        for (int d = 0; d < 3; ++d) p[a][d] = verts[3 * vi + d];
    }
    for (int a = 0; a < 3; ++a)
        for (int d = 0; d < 3; ++d) v9[9 * t + 3 * a + d] = p[a][d];
    double e1[3], e2[3], e3[3];
    for (int d = 0; d < 3; ++d) {
        e1[d] = p[1][d] - p[0][d];
        e2[d] = p[2][d] - p[0][d];
        e3[d] = p[2][d] - p[1][d];
    }
    double nu[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
    double len = sqrt(nu[0] * nu[0] + nu[1] * nu[1] + nu[2] * nu[2]);
    double l1 = e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2];
    double l2 = e2[0] * e2[0] + e2[1] * e2[1] + e2[2] * e2[2];
    double l3 = e3[0] * e3[0] + e3[1] * e3[1] + e3[2] * e3[2];
    double hh = fmax(l1, fmax(l2, l3));
    if (!(len > 1e-14 * hh) || !(hh > 0)) atomicExch(bad, 1);
    for (int d = 0; d < 3; ++d) {
        cent[3 * t + d] = (p[0][d] + p[1][d] + p[2][d]) / 3.0;
        nrm[3 * t + d] = -nu[d] / len;
    }
    area[t] = 0.5 * len;
    h2[t] = hh;
}

__global__ void k_bbox(const double *cent, int64_t n, double *out)
{
    __shared__ double mn[3][256], mx[3][256];
    double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x)
        for (int d = 0; d < 3; ++d) {
            double v = cent[3 * i + d];
            lo[d] = fmin(lo[d], v);
            hi[d] = fmax(hi[d], v);
        }
    for (int d = 0; d < 3; ++d) {
        mn[d][threadIdx.x] = lo[d];
        mx[d][threadIdx.x] = hi[d];
    }
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s)
            for (int d = 0; d < 3; ++d) {
                mn[d][threadIdx.x] = fmin(mn[d][threadIdx.x], mn[d][threadIdx.x + s]);
                mx[d][threadIdx.x] = fmax(mx[d][threadIdx.x], mx[d][threadIdx.x + s]);
            }
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int d = 0; d < 3; ++d) {
            out[d] = mn[d][0];
            out[3 + d] = mx[d][0];
        }
}

__device__ inline uint64_t spread3(uint64_t v)
{
    // spread the low 21 bits of v so that bit j moves to bit 3j
    v &= 0x1fffffull;
    v = (v | (v << 32)) & 0x1f00000000ffffull;
    v = (v | (v << 16)) & 0x1f0000ff0000ffull;
    v = (v | (v << 8)) & 0x100f00f00f00f00full;
    v = (v | (v << 4)) & 0x10c30c30c30c30c3ull;
    v = (v | (v << 2)) & 0x1249249249249249ull;
    return v;
}

// Morton key at depth 20: bit 3j+2 = x_j, 3j+1 = y_j, 3j = z_j
__global__ void k_morton(const double *cent, int64_t n, double lx, double ly, double lz, double W, uint64_t *keys,
                         int32_t *idx)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double scale = (double)(1 << 20) / W;
    int64_t c[3];
    double lo[3] = {lx, ly, lz};
    for (int d = 0; d < 3; ++d) {
        int64_t v = (int64_t)floor((cent[3 * i + d] - lo[d]) * scale);
        c[d] = v < 0 ? 0 : (v > (1 << 20) - 1 ? (1 << 20) - 1 : v);
    }
    keys[i] = (spread3((uint64_t)c[0]) << 2) | (spread3((uint64_t)c[1]) << 1) | spread3((uint64_t)c[2]);
    idx[i] = (int32_t)i;
}

template <int W>
__global__ void k_gather_rows(const double *src, double *dst, const int32_t *perm, int64_t n)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    int64_t s = perm[i];
    for (int d = 0; d < W; ++d) dst[W * i + d] = src[W * s + d];
}

__global__ void k_inverse_perm(const int32_t *perm, int32_t *iperm, int64_t n)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) iperm[perm[i]] = (int32_t)i;
}

__global__ void k_quad_points(const double *v9, const double *area, int64_t n, double *qpt, double *qw)
{
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= n) return;
    const double *p = v9 + 9 * t;
    int q = 0;
    for (int g = 0; g < 2; ++g) {
        double a = c_r6a[g], b = 1.0 - 2.0 * c_r6a[g];
        double bary[3][3] = {{b, a, a}, {a, b, a}, {a, a, b}};
        for (int r = 0; r < 3; ++r, ++q) {
            for (int d = 0; d < 3; ++d)
                qpt[18 * t + 3 * q + d] = bary[r][0] * p[d] + bary[r][1] * p[3 + d] + bary[r][2] * p[6 + d];
            qw[6 * t + q] = c_r6w[g] * area[t];
        }
    }
}

// b_i = e^{ik d.x_i} (1 + alpha ik d.n_i), alpha = i/k (Eq. eq_bm, sound-hard)
__global__ void k_rhs(const double *cent, const double *nrm, int64_t n, const double *dirs, int nrhs, double k,
                      double as, c64d *b)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int m = blockIdx.y;
    if (i >= n || m >= nrhs) return;
    const double *d = dirs + 3 * m;
    double dx = d[0] * cent[3 * i] + d[1] * cent[3 * i + 1] + d[2] * cent[3 * i + 2];
    double dn = d[0] * nrm[3 * i] + d[1] * nrm[3 * i + 1] + d[2] * nrm[3 * i + 2];
    double s, c;
    sincos(k * dx, &s, &c);
    c64d uinc(c, s);
    // alpha * du_inc/dn = as (i/k)(ik dn) u_inc = -as dn u_inc
    c64d f(1.0 - as * dn, 0.0);
    b[(int64_t)m * n + i] = uinc * f;
}

__global__ void k_permute_c(const c64d *src, c64d *dst, const int32_t *map, int64_t n, int64_t lds, int64_t ldd,
                            int nrhs, int gather)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int m = blockIdx.y;
    if (i >= n || m >= nrhs) return;
    if (gather)
        dst[m * ldd + i] = src[m * lds + map[i]];
    else
        dst[m * ldd + map[i]] = src[m * lds + i];
}

// Right-hand side written straight into the caller's element order (no
// Morton-order staging vector): b[m][perm[i]] for sorted element i.
__global__ void k_rhs_direct(const double *cent, const double *nrm, const int32_t *perm, int64_t n,
                             const double *dirs, int nrhs, double k, double as, c64d *b)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int m = blockIdx.y;
    if (i >= n || m >= nrhs) return;
    const double *d = dirs + 3 * m;
    double dx = d[0] * cent[3 * i] + d[1] * cent[3 * i + 1] + d[2] * cent[3 * i + 2];
    double dn = d[0] * nrm[3 * i] + d[1] * nrm[3 * i + 1] + d[2] * nrm[3 * i + 2];
    double s, c;
    sincos(k * dx, &s, &c);
    b[(int64_t)m * n + perm[i]] = c64d(c * (1.0 - as * dn), s * (1.0 - as * dn));
}

// Point-source incidence u_inc = G(x, x_s) on a sound-hard body:
// b[m][perm[i]] = G(x_i, x_s) + alpha dG/dn_x(x_i, x_s), r = x_i - x_s.
__global__ void k_rhs_point(const double *cent, const double *nrm, const int32_t *perm, int64_t n,
                            const double *src, int nrhs, double k, double as, c64d *b)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int m = blockIdx.y;
    if (i >= n || m >= nrhs) return;
    const double *xs = src + 3 * m, *x = cent + 3 * i, *nx = nrm + 3 * i;
    double r0 = x[0] - xs[0], r1 = x[1] - xs[1], r2 = x[2] - xs[2];
    double R2 = r0 * r0 + r1 * r1 + r2 * r2, R = sqrt(R2);
    double sn, cs;
    sincos(k * R, &sn, &cs);
    double g = 1.0 / (4.0 * FDA_PI * R);
    double f = -(r0 * nx[0] + r1 * nx[1] + r2 * nx[2]) * g / R2;
    double dre = f * (cs + k * R * sn), dim = f * (sn - k * R * cs);
    b[(int64_t)m * n + perm[i]] = c64d(cs * g - as * dim / k, sn * g + as * dre / k);
}

}  // namespace

void fda_rhs_point(fda_handle *h, const double *src_dev, int nrhs, c64d *b)
{
    dim3 g(fda_blocks(h->N, 256), nrhs);
    k_rhs_point<<<g, 256, 0, h->stream>>>(h->cent.as<double>(), h->nrm.as<double>(), h->perm.as<int32_t>(), h->N,
                                           src_dev, nrhs, h->k, h->cfg.alpha_sign, b);
    FDA_CHECK_LAUNCH();
}

// Device-resident staging area for the incidence directions of
// fda_rhs_plane_wave_noalloc: FDA_NOALLOC_MAX_DIRS unit vectors (6 KB), held
// by every GPU that loads the library until the process exits.  All calls
// share it, so calls that overlap on the GPU (different streams, or several
// host threads) race on its contents.
static __device__ __align__(256) double g_noalloc_dirs[3 * FDA_NOALLOC_MAX_DIRS];

// Device address of g_noalloc_dirs, looked up once per device (with that
// device current) on the first call made on it.
static double *noalloc_dirs_ptr()
{
    static std::mutex mu;
    static double *ptrs[256] = {nullptr};
    int dev = 0;
    FDA_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 256) fda_fail(FDA_ERR_CUDA, "device index out of range");
    std::lock_guard<std::mutex> lock(mu);
    if (!ptrs[dev]) {
        double *p = nullptr;
        FDA_CUDA(cudaGetSymbolAddress((void **)&p, g_noalloc_dirs));
        ptrs[dev] = p;
    }
    return ptrs[dev];
}

// b (caller order, device) for nrhs <= FDA_NOALLOC_MAX_DIRS directions;
// allocates nothing.
void fda_rhs_noalloc(fda_handle *h, const double *dirs_host, int nrhs, c64d *b)
{
    double *dd = noalloc_dirs_ptr();
    FDA_CUDA(cudaMemcpyAsync(dd, dirs_host, sizeof(double) * 3 * nrhs, cudaMemcpyHostToDevice, h->stream));
    dim3 g(fda_blocks(h->N, 256), nrhs);
    k_rhs_direct<<<g, 256, 0, h->stream>>>(h->cent.as<double>(), h->nrm.as<double>(), h->perm.as<int32_t>(), h->N,
                                            dd, nrhs, h->k, h->cfg.alpha_sign, b);
    FDA_CHECK_LAUNCH();
}

void fda_geometry_build(fda_handle *h, const double *verts, int64_t nv, const int32_t *tris, int64_t nt)
{
    cudaStream_t s = h->stream;
    for (int64_t t = 0; t < 3 * nt; ++t)
        if (tris[t] < 0 || tris[t] >= nv) fda_fail(FDA_ERR_ARG, "triangle vertex index out of range");
    for (int64_t i = 0; i < 3 * nv; ++i)
        if (!std::isfinite(verts[i])) fda_fail(FDA_ERR_ARG, "non-finite vertex coordinate");
    h->N = nt;
    h->NV = nv;
    dbuf dv, dt, v9, cent, nrm, area, h2, bad;
    dv.alloc(sizeof(double) * 3 * nv);
    dt.alloc(sizeof(int32_t) * 3 * nt);
    FDA_CUDA(cudaMemcpyAsync(dv.p, verts, sizeof(double) * 3 * nv, cudaMemcpyHostToDevice, s));
    FDA_CUDA(cudaMemcpyAsync(dt.p, tris, sizeof(int32_t) * 3 * nt, cudaMemcpyHostToDevice, s));
    v9.alloc(sizeof(double) * 9 * nt);
    cent.alloc(sizeof(double) * 3 * nt);
    nrm.alloc(sizeof(double) * 3 * nt);
    area.alloc(sizeof(double) * nt);
    h2.alloc(sizeof(double) * nt);
    bad.alloc(sizeof(int));
    FDA_CUDA(cudaMemsetAsync(bad.p, 0, sizeof(int), s));
    k_geometry<<<fda_blocks(nt, 256), 256, 0, s>>>(dv.as<double>(), dt.as<int32_t>(), nt, v9.as<double>(),
                                                  cent.as<double>(), nrm.as<double>(), area.as<double>(),
                                                  h2.as<double>(), bad.as<int>());
    FDA_CHECK_LAUNCH();
    int hbad = 0;
    double bb[6];
    dbuf dbb;
    dbb.alloc(sizeof(double) * 6);
    k_bbox<<<1, 256, 0, s>>>(cent.as<double>(), nt, dbb.as<double>());
    FDA_CHECK_LAUNCH();
    FDA_CUDA(cudaMemcpyAsync(&hbad, bad.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    FDA_CUDA(cudaMemcpyAsync(bb, dbb.p, sizeof(bb), cudaMemcpyDeviceToHost, s));
    FDA_CUDA(cudaStreamSynchronize(s));
    if (hbad) fda_fail(FDA_ERR_ARG, "degenerate triangle (zero area)");
    double ext = std::max(bb[3] - bb[0], std::max(bb[4] - bb[1], bb[5] - bb[2]));
    double W = ext > 0 ? ext * (1.0 + 1e-6) : 1.0;
    for (int d = 0; d < 3; ++d) h->root_lo[d] = 0.5 * (bb[d] + bb[3 + d]) - 0.5 * W;
    h->W = W;
    h->diam = sqrt((bb[3] - bb[0]) * (bb[3] - bb[0]) + (bb[4] - bb[1]) * (bb[4] - bb[1]) +
                   (bb[5] - bb[2]) * (bb[5] - bb[2]));

    // Morton order
    h->keys.alloc(sizeof(uint64_t) * nt);
    h->perm.alloc(sizeof(int32_t) * nt);
    k_morton<<<fda_blocks(nt, 256), 256, 0, s>>>(cent.as<double>(), nt, h->root_lo[0], h->root_lo[1],
                                                h->root_lo[2], W, h->keys.as<uint64_t>(), h->perm.as<int32_t>());
    FDA_CHECK_LAUNCH();
    fda_radix_sort_u64(h->keys.as<uint64_t>(), h->perm.as<int32_t>(), nt, 60, s);
    h->iperm.alloc(sizeof(int32_t) * nt);
    k_inverse_perm<<<fda_blocks(nt, 256), 256, 0, s>>>(h->perm.as<int32_t>(), h->iperm.as<int32_t>(), nt);
    FDA_CHECK_LAUNCH();

    h->verts9.alloc(sizeof(double) * 9 * nt);
    h->cent.alloc(sizeof(double) * 3 * nt);
    h->nrm.alloc(sizeof(double) * 3 * nt);
    h->area.alloc(sizeof(double) * nt);
    h->h2.alloc(sizeof(double) * nt);
    const int32_t *pm = h->perm.as<int32_t>();
    unsigned g = fda_blocks(nt, 256);
    k_gather_rows<9><<<g, 256, 0, s>>>(v9.as<double>(), h->verts9.as<double>(), pm, nt);
    k_gather_rows<3><<<g, 256, 0, s>>>(cent.as<double>(), h->cent.as<double>(), pm, nt);
    k_gather_rows<3><<<g, 256, 0, s>>>(nrm.as<double>(), h->nrm.as<double>(), pm, nt);
    k_gather_rows<1><<<g, 256, 0, s>>>(area.as<double>(), h->area.as<double>(), pm, nt);
    k_gather_rows<1><<<g, 256, 0, s>>>(h2.as<double>(), h->h2.as<double>(), pm, nt);
    FDA_CHECK_LAUNCH();
    h->qpt.alloc(sizeof(double) * 18 * nt);
    h->qw.alloc(sizeof(double) * 6 * nt);
    k_quad_points<<<g, 256, 0, s>>>(h->verts9.as<double>(), h->area.as<double>(), nt, h->qpt.as<double>(),
                                    h->qw.as<double>());
    FDA_CHECK_LAUNCH();
    FDA_CUDA(cudaStreamSynchronize(s));
}

void fda_rhs_sorted(fda_handle *h, const double *dirs_dev, int nrhs, c64d *b_sorted)
{
    dim3 g(fda_blocks(h->N, 256), nrhs);
    k_rhs<<<g, 256, 0, h->stream>>>(h->cent.as<double>(), h->nrm.as<double>(), h->N, dirs_dev, nrhs, h->k,
                                     h->cfg.alpha_sign, b_sorted);
    FDA_CHECK_LAUNCH();
}

// x (caller order, one column) -> xs (Morton order)
void fda_gather_to_sorted(fda_handle *h, const c64d *x, c64d *xs)
{
    dim3 g(fda_blocks(h->N, 256), 1);
    k_permute_c<<<g, 256, 0, h->stream>>>(x, xs, h->perm.as<int32_t>(), h->N, h->N, h->N, 1, 1);
    FDA_CHECK_LAUNCH();
}

// nrhs columns at once: x (caller order, leading dimension ld) -> xs (Morton
// order, leading dimension N), on stream s
void fda_gather_cols(fda_handle *h, const c64d *x, int64_t ld, c64d *xs, int nrhs, cudaStream_t s)
{
    dim3 g(fda_blocks(h->N, 256), nrhs);
    k_permute_c<<<g, 256, 0, s>>>(x, xs, h->perm.as<int32_t>(), h->N, ld, h->N, nrhs, 1);
    FDA_CHECK_LAUNCH();
}

// ys (Morton order, leading dimension N) -> y (caller order, leading dimension ld)
void fda_scatter_cols(fda_handle *h, const c64d *ys, c64d *y, int64_t ld, int nrhs, cudaStream_t s)
{
    dim3 g(fda_blocks(h->N, 256), nrhs);
    k_permute_c<<<g, 256, 0, s>>>(ys, y, h->perm.as<int32_t>(), h->N, h->N, ld, nrhs, 0);
    FDA_CHECK_LAUNCH();
}

// ys (Morton order) -> y (caller order)
void fda_scatter_from_sorted(fda_handle *h, const c64d *ys, c64d *y)
{
    dim3 g(fda_blocks(h->N, 256), 1);
    k_permute_c<<<g, 256, 0, h->stream>>>(ys, y, h->perm.as<int32_t>(), h->N, h->N, h->N, 1, 0);
    FDA_CHECK_LAUNCH();
}
