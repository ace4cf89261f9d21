// Fields off the surface from the boundary solution: Green's representation
// of Eq. cbie in the acoustic domain (c = 1, n into the body),
//   u(x) = u_inc(x) + int G(x, y) q(y) dy - int dG/dn_y(x, y) u(y) dy,
// and its large-|x| limit, the far-field pattern F of u_sc ~ e^{ik|x|}/|x| F,
//   F(xh) = (1/(4 pi)) int [ q(y) + ik (xh . n_y) u(y) ] e^{-ik xh . y} dy,
// each element integral by the six-point rule of the regular near field.
// Direct summation over all elements for every target (no fast algorithm):
// N x M x 6 FP64 kernel evaluations, sincos-bound.
#include <math.h>

#include <algorithm>
#include <utility>
#include <vector>

#include "fda_internal.cuh"

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
