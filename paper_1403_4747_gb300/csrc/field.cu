// Fields off the surface from the boundary solution: Green's representation
// of Eq. cbie in the acoustic domain (c = 1, n into the body),
//   u(x) = u_inc(x) + int G(x, y) q(y) dy - int dG/dn_y(x, y) u(y) dy,
// and its large-|x| limit, the far-field pattern F of u_sc ~ e^{ik|x|}/|x| F,
//   F(xh) = (1/(4 pi)) int [ q(y) + ik (xh . n_y) u(y) ] e^{-ik xh . y} dy,
// each element integral by the six-point rule of the regular near field.
// Direct summation over all elements for every target (no fast algorithm):
// N x M x 6 FP64 kernel evaluations, sincos-bound.
#include <math.h>

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
