// Learned sparse approximate inverse (SAI) preconditioner on the leaf-block
// pattern.  The paper solves without a preconditioner (Sec. 5.3); this is
// the learned preconditioner of the scope's solver row, with the leaf
// block-diagonal inverse (precond.cu) as its plain counterpart.
//
// A small network predicts the entries M_ij of a right preconditioner on the
// pattern {(i, j): i, j in the same leaf B} from the local geometry of the
// pair and the wavenumber:
//   features f(i, j) = [k d, (r.n_i)/d, (r.n_j)/d, n_i.n_j, k sqrt(a_i),
//                       k sqrt(a_j), [i == j], sqrt(a_j)/max(d, sqrt(a_j))]
//   (r = x_j - x_i, d = |r|, x centroids, n normals into the body, a areas;
//   the direction terms are 0 for i == j; all are invariant under rotations
//   of the pair, as the kernel is),
//   h1 = tanh(W1 f + b1), h2 = tanh(W2 h1 + b2), (Re M_ij, Im M_ij) = W3 h2 + b3,
// with 8 features and two hidden layers of 32.  It is trained to minimise
//   L = (1 / sum_B n_B) sum_B || M_B A_BB - I ||_F^2,
// A_BB the leaf's own block of the near-field matrix (Eq. eq_sum), by full-
// batch Adam with the forward, residual, backward and update kernels below
// (FP32); the FP64 instantiation of the same kernels serves the gradient
// check against an independent CPU implementation.
#include <math.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <vector>

#include "fda_internal.cuh"

namespace {

constexpr int SF = 8;   // features
constexpr int SH = 32;  // hidden width
constexpr int OW1 = 0, OB1 = OW1 + SH * SF, OW2 = OB1 + SH, OB2 = OW2 + SH * SH, OW3 = OB2 + SH,
              OB3 = OW3 + 2 * SH, SP = OB3 + 2;  // parameter layout, SP = 1410
constexpr int BT = 128;                          // threads per CTA in the per-entry kernels

// blocks of one problem: element geometry, the elements of each block and
// the offsets of each block's n_B x n_B row-major entries
struct sai_set {
    const double *cent, *nrm, *area;  // [n][3], [n][3], [n]
    const int64_t *bptr;              // [nb + 1] into belem
    const int32_t *belem;
    const int64_t *moff;              // [nb + 1] entry offsets
    double k;
    int nb;
    int maxn;                         // largest block
};

template <typename T>
__device__ inline void sai_features(const sai_set &S, int i, int j, T f[SF])
{
    const double *xi = S.cent + 3 * (int64_t)i, *xj = S.cent + 3 * (int64_t)j;
    const double *ni = S.nrm + 3 * (int64_t)i, *nj = S.nrm + 3 * (int64_t)j;
    const double r0 = xj[0] - xi[0], r1 = xj[1] - xi[1], r2 = xj[2] - xi[2];
    const double d = sqrt(r0 * r0 + r1 * r1 + r2 * r2);
    const double hi = sqrt(S.area[i]), hj = sqrt(S.area[j]);
    const bool self = i == j;
    f[0] = (T)(S.k * d);
    f[1] = self ? (T)0 : (T)((r0 * ni[0] + r1 * ni[1] + r2 * ni[2]) / d);
    f[2] = self ? (T)0 : (T)((r0 * nj[0] + r1 * nj[1] + r2 * nj[2]) / d);
    f[3] = (T)(ni[0] * nj[0] + ni[1] * nj[1] + ni[2] * nj[2]);
    f[4] = (T)(S.k * hi);
    f[5] = (T)(S.k * hj);
    f[6] = self ? (T)1 : (T)0;
    f[7] = (T)(hj / fmax(d, hj));
}

template <typename T>
__device__ inline void sai_forward_entry(const T *W, const T f[SF], T h1[SH], T h2[SH], T o[2])
{
    for (int a = 0; a < SH; ++a) {
        T z = W[OB1 + a];
        for (int b = 0; b < SF; ++b) z += W[OW1 + a * SF + b] * f[b];
        h1[a] = tanh(z);
    }
    for (int a = 0; a < SH; ++a) {
        T z = W[OB2 + a];
        for (int b = 0; b < SH; ++b) z += W[OW2 + a * SH + b] * h1[b];
        h2[a] = tanh(z);
    }
    for (int c = 0; c < 2; ++c) {
        T z = W[OB3 + c];
        for (int b = 0; b < SH; ++b) z += W[OW3 + c * SH + b] * h2[b];
        o[c] = z;
    }
}

// entry e of block b -> (row element, column element)
__device__ inline void sai_entry(const sai_set &S, int b, int e, int &i, int &j)
{
    const int64_t p0 = S.bptr[b];
    const int n = (int)(S.bptr[b + 1] - p0);
    i = S.belem[p0 + e / n];
    j = S.belem[p0 + e % n];
}

// M = network(features) on every entry of every block (one CTA per block)
template <typename T, typename TO>
__global__ void __launch_bounds__(BT) k_sai_forward(sai_set S, const T *Wg, cx<TO> *M)
{
    __shared__ T W[SP];
    for (int p = threadIdx.x; p < SP; p += BT) W[p] = Wg[p];
    __syncthreads();
    const int b = blockIdx.x;
    const int n = (int)(S.bptr[b + 1] - S.bptr[b]);
    for (int e = threadIdx.x; e < n * n; e += BT) {
        int i, j;
        sai_entry(S, b, e, i, j);
        T f[SF], h1[SH], h2[SH], o[2];
        sai_features(S, i, j, f);
        sai_forward_entry(W, f, h1, h2, o);
        M[S.moff[b] + e] = cx<TO>((TO)o[0], (TO)o[1]);
    }
}

// R = M_B A_BB - I, loss += scale ||R||^2, G = 2 scale R A_BB^H (dL/dM as
// dL/dRe M + i dL/dIm M); one CTA per block, A_BB and R staged in shared memory
template <typename T>
__global__ void __launch_bounds__(BT) k_sai_residual(sai_set S, const cx<T> *A, const cx<T> *M, cx<T> *G,
                                                     double *loss, T scale)
{
    extern __shared__ unsigned char sm_raw[];
    cx<T> *As = reinterpret_cast<cx<T> *>(sm_raw);
    const int b = blockIdx.x;
    const int n = (int)(S.bptr[b + 1] - S.bptr[b]);
    cx<T> *Rs = As + n * n;
    __shared__ double red[BT];
    const int64_t base = S.moff[b];
    for (int e = threadIdx.x; e < n * n; e += BT) As[e] = A[base + e];
    __syncthreads();
    double part = 0.0;
    for (int e = threadIdx.x; e < n * n; e += BT) {
        const int i = e / n, j = e % n;
        cx<T> r;
        for (int q = 0; q < n; ++q) cfma(r, M[base + i * n + q], As[q * n + j]);
        if (i == j) r.re -= (T)1;
        Rs[e] = r;
        part += (double)r.re * r.re + (double)r.im * r.im;
    }
    red[threadIdx.x] = part;
    __syncthreads();
    for (int s = BT / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) atomicAdd(loss, (double)scale * red[0]);
    for (int e = threadIdx.x; e < n * n; e += BT) {
        const int i = e / n, j = e % n;
        cx<T> g;
        for (int q = 0; q < n; ++q) {
            const cx<T> a = As[j * n + q];
            cfma(g, Rs[i * n + q], cx<T>(a.re, -a.im));
        }
        G[base + e] = cx<T>((T)2 * scale * g.re, (T)2 * scale * g.im);
    }
}

// dL/dW: per chunk of BT entries every thread runs its entry forward and
// back, stages activations and deltas in shared memory, then thread t sums
// the chunk's contribution to parameters t, t + BT, ...; CTAs stride over
// the blocks and add their sums to grad once at the end
template <typename T>
__global__ void __launch_bounds__(BT) k_sai_backward(sai_set S, const T *Wg, const cx<T> *G, T *grad)
{
    __shared__ T W[SP];
    extern __shared__ unsigned char sm_raw[];
    T *sf = reinterpret_cast<T *>(sm_raw);  // [BT][SF]
    T *sh1 = sf + BT * SF;                   // [BT][SH]
    T *sh2 = sh1 + BT * SH;
    T *sd1 = sh2 + BT * SH;
    T *sd2 = sd1 + BT * SH;
    T *sd3 = sd2 + BT * SH;                  // [BT][2]
    for (int p = threadIdx.x; p < SP; p += BT) W[p] = Wg[p];
    constexpr int PPT = (SP + BT - 1) / BT;
    T acc[PPT];
    for (int m = 0; m < PPT; ++m) acc[m] = (T)0;
    __syncthreads();
    const int t = threadIdx.x;
    for (int b = blockIdx.x; b < S.nb; b += gridDim.x) {
        const int n = (int)(S.bptr[b + 1] - S.bptr[b]);
        for (int e0 = 0; e0 < n * n; e0 += BT) {
            const int e = e0 + t;
            const int cnt = min(BT, n * n - e0);
            if (e < n * n) {
                int i, j;
                sai_entry(S, b, e, i, j);
                T f[SF], h1[SH], h2[SH], o[2];
                sai_features(S, i, j, f);
                sai_forward_entry(W, f, h1, h2, o);
                const cx<T> g = G[S.moff[b] + e];
                const T d3[2] = {g.re, g.im};
                T d2[SH], d1[SH];
                for (int a = 0; a < SH; ++a) {
                    const T s = W[OW3 + a] * d3[0] + W[OW3 + SH + a] * d3[1];
                    d2[a] = s * ((T)1 - h2[a] * h2[a]);
                }
                for (int a = 0; a < SH; ++a) {
                    T s = (T)0;
                    for (int c = 0; c < SH; ++c) s += W[OW2 + c * SH + a] * d2[c];
                    d1[a] = s * ((T)1 - h1[a] * h1[a]);
                }
                for (int a = 0; a < SF; ++a) sf[t * SF + a] = f[a];
                for (int a = 0; a < SH; ++a) {
                    sh1[t * SH + a] = h1[a];
                    sh2[t * SH + a] = h2[a];
                    sd1[t * SH + a] = d1[a];
                    sd2[t * SH + a] = d2[a];
                }
                sd3[t * 2] = d3[0];
                sd3[t * 2 + 1] = d3[1];
            }
            __syncthreads();
            for (int m = 0; m < PPT; ++m) {
                const int p = t + m * BT;
                if (p >= SP) break;
                T s = (T)0;
                if (p < OB1) {
                    const int a = (p - OW1) / SF, c = (p - OW1) % SF;
                    for (int q = 0; q < cnt; ++q) s += sd1[q * SH + a] * sf[q * SF + c];
                } else if (p < OW2) {
                    const int a = p - OB1;
                    for (int q = 0; q < cnt; ++q) s += sd1[q * SH + a];
                } else if (p < OB2) {
                    const int a = (p - OW2) / SH, c = (p - OW2) % SH;
                    for (int q = 0; q < cnt; ++q) s += sd2[q * SH + a] * sh1[q * SH + c];
                } else if (p < OW3) {
                    const int a = p - OB2;
                    for (int q = 0; q < cnt; ++q) s += sd2[q * SH + a];
                } else if (p < OB3) {
                    const int a = (p - OW3) / SH, c = (p - OW3) % SH;
                    for (int q = 0; q < cnt; ++q) s += sd3[q * 2 + a] * sh2[q * SH + c];
                } else {
                    const int a = p - OB3;
                    for (int q = 0; q < cnt; ++q) s += sd3[q * 2 + a];
                }
                acc[m] += s;
            }
            __syncthreads();
        }
    }
    for (int m = 0; m < PPT; ++m) {
        const int p = t + m * BT;
        if (p < SP) atomicAdd(grad + p, acc[m]);
    }
}

__global__ void k_sai_adam(float *W, const float *g, float *m1, float *m2, float lr, float b1, float b2, float eps,
                           float c1, float c2)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= SP) return;
    const float gp = g[p];
    m1[p] = b1 * m1[p] + (1.0f - b1) * gp;
    m2[p] = b2 * m2[p] + (1.0f - b2) * gp * gp;
    W[p] -= lr * (m1[p] / c1) / (sqrtf(m2[p] / c2) + eps);
}

// leaf self blocks A_BB of the near-field matrix, row-major per leaf
__global__ void k_sai_extract(const int32_t *leaf_box, const int32_t *bbeg, const int32_t *bend,
                              const int64_t *colptr, const int64_t *rptr, const int32_t *rb, const int32_t *re,
                              const int64_t *off, const c64d *A, const int64_t *moff, c64d *out, int *status)
{
    const int li = blockIdx.x;
    const int B = leaf_box[li];
    const int b0 = bbeg[B], n = bend[B] - b0;
    const int64_t nc = colptr[li + 1] - colptr[li];
    __shared__ int64_t cself;
    if (threadIdx.x == 0) {
        int64_t c = 0;
        cself = -1;
        for (int64_t g = rptr[li]; g < rptr[li + 1]; ++g) {
            if (rb[g] == b0) {
                cself = c;
                break;
            }
            c += re[g] - rb[g];
        }
    }
    __syncthreads();
    if (cself < 0) {
        if (threadIdx.x == 0) atomicExch(status, 1);
        return;
    }
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
        const int i = e / n, j = e % n;
        out[moff[li] + e] = A[off[li] + (int64_t)i * nc + cself + j];
    }
}

__global__ void k_c64_to_c32_n(const c64d *a, c32f *b, int64_t n)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
        b[e] = c32f((float)a[e].re, (float)a[e].im);
}

// device copies describing one problem's blocks
struct sai_data {
    dbuf bptr, belem, moff, A64, A32;
    dbuf cent, nrm, area;  // only for host-supplied geometry
    sai_set S{};
    int64_t nent = 0, nrows = 0;
};

// leaves of a handle as blocks (geometry stays in the handle)
void sai_from_handle(fda_handle *h, sai_data &D)
{
    const int NL = h->nleaf;
    std::vector<int32_t> lb(NL), bb(h->nbox_total), be(h->nbox_total);
    FDA_CUDA(cudaMemcpy(lb.data(), h->leaf_box.p, 4 * (size_t)NL, cudaMemcpyDeviceToHost));
    FDA_CUDA(cudaMemcpy(bb.data(), h->box_begin.p, 4 * bb.size(), cudaMemcpyDeviceToHost));
    FDA_CUDA(cudaMemcpy(be.data(), h->box_end.p, 4 * be.size(), cudaMemcpyDeviceToHost));
    std::vector<int64_t> bptr(NL + 1, 0), moff(NL + 1, 0);
    std::vector<int32_t> belem;
    int maxn = 0;
    for (int li = 0; li < NL; ++li) {
        const int b0 = bb[lb[li]], n = be[lb[li]] - b0;
        if (n > 64) fda_fail(FDA_ERR_ARG, "the learned preconditioner needs leaves of at most 64 elements");
        for (int q = 0; q < n; ++q) belem.push_back(b0 + q);
        bptr[li + 1] = bptr[li] + n;
        moff[li + 1] = moff[li] + (int64_t)n * n;
        maxn = std::max(maxn, n);
    }
    D.bptr.alloc(8 * bptr.size());
    D.moff.alloc(8 * moff.size());
    D.belem.alloc(4 * std::max<size_t>(belem.size(), 1));
    FDA_CUDA(cudaMemcpy(D.bptr.p, bptr.data(), 8 * bptr.size(), cudaMemcpyHostToDevice));
    FDA_CUDA(cudaMemcpy(D.moff.p, moff.data(), 8 * moff.size(), cudaMemcpyHostToDevice));
    if (!belem.empty())
        FDA_CUDA(cudaMemcpy(D.belem.p, belem.data(), 4 * belem.size(), cudaMemcpyHostToDevice));
    D.nent = moff[NL];
    D.nrows = bptr[NL];
    D.S = sai_set{h->cent.as<double>(), h->nrm.as<double>(), h->area.as<double>(), D.bptr.as<int64_t>(),
                  D.belem.as<int32_t>(), D.moff.as<int64_t>(), h->k, NL, maxn};
}

void sai_blocks_of_handle(fda_handle *h, sai_data &D)
{
    sai_from_handle(h, D);
    dbuf status;
    status.alloc(sizeof(int));
    FDA_CUDA(cudaMemsetAsync(status.p, 0, sizeof(int), h->stream));
    D.A64.alloc(sizeof(c64d) * std::max<int64_t>(D.nent, 1));
    k_sai_extract<<<h->nleaf, 256, 0, h->stream>>>(h->leaf_box.as<int32_t>(), h->box_begin.as<int32_t>(),
                                                   h->box_end.as<int32_t>(), h->nf_colptr.as<int64_t>(),
                                                   h->nr_ptr.as<int64_t>(), h->nr_begin.as<int32_t>(),
                                                   h->nr_end.as<int32_t>(), h->nf_off.as<int64_t>(),
                                                   h->op64.near.as<c64d>(), D.moff.as<int64_t>(), D.A64.as<c64d>(),
                                                   status.as<int>());
    FDA_CHECK_LAUNCH();
    int hs = 0;
    FDA_CUDA(cudaMemcpyAsync(&hs, status.p, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    FDA_CUDA(cudaStreamSynchronize(h->stream));
    if (hs) fda_fail(FDA_ERR_NUMERIC, "leaf self block not found in the near field");
}

size_t residual_smem(int maxn, size_t esz) { return 2 * (size_t)maxn * maxn * esz; }
size_t backward_smem(size_t tsz) { return tsz * BT * (SF + 4 * SH + 2); }

// loss and gradient of one set of blocks, accumulated into loss and grad
template <typename T>
void sai_loss_grad(const sai_set &S, const cx<T> *A, const T *W, cx<T> *M, cx<T> *G, double *loss, T *grad, T scale,
                   cudaStream_t s)
{
    if (S.nb == 0) return;
    k_sai_forward<T, T><<<S.nb, BT, 0, s>>>(S, W, M);
    FDA_CHECK_LAUNCH();
    const size_t rs = residual_smem(S.maxn, sizeof(cx<T>));
    FDA_CUDA(cudaFuncSetAttribute(k_sai_residual<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rs));
    k_sai_residual<T><<<S.nb, BT, rs, s>>>(S, A, M, G, loss, scale);
    FDA_CHECK_LAUNCH();
    const size_t bs = backward_smem(sizeof(T));
    FDA_CUDA(cudaFuncSetAttribute(k_sai_backward<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bs));
    k_sai_backward<T><<<std::min(S.nb, 1024), BT, bs, s>>>(S, W, G, grad);
    FDA_CHECK_LAUNCH();
}

// splitmix64: a fixed, documented generator for the initial weights
uint64_t splitmix64(uint64_t &x)
{
    uint64_t z = (x += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

}  // namespace

int fda_sai_nparams() { return SP; }

// Xavier-uniform weights, zero biases
void fda_sai_init(uint64_t seed, float *W)
{
    uint64_t st = seed;
    auto uni = [&]() { return (double)(splitmix64(st) >> 11) * (1.0 / 9007199254740992.0) * 2.0 - 1.0; };
    for (int p = 0; p < SP; ++p) W[p] = 0.0f;
    const double a1 = sqrt(6.0 / (SF + SH)), a2 = sqrt(6.0 / (SH + SH)), a3 = sqrt(6.0 / (SH + 2));
    for (int p = OW1; p < OB1; ++p) W[p] = (float)(a1 * uni());
    for (int p = OW2; p < OB2; ++p) W[p] = (float)(a2 * uni());
    for (int p = OW3; p < OB3; ++p) W[p] = (float)(a3 * uni());
}

// full-batch Adam on the leaf blocks of the given handles (FP32)
void fda_sai_train_impl(fda_handle *const *hs, int nh, int epochs, double lr, float *W, double *loss0,
                        double *loss1, double *train_s)
{
    cudaStream_t s = hs[0]->stream;
    const auto t0 = std::chrono::steady_clock::now();
    std::vector<sai_data> D(nh);
    int64_t rows = 0;
    for (int q = 0; q < nh; ++q) {
        sai_blocks_of_handle(hs[q], D[q]);
        FDA_CUDA(cudaStreamSynchronize(hs[q]->stream));
        D[q].A32.alloc(sizeof(c32f) * std::max<int64_t>(D[q].nent, 1));
        k_c64_to_c32_n<<<1024, 256, 0, s>>>(D[q].A64.as<c64d>(), D[q].A32.as<c32f>(), D[q].nent);
        FDA_CHECK_LAUNCH();
        rows += D[q].nrows;
    }
    int64_t maxent = 1;
    for (int q = 0; q < nh; ++q) maxent = std::max(maxent, D[q].nent);
    dbuf dW, dG, m1, m2, Mb, Gb, dl;
    dW.alloc(4 * SP);
    dG.alloc(4 * SP);
    m1.alloc(4 * SP);
    m2.alloc(4 * SP);
    Mb.alloc(sizeof(c32f) * maxent);
    Gb.alloc(sizeof(c32f) * maxent);
    dl.alloc(sizeof(double));
    FDA_CUDA(cudaMemcpyAsync(dW.p, W, 4 * SP, cudaMemcpyHostToDevice, s));
    FDA_CUDA(cudaMemsetAsync(m1.p, 0, 4 * SP, s));
    FDA_CUDA(cudaMemsetAsync(m2.p, 0, 4 * SP, s));
    const float scale = (float)(1.0 / (double)std::max<int64_t>(rows, 1));
    const float b1 = 0.9f, b2 = 0.999f;
    double c1 = 1.0, c2 = 1.0;
    for (int ep = 0; ep <= epochs; ++ep) {
        FDA_CUDA(cudaMemsetAsync(dG.p, 0, 4 * SP, s));
        FDA_CUDA(cudaMemsetAsync(dl.p, 0, sizeof(double), s));
        for (int q = 0; q < nh; ++q)
            sai_loss_grad<float>(D[q].S, D[q].A32.as<c32f>(), dW.as<float>(), Mb.as<c32f>(), Gb.as<c32f>(),
                                 dl.as<double>(), dG.as<float>(), scale, s);
        if (ep == 0 || ep == epochs) {
            double l = 0;
            FDA_CUDA(cudaMemcpyAsync(&l, dl.p, sizeof(double), cudaMemcpyDeviceToHost, s));
            FDA_CUDA(cudaStreamSynchronize(s));
            if (!std::isfinite(l)) fda_fail(FDA_ERR_NUMERIC, "learned preconditioner training diverged");
            (ep == 0 ? *loss0 : *loss1) = l;
        }
        if (ep == epochs) break;
        c1 *= b1;
        c2 *= b2;
        k_sai_adam<<<(SP + 255) / 256, 256, 0, s>>>(dW.as<float>(), dG.as<float>(), m1.as<float>(), m2.as<float>(),
                                                     (float)lr, b1, b2, 1e-8f, (float)(1.0 - c1), (float)(1.0 - c2));
        FDA_CHECK_LAUNCH();
    }
    FDA_CUDA(cudaMemcpyAsync(W, dW.p, 4 * SP, cudaMemcpyDeviceToHost, s));
    FDA_CUDA(cudaStreamSynchronize(s));
    *train_s = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

// network -> M on the leaf blocks of h (FP64 storage for the GMRES apply);
// returns the loss of M against the FP64 blocks
double fda_sai_set_impl(fda_handle *h, const float *W)
{
    cudaStream_t s = h->stream;
    sai_data D;
    sai_blocks_of_handle(h, D);
    if (D.S.nb == 0) fda_fail(FDA_ERR_STATE, "no leaf blocks");
    dbuf dW, dl, G;
    dW.alloc(4 * SP);
    FDA_CUDA(cudaMemcpyAsync(dW.p, W, 4 * SP, cudaMemcpyHostToDevice, s));
    h->sai_M.alloc(sizeof(c64d) * std::max<int64_t>(D.nent, 1));
    h->sai_off.alloc(8 * (size_t)(h->nleaf + 1));
    FDA_CUDA(cudaMemcpyAsync(h->sai_off.p, D.moff.p, 8 * (size_t)(h->nleaf + 1), cudaMemcpyDeviceToDevice, s));
    k_sai_forward<float, double><<<D.S.nb, BT, 0, s>>>(D.S, dW.as<float>(), h->sai_M.as<c64d>());
    FDA_CHECK_LAUNCH();
    // loss of the stored M against the FP64 blocks (FP64 residual kernel)
    dl.alloc(sizeof(double));
    G.alloc(sizeof(c64d) * std::max<int64_t>(D.nent, 1));
    FDA_CUDA(cudaMemsetAsync(dl.p, 0, sizeof(double), s));
    const size_t rs = residual_smem(D.S.maxn, sizeof(c64d));
    FDA_CUDA(cudaFuncSetAttribute(k_sai_residual<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rs));
    k_sai_residual<double><<<D.S.nb, BT, rs, s>>>(D.S, D.A64.as<c64d>(), h->sai_M.as<c64d>(),
                                                               G.as<c64d>(), dl.as<double>(),
                                                               1.0 / (double)std::max<int64_t>(D.nrows, 1));
    FDA_CHECK_LAUNCH();
    double l = 0;
    FDA_CUDA(cudaMemcpyAsync(&l, dl.p, sizeof(double), cudaMemcpyDeviceToHost, s));
    FDA_CUDA(cudaStreamSynchronize(s));
    return l;
}

// FP64 loss and gradient for caller-supplied geometry, blocks and A_BB (the
// gradient check); everything is copied in and the result copied out
void fda_sai_loss_grad_impl(int64_t n, const double *cent, const double *nrm, const double *area, double k, int nb,
                            const int64_t *bptr, const int32_t *belem, const c64d *A, const double *W, int fp32,
                            double *loss, double *grad)
{
    sai_data D;
    D.cent.alloc(24 * (size_t)n);
    D.nrm.alloc(24 * (size_t)n);
    D.area.alloc(8 * (size_t)n);
    FDA_CUDA(cudaMemcpy(D.cent.p, cent, 24 * (size_t)n, cudaMemcpyHostToDevice));
    FDA_CUDA(cudaMemcpy(D.nrm.p, nrm, 24 * (size_t)n, cudaMemcpyHostToDevice));
    FDA_CUDA(cudaMemcpy(D.area.p, area, 8 * (size_t)n, cudaMemcpyHostToDevice));
    std::vector<int64_t> moff(nb + 1, 0);
    int maxn = 0;
    for (int b = 0; b < nb; ++b) {
        const int64_t m = bptr[b + 1] - bptr[b];
        if (m < 1 || m > 64) fda_fail(FDA_ERR_ARG, "blocks must hold 1 to 64 elements");
        moff[b + 1] = moff[b] + m * m;
        maxn = std::max<int>(maxn, (int)m);
    }
    for (int64_t q = 0; q < bptr[nb]; ++q)
        if (belem[q] < 0 || belem[q] >= n) fda_fail(FDA_ERR_ARG, "block element index out of range");
    D.bptr.alloc(8 * (size_t)(nb + 1));
    D.moff.alloc(8 * (size_t)(nb + 1));
    D.belem.alloc(4 * (size_t)std::max<int64_t>(bptr[nb], 1));
    FDA_CUDA(cudaMemcpy(D.bptr.p, bptr, 8 * (size_t)(nb + 1), cudaMemcpyHostToDevice));
    FDA_CUDA(cudaMemcpy(D.moff.p, moff.data(), 8 * (size_t)(nb + 1), cudaMemcpyHostToDevice));
    FDA_CUDA(cudaMemcpy(D.belem.p, belem, 4 * (size_t)bptr[nb], cudaMemcpyHostToDevice));
    D.nent = moff[nb];
    D.A64.alloc(sizeof(c64d) * std::max<int64_t>(D.nent, 1));
    FDA_CUDA(cudaMemcpy(D.A64.p, A, sizeof(c64d) * (size_t)D.nent, cudaMemcpyHostToDevice));
    D.S = sai_set{D.cent.as<double>(), D.nrm.as<double>(), D.area.as<double>(), D.bptr.as<int64_t>(),
                  D.belem.as<int32_t>(), D.moff.as<int64_t>(), k, nb, maxn};
    dbuf dW, dG, Mb, Gb, dl, A32;
    dl.alloc(sizeof(double));
    FDA_CUDA(cudaMemset(dl.p, 0, sizeof(double)));
    const double scale = 1.0 / (double)std::max<int64_t>(bptr[nb], 1);
    if (!fp32) {
        dW.alloc(8 * SP);
        dG.alloc(8 * SP);
        Mb.alloc(sizeof(c64d) * std::max<int64_t>(D.nent, 1));
        Gb.alloc(sizeof(c64d) * std::max<int64_t>(D.nent, 1));
        FDA_CUDA(cudaMemcpy(dW.p, W, 8 * SP, cudaMemcpyHostToDevice));
        FDA_CUDA(cudaMemset(dG.p, 0, 8 * SP));
        sai_loss_grad<double>(D.S, D.A64.as<c64d>(), dW.as<double>(), Mb.as<c64d>(), Gb.as<c64d>(), dl.as<double>(),
                              dG.as<double>(), scale, 0);
        FDA_CUDA(cudaDeviceSynchronize());
        FDA_CUDA(cudaMemcpy(grad, dG.p, 8 * SP, cudaMemcpyDeviceToHost));
    } else {
        // the training precision: FP32 weights, blocks, activations and gradient
        std::vector<float> w32(SP), g32(SP);
        for (int p = 0; p < SP; ++p) w32[p] = (float)W[p];
        dW.alloc(4 * SP);
        dG.alloc(4 * SP);
        Mb.alloc(sizeof(c32f) * std::max<int64_t>(D.nent, 1));
        Gb.alloc(sizeof(c32f) * std::max<int64_t>(D.nent, 1));
        A32.alloc(sizeof(c32f) * std::max<int64_t>(D.nent, 1));
        k_c64_to_c32_n<<<256, 256>>>(D.A64.as<c64d>(), A32.as<c32f>(), D.nent);
        FDA_CHECK_LAUNCH();
        FDA_CUDA(cudaMemcpy(dW.p, w32.data(), 4 * SP, cudaMemcpyHostToDevice));
        FDA_CUDA(cudaMemset(dG.p, 0, 4 * SP));
        sai_loss_grad<float>(D.S, A32.as<c32f>(), dW.as<float>(), Mb.as<c32f>(), Gb.as<c32f>(), dl.as<double>(),
                             dG.as<float>(), (float)scale, 0);
        FDA_CUDA(cudaDeviceSynchronize());
        FDA_CUDA(cudaMemcpy(g32.data(), dG.p, 4 * SP, cudaMemcpyDeviceToHost));
        for (int p = 0; p < SP; ++p) grad[p] = g32[p];
    }
    FDA_CUDA(cudaMemcpy(loss, dl.p, sizeof(double), cudaMemcpyDeviceToHost));
}
