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

// blocks of one problem: element geometry, the row elements and the column
// elements of each block (the same list for the leaf-block pattern, the
// leaf's near-field columns for the near-field pattern) and the offsets of
// each block's n_B x nc_B row-major entries
struct sai_set {
    const double *cent, *nrm, *area;  // [n][3], [n][3], [n]
    const int64_t *bptr;              // [nb + 1] into belem (rows)
    const int32_t *belem;
    const int64_t *cptr;              // [nb + 1] into celem (columns)
    const int32_t *celem;
    const int64_t *moff;              // [nb + 1] entry offsets
    double k;
    int nb;
    int maxn;                         // most rows of a block
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
    const int64_t c0 = S.cptr[b];
    const int nc = (int)(S.cptr[b + 1] - c0);
    i = S.belem[S.bptr[b] + e / nc];
    j = S.celem[c0 + e % nc];
}

// entries of block b
__device__ inline int sai_count(const sai_set &S, int b)
{
    return (int)(S.bptr[b + 1] - S.bptr[b]) * (int)(S.cptr[b + 1] - S.cptr[b]);
}

// M = network(features) on every entry of every block (one CTA per block)
template <typename T, typename TO>
__global__ void __launch_bounds__(BT) k_sai_forward(sai_set S, const T *Wg, cx<TO> *M)
{
    __shared__ T W[SP];
    for (int p = threadIdx.x; p < SP; p += BT) W[p] = Wg[p];
    __syncthreads();
    const int b = blockIdx.x;
    const int ne = sai_count(S, b);
    for (int e = threadIdx.x; e < ne; e += BT) {
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
        const int ne = sai_count(S, b);
        for (int e0 = 0; e0 < ne; e0 += BT) {
            const int e = e0 + t;
            const int cnt = min(BT, ne - e0);
            if (e < ne) {
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

// ---- near-field pattern: M[B, C_B] for the rows of leaf B and its near-field
// columns C_B (whole leaves, element order); the objective compares
// M[B, C_B] A_near[C_B, C_B] with I[B, C_B], where a row l of A_near (in leaf
// C) holds the entries of C's own near-field columns and 0 elsewhere

// the handle's near-field layout: a leaf's columns are its near ranges
// (whole boxes, each in element order) one after another, in the order the
// ranges are listed, not sorted
struct near_view {
    const int32_t *leaf_box, *bbeg, *bend;
    const int64_t *colptr;     // [NL + 1] columns of each leaf
    const int64_t *rptr;       // [NL + 1] near ranges of each leaf
    const int32_t *rb, *re;    // element range [rb, re) of each near range
    const int64_t *off;        // [NL + 1] entry offsets of each leaf's rows (row-major, nc columns)
    const int32_t *elem_leaf;  // [N] leaf index of each element
};

constexpr int NT = 256;     // threads of the near-pattern product kernels
constexpr int QC = 64;      // B's columns per chunk
constexpr int QS = QC + 1;  // padded row stride of the A tile in shared memory
constexpr int MAXR = 512;   // near ranges of one leaf staged in shared memory

// the leaf whose rows start at column p of block b's columns, and the map of
// the chunk's columns q0 .. q0 + QC into that leaf's own columns (-1 where
// the pair is not in the near field), found through the leaf's near ranges
// (staged in rbs / res); returns whether any column maps, or -1 if the
// columns are not whole leaves or the leaf has more than MAXR ranges (then
// err is set)
struct row_leaf {
    int lc, nC, ncC;
    int64_t off;
};

__device__ inline int chunk_map(const sai_set &S, const near_view &V, int b, int p, int q0, row_leaf &L, int *map,
                                int *rbs, int *res, int *err)
{
    const int64_t c0 = S.cptr[b];
    const int nc = (int)(S.cptr[b + 1] - c0);
    const int e = S.celem[c0 + p];
    L.lc = V.elem_leaf[e];
    const int C = V.leaf_box[L.lc];
    const int cb0 = V.bbeg[C];
    L.nC = V.bend[C] - cb0;
    L.ncC = (int)(V.colptr[L.lc + 1] - V.colptr[L.lc]);
    L.off = V.off[L.lc];
    const int64_t r0 = V.rptr[L.lc];
    const int nr = (int)(V.rptr[L.lc + 1] - r0);
    if (e != cb0 || p + L.nC > nc || L.nC > 64 || nr > MAXR) {
        if (threadIdx.x == 0) atomicExch(err, nr > MAXR ? 2 : 1);
        return -1;
    }
    for (int r = threadIdx.x; r < nr; r += blockDim.x) {
        rbs[r] = V.rb[r0 + r];
        res[r] = V.re[r0 + r];
    }
    __syncthreads();
    int any = 0;
    if (threadIdx.x < QC) {
        const int q = q0 + (int)threadIdx.x;
        int pos = -1;
        if (q < nc) {
            const int j = S.celem[c0 + q];
            int o = 0;
            for (int r = 0; r < nr; ++r) {
                const int a = rbs[r], z = res[r];
                if (j >= a && j < z) {
                    pos = o + (j - a);
                    break;
                }
                o += z - a;
            }
        }
        map[threadIdx.x] = pos;
        any = pos >= 0;
    }
    return __syncthreads_or(any) ? 1 : 0;
}

// R = M[B, C_B] A_near[C_B, C_B] - I[B, C_B] over QC-column chunks (each
// thread a 4 x 4 register tile of the 64 x QC chunk), loss += scale ||R||^2;
// R is stored (n_B x nc_B at moff[b]) unless Rg is null.  One CTA per block.
template <typename T>
__global__ void __launch_bounds__(NT) k_sain_residual(sai_set S, near_view V, const cx<T> *A, const cx<T> *M,
                                                      cx<T> *Rg, double *loss, T scale, int *err)
{
    extern __shared__ __align__(16) unsigned char sm_raw[];
    cx<T> *Ms = reinterpret_cast<cx<T> *>(sm_raw);  // [64 rows of B][64 rows of C]
    cx<T> *As = Ms + 64 * 64;                        // [64 rows of C][QS]
    __shared__ int map[QC], rbs[MAXR], res[MAXR];
    __shared__ double red[NT];
    const int b = blockIdx.x, t = threadIdx.x, ti = t >> 4, tq = t & 15;
    const int64_t r0 = S.bptr[b], c0 = S.cptr[b], mo = S.moff[b];
    const int n = (int)(S.bptr[b + 1] - r0), nc = (int)(S.cptr[b + 1] - c0);
    double part = 0.0;
    bool bad = false;
    for (int q0 = 0; q0 < nc && !bad; q0 += QC) {
        cx<T> acc[4][4];
        for (int p = 0; p < nc;) {
            row_leaf L;
            const int any = chunk_map(S, V, b, p, q0, L, map, rbs, res, err);
            if (any < 0) {
                bad = true;
                break;
            }
            if (any) {
                for (int x = t; x < 64 * 64; x += NT) {
                    const int i = x >> 6, r = x & 63;
                    Ms[x] = i < n && r < L.nC ? M[mo + (int64_t)i * nc + p + r] : cx<T>();
                }
                for (int x = t; x < 64 * QC; x += NT) {
                    const int r = x / QC, qq = x % QC, m = map[qq];
                    As[r * QS + qq] = r < L.nC && m >= 0 ? A[L.off + (int64_t)r * L.ncC + m] : cx<T>();
                }
                __syncthreads();
                for (int r = 0; r < L.nC; ++r) {
                    cx<T> mv[4], av[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) mv[u] = Ms[(ti * 4 + u) * 64 + r];
#pragma unroll
                    for (int v = 0; v < 4; ++v) av[v] = As[r * QS + tq * 4 + v];
#pragma unroll
                    for (int u = 0; u < 4; ++u)
#pragma unroll
                        for (int v = 0; v < 4; ++v) cfma(acc[u][v], mv[u], av[v]);
                }
            }
            __syncthreads();  // map and tiles are rewritten for the next leaf
            p += L.nC;
        }
        if (bad) break;
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                const int i = ti * 4 + u, q = q0 + tq * 4 + v;
                if (i < n && q < nc) {
                    cx<T> r = acc[u][v];
                    if (S.celem[c0 + q] == S.belem[r0 + i]) r.re -= (T)1;
                    part += (double)r.re * r.re + (double)r.im * r.im;
                    if (Rg) Rg[mo + (int64_t)i * nc + q] = r;
                }
            }
    }
    red[t] = part;
    __syncthreads();
    for (int w = NT / 2; w > 0; w >>= 1) {
        if (t < w) red[t] += red[t + w];
        __syncthreads();
    }
    if (t == 0) atomicAdd(loss, (double)scale * red[0]);
}

// G[B, C] = 2 scale R[B, :] A_near[C, :]^H restricted to B's columns, for each
// leaf C among B's columns (dL/dRe M + i dL/dIm M); one CTA per block, each
// thread a 4 x 4 register tile of the 64 x 64 (row of B, row of C) block
template <typename T>
__global__ void __launch_bounds__(NT) k_sain_gradm(sai_set S, near_view V, const cx<T> *A, const cx<T> *Rg,
                                                   cx<T> *G, T scale, int *err)
{
    extern __shared__ __align__(16) unsigned char sm_raw[];
    cx<T> *Rs = reinterpret_cast<cx<T> *>(sm_raw);  // [64 rows of B][QC]
    cx<T> *As = Rs + 64 * QC;                        // [64 rows of C][QS]
    __shared__ int map[QC], rbs[MAXR], res[MAXR];
    const int b = blockIdx.x, t = threadIdx.x, ti = t >> 4, tr = t & 15;
    const int64_t r0 = S.bptr[b], c0 = S.cptr[b], mo = S.moff[b];
    const int n = (int)(S.bptr[b + 1] - r0), nc = (int)(S.cptr[b + 1] - c0);
    for (int p = 0; p < nc;) {
        cx<T> acc[4][4];
        row_leaf L{0, 0, 0, 0};
        bool bad = false;
        for (int q0 = 0; q0 < nc; q0 += QC) {
            const int any = chunk_map(S, V, b, p, q0, L, map, rbs, res, err);
            if (any < 0) {
                bad = true;
                break;
            }
            if (any) {
                for (int x = t; x < 64 * QC; x += NT) {
                    const int i = x / QC, qq = x % QC;
                    Rs[x] = i < n && q0 + qq < nc ? Rg[mo + (int64_t)i * nc + q0 + qq] : cx<T>();
                }
                for (int x = t; x < 64 * QC; x += NT) {
                    const int r = x / QC, qq = x % QC, m = map[qq];
                    As[r * QS + qq] = r < L.nC && m >= 0 ? A[L.off + (int64_t)r * L.ncC + m] : cx<T>();
                }
                __syncthreads();
                for (int qq = 0; qq < QC; ++qq) {
                    cx<T> rv[4], av[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) rv[u] = Rs[(ti * 4 + u) * QC + qq];
#pragma unroll
                    for (int v = 0; v < 4; ++v) {
                        const cx<T> a = As[(tr * 4 + v) * QS + qq];
                        av[v] = cx<T>(a.re, -a.im);
                    }
#pragma unroll
                    for (int u = 0; u < 4; ++u)
#pragma unroll
                        for (int v = 0; v < 4; ++v) cfma(acc[u][v], rv[u], av[v]);
                }
            }
            __syncthreads();
        }
        if (bad) break;
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                const int i = ti * 4 + u, r = tr * 4 + v;
                if (i < n && r < L.nC)
                    G[mo + (int64_t)i * nc + p + r] =
                        cx<T>((T)2 * scale * acc[u][v].re, (T)2 * scale * acc[u][v].im);
            }
        p += L.nC;
    }
}

// leaf index of every element
__global__ void k_elem_leaf(const int32_t *leaf_box, const int32_t *bbeg, const int32_t *bend, int NL, int32_t *out)
{
    const int li = blockIdx.x;
    if (li >= NL) return;
    const int B = leaf_box[li];
    for (int e = bbeg[B] + threadIdx.x; e < bend[B]; e += blockDim.x) out[e] = li;
}

// the near-field columns of the chosen leaves, packed block after block
__global__ void k_gather_cols(const int32_t *leaves, const int64_t *colptr, const int32_t *cols, const int64_t *cptr,
                              int nb, int32_t *out)
{
    const int b = blockIdx.x;
    if (b >= nb) return;
    const int64_t src = colptr[leaves[b]], dst = cptr[b], n = cptr[b + 1] - dst;
    for (int64_t q = threadIdx.x; q < n; q += blockDim.x) out[dst + q] = cols[src + q];
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
                  D.belem.as<int32_t>(), D.bptr.as<int64_t>(), D.belem.as<int32_t>(), D.moff.as<int64_t>(), h->k,
                  NL, maxn};
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

// ---- near-field pattern, host side

// grow-only device buffer
void ensure(dbuf &b, size_t bytes)
{
    if (b.bytes < bytes) b.alloc(bytes);
}

// a handle's leaf layout on the host and the element -> leaf map on the device
struct near_host {
    fda_handle *h = nullptr;
    std::vector<int32_t> lb, bb, be;
    std::vector<int64_t> colptr;
    dbuf elem_leaf;
    near_view V{};
};

void near_host_init(fda_handle *h, near_host &H)
{
    const int NL = h->nleaf;
    H.h = h;
    H.lb.resize(NL);
    H.bb.resize(h->nbox_total);
    H.be.resize(h->nbox_total);
    H.colptr.resize(NL + 1);
    FDA_CUDA(cudaMemcpy(H.lb.data(), h->leaf_box.p, 4 * (size_t)NL, cudaMemcpyDeviceToHost));
    FDA_CUDA(cudaMemcpy(H.bb.data(), h->box_begin.p, 4 * H.bb.size(), cudaMemcpyDeviceToHost));
    FDA_CUDA(cudaMemcpy(H.be.data(), h->box_end.p, 4 * H.be.size(), cudaMemcpyDeviceToHost));
    FDA_CUDA(cudaMemcpy(H.colptr.data(), h->nf_colptr.p, 8 * H.colptr.size(), cudaMemcpyDeviceToHost));
    for (int li = 0; li < NL; ++li)
        if (H.be[H.lb[li]] - H.bb[H.lb[li]] > 64)
            fda_fail(FDA_ERR_ARG, "the learned preconditioner needs leaves of at most 64 elements");
    H.elem_leaf.alloc(4 * (size_t)std::max<int64_t>(h->N, 1));
    k_elem_leaf<<<std::max(NL, 1), 128, 0, h->stream>>>(h->leaf_box.as<int32_t>(), h->box_begin.as<int32_t>(),
                                                        h->box_end.as<int32_t>(), NL, H.elem_leaf.as<int32_t>());
    FDA_CHECK_LAUNCH();
    H.V = near_view{h->leaf_box.as<int32_t>(), h->box_begin.as<int32_t>(), h->box_end.as<int32_t>(),
                    h->nf_colptr.as<int64_t>(), h->nr_ptr.as<int64_t>(), h->nr_begin.as<int32_t>(),
                    h->nr_end.as<int32_t>(), h->nf_off.as<int64_t>(), H.elem_leaf.as<int32_t>()};
}

// the near-field blocks of the chosen leaves (rows of the leaf x its
// near-field columns), packed; buffers grow and are reused across calls
struct near_set {
    dbuf leaves, bptr, belem, cptr, celem, moff;
    sai_set S{};
    int64_t nent = 0, nrows = 0;
};

void near_set_build(const near_host &H, const std::vector<int32_t> &leaves, near_set &D, cudaStream_t s)
{
    fda_handle *h = H.h;
    const int nb = (int)leaves.size();
    std::vector<int64_t> bptr(nb + 1, 0), cptr(nb + 1, 0), moff(nb + 1, 0);
    std::vector<int32_t> belem;
    int maxn = 0;
    for (int b = 0; b < nb; ++b) {
        const int li = leaves[b];
        if (li < 0 || li >= h->nleaf) fda_fail(FDA_ERR_ARG, "leaf index out of range");
        const int b0 = H.bb[H.lb[li]], n = H.be[H.lb[li]] - b0;
        const int64_t nc = H.colptr[li + 1] - H.colptr[li];
        for (int q = 0; q < n; ++q) belem.push_back(b0 + q);
        bptr[b + 1] = bptr[b] + n;
        cptr[b + 1] = cptr[b] + nc;
        moff[b + 1] = moff[b] + n * nc;
        maxn = std::max(maxn, n);
    }
    ensure(D.leaves, 4 * (size_t)std::max(nb, 1));
    ensure(D.bptr, 8 * (size_t)(nb + 1));
    ensure(D.cptr, 8 * (size_t)(nb + 1));
    ensure(D.moff, 8 * (size_t)(nb + 1));
    ensure(D.belem, 4 * std::max<size_t>(belem.size(), 1));
    ensure(D.celem, 4 * (size_t)std::max<int64_t>(cptr[nb], 1));
    FDA_CUDA(cudaMemcpyAsync(D.leaves.p, leaves.data(), 4 * (size_t)nb, cudaMemcpyHostToDevice, s));
    FDA_CUDA(cudaMemcpyAsync(D.bptr.p, bptr.data(), 8 * (size_t)(nb + 1), cudaMemcpyHostToDevice, s));
    FDA_CUDA(cudaMemcpyAsync(D.cptr.p, cptr.data(), 8 * (size_t)(nb + 1), cudaMemcpyHostToDevice, s));
    FDA_CUDA(cudaMemcpyAsync(D.moff.p, moff.data(), 8 * (size_t)(nb + 1), cudaMemcpyHostToDevice, s));
    FDA_CUDA(cudaMemcpyAsync(D.belem.p, belem.data(), 4 * belem.size(), cudaMemcpyHostToDevice, s));
    k_gather_cols<<<std::max(nb, 1), 128, 0, s>>>(D.leaves.as<int32_t>(), h->nf_colptr.as<int64_t>(),
                                                  h->nf_cols.as<int32_t>(), D.cptr.as<int64_t>(), nb,
                                                  D.celem.as<int32_t>());
    FDA_CHECK_LAUNCH();
    FDA_CUDA(cudaStreamSynchronize(s));  // the host vectors go out of scope
    D.nent = moff[nb];
    D.nrows = bptr[nb];
    D.S = sai_set{h->cent.as<double>(), h->nrm.as<double>(), h->area.as<double>(), D.bptr.as<int64_t>(),
                  D.belem.as<int32_t>(), D.cptr.as<int64_t>(), D.celem.as<int32_t>(), D.moff.as<int64_t>(), h->k,
                  nb, maxn};
}

size_t near_smem(size_t esz) { return (size_t)(64 * 64 + 64 * QS) * esz; }

template <typename T>
void near_attrs()
{
    static bool done = false;
    if (done) return;
    FDA_CUDA(cudaFuncSetAttribute(k_sain_residual<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)near_smem(sizeof(cx<T>))));
    FDA_CUDA(cudaFuncSetAttribute(k_sain_gradm<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)near_smem(sizeof(cx<T>))));
    const size_t bs = backward_smem(sizeof(T));
    FDA_CUDA(cudaFuncSetAttribute(k_sai_backward<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bs));
    done = true;
}

// loss (and, with R and G given, dL/dW added into grad) of the near-field
// objective over the blocks of S; A is the handle's near-field matrix
template <typename T>
void near_loss_grad(const sai_set &S, const near_view &V, const cx<T> *A, const T *W, cx<T> *M, cx<T> *R, cx<T> *G,
                    double *loss, T *grad, T scale, int *err, cudaStream_t s)
{
    if (S.nb == 0) return;
    near_attrs<T>();
    k_sai_forward<T, T><<<S.nb, BT, 0, s>>>(S, W, M);
    FDA_CHECK_LAUNCH();
    const size_t ns = near_smem(sizeof(cx<T>));
    k_sain_residual<T><<<S.nb, NT, ns, s>>>(S, V, A, M, R, loss, scale, err);
    FDA_CHECK_LAUNCH();
    if (!G) return;
    k_sain_gradm<T><<<S.nb, NT, ns, s>>>(S, V, A, R, G, scale, err);
    FDA_CHECK_LAUNCH();
    k_sai_backward<T><<<std::min(S.nb, 1024), BT, backward_smem(sizeof(T)), s>>>(S, W, G, grad);
    FDA_CHECK_LAUNCH();
}

void check_err(const dbuf &err, cudaStream_t s)
{
    int e = 0;
    FDA_CUDA(cudaMemcpyAsync(&e, err.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    FDA_CUDA(cudaStreamSynchronize(s));
    if (e == 2) fda_fail(FDA_ERR_STATE, "a leaf has more near-field ranges than the kernels stage");
    if (e) fda_fail(FDA_ERR_STATE, "near-field columns of a leaf are not whole leaves in element order");
}

// the near-field matrix of h in FP32 (the chosen form keeps one; else a copy)
const c32f *near_f32(fda_handle *h, dbuf &tmp)
{
    if (h->op32.near.p) return h->op32.near.as<c32f>();
    tmp.alloc(sizeof(c32f) * std::max<int64_t>(h->nnz_near, 1));
    k_c64_to_c32_n<<<1024, 256, 0, h->stream>>>(h->op64.near.as<c64d>(), tmp.as<c32f>(), h->nnz_near);
    FDA_CHECK_LAUNCH();
    return tmp.as<c32f>();
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
    h->sai_M32.release();
    h->sai_pattern = 0;
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
                  D.belem.as<int32_t>(), D.bptr.as<int64_t>(), D.belem.as<int32_t>(), D.moff.as<int64_t>(), k, nb,
                  maxn};
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

// ---- near-field pattern: training, setting, loss and gradient

namespace {

// k distinct leaves of NL, uniformly (partial Fisher-Yates on splitmix64)
std::vector<int32_t> sample_leaves(int NL, int k, uint64_t &st)
{
    std::vector<int32_t> all(NL);
    for (int i = 0; i < NL; ++i) all[i] = i;
    k = std::min(k, NL);
    for (int i = 0; i < k; ++i) {
        const int j = i + (int)(splitmix64(st) % (uint64_t)(NL - i));
        std::swap(all[i], all[j]);
    }
    all.resize(k);
    std::sort(all.begin(), all.end());
    return all;
}

}  // namespace

// Adam on the near-field objective: every step draws per_step leaves of each
// handle; loss0 / loss1 are taken on one fixed draw before and after (FP32)
void fda_sai_train_near_impl(fda_handle *const *hs, int nh, int epochs, double lr, int per_step, uint64_t seed,
                             float *W, double *loss0, double *loss1, double *train_s)
{
    cudaStream_t s = hs[0]->stream;
    const auto t0 = std::chrono::steady_clock::now();
    std::vector<near_host> H(nh);
    std::vector<dbuf> A32tmp(nh);
    std::vector<const c32f *> A32(nh);
    for (int q = 0; q < nh; ++q) {
        near_host_init(hs[q], H[q]);
        A32[q] = near_f32(hs[q], A32tmp[q]);
        FDA_CUDA(cudaStreamSynchronize(hs[q]->stream));
    }
    std::vector<near_set> D(nh), E(nh);
    uint64_t st = seed ^ 0x5A17C0DEull;
    int64_t eval_rows = 0;
    for (int q = 0; q < nh; ++q) {
        near_set_build(H[q], sample_leaves(hs[q]->nleaf, per_step, st), E[q], s);
        eval_rows += E[q].nrows;
    }
    dbuf dW, dG, m1, m2, Mb, Rb, Gb, dl, err;
    dW.alloc(4 * SP);
    dG.alloc(4 * SP);
    m1.alloc(4 * SP);
    m2.alloc(4 * SP);
    dl.alloc(sizeof(double));
    err.alloc(sizeof(int));
    FDA_CUDA(cudaMemcpyAsync(dW.p, W, 4 * SP, cudaMemcpyHostToDevice, s));
    FDA_CUDA(cudaMemsetAsync(m1.p, 0, 4 * SP, s));
    FDA_CUDA(cudaMemsetAsync(m2.p, 0, 4 * SP, s));
    FDA_CUDA(cudaMemsetAsync(err.p, 0, sizeof(int), s));
    auto evaluate = [&]() {
        FDA_CUDA(cudaMemsetAsync(dl.p, 0, sizeof(double), s));
        for (int q = 0; q < nh; ++q) {
            ensure(Mb, sizeof(c32f) * (size_t)std::max<int64_t>(E[q].nent, 1));
            near_loss_grad<float>(E[q].S, H[q].V, A32[q], dW.as<float>(), Mb.as<c32f>(), nullptr, nullptr,
                                  dl.as<double>(), nullptr, (float)(1.0 / (double)std::max<int64_t>(eval_rows, 1)),
                                  err.as<int>(), s);
        }
        double l = 0;
        FDA_CUDA(cudaMemcpyAsync(&l, dl.p, sizeof(double), cudaMemcpyDeviceToHost, s));
        check_err(err, s);
        if (!std::isfinite(l)) fda_fail(FDA_ERR_NUMERIC, "learned preconditioner training diverged");
        return l;
    };
    *loss0 = evaluate();
    const float b1 = 0.9f, b2 = 0.999f;
    double c1 = 1.0, c2 = 1.0;
    for (int ep = 0; ep < epochs; ++ep) {
        int64_t rows = 0;
        for (int q = 0; q < nh; ++q) {
            near_set_build(H[q], sample_leaves(hs[q]->nleaf, per_step, st), D[q], s);
            rows += D[q].nrows;
        }
        const float scale = (float)(1.0 / (double)std::max<int64_t>(rows, 1));
        FDA_CUDA(cudaMemsetAsync(dG.p, 0, 4 * SP, s));
        FDA_CUDA(cudaMemsetAsync(dl.p, 0, sizeof(double), s));
        for (int q = 0; q < nh; ++q) {
            const size_t eb = sizeof(c32f) * (size_t)std::max<int64_t>(D[q].nent, 1);
            ensure(Mb, eb);
            ensure(Rb, eb);
            ensure(Gb, eb);
            near_loss_grad<float>(D[q].S, H[q].V, A32[q], dW.as<float>(), Mb.as<c32f>(), Rb.as<c32f>(),
                                  Gb.as<c32f>(), dl.as<double>(), dG.as<float>(), scale, err.as<int>(), s);
        }
        c1 *= b1;
        c2 *= b2;
        k_sai_adam<<<(SP + 255) / 256, 256, 0, s>>>(dW.as<float>(), dG.as<float>(), m1.as<float>(), m2.as<float>(),
                                                     (float)lr, b1, b2, 1e-8f, (float)(1.0 - c1), (float)(1.0 - c2));
        FDA_CHECK_LAUNCH();
    }
    check_err(err, s);
    *loss1 = evaluate();
    FDA_CUDA(cudaMemcpyAsync(W, dW.p, 4 * SP, cudaMemcpyDeviceToHost, s));
    FDA_CUDA(cudaStreamSynchronize(s));
    *train_s = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

// network -> M on h's whole near-field pattern, FP32, in the near-field
// matrix's own layout (the GMRES apply runs the near-field product with it);
// with want_loss, the objective of the stored M over all leaves (FP32)
double fda_sai_set_near_impl(fda_handle *h, const float *W, bool want_loss)
{
    cudaStream_t s = h->stream;
    sai_data D;
    sai_from_handle(h, D);  // rows of every leaf, in leaf order
    if (D.S.nb == 0) fda_fail(FDA_ERR_STATE, "no leaves");
    sai_set S = D.S;
    S.cptr = h->nf_colptr.as<int64_t>();
    S.celem = h->nf_cols.as<int32_t>();
    S.moff = h->nf_off.as<int64_t>();
    dbuf dW;
    dW.alloc(4 * SP);
    FDA_CUDA(cudaMemcpyAsync(dW.p, W, 4 * SP, cudaMemcpyHostToDevice, s));
    h->sai_M.release();
    h->sai_M32.alloc(sizeof(c32f) * std::max<int64_t>(h->nnz_near, 1));
    k_sai_forward<float, float><<<S.nb, BT, 0, s>>>(S, dW.as<float>(), h->sai_M32.as<c32f>());
    FDA_CHECK_LAUNCH();
    h->sai_pattern = 1;
    if (!want_loss) {
        FDA_CUDA(cudaStreamSynchronize(s));
        return 0.0;
    }
    near_host H;
    near_host_init(h, H);
    dbuf A32tmp, dl, err;
    const c32f *A32 = near_f32(h, A32tmp);
    dl.alloc(sizeof(double));
    err.alloc(sizeof(int));
    FDA_CUDA(cudaMemsetAsync(dl.p, 0, sizeof(double), s));
    FDA_CUDA(cudaMemsetAsync(err.p, 0, sizeof(int), s));
    near_attrs<float>();
    k_sain_residual<float><<<S.nb, NT, near_smem(sizeof(c32f)), s>>>(
        S, H.V, A32, h->sai_M32.as<c32f>(), nullptr, dl.as<double>(), (float)(1.0 / (double)std::max<int64_t>(h->N, 1)),
        err.as<int>());
    FDA_CHECK_LAUNCH();
    double l = 0;
    FDA_CUDA(cudaMemcpyAsync(&l, dl.p, sizeof(double), cudaMemcpyDeviceToHost, s));
    check_err(err, s);
    return l;
}

// loss and gradient of the near-field objective over the given leaves of h,
// FP64 (the handle's FP64 near-field matrix) or FP32 (the training kernels)
void fda_sai_loss_grad_near_impl(fda_handle *h, const double *W, int nleaves, const int32_t *leaves, int fp32,
                                 double *loss, double *grad)
{
    cudaStream_t s = h->stream;
    near_host H;
    near_host_init(h, H);
    near_set D;
    near_set_build(H, std::vector<int32_t>(leaves, leaves + nleaves), D, s);
    const double scale = 1.0 / (double)std::max<int64_t>(D.nrows, 1);
    dbuf dW, dG, Mb, Rb, Gb, dl, err, A32tmp;
    dl.alloc(sizeof(double));
    err.alloc(sizeof(int));
    FDA_CUDA(cudaMemsetAsync(dl.p, 0, sizeof(double), s));
    FDA_CUDA(cudaMemsetAsync(err.p, 0, sizeof(int), s));
    const size_t ne = (size_t)std::max<int64_t>(D.nent, 1);
    if (!fp32) {
        dW.alloc(8 * SP);
        dG.alloc(8 * SP);
        Mb.alloc(sizeof(c64d) * ne);
        Rb.alloc(sizeof(c64d) * ne);
        Gb.alloc(sizeof(c64d) * ne);
        FDA_CUDA(cudaMemcpyAsync(dW.p, W, 8 * SP, cudaMemcpyHostToDevice, s));
        FDA_CUDA(cudaMemsetAsync(dG.p, 0, 8 * SP, s));
        near_loss_grad<double>(D.S, H.V, h->op64.near.as<c64d>(), dW.as<double>(), Mb.as<c64d>(), Rb.as<c64d>(),
                               Gb.as<c64d>(), dl.as<double>(), dG.as<double>(), scale, err.as<int>(), s);
        FDA_CUDA(cudaMemcpyAsync(grad, dG.p, 8 * SP, cudaMemcpyDeviceToHost, s));
        check_err(err, s);
    } else {
        std::vector<float> w32(SP), g32(SP);
        for (int p = 0; p < SP; ++p) w32[p] = (float)W[p];
        const c32f *A32 = near_f32(h, A32tmp);
        dW.alloc(4 * SP);
        dG.alloc(4 * SP);
        Mb.alloc(sizeof(c32f) * ne);
        Rb.alloc(sizeof(c32f) * ne);
        Gb.alloc(sizeof(c32f) * ne);
        FDA_CUDA(cudaMemcpyAsync(dW.p, w32.data(), 4 * SP, cudaMemcpyHostToDevice, s));
        FDA_CUDA(cudaMemsetAsync(dG.p, 0, 4 * SP, s));
        near_loss_grad<float>(D.S, H.V, A32, dW.as<float>(), Mb.as<c32f>(), Rb.as<c32f>(), Gb.as<c32f>(),
                              dl.as<double>(), dG.as<float>(), (float)scale, err.as<int>(), s);
        FDA_CUDA(cudaMemcpyAsync(g32.data(), dG.p, 4 * SP, cudaMemcpyDeviceToHost, s));
        check_err(err, s);
        for (int p = 0; p < SP; ++p) grad[p] = g32[p];
    }
    FDA_CUDA(cudaMemcpyAsync(loss, dl.p, sizeof(double), cudaMemcpyDeviceToHost, s));
    FDA_CUDA(cudaStreamSynchronize(s));
}
