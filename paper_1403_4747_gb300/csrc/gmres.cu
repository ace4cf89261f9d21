// GMRES solve of Sec. 5 (no preconditioner, tolerance on the relative
// residual of the unpreconditioned system).  Readings of what the paper
// leaves open: restarted GMRES(m), zero or caller initial guess, classical
// Gram-Schmidt with one re-orthogonalisation (CGS2).  Everything inside a
// restart cycle stays on the device in FP64: the Krylov basis, the operator,
// the Gram-Schmidt coefficients, the Hessenberg column, the Givens rotations
// and the residual estimate |g_{j+1}| / ||r_0|| of the small least-squares
// problem.  The host only enqueues each Arnoldi step (two graph launches: the
// product, then the rest of the step, whose kernels read the step index from
// device memory) and reads the estimate of the step before (so the GPU
// always has the next step queued); once the
// estimate predicts convergence within a step it reads every step's estimate
// as soon as that step ends.  A restart cycle ends with one synchronisation:
// the back substitution on the (at most 255 x 255) triangular system and the
// true residual of the next cycle.
//
// Chosen precision: GMRES runs on the FP32 FDA operator, inside an outer
// loop that re-evaluates the true residual b - A x with the FP64 operator
// (iterative refinement); convergence is judged on that FP64 residual.  The
// inner solves form their Gram-Schmidt products in FP32 (summed in FP64).
#include <math.h>

#include <chrono>
#include <complex>
#include <vector>

#include "fda_internal.cuh"

namespace {

constexpr int RT = 256;
constexpr int RCH = 1024;  // most chunks per vector for the two-stage dot products
constexpr int DEL = 4;     // elements per thread and chunk (chunks of RT x DEL elements)
// partial[i * rch + c] = sum over chunk c of conj(V_i[n]) w[n] for the G
// vectors of this CTA's group (blockIdx.y).  Every thread reads its w values
// once and accumulates the G products from them in the type P, then sums
// across its warp in P; the warps' sums are added in FP64.  P = double for
// the FP64 solve; P = float for the inner solves of the chosen form, whose
// tolerance (>= 1e-5) is far above FP32 rounding and whose result the FP64
// residual of the outer loop judges: GB300's FP64 rate (about 1/64 of FP32)
// would otherwise make these memory-sized passes compute-bound.
constexpr int DVG = 8;  // vectors per CTA
template <int G, typename P>
__device__ __forceinline__ void dots_group(const c64d *V, int64_t ldv, int nv, const c64d *w, int64_t n,
                                           c64d *partial, int rch, int i0)
{
    __shared__ double sr[RT / 32][G], si[RT / 32][G];
    const int c = blockIdx.x, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ng = min(G, nv - i0);
    const int64_t per = (n + rch - 1) / rch;
    const int64_t b = (int64_t)c * per, e = b + per < n ? b + per : n;
    P ar[G], ai[G];
#pragma unroll
    for (int g = 0; g < G; ++g) ar[g] = ai[g] = (P)0;
    for (int64_t t = b + threadIdx.x; t < e; t += RT) {
        const c64d xd = w[t];
        const P xr = (P)xd.re, xi = (P)xd.im;
#pragma unroll
        for (int g = 0; g < G; ++g)
            if (g < ng) {
                const c64d a = V[(int64_t)(i0 + g) * ldv + t];
                const P vr = (P)a.re, vi = (P)a.im;
                ar[g] += vr * xr + vi * xi;
                ai[g] += vr * xi - vi * xr;
            }
    }
#pragma unroll
    for (int g = 0; g < G; ++g)
        for (int o = 16; o > 0; o >>= 1) {
            ar[g] += __shfl_xor_sync(0xffffffffu, ar[g], o);
            ai[g] += __shfl_xor_sync(0xffffffffu, ai[g], o);
        }
    if (lane == 0)
#pragma unroll
        for (int g = 0; g < G; ++g) {
            sr[warp][g] = (double)ar[g];
            si[warp][g] = (double)ai[g];
        }
    __syncthreads();
    if (threadIdx.x < ng) {
        double r = 0.0, im = 0.0;
        for (int q = 0; q < RT / 32; ++q) {
            r += sr[q][threadIdx.x];
            im += si[q][threadIdx.x];
        }
        partial[(int64_t)(i0 + threadIdx.x) * rch + c] = c64d(r, im);
    }
}
template <int G, typename P>
__global__ void __launch_bounds__(RT) k_dots(const c64d *V, int64_t ldv, int nv, const c64d *w, int64_t n,
                                             c64d *partial, int rch)
{
    dots_group<G, P>(V, ldv, nv, w, n, partial, rch, blockIdx.y * G);
}

__device__ __forceinline__ void finish_one(const c64d *partial, int i, c64d *out, int rch)
{
    __shared__ double sr[RT], si[RT];
    double ar = 0.0, ai = 0.0;
    for (int c = threadIdx.x; c < rch; c += RT) {
        ar += partial[(int64_t)i * rch + c].re;
        ai += partial[(int64_t)i * rch + c].im;
    }
    sr[threadIdx.x] = ar;
    si[threadIdx.x] = ai;
    __syncthreads();
    for (int s = RT / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) {
            sr[threadIdx.x] += sr[threadIdx.x + s];
            si[threadIdx.x] += si[threadIdx.x + s];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) out[i] = c64d(sr[0], si[0]);
}

__global__ void k_dots_finish(const c64d *partial, int nv, c64d *out, int rch)
{
    finish_one(partial, blockIdx.x, out, rch);
}

// w[n] += sign * sum_i V_i[n] c[i]; the coefficients are staged in shared
// memory and the vectors read four at a time; the sum is formed in P (as in
// k_dots) and added to w in FP64
template <typename P>
__device__ __forceinline__ void combine_body(const c64d *V, int64_t ldv, int nv, const c64d *c, double sign,
                                             c64d *w, int64_t n)
{
    __shared__ P csr[256], csi[256];
    for (int i = threadIdx.x; i < nv && i < 256; i += RT) {
        csr[i] = (P)c[i].re;
        csi[i] = (P)c[i].im;
    }
    __syncthreads();
    auto cs = [&](int i) { return cx<P>(csr[i], csi[i]); };
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= n) return;
    auto ld = [&](int i) {
        const c64d a = V[(int64_t)i * ldv + t];
        return cx<P>((P)a.re, (P)a.im);
    };
    cx<P> acc;
    int i = 0;
    for (; i + 3 < nv; i += 4) {
        const cx<P> a0 = ld(i), a1 = ld(i + 1), a2 = ld(i + 2), a3 = ld(i + 3);
        cfma(acc, a0, cs(i));
        cfma(acc, a1, cs(i + 1));
        cfma(acc, a2, cs(i + 2));
        cfma(acc, a3, cs(i + 3));
    }
    for (; i < nv; ++i) cfma(acc, ld(i), cs(i));
    w[t] = c64d(w[t].re + sign * (double)acc.re, w[t].im + sign * (double)acc.im);
}

template <typename P>
__global__ void __launch_bounds__(RT) k_combine(const c64d *V, int64_t ldv, int nv, const c64d *c, double sign,
                                                c64d *w, int64_t n)
{
    combine_body<P>(V, ldv, nv, c, sign, w, n);
}

// ---- the Gram-Schmidt part of Arnoldi step j with j read from device
// memory (*jd), so that one captured graph serves every step of a cycle:
// w = V_{j+1} (the new product), nv = j + 1 basis vectors (1 with self: the
// dot product of w with itself)
template <int G, typename P>
__global__ void __launch_bounds__(RT) k_dots_j(const c64d *V, int64_t n, const int *jd, int self, c64d *partial,
                                               int rch)
{
    const int j = *jd;
    const c64d *w = V + (int64_t)(j + 1) * n;
    const int nv = self ? 1 : j + 1;
    for (int i0 = 0; i0 < nv; i0 += G) {  // the groups one after another: w is re-read from L2
        dots_group<G, P>(self ? w : V, n, nv, w, n, partial, rch, i0);
        __syncthreads();
    }
}

__global__ void k_dots_finish_j(const c64d *partial, const int *jd, int self, c64d *out, int rch)
{
    const int nv = self ? 1 : *jd + 1;
    if ((int)blockIdx.x < nv) finish_one(partial, blockIdx.x, out, rch);
}

template <typename P>
__global__ void __launch_bounds__(RT) k_combine_j(c64d *V, int64_t n, const int *jd, const c64d *c, double sign)
{
    const int j = *jd;
    combine_body<P>(V, n, j + 1, c, sign, V + (int64_t)(j + 1) * n, n);
}

// Device state of one Arnoldi step, copied to pinned host memory after the
// step: the residual estimate, ||w|| after orthogonalisation, and flags
// (bit 0: a non-finite Hessenberg entry, bit 1: breakdown, ||w|| tiny).
struct gm_status {
    double est, hn;
    int flags, j;
};

// The small work of Arnoldi step j on one thread: the Hessenberg column
// h = c1 + c2 (the two Gram-Schmidt passes) with h_{j+1} = ||w||, the
// previous Givens rotations applied to it, the new rotation that zeroes
// h_{j+1}, and the rotated right-hand side g of the least-squares problem.
// H is column-major with leading dimension ldh; *scale receives 1/||w||.
__device__ void arnoldi_body(int j, int ldh, const c64d *c1, const c64d *c2, const c64d *nrm2, c64d *H, c64d *cs,
                             c64d *sn, c64d *g, double rnorm0, double beta, double *scale, gm_status *st)
{
    c64d *hc = H + (int64_t)j * ldh;
    int bad = 0;
    for (int i = 0; i <= j; ++i) {
        const c64d v = c1[i] + c2[i];
        hc[i] = v;
        bad |= !isfinite(v.re) || !isfinite(v.im);
    }
    const double hn = sqrt(fmax(nrm2->re, 0.0));
    bad |= !isfinite(hn);
    *scale = hn > 0.0 ? 1.0 / hn : 1.0;
    c64d hj1(hn, 0.0);
    for (int i = 0; i < j; ++i) {
        // (h_i, h_{i+1}) <- (c h_i + s h_{i+1}, -conj(s) h_i + conj(c) h_{i+1})
        const c64d a = hc[i], b = hc[i + 1];
        hc[i] = cs[i] * a + sn[i] * b;
        hc[i + 1] = conjg(cs[i]) * b - conjg(sn[i]) * a;
    }
    const c64d hjj = hc[j];
    const double den = sqrt(hjj.re * hjj.re + hjj.im * hjj.im + hj1.re * hj1.re + hj1.im * hj1.im);
    c64d c(1.0, 0.0), s(0.0, 0.0);
    if (den > 0.0) {
        c = c64d(hjj.re / den, -hjj.im / den);
        s = c64d(hj1.re / den, -hj1.im / den);
    }
    cs[j] = c;
    sn[j] = s;
    hc[j] = c * hjj + s * hj1;
    hc[j + 1] = c64d();
    const c64d gj = g[j];
    g[j + 1] = c64d() - conjg(s) * gj;
    g[j] = c * gj;
    const c64d gn = g[j + 1];
    st->est = sqrt(gn.re * gn.re + gn.im * gn.im) / rnorm0;
    st->hn = hn;
    st->flags = (bad ? 1 : 0) | (hn <= 1e-14 * beta ? 2 : 0);
    st->j = j;
}

// the same with j read from *jd and its status in slot j % ring of st; the
// step then advances *jd (the next step's Gram-Schmidt kernels read it)
__global__ void k_arnoldi_step_j(int *jd, int ldh, const c64d *c1, const c64d *c2, const c64d *nrm2, c64d *H,
                                 c64d *cs, c64d *sn, c64d *g, const double *rb, double *scale, gm_status *st,
                                 int ring)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const int j = *jd;
    arnoldi_body(j, ldh, c1, c2, nrm2, H, cs, sn, g, rb[0], rb[1], scale, st + j % ring);
    *jd = j + 1;
}

// V_{*jd} *= *s (the new basis vector, after the step advanced *jd)
__global__ void k_scale_j(c64d *V, int64_t n, const int *jd, const double *s)
{
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t < n) {
        c64d *x = V + (int64_t)(*jd) * n;
        const double f = *s;
        x[t] = c64d(x[t].re * f, x[t].im * f);
    }
}

// start of a restart cycle: g = beta e_1, step index 0, and the cycle's
// ||r_0|| and beta for the Arnoldi kernel (rb)
__global__ void k_gmres_init(c64d *g, int n, double beta, int *jd, double *rb, double rnorm0)
{
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) g[t] = c64d(t == 0 ? beta : 0.0, 0.0);
    if (t == 0) {
        *jd = 0;
        rb[0] = rnorm0;
        rb[1] = beta;
    }
}

__global__ void k_axpby(const c64d *x, double a, const c64d *y, double b, c64d *out, int64_t n)
{
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t < n) out[t] = c64d(a * x[t].re + b * y[t].re, a * x[t].im + b * y[t].im);
}

__global__ void k_scale(c64d *x, double s, int64_t n)
{
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t < n) x[t] = c64d(x[t].re * s, x[t].im * s);
}

struct solver {
    fda_handle *h;
    int64_t n;
    dbuf partial, hd;
    double matvec_time = 0;
    int nmatvec = 0;
    // device state of the current restart cycle: Hessenberg columns (ldh =
    // m + 1), Givens rotations, rotated right-hand side, Gram-Schmidt
    // coefficients of the two passes, ||w||^2, 1/||w||, step status
    dbuf Hd, csd, snd, gd, c1d, c2d, nrm2d, scaled, st_ring, yd, jd, rb;
    // the Gram-Schmidt part of a step as one graph per basis (V) and
    // product arithmetic (FP64, FP32), captured on a private stream
    cudaStream_t cap = nullptr;
    cudaGraphExec_t gsx[2] = {};
    const c64d *gsV[2] = {};
    gm_status *hst = nullptr;   // pinned: status of the last RING steps
    c64d *hH = nullptr, *hg = nullptr, *hy = nullptr;  // pinned: H, g, y of a cycle
    static constexpr int RING = 4;
    cudaEvent_t sev[RING] = {};
    // matvec timing: event pairs around each product, read back in batches
    static constexpr int MVR = 64;
    cudaEvent_t mv0[MVR] = {}, mv1[MVR] = {};
    int mv_pending = 0;
    int ldh = 0;

    ~solver()
    {
        for (int i = 0; i < RING; ++i)
            if (sev[i]) cudaEventDestroy(sev[i]);
        for (int i = 0; i < MVR; ++i) {
            if (mv0[i]) cudaEventDestroy(mv0[i]);
            if (mv1[i]) cudaEventDestroy(mv1[i]);
        }
        for (int i = 0; i < 2; ++i)
            if (gsx[i]) cudaGraphExecDestroy(gsx[i]);
        if (cap) cudaStreamDestroy(cap);
        if (hst) cudaFreeHost(hst);
        if (hH) cudaFreeHost(hH);
        if (hg) cudaFreeHost(hg);
        if (hy) cudaFreeHost(hy);
    }

    void setup(int m)
    {
        ldh = m + 1;
        partial.alloc(sizeof(c64d) * RCH * (size_t)(m + 2));
        hd.alloc(sizeof(c64d) * (size_t)(m + 2));
        Hd.alloc(sizeof(c64d) * (size_t)ldh * m);
        csd.alloc(sizeof(c64d) * m);
        snd.alloc(sizeof(c64d) * m);
        gd.alloc(sizeof(c64d) * (m + 1));
        c1d.alloc(sizeof(c64d) * (m + 1));
        c2d.alloc(sizeof(c64d) * (m + 1));
        nrm2d.alloc(sizeof(c64d));
        scaled.alloc(sizeof(double));
        st_ring.alloc(sizeof(gm_status) * RING);
        jd.alloc(sizeof(int));
        rb.alloc(2 * sizeof(double));
        FDA_CUDA(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
        yd.alloc(sizeof(c64d) * (m + 1));
        FDA_CUDA(cudaMallocHost(&hst, sizeof(gm_status) * RING));
        FDA_CUDA(cudaMallocHost(&hH, sizeof(c64d) * (size_t)ldh * m));
        FDA_CUDA(cudaMallocHost(&hg, sizeof(c64d) * (m + 1)));
        FDA_CUDA(cudaMallocHost(&hy, sizeof(c64d) * (m + 1)));
        for (int i = 0; i < RING; ++i) FDA_CUDA(cudaEventCreateWithFlags(&sev[i], cudaEventDisableTiming));
        for (int i = 0; i < MVR; ++i) {
            FDA_CUDA(cudaEventCreate(&mv0[i]));
            FDA_CUDA(cudaEventCreate(&mv1[i]));
        }
    }

    // out[i] = V_i^H w for i < nv; lowp: products in FP32 (inner solves of
    // the chosen form), else FP64
    void dots_dev(const c64d *V, int nv, const c64d *w, c64d *out, bool lowp = false)
    {
        // chunks of RT x DEL elements, at most 2048 CTAs over all groups
        const int ng = nv == 1 ? 1 : (nv + DVG - 1) / DVG;
        const int64_t want = (n + (int64_t)RT * DEL - 1) / ((int64_t)RT * DEL);
        const int rch = (int)std::max<int64_t>(1, std::min<int64_t>(want, std::min(RCH, std::max(1, 2048 / ng))));
        dim3 g(rch, ng);
        if (nv == 1) {
            if (lowp) k_dots<1, float><<<g, RT, 0, h->stream>>>(V, n, nv, w, n, partial.as<c64d>(), rch);
            else k_dots<1, double><<<g, RT, 0, h->stream>>>(V, n, nv, w, n, partial.as<c64d>(), rch);
        } else {
            if (lowp) k_dots<DVG, float><<<g, RT, 0, h->stream>>>(V, n, nv, w, n, partial.as<c64d>(), rch);
            else k_dots<DVG, double><<<g, RT, 0, h->stream>>>(V, n, nv, w, n, partial.as<c64d>(), rch);
        }
        FDA_CHECK_LAUNCH();
        k_dots_finish<<<nv, RT, 0, h->stream>>>(partial.as<c64d>(), nv, out, rch);
        FDA_CHECK_LAUNCH();
    }
    // ||w|| on the host (synchronises; once per restart cycle)
    double norm(const c64d *w)
    {
        dots_dev(w, 1, w, hd.as<c64d>());
        c64d d;
        FDA_CUDA(cudaMemcpyAsync(&d, hd.p, sizeof(c64d), cudaMemcpyDeviceToHost, h->stream));
        FDA_CUDA(cudaStreamSynchronize(h->stream));
        return sqrt(std::max(d.re, 0.0));
    }
    // w += sign * V c, coefficients c on the device
    void combine_dev(const c64d *V, int nv, const c64d *c, double sign, c64d *w, bool lowp = false)
    {
        if (lowp) k_combine<float><<<fda_blocks(n, RT), RT, 0, h->stream>>>(V, n, nv, c, sign, w, n);
        else k_combine<double><<<fda_blocks(n, RT), RT, 0, h->stream>>>(V, n, nv, c, sign, w, n);
        FDA_CHECK_LAUNCH();
    }
    void collect_matvec_times()
    {
        for (int i = 0; i < mv_pending; ++i) {
            float ms = 0.0f;
            FDA_CUDA(cudaEventSynchronize(mv1[i]));
            FDA_CUDA(cudaEventElapsedTime(&ms, mv0[i], mv1[i]));
            matvec_time += 1e-3 * ms;
        }
        mv_pending = 0;
    }
    dbuf ptmp;
    // y = A M x when the preconditioner is on (right preconditioning), else A x
    void apply_op(const c64d *x, c64d *y, int precision)
    {
        if (h->cfg.precond != 0) {
            if (!ptmp.p) ptmp.alloc(sizeof(c64d) * n);
            fda_precond_apply(h, x, ptmp.as<c64d>());
            apply(ptmp.as<c64d>(), y, precision);
        } else {
            apply(x, y, precision);
        }
    }
    // stream-ordered product (no synchronisation); its device time is
    // measured with an event pair
    void apply(const c64d *x, c64d *y, int precision)
    {
        if (mv_pending == MVR) collect_matvec_times();
        FDA_CUDA(cudaEventRecord(mv0[mv_pending], h->stream));
        // through the handle's staging vectors, so every product replays the
        // same captured graph
        FDA_CUDA(cudaMemcpyAsync(h->xs.p, x, sizeof(c64d) * n, cudaMemcpyDeviceToDevice, h->stream));
        fda_apply_staged(h, precision, 1);
        FDA_CUDA(cudaMemcpyAsync(y, h->ys.p, sizeof(c64d) * n, cudaMemcpyDeviceToDevice, h->stream));
        FDA_CUDA(cudaEventRecord(mv1[mv_pending], h->stream));
        ++mv_pending;
        ++nmatvec;
    }

    // the Gram-Schmidt part of the step whose product is V_{*jd + 1}: two
    // CGS passes, ||w||, the Hessenberg column and Givens rotation, the
    // scaling of the new basis vector, and the status ring to the host
    void gs_launch(cudaStream_t s, c64d *V, bool lowp)
    {
        const int rch = (int)std::max<int64_t>(1, std::min<int64_t>(RCH, (n + (int64_t)RT * DEL - 1) /
                                                                             ((int64_t)RT * DEL)));
        for (int pass = 0; pass < 2; ++pass) {
            c64d *c = (pass ? c2d : c1d).as<c64d>();
            if (lowp) k_dots_j<DVG, float><<<rch, RT, 0, s>>>(V, n, jd.as<int>(), 0, partial.as<c64d>(), rch);
            else k_dots_j<DVG, double><<<rch, RT, 0, s>>>(V, n, jd.as<int>(), 0, partial.as<c64d>(), rch);
            FDA_CHECK_LAUNCH();
            k_dots_finish_j<<<ldh, RT, 0, s>>>(partial.as<c64d>(), jd.as<int>(), 0, c, rch);
            FDA_CHECK_LAUNCH();
            if (lowp) k_combine_j<float><<<fda_blocks(n, RT), RT, 0, s>>>(V, n, jd.as<int>(), c, -1.0);
            else k_combine_j<double><<<fda_blocks(n, RT), RT, 0, s>>>(V, n, jd.as<int>(), c, -1.0);
            FDA_CHECK_LAUNCH();
        }
        k_dots_j<1, double><<<rch, RT, 0, s>>>(V, n, jd.as<int>(), 1, partial.as<c64d>(), rch);
        FDA_CHECK_LAUNCH();
        k_dots_finish_j<<<1, RT, 0, s>>>(partial.as<c64d>(), jd.as<int>(), 1, nrm2d.as<c64d>(), rch);
        FDA_CHECK_LAUNCH();
        k_arnoldi_step_j<<<1, 32, 0, s>>>(jd.as<int>(), ldh, c1d.as<c64d>(), c2d.as<c64d>(), nrm2d.as<c64d>(),
                                          Hd.as<c64d>(), csd.as<c64d>(), snd.as<c64d>(), gd.as<c64d>(),
                                          rb.as<double>(), scaled.as<double>(), st_ring.as<gm_status>(), RING);
        FDA_CHECK_LAUNCH();
        k_scale_j<<<fda_blocks(n, RT), RT, 0, s>>>(V, n, jd.as<int>(), scaled.as<double>());
        FDA_CHECK_LAUNCH();
        FDA_CUDA(cudaMemcpyAsync(hst, st_ring.p, sizeof(gm_status) * RING, cudaMemcpyDeviceToHost, s));
    }
    // capture gs_launch for this basis once; on failure the kernels are
    // launched one by one
    void gs_graph(c64d *V, bool lowp)
    {
        const int i = lowp ? 1 : 0;
        if (gsV[i] == V && gsx[i]) return;
        if (gsx[i]) cudaGraphExecDestroy(gsx[i]);
        gsx[i] = nullptr;
        gsV[i] = V;
        cudaGraph_t g = nullptr;
        bool ok = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
        if (ok) {
            try {
                gs_launch(cap, V, lowp);
            } catch (...) {
                ok = false;
            }
            ok = cudaStreamEndCapture(cap, &g) == cudaSuccess && ok && g;
        }
        if (ok) ok = cudaGraphInstantiate(&gsx[i], g, 0) == cudaSuccess;
        if (g) cudaGraphDestroy(g);
        if (!ok) {
            (void)cudaGetLastError();
            gsx[i] = nullptr;
        }
    }

    // one Arnoldi step j of the current cycle, enqueued without
    // synchronisation; the status ring lands in hst, signalled by sev[j % RING]
    void arnoldi_step(c64d *V, int j, int precision)
    {
        c64d *vj = V + (int64_t)j * n, *vn = V + (int64_t)(j + 1) * n;
        const bool lowp = precision == FDA_CHOSEN_FP32;
        apply_op(vj, vn, precision);
        const int i = lowp ? 1 : 0;
        if (gsx[i] && gsV[i] == V) FDA_CUDA(cudaGraphLaunch(gsx[i], h->stream));
        else gs_launch(h->stream, V, lowp);
        FDA_CUDA(cudaEventRecord(sev[j % RING], h->stream));
    }
    const gm_status &status(int j)
    {
        FDA_CUDA(cudaEventSynchronize(sev[j % RING]));
        const gm_status &s = hst[j % RING];
        if (s.flags & 1) fda_fail(FDA_ERR_NUMERIC, "non-finite Hessenberg entry in GMRES");
        return s;
    }

    // GMRES(m) on A_prec: solve A d = r to ||r - A d|| <= tol_rel ||r||; d in/out
    // (d_zero: the caller knows d = 0, so the first residual is r itself)
    int gmres(const c64d *r, c64d *d, double tol_rel, int precision, int maxit, int &iters_out, double &est,
              bool d_zero = false)
    {
        const int m = std::max(1, h->cfg.restart);
        if (ldh != m + 1) setup(m);
        dbuf Vb, w;
        Vb.alloc(sizeof(c64d) * (size_t)(m + 1) * n);
        w.alloc(sizeof(c64d) * n);
        c64d *V = Vb.as<c64d>();
        gs_graph(V, precision == FDA_CHOSEN_FP32);
        double rnorm0 = norm(r);
        iters_out = 0;
        est = 0.0;
        if (rnorm0 == 0.0) {
            FDA_CUDA(cudaMemsetAsync(d, 0, sizeof(c64d) * n, h->stream));
            return 0;
        }
        int it = 0;
        bool first = true;
        while (true) {
            // residual of the current d: v0 = r - A d (no product while d = 0)
            if (first && d_zero) {
                FDA_CUDA(cudaMemcpyAsync(V, r, sizeof(c64d) * n, cudaMemcpyDeviceToDevice, h->stream));
            } else {
                apply(d, w.as<c64d>(), precision);
                k_axpby<<<fda_blocks(n, RT), RT, 0, h->stream>>>(r, 1.0, w.as<c64d>(), -1.0, V, n);
                FDA_CHECK_LAUNCH();
            }
            first = false;
            double beta = norm(V);
            if (!std::isfinite(beta)) fda_fail(FDA_ERR_NUMERIC, "non-finite residual in GMRES");
            est = beta / rnorm0;
            if (est <= tol_rel) break;
            if (it >= maxit) return 1;
            k_scale<<<fda_blocks(n, RT), RT, 0, h->stream>>>(V, 1.0 / beta, n);
            FDA_CHECK_LAUNCH();
            k_gmres_init<<<1, 256, 0, h->stream>>>(gd.as<c64d>(), m + 1, beta, jd.as<int>(), rb.as<double>(),
                                                   rnorm0);
            FDA_CHECK_LAUNCH();
            // Arnoldi steps: step j is enqueued before the host waits for the
            // status of step j - 1, so the device always has work queued; once
            // the estimates predict convergence at the next step, each step is
            // waited for right after it is enqueued.
            int jend = 0;          // columns of this cycle's least-squares problem
            bool eager = false;    // wait for each step's own status
            double e_prev = est, e_prev2 = est;
            for (int j = 0; j < m && it < maxit; ++j) {
                arnoldi_step(V, j, precision);
                ++it;
                ++iters_out;
                jend = j + 1;
                const int jc = eager ? j : j - 1;  // step whose status is read now
                if (jc < 0) continue;
                const gm_status &s = status(jc);
                const bool done = s.est <= tol_rel || (s.flags & 2);
                if (done) {
                    est = s.est;
                    if (jc < j) {  // step j was enqueued past convergence: not used
                        --it;
                        --iters_out;
                        jend = j;
                    }
                    break;
                }
                est = s.est;
                e_prev2 = e_prev;
                e_prev = s.est;
                // predicted estimate one step on, at the last step's rate
                const double rate = e_prev2 > 0.0 ? std::min(1.0, e_prev / e_prev2) : 1.0;
                if (!eager && e_prev * rate * rate <= 2.0 * tol_rel) eager = true;
            }
            // the cycle's last status (when the loop ended at m or maxit)
            if (jend > 0) {
                const gm_status &s = status(jend - 1);
                est = s.est;
            }
            // back substitution H y = g on the host, then d += V y (or M V y)
            const int j = jend;
            FDA_CUDA(cudaMemcpyAsync(hH, Hd.p, sizeof(c64d) * (size_t)ldh * j, cudaMemcpyDeviceToHost, h->stream));
            FDA_CUDA(cudaMemcpyAsync(hg, gd.p, sizeof(c64d) * j, cudaMemcpyDeviceToHost, h->stream));
            FDA_CUDA(cudaStreamSynchronize(h->stream));
            std::vector<std::complex<double>> y(j, 0.0);
            auto Hij = [&](int i, int k) { return std::complex<double>(hH[(size_t)k * ldh + i].re, hH[(size_t)k * ldh + i].im); };
            for (int i = j - 1; i >= 0; --i) {
                std::complex<double> s(hg[i].re, hg[i].im);
                for (int k = i + 1; k < j; ++k) s -= Hij(i, k) * y[k];
                y[i] = s / Hij(i, i);
                hy[i] = c64d(y[i].real(), y[i].imag());
            }
            FDA_CUDA(cudaMemcpyAsync(yd.p, hy, sizeof(c64d) * j, cudaMemcpyHostToDevice, h->stream));
            if (h->cfg.precond != 0) {
                // d += M (V y): form V y in w, then apply M into the basis slot V_m (free now)
                FDA_CUDA(cudaMemsetAsync(w.p, 0, sizeof(c64d) * n, h->stream));
                combine_dev(V, j, yd.as<c64d>(), 1.0, w.as<c64d>());
                c64d *tmp = V + (int64_t)m * n;
                fda_precond_apply(h, w.as<c64d>(), tmp);
                k_axpby<<<fda_blocks(n, RT), RT, 0, h->stream>>>(d, 1.0, tmp, 1.0, d, n);
                FDA_CHECK_LAUNCH();
            } else {
                combine_dev(V, j, yd.as<c64d>(), 1.0, d);
            }
        }
        return 0;
    }
};

__global__ void k_sub(const c64d *a, const c64d *b, c64d *o, int64_t n)
{
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t < n) o[t] = a[t] - b[t];
}

__global__ void k_add(c64d *a, const c64d *b, int64_t n)
{
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t < n) a[t] = a[t] + b[t];
}

}  // namespace

fda_status fda_solve_impl(fda_handle *h, const c64d *b, c64d *x, double tol, fda_info *info)
{
    auto t0 = std::chrono::steady_clock::now();
    const int64_t n = h->N;
    solver S;
    S.h = h;
    S.n = n;
    S.setup(std::max(1, h->cfg.restart));
    dbuf bs, xs, r, d, ax;
    bs.alloc(sizeof(c64d) * n);
    xs.alloc(sizeof(c64d) * n);
    r.alloc(sizeof(c64d) * n);
    d.alloc(sizeof(c64d) * n);
    ax.alloc(sizeof(c64d) * n);
    fda_gather_to_sorted(h, b, bs.as<c64d>());
    fda_gather_to_sorted(h, x, xs.as<c64d>());
    double bnorm = S.norm(bs.as<c64d>());
    int iters = 0, refinements = 0;
    double rel = 0.0;
    bool rel_of_x = false;  // rel already holds the FP64 residual of the current x
    fda_status st = FDA_OK;
    if (bnorm == 0.0) {
        FDA_CUDA(cudaMemsetAsync(xs.p, 0, sizeof(c64d) * n, h->stream));
    } else if (h->cfg.precision == FDA_PLAIN_FP64) {
        int it = 0;
        double est = 0;
        // solve A x = b directly: r = b, d = x
        const bool x_zero = S.norm(xs.as<c64d>()) == 0.0;
        int rc = S.gmres(bs.as<c64d>(), xs.as<c64d>(), tol, FDA_PLAIN_FP64, h->cfg.maxit, it, est, x_zero);
        iters = it;
        refinements = 0;
        (void)rc;
    } else {
        // outer FP64 residual, inner FP32 GMRES
        int budget = h->cfg.maxit;
        bool x_zero = S.norm(xs.as<c64d>()) == 0.0;
        for (int pass = 0; pass < 20; ++pass) {
            if (x_zero) {
                // r = b - A 0 = b: no FP64 product needed
                FDA_CUDA(cudaMemcpyAsync(r.p, bs.p, sizeof(c64d) * n, cudaMemcpyDeviceToDevice, h->stream));
                rel = 1.0;
            } else {
                S.apply(xs.as<c64d>(), ax.as<c64d>(), FDA_PLAIN_FP64);
                ++refinements;
                k_sub<<<fda_blocks(n, RT), RT, 0, h->stream>>>(bs.as<c64d>(), ax.as<c64d>(), r.as<c64d>(), n);
                FDA_CHECK_LAUNCH();
                rel = S.norm(r.as<c64d>()) / bnorm;
                rel_of_x = true;
            }
            if (rel <= tol || budget <= 0) break;
            // the FP32 operator reaches ~1e-6 relative at best: ask the inner
            // solve for at most 1e-5 and let the FP64 refinement passes do the rest
            double tin = std::min(0.5, std::max(1e-5, 0.5 * tol / rel));
            FDA_CUDA(cudaMemsetAsync(d.p, 0, sizeof(c64d) * n, h->stream));
            int it = 0;
            double est = 0;
            S.gmres(r.as<c64d>(), d.as<c64d>(), tin, FDA_CHOSEN_FP32, budget, it, est, true);
            iters += it;
            budget -= it;
            k_add<<<fda_blocks(n, RT), RT, 0, h->stream>>>(xs.as<c64d>(), d.as<c64d>(), n);
            FDA_CHECK_LAUNCH();
            x_zero = false;
            rel_of_x = false;
        }
    }
    // final FP64 residual (unless the refinement loop just computed it)
    if (bnorm > 0 && !rel_of_x) {
        S.apply(xs.as<c64d>(), ax.as<c64d>(), FDA_PLAIN_FP64);
        k_sub<<<fda_blocks(n, RT), RT, 0, h->stream>>>(bs.as<c64d>(), ax.as<c64d>(), r.as<c64d>(), n);
        FDA_CHECK_LAUNCH();
        rel = S.norm(r.as<c64d>()) / bnorm;
    }
    fda_scatter_from_sorted(h, xs.as<c64d>(), x);
    FDA_CUDA(cudaStreamSynchronize(h->stream));
    S.collect_matvec_times();
    if (!(rel <= tol)) st = FDA_ERR_NOT_CONVERGED;
    if (!std::isfinite(rel)) st = FDA_ERR_NUMERIC;
    if (info) {
        info->iters = iters;
        info->refinements = refinements;
        info->rel_resid_fp64 = rel;
        info->setup_s = h->tree_s + h->precompute_s;
        info->solve_s = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        info->matvec_s = S.nmatvec ? S.matvec_time / S.nmatvec : 0.0;
    }
    if (st == FDA_ERR_NOT_CONVERGED) h->err = "GMRES reached maxit above the tolerance";
    return st;
}
