// GMRES solve of Sec. 5 (no preconditioner, tolerance on the relative
// residual of the unpreconditioned system).  Readings of what the paper
// leaves open: restarted GMRES(m), zero or caller initial guess, classical
// Gram-Schmidt with one re-orthogonalisation (CGS2).  The Krylov basis, the
// operator and every vector operation live on the device in FP64; the small
// Hessenberg least-squares problem (Givens rotations on an (m+1) x m matrix)
// is updated on the host after each Arnoldi step, which is also where the
// convergence test reads the residual estimate.
//
// Chosen precision: GMRES runs on the FP32 FDA operator, inside an outer
// loop that re-evaluates the true residual b - A x with the FP64 operator
// (iterative refinement); convergence is judged on that FP64 residual.
#include <math.h>

#include <chrono>
#include <complex>
#include <vector>

#include "fda_internal.cuh"

namespace {

constexpr int RT = 256;
constexpr int RCH = 128;  // chunks per vector for the two-stage dot products

// partial[i * RCH + c] = sum over chunk c of conj(V_i[n]) w[n].  A CTA takes
// one chunk of the index range and a group of DVG vectors: every thread
// reads its w values once and accumulates DVG products from them, then the
// DVG sums are reduced across the CTA.
constexpr int DVG = 8;  // vectors per CTA

__global__ void __launch_bounds__(RT) k_dots(const c64d *V, int64_t ldv, int nv, const c64d *w, int64_t n,
                                             c64d *partial)
{
    __shared__ double sr[RT / 32][DVG], si[RT / 32][DVG];
    const int c = blockIdx.x, i0 = blockIdx.y * DVG, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ng = min(DVG, nv - i0);
    const int64_t per = (n + RCH - 1) / RCH;
    const int64_t b = (int64_t)c * per, e = b + per < n ? b + per : n;
    double ar[DVG], ai[DVG];
#pragma unroll
    for (int g = 0; g < DVG; ++g) ar[g] = ai[g] = 0.0;
    for (int64_t t = b + threadIdx.x; t < e; t += RT) {
        const c64d x = w[t];
#pragma unroll
        for (int g = 0; g < DVG; ++g)
            if (g < ng) {
                const c64d a = V[(int64_t)(i0 + g) * ldv + t];
                ar[g] += a.re * x.re + a.im * x.im;
                ai[g] += a.re * x.im - a.im * x.re;
            }
    }
#pragma unroll
    for (int g = 0; g < DVG; ++g)
        for (int o = 16; o > 0; o >>= 1) {
            ar[g] += __shfl_xor_sync(0xffffffffu, ar[g], o);
            ai[g] += __shfl_xor_sync(0xffffffffu, ai[g], o);
        }
    if (lane == 0)
#pragma unroll
        for (int g = 0; g < DVG; ++g) {
            sr[warp][g] = ar[g];
            si[warp][g] = ai[g];
        }
    __syncthreads();
    if (threadIdx.x < ng) {
        double r = 0.0, im = 0.0;
        for (int q = 0; q < RT / 32; ++q) {
            r += sr[q][threadIdx.x];
            im += si[q][threadIdx.x];
        }
        partial[(int64_t)(i0 + threadIdx.x) * RCH + c] = c64d(r, im);
    }
}

__global__ void k_dots_finish(const c64d *partial, int nv, c64d *out)
{
    __shared__ double sr[RT], si[RT];
    int i = blockIdx.x;
    double ar = 0.0, ai = 0.0;
    for (int c = threadIdx.x; c < RCH; c += RT) {
        ar += partial[(int64_t)i * RCH + c].re;
        ai += partial[(int64_t)i * RCH + c].im;
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

// w[n] += sign * sum_i V_i[n] c[i]; the coefficients are staged in shared
// memory and the vectors read four at a time
__global__ void __launch_bounds__(RT) k_combine(const c64d *V, int64_t ldv, int nv, const c64d *c, double sign,
                                                c64d *w, int64_t n)
{
    __shared__ c64d cs[256];
    for (int i = threadIdx.x; i < nv && i < 256; i += RT) cs[i] = c[i];
    __syncthreads();
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= n) return;
    c64d acc;
    int i = 0;
    for (; i + 3 < nv; i += 4) {
        const c64d a0 = V[(int64_t)i * ldv + t], a1 = V[(int64_t)(i + 1) * ldv + t];
        const c64d a2 = V[(int64_t)(i + 2) * ldv + t], a3 = V[(int64_t)(i + 3) * ldv + t];
        cfma(acc, a0, cs[i]);
        cfma(acc, a1, cs[i + 1]);
        cfma(acc, a2, cs[i + 2]);
        cfma(acc, a3, cs[i + 3]);
    }
    for (; i < nv; ++i) cfma(acc, V[(int64_t)i * ldv + t], cs[i]);
    w[t] = c64d(w[t].re + sign * acc.re, w[t].im + sign * acc.im);
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

    void dots(const c64d *V, int nv, const c64d *w, std::vector<std::complex<double>> &out)
    {
        dim3 g(RCH, (nv + DVG - 1) / DVG);
        k_dots<<<g, RT, 0, h->stream>>>(V, n, nv, w, n, partial.as<c64d>());
        FDA_CHECK_LAUNCH();
        k_dots_finish<<<nv, RT, 0, h->stream>>>(partial.as<c64d>(), nv, hd.as<c64d>());
        FDA_CHECK_LAUNCH();
        out.resize(nv);
        FDA_CUDA(cudaMemcpyAsync(out.data(), hd.p, sizeof(c64d) * nv, cudaMemcpyDeviceToHost, h->stream));
        FDA_CUDA(cudaStreamSynchronize(h->stream));
    }
    double norm(const c64d *w)
    {
        std::vector<std::complex<double>> d;
        dots(w, 1, w, d);
        return sqrt(std::max(d[0].real(), 0.0));
    }
    void combine(const c64d *V, const std::vector<std::complex<double>> &c, double sign, c64d *w)
    {
        FDA_CUDA(cudaMemcpyAsync(hd.p, c.data(), sizeof(c64d) * c.size(), cudaMemcpyHostToDevice, h->stream));
        k_combine<<<fda_blocks(n, RT), RT, 0, h->stream>>>(V, n, (int)c.size(), hd.as<c64d>(), sign, w, n);
        FDA_CHECK_LAUNCH();
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
    void apply(const c64d *x, c64d *y, int precision)
    {
        auto t0 = std::chrono::steady_clock::now();
        // through the handle's staging vectors, so every product replays the
        // same captured graph
        FDA_CUDA(cudaMemcpyAsync(h->xs.p, x, sizeof(c64d) * n, cudaMemcpyDeviceToDevice, h->stream));
        fda_apply_staged(h, precision, 1);
        FDA_CUDA(cudaMemcpyAsync(y, h->ys.p, sizeof(c64d) * n, cudaMemcpyDeviceToDevice, h->stream));
        FDA_CUDA(cudaStreamSynchronize(h->stream));
        matvec_time += std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        ++nmatvec;
    }

    // GMRES(m) on A_prec: solve A d = r to ||r - A d|| <= tol_rel ||r||; d in/out
    // (d_zero: the caller knows d = 0, so the first residual is r itself)
    int gmres(const c64d *r, c64d *d, double tol_rel, int precision, int maxit, int &iters_out, double &est,
              bool d_zero = false)
    {
        const int m = std::max(1, h->cfg.restart);
        dbuf Vb, w;
        Vb.alloc(sizeof(c64d) * (size_t)(m + 1) * n);
        w.alloc(sizeof(c64d) * n);
        c64d *V = Vb.as<c64d>();
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
            std::vector<std::complex<double>> H((size_t)(m + 1) * m, 0.0), cs(m), sn(m), g(m + 1, 0.0);
            g[0] = beta;
            int j = 0;
            for (; j < m && it < maxit; ++j, ++it) {
                c64d *vj = V + (int64_t)j * n, *vn = V + (int64_t)(j + 1) * n;
                apply_op(vj, vn, precision);
                std::vector<std::complex<double>> hcol(j + 2, 0.0), c;
                for (int pass = 0; pass < 2; ++pass) {
                    dots(V, j + 1, vn, c);
                    for (int i = 0; i <= j; ++i) hcol[i] += c[i];
                    combine(V, c, -1.0, vn);
                }
                double hn = norm(vn);
                hcol[j + 1] = hn;
                for (auto &v : hcol)
                    if (!std::isfinite(v.real()) || !std::isfinite(v.imag()))
                        fda_fail(FDA_ERR_NUMERIC, "non-finite Hessenberg entry in GMRES");
                if (hn > 0) {
                    k_scale<<<fda_blocks(n, RT), RT, 0, h->stream>>>(vn, 1.0 / hn, n);
                    FDA_CHECK_LAUNCH();
                }
                for (int i = 0; i < j; ++i) {
                    std::complex<double> t = cs[i] * hcol[i] + sn[i] * hcol[i + 1];
                    hcol[i + 1] = -std::conj(sn[i]) * hcol[i] + std::conj(cs[i]) * hcol[i + 1];
                    hcol[i] = t;
                }
                double den = std::sqrt(std::norm(hcol[j]) + std::norm(hcol[j + 1]));
                if (den == 0.0) {
                    cs[j] = 1.0;
                    sn[j] = 0.0;
                } else {
                    cs[j] = std::conj(hcol[j]) / den;
                    sn[j] = std::conj(hcol[j + 1]) / den;
                }
                hcol[j] = cs[j] * hcol[j] + sn[j] * hcol[j + 1];
                hcol[j + 1] = 0.0;
                g[j + 1] = -std::conj(sn[j]) * g[j];
                g[j] = cs[j] * g[j];
                for (int i = 0; i <= j; ++i) H[(size_t)i * m + j] = hcol[i];
                est = std::abs(g[j + 1]) / rnorm0;
                ++iters_out;
                if (est <= tol_rel || hn <= 1e-14 * beta) {
                    ++j;
                    ++it;
                    break;
                }
            }
            // back substitution H y = g, d += V y
            std::vector<std::complex<double>> y(j, 0.0);
            for (int i = j - 1; i >= 0; --i) {
                std::complex<double> s = g[i];
                for (int k = i + 1; k < j; ++k) s -= H[(size_t)i * m + k] * y[k];
                y[i] = s / H[(size_t)i * m + i];
            }
            if (h->cfg.precond != 0) {
                // d += M (V y): form V y in w, then apply M into the basis slot V_m (free now)
                FDA_CUDA(cudaMemsetAsync(w.p, 0, sizeof(c64d) * n, h->stream));
                combine(V, y, 1.0, w.as<c64d>());
                c64d *tmp = V + (int64_t)m * n;
                fda_precond_apply(h, w.as<c64d>(), tmp);
                std::vector<std::complex<double>> one(1, 1.0);
                combine(tmp, one, 1.0, d);
            } else {
                combine(V, y, 1.0, d);
            }
            if (it >= maxit && est > tol_rel) {
                // one last true-residual check happens at the top of the loop
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
    S.partial.alloc(sizeof(c64d) * RCH * (size_t)(h->cfg.restart + 2));
    S.hd.alloc(sizeof(c64d) * (size_t)(h->cfg.restart + 2));
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
