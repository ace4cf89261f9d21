// Leaf block-diagonal preconditioner.  The paper solves without a
// preconditioner (Sec. 5.3); this is the plain preconditioner of the scope's
// solver row: M = blockdiag(A_BB^-1) over the leaves B, where A_BB is the
// leaf's own block of the near-field matrix (self and neighbour element
// integrals of Eq. eq_sum among the leaf's elements).  GMRES uses it on the
// right (A M u = b, x = M u), so the residual it reports is still that of
// the unpreconditioned system.
#include <vector>

#include "fda_internal.cuh"

namespace {

constexpr int PT = 256;

// In-place Gauss-Jordan inversion with partial pivoting of each leaf's
// self block (FP64, n_B <= 64, in shared memory).  Writes M_B row-major.
__global__ void k_blockdiag_inv(const int32_t *leaf_box, const int32_t *bbeg, const int32_t *bend,
                                const int64_t *colptr, const int64_t *rptr, const int32_t *rb, const int32_t *re,
                                const int64_t *off, const c64d *A, const int64_t *moff, c64d *M, int *status)
{
    extern __shared__ unsigned char smem_raw[];
    c64d *S = reinterpret_cast<c64d *>(smem_raw);  // [64][64]
    __shared__ int piv[64];
    __shared__ c64d fcol[64];
    __shared__ int prow;
    __shared__ double pmax;
    int li = blockIdx.x;
    int B = leaf_box[li];
    int b0 = bbeg[B], n = bend[B] - b0;
    int64_t nc = colptr[li + 1] - colptr[li];
    // column offset of the leaf's own range among its near ranges
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
    const c64d *blk = A + off[li];
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
        int i = e / n, j = e % n;
        S[i * 64 + j] = blk[(int64_t)i * nc + cself + j];
    }
    __syncthreads();
    for (int k = 0; k < n; ++k) {
        if (threadIdx.x == 0) {
            int p = k;
            double best = -1.0;
            for (int i = k; i < n; ++i) {
                double m = S[i * 64 + k].re * S[i * 64 + k].re + S[i * 64 + k].im * S[i * 64 + k].im;
                if (m > best) {
                    best = m;
                    p = i;
                }
            }
            prow = p;
            pmax = best;
            piv[k] = p;
        }
        __syncthreads();
        if (!(pmax > 0.0)) {
            if (threadIdx.x == 0) atomicExch(status, 2);
            return;
        }
        int p = prow;
        if (p != k)
            for (int j = threadIdx.x; j < n; j += blockDim.x) {
                c64d t = S[k * 64 + j];
                S[k * 64 + j] = S[p * 64 + j];
                S[p * 64 + j] = t;
            }
        __syncthreads();
        c64d pv = S[k * 64 + k];
        double den = pv.re * pv.re + pv.im * pv.im;
        c64d inv(pv.re / den, -pv.im / den);
        __syncthreads();
        for (int j = threadIdx.x; j < n; j += blockDim.x) {
            c64d v = (j == k) ? c64d(1.0, 0.0) : S[k * 64 + j];
            S[k * 64 + j] = v * inv;
        }
        __syncthreads();
        for (int i = threadIdx.x; i < n; i += blockDim.x) fcol[i] = S[i * 64 + k];
        __syncthreads();
        for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
            int i = e / n, j = e % n;
            if (i == k) continue;
            c64d f = fcol[i];
            c64d rk = S[k * 64 + j];
            c64d cur = (j == k) ? c64d(0.0, 0.0) : S[i * 64 + j];
            S[i * 64 + j] = cur - f * rk;
        }
        __syncthreads();
    }
    // undo the row interchanges as column interchanges, last first
    for (int k = n - 1; k >= 0; --k) {
        int p = piv[k];
        if (p != k)
            for (int i = threadIdx.x; i < n; i += blockDim.x) {
                c64d t = S[i * 64 + k];
                S[i * 64 + k] = S[i * 64 + p];
                S[i * 64 + p] = t;
            }
        __syncthreads();
    }
    c64d *Mb = M + moff[li];
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) Mb[e] = S[(e / n) * 64 + (e % n)];
}

// z_B = M_B r_B for every leaf (one warp per row)
__global__ void k_blockdiag_apply(const int32_t *leaf_box, const int32_t *bbeg, const int32_t *bend,
                                  const int64_t *moff, const c64d *M, const c64d *r, c64d *z)
{
    int li = blockIdx.x;
    int B = leaf_box[li];
    int b0 = bbeg[B], n = bend[B] - b0;
    int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const c64d *Mb = M + moff[li];
    for (int i = warp; i < n; i += blockDim.x / 32) {
        c64d acc;
        for (int j = lane; j < n; j += 32) cfma(acc, Mb[i * n + j], r[b0 + j]);
        for (int o = 16; o > 0; o >>= 1) {
            acc.re += __shfl_xor_sync(0xffffffffu, acc.re, o);
            acc.im += __shfl_xor_sync(0xffffffffu, acc.im, o);
        }
        if (lane == 0) z[b0 + i] = acc;
    }
}

}  // namespace

void fda_precond_build(fda_handle *h)
{
    if (h->cfg.precond != 1) return;
    cudaStream_t s = h->stream;
    const int NL = h->nleaf;
    std::vector<int32_t> lb(NL), bb(h->nbox_total), be(h->nbox_total);
    FDA_CUDA(cudaMemcpy(lb.data(), h->leaf_box.p, 4 * (size_t)NL, cudaMemcpyDeviceToHost));
    FDA_CUDA(cudaMemcpy(bb.data(), h->box_begin.p, 4 * bb.size(), cudaMemcpyDeviceToHost));
    FDA_CUDA(cudaMemcpy(be.data(), h->box_end.p, 4 * be.size(), cudaMemcpyDeviceToHost));
    std::vector<int64_t> moff(NL + 1, 0);
    for (int li = 0; li < NL; ++li) {
        int64_t n = be[lb[li]] - bb[lb[li]];
        if (n > 64) fda_fail(FDA_ERR_ARG, "block-diagonal preconditioner needs leaves of at most 64 elements");
        moff[li + 1] = moff[li] + n * n;
    }
    h->pc_off.alloc(sizeof(int64_t) * (NL + 1));
    FDA_CUDA(cudaMemcpy(h->pc_off.p, moff.data(), sizeof(int64_t) * (NL + 1), cudaMemcpyHostToDevice));
    h->pc_M.alloc(sizeof(c64d) * std::max<int64_t>(moff[NL], 1));
    dbuf status;
    status.alloc(sizeof(int));
    FDA_CUDA(cudaMemsetAsync(status.p, 0, sizeof(int), s));
    size_t smem = sizeof(c64d) * 64 * 64;
    FDA_CUDA(cudaFuncSetAttribute(k_blockdiag_inv, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_blockdiag_inv<<<NL, PT, smem, s>>>(h->leaf_box.as<int32_t>(), h->box_begin.as<int32_t>(),
                                         h->box_end.as<int32_t>(), h->nf_colptr.as<int64_t>(),
                                         h->nr_ptr.as<int64_t>(), h->nr_begin.as<int32_t>(),
                                         h->nr_end.as<int32_t>(), h->nf_off.as<int64_t>(), h->op64.near.as<c64d>(),
                                         h->pc_off.as<int64_t>(), h->pc_M.as<c64d>(), status.as<int>());
    FDA_CHECK_LAUNCH();
    int hs = 0;
    FDA_CUDA(cudaMemcpyAsync(&hs, status.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    FDA_CUDA(cudaStreamSynchronize(s));
    if (hs == 1) fda_fail(FDA_ERR_NUMERIC, "leaf self block not found in the near field");
    if (hs == 2) fda_fail(FDA_ERR_NUMERIC, "singular leaf self block in the preconditioner");
}

// z = M r (both sorted order, complex double); M = the block-diagonal
// inverse (precond 1) or the learned SAI blocks (precond 2), same pattern
void fda_precond_apply(fda_handle *h, const c64d *r, c64d *z)
{
    const bool learned = h->cfg.precond == 2;
    if (learned && h->sai_pattern == 1) {
        // learned M on the near-field pattern: the near-field product with M
        fda_near_product_f32(h, h->sai_M32.as<c32f>(), r, z);
        return;
    }
    k_blockdiag_apply<<<h->nleaf, PT, 0, h->stream>>>(h->leaf_box.as<int32_t>(), h->box_begin.as<int32_t>(),
                                                      h->box_end.as<int32_t>(),
                                                      (learned ? h->sai_off : h->pc_off).as<int64_t>(),
                                                      (learned ? h->sai_M : h->pc_M).as<c64d>(), r, z);
    FDA_CHECK_LAUNCH();
}
