// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <deque>
#include <vector>

#include "../../include/fda_bem.h"

// ---------------------------------------------------------------------------
// complex arithmetic on interleaved (re, im) pairs
// ---------------------------------------------------------------------------
template <typename T>
struct cx {
    T re, im;
    __host__ __device__ cx() : re(0), im(0) {}
    __host__ __device__ cx(T r, T i) : re(r), im(i) {}
};
template <typename T> __host__ __device__ inline cx<T> operator+(cx<T> a, cx<T> b) { return {a.re + b.re, a.im + b.im}; }
template <typename T> __host__ __device__ inline cx<T> operator-(cx<T> a, cx<T> b) { return {a.re - b.re, a.im - b.im}; }
template <typename T> __host__ __device__ inline cx<T> operator*(cx<T> a, cx<T> b)
{
    return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
template <typename T> __host__ __device__ inline cx<T> operator*(T s, cx<T> a) { return {s * a.re, s * a.im}; }
template <typename T> __host__ __device__ inline cx<T> conjg(cx<T> a) { return {a.re, -a.im}; }
// a += b * c
template <typename T> __host__ __device__ inline void cfma(cx<T> &a, cx<T> b, cx<T> c)
{
    a.re = fma(b.re, c.re, fma(-b.im, c.im, a.re));
    a.im = fma(b.re, c.im, fma(b.im, c.re, a.im));
}
// a += conj(b) * c
template <typename T> __host__ __device__ inline void cfma_conj(cx<T> &a, cx<T> b, cx<T> c)
{
    a.re = fma(b.re, c.re, fma(b.im, c.im, a.re));
    a.im = fma(b.re, c.im, fma(-b.im, c.re, a.im));
}

typedef cx<double> c64d;  // complex double
typedef cx<float> c32f;   // complex float

#define FDA_PI 3.14159265358979323846

// ---------------------------------------------------------------------------
// error plumbing
// ---------------------------------------------------------------------------
struct fda_error {
    fda_status st;
    std::string msg;
};

#define FDA_CUDA(call)                                                                        \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess)                                                                \
            throw fda_error{e_ == cudaErrorMemoryAllocation ? FDA_ERR_OOM : FDA_ERR_CUDA,     \
                            std::string(#call) + ": " + cudaGetErrorString(e_)};              \
    } while (0)

// FDA_DEBUG_SYNC=1 in the environment makes every launch check synchronous,
// so that a failing kernel is reported at its own launch site.
int fda_debug_sync();
// counts every kernel launch of the library (one check follows each launch;
// a graph replay adds the kernels it holds)
void fda_count_launch();
void fda_count_launches(long long n);
long long fda_launches_so_far();
#define FDA_CHECK_LAUNCH()                                                                    \
    do {                                                                                      \
        fda_count_launch();                                                                   \
        FDA_CUDA(cudaGetLastError());                                                         \
        if (fda_debug_sync()) {                                                               \
            cudaError_t e2_ = cudaDeviceSynchronize();                                        \
            if (e2_ != cudaSuccess)                                                           \
                throw fda_error{FDA_ERR_CUDA, std::string(__FILE__) + ":" +                   \
                                                  std::to_string(__LINE__) + ": " +           \
                                                  cudaGetErrorString(e2_)};                   \
        }                                                                                     \
    } while (0)

inline void fda_fail(fda_status st, const std::string &m) { throw fda_error{st, m}; }

// ---------------------------------------------------------------------------
// device buffer owned by the handle
// ---------------------------------------------------------------------------
struct dbuf {
    void *p = nullptr;
    size_t bytes = 0;
    dbuf() {}
    dbuf(const dbuf &) = delete;
    dbuf &operator=(const dbuf &) = delete;
    ~dbuf() { release(); }
    void release()
    {
        if (p) cudaFree(p);
        p = nullptr;
        bytes = 0;
    }
    void alloc(size_t b)
    {
        release();
        if (b == 0) b = 16;
        FDA_CUDA(cudaMalloc(&p, b));
        bytes = b;
    }
    template <typename T> T *as() const { return reinterpret_cast<T *>(p); }
};

// a small fixed-capacity array of buffers, one per octree level
constexpr int FDA_MAX_LEVELS = 24;

// ---------------------------------------------------------------------------
// per-level description
// ---------------------------------------------------------------------------
struct level_info {
    int nbox = 0;        // boxes at this level
    int box0 = 0;        // offset of the level in the concatenated box arrays
    int nleaf = 0;
    double w = 0;        // box width
    int hf = 0;          // high-frequency regime
    int nc = 0;          // cells per cube-face edge (high frequency); cones = 6 nc^2
    int ncones = 1;      // 1 for low frequency
    double rho = 0;      // high-frequency far-field distance in widths
    int T = 0;           // retained rank (0: level has no far-field operators)
    int n_eq = 0, n_chk = 0;  // upward equivalent / check point counts
    int active = 0;      // densities are needed at this level
    int n_il = 0;        // interaction-list entries at this level
    int n_ops = 0;       // distinct M2L operators at this level
    int R_off = 0;       // offsets of the dense offset table lie in [-R_off, R_off]^3
};

// one batched-translation launch: tiles of (operator, pair range, row block)
// and (source offset, target offset) pairs, grouped by operator
// tiles of a batch cut for one (right-hand sides, columns per tile); kept
// until the handle is destroyed, because captured graphs point into them
struct tile_set {
    int mr = 0, nc = 0, rows = 1, n = 0;  // right-hand sides, columns and row tiles per tile, tiles
    dbuf buf;
};

struct tr_batch {
    dbuf pairs;
    int tm = 64;          // output rows per tile (32 or 64)
    int tout = 0;         // output rank
    int64_t npairs = 0;
    std::vector<int> op_start;  // pairs of operator o: [op_start[o], op_start[o+1])
    std::deque<tile_set> tilesets;  // columns per tile: 64 if an operator averages >= 48, else 32
    // tensor-core form of the batch: tile lists per (right-hand sides, columns,
    // row tiles) and the autotuner's shape for one right-hand side (0 = rule)
    std::deque<tile_set> tc_tilesets;
    int nc_tuned = 0, r_tuned = 1, st_tuned = 0;  // tuned tile shape at one right-hand side
    int nc_tm = 0, r_tm = 1, st_tm = 0;           // and at max_rhs right-hand sides
};

// tensor-core form of a set of translation operators: bf16 hi/lo panels
// (64 complex output rows x 32 complex input columns per panel); the tiles
// and tuned shapes belong to the batch that applies them
struct tc_ops {
    dbuf A;
    int Tout = 0, Tin = 0;
    int nrt = 0, nkc = 0;     // row tiles (64 complex rows), K stages (32 complex columns)
    int64_t op_bytes = 0;
};

// Low-rank reduced M2L operators of one level and rank bucket (Sec. 4.2):
// K~_o ~= U^_o V^_o with U^ (T x r) and V^ (r x T), zero-padded to the
// bucket's rank rpad, applied in two stages: t_p = V^_o q~_C into one
// intermediate vector per pair, then p~_D += U^_o t_p.
struct lr_bucket {
    int rpad = 0;
    std::vector<int> ops;       // operator indices of the level in this bucket
    dbuf U64, V64, U32, V32;    // [n][T x rpad] and [n][rpad x T], column-major
    tr_batch b1, b2;            // stage 1 (q~ -> t) and stage 2 (t -> p~) pairs, grouped by bucket operator
    tc_ops tc1, tc2;            // tensor-core panels of V^ and U^
    dbuf t64, t32, ts;          // intermediates [mr][pairs][rpad] (FP64, FP32) and the FP32 split into bf16
    int64_t npairs = 0;
};

template <typename T>
struct far_ops {
    // per level (index = level)
    dbuf Kt[FDA_MAX_LEVELS];     // [n_ops][T][T] column-major (K[j*T + i] = K~_ij)
    dbuf Mt[FDA_MAX_LEVELS];     // parent level: [8 * ncones][T_child][T] column-major
    dbuf Lt[FDA_MAX_LEVELS];     // parent level: [8 * ncones][T][T_child] column-major (rows = child rank)
    dbuf St;                     // per leaf: [n_B][T] (S~ transposed)
    dbuf St1;                    // the same for single-layer sources (right-hand side's layers; built on demand)
    dbuf Tt;                     // per leaf: [T][n_B] (T~ column-major)
    dbuf near;                   // near-field blocks, row-major per leaf
    dbuf near1;                  // right-hand side's layers on the same pattern (built on demand)
};

struct fda_handle {
    fda_config cfg;
    cudaStream_t stream = nullptr;
    std::string err;
    int state = 0;  // 0 created, 1 tree built, 2 precomputed

    // problem
    double k = 0, lambda = 0;
    int64_t N = 0, NV = 0;
    double root_lo[3] = {0, 0, 0};
    double W = 0, diam = 0;

    // geometry in Morton order (device)
    dbuf perm;      // int32 [N]: sorted position -> caller index
    dbuf iperm;     // int32 [N]: caller index -> sorted position
    dbuf verts9;    // double [N][9] triangle vertices
    dbuf cent;      // double [N][3]
    dbuf nrm;       // double [N][3] normal into the body
    dbuf area;      // double [N]
    dbuf h2;        // double [N] squared longest edge
    dbuf qpt;       // double [N][6][3] regular-rule quadrature points
    dbuf qw;        // double [N][6] weights (area included)
    dbuf keys;      // uint64 [N] sorted Morton keys

    // tree (device, concatenated over levels)
    int nlev = 0;
    level_info lev[FDA_MAX_LEVELS];
    int nbox_total = 0;
    dbuf box_begin, box_end;   // int32 element ranges
    dbuf box_key;              // uint64 Morton prefix at the box's level
    dbuf box_coord;            // int32 [nbox][3]
    dbuf box_parent;           // int32 global index (-1 root)
    dbuf box_child0, box_child1;  // int32 global child range [c0, c1)
    dbuf box_leaf;             // int32 flag
    dbuf box_level;            // int32
    int nleaf = 0;
    int max_leaf_rows = 0;     // largest leaf (elements)
    int64_t max_near_cols = 0; // widest near-field row of a leaf (columns)
    dbuf leaf_box;             // int32 [nleaf] global box index
    std::vector<int> h_leaf_level;  // leaf index -> level (host)
    dbuf leaf_of_box;          // int32 [nbox]: leaf index or -1

    // interaction lists (CSR over global boxes): source box (global) and operator index
    dbuf il_ptr, il_src, il_op, il_cone;  // il_cone: target cone (high frequency) or 0
    int64_t n_il_total = 0;
    // near-field lists (CSR over leaves): source element ranges
    dbuf nr_ptr, nr_begin, nr_end;
    dbuf nf_colptr;            // int64 [nleaf+1]: column offsets per leaf
    dbuf nf_cols;              // int32 [total cols]: source element of each column (the leaf's near
                               // ranges one after another, in list order, each in element order)
    dbuf nf_off;               // int64 [nleaf+1]: entry offsets per leaf block
    int64_t nnz_near = 0, ncols_total = 0;

    // canonical point sets per level (device, box-relative, scaled)
    dbuf eq_up[FDA_MAX_LEVELS], chk_up[FDA_MAX_LEVELS];
    dbuf rot[FDA_MAX_LEVELS];  // double [ncones][9] cone rotations (high frequency)
    // truncated SVD of G_up per level (FP64)
    dbuf Uup[FDA_MAX_LEVELS];  // [n_chk][T] column-major? stored as [T][n_chk] (column j contiguous)
    dbuf Vup[FDA_MAX_LEVELS];  // [T][n_eq]
    dbuf sig[FDA_MAX_LEVELS];  // [T]
    std::vector<int> leaf_T_off;   // per leaf: offset into St / Tt (elements)
    dbuf leaf_op_off;          // int64 [nleaf]
    // FP32 L2T operators without the 64-row padding (leaf li: [T][n_B] at
    // tt_c_off[li]), read by the one-right-hand-side L2T kernel
    dbuf tt32c, tt_c_off;

    far_ops<double> op64;
    far_ops<float> op32;
    int have32 = 0;
    int rhs_layers = 0;  // near field and S2M of the right-hand side's layers built
    int autotune_cached = 0, autotune_timed = 0;  // tensor-core batches from the cache / timed at setup
    std::string autotune_cache;                   // cfg.autotune_cache copied at fda_create ("" = none)

    // low-rank M2L (Sec. 4.2): per level the retained rank of every operator
    // (T: applied in full) and the rank buckets of the low-rank ones
    std::vector<int> op_rank[FDA_MAX_LEVELS];
    std::vector<int> op_bucket[FDA_MAX_LEVELS];  // bucket of each operator, -1 = full
    std::deque<lr_bucket> lr[FDA_MAX_LEVELS];
    // levels with low-rank buckets also keep every pair in one full-form
    // batch; the tensor-core path uses the low-rank form at level l only if
    // lr_tc[l] (set by the setup autotuner when it is faster)
    tr_batch b_m2l_all[FDA_MAX_LEVELS];
    int lr_tc[FDA_MAX_LEVELS] = {};       // one right-hand side
    int lr_tc_many[FDA_MAX_LEVELS] = {};  // several (decided at max_rhs)

    // tensor-core M2L (chosen precision)
    tc_ops tc_m2l[FDA_MAX_LEVELS], tc_m2m[FDA_MAX_LEVELS], tc_l2l[FDA_MAX_LEVELS];
    dbuf qs[FDA_MAX_LEVELS], ps[FDA_MAX_LEVELS];  // FP32 densities split into bf16 hi/lo
    dbuf tc_err;
    int have_tc = 0;
    int tc_force[3] = {0, 0, 0};  // tile shape forced by fda_set_tc_tiles (columns, row tiles, stages; 0 = auto)
    // tile lists of the tensor-core leaf products (near field, S2M, L2T) per
    // (kind, right-hand sides, columns per tile); kept because captured
    // graphs point into them
    struct leaf_tile_set {
        int kind = 0, mr = 0, nc = 0, n = 0;
        dbuf buf;
    };
    std::deque<leaf_tile_set> leaf_sets;

    // batched translations per level (M2L at l; M2M and L2L between l and l+1)
    tr_batch b_m2l[FDA_MAX_LEVELS], b_m2m[FDA_MAX_LEVELS], b_l2l[FDA_MAX_LEVELS];

    // densities (per level, [nbox][ncones][T])
    dbuf q64[FDA_MAX_LEVELS], p64[FDA_MAX_LEVELS];
    dbuf q32[FDA_MAX_LEVELS], p32[FDA_MAX_LEVELS];
    int lev_lo = -1;           // coarsest level with interaction-list entries
    std::vector<int3> h_ops[FDA_MAX_LEVELS];  // per level: offset of each distinct M2L operator

    // leaf block-diagonal preconditioner (row-major n_B x n_B per leaf)
    dbuf pc_M, pc_off;
    // learned SAI preconditioner: on the leaf-block pattern (sai_M, FP64,
    // row-major n_B x n_B per leaf) or on the near-field pattern (sai_M32,
    // FP32, the near-field matrix's layout); sai_pattern says which is set
    dbuf sai_M, sai_off, sai_M32;
    int sai_pattern = 0;

    // captured applies (one CUDA graph per precision, right-hand sides and
    // tensor-core switch), replayed on gstream joined to stream by events
    struct apply_graph {
        int key;
        cudaGraphExec_t exec;
        long long kernels;  // kernel launches captured in it
    };
    std::vector<apply_graph> graphs;
    cudaStream_t gstream = nullptr;
    cudaEvent_t gev[2] = {};
    int graphs_broken = 0;
    int64_t graph_replays = 0;

    // timing
    int timing = 0;
    cudaEvent_t ev[8] = {};
    float pass_ms[6] = {0, 0, 0, 0, 0, 0};
    double tree_s = 0, precompute_s = 0, near_s = 0;

    // workspace
    dbuf work64;               // general FP64 workspace (x staging etc.)
    dbuf xs, ys;               // sorted-order staging vectors (complex double)
    dbuf xs32;                 // sorted-order complex float staging
    dbuf io_x, io_y;           // device copies of host vectors (fda_apply_host)
    dbuf solve_ws;             // GMRES basis
    dbuf red;                  // reduction scratch
};

// ---------------------------------------------------------------------------
// entry points between translation units
// ---------------------------------------------------------------------------
void fda_geometry_build(fda_handle *h, const double *verts, int64_t nv, const int32_t *tris, int64_t nt);
void fda_tree_build(fda_handle *h);
void fda_near_build(fda_handle *h, int side = 0);
void fda_near_convert_f32(fda_handle *h, int side = 0);
// S~ of the right-hand side's layers (single-layer sources) for every leaf
void fda_far_rhs_s2m(fda_handle *h);
void fda_far_rhs_convert_f32(fda_handle *h);
void fda_far_precompute(fda_handle *h);
// side 0: the Burton-Miller operator (unknown u); side 1: the right-hand
// side's layers acting on q = du/dn (needs fda_rhs_layers_prepare)
void fda_apply_sorted(fda_handle *h, const c64d *xs, c64d *ys, int precision, int mr = 1, int side = 0);
void fda_rhs_layers_prepare(fda_handle *h);
// h->ys = A h->xs (sorted order, mr right-hand sides) through the graph cache
void fda_apply_staged(fda_handle *h, int precision, int mr);
void fda_graphs_release(fda_handle *h);
void fda_rhs_sorted(fda_handle *h, const double *dirs_dev, int nrhs, c64d *b_sorted);
void fda_rhs_noalloc(fda_handle *h, const double *dirs_host, int nrhs, c64d *b);
// point sources (device [nrhs][3]) -> b in the caller's element order, ld = N
void fda_rhs_point(fda_handle *h, const double *src_dev, int nrhs, c64d *b);
// far = 1: far-field pattern at unit directions; far = 0: scattered field at points
void fda_field(fda_handle *h, const c64d *u, const c64d *q, const double *tgt_dev, int64_t ntgt, int far, c64d *out);
// far-field pattern through the fast algorithm's upward pass (device directions [ndir][3])
void fda_far_field_upward(fda_handle *h, const c64d *u, const c64d *q, const double *dirs_dev, int ndir, c64d *out);
// scattered field at points through the fast algorithm (local densities by
// the downward pass, L2T at each point's box, equivalent sources and direct
// sums for what those do not cover); device points [ntgt][3]
void fda_field_fast(fda_handle *h, const c64d *u, const c64d *q, const double *tgt_dev, int64_t ntgt, c64d *out);
// FP64 upward pass: S2M of side 0 (double layer) or 1 (single layer) of xs
// (Morton order) into q64 (add = 1: added to q64), then M2M on q64
void fda_upward_fp64(fda_handle *h, const c64d *xs, int side, int add);
void fda_m2m_fp64(fda_handle *h);
// FP64 downward pass on q64: M2L at every level and L2L, local densities in p64
void fda_downward_fp64(fda_handle *h);
// the same outgoing and local densities of -D[u] + S[q] in the chosen precision
// (FP32 S2M, tensor-core translations), copied into q64 and p64; xs = -u, qs = q
void fda_translate_chosen(fda_handle *h, const c64d *xs, const c64d *qs);
void fda_gather_to_sorted(fda_handle *h, const c64d *x, c64d *xs);
void fda_scatter_from_sorted(fda_handle *h, const c64d *ys, c64d *y);
void fda_gather_cols(fda_handle *h, const c64d *x, int64_t ld, c64d *xs, int nrhs, cudaStream_t s);
void fda_scatter_cols(fda_handle *h, const c64d *ys, c64d *y, int64_t ld, int nrhs, cudaStream_t s);
fda_status fda_solve_impl(fda_handle *h, const c64d *b, c64d *x, double tol, fda_info *info);
void fda_precond_build(fda_handle *h);
void fda_precond_apply(fda_handle *h, const c64d *r, c64d *z);

void fda_build_batches(fda_handle *h);
int fda_sai_nparams();
void fda_sai_init(uint64_t seed, float *W);
void fda_sai_train_impl(fda_handle *const *hs, int nh, int epochs, double lr, float *W, double *loss0,
                        double *loss1, double *train_s);
double fda_sai_set_impl(fda_handle *h, const float *W);
void fda_sai_loss_grad_impl(int64_t n, const double *cent, const double *nrm, const double *area, double k, int nb,
                            const int64_t *bptr, const int32_t *belem, const c64d *A, const double *W, int fp32,
                            double *loss, double *grad);
void fda_sai_train_near_impl(fda_handle *const *hs, int nh, int epochs, double lr, int per_step, uint64_t seed,
                             float *W, double *loss0, double *loss1, double *train_s);
double fda_sai_set_near_impl(fda_handle *h, const float *W, bool want_loss);
void fda_sai_loss_grad_near_impl(fda_handle *h, const double *W, int nleaves, const int32_t *leaves, int fp32,
                                 double *loss, double *grad);
// z = A x over the near-field pattern for an FP32 matrix A in the near-field
// matrix's layout (one right-hand side, FP64 vectors)
void fda_near_product_f32(fda_handle *h, const c32f *A, const c64d *x, c64d *z);
void fda_pack_tc(fda_handle *h);
// split nvec FP32 vectors of length T into bf16 hi/lo (the gather layout of the tensor-core kernel)
void fda_split_vectors(fda_handle *h, const c32f *src, int64_t nvec, int T, dbuf &out);
// split level l's FP32 densities (mr right-hand sides) into bf16 hi/lo
void fda_split_tc(fda_handle *h, int l, const c32f *src, dbuf &out, int mr);
// dst += op * src for every pair of batch B on the tensor cores; src is the
// split densities of the source level (svstride vectors per right-hand
// side), dst the FP32 densities of the target level (dstride elements each)
void fda_run_tc(fda_handle *h, tr_batch &B, tc_ops &P, const dbuf &src, int64_t svstride, c32f *dst, int mr,
                int64_t dstride, int nc = 0, int rows = 0, int st = 0);
// leaf products on the tensor cores for mr right-hand sides (kind 0 near
// field y = A x, 1 S2M into q32, 2 L2T y += T~ p32); A: FP32 operator of the side
void fda_leaf_tc(fda_handle *h, int kind, const dbuf &A, const c32f *x, c64d *y, int mr);
// time the tile shapes of every tensor-core batch once and keep the fastest
void fda_autotune_tc(fda_handle *h);
int fda_tc_error(fda_handle *h);
template <typename R>
void fda_run_batch(tr_batch &B, const cx<R> *ops, int Tout, int Tin, const cx<R> *src, cx<R> *dst, int mr,
                   int64_t sstride, int64_t dstride, cudaStream_t s);

// scans and sorts (sort.cu)
void fda_exclusive_scan_i32(const int32_t *in, int32_t *out, int64_t n, cudaStream_t s, int32_t *total_host);
void fda_exclusive_scan_i64(const int64_t *in, int64_t *out, int64_t n, cudaStream_t s, int64_t *total_host);
void fda_radix_sort_u64(uint64_t *keys, int32_t *vals, int64_t n, int key_bits, cudaStream_t s);

// kernel launch helper
inline unsigned fda_blocks(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }
