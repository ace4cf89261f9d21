/*
 * fda_bem.h - C ABI of the GB300 fast directional Burton-Miller BEM library.
 *
 * The library solves the exterior Helmholtz problem for a sound-hard body
 * with the Burton-Miller boundary integral equation (Sec. 2, Eq. eq_bm),
 * discretised by collocation at triangle centroids with piecewise-constant
 * elements (Sec. 5), alpha = i/k.  Its matrix-vector product is the left-hand
 * side sum of Eq. eq_sum, evaluated by the fast directional algorithm of
 * Sec. 3 (algorithm summary, Steps 1-4) with the compressed translations of
 * Sec. 4, inside a GMRES solve (Sec. 5).
 *
 * Conventions shared by every entry point:
 *   - Mesh: vertices double[nv][3], triangles int32[nt][3] (0-based), oriented
 *     so that (v1 - v0) x (v2 - v0) points out of the body into the acoustic
 *     domain.  The library's normal n is the opposite unit vector (into the
 *     body): the orientation under which Eq. cbie is Green's representation
 *     with G = e^{ikr}/(4 pi r).
 *   - Vectors: complex double, interleaved (re, im), one value per triangle in
 *     the caller's triangle order; several right-hand sides are stored
 *     column-major with leading dimension ld >= nt.
 *   - Pointers marked "device" are CUDA device pointers owned by the caller;
 *     "host" pointers are ordinary host memory.  The library copies what it
 *     keeps and owns all of its internal device memory.
 *   - Calls are stream-ordered on the stream given in fda_config.cuda_stream
 *     (NULL = legacy default stream).  Entry points that return results to
 *     the host (fda_solve's info, fda_get_stats) synchronise that stream.
 *   - Call order: fda_create -> fda_build_tree -> fda_precompute_translations
 *     -> fda_apply / fda_rhs_plane_wave / fda_solve (any number of times)
 *     -> fda_destroy.  Out-of-order calls return FDA_ERR_STATE.
 *   - No C++ exception crosses this interface.  Every failing call returns a
 *     status and leaves a message for fda_last_error.
 */
#ifndef FDA_BEM_H
#define FDA_BEM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct { double re, im; } fda_c128;

typedef enum {
    FDA_OK = 0,
    FDA_ERR_ARG = 1,            /* invalid argument (sizes, degenerate triangle, k <= 0, ...) */
    FDA_ERR_STATE = 2,          /* call out of order */
    FDA_ERR_CUDA = 3,           /* a CUDA runtime call failed */
    FDA_ERR_OOM = 4,            /* device allocation failed */
    FDA_ERR_NOT_CONVERGED = 5,  /* GMRES reached maxit above the tolerance */
    FDA_ERR_TIMEOUT = 6,        /* a bounded device-side wait gave up */
    FDA_ERR_NUMERIC = 7         /* NaN/Inf met, or GMRES breakdown */
} fda_status;

typedef enum { FDA_PLAIN_FP64 = 0, FDA_CHOSEN_FP32 = 1 } fda_precision;
typedef enum { FDA_MODE_FDA = 0, FDA_MODE_DENSE = 1 } fda_mode;

typedef struct {
    double eps;            /* SVD truncation threshold of Eq. epsg / epsk (default 1e-4), in [1e-7, 0.1]: the
                              SVDs are eigendecompositions of Gram matrices G^H G in FP64, which resolve
                              singular values down to about 1e-8 of the largest, so smaller eps is rejected */
    int p_lf;              /* low-frequency cube surfaces: points per edge (default 8) */
    int p_hf;              /* high-frequency equivalent sphere: points per cube edge before projection (10) */
    int hf_nr;             /* high-frequency cone sampling: radial shells (5) */
    int hf_na;             /* high-frequency cone sampling: directions per shell (300) */
    int leaf_max;          /* octree leaf capacity in elements, <= 64 (default 64) */
    double hf_wavelengths; /* a cube is high-frequency iff its width >= hf_wavelengths * lambda (1.0) */
    double rho_min;        /* high-frequency far field starts at max(rho_min, w/lambda) widths (2.2) */
    int precision;         /* fda_precision: plain FP64 or chosen FP32 far field and near storage */
    int mode;              /* fda_mode: FDA, or dense all-pairs direct sum (small meshes, testing) */
    int restart;           /* GMRES restart length, 1 to 255 (default 100) */
    int maxit;             /* GMRES iteration cap (default 1000) */
    int precond;           /* 0 none (the paper's setting), 1 leaf block-diagonal (right preconditioner);
                              the learned preconditioner (2) is selected with fda_set_precond after fda_sai_set */
    double alpha_sign;     /* coupling alpha = alpha_sign * i/k with G = e^{ikr}/(4 pi r) and the normal into
                              the body.  -1 (default): the paper's operator.  Its closed form of Sec. 5.1,
                              u = 1/(1 + ik), and its iteration counts (Table tab_usphpls, Sec. 5.3) hold for
                              the complex conjugate of the printed equations (G = e^{-ikr}, alpha = i/k), and
                              conjugating that gives alpha = -i/k here.  +1: alpha = +i/k as printed, which
                              puts sphere eigenvalues around 0 and slows GMRES down */
    int max_rhs;           /* right-hand sides one fda_apply pass processes together (1..256, default 1);
                              densities and staging vectors are sized for it */
    int tensor_cores;      /* chosen precision: run M2L on the tensor cores (split-bf16 tcgen05 GEMMs, FP32
                              accumulation); 1 (default) or 0 (FP32 SIMT) */
    void *cuda_stream;     /* cudaStream_t, or NULL */
    int graphs;            /* 1 (default): from the second apply with the same precision, right-hand-side
                              count and tensor-core switch on, each operator application (fda_apply and
                              every GMRES product) replays one captured CUDA graph on a library stream
                              joined to cuda_stream; 0: launch the kernels one by one (timing mode also
                              does) */
    int autotune;          /* 1 (default): at setup, time each tensor-core translation batch with 32-, 64-
                              and 128-column tiles, one to three 64-row tiles per CTA tile and 2 to 4 ring
                              stages, and keep the fastest (one right-hand side); 0: fixed rule (32, 64 or
                              128 columns as operators have few or many pairs; one row tile) */
    const char *autotune_cache; /* NULL (default) or a file path: the autotuner first looks each batch up
                              there (key: GPU name and SM count, pass, level, ranks, operator and pair
                              counts) and times only the batches it does not find, appending their choice
                              as one text line "key columns row_tiles stages" each.  A missing file is
                              created; an unreadable or unwritable one only disables the cache.  The
                              string is read during fda_precompute_translations only. */
    int lowrank;           /* 1 (default): Sec. 4.2, each reduced M2L operator K~ (T x T) is factorised as
                              U^ V^ (T x r, r x T) truncated at eps times its largest singular value (Eq. epsk,
                              error measured in the Frobenius norm) and applied as two products where that is
                              cheaper; 0: every K~ applied in full */
} fda_config;

typedef struct {
    int iters;              /* GMRES iterations (inner iterations, summed over refinement passes) */
    int refinements;        /* outer FP64 residual evaluations (chosen precision) */
    double rel_resid_fp64;  /* ||b - A x|| / ||b|| with the plain FP64 FDA operator */
    double setup_s;         /* wall time of build_tree + precompute_translations */
    double solve_s;         /* wall time of this solve */
    double matvec_s;        /* mean device time of one operator application inside the solve (CUDA events) */
} fda_info;

typedef struct {
    int64_t n_elements, n_boxes, n_leaves, n_levels;
    int64_t nnz_near;             /* near-field matrix entries (Step 4) */
    int64_t n_m2l;                /* M2L (box, source) pairs over all levels */
    int64_t n_m2l_ops;            /* distinct compressed M2L operators */
    int64_t bytes_near;           /* bytes of the near-field matrix read per apply */
    int64_t bytes_far;            /* bytes of far-field operators and densities read/written per apply */
    int64_t flops_far;            /* real flops of the far-field passes per apply */
    int64_t device_bytes;         /* device memory held by the handle */
    int32_t level_regime[32];     /* per level: 0 = low frequency, 1 = high frequency, -1 = unused */
    int32_t level_rank[32];       /* per level: retained SVD rank T */
    int32_t level_boxes[32];
    int32_t level_cones[32];
    double precompute_s, tree_s, near_s;
    int64_t level_m2l_pairs[32];  /* per level: M2L (target, source) pairs */
    int32_t level_m2l_ops[32];    /* per level: distinct M2L operators (after the cone symmetry) */
    int64_t graph_replays;        /* operator applications replayed from captured CUDA graphs so far */
    int32_t graph_fallback;       /* 1 if a capture failed and the handle launches kernels one by one */
    int32_t autotune_cached;      /* tensor-core batches whose tile shape came from the autotune cache */
    int32_t autotune_timed;       /* tensor-core batches timed by the autotuner at setup */
    int32_t level_lr_ops[32];     /* per level: M2L operators applied in low-rank form (Sec. 4.2) */
    int32_t level_lr_rank_max[32];   /* per level: largest retained rank r of those operators */
    float level_lr_rank_mean[32];    /* per level: mean retained rank r of every operator factorised */
    int64_t level_lr_pairs[32];   /* per level: M2L pairs applied in low-rank form */
    double level_m2l_flops[32];   /* per level: real flops of the M2L pass for one right-hand side in the
                                     form the handle's current precision applies (8 T^2 per pair in full
                                     form, 8 (2 r T) per pair in low-rank form with the operator's own rank r) */
    double level_m2l_bytes[32];   /* per level, same form: algorithmic bytes for one right-hand side at 8
                                     bytes per complex value: every operator applied read once (T^2, or
                                     2 r T in low-rank form), source densities read once, target densities
                                     read and written once, each low-rank pair's intermediate written and
                                     read once */
    int32_t level_lr_tc[32];      /* per level: bit 0 set if the tensor-core path applies the low-rank form
                                     there to one right-hand side, bit 1 if to several (the setup autotuner
                                     found it faster than the full form, at one and at max_rhs columns) */
    int32_t level_tc_shape[32][3]; /* per level: tile shape the setup autotuner chose for the tensor-core
                                      M2M (from level l+1 into l), M2L (the full-form batch) and L2L (from
                                      l into l+1) at one right-hand side, as columns * 100 + row tiles * 10
                                      + stages; 0 if not tuned */
} fda_stats;

typedef struct fda_handle fda_handle;

/* Fill *cfg with the defaults listed above. */
void fda_default_config(fda_config *cfg);

/* Create a handle.  cfg (host) is copied.  Returns FDA_ERR_ARG for invalid
 * settings (eps outside [1e-7, 0.1], leaf_max outside [1, 64], ...). */
fda_status fda_create(const fda_config *cfg, fda_handle **out);

/* Sec. 3.3 Step 1 (setup, first part): copy the mesh (host pointers) to the
 * device, compute centroids, normals, areas and quadrature points, sort the
 * elements along a Morton curve, build the adaptive octree, split it into
 * low- and high-frequency regimes for wavenumber k > 0, divide the
 * high-frequency far fields into directional cones, and build the
 * interaction and near-field lists.  All of this runs on the device.
 * Returns FDA_ERR_ARG for nt < 1, indices out of range, a degenerate
 * triangle or k <= 0. */
fda_status fda_build_tree(fda_handle *h, const double *verts, int64_t nv, const int32_t *tris, int64_t nt,
                          double k);

/* Sec. 3.3 Step 1 (setup, second part) and Sec. 4: equivalent and check
 * points, truncated-SVD pseudo-inverses (Eq. svdg, epsg, invg), compressed
 * S2M/M2M/M2L/L2L/L2T operators (Eq. cmpm2l and the compressed forms of
 * Sec. 4.3), and the near-field matrix of Eq. eq_sum with its singular and
 * near-singular element integrals, all in FP64 on the device. */
fda_status fda_precompute_translations(fda_handle *h);

/* y = A x (Sec. 3.3 Steps 2-4): x, y device pointers, nrhs columns with
 * leading dimension ld (complex elements).  x and y must not overlap.
 * Columns are processed max_rhs at a time in one pass (every operator read
 * serves all of them). */
fda_status fda_apply(fda_handle *h, const fda_c128 *x, fda_c128 *y, int nrhs, int64_t ld);

/* Same as fda_apply with x and y in host memory: the copies to and from the
 * device are part of the call (synchronises the stream). */
fda_status fda_apply_host(fda_handle *h, const fda_c128 *x, fda_c128 *y, int nrhs, int64_t ld);

/* Right-hand side of Eq. eq_bm for a sound-hard body and plane waves
 * u_inc = e^{ik d.x}: b = u_inc + alpha du_inc/dn at the centroids.
 * dirs: host double[nrhs][3] unit vectors; b: device, ld = nt. */
fda_status fda_rhs_plane_wave(fda_handle *h, const double *dirs, int nrhs, fda_c128 *b);

/* Right-hand side of Eq. eq_bm for a sound-hard body and point sources
 * u_inc = G(x, x_s) (the sphere comparison of Sec. 5.2):
 * b = u_inc + alpha du_inc/dn at the centroids.  src: host double[nrhs][3]
 * source positions (finite, off the surface: a source on a centroid gives a
 * non-finite b, which fda_solve reports as FDA_ERR_NUMERIC); b: device,
 * ld = nt.  Synchronises the stream. */
fda_status fda_rhs_point_source(fda_handle *h, const double *src, int nrhs, fda_c128 *b);

/* Fields off the surface from a solution u (device, nt values in the
 * caller's order, e.g. fda_solve's x) and its Neumann data q = du/dn (device,
 * NULL = 0, the sound-hard case): Green's representation of Eq. cbie in the
 * acoustic domain (c = 1),
 *   u_sc(x) = int G(x, y) q(y) dy - int dG/dn_y(x, y) u(y) dy
 * (add u_inc for the total field), and its far-field pattern, u_sc ~
 * e^{ik|x|}/|x| F(xh) with
 *   F(xh) = (1/(4 pi)) int [ q(y) + ik (xh . n_y) u(y) ] e^{-ik xh . y} dy.
 * Every element by the six-point rule, summed directly over all elements
 * for each target (N x M x 6 FP64 evaluations; no fast algorithm), so
 * points closer to the surface than about two element sizes lose accuracy.
 * dirs: host double[ndir][3] unit vectors; pts: host double[npts][3];
 * F, out: device, caller-owned, overwritten.  Needs fda_precompute_translations
 * (FDA_ERR_STATE before); synchronises the stream. */
fda_status fda_far_field(fda_handle *h, const fda_c128 *u, const fda_c128 *q, const double *dirs, int ndir,
                         fda_c128 *F);
fda_status fda_scattered_field(fda_handle *h, const fda_c128 *u, const fda_c128 *q, const double *pts, int64_t npts,
                               fda_c128 *out);
/* The same far-field pattern F through the fast algorithm's upward pass
 * (Sec. 3.3 Step 2): the outgoing densities of -D[u] + S[q] (S2M of the
 * operator for u, S2M of the right-hand side's layers for q, M2M in FP64)
 * at the coarsest level with interaction lists, whose equivalent sources
 * phi = V q~ give each box's pattern: F(xh) = (1/(4 pi)) sum over boxes and
 * equivalent points of phi e^{-ik xh.y} (at a high-frequency level the box's
 * densities of the cone containing xh).  Elements of leaves above that level
 * are summed directly.  Accurate to a few times the operator's eps (a
 * high-frequency cone's densities are fitted on check points out to the
 * body's size, and the pattern extrapolates them to infinity); about (boxes x T +
 * equivalent points x T) work per direction instead of N x 6.  A non-NULL q
 * builds the right-hand side's layers on first use, as fda_rhs_neumann.
 * Arguments, errors and synchronisation as fda_far_field. */
fda_status fda_far_field_fast(fda_handle *h, const fda_c128 *u, const fda_c128 *q, const double *dirs, int ndir,
                              fda_c128 *F);
/* The same scattered field u_sc at points through the fast algorithm
 * (Sec. 3.3 Steps 2-3 with the points as L2T targets): the outgoing densities
 * of -D[u] + S[q] by S2M and M2M, the local densities by M2L and L2L (once
 * per call: in FP64, or in the chosen precision as in its apply, FP32 S2M
 * and tensor-core translations), then per point (FP64 arithmetic, FP32 in
 * the chosen precision):
 *   * the point is placed in the deepest box of the tree whose cube contains
 *     it; if that box A is a low-frequency box with local densities, the
 *     field of every source A's local density covers (the interaction lists
 *     of A and its ancestors) is A's L2T at the point (Eq. l2t with the
 *     value of G as the target kernel);
 *   * the rest of the sources (A's near field as if A were a leaf, or the
 *     whole tree for a point outside every low-frequency box) are walked
 *     top-down: a box that is not near the point's cube of its level (the
 *     interaction-list test, directional at a high-frequency level) adds
 *     sum_e G(x, y_e) phi_e over its equivalent sources phi = V q~ (the
 *     cone towards the point at a high-frequency level), a near leaf is
 *     summed element by element by the six-point rule, a near box with
 *     children is opened.
 * Agrees with fda_scattered_field to about the operator's eps relative to the
 * field's scale (the same six-point rule on the near elements), so points
 * closer to the surface than about two element sizes lose accuracy in the
 * same way; a point on an element's quadrature point gives a non-finite
 * value.  Work per point: the L2T (n_chk x T) plus the boxes and elements
 * it walks, instead of N x 6.  FDA_ERR_STATE if more than 2,048 boxes of one
 * level are near one point (the values are then NaN).  A non-NULL q builds
 * the right-hand side's layers on first use, as fda_rhs_neumann.  Arguments,
 * errors and synchronisation as fda_scattered_field. */
fda_status fda_scattered_field_fast(fda_handle *h, const fda_c128 *u, const fda_c128 *q, const double *pts,
                                    int64_t npts, fda_c128 *out);

/* Right-hand side of Eq. eq_bm for a radiating body with given Neumann data
 * q = du/dn (no incident field), the layers of the equation's right-hand
 * side evaluated by the same fast directional algorithm (Sec. 3.3 Steps 2-4
 * with single-layer sources):
 *   b_i = -alpha q_i / 2 + sum_j int_{tri_j} [ G + alpha dG/dn_x ](x_i, y) dy q_j
 * (c = 1/2 at a centroid; the adjoint double layer vanishes on the element
 * itself).  q, b: device, nrhs columns with leading dimension ld >= nt, not
 * overlapping; the handle's precision applies (chosen: FP32 near field and
 * split-bf16 translations).  The first call builds this side's near field
 * and single-layer S2M operators (FP64 quadrature; about the cost and memory
 * of the operator's own near field) and synchronises; later calls are
 * stream-ordered.  For a body that also scatters an incident wave, add
 * fda_rhs_plane_wave's result. */
fda_status fda_rhs_neumann(fda_handle *h, const fda_c128 *q, fda_c128 *b, int nrhs, int64_t ld);

/* Allocation-free variant of fda_rhs_plane_wave, for callers that must not
 * have the library allocate device memory during the call: real-time loops
 * that forbid allocator calls (cudaMalloc / cudaFree can synchronise the
 * device), and applications whose device memory is owned by their own pool
 * allocator, where an allocation behind their back could exceed their
 * budget.  The paper has no counterpart; this is an interface convenience.
 *   - It calls no cudaMalloc / cudaFree and no allocating library routine.
 *     The directions are staged in a fixed device array of
 *     FDA_NOALLOC_MAX_DIRS unit vectors (6 KB) that every GPU loading the
 *     library keeps until the process exits, and b is written directly in
 *     the caller's triangle order.
 *   - nrhs must be in [1, FDA_NOALLOC_MAX_DIRS]; larger requests return
 *     FDA_ERR_ARG.  dirs: host double[nrhs][3] unit vectors; b: device,
 *     column-major with ld = nt, owned by the caller.
 *   - All calls share the staging array, which keeps the last call's
 *     directions; calls whose work overlaps on the GPU (other streams or
 *     host threads) race on it.  The first call on a device looks up the
 *     array's device address; make that first call before any stream
 *     capture.
 *   - dirs is copied into the staging array by cudaMemcpyAsync on the
 *     handle's stream.  From pageable host memory CUDA may first wait for
 *     the stream's earlier work and returns once dirs has been read, so the
 *     caller may reuse dirs on return.  From pinned host memory the copy runs
 *     later, in stream order: dirs must stay valid and unchanged until the
 *     stream has reached it (synchronise, or wait on an event recorded after
 *     the call).
 * The result equals fda_rhs_plane_wave's.  Stream-ordered. */
#define FDA_NOALLOC_MAX_DIRS 256
fda_status fda_rhs_plane_wave_noalloc(fda_handle *h, const double *dirs, int nrhs, fda_c128 *b);

/* GMRES (Sec. 5): solve A x = b to ||b - A x|| / ||b|| <= tol for each of
 * nrhs columns (device pointers, ld = nt; x holds the initial guess on
 * entry, zero is fine).  Plain precision: GMRES(restart) on the FP64 FDA
 * operator.  Chosen precision: GMRES on the FP32 operator inside an outer
 * loop that evaluates the residual with the FP64 operator.  info (host, may
 * be NULL) receives the last column's figures.  Returns
 * FDA_ERR_NOT_CONVERGED when maxit is reached above tol. */
fda_status fda_solve(fda_handle *h, const fda_c128 *b, fda_c128 *x, int nrhs, double tol, fda_info *info);

/* Select the operator precision used by later fda_apply / fda_solve calls.
 * FDA_CHOSEN_FP32 needs a handle created with precision = FDA_CHOSEN_FP32
 * (which also keeps the FP64 operators); otherwise FDA_ERR_STATE. */
fda_status fda_set_precision(fda_handle *h, int precision);

/* Switch the tensor-core M2L of the chosen precision on (1) or off (0) for
 * later calls (needs a handle created with tensor_cores = 1 to turn on). */
fda_status fda_set_tensor_cores(fda_handle *h, int on);

/* The octree and lists of Sec. 3.3 Step 1 as built on the device, copied to
 * the host for checking them against an independent construction (no
 * counterpart in the paper's interface).  fda_tree_sizes fills sizes[0] =
 * boxes over all levels, sizes[1] = leaves, sizes[2] = interaction-list
 * entries, sizes[3] = near-field columns over all leaves.  fda_get_tree
 * copies (host arrays, caller-owned, sized from fda_tree_sizes; any may be
 * NULL to skip it; synchronises the stream):
 *   box_level[nbox], box_coord[nbox][3] (integer cube coordinates at the
 *   box's level: the cube is root_lo + w_l [c, c + 1)), box_leaf[nbox] (0/1),
 *   box_parent[nbox] (-1 for the root), box_begin[nbox] / box_end[nbox] (the
 *   box's elements as a range of Morton positions), perm[nt] (Morton
 *   position -> caller's triangle index), il_ptr[nbox + 1] / il_src[n_il]
 *   (each box's M2L interaction list: source boxes of its level),
 *   leaf_box[nleaf] (box of each leaf), nf_colptr[nleaf + 1] / nf_cols[ncols]
 *   (each leaf's near-field columns as Morton positions).
 * Boxes are numbered level by level.  FDA_ERR_STATE before fda_build_tree. */
fda_status fda_tree_sizes(fda_handle *h, int64_t *sizes);
fda_status fda_get_tree(fda_handle *h, int32_t *box_level, int32_t *box_coord, int32_t *box_leaf,
                        int32_t *box_parent, int32_t *box_begin, int32_t *box_end, int32_t *perm, int64_t *il_ptr,
                        int32_t *il_src, int32_t *leaf_box, int64_t *nf_colptr, int32_t *nf_cols);

/* Force the tile shape of every tensor-core translation launch (Sec. 3.3
 * Steps 2-3 on the tensor cores) for later calls, in place of the
 * autotuner's choice: (columns per tile, 64-row tiles per CTA tile, ring
 * stages) one of (32,1,2), (32,1,4), (64,1,2), (64,1,4), (32,2,4), (64,2,3),
 * (64,2,4), (32,3,3), (32,3,4), (128,1,3), (128,1,4), (128,2,2), (128,2,3), (64,3,3),
 * (64,4,2) (the last four with one accumulator slot); (0,0,0) returns to the tuned shapes.  A shape with
 * more row tiles than an operator has falls back to one row tile there.
 * Captured graphs are released (the next applies capture again).  Results
 * equal the tuned shapes' up to the rounding order of the float atomics.
 * FDA_ERR_ARG for any other shape. */
fda_status fda_set_tc_tiles(fda_handle *h, int columns, int row_tiles, int stages);

/* Select the preconditioner used by later fda_solve calls: 0 none, 1 leaf
 * block-diagonal (needs a handle created with precond = 1, which builds the
 * block inverses during fda_precompute_translations; else FDA_ERR_STATE),
 * 2 learned SAI (needs fda_sai_set or fda_sai_set_pattern first; else
 * FDA_ERR_STATE; the pattern last set is used). */
fda_status fda_set_precond(fda_handle *h, int precond);

/* Tree, list and operator statistics (host struct). */
fda_status fda_get_stats(fda_handle *h, fda_stats *out);

/* Per-pass device time of the most recent fda_apply, in milliseconds,
 * measured with CUDA events on the library stream when timing is enabled:
 * out[0] S2M, out[1] M2M, out[2] M2L, out[3] L2L, out[4] L2T, out[5] near
 * field (S2T).  Returns FDA_ERR_STATE if timing is off. */
fda_status fda_set_timing(fda_handle *h, int enable);
fda_status fda_get_pass_times(fda_handle *h, float out[6]);

/* ---- Learned sparse approximate inverse (SAI) preconditioner ----
 * Not in the paper (which solves unpreconditioned, Sec. 5.3): a right
 * preconditioner M on the leaf-block pattern (i, j in the same leaf; the
 * near-field pattern is below, fda_sai_set_pattern) whose
 * entries a small network predicts from the pair's local geometry and k
 * (8 rotation-invariant features: k|x_j - x_i|, the two normal projections of
 * the unit separation, n_i.n_j, k sqrt(area_i), k sqrt(area_j), [i == j],
 * sqrt(area_j)/max(|x_j - x_i|, sqrt(area_j)); two tanh layers of 32; output
 * Re, Im of M_ij).  Training minimises
 *     L = (1/sum_B n_B) sum_B ||M_B A_BB - I||_F^2
 * over the leaf self blocks A_BB of the near-field matrix (Eq. eq_sum) that
 * fda_precompute_translations built.  Weights are fda_sai_num_params() floats,
 * caller-owned, layout W1[32][8], b1[32], W2[32][32], b2[32], W3[2][32], b3[2]. */
typedef struct {
    int epochs;               /* Adam steps (default 400) */
    double lr;                /* Adam step size (default 3e-3) */
    unsigned long long seed;  /* seed of fda_sai_init_weights used by callers, and of the leaf
                                 draws of pattern 1 (default 1) */
    int pattern;              /* 0: leaf blocks, full batch (default); 1: near-field pattern */
    int sample_leaves;        /* pattern 1: leaves drawn from each handle per step (default 256) */
} fda_sai_config;

typedef struct {
    double loss_init;   /* L of the initial weights over all training blocks */
    double loss_final;  /* L after training */
    double train_s;     /* wall time of the training call */
} fda_sai_report;

int fda_sai_num_params(void);
fda_status fda_sai_default_config(fda_sai_config *cfg);
/* Xavier-uniform weights from splitmix64(seed), zero biases (host). */
fda_status fda_sai_init_weights(unsigned long long seed, float *weights);
/* Train on the leaf blocks (cfg->pattern 0) or the near-field pattern
 * (cfg->pattern 1, below) of nhandles precomputed handles (their own
 * near-field matrices, FP32 kernels on the first handle's stream).  weights:
 * host, in = initial, out = trained.  FDA_ERR_STATE before precompute,
 * FDA_ERR_NUMERIC if the loss stops being finite; message on handles[0]. */
fda_status fda_sai_train(fda_handle *const *handles, int nhandles, const fda_sai_config *cfg, float *weights,
                         fda_sai_report *rep);
/* Evaluate the network on h's leaf blocks and keep the result as h's learned
 * preconditioner (select it with fda_set_precond(h, 2)).  loss (optional,
 * host) receives L of the stored M against the FP64 blocks. */
fda_status fda_sai_set(fda_handle *h, const float *weights, double *loss);
/* The same network on the near-field pattern.  For pattern 1 it predicts
 * M_ij for every row i of a leaf B and every column j of B's near-field
 * columns C_B (the leaf's own elements and those of its near leaves, the
 * columns of the near-field matrix's rows of B), and training minimises
 *     L = (1/sum_B n_B) sum_B ||M[B, C_B] A_near[C_B, C_B] - I[B, C_B]||_F^2,
 * A_near the near-field matrix (a row l of leaf C holds C's own near-field
 * columns, 0 elsewhere), by Adam on sample_leaves leaves of each handle per
 * step (loss_init / loss_final: L on one fixed draw of that many leaves per
 * handle, before and after).
 *   - fda_sai_set_pattern: pattern 0 is fda_sai_set; pattern 1 evaluates M on
 *     h's whole near-field pattern (FP32, nnz_near entries, the near-field
 *     matrix's layout) and keeps it as h's learned preconditioner, applied
 *     by the near-field product (select with fda_set_precond(h, 2)).  loss
 *     (optional, host) receives L over all leaves of h in FP32 (pattern 1)
 *     or as fda_sai_set (pattern 0).  FDA_ERR_ARG for another pattern.
 *   - fda_sai_loss_grad_near: L and dL/dweights (fda_sai_num_params()
 *     doubles, host) over the leaves leaves[0 .. nleaves) of h (indices into
 *     h's leaf list, as fda_get_tree's leaf_box; host), normalised by their
 *     rows; precision FDA_PLAIN_FP64 runs the FP64 kernels on h's FP64
 *     near-field matrix, FDA_CHOSEN_FP32 the FP32 training kernels (weights
 *     rounded to FP32).  FDA_ERR_STATE before precompute; FDA_ERR_ARG for
 *     indices out of range.
 * Both need leaves of at most 64 elements (FDA_ERR_ARG otherwise). */
fda_status fda_sai_set_pattern(fda_handle *h, const float *weights, int pattern, double *loss);
fda_status fda_sai_loss_grad_near(fda_handle *h, const double *weights, int nleaves, const int32_t *leaves,
                                  int precision, double *loss, double *grad);
/* Loss L and gradient dL/dweights (fda_sai_num_params() doubles) of the
 * training kernels for caller-supplied data (host arrays, copied in): n elements
 * with centroids [n][3], normals [n][3], areas [n], wavenumber k; nblocks
 * blocks, block b = elements block_elems[block_ptr[b] .. block_ptr[b+1]) (1 to
 * 64 each, block_ptr[0] = 0), blocks = each block's n_b x n_b matrix
 * row-major, concatenated.  precision = FDA_PLAIN_FP64 runs the FP64
 * instantiation of the kernels, FDA_CHOSEN_FP32 the FP32 one that training
 * uses (weights and blocks rounded to FP32).  Needs a GPU; no handle (returns
 * the status only). */
fda_status fda_sai_loss_grad(int64_t n, const double *centroids, const double *normals, const double *areas,
                             double k, int nblocks, const int64_t *block_ptr, const int32_t *block_elems,
                             const fda_c128 *blocks, const double *weights, int precision, double *loss,
                             double *grad);

/* ---- Several meshes behind one operator application ----
 * A batch holds one handle per mesh, all created from one configuration, and
 * applies the operator of Eq. eq_sum (Sec. 3.3 Steps 2-4) to every mesh's
 * right-hand sides in one call.  With cfg.graphs = 1 the passes of all meshes
 * form one CUDA graph per call (captured on the second call with the same
 * right-hand-side count and per-mesh precision), one parallel branch per
 * mesh, so small meshes share the GPU instead of running one after another.
 * The paper treats one mesh; the batch is an execution arrangement of the
 * same per-mesh operator, and each mesh's result equals fda_apply on its
 * handle up to the rounding order of the float atomics.
 *   - fda_create_batch: nmesh in [1, 64]; cfg as for fda_create (NULL =
 *     defaults).  Every call on the batch or on a mesh's handle is ordered on
 *     cfg.cuda_stream; fda_apply_batch forks one private stream per mesh from
 *     it and joins them back before returning control of the stream.
 *   - fda_build_batch: per mesh i, verts[i] (host double[nv[i]][3]),
 *     tris[i] (host int32[nt[i]][3]) and wavenumber k[i], as fda_build_tree.
 *   - fda_precompute_batch: fda_precompute_translations on every mesh.
 *   - fda_apply_batch: y[i] = A_i x[i] for every mesh i: x[i], y[i] device
 *     pointers (caller-owned, column-major, nrhs columns, leading dimension
 *     ld[i] >= nt[i], x[i] and y[i] not overlapping); x, y, ld are host
 *     arrays of nmesh entries.  Columns go max_rhs at a time.
 *   - fda_batch_mesh: the handle of mesh i, owned by the batch (valid until
 *     fda_destroy_batch; do not destroy it), for fda_solve, fda_get_stats,
 *     fda_rhs_plane_wave, fda_set_precision ...; NULL if i is out of range.
 * Errors: FDA_ERR_ARG for bad sizes or pointers, FDA_ERR_STATE out of order,
 * a mesh's own status (its message prefixed by "mesh i: ") otherwise; the
 * message is read with fda_batch_last_error. */
typedef struct fda_batch fda_batch;

typedef struct {
    int nmesh;
    int64_t n_total;          /* elements over all meshes */
    int64_t graph_replays;    /* batch graph launches so far */
    int graph_fallback;       /* 1 if capture failed and calls run the passes directly */
    size_t device_bytes;      /* device memory held by all meshes */
} fda_batch_stats;

fda_status fda_create_batch(const fda_config *cfg, int nmesh, fda_batch **out);
fda_status fda_build_batch(fda_batch *b, const double *const *verts, const int64_t *nv, const int32_t *const *tris,
                           const int64_t *nt, const double *k);
fda_status fda_precompute_batch(fda_batch *b);
fda_status fda_apply_batch(fda_batch *b, const fda_c128 *const *x, fda_c128 *const *y, int nrhs,
                           const int64_t *ld);
fda_handle *fda_batch_mesh(fda_batch *b, int i);
fda_status fda_get_batch_stats(fda_batch *b, fda_batch_stats *out);
const char *fda_batch_last_error(const fda_batch *b);
/* Release the batch and its meshes' handles (NULL is ignored). */
void fda_destroy_batch(fda_batch *b);

/* Symmetry table of the cone partition of a high-frequency level with
 * nc x nc cells per cube face (6 nc^2 cones, Sec. 3.1; cone index =
 * (2 axis + [sign > 0]) nc^2 + a nc + b, a and b the cell along the two other
 * axes in increasing order).  For every cone u: rep[u] = its representative
 * cone on the +z face and g[9u..9u+8] = the signed axis permutation
 * (row-major, entries -1/0/1) with g_u (centre of rep[u]) = centre of u and
 * g of the opposite cone = -g_u.  The library gives cone u the frame
 * g_u R_rep(u), so M2L offsets related by these maps (the rotation
 * invariance of Sec. 4.1.1) share one operator.  Host only (no GPU needed);
 * rep holds 6 nc^2 ints and g 54 nc^2 ints, both caller-owned.  Returns
 * FDA_ERR_ARG for nc outside [1, 64] or NULL pointers. */
int fda_cone_symmetry_table(int nc, int *rep, int *g);

/* Number of CUDA kernels the library has launched since it was loaded, over
 * all handles and threads (a monotonic counter; the difference around a
 * region is the launches made inside it; a CUDA-graph replay counts the
 * kernels the graph holds).  Never fails. */
long long fda_launch_count(void);

/* Size in bytes of a public struct, for bindings to check their copy of
 * its layout: which = 0 fda_config, 1 fda_info, 2 fda_stats,
 * 3 fda_sai_config, 4 fda_sai_report, 5 fda_batch_stats; 0 for any other
 * value.  Never fails. */
size_t fda_struct_size(int which);

/* Message of the last failing call on this handle (never NULL). */
const char *fda_last_error(const fda_handle *h);

/* Release every resource of the handle (NULL is ignored). */
void fda_destroy(fda_handle *h);

#ifdef __cplusplus
}
#endif

#endif /* FDA_BEM_H */
