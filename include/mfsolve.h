/*
 * mfsolve -- multifrontal direct solver for finite-element matrices on one
 * B300 GPU (sm_103a).  C ABI of libmfsolve.so.
 *
 * The method is the multifrontal LU of arXiv 2306.08994: an elimination tree
 * built bottom-up from element fronts (Sec. 2.4), fronts processed level by
 * level, every level being one Foata normal-form class whose fronts are
 * independent (Sec. 3.3), each front assembled from its children's Schur
 * complements (extend-add, "join_fronts", Table 1), partially factored on its
 * fully assembled pivots with the division / multiplication / subtraction
 * tasks of Sec. 3 and Table 2 (no pivoting, L non-unit, U unit diagonal), and
 * its Schur complement S = F22 - F21 F11^-1 F12 (Sec. 2.2) handed to the
 * parent; the root is factored completely (Table 1).  The solution is
 * obtained by forward and backward substitution (`get_solution`, Table 2).
 *
 * Conventions for every entry point
 *  - Return value: MF_OK (0) or a negative MF_E* code; nothing throws across
 *    the ABI.  mf_strerror() names a code.
 *  - Pointers named d_* are device pointers (CUDA global memory of the
 *    current device); every other pointer is host memory.  Inputs are owned
 *    by the caller and only borrowed for the duration of the call (device
 *    inputs: until the work enqueued on `stream` has finished).
 *  - Opaque handles are owned by the library until mf_free_*().
 *  - Device work is enqueued asynchronously on `stream` (NULL = legacy
 *    default stream); device-detected conditions (perturbed or zero pivots,
 *    non-finite values) are reported by mf_status(), which synchronises.
 *  - Handles are not thread-safe; use one handle per host thread.
 *  - Element matrices: n_elem blocks of npe*npe doubles, block e column-major
 *    (entry (a,b) of element e at e*npe*npe + a + b*npe), rows/columns in the
 *    order of that element's nodes.  Dirichlet conditions are the caller's:
 *    the library solves the assembled system sum_e P_e^T K_e P_e exactly as
 *    given.
 *  - Vectors: n_dof x nrhs doubles, column-major (dof fastest).
 */
#ifndef MFSOLVE_H
#define MFSOLVE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ABI-compatible with cudaStream_t / CUstream. */
typedef struct CUstream_st* mf_stream_t;

#define MF_OK 0
#define MF_EINVAL (-1)       /* bad argument or handle */
#define MF_ENOMEM (-2)       /* device or host allocation failed */
#define MF_ECUDA (-3)        /* a CUDA runtime call failed */
#define MF_EZERO_PIVOT (-4)  /* |pivot| below the static threshold with pivot_fail set */
#define MF_ENOCONV (-5)      /* refinement did not reach the tolerance within maxit */
#define MF_ETIMEOUT (-6)     /* a bounded device wait ran out */
#define MF_ENOTSUP (-7)      /* option or input form not supported */
#define MF_ETOOLARGE (-8)    /* problem larger than mf_residual_noalloc's static scratch */

/* Arithmetic of the fronts (factor storage, extend-add, partial LU, Schur
 * update, triangular solves).  Residuals and solution updates are always FP64. */
#define MF_F64 0   /* FP64 throughout: the plain path */
#define MF_F32 1   /* FP32 fronts, FP32 SIMT Schur GEMMs */
#define MF_TF32 2  /* FP32 fronts, Schur GEMMs of large fronts on the tensor cores (tcgen05,
                      three-pass split TF32 = FP32-accurate products), FP32 accumulation */
#define MF_TF32_BF16 3  /* as MF_TF32, but the Schur updates S -= L21 U12 (Sec. 2.2) of fronts with a
                      contribution block of at least bf16_min_cb rows use BF16 tensor-core products
                      (kind::f16, FP32 accumulation): one BF16 product (bf16_passes 1) or three
                      split-BF16 products (bf16_passes 3) */

/* Front-size buckets of the fused small-front kernel (upper bounds on m). */
#define MF_FUSED_BUCKETS 9

typedef struct {
    int precision;        /* MF_F64 (default), MF_F32, MF_TF32 or MF_TF32_BF16 */
    double pivot_tol;     /* static pivot check: a pivot with |p| < pivot_tol * max|F| (max over its
                             front at assembly) is replaced by sign(p) * that bound (counted in
                             mf_status) or fails; <= 0 selects the unit roundoff of `precision` */
    int pivot_fail;       /* nonzero: a small pivot makes mf_status return MF_EZERO_PIVOT */
    int small_front_max;  /* fronts with m <= this run in the fused one-CTA kernel; 0 = default */
    int panel_width;      /* pivot block width of the large-front partial LU; 0 = default */
    int use_graph;        /* nonzero: replay factor/solve as captured CUDA graphs */
    int max_nrhs;         /* largest nrhs passed to mf_solve / mf_refine_solve; 0 = 4 */
    int subtree_levels;   /* bottom classes fused per subtree (one CTA walks classes 1..n of a
                             subtree with a block barrier between them): n > 0 = at most n
                             (fewer if a subtree would not fit shared memory); <= 0 = off */
    int sweep_kernel;     /* substitutions of the top classes in one persistent cooperative launch
                             per sweep (bounded grid barriers between dependent phases) instead of
                             one launch per class and kind: 0 = off (default), n > 0 = the top n
                             classes, -1 = every class with at most 2048 fronts */
    int subtree_solve_levels; /* bottom classes fused per subtree in the substitutions (one CTA
                             walks a subtree, update vectors stay in shared memory): n > 0 = at
                             most n, < 0 = off, 0 = as in the factorization (subtree_levels) */
    int tc_min_cb;        /* MF_TF32: smallest contribution block (m - k) whose Schur update runs
                             on the tensor cores; smaller ones use the SIMT GEMM; 0 = 256 */
    int super_panel;      /* pivots per super-panel of the large-front partial LU (a multiple of the
                             panel width): inside a super-panel each panel is updated just before
                             it is factored, the rest of the pivot block once per super-panel;
                             0 = default (256 for FP32 fronts, the panel width for FP64) */
    int fused_threads[MF_FUSED_BUCKETS];
                          /* threads per CTA of the fused small-front kernel for each front-size
                             bucket (m <= 16, 32, 48, 64, 96, 128, 160, 192, 224): 32, 64, 128 or
                             256; 0 = default (128 up to m = 64, 256 above).  Fronts with m <= 32
                             run in the lane-group kernel instead (one group of 4, 8, 16 or 32
                             lanes per front), so the first two entries are not used. */
    int lookahead;        /* one-panel lookahead in the large-front partial LU: the next pivot block
                             takes its share of the pending update (every pivot of its super-panel
                             so far) and is factored on a second stream while the rest of the update
                             runs; 0 = on (default), < 0 = off */
    int bf16_min_cb;      /* MF_TF32_BF16: smallest contribution block whose Schur update uses BF16
                             products; 0 = 2048 */
    int bf16_passes;      /* MF_TF32_BF16: 1 (default, also 0) = one BF16 product, 3 = hi/lo split */
    int foata_classes;    /* the bottom foata_classes classes run the paper's scalar-task schedule
                             (Sec. 3.3): per pivot step one launch each for the assertion (static
                             pivot check), division, multiplication and subtraction tasks of every
                             front of the class, after an extend-add launch; 0 = off (default: the
                             fused per-front kernels); turns off subtree fusion */
    int symmetric;        /* nonzero: the caller promises A = A^T.  Then U = D^-1 L^T (D = diag L),
                             so beyond the pivot block the large fronts factor only L, take U12 =
                             D^-1 L21^T by a transposing copy, and compute only the lower half of
                             their Schur update (mirrored after); solves run x = L^-T D L^-1 b and
                             never read U; mf_solve_adjoint equals mf_solve.  0 = general LU */
    int refine_cg;        /* with symmetric (and A positive definite): mf_refine_solve runs the FP64
                             preconditioned conjugate-gradient method with the factorization as
                             preconditioner (M^-1 = L^-T D L^-1, symmetric positive definite)
                             instead of stationary refinement; the stop test uses the normwise
                             backward error of the recursively updated residual, confirmed on the
                             true residual b - A x (restarting from x if they disagree);
                             iterations = preconditioner applications after the first; 0 = off */
    int panel_trsm;       /* large-front partial LU: 0 (default) = the pivot-block kernel also inverts
                             both triangles and the panel is finished by products with the inverses;
                             nonzero = the panel is finished by triangular solves against the factored
                             block (one thread per row or column; slower here, kept as an option) */
    int tc_direct;        /* MF_TF32 products: 0 (default) = a separate pass packs the tf32 hi/lo split
                             operands into the MMA's shared-memory image, which the product kernel
                             streams with bulk copies; nonzero = the product kernel loads the FP32
                             operands and splits them in shared memory itself (no pack pass; slower
                             here: its element loads keep too few bytes in flight) */
    int root_f64;         /* FP32-family fronts: the pivot blocks of the large fronts in the top
                             root_f64 Foata classes (1 = the root's class) are factored and inverted
                             in FP64 from the FP32 front and rounded once to FP32; 0 = none (default) */
} mf_options;

typedef struct {
    int dim;                      /* 2 or 3 */
    int64_t n_nodes;              /* number of dofs (one per node) */
    int64_t n_elem;
    int nodes_per_elem;           /* npe, <= 64 */
    const int64_t* elem_nodes;    /* n_elem * npe node ids, element e at [e*npe, (e+1)*npe) */
    const double* elem_centroid;  /* n_elem * dim coordinates used for recursive coordinate
                                     bisection when grid_dims is NULL; may be NULL otherwise */
    const int32_t* grid_dims;     /* {nx, ny, nz} (nz = 1 in 2D) for a structured grid whose
                                     element (ex,ey,ez) has id ex + nx*(ey + ny*ez): the tree is
                                     the recursive floor bisection of the element box along its
                                     longest axis (ties x, y, z) -- or NULL */
} mf_mesh_desc;

typedef struct {
    int64_t n_dof, n_elem, n_front, n_meshes;
    int32_t n_classes;    /* Foata classes = tree height (leaves are class 1) */
    int32_t max_m, max_k, root_m;
    int64_t sum_k;        /* equals n_dof */
    int64_t nnz_lu;       /* sum over fronts of m*k + k*(m-k) */
    int64_t sum_cb;       /* sum over fronts of (m-k)^2 */
    double factor_flops;  /* sum over pivots of (m-p-1) + 2 (m-p-1)^2 */
    double solve_flops;   /* per right-hand side: 2 nnz_lu (approx.) */
} mf_info;

typedef struct {
    int64_t n_perturbed;  /* pivots replaced by the static check */
    int32_t first_front;  /* front (analysis numbering) of the first small pivot, or -1 */
    int32_t first_pivot;  /* its pivot index inside the front, or -1 */
    int32_t nonfinite;    /* nonzero if a non-finite pivot was met */
    int32_t timeout;      /* nonzero if a bounded device wait ran out */
} mf_status_info;

typedef struct {
    int iterations;       /* refinement corrections applied */
    double backward_error;/* final ||b - A x||_inf / (||A||_inf ||x||_inf + ||b||_inf), max over rhs */
    double rel_residual;  /* final ||b - A x||_2 / ||b||_2, max over rhs */
} mf_refine_info;

typedef struct mf_analysis mf_analysis;
typedef struct mf_factors mf_factors;

void mf_default_options(mf_options* opt);
const char* mf_strerror(int code);

/* Symbolic analysis of one mesh (Sec. 2.4 tree, Table 2 pivot rule, Sec. 3.2
 * pivots-first ordering, Sec. 3.3 Foata classes at front granularity).  Host
 * only; copies everything it needs from `mesh`.  `opt` may be NULL. */
int mf_analyze_mesh(const mf_mesh_desc* mesh, const mf_options* opt, mf_analysis** out);

/* Analysis of `count` independent meshes solved together: one forest whose
 * fronts of equal height (aligned from the leaves) form one class, so each
 * class runs as one batched pass across all meshes.  Dofs, elements and
 * vectors are the meshes' concatenated in order. */
int mf_analyze_batch(const mf_mesh_desc* meshes, int count, const mf_options* opt, mf_analysis** out);

/* Symbolic analysis of a general sparse n x n matrix given by its CSR pattern
 * (host arrays, copied): rowptr (n+1 int64, rowptr[0] = 0, non-decreasing)
 * and col (rowptr[n] int32 column ids in [0, n), strictly increasing within a
 * row; entry q of the value array sits at row i, column col[q] for
 * rowptr[i] <= q < rowptr[i+1]).  The paper applies the method to symmetric
 * invertible finite-element matrices (Sec. 2.1) and builds the tree from
 * element fronts (Sec. 2.4); without elements or coordinates, the tree here
 * cuts the graph of A + A^T in two recursively (breadth-first level structure
 * from a pseudo-peripheral vertex, split in half) down to single vertices,
 * and vertex w's element holds a_ww and, for each off-diagonal pair {u, w}
 * placed on the left side of the cut that separates u and w, the entries
 * a_wu and a_uw; the right-side boundary of every cut becomes its separator.
 * The mesh analysis then runs on those elements.  Numeric calls on factors of
 * this analysis (mf_factor, mf_refine_solve, mf_refine_solve_adjoint,
 * mf_residual, mf_autotune) take d_values = the CSR values (rowptr[n]
 * doubles, device, in the order of col); mf_element_grad and
 * mf_element_outer return MF_ENOTSUP.  A structurally unsymmetric pattern is
 * symmetrised (missing mirror entries are zeros).  Limits: n < 2^30, and each
 * vertex's element may hold at most 63 pairs (else MF_ENOTSUP); bad arrays
 * give MF_EINVAL.  The element array (n * npe^2 doubles, npe = the largest
 * element) is allocated by mf_factors_create. */
int mf_analyze_csr(int64_t n, const int64_t* rowptr, const int32_t* col, const mf_options* opt, mf_analysis** out);

int mf_analysis_info(const mf_analysis* a, mf_info* out);

/* Export the front structure (fronts numbered class by class).  Every array
 * may be NULL.  parent, cls, m, k: n_front entries (parent -1 at a root);
 * dof_ptr: n_front+1 offsets into dofs; dofs: sum of m entries, each front's
 * pivots (ascending dof id) followed by its contribution-block dofs
 * (ascending). */
int mf_analysis_export(const mf_analysis* a, int32_t* parent, int32_t* cls, int32_t* m, int32_t* k,
                       int64_t* dof_ptr, int32_t* dofs);

/* Allocate the device storage for one factorization of `a` (factor arena,
 * contribution-block arena, solve and refinement work space) and upload the
 * front maps.  Allocation happens here and only here, so mf_factor /
 * mf_solve / mf_refine_solve allocate nothing.  `opt` may be NULL (the
 * analysis options are used). */
int mf_factors_create(const mf_analysis* a, const mf_options* opt, mf_factors** out);

/* Numeric factorization (Tables 1-2): class by class, one batched pass per
 * class of extend-add, partial LU with the static pivot check, and Schur
 * update.  d_values: the element matrices (see conventions), device. */
int mf_factor(mf_factors* f, const double* d_values, mf_stream_t stream);

/* x = A^-1 b in place: forward substitution with L leaves->root, backward
 * with U root->leaves (get_solution, Table 2).  d_rhs: n_dof x nrhs. */
int mf_solve(mf_factors* f, double* d_rhs, int nrhs, mf_stream_t stream);

/* x = A^-T b in place with the same factors: U^T forward, L^T backward. */
int mf_solve_adjoint(mf_factors* f, double* d_rhs, int nrhs, mf_stream_t stream);

/* Iterative refinement in FP64: x = solve(b); repeat r = b - A x (FP64,
 * element by element), x += solve(r) until the normwise backward error
 * ||r||_inf / (||A||_inf ||x||_inf + ||b||_inf) <= tol or maxit corrections.
 * Returns MF_ENOCONV if tol was not reached (x still holds the last iterate).
 * Synchronises `stream` once per correction to test convergence. */
int mf_refine_solve(mf_factors* f, const double* d_values, const double* d_b, double* d_x, int nrhs,
                    double tol, int maxit, mf_refine_info* info, mf_stream_t stream);

/* The same refinement for the adjoint system A^T x = b (the adjoint solve of
 * the gradient, Sec. 4): x = solve_adjoint(b); repeat r = b - A^T x (FP64,
 * element by element with the transposed element matrices), x +=
 * solve_adjoint(r) until ||r||_inf / (||A^T||_inf ||x||_inf + ||b||_inf) <=
 * tol or maxit corrections.  Arguments, layout and return codes as
 * mf_refine_solve. */
int mf_refine_solve_adjoint(mf_factors* f, const double* d_values, const double* d_b, double* d_x, int nrhs,
                            double tol, int maxit, mf_refine_info* info, mf_stream_t stream);

/* r = b - A x in FP64 with A given element by element. */
int mf_residual(const mf_factors* f, const double* d_values, const double* d_x, const double* d_b,
                double* d_r, int nrhs, mf_stream_t stream);

/* Adjoint gradient for per-element parameters: g_e = -lambda_e^T dK_e x_e,
 * dK_e = dK/dtheta_e given as element matrices (same layout as values);
 * lambda solves A^T lambda = dJ/dx (mf_solve_adjoint).  One right-hand side. */
int mf_element_grad(const mf_factors* f, const double* d_dvalues, const double* d_lambda, const double* d_x,
                    double* d_grad, mf_stream_t stream);

/* Gradient with respect to the element matrices themselves:
 * G_e = -lambda_e x_e^T (npe x npe, column-major per element), summed over
 * nrhs right-hand sides. */
int mf_element_outer(const mf_factors* f, const double* d_lambda, const double* d_x, int nrhs,
                     double* d_gradK, mf_stream_t stream);

/* Synchronise and report what the device saw during the last mf_factor.
 * Returns MF_EZERO_PIVOT if a pivot was small and pivot_fail is set. */
int mf_status(mf_factors* f, mf_status_info* out);

/* Copy front `front`'s factor to the host as FP64: L (m x k, column-major:
 * the pivot columns, L on/below the diagonal, U11 strictly above) and U
 * (k x m, column-major: the pivot rows).  Synchronises.  For tests. */
int mf_factors_export_front(const mf_factors* f, int32_t front, double* L, double* U);

/* r = b - A x (A given element by element, FP64) without any device
 * allocation.  The paper has no counterpart: this serves callers that may not
 * call cudaMalloc or any allocating routine when they evaluate a residual --
 * code under a memory budget fixed in advance, host frameworks that own
 * every device allocation through their own pool, real-time loops that
 * cannot afford an allocation's implicit synchronisation -- and that hold no
 * mf_factors handle.  Every pointer is the caller's: d_elem_nodes (device,
 * n_elem * npe global dof ids, as in mf_mesh_desc), d_values (element
 * matrices, as for mf_factor), d_x, d_b, d_r (n_dof x nrhs).
 * Limits: 1 <= nodes_per_elem <= 64 and 1 <= nrhs <= 65535, else MF_EINVAL
 * with nothing launched.  Work space is one file-scope device array of
 * MF_NOALLOC_MAX_ENTRIES doubles (8 MiB) that a device holds from the moment
 * the library's device code is loaded there until exit; with CUDA's lazy
 * module loading (the default) that moment is the first call of this entry
 * point on the device, which may therefore take device memory once; later
 * calls take none.  n_dof * nrhs beyond the array returns MF_ETOOLARGE and
 * launches nothing.  The caller must keep every id in d_elem_nodes in
 * [0, n_dof): the kernel checks each id before using it, never reads or
 * writes through one outside that range, and then fills all of d_r with NaN
 * (the call returns before the GPU runs, so the NaN output is the report).
 * The first call on a device looks the array's address up
 * (cudaGetSymbolAddress, that device current) and caches it: make that first
 * call before any stream capture.  The cached address belongs to the CUDA
 * context of that first call; after cudaDeviceReset, load the library afresh.
 * Calls share the array (each clears what it uses first), so calls that
 * overlap on the GPU race.  Sums use FP64 atomics: results equal
 * mf_residual's up to rounding order. */
#define MF_NOALLOC_MAX_ENTRIES (1 << 20)
int mf_residual_noalloc(int64_t n_dof, int64_t n_elem, int nodes_per_elem, const int64_t* d_elem_nodes,
                        const double* d_values, const double* d_x, const double* d_b, double* d_r, int nrhs,
                        mf_stream_t stream);

/* Per-kernel-family accounting for roofline reports.  While enabled, every
 * launch issued by mf_factor / mf_solve / mf_solve_adjoint / mf_refine_solve
 * is bracketed by CUDA events on the launching stream and its algorithmic
 * work is added up: bytes = the data the operation must move at minimum
 * (inputs read once, outputs written once), flops = the arithmetic the
 * algorithm performs.  Families: 0 fused small fronts, 1 large-front
 * assembly, 2 panel LU, 3 trailing GEMM, 4 Schur GEMM, 5 forward
 * substitution, 6 backward substitution, 7 residual and norms, 8 other,
 * 9 pivot-block inverses (for the substitutions).
 * mf_profile_read synchronises, writes MF_PROFILE_FAMILIES entries to each
 * non-NULL array (summed since the last read) and resets the sums. */
#define MF_PROFILE_FAMILIES 10
int mf_profile_enable(mf_factors* f, int enable);
int mf_profile_read(mf_factors* f, double* ms, int64_t* launches, double* bytes, double* flops);

/* Launch trace of the profiled region: one record per event-bracketed launch
 * (a factorization launch, or all kernels of one class of a substitution),
 * in issue order.  kind: 0 fused small fronts, 1 large-front assembly,
 * 2 panel diagonal block, 3 SIMT GEMM, 4 pivot-block inverses, 5 subtree
 * factorization, 6 tensor-core GEMM, 7 lane-group tiny fronts, 8 tensor-core
 * operand packing, 9 scalar-task Foata executor, 13 symmetric-mode U12 copy,
 * 14 symmetric-mode contribution-block mirror, 15 panel triangular solves,
 * 16 tensor-core GEMM splitting its own operands, or one of the
 * MF_TRACE_* codes below;
 * cls: 0-based Foata class or -1; tasks: fronts, tiles or tasks in the launch.
 * Call before mf_profile_read (which clears the trace).  Writes at most `cap`
 * records and stores the number recorded in *n; synchronises. */
#define MF_TRACE_FWD_CLASS 100
#define MF_TRACE_BWD_CLASS 101
#define MF_TRACE_SUBTREE_FWD 102
#define MF_TRACE_SUBTREE_BWD 103
#define MF_TRACE_FWD_SWEEP 104   /* persistent forward sweep (all classes above the subtrees) */
#define MF_TRACE_BWD_SWEEP 105
#define MF_TRACE_OTHER 199
typedef struct {
    int family, kind, cls, tasks;
    double ms;
    double bytes, flops;  /* algorithmic work of the record, as in mf_profile_read */
} mf_trace_rec;
int mf_profile_trace(mf_factors* f, mf_trace_rec* out, int cap, int* n);

/* Plan autotuner.  Sec. 3.3 fixes the class order of the fronts and leaves
 * open how the tasks of one class are cut into launches; the launch plan's
 * free choices are timed here on the caller's problem and the fastest kept:
 *   fused_threads[]  per front-size bucket (per-bucket times of profiled
 *                    factorizations, all buckets in one sweep),
 *   small_front_max  fused / blocked crossover,
 *   subtree_levels, subtree_solve_levels  depth of the bottom-class subtree
 *                    fusion of the factorization and of the substitutions,
 *   super_panel      depth of the deferred trailing updates of large fronts,
 *   precision and tc_min_cb  (FP32 family only) SIMT or tensor-core Schur GEMMs.
 * Candidates are timed as one factorization plus one refined solve
 * (mf_refine_solve to a normwise backward error of 1e-12, so a plan that
 * needs more corrections pays for them; CUDA events on `stream`, CUDA graph
 * replay, median of `reps` after one untimed run).
 * Arguments: a (analysis), d_values (device, element matrices as for
 * mf_factor), d_b (device, n_dof values: the right-hand side of the timed
 * solves; not modified), base (options to start from: its precision family,
 * FP64 or FP32/TF32, is kept; NULL = defaults), reps (>= 1), cache_path (a
 * JSON Lines file, one object per tuned problem keyed by the device and the
 * analysis' shape; an entry with this key is returned without timing, a new
 * result is appended; NULL = no cache), best (out: base with the tuned fields
 * set), info (out, may be NULL).  Allocates and frees one factor set per
 * candidate; returns MF_EINVAL, MF_ENOMEM or MF_ECUDA on failure, in which
 * case `best` is left unchanged.  Synchronises `stream`. */
typedef struct {
    double ms_default;   /* factor + refined solve with `base` (0 when taken from the cache) */
    double ms_best;      /* factor + refined solve with `best` */
    int candidates;      /* plans timed */
    int from_cache;      /* nonzero if `best` came from cache_path */
} mf_tune_info;
int mf_autotune(const mf_analysis* a, const double* d_values, const double* d_b, const mf_options* base, int reps,
                const char* cache_path, mf_options* best, mf_tune_info* info, mf_stream_t stream);

void mf_free_factors(mf_factors* f);
void mf_free_analysis(mf_analysis* a);

/* ---- Testing hooks.  The paper has no counterpart: they let tests drive the
 * library's error paths from the host without faulting, trapping or hanging
 * the GPU. */

/* Host-side allocation-failure injection: the n-th device allocation the
 * library makes from now on (0 = the next one) fails as if the device were
 * out of memory, so the entry point that made it releases what it had
 * allocated and returns MF_ENOMEM.  n < 0 disarms.  Process-wide, not
 * thread-safe with respect to concurrent allocations in other threads. */
void mf_test_fail_alloc(int64_t n);

/* Enqueues on `stream` one bounded device wait that nothing will release: a
 * single CTA waits at the grid barrier of the persistent substitution sweep
 * for a second CTA that is never launched, gives up after limit_ms
 * milliseconds (0 < limit_ms <= 10000, else MF_EINVAL), records a timeout in
 * f's status word and returns; no copy is in flight in that kernel.
 * mf_status(f) then returns MF_ETIMEOUT; the next mf_factor clears the status
 * and the handle stays usable. */
int mf_test_bounded_wait(mf_factors* f, double limit_ms, mf_stream_t stream);

#ifdef __cplusplus
}
#endif
#endif /* MFSOLVE_H */
