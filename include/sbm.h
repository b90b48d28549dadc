/*
 * sbm.h -- C ABI of the GB300 matrix-free shifted boundary method (SBM) operator.
 *
 * The library evaluates y = A x for the SBM discretisation of the Poisson
 * problem -Lap u = f in Omega, u = g on Gamma (paper, Section 2) on a
 * Cartesian background mesh of [-1,1]^d, with tensor-product Q_p elements,
 * in a continuous Galerkin (CG) or symmetric interior penalty discontinuous
 * Galerkin (DG) form, matrix-free (Section 3, Algorithms 1-3).
 *
 * Conventions for every entry point:
 *  - Every function returns an int status (SBM_OK = 0 or an SBM_ERR_* code);
 *    no C++ exception crosses this boundary.  sbm_error_string() names a code;
 *    sbm_last_error_detail() gives a message for the calling thread's last error.
 *  - The library owns all set-up data (host and device) of an sbm_problem and
 *    frees it in sbm_destroy().  The caller owns every vector argument (x, y,
 *    b, diag, ...) and the CUDA stream.  "device" pointers are CUDA device
 *    (or managed) memory on the current device; "host" pointers are ordinary
 *    CPU memory (pinned memory gives faster copies but is not required).
 *  - Device work is enqueued on the given stream (a cudaStream_t passed as
 *    void*; NULL = the legacy default stream) and is asynchronous unless the
 *    entry point says otherwise.
 *  - Vectors are in the problem's global DoF order:
 *      CG: nodes of the global Gauss-Lobatto lattice ((pN+1)^d nodes, axis 0
 *          fastest) that belong to an active cell, in increasing lattice order;
 *      DG: active cells in lexicographic order (axis 0 fastest), (p+1)^d
 *          values each, local lexicographic order inside a cell.
 *  - Thread safety: distinct problems may be used from different threads;
 *    one problem must not be used by two threads at once, and two applies of
 *    one problem must not run concurrently on different streams (they share
 *    the problem's per-face scratch buffer).
 */
#ifndef SBM_H
#define SBM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
enum {
  SBM_OK = 0,
  SBM_ERR_ARG = 1,            /* invalid argument (null pointer, size, degree, ...) */
  SBM_ERR_OOM = 2,            /* host or device allocation failed */
  SBM_ERR_CUDA = 3,           /* a CUDA runtime call or kernel launch failed */
  SBM_ERR_EMPTY_DOMAIN = 4,   /* no active cell: the true domain misses every cell centre */
  SBM_ERR_NOT_CONVERGED = 5,  /* iterative solver hit maxit (last iterate is still written) */
  SBM_ERR_TIMEOUT = 6,        /* a bounded device-side wait expired */
  SBM_ERR_STATE = 7,          /* call not valid in the problem's current state */
  SBM_ERR_UNSUPPORTED = 8,    /* combination not built (e.g. degree > 6) */
  SBM_ERR_GEOMETRY = 9        /* closest-point projection failed for a surrogate point */
};

/* ---- problem description ------------------------------------------------ */
enum {
  SBM_GEOM_BALL = 0,
  SBM_GEOM_ELLIPSOID = 1,
  SBM_GEOM_TORUS = 2,
  SBM_GEOM_BOX = 3,
  SBM_GEOM_BALLS = 4
};

/*
 * Geometry parameters (geom[]), d = dim:
 *   BALL      : centre c[d], radius r                 phi = |x - c| - r
 *   ELLIPSOID : semi-axes a[d], rotation R[d*d] (row-major, x = c + R y with
 *               y in the ellipsoid's frame), centre c[d]
 *                                                     phi = sum (y_i/a_i)^2 - 1
 *   TORUS     : major radius R, minor radius r (d = 3, axis z, centred at 0)
 *                                                     phi = (sqrt(x^2+y^2)-R)^2 + z^2 - r^2
 *   BOX       : centre c[d], half-widths b[d]        phi = max_i |x_i - c_i| - b_i
 *   BALLS     : the union of nballs balls given in balls[] (not geom[]), the
 *               multiple-ball benchmark of Section 4.3
 *                                                     phi = min_i |x - c_i| - r_i
 *               closest point on the union's boundary: the nearest of the
 *               projections onto each sphere, the nearest points of the
 *               pairwise intersection circles (3D) and the vertices where
 *               three spheres (3D) or two circles (2D) meet, keeping only
 *               candidates not strictly inside another ball; ties go to the
 *               first candidate in that order.
 * A background cell is active iff phi(cell centre) < 0 (strictly), unless
 * the volume-fraction criterion is chosen (activity, below).
 * Penalties: CG sigma = pen_shift * p^2 / h; DG surrogate faces
 * sigma = pen_shift * (p+1)^2 / h and interior faces
 * sigma_F = pen_interior * (p+1)^2 / h; h = 2 / cells_per_side.
 */
typedef struct {
  int dim;              /* 2 or 3 */
  int degree;           /* p, 1..6 */
  int cells_per_side;   /* N >= 1; the mesh is N^d cells of [-1,1]^d */
  int dg;               /* 0 = continuous Galerkin, 1 = SIPG discontinuous Galerkin */
  int geom_kind;        /* SBM_GEOM_* */
  double geom[16];      /* geometry parameters, see above */
  double pen_shift;     /* C in sigma = C p^2/h (CG) or C (p+1)^2/h (DG); paper leaves it open */
  double pen_interior;  /* C_F in sigma_F = C_F (p+1)^2/h (DG interior faces) */
  int extension;        /* SBM_EXT_*: the extension operator E of the shifted terms */
  int nballs;           /* SBM_GEOM_BALLS: number of balls (geom[] unused) */
  const double* balls;  /* SBM_GEOM_BALLS: host [nballs][dim + 1] centre, radius; copied */
  int activity;         /* SBM_ACTIVE_*: which background cells form the surrogate domain */
  double vf_threshold;  /* SBM_ACTIVE_VOLUME: minimum volume fraction, in (0, 1] */
} sbm_desc;

/*
 * Active cells (Section 2: "lying entirely within Omega or intersecting it
 * significantly, based on a chosen criterion, e.g. volume fraction"):
 *   SBM_ACTIVE_CENTRE  phi(cell centre) < 0 (strictly);
 *   SBM_ACTIVE_VOLUME  the volume fraction of Omega in the cell, estimated
 *                      by the midpoint rule on 8^d sub-cells (the share of
 *                      sub-cell midpoints with phi < 0), is >= vf_threshold.
 */
enum { SBM_ACTIVE_CENTRE = 0, SBM_ACTIVE_VOLUME = 1 };

/*
 * Extension operator E u_h(x~) on the surrogate boundary (Section 2.1, the
 * Taylor expansion of u about x~ evaluated at the true-boundary point x):
 *   SBM_EXT_EXACT   the whole series for the discrete polynomial: cell K's
 *                   polynomial evaluated at x_q (O((p+1)^(2d-1)) per face);
 *   SBM_EXT_TAYLOR1 truncated after the gradient term:
 *                   u_h(x~_q) + d_q . grad u_h(x~_q), d_q = x_q - x~_q
 *                   (sum-factorised, O(d (p+1)^d) per face; exact for affine u).
 */
enum { SBM_EXT_EXACT = 0, SBM_EXT_TAYLOR1 = 1 };

typedef struct sbm_problem sbm_problem;

/*
 * Build a problem on the host, in FP64: active cells and surrogate faces
 * (Section 2), the closest points on Gamma of the surrogate-face Gauss points
 * and their reference coordinates in the owning cell's frame (Sections 2.1
 * and 3.4), and the global DoF numbering.  No CUDA call is made (this works
 * without a GPU).  *out receives the handle (NULL on error).
 * Errors: SBM_ERR_ARG (bad desc), SBM_ERR_UNSUPPORTED (degree/dim),
 * SBM_ERR_EMPTY_DOMAIN, SBM_ERR_GEOMETRY, SBM_ERR_OOM.
 */
int sbm_create(const sbm_desc* desc, sbm_problem** out);

/*
 * Build the precomputed operator data (Section 3.4: per surrogate-face
 * quadrature point, the 1D basis values at the shifted point's reference
 * coordinates; the cell order and DoF line table the kernels use) and upload
 * it to the current CUDA device, synchronously.  Must be called once before
 * any apply/diagonal/solve call; the problem is then bound to that device.
 * Errors: SBM_ERR_STATE (called twice), SBM_ERR_OOM, SBM_ERR_CUDA.
 */
int sbm_setup_face_data(sbm_problem* prob);

/*
 * sbm_create with the geometry stage on GPU `device` (the operator
 * initialisation of Section 4.4): active-cell marking, surrogate-face
 * enumeration (deterministic scans), the closest-point projection of every
 * surrogate quadrature point and the CG DoF numbering (lattice marks, scan)
 * run as kernels.  The result is identical, bit for bit, to sbm_create's (the level-set
 * and projection code is shared and compiled without fused multiply-adds).
 * Synchronous; temporary device memory about 16 bytes per background cell,
 * 72 bytes per surrogate quadrature point and (CG) 12 bytes per lattice node
 * of the (pN+1)^d background lattice, freed before returning.
 * Errors: as sbm_create, plus SBM_ERR_ARG (device < 0) and SBM_ERR_CUDA.
 */
int sbm_create_gpu(const sbm_desc* desc, int device, sbm_problem** out);

/* Free every host and device resource of the problem (NULL is ignored).
 * The caller must make sure no work that uses the problem is still running. */
void sbm_destroy(sbm_problem* prob);

/* Sizes: global DoFs, active cells, surrogate faces, DG interior faces
 * (0 for CG).  Any output pointer may be NULL. */
int sbm_sizes(const sbm_problem* prob, int64_t* n_dofs, int64_t* n_cells,
              int64_t* n_sfaces, int64_t* n_ifaces);

/*
 * Copy the geometry to host buffers (for tests and diagnostics; any may be
 * NULL):
 *   cells  [n_cells * dim]         int32 cell multi-indices, lexicographic order
 *   sfaces [n_sfaces * 3]          int32 (active-cell rank, normal axis k, side s)
 *                                  per surrogate face; outward normal (2s-1) e_k;
 *                                  order: by cell, then k, then s
 *   face_x [n_sfaces * Q * dim]    double closest points x_q on Gamma of the
 *                                  face Gauss points, Q = (p+1)^(d-1), first
 *                                  tangential index fastest
 */
int sbm_export_geometry(const sbm_problem* prob, int32_t* cells, int32_t* sfaces,
                        double* face_x);

/*
 * Matrix-free apply in FP64: y = A x (Section 3.5 workflow; cell term by sum
 * factorisation, Algorithm 1; surrogate faces, Algorithm 3; DG interior
 * faces, Algorithm 2).  x and y are device arrays of n_dofs doubles; they
 * must not overlap.  Atomic-free: repeated calls give bitwise-equal y.
 * Asynchronous on stream.  Errors: SBM_ERR_ARG, SBM_ERR_STATE (no device data),
 * SBM_ERR_CUDA.
 */
int sbm_apply_f64(sbm_problem* prob, const double* x, double* y, void* stream);

/*
 * Same as sbm_apply_f64 with host arrays: copies x to the device, applies,
 * copies y back and synchronises the stream before returning (the path a
 * caller without device buffers takes; the staging buffers are allocated
 * once per problem on first use).  Continuous Galerkin problems run it as a
 * pipeline over slabs of whole cell layers along the last axis: the copy of
 * the next slab's part of x, the current slab's kernels (its faces beside
 * the previous slab's cells) and the copy of the part of y the slab
 * completes overlap, on streams of the problem ordered after the caller's
 * stream.  The result is bitwise that of sbm_apply_f64.  Page-locked host
 * arrays let the copies run concurrently with the kernels; with them the
 * pipeline is captured into a CUDA graph on the first call for a given
 * (x_host, y_host) pair and tile shape and replayed afterwards (the four
 * most recent pairs are kept).  Calls on one problem must not overlap (they
 * share the staging buffers and streams).
 */
int sbm_apply_f64_host(sbm_problem* prob, const double* x_host, double* y_host, void* stream);

/* Face arithmetic of the FP32 apply: FP32 CUDA cores, or the shifted point
 * evaluation on tensor cores in TF32 / BF16 with FP32 accumulation. */
enum { SBM_FACE_FP32 = 0, SBM_FACE_TF32 = 1, SBM_FACE_BF16 = 2 };

/*
 * Matrix-free apply in FP32 (same operator and algorithm as sbm_apply_f64;
 * the 1D tables and the per-face shifted-point tables rounded to FP32):
 * y = A x with x, y device arrays of n_dofs floats.  face_mode selects the
 * arithmetic of the surrogate faces' shifted point evaluation (Algorithm 3's
 * O((p+1)^(2d-1)) step): SBM_FACE_FP32 on the CUDA cores, or SBM_FACE_TF32 /
 * SBM_FACE_BF16 on the tensor cores (tcgen05, FP32 accumulation; 3D only),
 * where the Lagrange values at the shifted points and the cell values are
 * rounded to TF32 / BF16.  Asynchronous on stream.  A tensor-core apply whose
 * bounded wait expired records SBM_ERR_TIMEOUT, reported by
 * sbm_device_status.
 * Errors: SBM_ERR_ARG, SBM_ERR_STATE, SBM_ERR_UNSUPPORTED (tensor-core mode on
 * a 2D problem), SBM_ERR_CUDA.
 */
int sbm_apply_f32(sbm_problem* prob, const float* x, float* y, int face_mode, void* stream);

/*
 * sbm_apply_f64 for callers that cannot allocate device memory when they
 * apply the operator (the paper has no counterpart: this is a library
 * convenience).  Some callers cannot call cudaMalloc at that point -- code
 * that runs while another component captures a CUDA graph into a memory
 * pool, real-time loops whose allocator is frozen after start-up, or host
 * frameworks that only hand out fixed buffers.  This entry point allocates
 * nothing: the apply's scratch (per-face results and per-colour accumulation
 * buffers) lives in one static device array of 64 MiB that every GPU loading
 * the library holds until the process exits.  The problem's set-up data
 * still comes from sbm_setup_face_data; the caller passes x and y (device,
 * n_dofs doubles, not overlapping) as for sbm_apply_f64, and gets the same y.
 * Limits and behaviour:
 *  - continuous Galerkin problems only (SBM_ERR_UNSUPPORTED for DG);
 *  - the scratch needed, 2^d * n_dofs * 8 bytes plus the per-face results,
 *    must fit in 64 MiB (about 1 M DoFs in 3D, 2 M in 2D); larger
 *    problems get SBM_ERR_ARG with the byte counts in sbm_last_error_detail;
 *  - the current device must be the problem's device (SBM_ERR_STATE);
 *  - the first call on a device looks the array's address up
 *    (cudaGetSymbolAddress) with that device current and caches it: make
 *    that first call before any stream capture;
 *  - every call uses the same array: two calls whose work overlaps on the
 *    GPU (different streams, or different problems on one device) race.
 *    Nothing in the array needs clearing between calls.
 * Asynchronous on stream.  Errors: SBM_ERR_ARG, SBM_ERR_STATE,
 * SBM_ERR_UNSUPPORTED, SBM_ERR_CUDA.
 */
int sbm_apply_f64_noalloc(sbm_problem* prob, const double* x, double* y, void* stream);

/*
 * The diagonal of A (FP64, device array of n_dofs), for Jacobi scaling.
 * Asynchronous on stream.
 */
int sbm_diagonal(sbm_problem* prob, double* diag, void* stream);

/* ---- batches of problems ------------------------------------------------ */
typedef struct sbm_batch sbm_batch;

/*
 * A batch of independent continuous Galerkin problems (any sizes, degrees,
 * geometries), each with nrhs right-hand sides, applied together in ONE
 * persistent kernel launch (the paper applies one problem at a time; this
 * batches many).  The launch's blocks
 * stay resident and take work items from a device ticket counter: first
 * the surrogate-face items (ranges of faces, Algorithm 3), then the cell
 * chunk items (ranges of chunks: gather, cell term of Algorithm 1, face
 * folds, single-writer stores; each waits until its system's face items are
 * done), then the assembly items (the DoFs several colours share; each
 * waits for its system's chunk items).  Items are sized and ordered by the
 * paper's load-balancing weights (Section 3.5: 10 per cell, plus 40 per
 * surrogate face in 3D and 20 in 2D), scaled across degrees by the cell's
 * sum-factorisation cost (p+1)^(d+1), heaviest first within each phase.
 * Every dependency wait is bounded: on expiry the kernel records
 * SBM_ERR_TIMEOUT (sbm_batch_device_status) instead of hanging.  The
 * counter reset and the launch are captured into a CUDA graph on the first
 * call for a given set of vector pointers (eight kept per precision) and
 * replayed afterwards.
 * probs: nprob problems, all set up (sbm_setup_face_data) on the current
 * device; the batch keeps the pointers (do not destroy a problem before its
 * batch).  flags: SBM_BATCH_AUTOTUNE runs the autotuner: per precision and
 * per degree it times every combination of the cell kernel's tile shape
 * (chunks of R or R/2 cells, R = 256 / (p+1)^(d-1)), the face batch (256 or
 * 128 threads' worth of faces per pass) and, with SBM_BATCH_TENSOR_CORES,
 * tensor-core faces for the FP32 applies (the shifted point evaluation's
 * first contraction as one TF32 tcgen05.mma per face, FP32 accumulation in
 * tensor memory; 3D, exact extension; this changes the FP32 results to TF32
 * accuracy) on that degree's problems and keeps the fastest
 * (sbm_batch_knobs reports the choice and the timings); without it every
 * degree uses shape 0, the full face batch and CUDA-core faces.  Device scratch: nrhs
 * copies of each problem's per-face results and colour buffers, per
 * precision, allocated on first use (all or nothing).  Synchronous.
 * Errors: SBM_ERR_ARG, SBM_ERR_STATE, SBM_ERR_UNSUPPORTED (DG problem),
 * SBM_ERR_OOM, SBM_ERR_CUDA, SBM_ERR_TIMEOUT (a wait expired while tuning).
 */
enum { SBM_BATCH_AUTOTUNE = 1, SBM_BATCH_TENSOR_CORES = 2 };
int sbm_batch_create(sbm_problem* const* probs, int nprob, int nrhs, int flags,
                     sbm_batch** out);

/*
 * y_k = A_k x_k for every problem k and right-hand side: x[k] and y[k] are
 * device arrays of nrhs * n_dofs_k values (right-hand side r at offset
 * r * n_dofs_k), x[k] != y[k].  The same operator, arithmetic and summation
 * order as sbm_apply_f32 / sbm_apply_f64: bitwise-equal results for the
 * same tile shape.  One graph launch (a counter reset and the persistent
 * kernel) on stream, asynchronous; two batch applies must not overlap
 * (shared scratch and counters).
 */
int sbm_batch_apply_f32(sbm_batch* batch, const float* const* x, float* const* y, void* stream);
int sbm_batch_apply_f64(sbm_batch* batch, const double* const* x, double* const* y,
                        void* stream);

/* Tile shape (0, 1; 3 after the FP32 autotuner chose it) of a problem's
 * cell chunks (the FP32 choice; both precisions after an override);
 * override it for both precisions with 0 or 1 (drops the cached graphs;
 * synchronises the device). */
int sbm_batch_tile_shape(const sbm_batch* batch, int problem, int* variant);
int sbm_batch_set_tile_shape(sbm_batch* batch, int problem, int variant);

/*
 * The autotuner's record for one degree and precision (32 or 64):
 * *tile_shape (0: R cells per chunk, 1: R/2, 3: R cells without staged
 * runs -- FP32 batches of 3D problems), *face_batch (0: 256/L faces per
 * pass, 1: 128/L), *tensor_cores (tensor-core face path on: 1, off: 0);
 * ms[10] (may be NULL): the measured time in ms of that degree's sub-batch
 * for option index tile_shape + 2 face_batch + 4 tensor_cores (tile shapes
 * 0 and 1) or 8 + face_batch (tile shape 3), < 0 where the option was not
 * timed.  Any output may be NULL.
 * Errors: SBM_ERR_ARG (bad precision, no tuned problem of that degree).
 */
int sbm_batch_knobs(const sbm_batch* batch, int precision, int degree, int* tile_shape,
                    int* face_batch, int* tensor_cores, float* ms);

/*
 * Pin the knobs of one degree and precision (32 or 64) instead of the
 * autotuner's choice: tile shape (0, 1, or 3 for FP32 batches of 3D
 * problems), face batch (0, 1), tensor-core faces (0, 1; FP32 batches
 * created with SBM_BATCH_TENSOR_CORES only, not with tile shape 3).
 * Drops the cached graphs; synchronises the device.
 * Errors: SBM_ERR_ARG (bad value, no problem of that degree),
 * SBM_ERR_UNSUPPORTED (tensor cores not allowed, tile shape 3 where it does
 * not run).
 */
int sbm_batch_set_knobs(sbm_batch* batch, int precision, int degree, int tile_shape,
                        int face_batch, int tensor_cores);

/*
 * Synchronise the device and report (then clear) the batch's device error
 * word: SBM_ERR_TIMEOUT if a bounded dependency wait (or a tensor-core MMA's
 * completion wait) of an earlier batched apply expired, SBM_OK otherwise.
 */
int sbm_batch_device_status(sbm_batch* batch);

/*
 * Diagnostic of the persistent kernel's failure path (the paper has no
 * counterpart): one launch whose only work item waits for a dependency that
 * nothing produces; the bounded wait expires (about a second), the kernel
 * records SBM_ERR_TIMEOUT in the batch's error word and returns without
 * touching any vector.  No fault, no hang; the context stays usable.
 * Synchronous on stream.
 */
int sbm_batch_selftest_timeout(sbm_batch* batch, void* stream);

/* Free the batch (not its problems). */
void sbm_batch_destroy(sbm_batch* batch);

enum { SBM_BATCH_SOLVE_FP64 = 0, SBM_BATCH_SOLVE_MIXED = 1 };

/*
 * Solve A_k x = b for every problem k and right-hand side of the batch (the
 * paper states no solver; Section 4.2 notes that the operator application
 * dominates iterative solvers).  Every system runs its own BiCGStab
 * iteration -- its own scalars, residual tests and stopping -- but the
 * iterations advance together: each step applies the whole batch at once
 * (sbm_batch_apply_*) and runs every vector operation as one launch over all
 * systems, with per-system deterministic reductions (bitwise-reproducible
 * results); systems that have finished stop updating.
 *  mode SBM_BATCH_SOLVE_FP64: BiCGStab with FP64 applies from x = 0 to
 *    |b - A x| <= rtol |b| per system, at most maxit iterations (restarted
 *    from the best iterate after a breakdown, up to 20 times).
 *  mode SBM_BATCH_SOLVE_MIXED: FP64 iterative refinement: r = b - A x in
 *    FP64, an inner BiCGStab with FP64 vectors and FP32 applies for A d = r
 *    to inner_rtol |r| or inner_maxit iterations, x += d where the inner
 *    solve reduced its residual; a system leaves the refinement once its
 *    residual no longer halves per step; at most maxit refinements; systems
 *    above rtol then finish with the FP64 BiCGStab from their current x
 *    (at most min(20000, maxit * inner_maxit) iterations).
 * b[k], x[k]: device arrays of nrhs * n_dofs_k doubles, laid out as for
 * sbm_batch_apply (x is output only; the solve starts from 0).
 * iters[k * nrhs + r] (optional, host): BiCGStab iterations of that system
 * (two applies each; inner and finishing ones summed); relres[k * nrhs + r]
 * (optional, host): true relative residual |b - A x| / |b| in FP64 at exit;
 * outer (optional): refinement steps taken.  Device workspace: 11 FP64 and
 * 2 FP32 vectors of the batch's total length, allocated on first use and
 * kept with the batch.  Synchronous on stream.
 * Errors: SBM_ERR_ARG, SBM_ERR_STATE (other device), SBM_ERR_OOM,
 * SBM_ERR_CUDA, SBM_ERR_NOT_CONVERGED (a system above rtol; x holds the
 * last iterates and relres says which).
 */
int sbm_batch_solve(sbm_batch* batch, const double* const* b, double* const* x, int mode,
                    double rtol, int maxit, double inner_rtol, int inner_maxit, int* iters,
                    double* relres, int* outer, void* stream);

/* ---- solvers (the paper gives none; these drive the operator) ----------- */
enum { SBM_PRECOND_NONE = 0, SBM_PRECOND_JACOBI = 1 };

/*
 * Conjugate gradients on A x = b in FP64 (optionally Jacobi-preconditioned),
 * all vectors on the device, CUDA-graph-captured iterations, deterministic
 * reductions.  x (device, n_dofs) holds the initial guess on entry and the
 * last iterate on exit.  Stops when the true relative residual
 * |b - A x| / |b| <= rtol (checked after the recursive residual reaches it,
 * restarting if the two disagree), or after maxit iterations.  CG assumes a
 * symmetric positive definite A; the SBM operator is not symmetric when the
 * shift is non-zero, and CG can diverge on it: that ends the solve with
 * SBM_ERR_NOT_CONVERGED.  *iters and *relres (may be NULL) receive the
 * iteration count and the final true relative residual in every case.
 * Synchronous: returns after the solve (work runs on stream).
 * Errors: SBM_ERR_ARG, SBM_ERR_STATE, SBM_ERR_NOT_CONVERGED, SBM_ERR_CUDA.
 */
int sbm_cg(sbm_problem* prob, const double* b, double* x, double rtol, int maxit, int precond,
           int* iters, double* relres, void* stream);

/*
 * Restarted GMRES(restart) on A x = b in FP64 (no preconditioner; CGS2
 * orthogonalisation), the nonsymmetric counterpart of sbm_cg with the same
 * conventions; maxit counts operator applications inside Arnoldi steps.
 * Device workspace: (restart + 1) vectors of n_dofs doubles, allocated and
 * freed by the call.
 */
int sbm_gmres(sbm_problem* prob, const double* b, double* x, double rtol, int maxit, int restart,
              int* iters, double* relres, void* stream);

/*
 * BiCGStab (van der Vorst's stabilised bi-conjugate gradients) on A x = b,
 * for the nonsymmetric SBM operator (no preconditioner: the SBM diagonal has
 * negative entries near the surrogate boundary, and Jacobi scaling turns the
 * spectrum indefinite): two operator applications per
 * iteration, every scalar in FP64 on the device, BI_CHUNK = 8 iterations per
 * CUDA-graph launch, deterministic reductions.  sbm_bicgstab works on FP64
 * vectors with the FP64 apply; sbm_bicgstab_f32 on FP32 vectors with the
 * FP32 apply (face arithmetic face_mode, as in sbm_apply_f32) and FP64
 * scalars.  Same conventions as sbm_cg (x = initial guess in, iterate out;
 * true-residual stop test; device vectors of n_dofs).  A recursive residual
 * that the true one does not confirm restarts from the current iterate; a
 * breakdown, divergence or the iteration cap continues (or ends) from the
 * iterate of least recursive residual seen at a chunk end (at most 50
 * restarts).  *iters counts iterations, maxit
 * bounds them.  Device workspace: 7 vectors of n_dofs, allocated and freed
 * by the call.
 * Errors: SBM_ERR_ARG, SBM_ERR_STATE, SBM_ERR_UNSUPPORTED (tensor-core face
 * mode on a 2D problem), SBM_ERR_NOT_CONVERGED, SBM_ERR_CUDA.
 */
int sbm_bicgstab(sbm_problem* prob, const double* b, double* x, double rtol, int maxit,
                 int* iters, double* relres, void* stream);
int sbm_bicgstab_f32(sbm_problem* prob, const float* b, float* x, double rtol, int maxit,
                     int face_mode, int* iters, double* relres, void* stream);

/*
 * Inner solver of the mixed-precision refinement: GMRES(restart) or BiCGStab
 * on FP32 vectors, or BiCGStab on FP64 vectors and scalars whose operator
 * applications alone run in FP32 (the vector converted to FP32 before and the
 * result back to FP64 after each one).
 */
enum { SBM_INNER_GMRES = 0, SBM_INNER_BICGSTAB = 1, SBM_INNER_BICGSTAB_MIXED = 2 };

/*
 * Mixed precision: FP64 iterative refinement (defect correction).  Each
 * outer step computes r = b - A x with the FP64 apply, then solves
 * A c = r/|r| approximately in FP32 on the FP32 apply (face arithmetic
 * face_mode, as in sbm_apply_f32) with the inner solver inner_solver:
 * GMRES(restart), or BiCGStab (restart unused) (relative tolerance
 * inner_rtol, at most inner_maxit iterations), and updates x += |r| c in
 * FP64.  Stops when |b - A x|/|b| <= rtol (FP64).  If the refinement stalls
 * first (an inner solve without progress, or max_outer steps spent) -- the
 * FP32 operator's rounding, about condition number x 6e-8 of |b|, limits what
 * an inner solve can reach -- FP64 BiCGStab continues from x to rtol (at most
 * min(20000, max_outer * inner_maxit) iterations; counted as one more outer
 * step).  *iters = inner
 * iterations in total, including that finish (a BiCGStab iteration applies
 * the operator twice), *outer = outer steps; same conventions otherwise.
 */
int sbm_solve_ir(sbm_problem* prob, const double* b, double* x, double rtol, int max_outer,
                 int restart, double inner_rtol, int inner_maxit, int face_mode,
                 int inner_solver, int* iters, int* outer, double* relres, void* stream);

/*
 * BiCGStab with FP64 vectors and scalars whose iterations apply the FP32
 * operator (sbm_apply_f32 with face_mode, converted in and out), with
 * reliable updates: whenever the recursive residual has fallen tenfold since
 * the last update it is replaced by the true residual b - A x computed with
 * the FP64 operator (sbm_apply_f64), so the iteration keeps its Krylov space
 * (no restart) while converging to the FP64 solution; the initial and final
 * residuals are FP64.  A breakdown restarts from the best iterate, as
 * sbm_bicgstab.  When the true residual stops halving between updates (the
 * FP32 operator's rounding limits the corrections on ill-conditioned
 * systems) FP64 BiCGStab finishes from the current x within the remaining
 * iteration budget.  b, x: device arrays of n_dofs doubles (x: initial guess
 * in, solution out).  iters: iterations (two applies each, FP32 then FP64);
 * replacements: reliable updates (one FP64 apply each); relres: true FP64
 * relative residual at exit.  Synchronous.  Errors: as sbm_bicgstab, plus
 * those of the face mode (SBM_ERR_ARG, SBM_ERR_UNSUPPORTED).
 */
int sbm_bicgstab_mixed(sbm_problem* prob, const double* b, double* x, double rtol, int maxit,
                       int face_mode, int* iters, int* replacements, double* relres,
                       void* stream);

/*
 * Manufactured data (host, FP64; no CUDA call).  manufactured = 0:
 * u = prod_i sin(pi x_i), f = d pi^2 u; manufactured = 1 (2D only):
 * u = 2 cos(x_1) sin(x_2), f = 2 u (the paper's Appendix A solution).
 * sbm_rhs writes the right-hand side of the weak form (Section 2.1)
 *   b_i = int f v_i - int_F (grad v_i . n~) g(x_q) + int_F sigma g(x_q) v_i
 * with g = u at the true-boundary points x_q; sbm_interpolate writes the
 * nodal interpolant of u.  Both fill host arrays of n_dofs doubles.
 * Errors: SBM_ERR_ARG (NULL, unknown id).
 */
int sbm_rhs(const sbm_problem* prob, int manufactured, double* b_host);
/* The same right-hand side into a device array b (n_dofs doubles) on
 * stream: assembled on the host in FP64 as sbm_rhs, then copied (the call
 * returns once the host data is staged).  Errors: SBM_ERR_ARG, SBM_ERR_STATE
 * (no device data), SBM_ERR_CUDA. */
int sbm_rhs_device(const sbm_problem* prob, int manufactured, double* b, void* stream);
int sbm_interpolate(const sbm_problem* prob, int manufactured, double* u_host);

/*
 * Kernel timing (diagnostics).  While enabled, every sbm_apply_f64 /
 * sbm_apply_f32 records CUDA events on its stream at the boundaries of its
 * three phases: the surrogate-face kernel, the cell kernel (the DG kernel
 * for DG), and the assembly of the colour buffers (none for DG).
 * sbm_profile_read waits for the recorded events and returns, summed over
 * the applies since the previous read, the milliseconds of each phase in
 * phase_ms[0..2] (face, cell, assembly) and the number of kernel launches,
 * then resets.  Either output may be NULL.  Enabling adds four event records
 * per apply and nothing else.
 */
int sbm_profile_enable(sbm_problem* prob, int on);
int sbm_profile_read(sbm_problem* prob, double* phase_ms, int64_t* launches);

/*
 * Synchronise the device and report (then clear) the problem's device error
 * word: SBM_ERR_TIMEOUT if a bounded device-side wait of an earlier call
 * expired, SBM_OK otherwise.
 */
int sbm_device_status(sbm_problem* prob);

/*
 * Tile-shape autotuner for the single applies (continuous Galerkin; a no-op
 * for DG): times, in FP64 and in FP32, on this problem (temporary device
 * buffers of n_dofs doubles, freed before returning) the cell term's tile
 * shapes and keeps the faster per precision:
 *   0  chunks of R consecutive cells of a mesh row (R (p+1)^(d-1) threads),
 *      x-line runs staged in shared memory;
 *   1  chunks of R/2 cells;
 *   2  (3D; FP32 p <= 4, FP64 p <= 3) the cells of shape 0's chunks, one
 *      thread per cell with the tile in registers;
 *   3  (3D) shape 0's chunks without staged runs: each thread loads and
 *      stores its own lines.
 * and for shapes 0 and 3 each way of completing the DoFs several chunk
 * colours share (see sbm_set_ordered_stores).  All compute the same
 * operator; shapes 0, 2 and 3 give bitwise-equal results with either store
 * mode, shape 1 differs in the rounding of the few shared nodes it sums in
 * the assembly instead of in shared memory.  *shape64 / *shape32 (may be
 * NULL) receive the shape choices, sbm_ordered_stores the store modes.
 * Synchronous, legacy default stream.
 */
int sbm_autotune(sbm_problem* prob, int* shape64, int* shape32);

/*
 * Pin the tile shapes of the single applies instead (0..3 as for
 * sbm_autotune; -1 keeps the current one), e.g. to reproduce a run bitwise.
 * DG problems accept only 0 or -1.
 * Errors: SBM_ERR_ARG (NULL, shape outside -1..3), SBM_ERR_STATE,
 * SBM_ERR_UNSUPPORTED (a shape the problem's dimension, degree or
 * discretisation does not have).
 */
int sbm_set_tile_shape(sbm_problem* prob, int shape64, int shape32);

/*
 * How the single applies (continuous Galerkin, tile shapes 0 and 3, one
 * right-hand side, device buffers) complete the DoFs that chunks of several
 * colours share -- the scatter of Algorithm 1's cell results (and the face
 * terms of Algorithm 3 folded into them) into the global vector:
 *   0  every chunk stores such DoFs into its colour's buffer
 *      ([2^d][n_dofs] scratch) and an assembly pass sums the buffers in
 *      colour order;
 *   1  colour-ordered stores: one persistent launch takes the chunks in
 *      ascending colour order from a ticket counter; the lowest colour's
 *      chunk stores a shared DoF, each higher colour's chunk reads, adds and
 *      stores it after a bounded wait for its lower-colour neighbours (per-
 *      chunk completion counts), so y receives the same sums in the same
 *      order as with 0, bitwise, without the colour buffers' traffic or the
 *      assembly launch.  An expired wait records SBM_ERR_TIMEOUT
 *      (sbm_device_status).  The host-buffer pipeline, shapes 1 and 2 and
 *      multi-RHS launches always use 0.
 * -1 keeps the current mode; the default is 0 until sbm_autotune chooses.
 * Two applies of one problem must not run concurrently in mode 1 (they
 * share its counters), as in mode 0 they share its colour buffers.
 * Errors: SBM_ERR_ARG (NULL, mode outside -1..1), SBM_ERR_STATE,
 * SBM_ERR_UNSUPPORTED (1 where the tables were not built: DG, or a chunk
 * with more than 64 lower-colour neighbours).
 */
int sbm_set_ordered_stores(sbm_problem* prob, int ordered64, int ordered32);
/* The current store modes (0 or 1) of the FP64 and FP32 applies (either
 * pointer may be NULL).  Errors: SBM_ERR_ARG (prob NULL). */
int sbm_ordered_stores(const sbm_problem* prob, int* ordered64, int* ordered32);

/*
 * Diagnostic of the failure path (the paper has no counterpart): enqueue one
 * device-side bounded wait on a barrier that nothing releases.  The wait
 * gives up after a fixed number of polls (well under a second), records
 * SBM_ERR_TIMEOUT in the problem's device error word and returns; the next
 * sbm_device_status reports it.  No fault, no hang; the context stays usable.
 */
int sbm_selftest_timeout(sbm_problem* prob, void* stream);

/* ---- measurement aids ---------------------------------------------------- */

/*
 * Fused multiply-add throughput of the current GPU (a measurement aid for
 * the roofline of the cell kernels; the paper has no counterpart): a kernel
 * of independent fma.rn chains (8 per thread, 8 blocks of 256 threads per
 * SM), timed with CUDA events on stream (best of five launches after a
 * warm-up).  *gfma_per_s receives G FMA thread-operations per second
 * (x 2 = GFLOP/s).  precision: 64 (double) or 32 (float).  Synchronous;
 * about 0.1 s.  Errors: SBM_ERR_ARG, SBM_ERR_CUDA.
 */
int sbm_peak_probe(int precision, double* gfma_per_s, void* stream);

/* ---- seeded inputs ------------------------------------------------------- */
enum { SBM_DIST_UNIFORM = 0, SBM_DIST_NORMAL = 1 };

/*
 * The input generator of the benchmark workloads ("x ~ U(-1,1) from seed s";
 * the paper names no generator, so this is the library's convention), for C
 * callers that want the same vectors as the Python workload descriptions.
 * Counter-based splitmix64 (Steele, Lea, Flood, OOPSLA 2014): value k of
 * stream `seed` is the splitmix64 finaliser of seed + (k+1) * 0x9E3779B97F4A7C15
 * (mod 2^64); u_k = (value >> 11) * 2^-53 in [0, 1).
 *   SBM_DIST_UNIFORM  out[i] = 2 u_{offset+i} - 1                      (U(-1,1))
 *   SBM_DIST_NORMAL   out[i] = sqrt(-2 log1p(-u_2j)) cos(2 pi u_2j+1), j = offset+i
 *                     (Box--Muller, cosine branch; N(0,1))
 * out_host: n doubles of host memory, written in order (a problem's vector
 * is filled in its global DoF order).  Host only, synchronous, no CUDA call;
 * uses the C library's log1p and cos, compiled without fused multiply-adds.
 * Errors: SBM_ERR_ARG (n < 0, NULL output with n > 0, unknown dist).
 */
int sbm_fill_random(int64_t n, uint64_t seed, uint64_t offset, int dist, double* out_host);

/* Human-readable name of a status code (static string). */
const char* sbm_error_string(int status);

/* Detail message of the calling thread's most recent failed call ("" if none). */
const char* sbm_last_error_detail(void);

#ifdef __cplusplus
}
#endif

#endif /* SBM_H */
