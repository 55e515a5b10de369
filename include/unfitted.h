/*
 * unfitted.h - C ABI of the GB300 matrix-free unfitted DG Poisson operator.
 *
 * The operator is the one of arXiv 2404.07911, Sec. 2.1 (Eq. bilinear_cg, Eq. bilinear_dg):
 * a discontinuous Galerkin SIPG discretisation of -Lap u = f on Omega = {phi < 0} embedded in a
 * Cartesian background grid, with the Dirichlet condition on Gamma imposed by Nitsche's method,
 * stabilised by the face-based ghost penalty (Sec. 2.2) on jumps of normal derivatives of
 * orders 1..J across every face of a cut cell, and an optional per-cell diffusion coefficient
 * kappa that multiplies every term linearly (arithmetic face average {kappa} on face terms).
 * Shape functions are tensor-product Lagrange polynomials of degree p in the Gauss-Lobatto
 * points (Sec. 3.2); inside cells and full faces are integrated with structured (tensor Gauss)
 * quadrature, cut cells, Gamma and cut faces with unstructured dimension-reduction quadrature
 * generated once at creation (Sec. 2.3).
 *
 * DoF layout of every vector (x, y, g): active cells (inside + cut) numbered lexicographically
 * over the background grid with the x index fastest; active cell e owns the contiguous block
 * [e * n^d, (e + 1) * n^d), local index l = i + n j + n^2 k (n = p + 1), Sec. 3.2.
 *
 * Conventions for every call:
 *   - Return value: UF_OK or an error code; errors never abort the process.  uf_last_error()
 *     returns a thread-local message describing the last failure of the calling thread.
 *   - Device pointers refer to memory of the operator's CUDA device; the caller owns them.
 *   - `stream` is a cudaStream_t passed as void* (NULL = the legacy default stream).  Stream-
 *     ordered calls return once the work is enqueued; they never allocate and never synchronise.
 */
#ifndef UNFITTED_H
#define UNFITTED_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct uf_operator uf_operator; /* opaque, owned by the library */

typedef enum {
  UF_OK = 0,
  UF_EINVAL = 1,        /* invalid argument (NULL pointer, bad size, aliasing, bad parameter) */
  UF_ENOMEM = 2,        /* host or device allocation failed during creation */
  UF_ECUDA = 3,         /* a CUDA runtime call failed (message in uf_last_error) */
  UF_EUNSUPPORTED = 4,  /* valid but not supported (e.g. anisotropic grid, degree > 8) */
  UF_EGEOMETRY = 5,     /* quadrature generation failed (subdivision depth exceeded) */
  UF_ENODEVICE = 6      /* the operator was created host-only (device = -1) */
} uf_status;

enum { UF_FP64 = 1, UF_FP32 = 2 };     /* precision flags (bit mask in uf_params.precisions) */
enum { UF_LS_SPHERE = 0, UF_LS_PLANE = 1, UF_LS_SPHERES = 2 };  /* level set kinds */
enum { UF_DG = 0, UF_CG = 1 };         /* discretizations (uf_params.discretization) */
enum { UF_GP_FACE = 0, UF_GP_VOLUME = 1 }; /* ghost penalties (uf_params.gp_kind) */

/* Parameters of uf_create_unfitted_operator.  Penalties follow the paper's forms:
 * SIPG penalty sigma/h (Eq. bilinear_dg), Nitsche penalty tau/h (Eq. bilinear_cg), ghost
 * penalty gamma_j = gp_gamma * h^(2j-1) / (j!)^2 on [d^j u / dn^j], j = 1..gp_max_order. */
typedef struct {
  int dim;                /* 2 or 3 */
  int degree;             /* polynomial degree p, 1..8 */
  int n_cells[3];         /* background cells per direction (entries >= dim ignored) */
  double lo[3], hi[3];    /* background box; cells must be cubes (isotropic h) */
  int ls_kind;            /* UF_LS_SPHERE: phi(x) = |x - ls_center| - ls_radius;
                             UF_LS_PLANE: phi(x) = ls_normal . x - ls_offset (fields at the end) */
  double ls_center[3];
  double ls_radius;
  int quad_order;         /* q: Gauss points per interval of the cut-cell / cut-face rules */
  double sipg_gamma;      /* sigma */
  double nitsche_gamma;   /* tau */
  int gp_max_order;       /* J (0 disables the ghost penalty), <= degree */
  double gp_gamma;
  int precisions;         /* UF_FP64 | UF_FP32: which device data to build */
  int device;             /* CUDA device ordinal, or -1 for a host-only operator (no GPU use) */
  const double *kappa;    /* host array [n_active] copied at creation, or NULL for kappa = 1 */
  int discretization;     /* UF_DG: SIPG (Eq. bilinear_dg), DoFs per cell; UF_CG: continuous Q_p
                             (Eq. bilinear_cg, no SIPG), DoFs on the Gauss-Lobatto lattice points of
                             the active cells numbered lexicographically (x fastest) */
  double ls_normal[3];    /* UF_LS_PLANE: normal (any length > 0; entries >= dim ignored) */
  double ls_offset;       /* UF_LS_PLANE: the domain is ls_normal . x < ls_offset */
  int gp_kind;            /* UF_GP_FACE: sum_j gamma_j {kappa} int_F [d^j u/dn^j][d^j v/dn^j] on every
                             face of a cut cell; UF_GP_VOLUME: gp_tau / h^2 {kappa} int_P [u]_P [v]_P on
                             stable-neighbour patches P (paper Sec. 2.2, Eq. volume_based_gp): every
                             cut cell with its active face neighbour of largest volume fraction, [u]_P
                             the own polynomial minus the neighbour's extended one (Sec. 3.3).  Either
                             is off when gp_max_order = 0. */
  double gp_tau;          /* tau_v of UF_GP_VOLUME */
  const double *ls_spheres;  /* UF_LS_SPHERES: host array [ls_n_spheres][4] = (cx, cy, cz, R), copied
                                at creation; the domain is the union of the balls, level set
                                min_i (|x - c_i| - R_i) (paper Sec. 6).  Balls may intersect: a cell
                                or face met by several spheres gets a rule split at their
                                intersection circles; a cell inside the union but inside no single
                                ball is a cut cell with a full volume rule and no surface points */
  int ls_n_spheres;
} uf_params;

/* Sizes and algorithmic traffic of an operator (uf_get_info). */
typedef struct {
  int64_t n_active, n_inside, n_cut, n_dofs;
  int64_t n_faces, n_faces_full, n_faces_cut, n_faces_empty, n_faces_gp;
  int64_t n_vol_points, n_surf_points, n_face_points; /* unstructured points (face: unique) */
  int64_t n_vol_lines, n_face_lines;  /* lines of the dimension-reduction rules (face: per side) */
  int32_t dim, degree, dofs_per_cell, quad_order;
  double h;
  /* Algorithmic bytes of one vmult: read x once, write y once, read the per-cell metadata and
   * the unstructured point data once (per point: coordinate along its line and weight, plus the
   * surface normal; per line: two outer coordinates and offsets), FP64 and FP32 data. */
  double bytes_fp64, bytes_fp32;
  /* Algorithmic floating-point operations of one vmult (FMA = 2) from the paper's arithmetic
   * complexity model (Sec. 5.1: structured cell 6 k^4, structured face 7 k^3, unstructured cell
   * point 2 k^3 + 3 k^2 + 4 k, unstructured face point 3 k^2 + 4 k plus k^3 per face side, each
   * for evaluation and again for integration, k = p + 1) applied to this operator's inside cells,
   * structured faces, ghost-penalty orders, and unstructured points. */
  double flops;
  /* Per kernel (index 0 = structured terms of all cells, 1 = unstructured terms of cut cells):
   * algorithmic bytes for FP64 / FP32 data and algorithmic floating-point operations (model
   * above) of one launch, and the floating-point operations the kernels execute as built: the
   * FP64 kernels read the 1D basis at lines and points from tables, the FP32 kernels evaluate
   * it (kernel_flops_built_fp32).  In 3D with k <= 4 the FP64 cut-cell kernel applies each cut
   * face's k^2 x k^2 mass matrix instead of the face's points: its bytes count those matrices
   * (k^4 values per cut cell and cut face) and its operations two products per face. */
  double kernel_bytes_fp64[2], kernel_bytes_fp32[2], kernel_flops[2], kernel_flops_built[2];
  double kernel_flops_built_fp32[2];
  /* Groups of volume lines (3D): lines of a cut cell along one axis that share one outer
   * coordinate; the cut-cell kernel contracts along that coordinate once per group. */
  int64_t n_vol_groups;
  /* Cut cells that the FP64 cut-cell kernel handles with 32, 16 and 8 lanes of a warp (a cell's
   * group is the smallest that holds all its volume lines and all its cut-face lines in one
   * chunk; several small cut cells share a warp), chosen at creation.  The FP32 kernel uses the
   * same classes except that the 16-lane class runs with 32 lanes. */
  int64_t cut_lane_classes[3];
} uf_info;

/* Per-kernel device times collected between uf_profile_begin and uf_profile_end, indexed
 * [precision: 0 = FP64, 1 = FP32][kernel: 0 = structured, 1 = cut cells][0 = vmult, 1 = adjoint]:
 * ms_total sums the bracketed times, launches counts the bracketed evaluations (one per vmult)
 * and kernel_launches the kernel launches inside them (the cut-cell kernel launches once per
 * non-empty lane class). */
typedef struct {
  double ms_total[2][2][2];
  int64_t launches[2][2][2];
  int64_t kernel_launches[2][2][2];
} uf_kernel_times;

/* Build the operator: classify the background cells against the level set, number the active
 * cells, type the interior faces, generate the dimension-reduction quadrature of every cut cell
 * and cut face, and (device >= 0) upload everything to the device in the precisions requested.
 * Untimed setup (the paper excludes it, Sec. 6.2).  On success *out owns all library memory.
 * Errors: UF_EINVAL (NULL, dim/degree/q/sizes out of range), UF_EUNSUPPORTED (anisotropic cells,
 * unknown level set), UF_EGEOMETRY, UF_ENOMEM, UF_ECUDA. */
uf_status uf_create_unfitted_operator(const uf_params *params, uf_operator **out);

/* Fill *info.  Errors: UF_EINVAL on NULL. */
uf_status uf_get_info(const uf_operator *op, uf_info *info);

/* y = A x (paper Eq. operatorevaluation / Eq. matrixfreeopcompact, Sec. 3.1), matrix-free.
 * precision: UF_FP64 (x, y are double[n_dofs]) or UF_FP32 (float[n_dofs]); the operator must
 * have been created with that precision.  x and y are device pointers that must not overlap.
 * Stream-ordered; no allocation, no synchronisation.  Errors: UF_EINVAL, UF_ENODEVICE,
 * UF_ECUDA (launch failure). */
uf_status uf_vmult(uf_operator *op, int precision, void *y, const void *x, void *stream);

/* y = A^T g.  Every term of the form is symmetric, so A^T = A; the adjoint is computed by the
 * transposed cell-centric evaluation (each cell gathers the transposed couplings of its
 * neighbours) and agrees with uf_vmult up to rounding.  Same arguments and errors as uf_vmult. */
uf_status uf_vmult_adjoint(uf_operator *op, int precision, void *y, const void *g, void *stream);

/* End-to-end y = A x with HOST buffers: copies x (host, pinned or pageable) to a library-owned
 * device buffer allocated at creation, applies A, copies y back, and synchronises before
 * returning.  Discontinuous operators with at least 8192 cells run it as a pipeline over 16
 * parts of consecutive cells: x is copied in part by part on a library-owned stream, each part's
 * kernels start on a library-owned stream of its own (earlier parts at higher priority) once x has
 * reached its face neighbours, and its rows of y are copied out on a second library-owned stream
 * while later parts compute (the copies overlap the kernels when the host buffers are pinned);
 * the result equals uf_vmult's bit for bit, and later work on `stream` is ordered after it.  The
 * first call creates the streams (non-blocking) and their events.  Errors as uf_vmult. */
uf_status uf_vmult_host(uf_operator *op, int precision, void *y_host, const void *x_host,
                        void *stream);

/* Same as uf_vmult_host for y = A^T g. */
uf_status uf_vmult_adjoint_host(uf_operator *op, int precision, void *y_host, const void *g_host,
                                void *stream);

/* Asynchronous uf_vmult_host / uf_vmult_adjoint_host: the same copies and kernels, queued after
 * the work already on `stream`, without waiting; y_host holds the result, and x_host / g_host
 * may be changed, after uf_host_wait(op, stream).  Pipelined operators keep two device staging
 * sets per precision and alternate them, so consecutive calls overlap (the copies of one with
 * the kernels of the previous one); a call on a set still in use waits on the device for it.
 * Host buffers must be pinned for the copies to be asynchronous (pageable buffers make the calls
 * block).  Errors as uf_vmult. */
uf_status uf_vmult_host_async(uf_operator *op, int precision, void *y_host, const void *x_host,
                              void *stream);
uf_status uf_vmult_adjoint_host_async(uf_operator *op, int precision, void *y_host,
                                      const void *g_host, void *stream);

/* Waits until every host-buffer product queued on `stream` (and the library's own pipeline
 * streams) has finished, its results on the host.  Errors: UF_EINVAL, UF_ENODEVICE, UF_ECUDA. */
uf_status uf_host_wait(uf_operator *op, void *stream);

/* Kernel timing: uf_profile_begin creates `capacity` pairs of CUDA events (not stream-ordered;
 * call it outside any timed region); every kernel that vmult / vmult_adjoint launches afterwards
 * is bracketed by an event pair recorded on its stream, until the pairs run out.
 * uf_profile_end waits for the recorded events, sums the elapsed times per kernel into *out and
 * releases the events.  Errors: UF_EINVAL (capacity < 1, NULL out, no profiling active),
 * UF_ENODEVICE, UF_ECUDA. */
uf_status uf_profile_begin(uf_operator *op, int capacity);
uf_status uf_profile_end(uf_operator *op, uf_kernel_times *out);

/* The split FP32 operator, y = A x with FP32 device vectors x, y [n_dofs]: the rows of the cells
 * that carry Nitsche or ghost-penalty terms (cut cells and cells with a ghost-penalty face; for
 * UF_CG the cell-local rows before the sum over shared nodes) are evaluated with the FP64
 * kernels on the FP32 input and rounded once to FP32, every other row with the FP32 kernels.
 * With uf_set_split_fraction only the cut cells below a volume fraction (and their face
 * neighbours) are split.  It is the inner operator of UF_SOLVE_IR_SPLIT (paper Sec. 3.6
 * iterative solution; FP64 only where the penalty terms of small cut fractions live).  The FP64 structured kernel runs on the list of split cells, the FP64 cut-cell kernel
 * on every cut cell, and only the split cells and their face neighbours are widened to FP64.
 * The first call builds the cell lists (a device allocation); the call uses the FP64 staging
 * buffers of uf_vmult_host (UF_DG) or the FP64 cell-local vectors (UF_CG), so no other call on
 * the operator may overlap it.
 * Errors: UF_EINVAL (missing precision, overlap), UF_ENODEVICE, UF_ENOMEM, UF_ECUDA. */
uf_status uf_vmult_split(uf_operator *op, float *y, const float *x, void *stream);

/* Which cut cells get FP64 rows in the split operator: those whose volume fraction
 * |K cap Omega| / h^d is below `fraction`, with their active face neighbours (whose rows hold the
 * ghost-penalty couplings to them); fraction >= 1 (the default) takes every cut cell.  The cell
 * lists are rebuilt on the next split call.  Errors: UF_EINVAL (NULL op, fraction <= 0).  (Not
 * in the paper: selects the "tiny cut fractions" of the split precision pattern.) */
uf_status uf_set_split_fraction(uf_operator *op, double fraction);

/* Assembled-matrix baseline (paper Sec. 3.1 / Sec. 5.1, matrix-based evaluation).
 * uf_assemble_csr builds the operator's matrix on the device in CSR form (int64 row offsets
 * [n_dofs + 1], int32 column indices, values in `precision`; columns ascending per row) by
 * applying the FP64 matrix-free operator to distance-2-coloured unit vectors (n^d applications
 * per colour; 7 colours in 3D, 5 in 2D).  Synchronous; allocates the matrix (library-owned) and a
 * temporary n^d x n_dofs FP64 staging block.  Needs the FP64 DG operator.  Errors: UF_EINVAL,
 * UF_ENODEVICE, UF_EUNSUPPORTED (UF_CG operator), UF_ENOMEM (checked against free device memory
 * first), UF_ECUDA.
 * uf_csr_info: nonzeros and algorithmic bytes of one SpMV (values + column indices + row
 * offsets + x + y).  uf_csr_spmv: y = A x with the assembled matrix (device pointers, stream-
 * ordered, one warp per row).  uf_export_csr: host copies (any pointer may be NULL; values as
 * double).  uf_release_csr: frees both precisions' matrices (NULL-safe). */
uf_status uf_assemble_csr(uf_operator *op, int precision);
uf_status uf_csr_info(const uf_operator *op, int precision, int64_t *nnz, double *bytes);
uf_status uf_csr_spmv(uf_operator *op, int precision, void *y, const void *x, void *stream);
uf_status uf_export_csr(const uf_operator *op, int precision, int64_t *row_ptr, int32_t *col,
                        double *val);
uf_status uf_release_csr(uf_operator *op);

/* Gradient of r^T A(kappa) x with respect to the per-cell coefficient (FP64):
 * dk[e] = r^T (dA / dkappa_e) x for every active cell e.  A is linear in kappa, so for the loss
 * J = 1/2 ||A(kappa) x - b||^2 the kappa gradient is this with r = A x - b (and A^T r is the
 * x gradient, uf_vmult_adjoint).  Quadrature-point values of r and x are recomputed, nothing is
 * stored by uf_vmult.  dk [n_active], r and x [n_dofs] are FP64 device pointers; stream-
 * ordered; no allocation (a per-cell partial buffer owned by the operator is overwritten, so
 * calls on one operator must not overlap on different streams).  Needs the FP64 operator.
 * For a UF_CG operator r and x are global vectors and dk_e = (P r)^T A_loc,e (P x) with their
 * cell-local gathers.  Errors: UF_EINVAL, UF_ENODEVICE, UF_ECUDA.  (Not in the paper: the
 * differentiable operator.) */
uf_status uf_kappa_gradient(uf_operator *op, double *dk, const double *r, const double *x,
                            void *stream);

/* uf_kappa_gradient without any device allocation by the library for the call: the per-cell
 * partial buffer is a fixed array in the library's device memory instead of the operator's own.
 * (The paper has no counterpart; this serves callers that cannot allocate device memory, such as
 * applications whose device memory is entirely held by another allocator, e.g. a framework's
 * caching pool, or time-critical loops that cannot accept the device-wide synchronisation that
 * allocation can cause.)  Same arguments, results and errors as uf_kappa_gradient, plus:
 *  - limit: n_active * (1 + 2 dim) <= 2^20 doubles (8 MiB; 149,796 active cells in 3D,
 *    209,715 in 2D); larger operators are rejected with UF_EINVAL and a message;
 *  - the fixed array exists once per device that loads the library and stays allocated until
 *    the process exits; the first call on a device looks up its address (cudaGetSymbolAddress,
 *    with that device current) and caches it, so that first call should come before any stream
 *    capture;
 *  - every call on a device shares the one array and leaves its contents behind: calls whose
 *    kernels overlap on the GPU (different streams, or different operators on one device) race
 *    and must be serialised by the caller;
 *  - for a UF_CG operator the call also gathers r and x into the operator's own cell-local work
 *    vectors, which uf_vmult, uf_vmult_adjoint, uf_kappa_gradient and uf_solve use too: on one
 *    CG operator it must not overlap any of those calls;
 *  - the cached address belongs to the device's current context: after cudaDeviceReset (or a
 *    reset of the primary context) the entry point must not be called again in that process.
 * The call itself performs no cudaMalloc / cudaFree; the operator was allocated at creation. */
uf_status uf_kappa_gradient_noalloc(uf_operator *op, double *dk, const double *r,
                                    const double *x, void *stream);

/* Replace kappa from a DEVICE array [n_active] (FP64), stream-ordered (the FP32 copy is
 * converted on the device); the operator then always takes the general per-cell coefficient
 * path.  The host copy used by uf_get_info is not updated.  Errors: UF_EINVAL, UF_ENODEVICE,
 * UF_ECUDA.  Positivity is the caller's responsibility. */
uf_status uf_set_kappa_device(uf_operator *op, const double *kappa_dev, void *stream);

/* Replace kappa: host array [n_active] of positive values.  Synchronous.  Errors: UF_EINVAL. */
uf_status uf_set_kappa(uf_operator *op, const double *kappa_host);

/* Export (host copies) of the setup product, for checks against an independent implementation.
 * uf_export_cells: type[n_active] (0 inside, 1 cut) and index[n_active * 3] (background
 *   multi-index i, j, k); either pointer may be NULL.
 * uf_export_cut_cell_rule: for the c-th cut cell in active order, kind 0 = volume rule
 *   (xi[count * dim] reference coordinates in [0,1]^d, w[count] physical weights), kind 1 =
 *   surface rule (also normal[count * dim]).  Call with xi == NULL to get *count first.
 * uf_export_cut_face_rule: rule on F cap Omega of the face of active cell e on (axis, side)
 *   (side 0 = lower), in-face reference coordinates eta[count * (dim - 1)] (the other axes in
 *   increasing order) and physical weights; *count = 0 unless the face is a cut face.
 * Errors: UF_EINVAL (index out of range, NULL count). */
uf_status uf_export_cells(const uf_operator *op, int32_t *type, int32_t *index);
/* Per cut cell c (active order), host arrays [n_cut], any may be NULL: volume points, volume
 * lines (points of the dimension-reduction rule that share all but one coordinate), cut-face
 * lines, and the lanes of the cell's class in the FP64 cut-cell kernel (32, 16 or 8; the FP32
 * kernel runs the 16-lane class with 32 lanes).  Errors: UF_EINVAL (NULL op).  (Not in the
 * paper: lets tests pick cells by the kernel's work decomposition.) */
uf_status uf_export_cut_cell_counts(const uf_operator *op, int32_t *vol_points, int32_t *vol_lines,
                                    int32_t *face_lines, int32_t *lanes);
/* The volume lines of cut cell c in the order the cut-cell kernel walks them: by line axis, and
 * within an axis in contiguous groups of lines that share one outer coordinate.  axis[count],
 * group_start[count] (1 for the first line of a group), points[count] (volume points on the
 * line); group_start and points may be NULL.  Call with axis == NULL to get *count first.
 * Errors: UF_EINVAL (index out of range, NULL count). */
uf_status uf_export_cut_cell_lines(const uf_operator *op, int64_t c, int32_t *axis,
                                   int32_t *group_start, int32_t *points, int64_t *count);
uf_status uf_export_cut_cell_rule(const uf_operator *op, int64_t c, int kind, double *xi,
                                  double *w, double *normal, int64_t *count);
uf_status uf_export_cut_face_rule(const uf_operator *op, int64_t e, int axis, int side,
                                  double *eta, double *w, int64_t *count);

/* Continuous (UF_CG) operators: host copies of the global node of every cell-local DoF
 * (l2g[n_active * n^d]), of the load vector for f = 1 (rhs[n_dofs], b_i = int_Omega phi_i; the
 * Dirichlet data is zero) and of the diagonal of A (diag[n_dofs]), all computed at creation in
 * FP64.  Any pointer may be NULL.  Errors: UF_EINVAL (NULL op, not a UF_CG operator). */
uf_status uf_export_cg(const uf_operator *op, int32_t *l2g, double *rhs, double *diag);

/* Solve A x = b with Jacobi-preconditioned CG (the solver of the paper's Sec. 3.6 is a PCG; its
 * multigrid preconditioner is out of scope), for a continuous (UF_CG) or a discontinuous (UF_DG)
 * operator.  The Jacobi diagonal is computed on the host in FP64 (for UF_DG, and the work
 * vectors with it, on the first call: that call allocates device memory) and follows
 * uf_set_kappa, not uf_set_kappa_device:
 *   UF_SOLVE_FP64  PCG in FP64 on the correction of the initial guess until
 *                  ||b - A x|| <= tol ||b||, restarted from the true FP64 residual while the
 *                  recursive residual of the PCG has drifted below it (outer counts the runs);
 *   UF_SOLVE_IR    iterative refinement: FP64 residual r = b - A x, FP32 PCG on A d = r / ||r||
 *                  to a relative reduction inner_tol, FP64 update x += ||r|| d, repeated until
 *                  the FP64 relative residual is <= tol (FP64 only for the outer residual and the
 *                  update; the FP32 operator carries the Nitsche and ghost-penalty terms);
 *   UF_SOLVE_IR_SPLIT the same refinement with the split inner operator: the rows of the cells
 *                  that carry Nitsche or ghost-penalty terms (cut cells and cells with a
 *                  ghost-penalty face) are evaluated in FP64 from the FP32 input and rounded
 *                  once to FP32, the other rows in FP32 (uf_vmult_split).  It uses the FP64
 *                  staging buffers of uf_vmult_host (UF_DG) or the FP64 cell-local vectors
 *                  (UF_CG), so no other call on the operator may overlap it.
 * x (in: initial guess, out: solution) and b are FP64 device vectors [n_dofs].  Synchronous on
 * return.  The dot products (deterministic two-pass FP64 reductions), alpha and beta stay in
 * device memory; the host reads the stopping state once per 32 iterations, so up to 31 operator
 * applications run past the stop (their updates are skipped).  max_iter caps the CG iterations
 * (all inner iterations in IR mode), max_outer the refinement steps / restarts.
 * UF_CG: work vectors are allocated at creation; UF_DG: on the first call.  Errors: UF_EINVAL
 * (missing precision, bad parameters, breakdown), UF_ENOMEM, UF_ENODEVICE, UF_ECUDA. */
enum { UF_SOLVE_FP64 = 0, UF_SOLVE_IR = 1, UF_SOLVE_IR_SPLIT = 2 };
typedef struct {
  int mode;
  double tol;
  double inner_tol;
  int max_iter;
  int max_outer;
} uf_solve_params;
typedef struct {
  int converged, outer, iterations;
  double rel_residual;  /* final ||b - A x|| / ||b|| in FP64 */
  double seconds;       /* device time of the solve (CUDA events on `stream`) */
} uf_solve_stats;
uf_status uf_solve(uf_operator *op, const uf_solve_params *params, double *x, const double *b,
                   uf_solve_stats *stats, void *stream);

/* Sphere accuracy benchmark (paper Sec. 4).  On the operator's ball (radius R = ls_radius around
 * ls_center), with r = |x - ls_center| and d = dim,
 *   u(r) = cos(omega R) - cos(omega r),   f(r) = -omega^2 (cos(omega r) + (d - 1) sin(omega r) / (omega r)),
 * solve -Lap u = f with u = 0 on the sphere (the Dirichlet data g = 0 of the Nitsche terms).
 * uf_manufactured_rhs writes b_i = int_Omega f phi_i (host FP64 [n_dofs]); uf_l2_error returns
 * ||u_h - u||_L2(Omega) and ||u||_L2(Omega) for the discrete function with DoF values x (host FP64
 * [n_dofs]).  Both integrate on the operator's own quadrature (tensor Gauss with p + 1 points per
 * direction on inside cells, the cut-cell rules on cut cells), in FP64 on the host; they are
 * set-up and post-processing of the accuracy study, not part of the operator's evaluation.
 * Errors: UF_EINVAL (NULL, non-finite omega), UF_EUNSUPPORTED (not a sphere level set). */
uf_status uf_manufactured_rhs(const uf_operator *op, double omega, double *b);
uf_status uf_l2_error(const uf_operator *op, double omega, const double *x, double *err,
                      double *norm);

/* Release every host and device resource of op.  NULL is accepted (no-op).  The library's own
 * pipeline streams (asynchronous host-buffer products) are waited for; the caller must make sure
 * none of its streams still runs other work of op. */
uf_status uf_destroy(uf_operator *op);

/* Thread-local message of the last failing call of this thread ("" if none). */
const char *uf_last_error(void);

/* Host-side fault injection for tests (the paper has no failure handling of its own).  Every
 * device allocation, pinned host allocation and operator object of the library counts as one
 * allocation.  After uf_debug_fail_allocation(k), the next k allocations succeed and the one after
 * them fails as if memory were exhausted, without calling the allocator.  The call that made it
 * then returns UF_ENOMEM after releasing what it had allocated, and the hook disarms itself; a
 * negative k disarms it.  uf_debug_live_allocations reports the library's allocations not yet
 * released.  Both act on process-wide state; calls on several threads may interleave.
 * Errors: UF_EINVAL (NULL live). */
uf_status uf_debug_fail_allocation(int64_t after);
uf_status uf_debug_live_allocations(int64_t *live);

#ifdef __cplusplus
}
#endif
#endif /* UNFITTED_H */
