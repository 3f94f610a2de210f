/*
 * msbem.h -- C ABI of the GB300 multiscreen hypersingular BEM library.
 *
 * The library solves the Galerkin system  W Phi = L  of the Laplace
 * hypersingular operator on a polygonal multiscreen Gamma (Averseng, Claeys,
 * Hiptmair, "Boundary Element Methods for the Laplace Hypersingular Integral
 * Equation on Multiscreens: a two-level Substructuring Preconditioner"),
 * by preconditioned conjugate gradients under the two-level additive Schwarz
 * (substructuring) preconditioner of the paper, on one GPU.
 *
 * Problem statement (Sec. 1 eq. PDE_intro, Sec. 3.3 Thm. thmBVP): find the
 * jump phi with a(phi, psi) = l_g(psi) for all psi, where a is the
 * hypersingular form (Def. defa) and l_g(psi) = <<gamma u, pi_n g>> (eq. defRhs).
 *
 * Conventions shared by every call
 *   - All functions return 0 (MSBEM_OK) on success or a negative status.
 *     After a failure msbem_last_error(ctx) holds a one-line message.
 *   - Host arrays passed in are only read during the call and copied; the
 *     caller keeps ownership.  Device memory is owned by the library and freed
 *     by msbem_geom_free / msbem_destroy.
 *   - A context is bound to one device and one CUDA stream; it is not thread
 *     safe (one host thread per context at a time).
 *   - Triangles are int32 vertex-id triples; vertices are float64 xyz triples
 *     (row-major, 3 per vertex).  Normals n_T = (x1-x0) x (x2-x0) orient each
 *     triangle; the side (T,+) is the one n_T points into (Def. Mstar).
 *   - Dof numbering (Sec. 4.2 eq. defCurlyHtildeGamma): dofs are the
 *     generalized vertices (i,j), j < q_i, of the vertices with q_i > 1, in
 *     increasing vertex id, then increasing sector index; sectors of a vertex are
 *     numbered by the smallest key 2*T + (0 for side +, 1 for side -) of their
 *     oriented triangles, so sector q_i is the one with the largest such key.
 */
#ifndef MSBEM_H
#define MSBEM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MSBEM_OK 0
#define MSBEM_INVALID_ARG (-1)     /* bad pointer, size or option            */
#define MSBEM_NONCONFORMING (-2)   /* degenerate/duplicate/overlapping tris,  */
                                   /* or fine mesh not nested in coarse mesh  */
#define MSBEM_POINT_CONTACT (-3)   /* vertex whose triangles are not edge-    */
                                   /* connected (excluded, Sec. 4.3 footnote) */
#define MSBEM_OOM (-4)             /* device allocation failed                */
#define MSBEM_NOT_CONVERGED (-5)   /* maxit reached; density still written    */
#define MSBEM_BREAKDOWN (-6)       /* p^T W p <= 0 or non-finite in PCG       */
#define MSBEM_DEVICE_TIMEOUT (-7)  /* a bounded device-side wait expired      */
#define MSBEM_CUDA_ERROR (-8)      /* a CUDA call failed                      */
#define MSBEM_NOT_READY (-9)       /* call order violated (e.g. solve before  */
                                   /* assemble)                               */

typedef struct msbem_ctx msbem_ctx;
typedef struct msbem_geom msbem_geom;

/* Create a context on CUDA device `device`, issuing all work on `cuda_stream`
 * (a cudaStream_t; NULL = the legacy default stream).  *ctx receives the
 * handle.  Errors: INVALID_ARG, CUDA_ERROR. */
int msbem_create(msbem_ctx** ctx, int device, void* cuda_stream);

/* Destroy a context and every geometry still attached to it. */
int msbem_destroy(msbem_ctx* ctx);

/* Message of the last failure on this context ("" if none).  The string is
 * owned by the context and valid until the next call on it. */
const char* msbem_last_error(const msbem_ctx* ctx);

/* Upload a multiscreen and its substructuring (Sec. 3.1 Def. polygonalMS,
 * Sec. 5 "Coarse mesh", eq. jumpSplit).
 *   xyz[3*nv], tri[3*nt]           fine mesh M_{Gamma,h}
 *   coarse_xyz[3*ncv], coarse_tri[3*nct]  coarse mesh M_{Gamma,H}; the fine
 *                                  mesh must refine it (nested)
 *   parent_coarse_tri[nt]          coarse triangle containing each fine one
 *   patch_of_tri[nt]               patch id (>= 0) of each fine triangle; the
 *                                  face space of patch p holds the dofs whose
 *                                  vertex has all incident triangles in p, the
 *                                  remaining dofs form the wire basket
 * Builds the topology on the host (sectors by angular wedge linking around
 * every edge, dofs, surface-curl lists, pair classes, face/wire-basket classes,
 * coarse prolongation) and copies the mesh data to the device.
 * Errors: INVALID_ARG, NONCONFORMING, POINT_CONTACT, OOM, CUDA_ERROR. */
int msbem_upload(msbem_ctx* ctx, const double* xyz, int64_t nv, const int32_t* tri, int64_t nt,
                 const double* coarse_xyz, int64_t ncv, const int32_t* coarse_tri, int64_t nct,
                 const int32_t* parent_coarse_tri, const int32_t* patch_of_tri, msbem_geom** out);

/* Host-only mesh analysis (no context, no GPU): builds the topology of a
 * triangle mesh exactly as msbem_upload does (sectors, Sec. 4.2 generalized
 * vertices, dofs) and reports the dof count and, if cap >= *ndof, the dof map
 * (vertex id and sector index of every dof).  errbuf (may be NULL) receives a
 * message of at most errcap bytes on failure.
 * Errors: INVALID_ARG, NONCONFORMING, POINT_CONTACT. */
int msbem_mesh_dofs(const double* xyz, int64_t nv, const int32_t* tri, int64_t nt, int64_t* ndof,
                    int32_t* vertex_of_dof, int32_t* sector_of_dof, int64_t cap, char* errbuf,
                    int errcap);

/* Release a geometry and its device memory. */
int msbem_geom_free(msbem_geom* g);

/* Number of dofs N = |H~([Gamma])| (Sec. 4.2). */
int msbem_ndofs(const msbem_geom* g, int64_t* n);

/* Dof map (host arrays of length N): vertex id and 0-based sector index of
 * every dof, in the numbering described at the top of this file. */
int msbem_dof_map(const msbem_geom* g, int32_t* vertex_of_dof, int32_t* sector_of_dof);

/* Sizes of the splitting (eq. jumpSplit): number of face spaces (patches with
 * at least one dof), wire-basket size, coarse-space size, largest face block.
 * Any pointer may be NULL. */
int msbem_split_info(const msbem_geom* g, int64_t* n_faces, int64_t* n_wire_basket,
                     int64_t* n_coarse, int64_t* max_face);

typedef struct msbem_assemble_opts {
  int ss_order;    /* Gauss-Legendre points per dimension of the singular     */
                   /* (Sauter-Schwab-type) rules, 2..16; <= 0: default 5      */
  int far_kernel;  /* pair integrals: 0 = double-float arithmetic on the FP32 */
                   /* pipe (default), 1 = native FP64 (far and near field)    */
  int64_t panel_rows; /* 0 (default): V (nt x nt float pairs) in one piece    */
                   /* when it fits in free device memory, else in row panels  */
                   /* sized to fit; > 0: panels of that many triangle rows    */
                   /* (a multiple of 64).  Panels need far_kernel 0; W is     */
                   /* then summed panel by panel (equal to rounding, not bit  */
                   /* for bit symmetric).                                     */
} msbem_assemble_opts;

/* Assemble W[nu,nu'] = a(psi~_nu, psi~_nu') (Sec. 4.3 eq. eval_a_phiij with
 * Cor. corW): W = sum_{T,T'} V_{TT'} s_{T,nu} . s_{T',nu'}, V_{TT'} =
 * int_T int_T' 1/(4 pi |x-y|), with the 6-point degree-4 rule on pairs that
 * share no vertex and Sauter-Schwab-type rules on the others.  opts may be
 * NULL (defaults).  W (N x N, row-major) stays on the device, held as pairs of
 * floats (hi, lo) whose sum carries a 48-bit significand (relative precision
 * 2^-47, FP64-level for the solve); msbem_copy_matrix returns it as FP64.
 * A new assembly discards the preconditioner (msbem_factor again); a failed
 * one leaves the geometry neither assembled nor factored.
 * Errors: INVALID_ARG (options), NOT_READY, OOM, CUDA_ERROR. */
int msbem_assemble(msbem_geom* g, const msbem_assemble_opts* opts);

/* Copy rows [row0, row0+nrows) of W into out (host or device, nrows*N
 * doubles, row-major), converted to FP64.  A host destination needs a
 * temporary device buffer of nrows*N doubles.
 * Errors: NOT_READY, INVALID_ARG, OOM, CUDA_ERROR. */
int msbem_copy_matrix(const msbem_geom* g, int64_t row0, int64_t nrows, double* out);

/* Right-hand side L_nu = l_g(psi~_nu) = sum_T (c_+ - c_-)(g . n_T)|T|/3 for a
 * constant Neumann datum g (Sec. 4.3, last display) into out[N] (host or
 * device). */
int msbem_rhs(const msbem_geom* g, const double gvec[3], double* out);

typedef struct msbem_precond_opts {
  int wire_basket;   /* 0 = exact solve on the wire basket (Thm. main),      */
                     /* 1 = diagonal ("pointwise scalar product", Remark     */
                     /*     "Approximate solvers", Sec. 2.1)                  */
  int use_coarse;    /* 1 (default) = include the coarse space V~_H          */
  int precision;     /* 0 (default) = face and wire-basket inverses in       */
                     /*     double-float (FP64 accuracy);                     */
                     /* 1 = those inverses in FP32 (Gauss-Jordan in FP32,    */
                     /*     symmetrised): for the mixed-precision solves     */
                     /*     (precision 2, 4, 5), whose inner PCG reads FP32   */
                     /*     inverses anyway; the other solves still converge  */
                     /*     but with a less exact preconditioner.  The coarse */
                     /*     block A_H stays double-float.                     */
} msbem_precond_opts;

/* Set up M(H;h) (Sec. 2.1 Remark on PCG, eq. jumpSplit): the principal blocks
 * A_F = W[F,F] of every face space and A_W of the wire basket, and the coarse
 * matrix A_H = P^T W P, all inverted (FP64 accuracy unless opts->precision
 * is 1).  opts may be NULL.
 * Rejected options (INVALID_ARG) change nothing; any other failure leaves the
 * geometry unfactored (solves with the preconditioner return NOT_READY).
 * Errors: INVALID_ARG, NOT_READY (no W), BREAKDOWN (a block is not positive
 * definite), OOM, CUDA_ERROR. */
int msbem_factor(msbem_geom* g, const msbem_precond_opts* opts);

/* msbem_factor for n geometries of ONE context at once: the face, wire-basket
 * and coarse blocks of all of them (Sec. 5, eq. jumpSplit) are inverted by one
 * grouped sequence of launches (per 32-column step of the blocked Gauss-Jordan
 * recursion, the pivot, panel and update launches cover every block of every
 * geometry at once), so that many small instances fill the GPU together.  The
 * inverses are the same, bit for bit, as those msbem_factor gives each
 * geometry alone.
 *   geoms   n distinct geometries (caller-owned array), all assembled, all
 *           uploaded to the same context;
 *   opts    applied to every geometry, may be NULL;
 *   status  NULL or n ints (caller-owned): per geometry MSBEM_OK or
 *           MSBEM_BREAKDOWN.
 * Geometries whose status is MSBEM_OK are factored even when others broke
 * down.  The set-up time (msbem_last_timings, factor_ms) of each geometry is
 * that of the whole group, and the group's inversion launches count in the
 * first geometry's msbem_counters.
 * Errors: INVALID_ARG (n < 1, a NULL or repeated geometry, geometries of
 * different contexts), NOT_READY (one is not assembled; nothing is factored),
 * BREAKDOWN (a block of some geometry is not positive definite), OOM,
 * CUDA_ERROR. */
int msbem_factor_group(msbem_geom* const* geoms, int n, const msbem_precond_opts* opts, int* status);

typedef struct msbem_solve_opts {
  double rtol;        /* stop when ||L - W Phi_k|| <= rtol ||L|| (default 1e-8)*/
  int maxit;          /* iteration cap (default 1000)                          */
  int fixed_iters;    /* 1: run exactly maxit iterations (parity checks)       */
  int precondition;   /* 1 (default): PCG with M(H;h); 0: plain CG             */
  int precision;      /* arithmetic of the matrix-vector products:             */
                      /*  0 (default) double-float W (hi + lo FP32 planes,     */
                      /*    FP64-equivalent accuracy) and double-float         */
                      /*    preconditioner;                                    */
                      /*  1 plain FP64: an FP64 copy of W (made on first use,  */
                      /*    N*N*8 more bytes) and the FP64 block inverses;     */
                      /*  2 mixed: iterative refinement whose residual is the  */
                      /*    double-float product and whose correction equation */
                      /*    is solved by PCG with FP32 products (hi plane of   */
                      /*    W) to inner_rtol; iters counts inner iterations,   */
                      /*    resid_hist holds the true relative residual after  */
                      /*    each refinement step; fixed_iters is not allowed;  */
                      /*  3 tensor cores, double-float: as 0 with the products */
                      /*    formed by tcgen05 MMAs from six exact 8-bit        */
                      /*    integer slices of W and of the vectors (W's slices */
                      /*    take N*N*12 more bytes, made on first use);        */
                      /*  4 mixed, tensor-core residual: as 2 with the         */
                      /*    residual products as in 3;                         */
                      /*  5 mixed, scaled FP16: as 4 with the inner products   */
                      /*    on the tensor cores from an fp16 copy of W scaled  */
                      /*    by a power of two per row (each entry to 2^-11 of  */
                      /*    itself; N*N*2 more bytes)                          */
  double inner_rtol;  /* precision 2, 4, 5: inner tolerance (<= 0: 1e-4)       */
  double density_tol; /* precision 2, 4, 5: when > 0, a result also needs its  */
                      /*   estimated relative error (l2) <= density_tol: with  */
                      /*   the refinement's corrections D_k and their          */
                      /*   contraction eta = ||D_k|| / ||D_k-1||, the error of */
                      /*   X_k+1 is estimated as eta/(1-eta) ||D_k|| / ||X_k+1||*/
                      /*   (so at least two refinement steps); 0: residual     */
                      /*   test alone (default); must be < 1                   */
} msbem_solve_opts;

/* Solve W Phi = L for constant Neumann data g by PCG from Phi_0 = 0
 * (Sec. 2.1 Remark "Bound on the number of PCG iterations").
 *   density[N]      output Phi (host or device pointer)
 *   iters           iterations performed
 *   resid_hist      relative residual after 0..iters iterations (first
 *                   min(hist_cap, iters+1) entries written; may be NULL)
 *   kappa_est       condition number of the Lanczos tridiagonal built from the
 *                   PCG coefficients (may be NULL)
 * opts may be NULL.  Returns NOT_CONVERGED (density still written) if maxit is
 * reached first, BREAKDOWN on p^T W p <= 0 or a non-finite value. */
int msbem_solve(msbem_geom* g, const double gvec[3], const msbem_solve_opts* opts, double* density,
                int* iters, double* resid_hist, int hist_cap, double* kappa_est);

/* Solve W Phi_c = L(g_c) for k constant Neumann data g_c at once (block PCG):
 * every column follows the recursion of msbem_solve (own scalars and stopping
 * test) while the k columns share each pass over W (and over the block
 * inverses of the preconditioner), so k solves cost far less than k calls of
 * msbem_solve.  Columns are processed in groups of up to 16.
 *   gvecs[3*k]         the data g_c
 *   densities[k*N]     output, row c = Phi_c (host or device pointer)
 *   iters[k], relres[k], kappa_est[k]  per-column results (each may be NULL)
 * opts->precision as in msbem_solve: 0 and 3 run the double-float recursion
 * (CUDA-core or tensor-core products), 2, 4 and 5 the mixed refinement, 1 the
 * plain FP64 comparator one column at a time.  A column's result does not
 * depend on the other columns of its call (bit for bit).
 * Returns the worst status over the columns (NOT_CONVERGED / BREAKDOWN as in
 * msbem_solve; densities always written). */
int msbem_solve_batch(msbem_geom* g, const double* gvecs, int k, const msbem_solve_opts* opts,
                      double* densities, int* iters, double* relres, double* kappa_est);

/* Closed cells.  When the screen encloses bounded regions of R^3 (the cube
 * with its mid-planes encloses eight), the indicators of those cells have
 * vanishing surface curls and span the kernel of the hypersingular form; the
 * paper's connectedness assumption fails.  Reading used: msbem_assemble then
 * stores W + rho Q Q^T, rho = mean diag(W), Q = Z L^-T (Z^T Z = L L^T) an
 * orthonormal basis of the span of Z, the psi-coordinates of the cells'
 * indicators (value [sector j in K] minus its mean over the q_i sectors of the
 * vertex): the kernel directions take the eigenvalue rho; for constant g,
 * Z^T L = 0 and the solution is the one with Z^T Phi = 0.  Cells are the components of R^3 minus the screen found from the
 * sectors whose flux sum |T| (x_T . n) / 3 is negative (bounded, divergence
 * theorem).  Outputs: *ncells; Z[N * ncells] row-major (host, may be NULL);
 * *rho (valid after msbem_assemble). */
int msbem_cells(const msbem_geom* g, int* ncells, double* Z, double* rho);
/* The same, host only, from a mesh (no device): Z written when cap >= N * ncells. */
int msbem_mesh_cells(const double* xyz, int64_t nv, const int32_t* tri, int64_t nt, int* ncells, double* Z,
                     int64_t cap);

/* Y = W X: the Galerkin matrix applied to k <= 16 vectors at once (the
 * matrix-vector product of PCG, Sec. 2.1), e.g. for energies Phi^T W Phi.
 *   X[k*N], Y[k*N]  row c = vector c (host or device pointers, independently)
 *   precision       0 double-float products (FP64-equivalent), 1 the plain
 *                   FP64 copy of W (made on first use), 2 FP32 products with
 *                   the hi plane of W (about 1e-7 relative), 3 double-float
 *                   accuracy on the tensor cores: W and X cut into six exact
 *                   8-bit integer slices (bf16), slice products summed exactly
 *                   in FP32 accumulators (the slices of W, 12 bytes per entry,
 *                   are made on first use and kept until the next assembly),
 *                   4 scaled FP16 on the tensor cores (an fp16 copy of W
 *                   scaled by a power of two per row: each entry to 2^-11 of
 *                   itself; the vectors as two fp16 terms; FP32 accumulation)
 *   kernel_ms       device time of the product kernel(s) alone (may be NULL)
 * Errors: INVALID_ARG (k outside 1..16, bad precision), NOT_READY (no W),
 * DEVICE_TIMEOUT, OOM, CUDA_ERROR. */
int msbem_apply(msbem_geom* g, const double* X, int k, int precision, double* Y, double* kernel_ms);

/* The field U = DL Phi off the screen (Lemma lemrepDL, eq. formulaDL): for
 * targets x_m off Gamma,
 *   U(x) = sum_T sum_a J_{T,a} int_T n_T.(y - x) lambda_a(y) / (4 pi |x-y|^3) dy,
 *   J_{T,a} = sum_nu Phi_nu (c_+ - c_-)(T, a, nu)  (the jump of the density),
 * each triangle integrated by the 6-point rule on its 4^refine congruent
 * sub-triangles (refine 0..4; raise it for targets within a few h of Gamma).
 *   density[N]      Phi, e.g. from msbem_solve (host or device)
 *   targets[3*M]    target points, xyz triples (host or device)
 *   out[M]          U(x_m) (host or device)
 *   kernel_ms       device time of the evaluation kernel (may be NULL)
 * FP64 throughout.  Errors: INVALID_ARG, OOM, CUDA_ERROR. */
int msbem_dl_potential(msbem_geom* g, const double* density, const double* targets, int64_t M, int refine,
                       double* out, double* kernel_ms);

/* Timing of the last assemble / factor / solve on this geometry, in
 * milliseconds measured with CUDA events on the context's stream:
 * t[0] far field, t[1] near field, t[2] contraction to W, t[3] factor,
 * t[4] solve.  Any entry not yet measured is 0. */
int msbem_last_timings(const msbem_geom* g, double t[5]);

/* In-place inverses of `count` symmetric positive definite matrices by the
 * grouped blocked Gauss-Jordan recursion that msbem_factor runs over the face,
 * wire-basket and coarse blocks (Sec. 5, eq. jumpSplit: the blocks of M(H;h)
 * are inverted explicitly): per 32-column step, the pivot, panel and update
 * launches cover all matrices at once.  With precision 0 (double-float) the
 * update of a matrix of order >= 2048 is the tensor-core form (each rank-32
 * product from exact 8-bit slices of both operands, folded into double-float)
 * and that of a smaller one the CUDA-core form; the result depends on each
 * matrix's own order only, and is accurate to about 1e-15 cond(A) relative.
 * Precision 1 inverts in FP32 and symmetrises.
 *   ctx       context: its device, stream and memory pool are used
 *   A[count]  host array of device pointers, each an n[i] x n[i] row-major
 *             FP64 matrix on the context's device, overwritten by its inverse;
 *             distinct, non-overlapping
 *   n[count]  host array of orders, each >= 1
 *   status    NULL or count ints (host): MSBEM_OK or MSBEM_BREAKDOWN (a pivot
 *             that was not positive; that matrix then holds no inverse)
 * The call allocates its scratch (operand slices, panels, index words) from
 * the context's pool and waits for the stream before it returns.
 * Errors: INVALID_ARG (ctx or an array NULL, count < 1, an order < 1, a
 * precision other than 0 or 1), BREAKDOWN (some matrix), OOM, DEVICE_TIMEOUT,
 * CUDA_ERROR. */
int msbem_spd_inverse_group(msbem_ctx* ctx, double* const* A, const int64_t* n, int count, int precision,
                            int* status);

/* Largest matrix order msbem_spd_inverse_noalloc accepts. */
#define MSBEM_NOALLOC_MAX_N 2048

/* Inverse of one symmetric positive definite matrix, allocating no device
 * memory.  The paper has no counterpart: this is for callers that cannot
 * allocate, such as a process that has reserved all of its GPU memory for its
 * own pool up front, or a latency-critical loop that cannot afford cudaMalloc /
 * cudaFree (they synchronize the device and can fail under memory pressure).
 *   A[n*n]     device pointer, row-major FP64, symmetric positive definite
 *   Ainv[n*n]  device pointer receiving A^{-1} (may equal A: in place)
 *   n          1 <= n <= MSBEM_NOALLOC_MAX_N, else INVALID_ARG
 *   cuda_stream  stream for all work (NULL = legacy default stream)
 * The method is the same blocked Gauss-Jordan recursion msbem_factor uses
 * (32-wide panels, rank-32 updates in double-float).  Its scratch -- about
 * 1 MiB: the pivot block, two n x 32 panels, index words and the breakdown
 * flag -- is one file-scope device array.  It exists on a GPU once the
 * library's device code is loaded there and stays until the process exits.
 * Each call looks up that array's device address (cudaGetSymbolAddress) on the
 * current device, so A, Ainv and the stream must belong to the current device.
 * Every call shares the array and clears what must start at zero, so calls
 * that overlap on the GPU (on different streams or from different threads)
 * race and must not be issued.  The call copies a few index words from
 * pageable host memory and waits for the stream to read the breakdown flag,
 * so it cannot be called while the stream (or, for the legacy stream, any
 * stream) is being captured: it then returns INVALID_ARG (or CUDA_ERROR)
 * without doing any work.  Returns BREAKDOWN if a pivot is not positive (Ainv
 * then holds no inverse), CUDA_ERROR on a CUDA failure. */
int msbem_spd_inverse_noalloc(const double* A, int64_t n, double* Ainv, void* cuda_stream);

/* Counters of this geometry: *launches = number of CUDA kernels the library
 * has launched for it so far (all calls), *far_pairs = number of unordered
 * triangle pairs sharing no vertex (the units of the far-field kernel).
 * Either pointer may be NULL. */
int msbem_counters(const msbem_geom* g, int64_t* launches, int64_t* far_pairs);

/* ------------------------------------------------------------------------
 * Test hooks of the error paths (no counterpart in the paper).  They let the
 * tests drive the library's failure handling without a GPU fault: an
 * allocation that fails on the host side, and a bounded device-side wait that
 * runs out.  Process-wide; not for production use.
 * ------------------------------------------------------------------------ */

/* The (after + 1)-th device allocation the library makes from its memory
 * pools from now on fails as if the device were out of memory, once (the
 * hook then turns itself off); after = -1 turns a pending failure off.  The
 * failing call returns OOM and leaves its object as a failed call would
 * (e.g. a geometry neither assembled nor factored).  INVALID_ARG for after < -1. */
int msbem_test_fail_alloc(int64_t after);

/* ns > 0: on the current device, every CTA of the matrix-vector product
 * kernels (CUDA-core and tensor-core) first waits up to ns nanoseconds on a
 * device flag that nothing sets, then takes the path of a copy that never
 * completed: it lets its copies in flight land (bounded waits), frees what it
 * holds, sets the error flag and returns.  The calls whose products ran then
 * return DEVICE_TIMEOUT and the context stays usable.  ns = 0 turns it off.
 * Synchronizes the device.  INVALID_ARG for ns < 0. */
int msbem_test_expire_waits(int64_t ns);

/* ------------------------------------------------------------------------
 * Serving engine (no counterpart in the paper: it serves many solves of the
 * paper's problem).  Geometries (mesh + partition) are registered under a
 * key; solve requests (key, g) are queued, and msbem_server_progress admits
 * geometries against an HBM budget (assembly + factorisation on first use,
 * least-recently-used eviction of idle ones), runs a 16-slot multi-vector
 * PCG per resident geometry on its own stream, and refills slots as requests
 * finish (continuous batching).  A request's result does not depend on the
 * other requests it shares a batch with (bit for bit).
 * ------------------------------------------------------------------------ */
typedef struct msbem_server msbem_server;

typedef struct msbem_server_opts {
  double hbm_budget_bytes;  /* admission limit for resident geometries (0: 80% of free) */
  int precision;            /* as msbem_solve_opts.precision, except 1: 0 double-float */
                            /* PCG, 2 mixed (FP32 inner + refinement), 3, 4, 5 their   */
                            /* tensor-core forms                                        */
  double rtol;              /* relative residual per request (0: 1e-8)                 */
  double inner_rtol;        /* mixed precisions: inner tolerance (0: 1e-4)             */
  int maxit;                /* iterations per request (inner, summed; 0: 1000)         */
  int chunk;                /* PCG iterations between scheduling points (0: 4)         */
  int admission_threads;    /* host threads admitting new geometries, each with its   */
                            /* own context and stream (0: 4; at most 8)                */
  double density_tol;       /* mixed precisions: as msbem_solve_opts.density_tol (0:   */
                            /* residual test alone)                                     */
} msbem_server_opts;

typedef struct msbem_server_stats {
  int64_t submitted, completed, admissions, evictions;
  double resident_bytes;
  int resident_geometries;
  /* work of the admissions finished so far (CUDA events inside each call, on
   * the stream the kernels ran on): far-field kernel time and its unit count
   * (unordered triangle pairs sharing no vertex), whole assemblies and
   * preconditioner set-ups; kernels launched for all geometries, resident or
   * evicted */
  double far_ms;
  int64_t far_pairs;
  double assemble_ms, factor_ms;
  int64_t launches;
} msbem_server_stats;

/* Create an engine on ctx (opts may be NULL).  Errors: INVALID_ARG, CUDA_ERROR. */
int msbem_server_create(msbem_ctx* ctx, const msbem_server_opts* opts, msbem_server** out);
/* Free every resident geometry and the engine. */
int msbem_server_destroy(msbem_server* s);
/* Register a geometry under `key` (arrays as msbem_upload; copied, nothing
 * goes to the device yet).  Errors: INVALID_ARG (duplicate key), topology
 * errors of msbem_upload. */
int msbem_server_add_geometry(msbem_server* s, uint64_t key, const double* xyz, int64_t nv, const int32_t* tri,
                              int64_t nt, const double* coarse_xyz, int64_t ncv, const int32_t* coarse_tri,
                              int64_t nct, const int32_t* parent_coarse_tri, const int32_t* patch_of_tri);
/* The engine's clock (seconds, monotonic) for arrival time stamps. */
double msbem_server_now(void);
/* Bytes the admission of a registered geometry asks of the budget (resident
 * W, preconditioner and batch, plus the assembly's transient pair matrix);
 * -1 for an unknown key. */
double msbem_server_footprint(const msbem_server* s, uint64_t key);
/* Queue a request; density (N doubles, host or device, may be NULL) receives
 * Phi when it finishes.  t_arrival: arrival time on the engine's clock (<= 0:
 * now); latency is measured from it.  *id identifies the request. */
int msbem_server_submit(msbem_server* s, uint64_t key, const double gvec[3], double* density, double t_arrival,
                        uint64_t* id);
/* Admit, launch and harvest.  block = 0: one pass, returns at once; block = 1:
 * until every queued request has finished.  *completed: requests finished in
 * this call.  Returns the last admission error (OOM when a geometry never fits). */
int msbem_server_progress(msbem_server* s, int block, int* completed);
/* Result of a request: status (1 while pending, else a msbem status),
 * iterations (inner iterations summed in precision 2), true relative
 * residual, latency from arrival to the density being written, and the
 * number of refinement steps (precision 2). */
int msbem_server_result(msbem_server* s, uint64_t id, int* status, int* iters, double* relres, double* latency_ms,
                        int* refinements);
int msbem_server_stats_get(const msbem_server* s, msbem_server_stats* out);

#ifdef __cplusplus
}
#endif

#endif /* MSBEM_H */
