// Internal declarations of the msbem library (not part of the C ABI).
#pragma once

#include <array>
#include <cstdint>
#include <string>
#include <vector>

#include <cuda.h>
#include <cuda_runtime.h>

#include "../../include/msbem.h"

namespace msbem {

// ---------------------------------------------------------------------------
// Host topology of a triangle mesh (Sec. 4.2-4.3): sectors at every vertex,
// generalized vertices, dofs and the constant surface curls of the jumps of
// the basis functions on every triangle.
// ---------------------------------------------------------------------------
struct Topo {
  int64_t nv = 0, nt = 0;
  std::vector<double> xyz;       // 3*nv
  std::vector<int32_t> tri;      // 3*nt
  std::vector<double> area;      // nt
  std::vector<double> normal;    // 3*nt, unit, n_T = (x1-x0) x (x2-x0) / |.|
  std::vector<int32_t> q;        // sectors per vertex
  std::vector<int32_t> sector;   // 6*nt: sector[(T*2+side)*3 + a] at vertex tri[3T+a]
  std::vector<int64_t> first_dof;  // nv+1
  int64_t ndof = 0;
  std::vector<int32_t> dof_vertex, dof_sector;
  // jump coefficients: for dof nu, entries k in [jptr[nu], jptr[nu+1]):
  // triangle jtri[k], local vertex jloc[k], coefficient jcoef[k] = c_+ - c_-
  std::vector<int64_t> jptr;
  std::vector<int32_t> jtri, jloc;
  std::vector<double> jcoef;
  // closed cells (bounded regions of R^3 minus the screen) and the
  // psi-coordinates of their indicators, cellZ[nu * ncells + c]
  int ncells = 0;
  std::vector<double> cellZ;
  std::vector<double> cellQ;    // orthonormal basis Z L^-T of their span (Z^T Z = L L^T)
};

// Builds the topology; returns MSBEM_OK or an error status with a message.
int build_topology(const double* xyz, int64_t nv, const int32_t* tri, int64_t nt, Topo& out,
                   std::string& err);

// Closed cells of the screen (fills Topo::ncells and Topo::cellZ; topology.cpp).
void build_cells(Topo& t);

// Near pairs (pairs sharing at least one vertex, including T = T), with the
// canonical local vertex orderings used by the singular rules:
//   identical: (v0,v1,v2) as stored;
//   edge:      A = smaller shared vertex id, B = larger, C / D the others;
//   vertex:    O shared, then its cyclic successors in each triangle.
// The triangle with the smaller index comes first.
struct NearPair {
  int32_t T, S;       // T <= S
  int32_t cls;        // 3 identical, 2 edge, 1 vertex
  int32_t v[6];       // canonical vertex ids: T's three then S's three
};
void build_near_pairs(const Topo& t, std::vector<NearPair>& out);

// Face / wire-basket split (Sec. 5, eq. jumpSplit) and coarse prolongation.
struct Split {
  int64_t n_faces = 0;
  std::vector<int64_t> block_ptr;    // n_blocks+1 (faces first, wire basket last)
  std::vector<int32_t> block_dofs;   // dofs of every block, ascending within a block
  int64_t n_wb = 0;
  int64_t max_face = 0;
  // coarse prolongation P (N x NH), CSR by fine row
  int64_t n_coarse = 0;
  std::vector<int64_t> p_ptr;
  std::vector<int32_t> p_col;
  std::vector<double> p_val;
};
int build_split(const Topo& fine, const Topo& coarse, const int32_t* parent, const int32_t* patch,
                Split& out, std::string& err);

// Quadrature constants computed on the host (own implementation).
void gauss_legendre01(int n, double* x, double* w);
void six_point_rule(double bary[6][3], double w[6]);

// ---------------------------------------------------------------------------
// Device-side state of one geometry
// ---------------------------------------------------------------------------
// Stream-ordered allocation from the context's pool (which keeps freed memory
// for reuse, so repeated uploads of similar geometries do not remap HBM).
// Test hook (msbem_test_fail_alloc, api.cu): true when the injected failure
// is due, which makes this allocation fail as if the device were out of memory.
bool test_alloc_fails();
inline cudaError_t pool_alloc(void** p, size_t bytes, cudaMemPool_t pool, cudaStream_t s) {
  if (test_alloc_fails()) return cudaErrorMemoryAllocation;
  return pool ? cudaMallocFromPoolAsync(p, bytes, pool, s) : cudaMallocAsync(p, bytes, s);
}

struct DevGeom {
  cudaMemPool_t pool = nullptr;  // owned by the context
  // triangle data for the far field, arranged in tiles of 64 triangles
  int64_t nt = 0, nt_pad = 0;
  double* d_qp = nullptr;        // [nt_pad][6][3] quadrature points (FP64)
  double* d_cen = nullptr;       // [nt_pad][3] centroids
  float* d_qoff = nullptr;       // [nt_pad][6][3][2] point - centroid as (hi, lo) floats
  double* d_area = nullptr;      // [nt_pad]
  float2* d_cendf = nullptr;     // [nt_pad][3] centroids as (hi, lo) floats
  float2* d_areadf = nullptr;    // [nt_pad] areas as (hi, lo) floats
  int32_t* d_tri = nullptr;      // [nt_pad][3] (padding: -1)
  double* d_xyz = nullptr;       // [nv][3]
  NearPair* d_near = nullptr;    // [n_near]
  int64_t n_near = 0;
  float2* d_V = nullptr;         // [nt][nt] pair matrix as (hi, lo) floats (scratch)
  // jump/curl lists
  int64_t ndof = 0;
  int64_t* d_jptr = nullptr;
  int32_t* d_jtri = nullptr;
  double* d_jvec = nullptr;      // [entries][3] curl vectors s_{T,nu}
  float2* d_jvecf = nullptr;     // [entries][3] the same as (hi, lo) floats
  double* d_jrhs = nullptr;      // [entries][3] coef |T|/3 n_T (RHS weights)
  // Galerkin matrix as two FP32 planes [2][N][ldw] (hi, then lo; W = hi + lo
  // to ~2^-48 relative), ldw = N rounded up to 32, padding columns zero
  int64_t ldw = 0;
  float* d_Wh = nullptr;
  float* wlo() const { return d_Wh + ndof * ldw; }
  CUtensorMap tm_W;              // 16 x 128 x 2 boxes of both planes (matvec.cu)
  CUtensorMap tm_Whi;            // 32 x 128 x 1 boxes of the hi plane
  double* d_W64 = nullptr;       // FP64 copy of W for the plain comparator (made on first use)
  // integer slices of W for the tensor-core products (matvec_tc.cu; made on
  // first use, dropped with W): six bf16 8-bit slices, one fp16 11-bit slice,
  // the row exponents they share, and their tensor maps
  void* d_wsl = nullptr;
  void* d_wf16 = nullptr;
  int* d_wexp = nullptr;
  CUtensorMap tm_wsl, tm_wf16;
  int64_t panel_rows = 0;        // rows of V per panel in the last assembly (0: V in one piece)
  int mv_split[2] = {0, 0};      // column splits of the CUDA-core products (modes 0, 1) picked
                                 // by the autotuner at assembly (0: the N-only default)
  int ncells = 0;                // closed cells: W holds W + rho Q Q^T (Q: [N][ncells], orthonormal)
  double* d_cellZ = nullptr;     // Q
  double rho = 0.0;
  // preconditioner
  int64_t n_blocks = 0;
  int64_t* d_bptr = nullptr;     // n_blocks+1
  int32_t* d_bdofs = nullptr;
  int64_t* d_boff = nullptr;     // offset of each block's inverse in d_binv
  double* d_binv = nullptr;
  float2* d_binvf = nullptr;     // float-pair copy of the face / wire-basket inverses
  int64_t binv_size = 0;
  int32_t* d_btile = nullptr;    // 16-row tiles of the blocks: (block, first row) pairs
  int64_t n_btiles = 0;
  int wb_diag = 0;
  int64_t n_coarse = 0;
  int64_t* d_pptr = nullptr;     // P in CSR (by fine row)
  int32_t* d_pcol = nullptr;
  double* d_pval = nullptr;
  int64_t* d_cptr = nullptr;     // P in CSC (by coarse column)
  int32_t* d_crow = nullptr;
  double* d_cval = nullptr;
  float2* d_cvalf = nullptr;     // CSC values as (hi, lo) floats
  double* d_AHinv = nullptr;     // [NH][NH]
  double* d_WP = nullptr;        // [NH][N] scratch
  int use_coarse = 1;
  // PCG vectors
  double* d_vec = nullptr;       // vectors of N: x r z p q, coarse scratch
  float* d_pfp = nullptr;        // search direction p as planes [2][ldw] (hi, lo; zero padding)
  CUtensorMap tm_p;              // 1 x 128 x 2 boxes of d_pfp
  float2* d_rf = nullptr;        // residual r as (hi, lo) floats
  double* d_scal = nullptr;      // device scalars
  int assembled = 0, factored = 0;
  // PCG iteration chunk captured as a CUDA graph (one per preconditioning mode),
  // valid until the next factorisation; captured on a private stream
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t pcg_exec[4] = {nullptr, nullptr, nullptr, nullptr};  // [precondition + 2 plain]
  double* d_hist = nullptr;      // persistent residual / alpha / beta history
  int hist_cap = 0;              // iterations the persistent history can hold
  int64_t launches = 0;          // kernels launched by this geometry so far
  int64_t n_far_pairs = 0;       // unordered pairs sharing no vertex
  float times[5] = {0, 0, 0, 0, 0};
};

// launch wrappers (assemble.cu, factor.cu, pcg.cu); all return cudaError_t
cudaError_t launch_far_fp64(const DevGeom& g, cudaStream_t s);
// err: a device int set to 1 when a tile's staging copy never completed
cudaError_t launch_far_df(const DevGeom& g, int* err, cudaStream_t s);
// t0, t1: the rows of V held (panel mode); t1 < 0: all rows
cudaError_t launch_near(const DevGeom& g, int ss_order, const double* gl_x, const double* gl_w,
                        int fp64, cudaStream_t s, int64_t t0 = 0, int64_t t1 = -1);
cudaError_t launch_contract(const DevGeom& g, cudaStream_t s);
// panel mode (V holds triangle rows tb0*64 .. (tb0+ntb)*64 - 1)
cudaError_t launch_far_df_panel(const DevGeom& g, int tb0, int ntb, int* err, cudaStream_t s);
cudaError_t launch_contract_panel(const DevGeom& g, int64_t t0, int64_t t1, int rt0, int nrt, cudaStream_t s);
cudaError_t launch_rhs(const DevGeom& g, const double gvec[3], double* out, cudaStream_t s);
cudaError_t copy_rows_to_double(const DevGeom& g, int64_t row0, int64_t nrows, double* out,
                                cudaStream_t s);
// diag(W) as FP64 (N values) and the rank-ncells update W += rho Q Q^T
cudaError_t copy_diagonal(const DevGeom& g, double* out, cudaStream_t s);
cudaError_t launch_augment(const DevGeom& g, double rho, cudaStream_t s);
cudaError_t set_far_constants(const double bary[6][3], const double w[6]);
cudaError_t set_far_df_constants(const double w[6]);

// Q = W P for kb <= 16 vectors (matvec.cu): mode 0 double-float on both W
// planes (tmW over both), mode 1 FP32 on the hi plane (tmW over one plane);
// tmP boxes are 128 x kb x planes.  Partial sums of p_c . q_c go to
// part[c * matvec_blocks(N, mode) + block].  The kernel returns at once when *stop
// is non-zero and sets *err when a copy never completes.
cudaError_t encode_planes(CUtensorMap* map, const float* base, int64_t ld, int64_t rows,
                          int64_t plane_stride, int nplanes, int box_rows);
unsigned matvec_blocks(int64_t N, int mode);
int matvec_pad(int kb);      // box rows of tmP for kb vectors (1, 2, 4, 8 or 16)
int matvec_rows(int mode);   // box rows of tmW (16 double-float, 32 FP32)
cudaError_t matvec_init();   // per device, before the first launch_matvec
// test hooks of the bounded waits (current device): 0 off
cudaError_t set_matvec_expire_ns(long long ns);
cudaError_t set_matvec_tc_expire_ns(long long ns);
// split > 1 divides the columns among split CTAs per row block (scratch of
// matvec_scratch_bytes; a second kernel adds the partials in split order).
cudaError_t launch_matvec(int mode, const CUtensorMap& tmW, const CUtensorMap& tmP, int64_t N, int kb,
                          const double* P, double* Q, double* part, const int* stop, int* err,
                          cudaStream_t s, int split = 1, void* scratch = nullptr);
int matvec_split(int64_t N, int mode);
size_t matvec_scratch_bytes(int64_t N, int kb, int split);
// the split this geometry's products use: the autotuned one, else the default
int matvec_split_of(const DevGeom& g, int mode);
// Autotuner: times the candidate column splits of both CUDA-core products on
// this geometry's W (16 vectors and 1 vector) and keeps the fastest in
// g.mv_split; results are cached per (device, N, mode) for the process.
cudaError_t matvec_autotune(DevGeom& g, cudaStream_t s);

// Q = W P on the tensor cores from integer slices of W and P (matvec_tc.cu);
// prec 0 double-float accuracy, 1 scaled FP16 (W to 11 bits under its row
// scale); same outputs and part layout as mode 0 of launch_matvec.
// ensure_w_slices makes the slices of W of that precision (once per
// assembly); work holds tc_work_bytes(g) of scratch.
cudaError_t ensure_w_slices(DevGeom& g, int prec, cudaStream_t s);
void drop_w_slices(DevGeom& g, cudaStream_t s);
size_t tc_slices_bytes(const DevGeom& g, int prec);
size_t tc_work_bytes(const DevGeom& g);
cudaError_t launch_matvec_tc(DevGeom& g, int prec, int kb, const double* P, double* Q, double* part,
                             const int* stop, int* err, void* work, cudaStream_t s);

// Preconditioner set-up (factor.cu).  factor_blocks = factor_gather +
// factor_invert + factor_finish for one geometry; a group of geometries
// gathers each into one InvPlan, inverts them all in one grouped sequence of
// launches and finishes each.
struct InvPlan {
  std::vector<double*> ptr;    // per matrix id: the n x n matrix, row-major
  std::vector<int64_t> size;   // per matrix id: n
  std::vector<int> owner;      // per matrix id: the tag given to factor_gather
  std::vector<int32_t> inv;    // the ids to invert in place
  std::vector<char> f32;       // per matrix id: inverted in FP32 (else double-float)
};
// prec32: the face and wire-basket blocks are inverted in FP32 (the coarse
// block stays double-float)
cudaError_t factor_gather(DevGeom& g, const std::vector<int64_t>& bptr, int wb_diag, cudaStream_t s,
                          InvPlan& plan, int owner, int prec32 = 0);
cudaError_t factor_invert(const InvPlan& plan, cudaMemPool_t pool, cudaStream_t s, std::vector<int>& bad,
                          int64_t* launches);
cudaError_t factor_finish(DevGeom& g, const std::vector<int64_t>& bptr, cudaStream_t s);
cudaError_t factor_blocks(DevGeom& g, const std::vector<int64_t>& bptr, int wb_diag,
                          cudaStream_t s, int* not_spd, int prec32 = 0);

// The rank-32 update of the double-float Gauss-Jordan recursion on the tensor
// cores (factor_tcp.cu): device pointers of one grouped inversion, matrices in
// sorted order (largest first); pl / pr / pt are prefixes over the sorted
// matrices of rows rounded up to 128, columns rounded up to tcp_tile_cols()
// and 128 x tcp_tile_cols() output tiles; Lsl / Rsl hold the digit tiles
// (tcp_slice_bytes(pl[nb], pr[nb]) bytes, Lsl first, Rsl at
// tcp_slice_bytes(pl[nb], 0)), exL / exR one exponent per padded row / column.
template <class Elem, class Op>
struct TcpDev {
  Elem* const* Ap;
  const int64_t* bsize;
  const int32_t* order;
  const int64_t* soff;
  const Op* Pf;
  const Op* Cf;
  const Op* Rf;
  const int64_t* pl;
  const int64_t* pr;
  const int64_t* pt;
  unsigned char* Lsl;
  unsigned char* Rsl;
  int* exL;
  int* exR;
  int* err;        // set to 1 when a bounded wait gave up
};
size_t tcp_slice_bytes(int64_t rows, int64_t cols);
int tcp_tile_cols();
cudaError_t tcp_init(int* sms);   // per device, before the first launch; *sms = SM count
// one step (pivot columns k0 ..) over the first `active` sorted matrices:
// rows = pl[active], cols = pr[active], tiles = pt[active]; three launches
cudaError_t launch_tcp_update(const TcpDev<double, float2>& d, int active, int64_t k0, int64_t rows, int64_t cols,
                              int64_t tiles, int sms, cudaStream_t s);

// Single-matrix blocked Gauss-Jordan inversion with caller-provided scratch
// (factor.cu); used by the allocation-free entry point.
size_t bgj_scratch_bytes(int64_t n);
cudaError_t bgj_invert_single(double* A, int64_t n, unsigned char* scratch, size_t bytes,
                              cudaStream_t s, int* not_spd);

struct PcgOut {
  int iters = 0;
  int status = 0;
  double err_est = 0.0;   // refinement with a density test: estimated relative error of the result
  std::vector<double> hist, alpha, beta;
};
// precision: 0 double-float matrix products (default), 1 the plain FP64
// comparator (FP64 copy of W, FP64 block inverses)
cudaError_t run_pcg(DevGeom& g, const double gvec[3], double rtol, int maxit, int fixed,
                    int precondition, int precision, double* x_out_dev, PcgOut& out, cudaStream_t s);
cudaError_t ensure_w64(DevGeom& g, cudaStream_t s);
void launch_gemv64(const DevGeom& g, const double* p, double* q, double* part, const int* stop, cudaStream_t s);
// Y = W X for kb <= 16 vectors (pcg_batch.cu); mode 0 double-float, 1 FP32 hi
// plane, 2 plain FP64, 3 double-float from integer slices on the tensor cores,
// 4 scaled FP16 on the tensor cores
cudaError_t apply_w(DevGeom& g, const double* X_in, bool in_dev, int kb, int mode, double* Y_out, bool out_dev,
                    float* kernel_ms, cudaStream_t s);
void drop_pcg_graphs(DevGeom& g);
// k <= 16 independent right-hand sides sharing the matrix-vector products
// (pcg_batch.cu); X_out is k x N (row c = density of g_c)
// (tensor: double-float products on the tensor cores)
cudaError_t run_pcg_batch(DevGeom& g, const double* gvecs, int kb, double rtol, int maxit, int fixed,
                          int precondition, double* X_out, bool out_on_device, std::vector<PcgOut>& outs,
                          cudaStream_t s, int tensor = 0);
// mixed precision: FP32 inner PCG inside double-float iterative refinement
// (pcg_batch.cu); *refinements receives the number of refinement steps
cudaError_t run_ir_batch(DevGeom& g, const double* gvecs, int kb, double rtol, int maxit, double inner_rtol,
                         int precondition, double* X_out, bool out_on_device, std::vector<PcgOut>& outs,
                         int* refinements, cudaStream_t s, int tensor = 0, int inner_fp16 = 0,
                         double density_tol = 0.0);

// double-layer potential at M targets (device arrays) from the jump values
// J[T][a] (host, 3 per triangle); refine: 4^refine sub-triangles (potential.cu)
cudaError_t dl_potential(DevGeom& g, const std::vector<double>& J, const double* X_dev, int64_t M, int refine,
                         double* out_dev, float* kernel_ms, cudaStream_t s);

// accessors of the opaque handles (api.cu)
DevGeom& msbem_geom_dev(msbem_geom* g);
int msbem_ctx_device(const msbem_ctx* c);

}  // namespace msbem
