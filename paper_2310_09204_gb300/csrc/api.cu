// C ABI of the msbem library (include/msbem.h): context and geometry handles,
// host topology at upload, orchestration of the device kernels.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <memory>
#include <mutex>
#include <thread>
#include <string>
#include <vector>

#include "msbem_internal.h"

using namespace msbem;

struct msbem_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  cudaStream_t cap_stream = nullptr;  // private stream for CUDA-graph capture
  cudaMemPool_t pool = nullptr;
  std::string err;
  std::vector<msbem_geom*> geoms;
  cudaEvent_t ev[8] = {};
};

struct msbem_geom {
  msbem_ctx* ctx = nullptr;
  Topo fine, coarse;
  Split split;
  DevGeom dev;
  std::vector<int64_t> bptr;
  int ss_order = 5;
};

namespace {

int fail(msbem_ctx* c, int status, const std::string& msg) {
  if (c) c->err = msg;
  return status;
}

int cuda_fail(msbem_ctx* c, cudaError_t e, const char* where) {
  if (e == cudaErrorMemoryAllocation)
    return fail(c, MSBEM_OOM, std::string(where) + ": out of device memory");
  if (e == cudaErrorTimeout)
    return fail(c, MSBEM_DEVICE_TIMEOUT, std::string(where) + ": a bounded device-side wait expired");
  return fail(c, MSBEM_CUDA_ERROR, std::string(where) + ": " + cudaGetErrorString(e));
}

template <class T>
cudaError_t dalloc(T** p, size_t n, cudaMemPool_t pool, cudaStream_t s) {
  return pool_alloc((void**)p, sizeof(T) * std::max<size_t>(n, 1), pool, s);
}

template <class T>
cudaError_t dput(T** p, const std::vector<T>& h, cudaMemPool_t pool, cudaStream_t s) {
  cudaError_t e = dalloc(p, h.size(), pool, s);
  if (e != cudaSuccess || h.empty()) return e;
  return cudaMemcpyAsync(*p, h.data(), sizeof(T) * h.size(), cudaMemcpyHostToDevice, s);
}

bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// freed memory a context's pool keeps for reuse beyond what is in use
constexpr uint64_t kPoolSpare = 8ull << 30;

void free_dev(DevGeom& d, cudaStream_t s) {
  drop_pcg_graphs(d);
  void* ptrs[] = {d.d_hist, d.d_qp, d.d_cen, d.d_qoff, d.d_area, d.d_tri, d.d_xyz, d.d_near, d.d_V,
                  d.d_jptr, d.d_jtri, d.d_jvec, d.d_jvecf, d.d_jrhs, d.d_Wh, d.d_bptr, d.d_bdofs, d.d_boff,
                  d.d_binv, d.d_pptr, d.d_pcol, d.d_pval, d.d_cptr, d.d_crow, d.d_cval, d.d_cvalf, d.d_pfp, d.d_rf, d.d_binvf,
                  d.d_btile, d.d_W64, d.d_wsl, d.d_wf16, d.d_wexp, d.d_cellZ, d.d_WP, d.d_vec, d.d_scal,
                  d.d_cendf, d.d_areadf};
  for (void* p : ptrs)
    if (p) cudaFreeAsync(p, s);
  cudaStreamSynchronize(s);
  d = DevGeom();
}

// Extreme eigenvalues of the symmetric tridiagonal (d, e) by Sturm bisection.
double sturm_count(const std::vector<double>& d, const std::vector<double>& e, double x) {
  int cnt = 0;
  double q = d[0] - x;
  if (q < 0) ++cnt;
  for (size_t i = 1; i < d.size(); ++i) {
    double qq = (q == 0.0) ? 1e-300 : q;
    q = d[i] - x - e[i - 1] * e[i - 1] / qq;
    if (q < 0) ++cnt;
  }
  return cnt;
}

double tridiag_kappa(const std::vector<double>& alpha, const std::vector<double>& beta) {
  const size_t m = alpha.size();
  if (m == 0) return NAN;
  std::vector<double> d(m), e(m > 1 ? m - 1 : 0);
  for (size_t j = 0; j < m; ++j) {
    d[j] = 1.0 / alpha[j] + (j > 0 ? beta[j - 1] / alpha[j - 1] : 0.0);
    if (j + 1 < m) e[j] = std::sqrt(beta[j]) / alpha[j];
  }
  double lo = 1e300, hi = -1e300;
  for (size_t j = 0; j < m; ++j) {  // Gershgorin bounds
    double r = (j > 0 ? std::fabs(e[j - 1]) : 0.0) + (j + 1 < m ? std::fabs(e[j]) : 0.0);
    lo = std::min(lo, d[j] - r);
    hi = std::max(hi, d[j] + r);
  }
  auto kth = [&](int k) {  // k-th smallest eigenvalue, 0-based
    double a = lo, b = hi;
    for (int it = 0; it < 200; ++it) {
      double mid = 0.5 * (a + b);
      if (sturm_count(d, e, mid) > k) b = mid; else a = mid;
      if (b - a <= 1e-15 * std::max(std::fabs(a), std::fabs(b))) break;
    }
    return 0.5 * (a + b);
  };
  return kth((int)m - 1) / kth(0);
}

}  // namespace

namespace msbem {
DevGeom& msbem_geom_dev(msbem_geom* g) { return g->dev; }
int msbem_ctx_device(const msbem_ctx* c) { return c->device; }
}  // namespace msbem

extern "C" {

int msbem_create(msbem_ctx** ctx, int device, void* stream) {
  if (!ctx) return MSBEM_INVALID_ARG;
  *ctx = nullptr;
  cudaError_t e = cudaSetDevice(device);
  if (e != cudaSuccess) return MSBEM_CUDA_ERROR;
  auto* c = new msbem_ctx();
  c->device = device;
  c->stream = (cudaStream_t)stream;
  for (auto& ev : c->ev) cudaEventCreate(&ev);
  if (cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    c->cap_stream = nullptr;
  }
  // a private stream-ordered pool that keeps freed memory for reuse
  cudaMemPoolProps props = {};
  props.allocType = cudaMemAllocationTypePinned;
  props.location.type = cudaMemLocationTypeDevice;
  props.location.id = device;
  if (cudaMemPoolCreate(&c->pool, &props) == cudaSuccess) {
    uint64_t keep = UINT64_MAX;
    cudaMemPoolSetAttribute(c->pool, cudaMemPoolAttrReleaseThreshold, &keep);
  } else {
    cudaGetLastError();
    c->pool = nullptr;
  }
  *ctx = c;
  return MSBEM_OK;
}

int msbem_destroy(msbem_ctx* c) {
  if (!c) return MSBEM_INVALID_ARG;
  cudaSetDevice(c->device);
  for (auto* g : c->geoms) {
    free_dev(g->dev, c->stream);
    delete g;
  }
  for (auto& ev : c->ev) cudaEventDestroy(ev);
  if (c->pool) {
    cudaStreamSynchronize(c->stream);
    cudaMemPoolDestroy(c->pool);
  }
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  delete c;
  return MSBEM_OK;
}

const char* msbem_last_error(const msbem_ctx* c) { return c ? c->err.c_str() : "null context"; }

int msbem_upload(msbem_ctx* c, const double* xyz, int64_t nv, const int32_t* tri, int64_t nt,
                 const double* cxyz, int64_t ncv, const int32_t* ctri, int64_t nct,
                 const int32_t* parent, const int32_t* patch, msbem_geom** out) {
  if (!c) return MSBEM_INVALID_ARG;
  if (!out || !xyz || !tri || !cxyz || !ctri || !parent || !patch || nv <= 0 || nt <= 0 ||
      ncv <= 0 || nct <= 0)
    return fail(c, MSBEM_INVALID_ARG, "msbem_upload: null pointer or empty mesh");
  *out = nullptr;
  cudaSetDevice(c->device);
  auto g = std::make_unique<msbem_geom>();
  g->ctx = c;
  std::string err;
  int st = build_topology(xyz, nv, tri, nt, g->fine, err);
  if (st) return fail(c, st, "fine mesh: " + err);
  // the near-pair list (read-only use of the fine topology) on a second host
  // thread while the cells, the coarse topology and the split are built
  std::vector<NearPair> near;
  std::thread near_th([&] { build_near_pairs(g->fine, near); });
  build_cells(g->fine);
  st = build_topology(cxyz, ncv, ctri, nct, g->coarse, err);
  if (st) err = "coarse mesh: " + err;
  else st = build_split(g->fine, g->coarse, parent, patch, g->split, err);
  near_th.join();
  if (st) return fail(c, st, err);
  const Topo& f = g->fine;
  const Split& sp = g->split;
  DevGeom& d = g->dev;
  cudaStream_t s = c->stream;
  d.pool = c->pool;
  d.cap_stream = c->cap_stream;
  d.nt = nt;
  d.nt_pad = (nt + 63) / 64 * 64;
  d.ndof = f.ndof;
  // triangle data: quadrature points, centroids, offsets
  double bary[6][3], w6[6];
  six_point_rule(bary, w6);
  std::vector<double> qp(d.nt_pad * 18, 0.0), cen(d.nt_pad * 3, 0.0), area(d.nt_pad, 0.0);
  std::vector<float> qoff(d.nt_pad * 36, 0.0f);
  std::vector<int32_t> tpad(d.nt_pad * 3, -1);
  // centroids and areas also as float pairs (the separated pairs of the far
  // field are formed in FP32 arithmetic alone)
  std::vector<float2> cendf(d.nt_pad * 3, make_float2(0.f, 0.f)), areadf(d.nt_pad, make_float2(0.f, 0.f));
  auto to_pair = [](double x) {
    const float hi = (float)x;
    return make_float2(hi, (float)(x - (double)hi));
  };
  for (int64_t T = 0; T < nt; ++T) {
    const double* X[3] = {&f.xyz[3 * f.tri[3 * T]], &f.xyz[3 * f.tri[3 * T + 1]],
                          &f.xyz[3 * f.tri[3 * T + 2]]};
    for (int k = 0; k < 3; ++k) cen[3 * T + k] = (X[0][k] + X[1][k] + X[2][k]) / 3.0;
    for (int p = 0; p < 6; ++p)
      for (int k = 0; k < 3; ++k) {
        double v = bary[p][0] * X[0][k] + bary[p][1] * X[1][k] + bary[p][2] * X[2][k];
        qp[T * 18 + 3 * p + k] = v;
        double off = v - cen[3 * T + k];
        float hi = (float)off;
        float lo = (float)(off - (double)hi);
        qoff[T * 36 + 6 * p + 2 * k] = hi;
        qoff[T * 36 + 6 * p + 2 * k + 1] = lo;
      }
    area[T] = f.area[T];
    for (int a = 0; a < 3; ++a) tpad[3 * T + a] = f.tri[3 * T + a];
    for (int k = 0; k < 3; ++k) cendf[3 * T + k] = to_pair(cen[3 * T + k]);
    areadf[T] = to_pair(area[T]);
  }
  // curl vectors s_{T,nu} = coef (x_{a+1} - x_{a+2}) / (2|T|) and RHS weights
  const int64_t ne = f.jptr[f.ndof];
  std::vector<double> jvec(3 * ne), jrhs(3 * ne);
  std::vector<float2> jvecf(3 * ne);
  for (int64_t k = 0; k < ne; ++k) {
    int64_t T = f.jtri[k];
    int a = f.jloc[k];
    const double* xa1 = &f.xyz[3 * f.tri[3 * T + (a + 1) % 3]];
    const double* xa2 = &f.xyz[3 * f.tri[3 * T + (a + 2) % 3]];
    for (int m = 0; m < 3; ++m) {
      jvec[3 * k + m] = f.jcoef[k] * (xa1[m] - xa2[m]) / (2.0 * f.area[T]);
      jrhs[3 * k + m] = f.jcoef[k] * f.area[T] / 3.0 * f.normal[3 * T + m];
      float hi = (float)jvec[3 * k + m];
      jvecf[3 * k + m] = make_float2(hi, (float)(jvec[3 * k + m] - (double)hi));
    }
  }
  // coarse prolongation in CSC form
  const int64_t NH = sp.n_coarse;
  std::vector<int64_t> cptr(NH + 1, 0);
  std::vector<int32_t> crow(sp.p_col.size());
  std::vector<double> cval(sp.p_col.size());
  for (int32_t col : sp.p_col) cptr[col + 1]++;
  for (int64_t m = 0; m < NH; ++m) cptr[m + 1] += cptr[m];
  {
    std::vector<int64_t> pos(cptr.begin(), cptr.end() - 1);
    for (int64_t r = 0; r < f.ndof; ++r)
      for (int64_t k = sp.p_ptr[r]; k < sp.p_ptr[r + 1]; ++k) {
        int64_t dst = pos[sp.p_col[k]]++;
        crow[dst] = (int32_t)r;
        cval[dst] = sp.p_val[k];
      }
  }
  g->bptr = sp.block_ptr;
  d.n_blocks = (int64_t)sp.block_ptr.size() - 1;
  d.n_coarse = NH;
  cudaError_t e = cudaSuccess;
  auto chk = [&](cudaError_t x) { if (e == cudaSuccess) e = x; };
  chk(dput(&d.d_qp, qp, c->pool, s));
  chk(dput(&d.d_cen, cen, c->pool, s));
  chk(dput(&d.d_qoff, qoff, c->pool, s));
  chk(dput(&d.d_area, area, c->pool, s));
  chk(dput(&d.d_cendf, cendf, c->pool, s));
  chk(dput(&d.d_areadf, areadf, c->pool, s));
  chk(dput(&d.d_tri, tpad, c->pool, s));
  chk(dput(&d.d_xyz, f.xyz, c->pool, s));
  d.n_near = (int64_t)near.size();
  {
    int64_t ident = 0;
    for (const NearPair& np : near) ident += (np.cls == 3);
    d.n_far_pairs = nt * (nt - 1) / 2 - (d.n_near - ident);
  }
  chk(dput(&d.d_near, near, c->pool, s));
  chk(dput(&d.d_jptr, f.jptr, c->pool, s));
  chk(dput(&d.d_jtri, f.jtri, c->pool, s));
  chk(dput(&d.d_jvec, jvec, c->pool, s));
  chk(dput(&d.d_jvecf, jvecf, c->pool, s));
  chk(dput(&d.d_jrhs, jrhs, c->pool, s));
  chk(dput(&d.d_bptr, sp.block_ptr, c->pool, s));
  chk(dput(&d.d_bdofs, sp.block_dofs, c->pool, s));
  chk(dput(&d.d_pptr, sp.p_ptr, c->pool, s));
  chk(dput(&d.d_pcol, sp.p_col, c->pool, s));
  chk(dput(&d.d_pval, sp.p_val, c->pool, s));
  chk(dput(&d.d_cptr, cptr, c->pool, s));
  chk(dput(&d.d_crow, crow, c->pool, s));
  chk(dput(&d.d_cval, cval, c->pool, s));
  {
    std::vector<float2> cvalf(cval.size());
    for (size_t k = 0; k < cval.size(); ++k) {
      float hi = (float)cval[k];
      cvalf[k] = make_float2(hi, (float)(cval[k] - (double)hi));
    }
    chk(dput(&d.d_cvalf, cvalf, c->pool, s));
  }
  const int64_t N = f.ndof;
  d.ncells = f.ncells;
  if (f.ncells) chk(dput(&d.d_cellZ, f.cellQ, c->pool, s));
  d.ldw = (N + 31) / 32 * 32;
  chk(dalloc(&d.d_Wh, (size_t)2 * N * d.ldw, c->pool, s));
  if (N > 0) chk(cudaMemsetAsync(d.d_Wh, 0, sizeof(float) * 2 * N * d.ldw, s));
  chk(dalloc(&d.d_WP, (size_t)std::max<int64_t>(NH, 1) * N, c->pool, s));
  chk(dalloc(&d.d_vec, (size_t)(5 * N + 2 * std::max<int64_t>(NH, 1) + 8), c->pool, s));
  chk(dalloc(&d.d_pfp, (size_t)2 * d.ldw, c->pool, s));
  if (N > 0) {
    chk(matvec_init());
    chk(cudaMemsetAsync(d.d_pfp, 0, sizeof(float) * 2 * d.ldw, s));
    chk(encode_planes(&d.tm_W, d.d_Wh, d.ldw, N, N * d.ldw, 2, matvec_rows(0)));
    chk(encode_planes(&d.tm_Whi, d.d_Wh, d.ldw, N, N * d.ldw, 1, matvec_rows(1)));
    chk(encode_planes(&d.tm_p, d.d_pfp, d.ldw, 1, d.ldw, 2, 1));
  }
  chk(dalloc(&d.d_rf, (size_t)N, c->pool, s));
  d.hist_cap = 1024;
  chk(dalloc(&d.d_hist, (size_t)(3 * d.hist_cap + 1), c->pool, s));
  chk(dalloc(&d.d_scal, (size_t)(16 + std::max<int64_t>(256, N / 8 + 8)), c->pool, s));
  chk(cudaStreamSynchronize(s));
  if (e != cudaSuccess) {
    free_dev(d, s);
    return cuda_fail(c, e, "msbem_upload");
  }
  c->geoms.push_back(g.get());
  *out = g.release();
  return MSBEM_OK;
}

int msbem_mesh_dofs(const double* xyz, int64_t nv, const int32_t* tri, int64_t nt, int64_t* ndof,
                    int32_t* vertex_of_dof, int32_t* sector_of_dof, int64_t cap, char* errbuf,
                    int errcap) {
  if (errbuf && errcap > 0) errbuf[0] = 0;
  if (!ndof) return MSBEM_INVALID_ARG;
  Topo t;
  std::string err;
  int st = build_topology(xyz, nv, tri, nt, t, err);
  if (st) {
    if (errbuf && errcap > 0) {
      std::strncpy(errbuf, err.c_str(), (size_t)errcap - 1);
      errbuf[errcap - 1] = 0;
    }
    return st;
  }
  *ndof = t.ndof;
  if (cap >= t.ndof) {
    if (vertex_of_dof) std::memcpy(vertex_of_dof, t.dof_vertex.data(), sizeof(int32_t) * t.ndof);
    if (sector_of_dof) std::memcpy(sector_of_dof, t.dof_sector.data(), sizeof(int32_t) * t.ndof);
  }
  return MSBEM_OK;
}

int msbem_mesh_cells(const double* xyz, int64_t nv, const int32_t* tri, int64_t nt, int* ncells, double* Z,
                     int64_t cap) {
  if (!ncells) return MSBEM_INVALID_ARG;
  Topo t;
  std::string err;
  int st = build_topology(xyz, nv, tri, nt, t, err);
  if (st) return st;
  build_cells(t);
  *ncells = t.ncells;
  if (Z && cap >= (int64_t)t.cellZ.size() && !t.cellZ.empty())
    std::memcpy(Z, t.cellZ.data(), sizeof(double) * t.cellZ.size());
  return MSBEM_OK;
}

int msbem_geom_free(msbem_geom* g) {
  if (!g) return MSBEM_INVALID_ARG;
  msbem_ctx* c = g->ctx;
  cudaSetDevice(c->device);
  free_dev(g->dev, c->stream);
  c->geoms.erase(std::remove(c->geoms.begin(), c->geoms.end(), g), c->geoms.end());
  delete g;
  return MSBEM_OK;
}

int msbem_ndofs(const msbem_geom* g, int64_t* n) {
  if (!g || !n) return MSBEM_INVALID_ARG;
  *n = g->fine.ndof;
  return MSBEM_OK;
}

int msbem_dof_map(const msbem_geom* g, int32_t* vertex_of_dof, int32_t* sector_of_dof) {
  if (!g) return MSBEM_INVALID_ARG;
  if (vertex_of_dof) std::memcpy(vertex_of_dof, g->fine.dof_vertex.data(), sizeof(int32_t) * g->fine.ndof);
  if (sector_of_dof) std::memcpy(sector_of_dof, g->fine.dof_sector.data(), sizeof(int32_t) * g->fine.ndof);
  return MSBEM_OK;
}

int msbem_split_info(const msbem_geom* g, int64_t* n_faces, int64_t* n_wb, int64_t* n_coarse,
                     int64_t* max_face) {
  if (!g) return MSBEM_INVALID_ARG;
  if (n_faces) *n_faces = g->split.n_faces;
  if (n_wb) *n_wb = g->split.n_wb;
  if (n_coarse) *n_coarse = g->split.n_coarse;
  if (max_face) *max_face = g->split.max_face;
  return MSBEM_OK;
}

int msbem_assemble(msbem_geom* g, const msbem_assemble_opts* opts) {
  if (!g) return MSBEM_INVALID_ARG;
  msbem_ctx* c = g->ctx;
  cudaSetDevice(c->device);
  int n = opts && opts->ss_order > 0 ? opts->ss_order : 5;
  int far_kernel = opts ? opts->far_kernel : 0;
  if (n < 2 || n > 16) return fail(c, MSBEM_INVALID_ARG, "ss_order must be in [2, 16]");
  if (far_kernel < 0 || far_kernel > 1) return fail(c, MSBEM_INVALID_ARG, "far_kernel must be 0 or 1");
  g->ss_order = n;
  DevGeom& d = g->dev;
  cudaStream_t s = c->stream;
  double bary[6][3], w6[6], glx[16], glw[16];
  six_point_rule(bary, w6);
  gauss_legendre01(n, glx, glw);
  // the 6-point rule is fixed: its weights go to the device's constant memory
  // once (assemblies of other contexts may be running on other threads)
  cudaError_t e = cudaSuccess;
  {
    static std::mutex mu;
    static std::vector<int> done;
    std::lock_guard<std::mutex> lock(mu);
    if (std::find(done.begin(), done.end(), c->device) == done.end()) {
      e = set_far_constants(bary, w6);
      if (e == cudaSuccess) e = set_far_df_constants(w6);
      if (e == cudaSuccess) done.push_back(c->device);
    }
  }
  if (e != cudaSuccess) return cuda_fail(c, e, "far constants");
  // W is rewritten from here on: until it is complete the geometry counts as
  // neither assembled nor factored (a failed assembly leaves it unusable)
  d.assembled = 0;
  d.factored = 0;
  // V (nt^2 float pairs) is scratch of the assembly only: taken from the pool
  // here and returned once W is formed, so a resident geometry holds W alone
  drop_pcg_graphs(d);
  if (d.d_W64) {  // the FP64 copy and the slices follow W
    cudaFreeAsync(d.d_W64, s);
    d.d_W64 = nullptr;
  }
  drop_w_slices(d, s);
  // V in one piece when it fits, else in row panels of triangles (a multiple
  // of 64 rows) computed and contracted one after the other
  int64_t panel = opts ? opts->panel_rows : 0;
  const int64_t nt_pad = d.nt_pad;
  if (panel <= 0) {
    size_t fr = 0, tot = 0;
    cudaMemGetInfo(&fr, &tot);
    uint64_t reserved = 0, used = 0;
    if (d.pool) {
      cudaMemPoolGetAttribute(d.pool, cudaMemPoolAttrReservedMemCurrent, &reserved);
      cudaMemPoolGetAttribute(d.pool, cudaMemPoolAttrUsedMemCurrent, &used);
    }
    const double avail = (double)fr + (double)(reserved > used ? reserved - used : 0);
    const double full = (double)sizeof(float2) * d.nt * d.nt;
    if (full > 0.8 * avail)
      panel = std::max<int64_t>(64, (int64_t)(0.6 * avail / (sizeof(float2) * (double)d.nt)) / 64 * 64);
  }
  const bool panels = panel > 0 && panel < nt_pad;
  if (panel % 64) return fail(c, MSBEM_INVALID_ARG, "panel_rows must be a multiple of 64");
  if (panels && far_kernel == 1)
    return fail(c, MSBEM_INVALID_ARG, "panel assembly uses the double-float pair kernel (far_kernel 0)");
  const int64_t vrows = panels ? panel : d.nt;
  // V, and 256 bytes after it for the far-field kernel's error flag
  const size_t vbytes = (sizeof(float2) * (size_t)std::max<int64_t>(1, vrows * d.nt) + 255) / 256 * 256;
  if (!d.d_V) {
    e = pool_alloc((void**)&d.d_V, vbytes + 256, d.pool, s);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(c, MSBEM_OOM, "assemble: no room for the pair matrix V");
    }
  }
  int* far_err = (int*)((char*)d.d_V + vbytes);
  if ((e = cudaMemsetAsync(far_err, 0, sizeof(int), s)) != cudaSuccess) return cuda_fail(c, e, "assemble");
  float t_far = 0.f, t_near = 0.f, t_con = 0.f;
  if (!panels) {
    cudaEventRecord(c->ev[0], s);
    e = (far_kernel == 1) ? launch_far_fp64(d, s) : launch_far_df(d, far_err, s);
    if (e != cudaSuccess) return cuda_fail(c, e, "far field");
    cudaEventRecord(c->ev[1], s);
    e = launch_near(d, n, glx, glw, far_kernel == 1, s);
    if (e != cudaSuccess) return cuda_fail(c, e, "near field");
    cudaEventRecord(c->ev[2], s);
    e = launch_contract(d, s);
    if (e != cudaSuccess) return cuda_fail(c, e, "contraction");
    cudaEventRecord(c->ev[3], s);
    d.launches += 1 + (d.n_near > 0) + (d.ndof > 0);
  } else {
    // dof rows each panel touches: the dofs of the vertices of its triangles
    const Topo& f = g->fine;
    const int64_t np = (d.nt + panel - 1) / panel;
    std::vector<int> rt0(np, INT32_MAX), rt1(np, -1);
    for (int64_t T = 0; T < d.nt; ++T) {
      const int64_t p = T / panel;
      for (int a = 0; a < 3; ++a) {
        const int32_t v = f.tri[3 * T + a];
        if (f.first_dof[v + 1] > f.first_dof[v]) {
          rt0[p] = std::min<int>(rt0[p], (int)(f.first_dof[v] / 32));
          rt1[p] = std::max<int>(rt1[p], (int)((f.first_dof[v + 1] - 1) / 32));
        }
      }
    }
    if (d.ndof > 0) e = cudaMemsetAsync(d.d_Wh, 0, sizeof(float) * 2 * d.ndof * d.ldw, s);
    std::vector<cudaEvent_t> evs(4 * np);
    for (auto& x : evs) cudaEventCreate(&x);
    for (int64_t p = 0; p < np && e == cudaSuccess; ++p) {
      const int64_t t0 = p * panel, t1 = std::min<int64_t>(d.nt, t0 + panel);
      cudaEventRecord(evs[4 * p], s);
      e = launch_far_df_panel(d, (int)(t0 / 64), (int)((std::min<int64_t>(nt_pad, t0 + panel) - t0) / 64),
                              far_err, s);
      cudaEventRecord(evs[4 * p + 1], s);
      if (e == cudaSuccess) e = launch_near(d, n, glx, glw, 0, s, t0, t1);
      cudaEventRecord(evs[4 * p + 2], s);
      if (e == cudaSuccess && rt1[p] >= rt0[p]) e = launch_contract_panel(d, t0, t1, rt0[p], rt1[p] - rt0[p] + 1, s);
      cudaEventRecord(evs[4 * p + 3], s);
      d.launches += 3;
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    for (int64_t p = 0; p < np && e == cudaSuccess; ++p) {
      float t;
      cudaEventElapsedTime(&t, evs[4 * p], evs[4 * p + 1]); t_far += t;
      cudaEventElapsedTime(&t, evs[4 * p + 1], evs[4 * p + 2]); t_near += t;
      cudaEventElapsedTime(&t, evs[4 * p + 2], evs[4 * p + 3]); t_con += t;
    }
    for (auto& x : evs) cudaEventDestroy(x);
    if (e != cudaSuccess) return cuda_fail(c, e, "panel assembly");
  }
  if (d.ncells > 0 && d.ndof > 0) {
    // closed cells: W + rho Q Q^T, rho = mean diag(W) (summed in dof order)
    std::vector<double> diag(d.ndof);
    double* dd = nullptr;
    e = pool_alloc((void**)&dd, sizeof(double) * d.ndof, d.pool, s);
    if (e == cudaSuccess) e = copy_diagonal(d, dd, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(diag.data(), dd, sizeof(double) * d.ndof, cudaMemcpyDeviceToHost, s);
    if (dd) cudaFreeAsync(dd, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(c, e, "cells");
    double sum = 0.0;
    for (double x : diag) sum += x;
    d.rho = sum / (double)d.ndof;
    if ((e = launch_augment(d, d.rho, s)) != cudaSuccess) return cuda_fail(c, e, "cells");
    ++d.launches;
  }
  int h_far_err = 0;
  e = cudaMemcpyAsync(&h_far_err, far_err, sizeof(int), cudaMemcpyDeviceToHost, s);
  cudaFreeAsync(d.d_V, s);
  d.d_V = nullptr;
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(c, e, "assemble");
  if (h_far_err) return fail(c, MSBEM_DEVICE_TIMEOUT, "assemble: a far-field staging copy did not complete");
  if (d.pool) {
    // the pool keeps at most kPoolSpare bytes of freed memory (V of the next
    // assembly of a similar geometry) beyond what is in use, so that the V of
    // a large geometry goes back to the device for other contexts
    uint64_t used = 0;
    cudaMemPoolGetAttribute(d.pool, cudaMemPoolAttrUsedMemCurrent, &used);
    cudaMemPoolTrimTo(d.pool, (size_t)(used + kPoolSpare));
  }
  if (!panels) {
    cudaEventElapsedTime(&t_far, c->ev[0], c->ev[1]);
    cudaEventElapsedTime(&t_near, c->ev[1], c->ev[2]);
    cudaEventElapsedTime(&t_con, c->ev[2], c->ev[3]);
  }
  d.times[0] = t_far;
  d.times[1] = t_near;
  d.times[2] = t_con;
  d.panel_rows = panels ? panel : 0;
  // column splits of the CUDA-core products for this W (timed once per
  // order N in the process); on any failure the N-only defaults stay
  if (matvec_autotune(d, s) != cudaSuccess) {
    cudaGetLastError();
    d.mv_split[0] = d.mv_split[1] = 0;
  }
  d.assembled = 1;
  d.factored = 0;
  return MSBEM_OK;
}

int msbem_copy_matrix(const msbem_geom* g, int64_t row0, int64_t nrows, double* out) {
  if (!g || !out) return MSBEM_INVALID_ARG;
  msbem_ctx* c = g->ctx;
  if (!g->dev.assembled) return fail(c, MSBEM_NOT_READY, "msbem_copy_matrix: not assembled");
  const int64_t N = g->fine.ndof;
  if (row0 < 0 || nrows < 0 || row0 + nrows > N) return fail(c, MSBEM_INVALID_ARG, "row range");
  cudaSetDevice(c->device);
  // W is held as (hi, lo) float pairs; convert rows to FP64 on the device
  double* tmp = nullptr;
  const bool dev_out = is_device_ptr(out);
  cudaError_t e = cudaSuccess;
  if (!dev_out)
    e = pool_alloc((void**)&tmp, sizeof(double) * std::max<int64_t>(1, nrows * N), c->pool, c->stream);
  if (e == cudaSuccess) e = copy_rows_to_double(g->dev, row0, nrows, dev_out ? out : tmp, c->stream);
  if (e == cudaSuccess && !dev_out)
    e = cudaMemcpyAsync(out, tmp, sizeof(double) * nrows * N, cudaMemcpyDeviceToHost, c->stream);
  if (tmp) cudaFreeAsync(tmp, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  return e == cudaSuccess ? MSBEM_OK : cuda_fail(c, e, "msbem_copy_matrix");
}

int msbem_rhs(const msbem_geom* g, const double gv[3], double* out) {
  if (!g || !gv || !out) return MSBEM_INVALID_ARG;
  msbem_ctx* c = g->ctx;
  cudaSetDevice(c->device);
  const int64_t N = g->fine.ndof;
  double* tmp = nullptr;
  cudaError_t e = pool_alloc((void**)&tmp, sizeof(double) * std::max<int64_t>(N, 1), c->pool, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "msbem_rhs");
  e = launch_rhs(g->dev, gv, tmp, c->stream);
  const_cast<msbem_geom*>(g)->dev.launches += (N > 0);
  if (e == cudaSuccess) e = cudaMemcpyAsync(out, tmp, sizeof(double) * N, cudaMemcpyDefault, c->stream);
  cudaFreeAsync(tmp, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  return e == cudaSuccess ? MSBEM_OK : cuda_fail(c, e, "msbem_rhs");
}

int msbem_factor(msbem_geom* g, const msbem_precond_opts* opts) {
  if (!g) return MSBEM_INVALID_ARG;
  msbem_ctx* c = g->ctx;
  if (!g->dev.assembled) return fail(c, MSBEM_NOT_READY, "msbem_factor: call msbem_assemble first");
  cudaSetDevice(c->device);
  DevGeom& d = g->dev;
  int wb_diag = opts ? opts->wire_basket : 0;
  if (wb_diag < 0 || wb_diag > 1) return fail(c, MSBEM_INVALID_ARG, "wire_basket must be 0 or 1");
  const int prec32 = opts ? opts->precision : 0;
  if (prec32 < 0 || prec32 > 1) return fail(c, MSBEM_INVALID_ARG, "precision must be 0 or 1");
  // nothing of the geometry changes before the options are checked: the old
  // inverses and their coarse layout stay usable after a rejected call
  d.use_coarse = opts ? (opts->use_coarse != 0) : 1;
  d.wb_diag = (g->split.n_wb > 0) ? 0 : -1;  // marks whether the last block is the wire basket
  d.factored = 0;      // until the new inverses are complete
  drop_pcg_graphs(d);  // the captured iterations address the old inverses
  cudaEventRecord(c->ev[4], c->stream);
  int not_spd = 0;
  cudaError_t e = factor_blocks(d, g->bptr, (g->split.n_wb > 0) ? wb_diag : 0, c->stream, &not_spd, prec32);
  if (e != cudaSuccess) return cuda_fail(c, e, "msbem_factor");
  const int nblk = (int)g->bptr.size() - 1;
  int64_t off = 0;
  for (int b = 0; b < nblk; ++b) off += (g->bptr[b + 1] - g->bptr[b]) * (g->bptr[b + 1] - g->bptr[b]);
  d.d_AHinv = d.d_binv + off;
  cudaEventRecord(c->ev[5], c->stream);
  cudaStreamSynchronize(c->stream);
  float t;
  cudaEventElapsedTime(&t, c->ev[4], c->ev[5]);
  d.times[3] = t;
  if (not_spd) return fail(c, MSBEM_BREAKDOWN, "msbem_factor: a block is not positive definite");
  d.factored = 1;
  return MSBEM_OK;
}

int msbem_factor_group(msbem_geom* const* geoms, int n, const msbem_precond_opts* opts, int* status) {
  if (!geoms || n < 1) return MSBEM_INVALID_ARG;
  for (int i = 0; i < n; ++i) {
    if (!geoms[i]) return MSBEM_INVALID_ARG;
    for (int j = 0; j < i; ++j)
      if (geoms[j] == geoms[i]) return fail(geoms[0]->ctx, MSBEM_INVALID_ARG, "msbem_factor_group: repeated geometry");
  }
  msbem_ctx* c = geoms[0]->ctx;
  for (int i = 0; i < n; ++i)
    if (geoms[i]->ctx != c) return fail(c, MSBEM_INVALID_ARG, "msbem_factor_group: geometries of different contexts");
  const int wb_diag = opts ? opts->wire_basket : 0;
  if (wb_diag < 0 || wb_diag > 1) return fail(c, MSBEM_INVALID_ARG, "wire_basket must be 0 or 1");
  const int prec32 = opts ? opts->precision : 0;
  if (prec32 < 0 || prec32 > 1) return fail(c, MSBEM_INVALID_ARG, "precision must be 0 or 1");
  for (int i = 0; i < n; ++i)
    if (!geoms[i]->dev.assembled) return fail(c, MSBEM_NOT_READY, "msbem_factor_group: call msbem_assemble first");
  cudaSetDevice(c->device);
  cudaEventRecord(c->ev[4], c->stream);
  InvPlan plan;
  for (int i = 0; i < n; ++i) {
    msbem_geom* g = geoms[i];
    DevGeom& d = g->dev;
    d.factored = 0;
    d.use_coarse = opts ? (opts->use_coarse != 0) : 1;
    d.wb_diag = (g->split.n_wb > 0) ? 0 : -1;
    drop_pcg_graphs(d);
    cudaError_t e = factor_gather(d, g->bptr, (g->split.n_wb > 0) ? wb_diag : 0, c->stream, plan, i, prec32);
    if (e != cudaSuccess) return cuda_fail(c, e, "msbem_factor_group");
  }
  std::vector<int> bad;
  cudaError_t e = factor_invert(plan, c->pool, c->stream, bad, &geoms[0]->dev.launches);
  if (e != cudaSuccess) return cuda_fail(c, e, "msbem_factor_group");
  std::vector<int> broke(n, 0);
  for (size_t m = 0; m < bad.size(); ++m)
    if (bad[m]) broke[plan.owner[m]] = 1;
  for (int i = 0; i < n; ++i) {
    msbem_geom* g = geoms[i];
    DevGeom& d = g->dev;
    if ((e = factor_finish(d, g->bptr, c->stream)) != cudaSuccess) return cuda_fail(c, e, "msbem_factor_group");
    const int nblk = (int)g->bptr.size() - 1;
    int64_t off = 0;
    for (int b = 0; b < nblk; ++b) off += (g->bptr[b + 1] - g->bptr[b]) * (g->bptr[b + 1] - g->bptr[b]);
    d.d_AHinv = d.d_binv + off;
  }
  cudaEventRecord(c->ev[5], c->stream);
  if ((e = cudaStreamSynchronize(c->stream)) != cudaSuccess) return cuda_fail(c, e, "msbem_factor_group");
  float t;
  cudaEventElapsedTime(&t, c->ev[4], c->ev[5]);
  int any = 0;
  for (int i = 0; i < n; ++i) {
    geoms[i]->dev.times[3] = t;
    geoms[i]->dev.factored = broke[i] ? 0 : 1;
    if (status) status[i] = broke[i] ? MSBEM_BREAKDOWN : MSBEM_OK;
    any |= broke[i];
  }
  if (any) return fail(c, MSBEM_BREAKDOWN, "msbem_factor_group: a block is not positive definite");
  return MSBEM_OK;
}

int msbem_spd_inverse_group(msbem_ctx* c, double* const* A, const int64_t* n, int count, int precision,
                            int* status) {
  if (!c || !A || !n || count < 1) return MSBEM_INVALID_ARG;
  if (precision < 0 || precision > 1) return fail(c, MSBEM_INVALID_ARG, "precision must be 0 or 1");
  InvPlan plan;
  for (int i = 0; i < count; ++i) {
    if (!A[i] || n[i] < 1) return fail(c, MSBEM_INVALID_ARG, "msbem_spd_inverse_group: NULL matrix or order < 1");
    plan.ptr.push_back(A[i]);
    plan.size.push_back(n[i]);
    plan.owner.push_back(i);
    plan.inv.push_back(i);
    plan.f32.push_back((char)precision);
  }
  cudaSetDevice(c->device);
  std::vector<int> bad;
  int64_t launches = 0;
  cudaError_t e = factor_invert(plan, c->pool, c->stream, bad, &launches);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "msbem_spd_inverse_group");
  int any = 0;
  for (int i = 0; i < count; ++i) {
    if (status) status[i] = bad[i] ? MSBEM_BREAKDOWN : MSBEM_OK;
    any |= bad[i];
  }
  if (any) return fail(c, MSBEM_BREAKDOWN, "msbem_spd_inverse_group: a matrix is not positive definite");
  return MSBEM_OK;
}

int msbem_solve(msbem_geom* g, const double gv[3], const msbem_solve_opts* opts, double* density,
                int* iters, double* hist, int hist_cap, double* kappa) {
  if (!g || !gv || !density) return MSBEM_INVALID_ARG;
  msbem_ctx* c = g->ctx;
  DevGeom& d = g->dev;
  double rtol = opts ? opts->rtol : 1e-8;
  int maxit = opts ? opts->maxit : 1000;
  int fixed = opts ? opts->fixed_iters : 0;
  int prec = opts ? opts->precondition : 1;
  const int precision = opts ? opts->precision : 0;
  const double inner = (opts && opts->inner_rtol > 0.0) ? opts->inner_rtol : 1e-4;
  const double dtol = opts ? opts->density_tol : 0.0;
  if (!(dtol >= 0.0 && dtol < 1.0)) return fail(c, MSBEM_INVALID_ARG, "density_tol must be in [0, 1)");
  if (!(rtol >= 0.0) || maxit < 1) return fail(c, MSBEM_INVALID_ARG, "rtol >= 0 and maxit >= 1 required");
  if (precision < 0 || precision > 5) return fail(c, MSBEM_INVALID_ARG, "precision must be 0 .. 5");
  if ((precision == 2 || precision >= 4) && (fixed || !(inner < 1.0)))
    return fail(c, MSBEM_INVALID_ARG, "mixed precision: no fixed_iters, inner_rtol < 1");
  if (!d.assembled) return fail(c, MSBEM_NOT_READY, "msbem_solve: not assembled");
  if (prec && !d.factored) return fail(c, MSBEM_NOT_READY, "msbem_solve: call msbem_factor first");
  cudaSetDevice(c->device);
  const int64_t N = g->fine.ndof;
  const bool dev_out = is_device_ptr(density);
  PcgOut po;
  cudaEventRecord(c->ev[6], c->stream);
  cudaError_t e;
  if (precision == 2 || precision >= 4) {
    std::vector<PcgOut> outs;
    e = run_ir_batch(d, gv, 1, rtol, maxit, inner, prec, d.d_vec, true, outs, nullptr, c->stream, precision >= 4,
                     precision == 5, dtol);
    if (e == cudaSuccess) po = outs[0];
  } else if (precision == 3) {
    std::vector<PcgOut> outs;
    e = run_pcg_batch(d, gv, 1, rtol, maxit, fixed, prec, d.d_vec, true, outs, c->stream, 1);
    if (e == cudaSuccess) po = outs[0];
  } else {
    e = run_pcg(d, gv, rtol, maxit, fixed, prec, precision, d.d_vec, po, c->stream);
  }
  if (e != cudaSuccess) return cuda_fail(c, e, "msbem_solve");
  e = cudaMemcpyAsync(density, d.d_vec, sizeof(double) * N,
                      dev_out ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream);
  cudaEventRecord(c->ev[7], c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "msbem_solve copy-out");
  float t;
  cudaEventElapsedTime(&t, c->ev[6], c->ev[7]);
  d.times[4] = t;
  if (iters) *iters = po.iters;
  if (hist && hist_cap > 0)
    for (int i = 0; i < hist_cap && i < (int)po.hist.size(); ++i) hist[i] = po.hist[i];
  if (kappa) *kappa = tridiag_kappa(po.alpha, po.beta);
  if (po.status == MSBEM_NOT_CONVERGED) return fail(c, po.status, "msbem_solve: maxit reached");
  if (po.status == MSBEM_BREAKDOWN) return fail(c, po.status, "msbem_solve: PCG breakdown");
  if (po.status == MSBEM_DEVICE_TIMEOUT)
    return fail(c, po.status, "msbem_solve: a matrix copy did not complete in time");
  return MSBEM_OK;
}

int msbem_counters(const msbem_geom* g, int64_t* launches, int64_t* far_pairs) {
  if (!g) return MSBEM_INVALID_ARG;
  if (launches) *launches = g->dev.launches;
  if (far_pairs) *far_pairs = g->dev.n_far_pairs;
  return MSBEM_OK;
}

int msbem_solve_batch(msbem_geom* g, const double* gvecs, int k, const msbem_solve_opts* opts,
                      double* density, int* iters, double* relres, double* kappa) {
  if (!g || !gvecs || !density || k < 1) return MSBEM_INVALID_ARG;
  msbem_ctx* c = g->ctx;
  DevGeom& d = g->dev;
  double rtol = opts ? opts->rtol : 1e-8;
  int maxit = opts ? opts->maxit : 1000;
  int fixed = opts ? opts->fixed_iters : 0;
  int prec = opts ? opts->precondition : 1;
  const int precision = opts ? opts->precision : 0;
  const double inner = (opts && opts->inner_rtol > 0.0) ? opts->inner_rtol : 1e-4;
  const double dtol = opts ? opts->density_tol : 0.0;
  if (!(dtol >= 0.0 && dtol < 1.0)) return fail(c, MSBEM_INVALID_ARG, "density_tol must be in [0, 1)");
  if (!(rtol >= 0.0) || maxit < 1) return fail(c, MSBEM_INVALID_ARG, "rtol >= 0 and maxit >= 1 required");
  if (precision < 0 || precision > 5) return fail(c, MSBEM_INVALID_ARG, "precision must be 0 .. 5");
  if ((precision == 2 || precision >= 4) && (fixed || !(inner < 1.0)))
    return fail(c, MSBEM_INVALID_ARG, "mixed precision: no fixed_iters, inner_rtol < 1");
  if (!d.assembled) return fail(c, MSBEM_NOT_READY, "msbem_solve_batch: not assembled");
  if (prec && !d.factored) return fail(c, MSBEM_NOT_READY, "msbem_solve_batch: call msbem_factor first");
  cudaSetDevice(c->device);
  const int64_t N = g->fine.ndof;
  const bool dev_out = is_device_ptr(density);
  int worst = MSBEM_OK;
  cudaEventRecord(c->ev[6], c->stream);
  for (int c0 = 0, kb = 0; c0 < k; c0 += kb) {
    kb = precision == 1 ? 1 : std::min(16, k - c0);
    std::vector<PcgOut> outs;
    cudaError_t e;
    if (precision == 1) {  // the plain comparator: one request at a time
      outs.resize(1);
      e = run_pcg(d, gvecs + 3 * c0, rtol, maxit, fixed, prec, 1, d.d_vec, outs[0], c->stream);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(density + (size_t)c0 * N, d.d_vec, sizeof(double) * N,
                            dev_out ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    } else if (precision == 2 || precision >= 4) {
      e = run_ir_batch(d, gvecs + 3 * c0, kb, rtol, maxit, inner, prec, density + (size_t)c0 * N, dev_out,
                       outs, nullptr, c->stream, precision >= 4, precision == 5, dtol);
    } else {
      e = run_pcg_batch(d, gvecs + 3 * c0, kb, rtol, maxit, fixed, prec, density + (size_t)c0 * N, dev_out,
                        outs, c->stream, precision == 3);
    }
    if (e != cudaSuccess) return cuda_fail(c, e, "msbem_solve_batch");
    for (int j = 0; j < kb; ++j) {
      const PcgOut& o = outs[j];
      if (iters) iters[c0 + j] = o.iters;
      if (relres) relres[c0 + j] = o.hist.empty() ? 0.0 : o.hist.back();
      if (kappa) kappa[c0 + j] = tridiag_kappa(o.alpha, o.beta);
      if (o.status == MSBEM_DEVICE_TIMEOUT) worst = MSBEM_DEVICE_TIMEOUT;
      else if (o.status == MSBEM_BREAKDOWN && worst != MSBEM_DEVICE_TIMEOUT) worst = MSBEM_BREAKDOWN;
      else if (o.status == MSBEM_NOT_CONVERGED && worst == MSBEM_OK) worst = MSBEM_NOT_CONVERGED;
    }
  }
  cudaEventRecord(c->ev[7], c->stream);
  cudaStreamSynchronize(c->stream);
  float t;
  cudaEventElapsedTime(&t, c->ev[6], c->ev[7]);
  d.times[4] = t;
  if (worst == MSBEM_DEVICE_TIMEOUT)
    return fail(c, worst, "msbem_solve_batch: a matrix copy did not complete in time");
  if (worst == MSBEM_BREAKDOWN) return fail(c, worst, "msbem_solve_batch: PCG breakdown");
  if (worst == MSBEM_NOT_CONVERGED) return fail(c, worst, "msbem_solve_batch: maxit reached");
  return MSBEM_OK;
}

int msbem_apply(msbem_geom* g, const double* X, int k, int precision, double* Y, double* kernel_ms) {
  if (!g || !X || !Y || k < 1 || k > 16 || precision < 0 || precision > 4) return MSBEM_INVALID_ARG;
  msbem_ctx* c = g->ctx;
  if (!g->dev.assembled) return fail(c, MSBEM_NOT_READY, "msbem_apply: not assembled");
  cudaSetDevice(c->device);
  // precision 0 -> kernel mode 0 (double-float), 1 -> plain FP64 copy, 2 -> FP32 hi plane,
  // 3 -> double-float from integer slices on the tensor cores, 4 -> scaled FP16 on the tensor cores
  const int mode = precision == 0 ? 0 : precision == 1 ? 2 : precision == 2 ? 1 : precision;
  float ms = 0.f;
  cudaError_t e = apply_w(g->dev, X, is_device_ptr(X), k, mode, Y, is_device_ptr(Y), &ms, c->stream);
  if (e == cudaErrorTimeout) return fail(c, MSBEM_DEVICE_TIMEOUT, "msbem_apply: a matrix copy did not complete");
  if (e != cudaSuccess) return cuda_fail(c, e, "msbem_apply");
  if (kernel_ms) *kernel_ms = ms;
  return MSBEM_OK;
}

int msbem_cells(const msbem_geom* g, int* ncells, double* Z, double* rho) {
  if (!g) return MSBEM_INVALID_ARG;
  if (ncells) *ncells = g->fine.ncells;
  if (Z && !g->fine.cellZ.empty()) std::memcpy(Z, g->fine.cellZ.data(), sizeof(double) * g->fine.cellZ.size());
  if (rho) *rho = g->dev.rho;
  return MSBEM_OK;
}

int msbem_dl_potential(msbem_geom* g, const double* density, const double* targets, int64_t M, int refine,
                       double* out, double* kernel_ms) {
  if (!g || !density || !targets || !out || M < 0 || refine < 0 || refine > 4) return MSBEM_INVALID_ARG;
  msbem_ctx* c = g->ctx;
  cudaSetDevice(c->device);
  const Topo& f = g->fine;
  const int64_t N = f.ndof;
  cudaStream_t s = c->stream;
  std::vector<double> phi(N);
  cudaError_t e = cudaMemcpy(phi.data(), density, sizeof(double) * N, cudaMemcpyDefault);
  if (e != cudaSuccess) return cuda_fail(c, e, "msbem_dl_potential density");
  // jump values J[T][a] from the curl lists, summed in list order
  std::vector<double> J(3 * f.nt, 0.0);
  for (int64_t nu = 0; nu < N; ++nu)
    for (int64_t k = f.jptr[nu]; k < f.jptr[nu + 1]; ++k) J[3 * f.jtri[k] + f.jloc[k]] += phi[nu] * f.jcoef[k];
  const bool xdev = is_device_ptr(targets), odev = is_device_ptr(out);
  double *dx = nullptr, *dout = nullptr;
  if (!xdev && (e = pool_alloc((void**)&dx, sizeof(double) * std::max<int64_t>(1, 3 * M), c->pool, s)) != cudaSuccess)
    return cuda_fail(c, e, "msbem_dl_potential");
  if (!odev && (e = pool_alloc((void**)&dout, sizeof(double) * std::max<int64_t>(1, M), c->pool, s)) != cudaSuccess) {
    if (dx) cudaFreeAsync(dx, s);
    return cuda_fail(c, e, "msbem_dl_potential");
  }
  if (!xdev) cudaMemcpyAsync(dx, targets, sizeof(double) * 3 * M, cudaMemcpyHostToDevice, s);
  float ms = 0.f;
  e = dl_potential(g->dev, J, xdev ? targets : dx, M, refine, odev ? out : dout, &ms, s);
  if (e == cudaSuccess && !odev) e = cudaMemcpyAsync(out, dout, sizeof(double) * M, cudaMemcpyDeviceToHost, s);
  if (dx) cudaFreeAsync(dx, s);
  if (dout) cudaFreeAsync(dout, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(c, e, "msbem_dl_potential");
  if (kernel_ms) *kernel_ms = ms;
  return MSBEM_OK;
}

int msbem_last_timings(const msbem_geom* g, double t[5]) {
  if (!g || !t) return MSBEM_INVALID_ARG;
  for (int i = 0; i < 5; ++i) t[i] = g->dev.times[i];
  return MSBEM_OK;
}


// ---- test hooks of the error paths ------------------------------------------
// (after + 1)-th pool allocation from now fails, once; -1: off
static std::atomic<long long> g_alloc_countdown{-1};

int msbem_test_fail_alloc(int64_t after) {
  if (after < -1) return MSBEM_INVALID_ARG;
  g_alloc_countdown.store(after);
  return MSBEM_OK;
}

int msbem_test_expire_waits(int64_t ns) {
  if (ns < 0) return MSBEM_INVALID_ARG;
  cudaError_t e = set_matvec_expire_ns((long long)ns);
  if (e == cudaSuccess) e = set_matvec_tc_expire_ns((long long)ns);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  return e == cudaSuccess ? MSBEM_OK : MSBEM_CUDA_ERROR;
}

}  // extern "C"

namespace msbem {

bool test_alloc_fails() {
  long long v = g_alloc_countdown.load(std::memory_order_relaxed);
  while (v >= 0) {
    // v == 0: this allocation fails and the hook turns itself off
    if (g_alloc_countdown.compare_exchange_weak(v, v - 1)) return v == 0;
  }
  return false;
}

}  // namespace msbem
