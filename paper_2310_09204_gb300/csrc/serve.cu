// Serving engine: solve requests (geometry key, Neumann data g) arriving over
// time are answered from geometries kept resident on the device (W, the
// factored preconditioner M(H;h) and a 16-slot batch of PCG vectors per
// geometry), admitted against an HBM budget with least-recently-used
// eviction of idle geometries.
//
// Continuous batching: every resident geometry runs its own multi-vector PCG
// on its own CUDA stream, so the iterations of different geometries overlap
// on the device.  Every `chunk` iterations the engine looks at the per-slot
// states: finished slots are harvested and refilled at once from the
// geometry's queue; a new request joins the running batch without disturbing
// the other slots (every per-slot sum runs in the same order whatever the
// batch holds, so each result is bit for bit the one it gets alone).
//
// precision 0 (3): each slot runs the double-float PCG of msbem_solve_batch
// (with the tensor-core products).
// precision 2 (4, 5): each slot runs the iterative refinement of the mixed
// mode -- inner PCG with FP32 products (FP32, scaled FP16 on the tensor
// cores) to inner_rtol, then X += D and the true residual R = L - W X with
// the double-float product (on the tensor cores); the slot finishes when
// ||R|| <= rtol ||L||, else restarts its inner solve on R.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cmath>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "batch.cuh"
#include "df.cuh"

using namespace msbem;

namespace msbem {

// ---- column-masked kernels (mask[c] != 0 selects column c) -----------------
__global__ void s_copy_cols(double* __restrict__ dst, const double* __restrict__ src, int64_t N, int kb,
                            const int* __restrict__ mask) {
  for (int64_t e = (int64_t)blockIdx.x * 256 + threadIdx.x; e < N * kb; e += (int64_t)gridDim.x * 256)
    if (mask[e % kb]) dst[e] = src ? src[e] : 0.0;
}

__global__ void s_axpy_cols(double* __restrict__ X, const double* __restrict__ D, int64_t N, int kb,
                            const int* __restrict__ mask) {
  for (int64_t e = (int64_t)blockIdx.x * 256 + threadIdx.x; e < N * kb; e += (int64_t)gridDim.x * 256)
    if (mask[e % kb]) X[e] += D[e];
}

__global__ void s_resid_cols(const double* __restrict__ L, const double* __restrict__ Q, double* __restrict__ R,
                             int64_t N, int kb, const int* __restrict__ mask) {
  for (int64_t e = (int64_t)blockIdx.x * 256 + threadIdx.x; e < N * kb; e += (int64_t)gridDim.x * 256)
    if (mask[e % kb]) R[e] = L[e] - Q[e];
}

// R[i][c] = L_c[i] for the masked columns (constant data g_c)
__global__ void s_rhs_cols(const int64_t* __restrict__ jptr, const double* __restrict__ jrhs, int64_t N,
                           const double* __restrict__ gv, int kb, const int* __restrict__ mask,
                           double* __restrict__ L) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= N * kb) return;
  const int64_t i = e / kb;
  const int c = (int)(e % kb);
  if (!mask[c]) return;
  double acc = 0.0;
  for (int64_t k = jptr[i]; k < jptr[i + 1]; ++k)
    acc += jrhs[3 * k] * gv[3 * c] + jrhs[3 * k + 1] * gv[3 * c + 1] + jrhs[3 * k + 2] * gv[3 * c + 2];
  L[e] = acc;
}

// fixed-order sum of a masked column's partials into a ColState field
__global__ void s_reduce_cols(const double* __restrict__ part, int nparts, ColState* cs, int field,
                              const int* __restrict__ mask) {
  __shared__ double sm[256];
  const int c = blockIdx.x;
  if (!mask[c]) return;
  double acc = 0.0;
  for (int i = threadIdx.x; i < nparts; i += 256) acc += part[(int64_t)c * nparts + i];
  sm[threadIdx.x] = acc;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) sm[threadIdx.x] += sm[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *(double*)((char*)&cs[c] + field) = sm[0];
}

// P_c = Z_c (first search direction) and its float-pair planes, masked columns
__global__ void s_setp_cols(double* __restrict__ P, float* __restrict__ Pf, int64_t ldp,
                            const double* __restrict__ Z, int64_t N, int kb, const int* __restrict__ mask) {
  for (int64_t e = (int64_t)blockIdx.x * 256 + threadIdx.x; e < N * kb; e += (int64_t)gridDim.x * 256) {
    const int64_t i = e / kb;
    const int c = (int)(e - i * kb);
    if (!mask[c]) continue;
    const double v = Z[e];
    P[e] = v;
    float h, l;
    split_df(v, h, l);
    Pf[(int64_t)c * ldp + i] = h;
    Pf[(int64_t)(kb + c) * ldp + i] = l;
  }
}

// masked columns start their recursion: iteration 0, running unless no data
__global__ void s_start_cols(ColState* cs, int kb, const int* __restrict__ mask) {
  const int c = threadIdx.x;
  if (c >= kb || !mask[c]) return;
  cs[c].iter = 0;
  cs[c].done = cs[c].nL2 == 0.0 ? 4 : 0;
}

// out = column c of X (N x kb)
__global__ void s_gather_col(const double* __restrict__ X, int64_t N, int kb, int c, double* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < N) out[i] = X[i * kb + c];
}

}  // namespace msbem

// ---------------------------------------------------------------------------
// host engine
// ---------------------------------------------------------------------------
namespace {

double now_s() {
  using namespace std::chrono;
  return duration<double>(steady_clock::now().time_since_epoch()).count();
}

enum SlotPhase { IDLE = 0, INNER = 1 };

struct Request {
  uint64_t id = 0, key = 0;
  double g[3] = {0, 0, 0};
  double* out = nullptr;
  double t_arrival = 0.0, t_done = -1.0;
  int status = 1;          // 1 = pending (not finished yet)
  int iters = 0;
  int refinements = 0;
  double relres = NAN;
};

struct Slot {
  uint64_t req = 0;        // 0 = free
  int phase = IDLE;
  int inner_total = 0;
  int refinements = 0;
  double nL = 0.0;         // ||L_c||^2
  double dprev = 0.0;      // ||D|| of the previous refinement step (density test)
};

struct Batch {
  cudaStream_t s = nullptr;
  cudaEvent_t ev = nullptr;
  char* base = nullptr;
  size_t bytes = 0;
  BatchBuffers b{};
  double *L = nullptr, *Xo = nullptr, *Ro = nullptr, *nrm = nullptr, *out = nullptr;
  float* Xf = nullptr;
  int* mask = nullptr;
  char* scratch = nullptr;
  BatchState* fl = nullptr;        // all_done = 0 flags for the utility kernels
  CUtensorMap tmP, tmX;
  int split = 1;
  ColState* h_cs = nullptr;        // pinned snapshots
  double* h_nrm = nullptr;
  int* h_mask = nullptr;
  BatchState* h_bs = nullptr;
  bool in_flight = false;
  // the `chunk` PCG iterations of a scheduling point, captured once as a CUDA
  // graph (the batch's buffers, split and mode never change) and replayed
  cudaGraphExec_t iter_exec = nullptr;
  Slot slot[BK];
};

// life cycle of a geometry in the engine
enum GeomState { G_OUT = 0, G_ADMITTING = 1, G_READY = 2, G_FAILED = 3, G_EVICTING = 4 };

struct GeomEntry {
  uint64_t key = 0;
  std::atomic<int> state{G_OUT};   // written by the admission thread, read by progress()
  int admit_status = 0;
  size_t reserved = 0;             // budget bytes held while admitting
  int owner = -1;                  // admission thread (context) holding the geometry
  std::vector<double> xyz, cxyz;
  std::vector<int32_t> tri, ctri, parent, patch;
  int64_t ndof = -1, nt = 0;
  size_t footprint = 0;    // resident bytes (W, preconditioner, batch)
  msbem_geom* geom = nullptr;
  std::unique_ptr<Batch> batch;
  std::deque<uint64_t> pending;
  double last_used = 0.0;
  int active = 0;          // busy slots
};

}  // namespace

struct msbem_server {
  msbem_ctx* ctx = nullptr;
  msbem_server_opts opts{};
  int device = 0;
  std::unordered_map<uint64_t, std::unique_ptr<GeomEntry>> geoms;
  std::unordered_map<uint64_t, Request> reqs;
  uint64_t next_id = 1;
  size_t resident = 0;             // bytes of resident + admitting geometries
  msbem_server_stats st{};
  // admission threads: each uploads, assembles and factors new geometries (and
  // frees the evicted ones it admitted) on its own context and stream, so the
  // PCG iterations of the resident geometries keep running meanwhile and the
  // host topology of one geometry overlaps the GPU assembly of another
  struct Worker {
    msbem_ctx* ctx = nullptr;
    cudaStream_t stream = nullptr;
    std::thread th;
    std::deque<std::pair<int, GeomEntry*>> tasks;   // (1 admit | 2 evict, entry)
    int queued_admissions = 0;
  };
  std::vector<std::unique_ptr<Worker>> workers;
  std::mutex mu;
  std::condition_variable cv;
  bool stop = false;
  // admission work (under mu) and kernels of released geometries
  double far_ms = 0.0, assemble_ms = 0.0, factor_ms = 0.0;
  int64_t far_pairs = 0, launches_released = 0;
};

namespace {

constexpr int kSlots = BK;

bool is_mixed(int precision) { return precision == 2 || precision == 4 || precision == 5; }
bool tc_residual(int precision) { return precision >= 3; }   // double-float products on the tensor cores
// the product mode of the slots' PCG iterations (enqueue_batch_iteration)
int inner_mode(int precision) {
  return precision == 0 ? 0 : precision == 3 ? 3 : precision == 5 ? 4 : 1;
}

size_t estimate_footprint(const GeomEntry& e, int precision) {
  const size_t N = (size_t)std::max<int64_t>(e.ndof, 1);
  const size_t ldw = (N + 31) / 32 * 32;
  // W planes, FP64 + float-pair block inverses (faces of ~600 dofs at most plus
  // a wire basket of ~sqrt(N) * 12 dofs, a bound), coarse scratch, batch vectors
  const size_t wb = (size_t)(12.0 * std::sqrt((double)N)) + 64;
  const size_t blocks = 16 * (N * 600 + wb * wb);
  const size_t batch = sizeof(double) * N * kSlots * 12 + sizeof(float) * 4 * kSlots * ldw;
  // integer slices of W for the tensor-core products (bf16: 12 bytes an
  // entry, fp16: 2), on padded 8 x 64 tiles
  const size_t tiles = ((N + 7) / 8 * 8) * ((N + 63) / 64 * 64);
  const size_t slices = (tc_residual(precision) ? 12 * tiles + 4 * N : 0) + (precision == 5 ? 2 * tiles : 0);
  return 8 * N * ldw + blocks + 8 * N * 64 + batch + slices + (2u << 20);
}

size_t transient_bytes(const GeomEntry& e) { return sizeof(float2) * (size_t)e.nt * e.nt; }

void free_batch(Batch* B) {
  if (!B) return;
  if (B->s) cudaStreamSynchronize(B->s);
  if (B->iter_exec) cudaGraphExecDestroy(B->iter_exec);
  B->iter_exec = nullptr;
  if (B->base) cudaFreeAsync(B->base, B->s);
  if (B->s) cudaStreamSynchronize(B->s);
  if (B->h_cs) cudaFreeHost(B->h_cs);
  if (B->ev) cudaEventDestroy(B->ev);
  if (B->s) cudaStreamDestroy(B->s);
}

int alloc_batch(msbem_server* S, GeomEntry& e) {
  DevGeom& g = msbem_geom_dev(e.geom);
  const int64_t N = g.ndof;
  const int kb = kSlots;
  auto B = std::make_unique<Batch>();
  if (cudaStreamCreateWithFlags(&B->s, cudaStreamNonBlocking) != cudaSuccess) return MSBEM_CUDA_ERROR;
  cudaEventCreateWithFlags(&B->ev, cudaEventDisableTiming);
  const int maxit = S->opts.maxit;
  const int64_t NH = std::max<int64_t>(g.n_coarse, 1);
  const size_t nvec = (size_t)N * kb;
  const size_t nparts = (size_t)kb * std::max<unsigned>(matvec_blocks(N, 0), BRED);
  const size_t hsz = (size_t)kb * (maxit + 1) + 2 * (size_t)kb * maxit;
  B->split = std::max(matvec_split_of(g, 0), matvec_split_of(g, 1));
  const int prec = S->opts.precision;
  size_t scr = matvec_scratch_bytes(N, kb, B->split);
  if (tc_residual(prec)) {
    // the slices of W, made here on the admission thread's context
    cudaError_t ce = ensure_w_slices(g, 0, B->s);
    if (ce == cudaSuccess && prec == 5) ce = ensure_w_slices(g, 1, B->s);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(B->s);
    if (ce != cudaSuccess) {
      cudaGetLastError();
      free_batch(B.get());
      return ce == cudaErrorMemoryAllocation ? MSBEM_OOM : MSBEM_CUDA_ERROR;
    }
    scr = std::max(scr, tc_work_bytes(g));
  }
  B->bytes = sizeof(double) * (8 * nvec + 2 * NH * kb + nparts + hsz + 3 * kb + 4 * kb + N) +
             sizeof(float) * 4 * kb * g.ldw + sizeof(float2) * nvec + sizeof(ColState) * kb +
             2 * sizeof(BatchState) + sizeof(int) * kb + scr + 1024;
  if (pool_alloc((void**)&B->base, B->bytes, g.pool, B->s) != cudaSuccess) {
    cudaGetLastError();
    free_batch(B.get());
    return MSBEM_OOM;
  }
  Carver cv{B->base};
  BatchBuffers& b = B->b;
  b.X = cv.take<double>(nvec);      // inner iterate (the correction D in the mixed mode)
  b.R = cv.take<double>(nvec);      // inner residual
  b.Z = cv.take<double>(nvec);
  b.P = cv.take<double>(nvec);
  b.Q = cv.take<double>(nvec);
  b.T = cv.take<double>(NH * kb);
  b.U = cv.take<double>(NH * kb);
  b.part = cv.take<double>(nparts);
  b.hist = cv.take<double>(hsz);
  b.gv = cv.take<double>(3 * kb);
  b.Pf = cv.take<float>(2 * kb * g.ldw);
  b.Rf = cv.take<float2>(nvec);
  b.cs = cv.take<ColState>(kb);
  b.bs = cv.take<BatchState>(1);
  B->L = cv.take<double>(nvec);
  B->Xo = cv.take<double>(nvec);
  B->Ro = cv.take<double>(nvec);
  B->nrm = cv.take<double>(4 * kb);     // ||.||^2 of R, L | D | X per column
  B->out = cv.take<double>(N);
  B->Xf = cv.take<float>(2 * kb * g.ldw);
  B->mask = cv.take<int>(kb);
  B->fl = cv.take<BatchState>(1);
  B->scratch = cv.take<char>(scr);
  cudaError_t ce = encode_planes(&B->tmP, b.Pf, g.ldw, kb, kb * g.ldw, inner_mode(prec) == 1 ? 1 : 2,
                                 matvec_pad(kb));
  if (ce == cudaSuccess) ce = encode_planes(&B->tmX, B->Xf, g.ldw, kb, kb * g.ldw, 2, matvec_pad(kb));
  // pinned snapshots: ColState[kb], nrm[4kb], mask[kb], BatchState
  void* pin = nullptr;
  if (ce == cudaSuccess)
    ce = cudaMallocHost(&pin, sizeof(ColState) * kb + sizeof(double) * 4 * kb + sizeof(int) * kb +
                                  sizeof(BatchState) + 64);
  if (ce != cudaSuccess) {
    cudaGetLastError();
    free_batch(B.get());
    return MSBEM_CUDA_ERROR;
  }
  B->h_cs = (ColState*)pin;
  B->h_nrm = (double*)(B->h_cs + kb);
  B->h_mask = (int*)(B->h_nrm + 4 * kb);
  B->h_bs = (BatchState*)(B->h_mask + kb);
  for (int c = 0; c < kb; ++c) B->h_cs[c] = ColState{0, 0, 0, 0, 0, 0, 0, 6, 0, 0, 0};
  const double inner = is_mixed(prec) ? S->opts.inner_rtol : S->opts.rtol;
  *B->h_bs = BatchState{1, kb, maxit, 0, inner, 0};
  cudaMemsetAsync(B->base, 0, B->bytes, B->s);
  cudaMemcpyAsync(b.cs, B->h_cs, sizeof(ColState) * kb, cudaMemcpyHostToDevice, B->s);
  cudaMemcpyAsync(b.bs, B->h_bs, sizeof(BatchState), cudaMemcpyHostToDevice, B->s);
  if (cudaStreamSynchronize(B->s) != cudaSuccess) {
    free_batch(B.get());
    return MSBEM_CUDA_ERROR;
  }
  e.batch = std::move(B);
  return MSBEM_OK;
}

// on the admission thread (or at destruction, after the threads have ended)
void release_geometry(msbem_server* S, GeomEntry& e) {
  free_batch(e.batch.get());
  e.batch.reset();
  if (e.geom) {
    const int64_t n = msbem_geom_dev(e.geom).launches;
    {
      std::lock_guard<std::mutex> lock(S->mu);
      S->launches_released += n;
    }
    msbem_geom_free(e.geom);
  }
  e.geom = nullptr;
}

int admit_now(msbem_server* S, msbem_ctx* actx, GeomEntry& e) {
  msbem_geom* g = nullptr;
  int st = msbem_upload(actx, e.xyz.data(), (int64_t)e.xyz.size() / 3, e.tri.data(), (int64_t)e.tri.size() / 3,
                        e.cxyz.data(), (int64_t)e.cxyz.size() / 3, e.ctri.data(), (int64_t)e.ctri.size() / 3,
                        e.parent.data(), e.patch.data(), &g);
  if (st) return st;
  // the mixed precisions' inner PCG reads FP32 block inverses: invert in FP32
  const msbem_precond_opts po{0, 1, is_mixed(S->opts.precision) ? 1 : 0};
  if ((st = msbem_assemble(g, nullptr)) || (st = msbem_factor(g, &po))) {
    msbem_geom_free(g);
    return st;
  }
  {
    const DevGeom& d = msbem_geom_dev(g);
    std::lock_guard<std::mutex> lock(S->mu);
    S->far_ms += d.times[0];
    S->assemble_ms += (double)d.times[0] + d.times[1] + d.times[2];
    S->factor_ms += d.times[3];
    S->far_pairs += d.n_far_pairs;
  }
  e.geom = g;
  if ((st = alloc_batch(S, e))) {
    msbem_geom_free(g);
    e.geom = nullptr;
    return st;
  }
  DevGeom& d = msbem_geom_dev(g);
  const size_t NH = (size_t)std::max<int64_t>(d.n_coarse, 1);
  const int prec = S->opts.precision;
  e.footprint = sizeof(float) * 2 * (size_t)d.ndof * d.ldw + (sizeof(double) + sizeof(float2)) * d.binv_size +
                sizeof(double) * (NH * d.ndof + 8 * (size_t)d.ndof) + e.batch->bytes +
                (tc_residual(prec) ? tc_slices_bytes(d, 0) : 0) + (prec == 5 ? tc_slices_bytes(d, 1) : 0);
  return MSBEM_OK;
}

void admission_thread(msbem_server* S, int w) {
  cudaSetDevice(S->device);
  msbem_server::Worker& W = *S->workers[w];
  for (;;) {
    std::pair<int, GeomEntry*> t;
    {
      std::unique_lock<std::mutex> lock(S->mu);
      S->cv.wait(lock, [S, &W] { return S->stop || !W.tasks.empty(); });
      if (W.tasks.empty()) return;          // stop requested and nothing left
      t = W.tasks.front();
      W.tasks.pop_front();
    }
    GeomEntry& e = *t.second;
    if (t.first == 2) {
      release_geometry(S, e);
      e.state.store(G_OUT);
    } else {
      const int st = admit_now(S, W.ctx, e);
      e.admit_status = st;
      {
        std::lock_guard<std::mutex> lock(S->mu);
        --W.queued_admissions;
      }
      e.state.store(st == MSBEM_OK ? G_READY : G_FAILED);
    }
  }
}

// admissions go to the thread with the fewest queued, evictions to the thread
// that owns the geometry
void post(msbem_server* S, int kind, GeomEntry* e) {
  {
    std::lock_guard<std::mutex> lock(S->mu);
    int w = e->owner;
    if (kind == 1) {
      w = 0;
      for (int i = 1; i < (int)S->workers.size(); ++i)
        if (S->workers[i]->queued_admissions < S->workers[w]->queued_admissions) w = i;
      e->owner = w;
      ++S->workers[w]->queued_admissions;
    }
    S->workers[w]->tasks.emplace_back(kind, e);
  }
  S->cv.notify_all();
}

// make room for `need` bytes by evicting idle resident geometries, least
// recently used first (the frees run on the admission thread, queued before
// the admission that needs the room)
bool make_room(msbem_server* S, size_t need) {
  while (S->resident + need > (size_t)S->opts.hbm_budget_bytes) {
    GeomEntry* victim = nullptr;
    for (auto& kv : S->geoms) {
      GeomEntry& e = *kv.second;
      if (e.state.load() != G_READY || e.active > 0 || !e.pending.empty()) continue;
      if (!victim || e.last_used < victim->last_used) victim = &e;
    }
    if (!victim) return false;
    victim->state.store(G_EVICTING);
    S->resident -= std::min(S->resident, victim->footprint);
    ++S->st.evictions;
    post(S, 2, victim);
  }
  return true;
}

void finish(msbem_server* S, GeomEntry& e, int c, int status, int iters, double relres, const double* src_cols) {
  Batch& B = *e.batch;
  Slot& sl = B.slot[c];
  Request& r = S->reqs[sl.req];
  DevGeom& g = msbem_geom_dev(e.geom);
  const int64_t N = g.ndof;
  s_gather_col<<<(unsigned)((N + 255) / 256), 256, 0, B.s>>>(src_cols, N, kSlots, c, B.out);
  if (r.out) cudaMemcpyAsync(r.out, B.out, sizeof(double) * N, cudaMemcpyDefault, B.s);
  cudaStreamSynchronize(B.s);
  r.status = status;
  r.iters = iters;
  r.relres = relres;
  r.refinements = sl.refinements;
  r.t_done = now_s();
  sl = Slot();
  B.h_cs[c].done = 6;
  --e.active;
  ++S->st.completed;
}

// one scheduling point of a resident geometry whose batch is not in flight
void schedule(msbem_server* S, GeomEntry& e) {
  Batch& B = *e.batch;
  DevGeom& g = msbem_geom_dev(e.geom);
  const int64_t N = g.ndof;
  const int kb = kSlots;
  const int prec = S->opts.precision;
  const bool mixed = is_mixed(prec);
  const unsigned grid = kStrideBlocks;
  const dim3 rgrid(BRED, kb);
  cudaStream_t s = B.s;
  // 1. slots whose inner recursion stopped
  std::vector<int> refine;
  for (int c = 0; c < kb; ++c) {
    Slot& sl = B.slot[c];
    if (sl.phase != INNER) continue;
    const ColState& cs = B.h_cs[c];
    if (cs.done == 0) continue;
    sl.inner_total += cs.iter;
    const double rel = cs.nL2 > 0.0 ? std::sqrt(cs.rr / cs.nL2) : 0.0;
    if (!mixed) {
      const int status = cs.done == 1 || cs.done == 4 ? MSBEM_OK
                       : cs.done == 2 ? MSBEM_BREAKDOWN
                       : cs.done == 5 ? MSBEM_DEVICE_TIMEOUT
                                      : MSBEM_NOT_CONVERGED;
      finish(S, e, c, status, sl.inner_total, cs.done == 4 ? 0.0 : rel, B.b.X);
    } else if (cs.done == 2 || cs.done == 5) {
      finish(S, e, c, cs.done == 2 ? MSBEM_BREAKDOWN : MSBEM_DEVICE_TIMEOUT, sl.inner_total, NAN, B.Xo);
    } else {
      refine.push_back(c);
    }
  }
  std::vector<int> start;   // columns whose inner recursion (re)starts on Ro
  if (!refine.empty()) {
    // X += D and the true residual R = L - W X (double-float product)
    for (int c = 0; c < kb; ++c) B.h_mask[c] = 0;
    for (int c : refine) B.h_mask[c] = 1;
    cudaMemcpyAsync(B.mask, B.h_mask, sizeof(int) * kb, cudaMemcpyHostToDevice, s);
    s_axpy_cols<<<grid, 256, 0, s>>>(B.Xo, B.b.X, N, kb, B.mask);
    if (tc_residual(prec)) {
      launch_matvec_tc(g, 0, kb, B.Xo, B.b.Q, B.b.part, &B.fl->all_done, &B.fl->err, B.scratch, s);
    } else {
      bsplit_kernel<<<grid, 256, 0, s>>>(B.Xo, B.Xf, g.ldw, N, kb);
      launch_matvec(0, g.tm_W, B.tmX, N, kb, B.Xo, B.b.Q, B.b.part, &B.fl->all_done, &B.fl->err, s,
                    matvec_split_of(g, 0), B.scratch);
    }
    s_resid_cols<<<grid, 256, 0, s>>>(B.L, B.b.Q, B.Ro, N, kb, B.mask);
    bdot_kernel<<<rgrid, 256, 0, s>>>(B.Ro, B.Ro, N, kb, B.b.part, B.fl);
    bsum_kernel<<<kb, 256, 0, s>>>(B.b.part, BRED, B.nrm);
    const double dtol = S->opts.density_tol;
    if (dtol > 0.0) {
      // norms of the correction D (in b.X) and of the updated X
      bdot_kernel<<<rgrid, 256, 0, s>>>(B.b.X, B.b.X, N, kb, B.b.part, B.fl);
      bsum_kernel<<<kb, 256, 0, s>>>(B.b.part, BRED, B.nrm + 2 * kb);
      bdot_kernel<<<rgrid, 256, 0, s>>>(B.Xo, B.Xo, N, kb, B.b.part, B.fl);
      bsum_kernel<<<kb, 256, 0, s>>>(B.b.part, BRED, B.nrm + 3 * kb);
      g.launches += 4;
    }
    cudaMemcpyAsync(B.h_nrm, B.nrm, sizeof(double) * 4 * kb, cudaMemcpyDeviceToHost, s);
    cudaStreamSynchronize(s);
    g.launches += 6;
    for (int c : refine) {
      Slot& sl = B.slot[c];
      ++sl.refinements;
      const double rel = sl.nL > 0.0 ? std::sqrt(B.h_nrm[c] / sl.nL) : 0.0;
      // density test as in msbem_solve_opts.density_tol: error of X estimated
      // from the contraction of consecutive corrections (from the second on)
      bool dens = dtol <= 0.0;
      if (!dens) {
        const double dn = std::sqrt(B.h_nrm[2 * kb + c]), xn = std::sqrt(B.h_nrm[3 * kb + c]);
        if (sl.refinements >= 2 && sl.dprev > 0.0) {
          const double eta = dn / sl.dprev;
          dens = eta < 1.0 && eta / (1.0 - eta) * dn <= dtol * xn;
        }
        sl.dprev = dn;
      }
      if (rel <= S->opts.rtol && dens)
        finish(S, e, c, MSBEM_OK, sl.inner_total, rel, B.Xo);
      else if (sl.inner_total >= S->opts.maxit || sl.refinements >= 12)
        finish(S, e, c, MSBEM_NOT_CONVERGED, sl.inner_total, rel, B.Xo);
      else
        start.push_back(c);
    }
  }
  // 2. free slots take queued requests
  std::vector<int> fresh;
  for (int c = 0; c < kb && !e.pending.empty(); ++c) {
    if (B.slot[c].req) continue;
    const uint64_t id = e.pending.front();
    e.pending.pop_front();
    Slot& sl = B.slot[c];
    sl = Slot();
    sl.req = id;
    sl.phase = INNER;
    ++e.active;
    fresh.push_back(c);
  }
  if (!fresh.empty()) {
    double gv[3 * BK];
    for (int c = 0; c < kb; ++c) {
      B.h_mask[c] = 0;
      for (int k = 0; k < 3; ++k) gv[3 * c + k] = 0.0;
    }
    for (int c : fresh) {
      B.h_mask[c] = 1;
      const Request& r = S->reqs[B.slot[c].req];
      for (int k = 0; k < 3; ++k) gv[3 * c + k] = r.g[k];
    }
    cudaMemcpyAsync(B.mask, B.h_mask, sizeof(int) * kb, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(B.b.gv, gv, sizeof(double) * 3 * kb, cudaMemcpyHostToDevice, s);
    s_rhs_cols<<<(unsigned)((N * kb + 255) / 256), 256, 0, s>>>(g.d_jptr, g.d_jrhs, N, B.b.gv, kb, B.mask, B.L);
    s_copy_cols<<<grid, 256, 0, s>>>(B.Ro, B.L, N, kb, B.mask);
    s_copy_cols<<<grid, 256, 0, s>>>(B.Xo, nullptr, N, kb, B.mask);
    bdot_kernel<<<rgrid, 256, 0, s>>>(B.L, B.L, N, kb, B.b.part, B.fl);
    bsum_kernel<<<kb, 256, 0, s>>>(B.b.part, BRED, B.nrm);
    cudaMemcpyAsync(B.h_nrm, B.nrm, sizeof(double) * kb, cudaMemcpyDeviceToHost, s);
    cudaStreamSynchronize(s);
    g.launches += 6;
    for (int c : fresh) {
      B.slot[c].nL = B.h_nrm[c];
      start.push_back(c);
    }
  }
  // 3. (re)start the inner recursion of the selected columns on Ro
  if (!start.empty()) {
    for (int c = 0; c < kb; ++c) B.h_mask[c] = 0;
    for (int c : start) {
      B.h_mask[c] = 1;
      B.slot[c].phase = INNER;
    }
    cudaMemcpyAsync(B.mask, B.h_mask, sizeof(int) * kb, cudaMemcpyHostToDevice, s);
    B.h_bs->all_done = 0;
    cudaMemcpyAsync(B.b.bs, B.h_bs, sizeof(BatchState), cudaMemcpyHostToDevice, s);
    const int f32 = inner_mode(prec) == 1 || inner_mode(prec) == 4 ? 1 : 0;
    s_copy_cols<<<grid, 256, 0, s>>>(B.b.R, B.Ro, N, kb, B.mask);
    s_copy_cols<<<grid, 256, 0, s>>>(B.b.X, nullptr, N, kb, B.mask);
    bdot_kernel<<<rgrid, 256, 0, s>>>(B.b.R, B.b.R, N, kb, B.b.part, B.fl);
    s_reduce_cols<<<kb, 256, 0, s>>>(B.b.part, BRED, B.b.cs, offsetof(ColState, nL2), B.mask);
    apply_M_batch(g, B.b, kb, 1, f32, s, false);
    s_setp_cols<<<grid, 256, 0, s>>>(B.b.P, B.b.Pf, g.ldw, B.b.Z, N, kb, B.mask);
    bdot_kernel<<<rgrid, 256, 0, s>>>(B.b.R, B.b.Z, N, kb, B.b.part, B.fl);
    s_reduce_cols<<<kb, 256, 0, s>>>(B.b.part, BRED, B.b.cs, offsetof(ColState, rz), B.mask);
    s_start_cols<<<1, BK, 0, s>>>(B.b.cs, kb, B.mask);
    g.launches += 9;
  }
  // 4. iterate the running slots: the chunk of iterations as one graph launch
  if (e.active > 0) {
    const int mv_mode = inner_mode(prec);
    const int split = mv_mode >= 3 ? 1 : matvec_split_of(g, mv_mode);
    auto enqueue_chunk = [&] {
      for (int it = 0; it < S->opts.chunk; ++it)
        enqueue_batch_iteration(g, B.b, kb, 1, mv_mode, B.tmP, split, B.scratch, S->opts.maxit, s);
    };
    if (!B.iter_exec) {
      cudaGraph_t graph = nullptr;
      if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
        enqueue_chunk();
        if (cudaStreamEndCapture(s, &graph) == cudaSuccess && graph) {
          if (cudaGraphInstantiate(&B.iter_exec, graph, 0) != cudaSuccess) B.iter_exec = nullptr;
          cudaGraphDestroy(graph);
        }
      }
      cudaGetLastError();
    }
    if (B.iter_exec)
      cudaGraphLaunch(B.iter_exec, s);
    else
      enqueue_chunk();   // without a graph, the same launches one by one
    cudaMemcpyAsync(B.h_cs, B.b.cs, sizeof(ColState) * kb, cudaMemcpyDeviceToHost, s);
    cudaEventRecord(B.ev, s);
    B.in_flight = true;
    e.last_used = now_s();
  }
}

}  // namespace

extern "C" {

int msbem_server_create(msbem_ctx* ctx, const msbem_server_opts* opts, msbem_server** out) {
  if (!ctx || !out) return MSBEM_INVALID_ARG;
  *out = nullptr;
  auto S = std::make_unique<msbem_server>();
  S->ctx = ctx;
  msbem_server_opts o{};
  if (opts) o = *opts;
  if (o.rtol <= 0.0) o.rtol = 1e-8;
  if (o.inner_rtol <= 0.0) o.inner_rtol = 1e-4;
  if (o.maxit <= 0) o.maxit = 1000;
  if (o.chunk <= 0) o.chunk = 4;
  if (o.precision < 0 || o.precision > 5 || o.precision == 1) return MSBEM_INVALID_ARG;
  if (!(o.inner_rtol < 1.0)) return MSBEM_INVALID_ARG;
  if (!(o.density_tol >= 0.0 && o.density_tol < 1.0)) return MSBEM_INVALID_ARG;
  if (o.hbm_budget_bytes <= 0.0) {
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) return MSBEM_CUDA_ERROR;
    o.hbm_budget_bytes = 0.8 * (double)fr;
  }
  S->opts = o;
  S->device = msbem_ctx_device(ctx);
  cudaSetDevice(S->device);
  const int nw = o.admission_threads > 0 ? std::min(o.admission_threads, 8) : 4;
  auto undo = [&](int st) {  // a failed set-up releases the workers made so far
    for (auto& w : S->workers) {
      msbem_destroy(w->ctx);
      cudaStreamDestroy(w->stream);
    }
    S->workers.clear();
    return st;
  };
  for (int i = 0; i < nw; ++i) {
    auto W = std::make_unique<msbem_server::Worker>();
    if (cudaStreamCreateWithFlags(&W->stream, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      return undo(MSBEM_CUDA_ERROR);
    }
    const int st = msbem_create(&W->ctx, S->device, W->stream);
    if (st) {
      cudaStreamDestroy(W->stream);
      return undo(st);
    }
    S->workers.push_back(std::move(W));
  }
  msbem_server* raw = S.release();
  for (int i = 0; i < nw; ++i) raw->workers[i]->th = std::thread(admission_thread, raw, i);
  *out = raw;
  return MSBEM_OK;
}

int msbem_server_destroy(msbem_server* S) {
  if (!S) return MSBEM_INVALID_ARG;
  {
    std::lock_guard<std::mutex> lock(S->mu);
    S->stop = true;
  }
  S->cv.notify_all();
  for (auto& w : S->workers)
    if (w->th.joinable()) w->th.join();
  cudaSetDevice(S->device);
  for (auto& kv : S->geoms) release_geometry(S, *kv.second);
  for (auto& w : S->workers) {
    msbem_destroy(w->ctx);
    cudaStreamDestroy(w->stream);
  }
  delete S;
  return MSBEM_OK;
}

int msbem_server_add_geometry(msbem_server* S, uint64_t key, const double* xyz, int64_t nv, const int32_t* tri,
                              int64_t nt, const double* cxyz, int64_t ncv, const int32_t* ctri, int64_t nct,
                              const int32_t* parent, const int32_t* patch) {
  if (!S || !xyz || !tri || !cxyz || !ctri || !parent || !patch || nv <= 0 || nt <= 0 || ncv <= 0 || nct <= 0)
    return MSBEM_INVALID_ARG;
  if (S->geoms.count(key)) return MSBEM_INVALID_ARG;
  auto e = std::make_unique<GeomEntry>();
  e->key = key;
  e->xyz.assign(xyz, xyz + 3 * nv);
  e->tri.assign(tri, tri + 3 * nt);
  e->cxyz.assign(cxyz, cxyz + 3 * ncv);
  e->ctri.assign(ctri, ctri + 3 * nct);
  e->parent.assign(parent, parent + nt);
  e->patch.assign(patch, patch + nt);
  e->nt = nt;
  int64_t n = 0;
  const int st = msbem_mesh_dofs(xyz, nv, tri, nt, &n, nullptr, nullptr, 0, nullptr, 0);
  if (st) return st;
  e->ndof = n;
  S->geoms[key] = std::move(e);
  return MSBEM_OK;
}

double msbem_server_now(void) { return now_s(); }

double msbem_server_footprint(const msbem_server* S, uint64_t key) {
  if (!S) return -1.0;
  auto it = S->geoms.find(key);
  if (it == S->geoms.end()) return -1.0;
  return (double)(estimate_footprint(*it->second, S->opts.precision) + transient_bytes(*it->second));
}

int msbem_server_submit(msbem_server* S, uint64_t key, const double g[3], double* density, double t_arrival,
                        uint64_t* id) {
  if (!S || !g || !id) return MSBEM_INVALID_ARG;
  auto it = S->geoms.find(key);
  if (it == S->geoms.end()) return MSBEM_INVALID_ARG;
  Request r;
  r.id = S->next_id++;
  r.key = key;
  for (int k = 0; k < 3; ++k) r.g[k] = g[k];
  r.out = density;
  r.t_arrival = t_arrival > 0.0 ? t_arrival : now_s();
  S->reqs[r.id] = r;
  GeomEntry& e = *it->second;
  e.pending.push_back(r.id);
  *id = r.id;
  ++S->st.submitted;
  return MSBEM_OK;
}

int msbem_server_progress(msbem_server* S, int block, int* completed) {
  if (!S) return MSBEM_INVALID_ARG;
  cudaSetDevice(msbem_ctx_device(S->ctx));
  const int64_t before = S->st.completed;
  int status = MSBEM_OK;
  for (;;) {
    bool busy = false;
    // admissions: geometries with queued requests that are not resident
    for (auto& kv : S->geoms) {
      GeomEntry& e = *kv.second;
      const int gs = e.state.load();
      if (gs == G_ADMITTING || gs == G_EVICTING) {
        busy = true;
        continue;
      }
      if (gs == G_FAILED) {                  // the geometry cannot be served
        for (uint64_t id : e.pending) {
          Request& r = S->reqs[id];
          r.status = e.admit_status;
          r.t_done = now_s();
          ++S->st.completed;
        }
        e.pending.clear();
        S->resident -= std::min(S->resident, e.reserved);
        e.reserved = 0;
        status = e.admit_status;
        e.state.store(G_OUT);
        continue;
      }
      if (gs != G_OUT || e.pending.empty()) continue;
      const size_t need = estimate_footprint(e, S->opts.precision) + transient_bytes(e);
      if (!make_room(S, need)) {
        // wait while other geometries have work and will go idle; a geometry
        // that can never fit fails its requests
        bool others = false;
        for (auto& kv2 : S->geoms) {
          const GeomEntry& o = *kv2.second;
          const int os = o.state.load();
          others = others || os == G_ADMITTING || os == G_EVICTING ||
                   (os == G_READY && (o.active > 0 || !o.pending.empty()));
        }
        if (others) {
          busy = true;
          continue;
        }
        e.admit_status = MSBEM_OOM;
        e.state.store(G_FAILED);
        busy = true;
        continue;
      }
      S->resident += need;
      e.reserved = need;
      e.state.store(G_ADMITTING);
      ++S->st.admissions;
      post(S, 1, &e);
      busy = true;
    }
    for (auto& kv : S->geoms) {
      GeomEntry& e = *kv.second;
      if (e.state.load() != G_READY) continue;
      if (e.reserved) {                     // admission finished: book the actual bytes
        S->resident = S->resident - std::min(S->resident, e.reserved) + e.footprint;
        e.reserved = 0;
      }
      Batch& B = *e.batch;
      if (B.in_flight) {
        const cudaError_t q = cudaEventQuery(B.ev);
        if (q == cudaErrorNotReady) {
          busy = true;
          continue;
        }
        B.in_flight = false;
        if (q != cudaSuccess) return MSBEM_CUDA_ERROR;
      }
      if (e.active > 0 || !e.pending.empty()) {
        schedule(S, e);
        busy = busy || B.in_flight || e.active > 0 || !e.pending.empty();
      }
    }
    if (!block || !busy) break;
  }
  if (completed) *completed = (int)(S->st.completed - before);
  S->st.resident_bytes = (double)S->resident;
  int nres = 0;
  for (auto& kv : S->geoms) nres += kv.second->state.load() == G_READY;
  S->st.resident_geometries = nres;
  return status;
}

int msbem_server_result(msbem_server* S, uint64_t id, int* status, int* iters, double* relres, double* latency_ms,
                        int* refinements) {
  if (!S) return MSBEM_INVALID_ARG;
  auto it = S->reqs.find(id);
  if (it == S->reqs.end()) return MSBEM_INVALID_ARG;
  const Request& r = it->second;
  if (status) *status = r.status;
  if (iters) *iters = r.iters;
  if (relres) *relres = r.relres;
  if (latency_ms) *latency_ms = r.t_done >= 0 ? 1e3 * (r.t_done - r.t_arrival) : -1.0;
  if (refinements) *refinements = r.refinements;
  return MSBEM_OK;
}

int msbem_server_stats_get(const msbem_server* S, msbem_server_stats* out) {
  if (!S || !out) return MSBEM_INVALID_ARG;
  msbem_server* M = const_cast<msbem_server*>(S);
  std::lock_guard<std::mutex> lock(M->mu);
  *out = S->st;
  out->far_ms = S->far_ms;
  out->far_pairs = S->far_pairs;
  out->assemble_ms = S->assemble_ms;
  out->factor_ms = S->factor_ms;
  int64_t launches = S->launches_released;
  for (auto& kv : S->geoms) {
    const GeomEntry& e = *kv.second;
    if (e.state.load() == G_READY && e.geom) launches += msbem_geom_dev(e.geom).launches;
  }
  out->launches = launches;
  return MSBEM_OK;
}

}  // extern "C"
