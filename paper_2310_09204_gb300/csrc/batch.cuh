// Shared pieces of the multi-vector PCG (pcg_batch.cu) and of the serving
// engine (serve.cu): per-column state, the work buffers of one batch, and the
// kernels both drive.  Vectors of a batch are row-major N x kb (kb <= 16).
#pragma once

#include <cstddef>

#include "msbem_internal.h"

namespace msbem {

#define BK 16                 // columns per batch
#define BRED 128              // blocks of the column reductions
static constexpr unsigned kStrideBlocks = 512;

// PCG scalars and stopping state of one column.  done: 0 running,
// 1 converged (or fixed count reached), 2 breakdown, 3 iteration cap,
// 4 no data, 5 device timeout, 6 idle slot (serving engine).
struct ColState {
  double rz, pq, alpha, rr, rz_new, beta, nL2;
  int done, iter, pad0, pad1;
};
struct BatchState {
  int all_done;
  int kb;
  int maxit;
  int fixed;
  double rtol;
  int err;      // set by the matrix-vector product when a copy never completed
};

__device__ __forceinline__ bool col_active(const ColState* cs, int c) { return cs[c].done == 0; }

struct BatchBuffers {
  double *X, *R, *Z, *P, *Q, *T, *U, *part, *gv, *hist;
  float* Pf;     // [2][kb][ldw] float-pair planes of P (transposed)
  float2* Rf;
  ColState* cs;
  BatchState* bs;
};

// carves one pool allocation into 16-byte aligned pieces
struct Carver {
  char* cur;
  template <class T>
  T* take(size_t n) {
    T* p = (T*)cur;
    cur += (sizeof(T) * n + 15) / 16 * 16;
    return p;
  }
};

__global__ void bdot_kernel(const double* __restrict__ A, const double* __restrict__ B, int64_t N, int kb,
                            double* __restrict__ part, const BatchState* __restrict__ bs);
__global__ void bsum_kernel(const double* __restrict__ part, int nparts, double* __restrict__ out);
__global__ void brhs_kernel(const int64_t* __restrict__ jptr, const double* __restrict__ jrhs, int64_t N,
                            const double* __restrict__ gv, int kb, double* __restrict__ R);
__global__ void bsplit_kernel(const double* __restrict__ X, float* __restrict__ Xf, int64_t ldp, int64_t N,
                              int kb);

// Z = M R for all columns (f32: FP32 block inverses and residual).
// in_iteration: within a PCG iteration -- the residual's float-pair split Rf
// is already written (by the residual update), and the launch that ends the
// application also leaves the partial sums of R . Z in b.part (bdot_kernel's
// layout); otherwise Rf is made here and no sums are formed.
void apply_M_batch(DevGeom& g, const BatchBuffers& b, int kb, int precondition, int f32, cudaStream_t s,
                   bool in_iteration);

// One PCG iteration on every running column of the batch (the recursion of
// Sec. 2.1 per column; columns that are not running are left untouched):
// Q = W P (mode 0 double-float, 1 FP32), alpha, X/R update, stopping test,
// Z = M R, beta, P update.  hist: [kb][hcap+1] residuals then [kb][hcap]
// alpha and beta.
void enqueue_batch_iteration(DevGeom& g, const BatchBuffers& b, int kb, int precondition, int mv_mode,
                             const CUtensorMap& tmP, int split, void* scratch, int hcap, cudaStream_t s);

}  // namespace msbem
