// The solver handle (opaque behind include/rr.h) and its device arena, shared by
// the translation units that sequence work on it.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "common.cuh"
#include "kernels.h"

namespace rr {
struct BatchState;
void batch_free(BatchState *b);
}  // namespace rr

struct DevArena {
  std::vector<void *> ptrs;
  template <class T>
  rr_status alloc(T **p, size_t n) {
    void *q = nullptr;
    const size_t bytes = sizeof(T) * (n ? n : 1);
    if (cudaMalloc(&q, bytes) != cudaSuccess) {
      cudaGetLastError();
      rr_set_error("cudaMalloc of %zu bytes failed", bytes);
      return RR_OOM;
    }
    ptrs.push_back(q);
    *p = static_cast<T *>(q);
    return RR_OK;
  }
  void release(void *p) {
    for (auto &q : ptrs)
      if (q == p) {
        cudaFree(q);
        q = nullptr;
      }
  }
  void free_all() {
    for (void *q : ptrs)
      if (q) cudaFree(q);
    ptrs.clear();
  }
};

struct rr_handle {
  cudaStream_t st = nullptr;
  rr_options opt{};
  int64_t N = 0, F = 0, nnz = 0;
  int32_t k_req = 0, k_eff = 0, kmeans_iters = 0;
  double lambda = 0.0, omega = 1.0, setup_ms = 0.0;
  // X and its transposed copy
  int64_t *row_ptr = nullptr;
  int32_t *col_idx = nullptr;
  int64_t *col_ptr = nullptr;
  int32_t *row_idx = nullptr;
  // clustering
  int32_t *labels = nullptr;
  int32_t *centers = nullptr;
  int64_t *n_S = nullptr;
  int64_t *cl_ptr = nullptr;
  int32_t *members = nullptr;
  double *s = nullptr;
  // coarse level
  double *G = nullptr, *Ac = nullptr, *Lw = nullptr, *Linv = nullptr, *Ainv = nullptr;
  double *mu = nullptr, *Qv = nullptr;   // RR_COARSE_EIGEN: eigenvalues, eigenvector rows
  double *Qt = nullptr, *dvec = nullptr, *ec_tmp = nullptr;   // Q row-major, 1/(mu+lambda)
  float *Ainv32 = nullptr;               // RR_PREC_MIXED: FP32 copy of Ainv, rows padded to 4
  int32_t eig_sweeps = 0;
  // coarse levels prepared ahead for other lambdas (rr_prepare_lambdas): built
  // on prep_st; rr_set_lambda to one of them swaps its buffers in
  struct Prepared {
    double lambda = 0.0;
    bool valid = false;
    double *Ainv = nullptr, *d = nullptr, *omega_dev = nullptr;
    float *Ainv32 = nullptr;
    unsigned long long *max_bits = nullptr;
    cudaEvent_t done = nullptr;
  };
  static constexpr int kPrepared = 8;
  Prepared prep[kPrepared];
  cudaStream_t prep_st = nullptr;
  double *prep_Ac = nullptr, *prep_Lw = nullptr, *prep_Linv = nullptr;   // shared scratch
  // smoother
  double *d = nullptr;
  int64_t *gsum = nullptr;   // sum_j |(X^T X)_ij| = sum of the row lengths over column i
  double *omega_dev = nullptr;
  unsigned long long *max_bits = nullptr;
  rr::RestrictPlan rplan;   // restriction items of the single-system path
  rr::RestrictPlan bplan;   // the batched path's (larger) items
  rr::SlicedPattern pcsr;   // X by row, vector v cut in feature slices
  rr::SlicedPattern pcsc;   // X^T by column, vector u cut in row slices
  rr::SplitOperator split;  // the FP32 operator's split form (mixed precision, binary X)
  // solve workspace
  double *b = nullptr, *r = nullptr, *z1 = nullptr, *z2 = nullptr, *z = nullptr, *p = nullptr,
         *q = nullptr, *r1 = nullptr, *u = nullptr, *rc = nullptr, *ec = nullptr, *rt = nullptr;
  double *part_rz = nullptr, *part_pq = nullptr, *part_rr = nullptr, *part_bb = nullptr;
  double *scal = nullptr;
  double *w_int = nullptr;         // the iterate (graphs capture fixed pointers)
  double *bayes_y = nullptr;       // rr_bayes: y + e1, then y - X w (N)
  cudaStream_t cap_stream = nullptr;
  cudaGraph_t loop_graph = nullptr;
  cudaGraphExec_t loop_exec = nullptr;
  int32_t *limit_host = nullptr;
  int64_t body_kernels = 0;
  double phase_ms[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  bool gram_on_tensor_cores = false;
  rr::PcgScalars *S = nullptr;
  rr::PcgScalars *S_host = nullptr;
  double *scal_host = nullptr;
  double *history = nullptr;
  int32_t hist_cap = 0;
  int32_t *err = nullptr;
  int32_t *err_host = nullptr;
  int n_parts = 0;
  rr::BatchState *batch = nullptr;   // rr_solve_batch workspace (created on first use)
  // dense X (RR_DENSE_F32_ROWMAJOR)
  bool dense = false;
  float *Xd = nullptr;                // [N x F] row-major
  double *dsq = nullptr, *dgs = nullptr, *dpart = nullptr;
  // rr_solve_fcg workspace (created on first use)
  double *p_prev = nullptr, *q_prev = nullptr, *part_zq = nullptr, *part3 = nullptr;
  rr::FcgScalars *Sf = nullptr, *Sf_host = nullptr;
  // TLFCG rougher (two CG steps on A z = r): iterate, residual, direction, A direction, copy of r
  double *tz = nullptr, *tr = nullptr, *tp = nullptr, *tq = nullptr, *tzz = nullptr;
  double *t_rz = nullptr, *t_pq = nullptr, *t_rr = nullptr;
  rr::PcgScalars *St = nullptr;
  void *fcg_cache = nullptr;   // the FCG loop graph without a network (kept until lambda changes)
  // rr_fork_lambda: the handle whose X-dependent setup this one shares (nullptr:
  // none); the event recorded after this handle's coarse factor (a fork's, or
  // the one rr_setup leaves running on fst, its own stream)
  rr_handle *fork_of = nullptr;
  cudaEvent_t ready = nullptr;
  cudaStream_t fst = nullptr;
  DevArena mem;
};
