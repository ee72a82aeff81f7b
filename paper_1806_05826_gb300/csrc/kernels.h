// Host-side launch wrappers of the library's kernels (internal interface).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"
#include "rr.h"

namespace rr {

// ---- k_util.cu ----------------------------------------------------------
// out[0] = 0, out[i+1] = out[i] + in[i] for i < n (n+1 outputs).
// scratch: >= scan_scratch_len(n) int64.
int64_t scan_scratch_len(int64_t n);
rr_status scan_exclusive(const int64_t *in, int64_t *out, int64_t n, int64_t *scratch,
                         cudaStream_t st);

// CSC of a binary CSR pattern: col_ptr int64[n_cols+1], row_idx int32[nnz] with
// rows ascending in every column. counts/cursor: int64[n_cols]; tmp: int32[nnz].
rr_status transpose_pattern(int64_t n_rows, int64_t n_cols, int64_t nnz, const int64_t *row_ptr,
                            const int32_t *col_idx, int64_t *col_ptr, int32_t *row_idx,
                            int64_t *counts, int64_t *cursor, int32_t *tmp,
                            int64_t *scan_scratch, cudaStream_t st);

// Records DEV_BAD_INDEX in *err unless every row's indices are strictly
// increasing and in [0, n_cols).
rr_status validate_csr(int64_t n_rows, int64_t n_cols, const int64_t *row_ptr,
                       const int32_t *col_idx, int32_t *err, cudaStream_t st);

rr_status iota_i64(int64_t *out, int64_t n, cudaStream_t st);
rr_status fill_f64(double *out, double v, int64_t n, cudaStream_t st);

// ---- k_kmeans.cu --------------------------------------------------------
struct KmeansBuffers {
  int64_t *d2;         // [F]   seeding squared distances
  int32_t *ov;         // [F]   overlaps with the newest centre
  double *part;        // [kMaxGrid] per-block D^2 sums (exact integers in FP64 range)
  int64_t *part_i;     // [kMaxGrid]
  int32_t *centers;    // [k]
  int32_t *labels;     // [F]
  int32_t *next;       // [F]
  int64_t *n_S;        // [k]
  int64_t *Q;          // [k]
  int32_t *D;          // [F*k]
  int64_t *changes;    // [1]
  int32_t *work_ctr;   // [1]
  int32_t *order;      // [F] features by descending work (heaviest first)
};
rr_status kmeanspp_seed(int64_t N, int64_t F, const int64_t *row_ptr, const int32_t *col_idx,
                        const int64_t *col_ptr, const int32_t *row_idx, int32_t k, uint64_t seed,
                        KmeansBuffers &b, cudaStream_t st);
// labels <- -1 except labels[centers[S]] = S.
rr_status kmeans_init_labels(int64_t F, int32_t k, KmeansBuffers &b, cudaStream_t st);
// One Lloyd assignment step; on return (stream synchronised) *changes_host holds
// the number of labels that changed.
rr_status kmeans_lloyd_step(int64_t N, int64_t F, const int64_t *row_ptr, const int32_t *col_idx,
                            const int64_t *col_ptr, const int32_t *row_idx, int32_t k,
                            KmeansBuffers &b, int64_t *changes_host, cudaStream_t st);
rr_status kmeans_work_order(int64_t F, const int64_t *row_ptr, const int64_t *col_ptr,
                            const int32_t *row_idx, KmeansBuffers &b, int64_t *scratch,
                            cudaStream_t st);

// ---- k_coarse.cu --------------------------------------------------------
// Compacts labels in place to 0..k_eff-1 (order kept); n_S compacted too.
// k_eff_host receives the count (stream synchronised).
rr_status compact_clusters(int64_t F, int32_t k, int32_t *labels, int64_t *n_S, int32_t *remap,
                           int32_t *k_eff_host, cudaStream_t st);
// s_S = 1/sqrt(n_S)
rr_status prolong_scale(int32_t k, const int64_t *n_S, double *s, cudaStream_t st);
// Ct[S, r] (k_pad x n_pad, FP16, K-major) = number of features of cluster S in row r.
rr_status coarse_counts(int64_t N, int64_t n_pad, int32_t k_pad, const int64_t *row_ptr,
                        const int32_t *col_idx, const int32_t *labels, void *Ct, int32_t *err,
                        cudaStream_t st);
// G = Ct Ct^T exact (CUDA cores, int32 chunks summed in int64) -> G as FP64 (k x k).
rr_status gram_exact_cuda_cores(int32_t k, int32_t k_pad, int64_t n_pad, const void *Ct, double *G,
                                cudaStream_t st);
// A_c lower triangle (G[S,T] s_S) s_T + lambda on the diagonal, mirrored.
rr_status coarse_operator(int32_t k, const double *G, const double *s, double lambda, double *Ac,
                          cudaStream_t st);
// In-place lower Cholesky of Ac (k x k); records DEV_NOT_SPD on a pivot <= 0.
rr_status cholesky(int32_t k, double *L, int32_t *err, cudaStream_t st);
// Ainv = L^{-T} L^{-1} (full symmetric). Linv: k x k workspace.
rr_status chol_inverse(int32_t k, const double *L, double *Linv, double *Ainv, cudaStream_t st);

// ---- k_spmv.cu ----------------------------------------------------------
// Work items of the transpose mat-vec: every column is cut into pieces of at
// most kCscChunk nonzeros; columns of one piece finish in place, longer ones
// in a second pass over their piece sums.
struct CscItem {
  int64_t begin, end;  // range in row_idx
  int32_t col;         // column
  int32_t slot;        // -1: whole column; else index into piece sums
};
struct CscPlan {
  CscItem *items = nullptr;
  int64_t n_items = 0;
  int32_t *heavy_col = nullptr;   // columns cut into >1 pieces
  int32_t *heavy_first = nullptr; // their first slot
  int32_t *heavy_n = nullptr;     // their number of slots
  int64_t n_heavy = 0;
  int64_t n_slots = 0;
  double *slot_sum = nullptr;     // [n_slots]
};
constexpr int kCscChunk = 2048;
rr_status csc_plan_build(int64_t F, const int64_t *col_ptr, CscPlan &plan, cudaStream_t st);
void csc_plan_free(CscPlan &plan);

// Epilogues of t_i = (X^T u)_i + lambda v_i, fused into the transpose mat-vec.
enum CscMode : int32_t {
  CSC_RHS = 0,     // out = X^T u                    (b = X^T y; v unused)
  CSC_APPLY = 1,   // out = t
  CSC_PRE = 2,     // out = r - t                     (r1 of the cycle)
  CSC_POST = 3,    // r2 = r - t; out = v + w*(r2/d)  (z of the cycle); dot r.out
  CSC_PCG = 4,     // out = t                         (q = A p); dot v.out
  CSC_RESID = 5,   // out = r - t, r = b              (true residual); dot out.out
};
struct CscEpilogue {
  int32_t mode;
  double lambda;
  double omega;
  const double *v;    // vector X was applied to
  const double *r;    // residual (PRE/POST) or b (RESID)
  const double *d;    // Jacobi diagonal (POST)
  double *out;
  double *dot_part;   // per-block partial dots (POST/PCG/RESID), 2 * kMaxGrid entries
  const int32_t *stop;  // if non-null and *stop != 0 the kernels return at once
};
rr_status csr_spmv(int64_t N, const int64_t *row_ptr, const int32_t *col_idx, const double *v,
                   double *u, const int32_t *stop, cudaStream_t st);
rr_status csc_spmv(int64_t F, const int32_t *row_idx, const double *u, const CscPlan &plan,
                   const CscEpilogue &ep, cudaStream_t st);
// Number of partial dots csc_spmv writes into ep.dot_part.
int csc_dot_parts(const CscPlan &plan);

// ---- k_pcg.cu -----------------------------------------------------------
struct PcgScalars {
  double rho_old;    // <r, z> of the previous iteration
  double rr;         // ||r||^2 after the last update
  double bnorm;      // ||b||
  double target;     // tol * ||b||
  int32_t iter;      // iterations done (all restarts together)
  int32_t converged; // 1 once ||r|| <= target: later kernels of the loop return at once
  int32_t nonfinite; // 1 if a NaN/Inf was met
  int32_t first;     // 1 before the first direction of a (re)start
};
constexpr int kVecGrid = kSMs * 4;   // fixed grid of the vector kernels (deterministic partials)

// r_c[S] = s_S * sum_{i in S} r1[i] (members ascending), one warp per cluster.
rr_status restrict_clusters(int32_t k, const int64_t *cl_ptr, const int32_t *members,
                            const double *s, const double *r1, double *rc, const int32_t *stop,
                            cudaStream_t st);
// e_c = Ainv r_c.
rr_status coarse_matvec(int32_t k, const double *Ainv, const double *rc, double *ec,
                        const int32_t *stop, cudaStream_t st);
// z2 = z1 + s[l(i)] e_c[l(i)].
rr_status prolong_add(int64_t F, const int32_t *labels, const double *s, const double *ec,
                      const double *z1, double *z2, const int32_t *stop, cudaStream_t st);
// z = omega * r / d; if rz_part: per-block <r, z> into rz_part[0..kVecGrid).
// d == nullptr means z = r (no preconditioner).
rr_status jacobi(int64_t F, double omega, const double *r, const double *d, double *z,
                 double *rz_part, const int32_t *stop, cudaStream_t st);
// rho = <r,z> (from n_rz partials); beta = rho / rho_old (0 on a (re)start); p = z + beta p.
rr_status pcg_direction(int64_t F, const double *rz_part, int n_rz, const double *z, double *p,
                        PcgScalars *S, cudaStream_t st);
// alpha = rho / <p,q>; w += alpha p; r -= alpha q; partial ||r||^2;
// z1 = omega r / d when z1 != nullptr.
rr_status pcg_update(int64_t F, const double *rz_part, int n_rz, const double *pq_part, int n_pq,
                     const double *p, const double *q, double *w, double *r, double omega,
                     const double *d, double *z1, double *rr_part, PcgScalars *S,
                     cudaStream_t st);
// rr = sum(rr_part); rho_old = sum(rz_part); iter++; convergence and finiteness flags;
// history[iter-1] = ||r|| / ||b|| when iter <= hist_cap.
rr_status pcg_finish(const double *rz_part, int n_rz, const double *rr_part, int n_rr,
                     PcgScalars *S, double *history, int32_t hist_cap, cudaStream_t st);
// per-block partial <a, b> into part[0..kVecGrid).
rr_status dot_parts(int64_t n, const double *a, const double *b, double *part, cudaStream_t st);
// (Re)starts PCG: bnorm/target from <b,b> partials if set_bnorm, rr from <r,r> partials.
rr_status pcg_start(const double *bb_part, int n_bb, const double *rr_part, int n_rr, double tol,
                    int32_t set_bnorm, PcgScalars *S, cudaStream_t st);
// *out = fixed-order sum of n partials.
rr_status sum_parts(const double *part, int n, double *out, cudaStream_t st);
rr_status copy_f64(double *dst, const double *src, int64_t n, cudaStream_t st);
// dst = src (or zero when src == nullptr) for vectors of F entries; device helper kernels.
rr_status axpby(int64_t n, double a, const double *x, double b, double *y, cudaStream_t st);

}  // namespace rr
