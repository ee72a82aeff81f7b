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

// Records DEV_BAD_INDEX in *err unless 0 <= row_ptr[r] <= row_ptr[r+1] <= nnz
// and every row's indices are strictly increasing and in [0, n_cols).
rr_status validate_csr(int64_t n_rows, int64_t n_cols, int64_t nnz, const int64_t *row_ptr,
                       const int32_t *col_idx, int32_t *err, cudaStream_t st);

rr_status iota_i64(int64_t *out, int64_t n, cudaStream_t st);
rr_status fill_f64(double *out, double v, int64_t n, cudaStream_t st);

// ---- k_leader.cu --------------------------------------------------------
// Leader-follower clustering (Algorithm 1), binary X, in steps of 64 features
// (each feature's rows in tasks of at most 2048).
constexpr int32_t kLfMaxLeaders = 16384;   // the count kernel's shared-memory counters
struct LfState {
  int32_t L;            // leaders so far
  int32_t nnew;         // leaders made by the current step
  int32_t min_n, min_s; // the smallest leader size and the earliest leader of that size
  int32_t overflow;     // 1 once more than the capacity would be needed
  int32_t newpos[64];   // the current step's new leaders (positions in the step)
};
struct LfBuffers {
  int32_t *rl = nullptr;                  // [nnz] per-row leader lists, laid out like col_idx
  int32_t *rl_cnt = nullptr;              // [N]
  unsigned long long *rowmask = nullptr;  // [N] the step features holding each row
  int32_t *nlead = nullptr;               // [cap] leader sizes
  unsigned long long *best = nullptr;     // [64] nearest committed leader of each step feature
  LfState *S = nullptr;
};
// labels[F] (cluster = leader index), centers[cap] (the leaders' feature ids);
// RR_UNSUPPORTED when more than cap leaders would be needed.
rr_status leader_follower(int64_t N, int64_t F, const int64_t *row_ptr, const int64_t *col_ptr,
                          const int32_t *row_idx, double tol2, int32_t cap, LfBuffers &lb,
                          int32_t *labels, int32_t *centers, int32_t *n_lead_out, int32_t *err,
                          cudaStream_t st);

// ---- k_kmeans.cu --------------------------------------------------------
struct KmeansBuffers {
  int64_t *d2;         // [F]   seeding squared distances
  int32_t *ov;         // [F]   overlaps with the newest centre
  double *part;        // [kMaxGrid] per-block D^2 sums (exact integers in FP64 range)
  int64_t *part_i;     // [kmeans_seed_tiles(F) + 1]
  int32_t *centers;    // [k]
  int32_t *labels;     // [F]   current labels (-1: not assigned yet)
  int32_t *prev;       // [F]   labels of the previous step
  int32_t *next;       // [F]
  int64_t *mcount;     // [N]   room for each row's delta list (2 x moved entries)
  int64_t *mptr;       // [N+1] start of each row's delta list
  int2 *dlist;         // [max(2 nnz, F) + 1] (cluster, delta) pairs of the rows' count changes
  int32_t *dcount;     // [N]   length of each row's delta list
  int64_t *work;       // [1]   total cost of applying the delta lists
  int64_t *scan_scratch;
  int64_t *n_S;        // [k]
  int64_t *Q;          // [k]
  float2 *qr;          // [k]   FP32 approximations of the score terms (argmin filter)
  int32_t *D;          // [F*k] D[i, S] = x_i . c_S for the current labels
  int64_t *changes;    // [1]
  int32_t *work_ctr;   // [1]
  int32_t *order;      // [F] features by descending work (heaviest first)
  uint16_t *hot;       // [F] shared-histogram bin of a frequent feature (0xFFFF: none)
  int32_t *hot_col;    // [2048] feature of each bin
  int32_t *hot_n;      // [1] bins in use (capped at 2048 when read)
  int32_t packed;      // host: delta lists in the 32-bit form (set by kmeans_work_order)
  int64_t *task_ptr;   // [F+1] first pull task of each feature in work order
  int32_t *task_it;    // [kmeans_pull_tasks_max(F, nnz)] feature (work-order index) of each task
  int64_t n_tasks;     // host: number of pull tasks (set by kmeans_work_order)
  int32_t *moved;      // [F]   features whose label changed (steps after few changes)
  int32_t *touched;    // [N]   rows holding them
  int32_t *sparse_n;   // [4]   lengths of moved[] and touched[], the moved columns' entries (u64)
};
// upper bound of the pull tasks: one per feature plus one per 1024 entries
int64_t kmeans_pull_tasks_max(int64_t F, int64_t nnz);
// K-means++ seeding (k centres into b.centers). Synchronises the stream.
// pull_work: a centre c is pulled when n_c nnz / N exceeds it (0: kSeedPullWork,
// < 0: never).
rr_status kmeanspp_seed(int64_t N, int64_t F, int64_t nnz, const int64_t *row_ptr,
                        const int32_t *col_idx, const int64_t *col_ptr, const int32_t *row_idx,
                        int32_t k, uint64_t seed, int64_t pull_work, KmeansBuffers &b,
                        cudaStream_t st);
// default pull threshold: a centre's overlaps are pulled when pushing them
// would take more than about 7e5 atomic increments
constexpr double kSeedPullWork = 7.0e5;

// labels <- -1 except labels[centers[S]] = S; prev <- -1; D <- 0.
// tiles of features of the seeding pass (tile sums in part_i)
int64_t kmeans_seed_tiles(int64_t F);
rr_status kmeans_init_labels(int64_t F, int32_t k, KmeansBuffers &b, cudaStream_t st);
// After kmeanspp_seed: the first Lloyd step's result (each feature's nearest
// centre, left by the seeding in b.prev) as labels, prev <- -1, D <- 0, and
// the labels that differ from the singleton labelling in *changes_host.
rr_status kmeans_seeded_labels(int64_t F, int32_t k, KmeansBuffers &b, int64_t *changes_host,
                               cudaStream_t st);
// One Lloyd assignment step; on return (stream synchronised) *changes_host holds
// the number of labels that changed. pull_work: count updates above which the
// step pulls per feature instead of pushing per row (<= 0: the default).
// moved: < 0 for the first step (every label -1 before it but the centres'),
// else the number of labels the previous step changed.
rr_status kmeans_lloyd_step(int64_t N, int64_t F, int64_t nnz, const int64_t *row_ptr,
                            const int32_t *col_idx, const int64_t *col_ptr, const int32_t *row_idx,
                            int32_t k, KmeansBuffers &b, int64_t *changes_host, int64_t pull_work,
                            int64_t moved, cudaStream_t st);
// order[] = features by descending work_i = sum of the row lengths of column i
// (heaviest first); work[] receives work_i, which is also the Gershgorin row
// sum of X^T X for binary X.
// work[i] = sum over the rows of column i of their lengths (= sum_j |(X^T X)_ij|)
rr_status feature_work(int64_t F, const int64_t *row_ptr, const int64_t *col_ptr,
                       const int32_t *row_idx, int64_t *work, cudaStream_t st);
rr_status kmeans_work_order(int64_t N, int64_t F, int32_t k, const int64_t *row_ptr,
                            const int64_t *col_ptr, const int32_t *row_idx, KmeansBuffers &b,
                            int64_t *work, int64_t *scratch, cudaStream_t st);

// ---- k_coarse.cu --------------------------------------------------------
// Compacts labels in place to 0..k_eff-1 (order kept); n_S compacted too.
// k_eff_host receives the count (stream synchronised).
rr_status compact_clusters(int64_t F, int32_t k, int32_t *labels, int64_t *n_S, int32_t *remap,
                           int32_t *k_eff_host, cudaStream_t st);
// s_S = 1/sqrt(n_S)
rr_status prolong_scale(int32_t k, const int64_t *n_S, double *s, cudaStream_t st);
// C32[S, r] (k_pad x n_pad, int32, K-major) = number of features of cluster S in
// row r; *max_count receives the largest count.
rr_status coarse_counts(int64_t N, int64_t n_pad, int32_t k_pad, const int64_t *row_ptr,
                        const int32_t *col_idx, const int32_t *labels, int32_t *C32,
                        int32_t *max_count, cudaStream_t st);
// FP16 copy of n counts (each <= 2048, so exact).
rr_status counts_to_half(int64_t n, const int32_t *C32, void *C16, cudaStream_t st);
// ---- k_gram_tc.cu -------------------------------------------------------
// K rows per tensor-core chunk that keep every FP32 partial sum exact (< 2^24)
// for counts up to max_count; < 64 means the tensor-core path cannot be exact.
int64_t gram_tc_chunk(int32_t max_count);
// G = Ct Ct^T (k x k, FP64, exact) with tcgen05 MMAs; k_pad % 128 == 0, n_pad % 64 == 0.
// wait_limit: spin iterations of the kernel's bounded waits on its pipeline
// (0: the default; negative: none, a test hook that makes them expire).
rr_status gram_tensor_cores(int32_t k, int32_t k_pad, int64_t n_pad, const void *Ct,
                            int32_t max_count, double *G, int32_t *err, cudaStream_t st,
                            int32_t wait_limit = 0);
// G = C32 C32^T exact (CUDA cores, int32 steps summed in int64) -> G as FP64 (k x k).
rr_status gram_exact_cuda_cores(int32_t k, int32_t k_pad, int64_t n_pad, const int32_t *C32,
                                double *G, cudaStream_t st);
// A_c lower triangle (G[S,T] s_S) s_T + lambda on the diagonal, mirrored.
rr_status coarse_operator(int32_t k, const double *G, const double *s, double lambda, double *Ac,
                          cudaStream_t st);
// In-place lower Cholesky of Ac (k x k); records DEV_NOT_SPD on a pivot <= 0.
// scratch: k x k doubles it may overwrite (the inverses of the diagonal blocks).
rr_status cholesky(int32_t k, double *L, double *scratch, int32_t *err, cudaStream_t st);
// Ainv = L^{-T} L^{-1} (full symmetric). Linv: k x k workspace.
rr_status chol_inverse(int32_t k, const double *L, double *Linv, double *Ainv, cudaStream_t st);

// ---- operator epilogues ------------------------------------------------
// Epilogues of t_i = (X^T u)_i + lambda v_i, applied where the transposed
// mat-vec's piece sums are combined (k_sliced.cu).
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

// ---- k_fcg.cu -----------------------------------------------------------
// Flexible CG (Algorithm 3, m = 1) scalars; see k_fcg.cu.
struct FcgScalars {
  double rr;         // ||r||^2 after the last update
  double bnorm;      // ||b||
  double target;     // tol * ||b||
  double pq_prev;    // <p, A p> of the previous direction
  int32_t iter, converged, nonfinite, first, limit;
  int32_t fallbacks; // learned steps redone with the Cholesky coarse solve
  int32_t skip_fb;   // 0 while the current step is being redone (fallback pass), else 1
  int32_t learned;   // 1 if the coarse correction is the network's
};
rr_status fcg_dot(int64_t F, const double *a, const double *b, double *part, const int32_t *stop,
                  cudaStream_t st);
rr_status fcg_direction(int64_t F, const double *part_zq, const FcgScalars *S, const double *z,
                        const double *p_prev, double *p, const int32_t *stop, cudaStream_t st);
rr_status fcg_dots(int64_t F, const double *p, const double *r, const double *q, double *part3,
                   const int32_t *stop, cudaStream_t st);
rr_status fcg_decide(const double *part_rz, const double *part_pq, const double *part3,
                     FcgScalars *S, cudaStream_t st);
rr_status fcg_update(int64_t F, const double *part_pq, const double *part3, const double *p,
                     const double *q, double *w, double *r, double omega, const double *d,
                     double *z1, double *p_prev, double *q_prev, double *part_rr,
                     const FcgScalars *S, cudaStream_t st);
rr_status fcg_finish(const double *part_rr, const double *part_pq, FcgScalars *S, double *history,
                     int32_t hist_cap, cudaStream_t st);
rr_status fcg_start(const double *bb_part, int n_bb, const double *rr_part, double tol,
                    int32_t set_bnorm, int32_t learned, FcgScalars *S, cudaStream_t st);
rr_status fcg_condition(cudaGraphConditionalHandle hc, const FcgScalars *S, cudaStream_t st);

// ---- k_sliced.cu --------------------------------------------------------
// Sliced binary pattern (see k_sliced.cu): the gathered dimension (n_inner)
// cut into nb slices of W <= kSliceMax entries, 16-bit offsets in 16-byte
// words, segments cut into pieces of <= kPieceWords words, one FP64 sum slot
// per piece, slots of an outer index contiguous.
constexpr int kSliceMax = 27648;   // FP64 slice + pad = 216 KiB of shared memory
constexpr int kPieceWords = 32;
struct SlicedView {
  int32_t W;
  int64_t n_inner;
  const int32_t *pw;
  const int32_t *slot;
  const uint4 *idx;
  const int32_t *task_slice;
  const int32_t *task_p;
  const int32_t *order;
};
struct SlicedPattern {
  int64_t n_outer = 0, n_inner = 0, nwords = 0, npieces = 0;
  int32_t nb = 0, W = 0, ntasks = 0;
  int32_t *pw = nullptr;         // [npieces+1] first word of each piece (slice-major)
  int32_t *slot = nullptr;       // [npieces]   sum slot of each piece (outer-major)
  int32_t *slot_ptr = nullptr;   // [n_outer+1] slots of each outer index
  uint4 *idx = nullptr;          // [nwords]
  double *psum = nullptr;        // [npieces]   piece sums
  int32_t *task_slice = nullptr; // [ntasks]
  int32_t *task_p = nullptr;     // [ntasks+1]
  int32_t *order = nullptr;      // [npieces]   the pieces of each task, longest first
  int64_t n_chunks = 0;          // chunks of whole pieces of the staged FP32 gather (0: none)
  int32_t *chunk_p = nullptr;    // [n_chunks+1] first piece of every chunk
  int32_t *chunk_w = nullptr;    // [n_chunks+1] first word of every chunk
  bool staged = false;           // FP32 passes use the staged gather (needs the chunks)
  bool psum32 = false;           // piece sums stored as FP32 (psum holds floats), else FP64
  int32_t n_heavy = 0;           // outer indices with many slots (summed one warp each)
  int32_t *heavy = nullptr;      // [n_heavy]
  int32_t *task_c = nullptr;     // [ntasks+1]  chunks of each task
  int32_t *err = nullptr;        // device error word (DEV_TIMEOUT from a bounded wait)
  void *xq = nullptr;            // [n_inner]   the gathered vector in the accumulation type
  // streaming gather (FP32 piece sums only; see sliced_build_stream)
  int32_t *wmeta = nullptr;      // [nwords] slot of the piece that ends at this word, else -1
  int32_t *wstart = nullptr;     // [ntasks * 33] first word of each warp's range of a task
  SlicedView view() const {
    return SlicedView{W, n_inner, pw, slot, idx, task_slice, task_p, order};
  }
};
// outer_ptr/inner: a pattern with inner indices ascending within each outer index.
// chunks: build the staged gather's chunks (and balance the words for it);
// false for a pattern only the streaming gather reads.
rr_status sliced_build(int64_t n_outer, int64_t n_inner, const int64_t *outer_ptr,
                       const int32_t *inner, SlicedPattern &P, int32_t *err, cudaStream_t st,
                       bool chunks = true);
void sliced_free(SlicedPattern &P);
// piece sums of P against x (or, when `in` is given, against the per-index
// sums of in's slots: the output of a previous pass); fp32: accumulate in FP32
// (the mixed-precision inner iterations), else in FP64. x32_ready (fp32 only):
// the FP32 copy of x is already in P.xq (written by the kernel that made x).
rr_status sliced_gather(const SlicedPattern &P, const double *x, const SlicedPattern *in,
                        const int32_t *stop, cudaStream_t st, bool fp32 = false,
                        bool x32_ready = false);
// out[o] = sum of the slots of outer index o.
rr_status sliced_slot_sum(const SlicedPattern &P, double *out, cudaStream_t st);
// Metadata of the streaming gather for P (FP32 piece sums): then every FP32
// gather of P streams the task's words warp by warp (see k_sliced.cu).
rr_status sliced_build_stream(SlicedPattern &P, cudaStream_t st);
// Chooses P.staged: mode RR_GATHER_LANES / RR_GATHER_STAGED, or (RR_GATHER_AUTO)
// the faster of the two FP32 gathers on this pattern, each timed on the stream.
rr_status sliced_choose_gather(SlicedPattern &P, int32_t mode, cudaStream_t st);
// t_i = slot sums of feature i, then the epilogue; kVecGrid partial dots.
rr_status sliced_epilogue(const SlicedPattern &P, const CscEpilogue &ep, cudaStream_t st);

// ---- k_eigen.cu ---------------------------------------------------------
// G_s = D_s G D_s = Q diag(mu) Q^T by parallel cyclic Jacobi (FP64): mu[k],
// Vk (k x k, row e = eigenvector e); *sweeps_out the sweeps taken.
rr_status coarse_eigen(int32_t k, const double *G, const double *s, double *mu, double *Vk,
                       int32_t *sweeps_out, cudaStream_t st);
// Qt = Vk^T (Q row-major); d = 1 / (mu + lambda).
rr_status eig_transpose(int32_t k, const double *Vk, double *Qt, cudaStream_t st);
rr_status eig_dvec(int32_t k, const double *mu, double lambda, double *d, cudaStream_t st);
// Ainv = Q diag(1 / (mu + lambda)) Q^T (exactly symmetric).
rr_status eig_inverse(int32_t k, const double *mu, const double *Vk, double lambda, double *Ainv,
                      cudaStream_t st);

// ---- k_bayes.cu ---------------------------------------------------------
// Gibbs sampling with noise injection (see k_bayes.cu for the draws).
rr_status bayes_noise_y(int64_t N, const double *y, uint64_t seed, int64_t step, double tau,
                        double *yt, cudaStream_t st);
rr_status bayes_add_e2(int64_t F, double *b, uint64_t seed, int64_t step, double lam, double tau,
                       cudaStream_t st);
rr_status bayes_resid(int64_t N, const double *y, const double *u, double *r, cudaStream_t st);
rr_status bayes_gamma(double a, double rate0, const double *part, int n_part, uint64_t seed,
                      uint64_t stream, double *out, cudaStream_t st);
rr_status bayes_accum(int64_t F, const double *w, double *acc, cudaStream_t st);
rr_status bayes_scale(int64_t F, double s, double *v, cudaStream_t st);

// ---- k_split.cu ---------------------------------------------------------
// Split form of the FP32 operator (see k_split.cu): the all-ones columns as a
// rank-one term, the H most frequent other columns as a row-major bitmap, the
// rest as sliced patterns with FP32 piece sums.
struct SplitOperator {
  bool active = false;
  int64_t N = 0, F = 0;
  int32_t H = 0, G = 0;           // head columns (32 G) and bitmap words per row
  int32_t n_ones = 0;
  int32_t *ones = nullptr;        // [n_ones] the all-ones columns
  int32_t *head = nullptr;        // [H] column of each head bit (-1: none)
  uint32_t *bits = nullptr;       // [N * G] row-major head bitmap
  int32_t nblk = 0;               // blocks of the row pass
  int64_t rows_per_blk = 0;       // rows of each block (a multiple of 32)
  int64_t max_slots = 0;          // most tail row slots of one block
  float *zpart = nullptr;         // [nblk * H] per-block head column sums of X^T u
  float *upart = nullptr;         // [nblk] per-block sums of u
  int32_t n_spec = 0;             // features finished one warp each
  int32_t *spec = nullptr;        // [n_spec]
  int32_t *spec_kind = nullptr;   // [n_spec] head index, -1 all-ones, -2 long tail column
  uint8_t *is_spec = nullptr;     // [F]
  double *wd = nullptr;           // [F] omega / d_i at the current lambda
  SlicedPattern xt;               // X over the tail columns (rows gather v)
  SlicedPattern xtt;              // X^T over the tail columns (columns gather u)
};
// head_opt: < 0 no split form (S stays inactive); 0 the head size by the
// byte rule; > 0 that head size (a power of two from 32 to 1024).
rr_status split_build(int64_t N, int64_t F, const int64_t *row_ptr, const int32_t *col_idx,
                      const int64_t *col_ptr, const int32_t *row_idx, int32_t head_opt,
                      int32_t gather_mode, SplitOperator &S, int32_t *err, cudaStream_t st);
void split_free(SplitOperator &S);
rr_status split_set_wd(SplitOperator &S, double omega, const double *d, cudaStream_t st);
// X^T X v + lambda v in the split form, finished by ep; x32_ready: S.xt.xq
// already holds v in FP32 (written by the kernel that made v).
rr_status split_apply(const SplitOperator &S, const double *v, const CscEpilogue &ep,
                      const int32_t *stop, cudaStream_t st, bool x32_ready);

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
  int32_t limit;     // iteration limit of the device-side loop
  uint32_t arrive;   // blocks of the update kernel done (0 between launches)
};
constexpr int kVecGrid = kSMs * 2;   // fixed grid of the vector kernels (deterministic partials)

// Restriction r_c[S] = s_S * sum_{i in S} r1[i] over the member list (members of
// S ascending). Clusters are cut into items of <= item_size members (one warp
// each: kRestrictItem = 256 members, two rounds of four loads per lane, for the
// single-system path; kRestrictItemBatch for the batched path, a block per
// item over a slab of systems); a second kernel sums each cluster's item sums
// (one warp per cluster, lanes strided over the items, a fixed shuffle tree)
// and scales them by s_S into rc.
constexpr int kRestrictItem = 256;
constexpr int kRestrictItemBatch = 4096;
struct RestrictItem {
  int32_t begin, end;   // range in the member list
};
struct RestrictPlan {
  int32_t k = 0;
  int32_t n_items = 0;
  int32_t *item_ptr = nullptr;    // [k+1] items of each cluster
  RestrictItem *items = nullptr;  // [n_items]
  double *item_sum = nullptr;     // [n_items]
  double *rc = nullptr;           // [k] the restricted vector
};
rr_status restrict_plan(int32_t k, const int64_t *cl_ptr, RestrictPlan &plan, int64_t *scratch,
                        cudaStream_t st, int32_t item_size = kRestrictItem);
void restrict_free(RestrictPlan &plan);
// plan.rc = P^T r1 (scaled by s)
rr_status restrict_clusters(const RestrictPlan &plan, const int32_t *members, const double *r1,
                            const double *s, const int32_t *stop, cudaStream_t st);
// e_c = Ainv r_c from plan.rc (also written to rc when non-null).
// FP32 form for the FP32 inner iterations: Ainv32 = FP32 copy of Ainv with
// rows padded to a multiple of 4 (coarse_to_f32), FP32 products and sums.
rr_status coarse_to_f32(int32_t k, const double *Ainv, float *Ainv32, cudaStream_t st);
rr_status coarse_matvec32(int32_t k, const float *Ainv32, const RestrictPlan &plan,
                          const double *s, double *ec, const int32_t *stop, cudaStream_t st);
// The same with the eigendecomposition: e_c = Q (dvec * (Q^T r_c)), Vk = Q^T
// (rows: eigenvectors), Qt = Q (row-major), dvec = 1 / (mu + lambda); tmp[k].
rr_status coarse_matvec_eigen(int32_t k, const double *Vk, const double *Qt, const double *dvec,
                              const RestrictPlan &plan, const double *s, double *tmp, double *ec,
                              const int32_t *stop, cudaStream_t st);
rr_status coarse_matvec(int32_t k, const double *Ainv, const RestrictPlan &plan, const double *s,
                        double *rc, double *ec, const int32_t *stop, cudaStream_t st);
// z2 = z1 + s[l(i)] e_c[l(i)].
// z2_32 (optional): also the FP32 copy of z2 (for an operator apply with x32_ready).
rr_status prolong_add(int64_t F, const int32_t *labels, const double *s, const double *ec,
                      const double *z1, double *z2, const int32_t *stop, cudaStream_t st,
                      float *z2_32 = nullptr);
// z = omega * r / d; if rz_part: per-block <r, z> into rz_part[0..kVecGrid).
// d == nullptr means z = r (no preconditioner).
rr_status jacobi(int64_t F, double omega, const double *r, const double *d, double *z,
                 double *rz_part, const int32_t *stop, cudaStream_t st, float *z32 = nullptr);
// rho = <r,z> (from n_rz partials); beta = rho / rho_old (0 on a (re)start); p = z + beta p.
rr_status pcg_direction(int64_t F, const double *rz_part, int n_rz, const double *z, double *p,
                        PcgScalars *S, cudaStream_t st, float *p32 = nullptr);
// alpha = rho / <p,q>; w += alpha p; r -= alpha q; partial ||r||^2;
// z1 = omega r / d when z1 != nullptr; then the iteration's scalars: rr =
// ||r||^2, rho_old = rho, iter++, convergence and finiteness flags,
// history[iter-1] = ||r|| / ||b|| when iter <= hist_cap.
rr_status pcg_update(int64_t F, const double *rz_part, int n_rz, const double *pq_part, int n_pq,
                     const double *p, const double *q, double *w, double *r, double omega,
                     const double *d, double *z1, double *rr_part, PcgScalars *S,
                     cudaStream_t st, float *z1_32 = nullptr, const double *wd = nullptr,
                     double *history = nullptr, int32_t hist_cap = 0);
// Fresh scalars for a fixed number of plain CG steps inside another solver's
// iteration (no stopping target; stopped when *outer_converged).
rr_status inner_start(PcgScalars *S, const int32_t *outer_converged, cudaStream_t st);
// per-block partial <a, b> into part[0..kVecGrid).
rr_status dot_parts(int64_t n, const double *a, const double *b, double *part, cudaStream_t st);
// (Re)starts PCG: bnorm/target from <b,b> partials if set_bnorm, rr from <r,r> partials.
rr_status pcg_start(const double *bb_part, int n_bb, const double *rr_part, int n_rr, double tol,
                    int32_t set_bnorm, PcgScalars *S, cudaStream_t st);
// *out = fixed-order sum of n partials.
rr_status sum_parts(const double *part, int n, double *out, cudaStream_t st);
rr_status copy_f64(double *dst, const double *src, int64_t n, cudaStream_t st);
// Sets the while-loop condition of a graph: !converged && iter < limit.
rr_status loop_condition(cudaGraphConditionalHandle hc, const PcgScalars *S, cudaStream_t st);
// dst = src (or zero when src == nullptr) for vectors of F entries; device helper kernels.
rr_status axpby(int64_t n, double a, const double *x, double b, double *y, cudaStream_t st);

// ---- k_mlp.cu -----------------------------------------------------------
// e_c = ||r_c|| net(r_c / ||r_c||) from the restriction's item sums.
rr_status mlp_coarse(const rr_mlp *m, const RestrictPlan &plan, const double *s, double *ec,
                     const int32_t *stop, cudaStream_t st);
int32_t mlp_k(const rr_mlp *m);

// ---- k_dense.cu ---------------------------------------------------------
// Dense X (N x F FP32 row-major): k-means in FP64 with blocked row sums (see
// k_dense.cu), the coarse Gram from X onehot, the smoother's statistics and
// the operator's two passes.
struct DenseKmeansScratch {
  int32_t *key;          // [F]
  int64_t *iota;         // [F+1]
  int64_t *cl_ptr;       // [k+2]
  int32_t *members;      // [F]
  int64_t *counts, *cursor;   // [k+1] each
  int32_t *tmp;          // [F]
  int64_t *scan_scratch; // scan_scratch_len(k+1)
  double *mu;            // [k*N]
  double *part;          // [k*nb]
  double *mm;            // [k]
  double *dot;           // [k*F]
  double *dpart;         // dense_dot_part_len(N, F): row-block partial dots
  unsigned long long *changes;
};
int64_t dense_dot_part_len(int64_t N, int64_t F);
rr_status dense_kmeanspp(int64_t N, int64_t F, const float *X, int32_t k, uint64_t seed,
                         int32_t *centers, double *d2, uint8_t *chosen, double *part, int32_t *err,
                         cudaStream_t st);
rr_status dense_lloyd(int64_t N, int64_t F, const float *X, int32_t k, const int32_t *centers,
                      int32_t max_iter, int32_t *labels, DenseKmeansScratch &w, int32_t *iters,
                      cudaStream_t st);
// C (k_eff x N) = cluster sums of the columns (members ascending); G = C C^T.
rr_status dense_coarse_gram(int64_t N, int64_t F, const float *X, int32_t k_eff,
                            const int64_t *cl_ptr, const int32_t *members, double *C, double *G,
                            cudaStream_t st);
// sq_i = ||x_i||^2; gs_i = sum_r |x_ri| sum_j |x_rj| (>= sum_j |(X^T X)_ij|).
// rowabs: [N]; part: [2 dense_col_blocks(N) F].
rr_status dense_colstats(int64_t N, int64_t F, const float *X, double *rowabs, double *part,
                         double *sq, double *gs, cudaStream_t st);
rr_status dense_jacobi(int64_t F, double lambda, const double *sq, const double *gs, double *d,
                       unsigned long long *max_bits, cudaStream_t st);
int64_t dense_col_blocks(int64_t N);
// u = X v (FP32 accumulation when fp32).
rr_status dense_matvec(int64_t N, int64_t F, const float *X, const double *v, double *u,
                       const int32_t *stop, bool fp32, cudaStream_t st);
// Rows of the partial-sum buffer that dense_operator and dense_transposed
// need: part holds dense_part_rows(N, F) * F doubles.
int64_t dense_part_rows(int64_t N, int64_t F);
// X^T X v, then the epilogue ep (one pass over X when F % 4 == 0 and F <= 8192;
// else u = X v into u and X^T u).
rr_status dense_operator(int64_t N, int64_t F, const float *X, const double *v, double *u,
                         double *part, const CscEpilogue &ep, bool fp32, cudaStream_t st);
// t = X^T u in row-block partials, then the epilogue ep (part: [dense_col_blocks(N) * F]).
rr_status dense_transposed(int64_t N, int64_t F, const float *X, const double *u, double *part,
                           const CscEpilogue &ep, bool fp32, cudaStream_t st);

}  // namespace rr
