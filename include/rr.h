/*
 * rr.h — C ABI of the GB300 two-level preconditioned CG solver for the
 * regularised normal equations
 *
 *     (X^T X + lambda I) w = X^T y                       (paper Eq. (1))
 *
 * from Tavernier, Simm, Meerbergen & Moreau, "Two-level preconditioning for
 * Ridge Regression" (arXiv 1806.05826). The paper calls lambda "beta".
 *
 * Conventions for every entry point:
 *  - Return a status code; never abort and never trap on the device. On any
 *    status other than RR_OK, rr_last_error() holds a one-line message
 *    (thread-local, valid until the next call on the same thread).
 *  - Vectors passed as `const double*` / `double*` are DEVICE pointers in FP64
 *    unless the comment says "host". They are caller-owned; the library reads
 *    and writes them only on the handle's stream (rr_options.stream), and the
 *    call returns before that work is complete unless it says otherwise.
 *  - Feature vectors (w, v, labels) are in the caller's feature order 0..F-1;
 *    sample vectors (y) in row order 0..N-1.
 *  - A handle is not thread-safe; different handles may be used from
 *    different threads. The handle owns all of its device memory.
 */
#ifndef RR_H_
#define RR_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rr_handle rr_handle;

typedef enum {
  RR_OK = 0,
  RR_INVALID_ARG = 1,    /* bad sizes, CSR not monotone / out of range, lambda <= 0, k < 1 */
  RR_CUDA_ERROR = 2,     /* a CUDA runtime call failed */
  RR_OOM = 3,            /* device allocation failed */
  RR_NOT_SPD = 4,        /* coarse Cholesky met a pivot <= 0 */
  RR_NOT_CONVERGED = 5,  /* iteration cap reached; w and info still written */
  RR_NONFINITE = 6,      /* NaN/Inf met in a norm or dot product */
  RR_TIMEOUT = 7,        /* a bounded device wait gave up */
  RR_UNSUPPORTED = 8     /* input outside the documented limits */
} rr_status;

/* rr_matrix.layout */
enum { RR_CSR_BINARY = 0,       /* pattern only: every stored entry is 1 */
       RR_DENSE_F32_ROWMAJOR = 1 };

/* rr_options.solver — the preconditioner inside CG */
enum { RR_SOLVER_TWOLEVEL = 0,  /* symmetric two-level cycle (Section 3.1) in PCG */
       RR_SOLVER_CG = 1,        /* no preconditioner (Table 2, "CG") */
       RR_SOLVER_DCG = 2,       /* Jacobi preconditioner (Table 2, "DCG") */
       RR_SOLVER_TLFCG = 3 };   /* the paper's TLFCG (Table 2, Section 4): flexible CG (Alg. 3,
                                   m = 1) whose preconditioner is two CG iterations on A z = r
                                   from z = 0 (the "rougher") followed by the coarse correction of
                                   their residual; no post-smoothing */

/* rr_options.gram — how rr_setup forms the exact coarse Gram C^T C */
enum { RR_GRAM_AUTO = 0,        /* tcgen05 tensor cores (FP16 counts, exact FP32 chunks) when
                                   the counts allow exact chunks, else CUDA cores */
       RR_GRAM_CUDA_CORES = 1 };/* int32 products summed in int64 on CUDA cores */

/* rr_options.gather — the FP32 sliced-gather kernel of the operator applies
 * (both give identical bits: the same sums in the same order) */
enum { RR_GATHER_AUTO = 0,      /* rr_setup times both on each pass of X and keeps the faster */
       RR_GATHER_LANES = 1,     /* each lane sums whole pieces, index words loaded by the lanes */
       RR_GATHER_STAGED = 2,    /* index words streamed through shared memory by bulk copies */
       RR_GATHER_LANES_STAGED = 3 };  /* lanes for the X pass, staged for the X^T pass (the usual
                                   timed choice on Zipf-like data; fixed, e.g. under a profiler,
                                   whose serialisation distorts the timing) */

/* rr_options.coarse — how A_c(lambda)^-1 is formed (Section 4) */
enum { RR_COARSE_CHOLESKY = 0,  /* per lambda: Cholesky factor of A_c, its triangular inverse,
                                   A_c^-1 = L^-T L^-1 */
       RR_COARSE_EIGEN = 1 };   /* once per clustering: X_c^T X_c = Q diag(mu) Q^T (parallel
                                   cyclic Jacobi, FP64); the coarse solve is then applied as
                                   Q (diag(1 / (mu + lambda)) (Q^T r_c)), two mat-vecs, so
                                   rr_set_lambda only rescales a vector (rr_solve_batch forms
                                   Q diag(1 / (mu + lambda)) Q^T once per weight) */

/* rr_options.clustering (Section 3.4) */
enum { RR_CLUSTER_KMEANS = 0,   /* k-means++ seeding and Lloyd steps into k clusters */
       RR_CLUSTER_LEADER = 1 }; /* leader-follower clustering (Algorithm 1), binary X only:
                                   features in index order join the nearest leader (squared
                                   Euclidean distance, the earliest leader on ties) when that
                                   distance is below lf_tol2, else become leaders; leaders are not
                                   updated; k bounds the number of leaders (RR_UNSUPPORTED if more
                                   would be needed) */

/* rr_options.precision */
enum { RR_PREC_FP64 = 0,        /* every operator apply accumulates in FP64 */
       RR_PREC_MIXED = 1 };     /* the operator applies inside the CG iterations gather FP32
                                   copies of the vector and accumulate in FP32; vectors, dot
                                   products, norms, the coarse Cholesky solve and every true
                                   residual b - A w stay FP64, and each restart on the true
                                   residual is an FP64 iterative-refinement step (so
                                   max_restarts bounds the refinement steps) */

/* The feature matrix X (N x F).
 *  CSR_BINARY: row_ptr int64[N+1] (row_ptr[0] = 0, non-decreasing,
 *    row_ptr[N] = nnz) and col_idx int32[nnz], strictly increasing within each
 *    row, each in [0, F). values must be NULL.
 *  DENSE_F32_ROWMAJOR: values float[N*F], row-major; row_ptr/col_idx NULL; nnz ignored;
 *    N*F < 2^34, N <= 4,194,240 and F <= 25600 (the operator stages a whole
 *    vector of F FP64 values in shared memory), else RR_UNSUPPORTED. The clustering runs in
 *    FP64 on the FP32 values (row sums in blocks of 64 rows, ascending).
 *  An unknown layout, or pointers that do not match the layout, give
 *  RR_INVALID_ARG.
 *  on_device = 1: the pointers are device pointers; 0: host pointers (copied
 *  inside rr_setup). rr_setup copies X into the handle; the caller may free
 *  its copy when rr_setup returns. */
typedef struct {
  int64_t n_rows, n_cols, nnz;
  const int64_t *row_ptr;
  const int32_t *col_idx;
  const float *values;
  int32_t layout;
  int32_t on_device;
} rr_matrix;

typedef struct {
  int32_t kmeans_max_iter;      /* Lloyd assignment steps at most (default 50) */
  int32_t max_iter;             /* Krylov iterations at most, all restarts together (default 20000) */
  uint64_t seed;                /* SplitMix64 seed of the k-means++ draws (default 0) */
  const int32_t *init_centers;  /* host int32[k] distinct feature ids, or NULL for k-means++ */
  int32_t solver;               /* RR_SOLVER_* (default RR_SOLVER_TWOLEVEL) */
  int32_t precision;            /* RR_PREC_* (default RR_PREC_FP64) */
  int32_t check_every;          /* iterations between convergence read-backs when use_graphs = 0
                                   (default 8) */
  int32_t max_restarts;         /* true-residual refinement restarts at most (default 5) */
  int32_t use_graphs;           /* 1: the iteration loop runs on the device as a CUDA graph with
                                   a conditional while node (default); 0: host-driven batches of
                                   check_every iterations (same results). The k-means++ rounds are
                                   host-issued kernel chains either way */
  int32_t gram;                 /* RR_GRAM_* (default RR_GRAM_AUTO) */
  int32_t gather;               /* RR_GATHER_* (default RR_GATHER_AUTO) */
  int32_t wait_limit;           /* test hook: spin iterations of the coarse Gram kernel's bounded
                                   mbarrier waits; 0 = default (2^22); negative = each such wait
                                   gives up at once, so rr_setup returns RR_TIMEOUT (the kernel
                                   still waits, with the default limit, for its own copies in
                                   flight, and frees its tensor memory, before it exits) */
  int64_t lloyd_pull_work;      /* a Lloyd step whose count updates (row entries x changed
                                   clusters) exceed this re-gathers the affected features per
                                   feature (pull), else it pushes the updates with integer atomics;
                                   0 = default (2e8). Labels are identical either way */
  int32_t coarse;               /* RR_COARSE_* (default RR_COARSE_CHOLESKY) */
  int32_t split_head;           /* RR_PREC_MIXED, binary X: the operator applies of the FP32
                                   iterations take the columns that hold every row as a rank-one
                                   term and the split_head most frequent other columns as a
                                   row-major bitmap (one read serves X v and X^T u), the rest as
                                   sliced index lists. 0 = automatic (default: the largest power
                                   of two from 32 to 1024 whose columns each hold at least N/8
                                   rows, or none); a power of two from 32 to 1024 = that many;
                                   -1 = no split form (every column as sliced index lists) */
  int32_t clustering;           /* RR_CLUSTER_* (default RR_CLUSTER_KMEANS) */
  double lf_tol2;               /* RR_CLUSTER_LEADER: the squared distance tolerance (a feature
                                   follows when d^2 < lf_tol2); default 1.0 */
  int64_t seed_pull_work;       /* a k-means++ round whose centre c's row entries (estimated as
                                   n_c nnz / N) exceed this counts the overlaps with c column by
                                   column against a bitmap of c's rows (pull), else row by row
                                   with integer atomics (push); 0 = default (7e5), negative =
                                   always push. Centres are identical either way */
  void *stream;                 /* cudaStream_t for all work; NULL = legacy default stream */
} rr_options;

typedef struct {
  int32_t iters;          /* Krylov iterations, all restarts together */
  int32_t restarts;       /* refinement restarts taken */
  int32_t k_eff;          /* non-empty clusters */
  int32_t kmeans_iters;   /* Lloyd assignment steps taken in rr_setup */
  double rel_res;         /* recurrence ||r|| / ||X^T y|| at exit */
  double true_rel_res;    /* ||X^T y - A w|| / ||X^T y|| at exit */
  double omega;           /* Jacobi damping used */
  double setup_ms;        /* wall time of rr_setup (host clock, synchronised) */
  double solve_ms;        /* wall time of this solve (host clock, synchronised) */
  int64_t launches;       /* kernels this call launched */
  int32_t gram_tensor_cores; /* 1 if rr_setup formed the coarse Gram on the tensor cores */
  int32_t fallbacks;      /* rr_solve_fcg with a network: steps redone with the Cholesky
                             coarse solve */
  int32_t gather_staged;  /* FP32 gather kernel in use: bit 0 set if the X pass is staged,
                             bit 1 if the X^T pass is (see rr_options.gather) */
  double setup_phase_ms[8]; /* rr_setup wall time by phase: 0 copy + validation of X, 1 CSC
                               build, 2 k-means++ seeding, 3 Lloyd steps, 4 compaction + member
                               lists, 5 counts + coarse Gram, 6 coarse factor + smoother,
                               7 sliced patterns + solve workspace */
} rr_info;

/* Fills *o with the defaults listed above. */
void rr_default_options(rr_options *o);

/* Builds the two-level preconditioner for X at regularisation lambda
 * (Section 3): k-means++ clustering of the F feature columns into k clusters
 * (Section 3.4, Euclidean distance), the prolongation P(i,S) = 1/sqrt(n_S)
 * (Eq. (prolong)), the Galerkin coarse operator P^T A P = X_c^T X_c +
 * lambda I (Section 3.2), its Cholesky factor (Section 4), and the damped
 * Jacobi smoother. Empty clusters are dropped (info k_eff). Synchronises the
 * stream before returning, except (binary X) for the coarse factor and
 * inverse, which are left running on a stream of the handle's own: every later
 * call that uses the coarse level waits for them (a solve's stream waits on
 * their event; rr_set_lambda, rr_prepare_lambdas, rr_solve_batch, rr_harvest,
 * rr_bayes and rr_get_coarse wait on the host; in rr_solve_many only this
 * handle's problem waits), so that forks (rr_fork_lambda) build their own
 * factors meanwhile. A non-positive pivot of that factor is reported by the
 * first solve (RR_NOT_SPD). o may be NULL (defaults). On success *out owns
 * the handle; release it with rr_free.
 * Errors: RR_INVALID_ARG (see rr_matrix; lambda <= 0 or not finite; k < 1 or
 * k > F; repeated or out-of-range init_centers), RR_UNSUPPORTED (nnz >= 2^31,
 * k > 16384, a row holding more than 8191 features of one cluster), RR_TIMEOUT (a bounded
 * device wait expired),
 * RR_NOT_SPD, RR_OOM, RR_CUDA_ERROR. */
rr_status rr_setup(const rr_matrix *X, double lambda, int32_t k, const rr_options *o,
                   rr_handle **out);

/* Re-targets the handle to another lambda, keeping the clustering: rebuilds
 * the coarse operator, its factor and the smoother (Section 4: the Cholesky
 * factor must be recomputed when beta changes). Synchronises the stream. */
rr_status rr_set_lambda(rr_handle *h, double lambda);

/* Prepares the coarse level of up to 8 further lambdas ahead of time (no
 * counterpart in the paper, which refactors the coarse operator whenever beta
 * changes, Section 4): the Cholesky factor, its inverse and the smoother of
 * each lambda are computed on a second stream, overlapping whatever the
 * handle's stream runs meanwhile (a solve); rr_set_lambda to exactly one of
 * these lambdas then waits for its work and swaps it in instead of
 * factoring. Returns without waiting for the factors; a later call replaces
 * the prepared set (after the earlier one has finished); an RR_COARSE_EIGEN
 * handle needs none (a no-op). lambdas: host double[n], each positive and
 * finite. Errors: RR_INVALID_ARG (NULL handle, n outside [0, 8], a bad
 * lambda), RR_OOM, RR_CUDA_ERROR; a factor that meets a non-positive pivot
 * is reported by the rr_set_lambda that installs it (RR_NOT_SPD). */
rr_status rr_prepare_lambdas(rr_handle *h, const double *lambdas, int32_t n);

/* A handle for another lambda on the same X (Section 2 poses one X with
 * several beta; Section 4 refactors only the coarse operator when beta
 * changes). The fork shares base's setup that does not depend on lambda: X
 * and its transpose, the clustering, the coarse Gram and the operator's
 * patterns. It owns the coarse operator, factor and inverse at `lambda`, the
 * smoother, the solve vectors and scalars, the operator's intermediate
 * vectors and a stream of its own (non-blocking): rr_solve and rr_set_lambda
 * on it behave as on a handle set up at that lambda with the same clustering
 * (the same bits), and rr_solve_many solves base and forks concurrently. The
 * smoother is built before returning; the coarse factor is left running on
 * the fork's stream, and rr_solve_many starts the fork's problem only once it
 * is done (the other problems start at once). base must outlive its forks, and
 * is not otherwise changed; a fork of a fork, or of a dense-X handle, is not
 * supported. rr_solve_batch, rr_harvest, rr_bayes and rr_prepare_lambdas
 * reject forks (RR_UNSUPPORTED).
 * rr_free(fork) frees only what the fork owns. Device memory: about 13 F + 3 N
 * doubles plus the coarse level (3 k_eff^2 doubles) and the operator's
 * intermediate vectors. Errors: RR_INVALID_ARG (NULL argument, lambda not
 * positive and finite), RR_UNSUPPORTED, RR_OOM, RR_CUDA_ERROR; a non-positive
 * pivot of the fork's factor is reported by its first solve (RR_NOT_SPD). */
rr_status rr_fork_lambda(rr_handle *base, double lambda, rr_handle **out);

/* Solves Eq. (1) for one right-hand side by CG preconditioned as
 * rr_options.solver says (RR_SOLVER_TLFCG: flexible CG, Algorithm 3 with
 * m = 1, as rr_solve_fcg without a network), from w_0 = 0 (Algorithm 3's
 * initialisation), until
 * the recurrence residual satisfies ||r|| <= tol ||X^T y||; then checks the
 * true residual and restarts on the correction while it is above tol
 * (at most max_restarts times).
 * y: device double[N]. w: device double[F], overwritten with the solution.
 * info may be NULL. Synchronises the stream before returning.
 * Errors: RR_INVALID_ARG (tol not in (0, 1)), RR_NOT_CONVERGED (cap reached;
 * w holds the last iterate), RR_NONFINITE, RR_CUDA_ERROR. */
rr_status rr_solve(rr_handle *h, const double *y, double *w, double tol, rr_info *info);

/* Solves Eq. (1) for many right-hand sides and many weights at once: for every
 * target j < nrhs and weight l < nlam, (X^T X + lambdas[l] I) w = X^T y_j
 * (Section 2 poses one X with several b and several beta). The nrhs * nlam
 * systems share the handle's clustering (Section 3.4) and advance together
 * through the two-level PCG of rr_solve: each operator apply is one
 * sparse-times-dense pass pair over X's pattern for a slab of 64 systems, the
 * coarse level has one Cholesky factor per weight, and each system keeps its
 * own CG scalars and stops on its own residual ||r|| <= tol ||X^T y_j||.
 * Precision, whatever the handle's: the operator applies inside CG (also
 * those of the smoother) gather FP32 copies of the vectors with FP32
 * accumulation; FP64 vectors, dot products, norms, coarse level (Cholesky
 * factors and coarse products); an FP64 true residual after CG
 * stops, restarting each system on its correction while it is above tol
 * (at most max_restarts times per system).
 *   Y        device double[nrhs * N], target j at Y + j*N.
 *   lambdas  host double[nlam], each > 0 and finite.
 *   W        device double[nlam * nrhs * F], overwritten: the solution of
 *            (j, l) at W + (l*nrhs + j)*F.
 *   infos    host rr_info[nlam * nrhs] (index l*nrhs + j) or NULL; solve_ms
 *            is the time of the whole batch.
 * The handle's own lambda and rr_solve state are untouched. Device work
 * space of about 13 F + 3 N doubles per system is kept in the handle and
 * reused by later calls with as many or fewer systems and weights.
 * Requires RR_SOLVER_TWOLEVEL and binary X. Synchronises the stream before
 * returning.
 * Errors: RR_INVALID_ARG, RR_UNSUPPORTED (other solver, dense X), RR_OOM, RR_NOT_SPD,
 * RR_NOT_CONVERGED (some system hit a cap; W holds the last iterates and
 * infos say which), RR_NONFINITE, RR_CUDA_ERROR. */
rr_status rr_solve_batch(rr_handle *h, int32_t nrhs, const double *Y, int32_t nlam,
                         const double *lambdas, double *W, double tol, rr_info *infos);

/* Solves nprob independent problems of different sizes, problem i being
 * Eq. (1) for the X, clustering, lambda and solver of handle hs[i] with target
 * ys[i] (device double[N_i]) into ws[i] (device double[F_i]), exactly as
 * rr_solve would, but in one CUDA graph: the CG loop of every problem is a
 * conditional while node of one graph, the loops being independent branches,
 * so the kernels of small problems run concurrently with those of others.
 * (The paper solves one problem at a time; this is the batched form for many
 * unrelated problems.) True-residual refinement per problem as rr_solve (a
 * relaunch of the graph continues the problems that restart). All work runs on
 * `stream` (cudaStream_t) during the call; the handles must be distinct, and
 * each must have been set up with use_graphs = 1 or 0 alike (the graph is
 * always used). infos: host rr_info[nprob] or NULL; solve_ms is the time of
 * the whole call. Returns RR_OK when every problem reached tol, else the
 * first failing status kind (RR_NOT_CONVERGED / RR_NONFINITE); RR_UNSUPPORTED
 * if a handle's solver is RR_SOLVER_TLFCG. Synchronises. */
rr_status rr_solve_many(int32_t nprob, rr_handle *const *hs, const double *const *ys,
                        double *const *ws, double tol, void *stream, rr_info *infos);

/* ---- Flexible CG and the learned coarse correction ----------------------
 * Algorithm 3 (flexible CG, FCG(m) with m = 1: each direction is
 * A-orthogonalised against the previous one, which allows a preconditioner
 * that changes from step to step) with the two-level cycle of Section 3.1 as
 * its preconditioner, from w_0 = 0. The cycle's coarse solve e_c = A_c^-1 r_c
 * is either the Cholesky solve (net == NULL: the paper's own method in FCG
 * form) or a learned correction e_c = ||r_c|| net(r_c / ||r_c||) from an
 * rr_mlp (the paper has no learned part). With a network, a step falls back
 * to the Cholesky coarse solve when <r, z> <= 0, when z or the step length is
 * not finite, or when the step would not reduce ||r||_2 (checked in FP64
 * before the update, from <p,r>, <r,q>, ||q||^2); info->fallbacks counts them.
 * Stopping, true-residual refinement, precision and graphs as in rr_solve.
 * y: device double[N]; w: device double[F]. The network's k must equal the
 * handle's k_eff. Errors as rr_solve, RR_INVALID_ARG on a k mismatch. */
typedef struct rr_mlp rr_mlp;
rr_status rr_solve_fcg(rr_handle *h, const rr_mlp *net, const double *y, double *w, double tol,
                       rr_info *info);

/* Training pairs for the learned correction, harvested from the batched
 * two-level PCG of rr_solve_batch at one weight: for every system j and
 * iteration i, x = r_c = P^T r1 (the restricted residual after
 * pre-smoothing) and t = P^T (e - z1), e = wref_j - w_i the error of the
 * iterate and z1 the pre-smoothing step (so that P t is the part of the
 * remaining error that the coarse space can carry).
 *   Y     device double[nrhs * N] (target j at Y + j*N)
 *   Wref  device double[nrhs * F], the solutions (e.g. from rr_solve_batch at
 *         a tighter tol)
 *   Xp,Tp device float[max_pairs * k_eff] each, pair p at row p
 *   n_pairs (host) receives the number of pairs written: every (j, i) with
 *   i below max_iter and system j still iterating (its recurrence residual
 *   above tol ||X^T y_j||), in order of i then j, cut at max_pairs.
 * Runs at most max_iter iterations (no refinement restarts). Binary X only
 * (RR_UNSUPPORTED on a dense handle). Synchronises. */
rr_status rr_harvest(rr_handle *h, int32_t nrhs, const double *Y, double lambda, const double *Wref,
                     double tol, int32_t max_iter, float *Xp, float *Tp, int64_t max_pairs,
                     int64_t *n_pairs);

/* The network: h1 = relu(W1 x + b1), h2 = relu(W2 h1 + b2), o = W3 h2 + b3,
 * x and o of length k, hidden width H (a positive multiple of 128). Weights in
 * FP32 (the master copy Adam updates) with BF16 copies for the tensor-core
 * products; training minimises 0.5/B sum_b ||o_b - t_b||^2.
 * params_host: the parameters packed as W1 [H x k] row-major, b1 [H],
 * W2 [H x H], b2 [H], W3 [k x H], b3 [k] (rr_mlp_param_count(k, H) floats).
 * max_batch bounds the rows of one forward / gradient / training step.
 * All work runs on `stream` (cudaStream_t, NULL = legacy default stream). */
int64_t rr_mlp_param_count(int32_t k, int32_t hidden);
rr_status rr_mlp_create(int32_t k, int32_t hidden, int32_t max_batch, const float *params_host,
                        void *stream, rr_mlp **out);
rr_status rr_mlp_set_params(rr_mlp *m, const float *params_host);
rr_status rr_mlp_get_params(const rr_mlp *m, float *params_host);
/* The loss metric (no counterpart in the paper): with W_host (host float[k x k]
 * row-major, symmetric, e.g. the coarse operator A_c scaled), rr_mlp_grad and
 * rr_mlp_train minimise 0.5/B sum_b (o_b - t_b)^T W (o_b - t_b), whose output
 * gradient W (o - t) / B is one more tensor-core product per batch (W in
 * BF16); NULL restores the plain loss. Errors: RR_INVALID_ARG (NULL network,
 * a non-finite entry, W not symmetric to 1e-6 of its largest entry),
 * RR_OOM, RR_CUDA_ERROR. */
rr_status rr_mlp_set_metric(rr_mlp *m, const float *W_host);
/* out (device float[B x k]) = o for the rows of X (device float[B x k]), as given. */
rr_status rr_mlp_forward(rr_mlp *m, int32_t B, const float *X, float *out);
/* Loss and its gradient for the rows of X with targets T (device float[B x k]),
 * as given; grads_host (packed like the parameters) and loss_host may be NULL. */
rr_status rr_mlp_grad(rr_mlp *m, int32_t B, const float *X, const float *T, float *grads_host,
                      float *loss_host);
/* `steps` Adam steps (lr, beta1 = 0.9, beta2 = 0.999, eps = 1e-8) on batches of
 * `batch` pairs drawn uniformly (SplitMix64 at counter step*batch + b) from the
 * n_pairs rows of Xp, Tp (device float[n_pairs x k]); each pair is divided by
 * ||x|| (the homogeneous scaling of the learned correction). loss_host: host
 * float[steps] of the batch losses, or NULL. Synchronises the stream. */
rr_status rr_mlp_train(rr_mlp *m, int64_t n_pairs, const float *Xp, const float *Tp, int32_t batch,
                       int32_t steps, float lr, uint64_t seed, float *loss_host);
void rr_mlp_free(rr_mlp *m);

/* out = (X^T X + lambda I) v (Eq. (1)'s operator, applied matrix-free as
 * u = X v then X^T u + lambda v). v, out: device double[F]; may not alias.
 * Accumulates in FP32 when the handle was set up with RR_PREC_MIXED (the
 * operator of its CG iterations), else in FP64; likewise rr_rhs and rr_matvec.
 * rr_solve's right-hand side and true residuals are always FP64. */
rr_status rr_apply(rr_handle *h, const double *v, double *out);

/* z = M^{-1} r for the handle's preconditioner (the two-level cycle of
 * Section 3.1 for RR_SOLVER_TWOLEVEL). r, z: device double[F]; may not alias. */
rr_status rr_precondition(rr_handle *h, const double *r, double *z);

/* b = X^T y (Eq. (1)'s right-hand side; also the transposed mat-vec alone).
 * y: device double[N]; b: device double[F]. */
rr_status rr_rhs(rr_handle *h, const double *y, double *b);

/* u = X v (the first half of the operator, Section 1's mat-vec).
 * v: device double[F]; u: device double[N]. */
rr_status rr_matvec(rr_handle *h, const double *v, double *u);

/* Copies the final cluster of every feature (compacted to 0..k_eff-1, empty
 * clusters dropped in order) to host int32[F]. Synchronises. */
rr_status rr_get_labels(const rr_handle *h, int32_t *labels_host);

/* Copies the k initial centres (feature ids) used by Lloyd to host int32[k]. */
rr_status rr_get_centers(const rr_handle *h, int32_t *centers_host);

/* Copies the coarse operator A_c (k_eff x k_eff, row-major, FP64, lower
 * triangle mirrored) and the exact coarse Gram G = C^T C (k_eff x k_eff,
 * int64) to host buffers; either may be NULL. G exists for binary X only:
 * a non-NULL G_host on a dense handle gives RR_UNSUPPORTED. Synchronises. */
rr_status rr_get_coarse(const rr_handle *h, double *Ac_host, int64_t *G_host);

/* Number of non-empty clusters, Jacobi damping and sizes of the handle. Any
 * pointer may be NULL. */
rr_status rr_query(const rr_handle *h, int64_t *n_rows, int64_t *n_cols, int32_t *k_eff,
                   double *omega, double *lambda);

/* out = (X^T X + lambda I) v for binary X given directly as device CSR
 * (row_ptr int64[n_rows+1], col_idx int32[nnz]) and its transposed copy CSC
 * (col_ptr int64[n_cols+1], row_idx int32[nnz]), without a handle and without
 * allocating any device memory. (No counterpart in the paper: this is an
 * interface for callers that may not allocate.)
 *
 * Who needs it: code that runs where cudaMalloc is off limits, for example
 * inside a framework that owns every byte of device memory through its own
 * pool and forbids other allocations, or code on a latency-critical path that
 * cannot afford cudaMalloc's implicit device synchronisation. rr_apply needs a
 * handle, and rr_setup allocates.
 *
 * The intermediate u = X v is kept in a fixed 32 MiB array inside the library,
 * so n_rows may not exceed 4,194,304 (RR_UNSUPPORTED beyond). With CUDA's lazy
 * module loading (the default), that array is reserved on a device when the
 * first call on that device loads this part of the library and looks up the
 * array's address (cudaGetSymbolAddress); it then stays reserved until the
 * process exits. So make one warm-up call on each device before a memory pool
 * takes the device's memory and before any stream capture; every later call
 * allocates nothing. All calls share the array: calls whose work overlaps on
 * the GPU (different streams, or different host threads on the same device)
 * race on it and must be serialised by the caller. Every call writes
 * u[0, n_rows) before reading it, so no state carries over.
 *
 * Preconditions the library does not check: row_ptr and col_ptr are
 * non-decreasing from 0 to the same nnz, and every col_idx lies in
 * [0, n_cols) and every row_idx in [0, n_rows). An index outside its range is
 * skipped (never read past a vector), so such input gives an undefined result
 * but no out-of-bounds access; pointer arrays that run past their index
 * arrays are undefined behaviour. The Python binding checks the lengths.
 * v, out: device double[n_cols], may not alias. stream: cudaStream_t or NULL.
 * Returns before the work completes. Errors: RR_INVALID_ARG (sizes < 1, a NULL
 * pointer, v == out), RR_UNSUPPORTED, RR_CUDA_ERROR. */
rr_status rr_apply_noalloc(int64_t n_rows, int64_t n_cols, const int64_t *row_ptr,
                           const int32_t *col_idx, const int64_t *col_ptr, const int32_t *row_idx,
                           double lambda, const double *v, double *out, void *stream);

/* The coarse eigendecomposition of an RR_COARSE_EIGEN handle (Section 4: a
 * decomposition of X_c reused for every lambda): mu_host[k_eff] the
 * eigenvalues of X_c^T X_c (unordered), Q_host[k_eff x k_eff] row-major with
 * column e the eigenvector of mu[e], *sweeps the Jacobi sweeps taken. Any
 * output may be NULL. Errors: RR_INVALID_ARG (NULL handle or no eigen
 * decomposition), RR_CUDA_ERROR. */
rr_status rr_get_eigen(const rr_handle *h, double *mu_host, double *Q_host, int32_t *sweeps);

/* ---- Bayesian ridge regression by Gibbs sampling (Section 2, Eq. (ni_xtx)).
 * Likelihood y ~ N(X w, tau^-1 I), prior w ~ N(0, lambda^-1 I), hyperpriors
 * lambda ~ Gamma(alpha, beta) and tau ~ Gamma(a_tau, b_tau) (shape, rate).
 * Sample t draws w given (lambda, tau) by noise injection, solving
 *   (X^T X + (lambda/tau) I) w = X^T (y + e1) + e2 / tau,
 *   e1 ~ N(0, tau^-1 I_N), e2 ~ N(0, lambda I_F),
 * with the handle's solver (the clustering is kept; the coarse operator is
 * rebuilt at lambda/tau, which an RR_COARSE_EIGEN handle does with two
 * mat-vec scalings and no factorisation), then lambda | w ~ Gamma(alpha +
 * F/2, beta + ||w||^2 / 2) and, unless a_tau <= 0 (tau fixed at tau0),
 * tau | w ~ Gamma(a_tau + N/2, b_tau + ||y - X w||^2 / 2). All draws come
 * from a counter-based generator on (seed, stream, index): SplitMix64 (Steele,
 * Lea & Flood 2014) with the stream base mix(mix(seed) xor stream *
 * 0xD1B54A32D192ED03) and uniform i = (mix(base + (i + 1) * 0x9E3779B97F4A7C15)
 * >> 11) 2^-53; normal i by Box-Muller from the uniforms i and 2^40 + i; e1 of
 * sample t on stream 2t, e2 on stream 2t + 1; Gamma by Marsaglia & Tsang
 * (2000) on stream 2^20 + 2t (lambda) and 2^20 + 2t + 1 (tau), attempt j
 * taking its normal from the uniforms 2j, 2j + 1 and its u from 2^32 + j. */
typedef struct {
  double alpha, beta;     /* lambda ~ Gamma(alpha, beta); alpha + F/2 >= 1 */
  double a_tau, b_tau;    /* tau ~ Gamma(a_tau, b_tau); a_tau <= 0: tau fixed */
  double lambda0, tau0;   /* the chain's starting values, > 0 */
  uint64_t seed;
  double tol;             /* each solve's relative residual, in (0, 1) */
} rr_bayes_params;

/* Runs n_samples Gibbs steps. y: device double[n_rows]. w_mean: device
 * double[n_cols] or NULL, the mean of w over the samples t >= burnin.
 * lam_trace, tau_trace: host double[n_samples] or NULL, lambda and tau drawn
 * at each step (after its solve); iters: host int32[n_samples] or NULL, the
 * PCG iterations of each solve. The handle's lambda is restored before
 * returning. Synchronous. Errors: RR_INVALID_ARG (NULL handle or y, a
 * parameter out of range, n_samples < 1, burnin outside [0, n_samples)),
 * RR_NOT_CONVERGED or RR_NONFINITE from a solve (the chain stops there, the
 * traces hold the steps done), RR_CUDA_ERROR. */
rr_status rr_bayes(rr_handle *h, const double *y, const rr_bayes_params *p, int32_t n_samples,
                   int32_t burnin, double *w_mean, double *lam_trace, double *tau_trace,
                   int32_t *iters);

/* The batched engine's sparse-times-dense variant chosen by its autotuner for
 * the last rr_solve_batch (or rr_harvest) on h: systems per slab (32, 64 or
 * 128: the columns one warp carries through a pass over X) and row segments
 * in flight per warp (4 or 8). Every candidate is timed on the two FP32
 * passes of one operator apply over all slabs at the first batched call for
 * a given (N, F, nnz, padded batch width) in the process, and the fastest is
 * kept; apply_ms is its time (both passes, every system of the batch). All
 * variants sum in the same order, so the choice does not change results.
 * (No counterpart in the paper.) Any output pointer may be NULL. Errors:
 * RR_INVALID_ARG (NULL handle, or no batched call yet). */
rr_status rr_query_batch(const rr_handle *h, int32_t *slab_width, int32_t *unroll,
                         double *apply_ms);

/* Number of kernels the library has launched from the calling thread since it
 * was loaded (counts every launch of every call, setup included). */
int64_t rr_launch_count(void);

/* Releases the handle and all of its device memory (synchronises its stream). */
void rr_free(rr_handle *h);

/* Message of the last failed call on this thread ("" if none). */
const char *rr_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* RR_H_ */
