// Leader-follower clustering of the features (Section 3.4, Algorithm 1) for
// binary X: the features are visited in index order; each joins the nearest
// leader when the squared Euclidean distance
//
//   d(i, s)^2 = n_i + n_s - 2 |R_i and R_s|     (R_j: the rows of column j)
//
// is below tol2, else it becomes a new leader; leaders are never updated, the
// first leader is feature 0, and ties go to the earliest leader. The result is
// that of the sequential loop, bit for bit (integer distances, one fixed rule).
//
// GPU form: the features in steps of kLfBlock = 64 consecutive ones. Per step
//   mark     each step feature ORs its bit into rowmask[r] for its rows;
//   count    one CTA per step feature: the overlaps with every committed
//            leader through the per-row leader lists (a leader's id sits in
//            the list of each of its rows), counted in shared memory, and the
//            overlaps with the earlier step features through rowmask; the
//            nearest committed leader (d^2, id) with the zero-overlap leaders
//            represented by the earliest leader of smallest size;
//   resolve  one thread walks the step's features in order against those
//            results and the step's new leaders (their overlaps from the pair
//            counts): the sequential decision, exactly;
//   commit   the step's new leaders are appended to the lists of their rows;
//            rowmask is cleared.
// A row holds at most its own length of leaders (each is one of its columns),
// so the lists live in an array laid out like col_idx.
#include <vector>

#include "common.cuh"
#include "handle.h"
#include "kernels.h"

namespace rr {

namespace {

constexpr int kLfBlock = 64;
constexpr int64_t kLfTaskRows = 2048;   // rows of one task (a feature's rows in tasks)

// A step feature's rows [e0, e1) of its CSC column; first: the task that
// starts the column.
struct LfTask {
  int32_t b, first;
  int64_t e0, e1;
};

__global__ void k_lf_mark(const LfTask *__restrict__ tasks, const int32_t *__restrict__ row_idx,
                          unsigned long long *__restrict__ rowmask) {
  pdl_wait();
  const LfTask t = tasks[blockIdx.x];
  const unsigned long long bit = 1ULL << t.b;
  for (int64_t e = t.e0 + threadIdx.x; e < t.e1; e += blockDim.x)
    atomicOr(&rowmask[row_idx[e]], bit);
}

// Overlaps of a task's rows with every committed leader (through the per-row
// leader lists) and with the earlier step features (through rowmask), counted
// in shared memory, then added into the step feature's global counters.
__global__ void k_lf_count(const LfTask *__restrict__ tasks, const int32_t *__restrict__ row_idx,
                           const int64_t *__restrict__ row_ptr, const int32_t *__restrict__ rl,
                           const int32_t *__restrict__ rl_cnt,
                           const unsigned long long *__restrict__ rowmask,
                           const LfState *__restrict__ S, int32_t cap, int32_t *__restrict__ gcnt,
                           int32_t *__restrict__ gpair) {
  pdl_wait();
  extern __shared__ int32_t cnt[];
  __shared__ int32_t pc[kLfBlock];
  const LfTask t = tasks[blockIdx.x];
  const int32_t L0 = S->L;
  for (int32_t s = threadIdx.x; s < L0; s += blockDim.x) cnt[s] = 0;
  if (threadIdx.x < kLfBlock) pc[threadIdx.x] = 0;
  __syncthreads();
  const unsigned long long below = t.b == 0 ? 0ULL : (~0ULL >> (64 - t.b));
  for (int64_t e = t.e0 + threadIdx.x; e < t.e1; e += blockDim.x) {
    const int32_t r = row_idx[e];
    const int64_t q0 = row_ptr[r];
    const int64_t len = row_ptr[r + 1] - q0;
    const int32_t qn = (int32_t)min((int64_t)rl_cnt[r], len);
    for (int32_t q = 0; q < qn; ++q) {
      const int32_t s = rl[q0 + q];
      if (s >= 0 && s < L0) atomicAdd(&cnt[s], 1);
    }
    unsigned long long m = rowmask[r] & below;
    while (m) {
      atomicAdd(&pc[__ffsll((long long)m) - 1], 1);
      m &= m - 1;
    }
  }
  __syncthreads();
  int32_t *g = gcnt + (int64_t)t.b * cap;
  for (int32_t s = threadIdx.x; s < L0; s += blockDim.x)
    if (cnt[s]) atomicAdd(&g[s], cnt[s]);
  if (threadIdx.x < kLfBlock && pc[threadIdx.x])
    atomicAdd(&gpair[t.b * kLfBlock + threadIdx.x], pc[threadIdx.x]);
}

// The nearest committed leader of each step feature, (d^2, id) packed so that
// the smallest key is the nearest, earliest leader; the leaders it shares no
// row with are represented by the earliest leader of smallest size. Clears
// the feature's counters for the next step.
__global__ void k_lf_best(int64_t F, int64_t f0, const int64_t *__restrict__ col_ptr,
                          const int32_t *__restrict__ nlead, const LfState *__restrict__ S,
                          int32_t cap, int32_t *__restrict__ gcnt,
                          unsigned long long *__restrict__ best) {
  pdl_wait();
  __shared__ unsigned long long red[kWarps];
  const int b = blockIdx.x;
  const int64_t i = f0 + b;
  if (i >= F) return;
  const int32_t L0 = S->L;
  const int64_t n_i = col_ptr[i + 1] - col_ptr[i];
  int32_t *g = gcnt + (int64_t)b * cap;
  unsigned long long key = ~0ULL;
  for (int32_t s = threadIdx.x; s < L0; s += blockDim.x) {
    const int32_t c = g[s];
    if (c > 0) {
      const int64_t d2 = n_i + nlead[s] - 2 * (int64_t)c;
      const unsigned long long k2 = ((unsigned long long)d2 << 32) | (uint32_t)s;
      key = k2 < key ? k2 : key;
      g[s] = 0;
    }
  }
  if (threadIdx.x == 0 && L0 > 0) {
    const unsigned long long k2 =
        ((unsigned long long)(n_i + S->min_n) << 32) | (uint32_t)S->min_s;
    key = k2 < key ? k2 : key;
  }
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long t = __shfl_xor_sync(0xffffffffu, key, o);
    key = t < key ? t : key;
  }
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = key;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long k2 = red[0];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) k2 = red[w] < k2 ? red[w] : k2;
    best[b] = k2;
  }
}

// The sequential decision over the step's features (one thread).
__global__ void k_lf_resolve(int64_t F, int64_t f0, const int64_t *__restrict__ col_ptr,
                             double tol2, int32_t cap, const unsigned long long *__restrict__ best,
                             const int32_t *__restrict__ pair, int32_t *__restrict__ lead,
                             int32_t *__restrict__ nlead, int32_t *__restrict__ labels,
                             LfState *__restrict__ S) {
  pdl_wait();
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  int32_t L = S->L;
  const int32_t Lstart = L;
  int32_t nnew = 0;
  int32_t min_n = S->min_n, min_s = S->min_s;
  const int nb = (int)(F - f0 < kLfBlock ? F - f0 : kLfBlock);
  for (int b = 0; b < nb; ++b) {
    const int64_t i = f0 + b;
    const int64_t n_i = col_ptr[i + 1] - col_ptr[i];
    int64_t d2b = -1;
    int32_t sb = -1;
    if (Lstart > 0) {
      d2b = (int64_t)(best[b] >> 32);
      sb = (int32_t)(best[b] & 0xffffffffULL);
    }
    // the step's earlier new leaders, in creation order (larger ids than
    // every committed leader: only a strictly smaller distance wins)
    for (int t = 0; t < nnew; ++t) {
      const int jb = S->newpos[t];
      const int64_t d2 = n_i + nlead[Lstart + t] - 2 * (int64_t)pair[b * kLfBlock + jb];
      if (sb < 0 || d2 < d2b) {
        d2b = d2;
        sb = Lstart + t;
      }
    }
    if (sb >= 0 && (double)d2b < tol2) {
      labels[i] = sb;
      continue;
    }
    if (L >= cap) {
      S->overflow = 1;
      labels[i] = 0;
      continue;
    }
    lead[L] = (int32_t)i;
    nlead[L] = (int32_t)n_i;
    labels[i] = L;
    S->newpos[nnew++] = b;
    if (L == 0 || n_i < min_n) {
      min_n = (int32_t)n_i;
      min_s = L;
    }
    ++L;
  }
  S->L = L;
  S->nnew = nnew;
  S->min_n = min_n;
  S->min_s = min_s;
}

// The step's new leaders join the lists of their rows; rowmask and the pair
// counters are cleared for the next step.
__global__ void k_lf_commit(const LfTask *__restrict__ tasks, const int32_t *__restrict__ row_idx,
                            const int64_t *__restrict__ row_ptr, int32_t *__restrict__ rl,
                            int32_t *__restrict__ rl_cnt, unsigned long long *__restrict__ rowmask,
                            const LfState *__restrict__ S, int32_t *__restrict__ gpair,
                            int32_t *__restrict__ err) {
  pdl_wait();
  const LfTask t = tasks[blockIdx.x];
  const int32_t nnew = S->nnew;
  int32_t id = -1;
  for (int q = 0; q < nnew; ++q)
    if (S->newpos[q] == t.b) id = S->L - nnew + q;
  for (int64_t e = t.e0 + threadIdx.x; e < t.e1; e += blockDim.x) {
    const int32_t r = row_idx[e];
    if (id >= 0) {
      const int32_t pos = atomicAdd(&rl_cnt[r], 1);
      if (pos < row_ptr[r + 1] - row_ptr[r])
        rl[row_ptr[r] + pos] = id;
      else
        set_dev_error(err, DEV_BAD_INDEX);
    }
    rowmask[r] = 0ULL;
  }
  if (t.first && threadIdx.x < kLfBlock) gpair[t.b * kLfBlock + threadIdx.x] = 0;
}

__global__ void k_lf_init(LfState *S) {
  S->L = 0;
  S->nnew = 0;
  S->min_n = 0;
  S->min_s = 0;
  S->overflow = 0;
}

}  // namespace

rr_status leader_follower(int64_t N, int64_t F, const int64_t *row_ptr, const int64_t *col_ptr,
                          const int32_t *row_idx, double tol2, int32_t cap, LfBuffers &lb,
                          int32_t *labels, int32_t *centers, int32_t *n_lead_out, int32_t *err,
                          cudaStream_t st) {
  if (cap < 1 || cap > kLfMaxLeaders) {
    rr_set_error("leader-follower: the leader capacity k must be in [1, %d]", kLfMaxLeaders);
    return RR_UNSUPPORTED;
  }
  // the tasks of every step, from the column pointers
  std::vector<int64_t> cp(F + 1);
  RR_CUDA(cudaMemcpyAsync(cp.data(), col_ptr, sizeof(int64_t) * (F + 1), cudaMemcpyDeviceToHost, st));
  RR_CUDA(cudaStreamSynchronize(st));
  const int64_t n_steps = (F + kLfBlock - 1) / kLfBlock;
  std::vector<LfTask> tasks;
  std::vector<int64_t> step_ptr(n_steps + 1, 0);
  for (int64_t s = 0; s < n_steps; ++s) {
    for (int64_t i = s * kLfBlock; i < std::min<int64_t>(F, (s + 1) * kLfBlock); ++i)
      for (int64_t e0 = cp[i]; e0 < cp[i + 1]; e0 += kLfTaskRows)
        tasks.push_back(LfTask{(int32_t)(i - s * kLfBlock), e0 == cp[i] ? 1 : 0, e0,
                               std::min<int64_t>(cp[i + 1], e0 + kLfTaskRows)});
    step_ptr[s + 1] = (int64_t)tasks.size();
  }
  LfTask *d_tasks = nullptr;
  int32_t *gcnt = nullptr, *gpair = nullptr;
  DevArena tmp;
  struct Release {
    DevArena &a;
    ~Release() { a.free_all(); }   // cudaFree waits for the work queued on the device
  } release_tmp{tmp};
  RR_TRY(tmp.alloc(&d_tasks, std::max<size_t>(tasks.size(), 1)));
  RR_TRY(tmp.alloc(&gcnt, (int64_t)kLfBlock * cap));
  RR_TRY(tmp.alloc(&gpair, kLfBlock * kLfBlock));
  if (!tasks.empty())
    RR_CUDA(cudaMemcpyAsync(d_tasks, tasks.data(), sizeof(LfTask) * tasks.size(),
                            cudaMemcpyHostToDevice, st));
  RR_CUDA(cudaMemsetAsync(gcnt, 0, sizeof(int32_t) * kLfBlock * cap, st));
  RR_CUDA(cudaMemsetAsync(gpair, 0, sizeof(int32_t) * kLfBlock * kLfBlock, st));
  const size_t smem = sizeof(int32_t) * (size_t)cap;
  RR_CUDA(cudaFuncSetAttribute(k_lf_count, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)std::max<size_t>(smem, 1)));
  RR_CUDA(cudaMemsetAsync(lb.rl_cnt, 0, sizeof(int32_t) * N, st));
  RR_CUDA(cudaMemsetAsync(lb.rowmask, 0, sizeof(unsigned long long) * N, st));
  RR_LAUNCH(k_lf_init, 1, 1, 0, st, lb.S);
  for (int64_t s = 0; s < n_steps; ++s) {
    const int64_t f0 = s * kLfBlock;
    const int nb = (int)std::min<int64_t>(kLfBlock, F - f0);
    const unsigned nt = (unsigned)(step_ptr[s + 1] - step_ptr[s]);
    const LfTask *ts = d_tasks + step_ptr[s];
    if (nt) {
      RR_LAUNCH_PDL(k_lf_mark, nt, kThreads, 0, st, ts, row_idx, lb.rowmask);
      RR_LAUNCH_PDL(k_lf_count, nt, kThreads, smem, st, ts, row_idx, row_ptr,
                    (const int32_t *)lb.rl, (const int32_t *)lb.rl_cnt,
                    (const unsigned long long *)lb.rowmask, (const LfState *)lb.S, cap, gcnt,
                    gpair);
    }
    RR_LAUNCH_PDL(k_lf_best, nb, kThreads, 0, st, F, f0, col_ptr, (const int32_t *)lb.nlead,
                  (const LfState *)lb.S, cap, gcnt, lb.best);
    RR_LAUNCH_PDL(k_lf_resolve, 1, 32, 0, st, F, f0, col_ptr, tol2, cap,
                  (const unsigned long long *)lb.best, (const int32_t *)gpair, centers,
                  lb.nlead, labels, lb.S);
    if (nt)
      RR_LAUNCH_PDL(k_lf_commit, nt, kThreads, 0, st, ts, row_idx, row_ptr, lb.rl, lb.rl_cnt,
                    lb.rowmask, (const LfState *)lb.S, gpair, err);
  }
  LfState Sh{};
  RR_CUDA(cudaMemcpyAsync(&Sh, lb.S, sizeof(LfState), cudaMemcpyDeviceToHost, st));
  RR_CUDA(cudaStreamSynchronize(st));
  if (Sh.overflow) {
    rr_set_error("leader-follower: more than k = %d leaders at tol2 = %g (raise the tolerance "
                 "or k)", cap, tol2);
    return RR_UNSUPPORTED;
  }
  *n_lead_out = Sh.L;
  return RR_OK;
}

}  // namespace rr
