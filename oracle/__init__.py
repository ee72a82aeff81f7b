"""FP64 CPU oracle for two-level preconditioned CG on (X^T X + lambda I) w = X^T y.

TEST INFRASTRUCTURE ONLY. Only tests/, __graft_entry__.smoke() and bench.py's
CPU-baseline leg and reference arm may import this package; the library under
paper_1806_05826_gb300/ never does, and the two share no code.

Follows Tavernier, Simm, Meerbergen & Moreau, "Two-level preconditioning for
Ridge Regression" (arXiv 1806.05826):

  problem     Eq. (1): (X^T X + beta I) w = X^T b; beta is called lambda here.
  P           Eq. (prolong), Section 3.2: P(i, S) = 1/sqrt(n_S) for i in S.
  coarse      Section 3.2: Galerkin P^T (X^T X + beta I) P = X_c^T X_c + beta I.
  cycle       Section 3.1: T = (I - w A)(I - P A_c^{-1} P^T A)(I - w A),
              with the Richardson smoother generalised to damped Jacobi.
  clustering  Section 3.4: k-means++ on the features, Euclidean distance; or
              leader-follower clustering (Algorithm 1, leader.py).
  coarse solve Section 4: Cholesky factorisation of the coarse operator; or the
              eigendecomposition of X_c^T X_c, reused for every lambda
              (eigen.py, cyclic Jacobi).
  Krylov      CG, Jacobi-preconditioned CG (DCG), PCG, and flexible CG
              (Algorithm 3) with truncation m_i = max(1, i mod (m+1)).
  residual    Section 4 figures: ||X^T b - (X^T X + beta I) x|| / ||X^T b||.
  learned     (no counterpart in the paper) the training pairs of the learned
              coarse correction, (P^T r1, P^T (e - z1)) along two-level PCG
              (learned.py), and the FP64 network with its gradients (mlp.py).

Parity unpinned: iteration counts and speed-ups against the paper's tables
(its datasets are not available), and k-means labels beyond "same initial
centres give the same labels" (Lloyd's optimum is not unique).
"""
from . import sparse, kmeans, twolevel, krylov, mlp, learned, eigen, bayes, leader  # noqa: F401
