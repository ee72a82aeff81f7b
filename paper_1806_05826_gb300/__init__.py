"""GB300 (sm_103a) two-level preconditioned CG for (X^T X + lambda I) w = X^T y.

Tavernier, Simm, Meerbergen & Moreau, "Two-level preconditioning for Ridge
Regression" (arXiv 1806.05826). The solver lives in librr.so (CUDA); `rr` is
its Python binding.
"""
from . import rr  # noqa: F401
