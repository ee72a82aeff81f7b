// The operator epilogues (CscEpilogue modes) applied where t_i = (X^T u)_i is
// complete, shared by the sliced (binary) and dense forms of the operator.
#pragma once

#include "common.cuh"
#include "kernels.h"

namespace rr {

// t = sum + lambda v_i, then the mode's update of out[i]; the mode's dot
// contribution is added to `dot`. With wd (omega / d_i, precomputed), POST
// multiplies by it instead of dividing by d_i (one FP64 multiply instead of a
// division; the FP32 inner iterations use this form).
__device__ __forceinline__ void epilogue(const CscEpilogue &ep, int64_t i, double sum, double &dot,
                                         const double *__restrict__ wd) {
  if (ep.mode == CSC_POST && wd) {
    const double r2 = ep.r[i] - (sum + ep.lambda * ep.v[i]);
    const double z = ep.v[i] + r2 * wd[i];
    ep.out[i] = z;
    dot += ep.r[i] * z;
    return;
  }
  switch (ep.mode) {
    case CSC_RHS:
      ep.out[i] = sum;
      break;
    case CSC_APPLY:
      ep.out[i] = sum + ep.lambda * ep.v[i];
      break;
    case CSC_PRE:
      ep.out[i] = ep.r[i] - (sum + ep.lambda * ep.v[i]);
      break;
    case CSC_POST: {
      const double r2 = ep.r[i] - (sum + ep.lambda * ep.v[i]);
      const double z = ep.v[i] + ep.omega * r2 / ep.d[i];
      ep.out[i] = z;
      dot += ep.r[i] * z;
      break;
    }
    case CSC_PCG: {
      const double t = sum + ep.lambda * ep.v[i];
      ep.out[i] = t;
      dot += ep.v[i] * t;
      break;
    }
    default: {  // CSC_RESID
      const double t = ep.r[i] - (sum + ep.lambda * ep.v[i]);
      ep.out[i] = t;
      dot += t * t;
      break;
    }
  }
}

__device__ __forceinline__ void epilogue(const CscEpilogue &ep, int64_t i, double sum, double &dot) {
  epilogue(ep, i, sum, dot, nullptr);
}

// The same epilogue on values loaded by the caller: vi = v[i], ri = r[i] and
// wdi = omega / d_i (POST), with the same operations in the same order.
__device__ __forceinline__ void epilogue_values(const CscEpilogue &ep, int64_t i, double sum,
                                                double vi, double ri, double wdi, double &dot) {
  switch (ep.mode) {
    case CSC_RHS:
      ep.out[i] = sum;
      break;
    case CSC_APPLY:
      ep.out[i] = sum + ep.lambda * vi;
      break;
    case CSC_PRE:
      ep.out[i] = ri - (sum + ep.lambda * vi);
      break;
    case CSC_POST: {
      const double r2 = ri - (sum + ep.lambda * vi);
      const double z = vi + r2 * wdi;
      ep.out[i] = z;
      dot += ri * z;
      break;
    }
    case CSC_PCG: {
      const double t = sum + ep.lambda * vi;
      ep.out[i] = t;
      dot += vi * t;
      break;
    }
    default: {  // CSC_RESID
      const double t = ri - (sum + ep.lambda * vi);
      ep.out[i] = t;
      dot += t * t;
      break;
    }
  }
}

}  // namespace rr
