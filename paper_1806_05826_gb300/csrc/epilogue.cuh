// The operator epilogues (CscEpilogue modes) applied where t_i = (X^T u)_i is
// complete, shared by the sliced (binary) and dense forms of the operator.
#pragma once

#include "common.cuh"
#include "kernels.h"

namespace rr {

// t = sum + lambda v_i, then the mode's update of out[i]; the mode's dot
// contribution is added to `dot`.
__device__ __forceinline__ void epilogue(const CscEpilogue &ep, int64_t i, double sum, double &dot) {
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

}  // namespace rr
