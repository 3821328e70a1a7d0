// The eigenvalue p of the preconditioner in the transformed basis (Sec. 3.1.1 for theta, Sec. 4
// for BDF2, Sec. 3.1.4 for P_theta) as 1/p, for the compute types of the preconditioner kernels
// (float64, float32 and double-float); shared by the CUDA-core and tensor-core time kernels.
#pragma once

#include <math.h>

#include "st_dd.cuh"
#include "st_internal.cuh"

namespace st {

__device__ __forceinline__ double rsq(double x) { return rsqrt(x); }
__device__ __forceinline__ float rsq(float x) { return rsqrtf(x); }
__device__ __forceinline__ dd rsq(dd x) { return rsqrt_dd(x); }

// 1/p for the eigenvalue of the preconditioner at time frequency k (1-based) and tau*mu.
template <class T>
__device__ __forceinline__ T inv_symbol(const Spec<T> &sp, int k, T tmu) {
  const T hk = sp.hk[k - 1], ck = sp.ck[k - 1], sk = sp.sk[k - 1];
  if (sp.prec == ST_PREC_PTHETA) {
    // lam_H = sqrt(2 - 2cos x) = 2 sin(x/2), lam_Htheta = sqrt(th^2 + (1-th)^2 + 2 th(1-th) cos x)
    return T(1) / (sp.lh[k - 1] + sp.lht[k - 1] * tmu);
  }
  T re, im;
  if (sp.scheme == ST_THETA) {
    // |a0 + a1 e^{ix}|, a0 = 1 + th tmu, a1 = -1 + (1-th) tmu;  a0 + a1 cos x = (1 - cos x) +
    // tmu (th + (1-th) cos x)
    re = hk + tmu * (sp.theta + (T(1) - sp.theta) * ck);
    im = (T(-1) + (T(1) - sp.theta) * tmu) * sk;
  } else {
    // |a0 + a1 e^{ix} + a2 e^{2ix}|, a0 = 3/2 + tmu, a1 = -2, a2 = 1/2:
    // re = (1 - cos x)^2 + tmu, im = -sin x (2 - cos x)
    re = hk * hk + tmu;
    im = -sk * (T(1) + hk);
  }
  return rsq(re * re + im * im);
}

}  // namespace st
