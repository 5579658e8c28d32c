// Node lookup on the model's rest-frame wavelength axis, shared by the forward
// epilogue and its adjoint so that both take the same interpolation brackets.
#pragma once
#include "sed_internal.cuh"

namespace sed {

// last node k with lam[k] <= x (lam ascending), for lam[0] <= x <= lam[n-1];
// clamped to n-2 so that k+1 is a valid node.
__device__ __forceinline__ int locate_ln(const GridDev& g, float lnx, const float* lnl_hi) {
  int q = (int)((lnx - g.lut_x0) * g.lut_inv_h);
  q = q < 0 ? 0 : (q >= g.lut_n ? g.lut_n - 1 : q);
  int k = g.lut[q];
  const int top = g.n_lam - 2;
  k = k > top ? top : k;
#pragma unroll 1
  for (int it = 0; it < 4 && k < top && lnl_hi[k + 1] <= lnx; ++it) ++k;
#pragma unroll 1
  for (int it = 0; it < 4 && k > 0 && lnl_hi[k] > lnx; ++it) --k;
  return k;
}

__device__ __forceinline__ int locate_lin(const GridDev& g, float x) {
  int k = locate_ln(g, logf(x), g.lnl_hi);
  const int top = g.n_lam - 2;
#pragma unroll 1
  for (int it = 0; it < 4 && k < top && g.lam_f[k + 1] <= x; ++it) ++k;
#pragma unroll 1
  for (int it = 0; it < 4 && k > 0 && g.lam_f[k] > x; ++it) --k;
  return k;
}

}  // namespace sed
