// Marginalised calibration polynomial (App. E, Eq. app_polymarg), shared by
// the forward epilogue and its adjoint.  The spectrum's model is
// mu_i (1 + sum_m c_m T_m(x_i)) with c ~ N(0, diag(s_m^2)); integrating c out,
//   lnL += b^T M^-1 b / 2 - ln|M| / 2 - ln|Lambda| / 2,
//   M_ab = sum_i w_i mu_i^2 T_a(x_i) T_b(x_i) + delta_ab / s_a^2,
//   b_a  = sum_i w_i mu_i r_i T_a(x_i),   w_i = 1/sigma_i^2,  r_i = d_i - mu_i,
// over the included pixels.  With T_a T_b = (T_{a+b} + T_{|a-b|}) / 2 the
// Gram matrix needs only the 2n-1 moments S_k = sum_i w_i mu_i^2 T_k(x_i).
#pragma once
#include "sed_internal.cuh"

namespace sed {

constexpr int CAL_NS = 2 * SED_MAX_CALIB - 1;   // moments S_k
constexpr int CAL_NV = CAL_NS + SED_MAX_CALIB;  // S_k then b_a

// One pixel's share of a block of NK consecutive sums: moments k = K0 .. K0+NK-1
// of coef * T_k(x), up to k < kmax (the moments S use coef = w mu^2 and
// kmax = 2n - 1, the vector b uses coef = w mu r and kmax = n).  The sums are
// taken in blocks of SED_MAX_CALIB to keep few of them live at a time.
template <int K0, int NK>
__device__ __forceinline__ void calib_accumulate(float x, float coef, int kmax, float (&v)[NK]) {
  float tp = 1.f, tc = x;   // T_{k-1}, T_k for k = 1
  if (K0 == 0) v[0] += coef;
#pragma unroll
  for (int k = 1; k < K0 + NK; ++k) {
    if (k >= K0 && k < kmax) v[k - K0] += coef * tc;
    const float tn = 2.f * x * tc - tp;
    tp = tc;
    tc = tn;
  }
}

// One block of calibration sums over the thread's own pixels (mu_s[i] != 0 for
// an included pixel): B = 0 gives the moments S_K0 .. S_K0+12 of w mu^2,
// B = 1 the vector b of w mu r; per-warp FP64 totals into part[warp][...].
template <int K0, int B, int NT>
__device__ __forceinline__ void calib_block(const ModelDev& md, const float* mu_s, int tid, int lane, int warp,
                                            double* part) {
  constexpr int NK = SED_MAX_CALIB;
  float v[NK];
#pragma unroll
  for (int q = 0; q < NK; ++q) v[q] = 0.f;
  const int kmax = B ? md.calib_n : 2 * md.calib_n - 1;
  for (int i = tid; i < md.n_pix; i += NT) {
    const float mu = mu_s[i];
    if (mu == 0.f) continue;
    // w mu^2 = (mu/sigma)^2 and w mu r = (mu/sigma)(r/sigma), formed from the
    // ratios (of the order of the S/N: cgs fluxes and 1/sigma^2 overflow FP32)
    const double is = md.spec_isig[i];
    const float mw = (float)((double)mu * is);
    const float coef = B ? mw * (float)((md.spec_d[i] - (double)mu) * is) : mw * mw;
    calib_accumulate<K0, NK>(md.pix_cx[i], coef, kmax, v);
  }
  const int base = B ? CAL_NS : K0;
#pragma unroll
  for (int q = 0; q < NK; ++q) {
    if (base + q >= (B ? CAL_NV : CAL_NS)) break;
    double x = (double)v[q];
#pragma unroll
    for (int o = 16; o; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if (lane == 0) part[warp * CAL_NV + base + q] = x;
  }
}

// Cholesky solve of the n x n system from the summed moments (one thread,
// FP64).  Writes the lower factor L (row-major n x n) and c* = M^-1 b; returns
// the lnL terms, or NaN when M is not positive definite.
__device__ inline double calib_solve(const ModelDev& md, const double* S, const double* B, double* L, double* c) {
  const int n = md.calib_n;
  double logdet = 0.0;
  for (int j = 0; j < n; ++j) {
    double d = 0.5 * (S[2 * j] + S[0]) + md.calib_isig2[j];
    for (int k = 0; k < j; ++k) d -= L[j * n + k] * L[j * n + k];
    if (!(d > 0.0)) return NAN;
    const double ljj = sqrt(d);
    L[j * n + j] = ljj;
    logdet += log(d);
    for (int i = j + 1; i < n; ++i) {
      double v = 0.5 * (S[i + j] + S[i - j]);
      for (int k = 0; k < j; ++k) v -= L[i * n + k] * L[j * n + k];
      L[i * n + j] = v / ljj;
    }
  }
  for (int i = 0; i < n; ++i) {
    double v = B[i];
    for (int k = 0; k < i; ++k) v -= L[i * n + k] * c[k];
    c[i] = v / L[i * n + i];
  }
  for (int i = n - 1; i >= 0; --i) {
    double v = c[i];
    for (int k = i + 1; k < n; ++k) v -= L[k * n + i] * c[k];
    c[i] = v / L[i * n + i];
  }
  double quad = 0.0;
  for (int a = 0; a < n; ++a) quad += B[a] * c[a];
  return 0.5 * quad - 0.5 * logdet - 0.5 * md.calib_logdet_lam;
}

}  // namespace sed
