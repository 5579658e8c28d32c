// Per-datum likelihood pieces shared by the forward epilogue and its adjoint:
// the one-sided residual of a photometric upper limit (phot_resid, below) and
// the systematic noise floor (App. sys_floor, Eq. app_noise_floor), under
// which each datum's variance becomes
//   sigma_eff^2 = s^2 sigma^2 + (f_calib |m|)^2 + (f_data |d|)^2 + j^2,
// fl = {s, f_calib, f_data, j} (s = 1 and the others 0 for a term that is off).
// The kernels work in units of the formal error: with mn = m/sigma,
// dn = d/sigma, rn = dn - mn and jn = j/sigma,
//   q = sigma_eff^2 / sigma^2 = s^2 + (f_calib mn)^2 + (f_data dn)^2 + jn^2,
//   term = -rn^2 / (2 q) - ln(q) / 2 - ln(2 pi sigma^2) / 2,
// the last part the per-datum constant the host prepares.  T is float for the
// spectral pixels and double for the bands' FP64 pass.
#pragma once
#include "sed_internal.cuh"

namespace sed {

template <typename T>
__device__ __forceinline__ T floor_q(const float (&fl)[4], T mn, T dn, T jn) {
  const T s = (T)fl[0], fc = (T)fl[1] * mn, fd = (T)fl[2] * dn;
  return s * s + fc * fc + fd * fd + jn * jn;
}

// d term / d q
template <typename T>
__device__ __forceinline__ T floor_gq(T rn, T q) {
  return (rn * rn / q - (T)1) / ((T)2 * q);
}

// d term / d mn: the residual's share and, through the model-anchored term,
// the variance's (dq/dmn = 2 f_calib^2 mn)
template <typename T>
__device__ __forceinline__ T floor_dm(const float (&fl)[4], T rn, T q, T gq, T mn) {
  return rn / q + gq * (T)2 * (T)fl[1] * (T)fl[1] * mn;
}

// adds d term / d log10 of each term to g: dq/dlog10 x = 2 ln(10) x^2 with x =
// s, f_calib mn, f_data dn, jn
template <typename T>
__device__ __forceinline__ void floor_dparam(const float (&fl)[4], T gq, T mn, T dn, T jn, T (&g)[4]) {
  const T c = gq * (T)4.605170185988091;   // 2 ln(10)
  const T fc = (T)fl[1] * mn, fd = (T)fl[2] * dn;
  g[0] += c * (T)fl[0] * (T)fl[0];
  g[1] += c * fc * fc;
  g[2] += c * fd * fd;
  g[3] += c * jn * jn;
}

// Residual (d - m)/sigma of photometric band b from dn = d/sigma and mn =
// m/sigma.  A band flagged as an upper limit (Sec. 4.1 likelihood, Eq.
// app_line_chi2_UL) costs nothing while the model stays at or below the limit:
// its residual is then 0, which also zeroes its share of d lnL / d m (the
// derivative of -min(r, 0)^2 / 2 is min(r, 0)).
template <typename T>
__device__ __forceinline__ T phot_resid(const ModelDev& md, int b, T dn, T mn) {
  const T r = dn - mn;
  return (md.phot_ul != nullptr && md.phot_ul[b] && r > (T)0) ? (T)0 : r;
}

}  // namespace sed
