// IGM transmission (Sec. 2.6): the Madau (1995) mean optical depth of the
// intergalactic medium at the observed wavelength lam_obs = lam_rest (1 + z),
// shared by the epilogues and their adjoints.
//   Lyman-series blanketing: A_j (lam_obs/lam_j)^3.46 for every line j with
//   lam_j < lam_obs < lam_j (1 + z), Ly-alpha to Ly-delta;
//   photoelectric absorption by Lyman-limit systems below lam_L (1 + z),
//   lam_L = 911.75 A: with x_c = lam_obs/lam_L (not below 1) and x_e = 1 + z,
//   0.25 x_c^3 (x_e^0.46 - x_c^0.46) + 9.4 x_c^1.5 (x_e^0.18 - x_c^0.18)
//   - 0.7 x_c^3 (x_c^-1.32 - x_e^-1.32) - 0.023 (x_e^1.68 - x_c^1.68).
// The transmission is exp(-f tau), f the row's igm_factor.  FP32, each power
// as exp2(p log2 x).
#pragma once
#include "sed_internal.cuh"

namespace sed {

constexpr float IGM_LYA = 1215.67f;

__device__ __forceinline__ float igm_pow(float x, float p) { return exp2f(p * __log2f(x)); }

// tau and d tau / dz at fixed rest wavelength lr (A) for 1 + z = opz; 0 redward of Ly-alpha
__device__ __forceinline__ void igm_madau(float lr, float opz, float& tau, float& dtau_dz) {
  tau = 0.f;
  dtau_dz = 0.f;
  if (lr >= IGM_LYA) return;
  const float lo = lr * opz;
  const float lj[4] = {1215.67f, 1025.72f, 972.537f, 949.743f};
  const float aj[4] = {3.6e-3f, 1.7e-3f, 1.1846e-3f, 9.316e-4f};
#pragma unroll
  for (int j = 0; j < 4; ++j)
    if (lr < lj[j] && lo > lj[j]) {
      const float t = aj[j] * igm_pow(lo / lj[j], 3.46f);
      tau += t;
      dtau_dz += 3.46f * t / opz;   // lam_obs = lr (1+z)
    }
  if (lr < 911.75f) {
    const float xe = opz, xr = lo * (1.f / 911.75f);
    const bool clamp = xr < 1.f;
    const float xc = clamp ? 1.f : xr;
    const float xc3 = xc * xc * xc, xc15 = xc * sqrtf(xc);
    const float e046 = igm_pow(xe, 0.46f), c046 = igm_pow(xc, 0.46f);
    const float e018 = igm_pow(xe, 0.18f), c018 = igm_pow(xc, 0.18f);
    const float em132 = igm_pow(xe, -1.32f), cm132 = igm_pow(xc, -1.32f);
    const float e168 = igm_pow(xe, 1.68f), c168 = igm_pow(xc, 1.68f);
    tau += 0.25f * xc3 * (e046 - c046) + 9.4f * xc15 * (e018 - c018) - 0.7f * xc3 * (cm132 - em132) -
           0.023f * (e168 - c168);
    // d/dx_e at fixed x_c, and d/dx_c (x_c = lr (1+z) / lam_L moves with z unless clamped)
    const float dxe = 0.25f * xc3 * 0.46f * e046 / xe + 9.4f * xc15 * 0.18f * e018 / xe -
                      0.7f * xc3 * 1.32f * em132 / xe - 0.023f * 1.68f * e168 / xe;
    float dxc = 0.f;
    if (!clamp)
      dxc = 0.75f * xc * xc * (e046 - c046) - 0.25f * xc3 * 0.46f * c046 / xc +
            14.1f * sqrtf(xc) * (e018 - c018) - 9.4f * xc15 * 0.18f * c018 / xc -
            2.1f * xc * xc * (cm132 - em132) + 0.7f * xc3 * 1.32f * cm132 / xc + 0.023f * 1.68f * c168 / xc;
    dtau_dz += dxe + dxc * (xr / opz);
  }
}

}  // namespace sed
