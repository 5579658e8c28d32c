// Emission lines of the nebular grid (App. C, App. line_proj, Eq.
// app_line_profile) and the line-catalogue arm (Sec. 3.3, App. line_lik),
// shared by the forward epilogue and its adjoint so that both evaluate the
// same FP32 arithmetic.
#pragma once
#include "atten.cuh"
#include "igm.cuh"
#include "sed_internal.cuh"

namespace sed {

// Instrumental dispersion (km/s) at a line's observed wavelength lam_obs
// (ln lam_obs = xh): the pixels' LSF interpolated linearly in wavelength
// (the pixel bracket by bisection on ln(lambda)), constant past the ends;
// dsi = its slope in lam_obs (0 past the ends).
__device__ __forceinline__ void line_sigma_inst(const ModelDev& md, float xh, float lam_obs, float& si, float& dsi) {
  int lo = 0, hi = md.n_pix - 1;
  dsi = 0.f;
  if (xh <= md.pix_ln2[0].x) { si = md.pix_sinst[0]; return; }
  if (xh >= md.pix_ln2[hi].x) { si = md.pix_sinst[hi]; return; }
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (md.pix_ln2[mid].x <= xh) lo = mid; else hi = mid;
  }
  const float l0 = md.pix_lamc[lo] * (float)C_AA, l1 = md.pix_lamc[hi] * (float)C_AA;
  const float w = (lam_obs - l0) / (l1 - l0);
  dsi = (md.pix_sinst[hi] - md.pix_sinst[lo]) / (l1 - l0);
  si = md.pix_sinst[lo] + fminf(fmaxf(w, 0.f), 1.f) * (md.pix_sinst[hi] - md.pix_sinst[lo]);
}

// ---- emission lines (App. C, App. line_proj, Eq. app_line_profile)
// Line l of the row: its flux F_l (erg/s/cm^2), the spectral profile's peak
// factor A_l = F_l / (sqrt(2 pi) s_l), 1/s_l, and ln(lam_obs) as an FP32 pair.
// L_l = Q_young 10^(bilinear log10 cube) in device units (the cube carries the
// device-unit offset of the continuum template), times the attenuation the
// nebular continuum meets at lam_l (atten.cuh's factor of neb), times
// s_spec / (1+z): the flux factor without its (1+z).  s_l takes sigma_inst
// at lam_obs by linear interpolation in wavelength between the pixels (their
// value past the ends).
__device__ __forceinline__ void line_setup(const ModelDev& md, const GridDev& g, const RowScal& rs, float eb, int l,
                                           float* F_s, float* A_s, float* is_s, float2* x_s) {
  const int nl = g.n_lam, NLn = g.n_line;
  float lg = 0.f;
#pragma unroll
  for (int c = 0; c < 4; ++c) lg = fmaf(rs.neb_w[c], g.line_tab[(rs.neb_off[c] / nl) * NLn + l], lg);
  const float L = ex2_approx(rs.log2_qy + 3.3219280948873623f * lg);
  const float4 c = g.line_att4[l];
  const float tbc = rs.tau_bc * __expf(rs.alpha_bc * c.x);
  const float td = rs.tau_d * dust_shape(md, c, eb, __expf(rs.delta * c.x));
  const float ed = __expf(-td), ebc = __expf(-tbc), f = rs.fob;
  const float fac = md.fesc_geom == SED_FESC_PICKET ? ed * (1.f - f) * ebc : ed * ((1.f - f) * ebc + f) * (1.f - f);
  float F = L * fac * rs.s_spec * rs.inv1pz;
  if (md.use_igm && c.w < IGM_LYA) {   // the IGM transmission at the line's observed wavelength
    float tau, dtau;
    igm_madau(c.w, 1.f / rs.inv1pz, tau, dtau);
    F *= __expf(-rs.igm_f * tau);
  }
  F_s[l] = F;
  // observed ln(lambda) = ln(lam_l) + ln(1+z): the FP32 pairs summed by two-sum
  const float2 lr = g.line_ln2[l];
  const float sh = lr.x + rs.ln1pz_hi, bv = sh - lr.x;
  const float e = (lr.x - (sh - bv)) + (rs.ln1pz_hi - bv);
  const float t = e + (lr.y + rs.ln1pz_lo);
  const float xh = sh + t, xl = t - (xh - sh);
  x_s[l] = make_float2(xh, xl);
  float inv_s = 0.f, A = 0.f;
  if (md.n_pix > 0) {
    float si, dsi;
    line_sigma_inst(md, xh, c.w / rs.inv1pz, si, dsi);
    const float s = sqrtf(rs.sgas * rs.sgas + si * si) * (float)(1.0 / C_KMS);
    if (s > 0.f) {
      inv_s = 1.f / s;
      A = F * inv_s * 0.3989422804014327f;
    }
  }
  A_s[l] = A;
  is_s[l] = inv_s;
}

// Sum of the line profiles at pixel i (cgs F_nu), lines in index order, each
// truncated at 5 s_l (Eq. app_line_profile, not renormalised).
__device__ __forceinline__ float lines_at_pixel(const ModelDev& md, int i, int NLn, const float* A_s, const float* is_s,
                                                const float2* x_s) {
  const float2 p = md.pix_ln2[i];
  float acc = 0.f;
  for (int l = 0; l < NLn; ++l) {
    const float u = ((p.x - x_s[l].x) + (p.y - x_s[l].y)) * is_s[l];
    if (fabsf(u) <= 5.f) acc = fmaf(A_s[l], __expf(-0.5f * u * u), acc);
  }
  return acc * md.pix_lamc[i];
}

// Band b's response to a line at observed wavelength x: rz = R_b(x) / Z_b, R_b
// linear between the band's samples (0 outside them), and its slope drz in x.
// The bracket (the last sample at or below x; the last interval at the band's
// end) is found from the position of x between the band's ends and a walk to
// it: one or two loads for evenly spaced samples instead of a bisection's chain
// of dependent loads, and the same bracket for any spacing.
__device__ __forceinline__ void line_band_resp(const ModelDev& md, int b, float x, float& rz, float& drz) {
  const int b0 = md.band_start[b], b1 = md.band_start[b + 1] - 1;
  rz = 0.f;
  drz = 0.f;
  const float xa = md.samp2[b0].x, xb = md.samp2[b1].x;
  if (!(x >= xa && x <= xb)) return;
  int j = b1 > b0 ? b0 + (int)((x - xa) / (xb - xa) * (float)(b1 - b0)) : b0;
  j = min(max(j, b0), max(b1 - 1, b0));
  while (j > b0 && md.samp2[j].x > x) --j;
  while (j + 1 < b1 && md.samp2[j + 1].x <= x) ++j;
  const int lo = j, hi = b1 > b0 ? j + 1 : b0;
  const float x0 = md.samp2[lo].x, x1 = md.samp2[hi].x;
  if (!(x1 > x0)) { rz = md.samp_rz[lo]; return; }
  const float t = (x - x0) / (x1 - x0);
  drz = (md.samp_rz[hi] - md.samp_rz[lo]) / (x1 - x0);
  rz = md.samp_rz[lo] + t * (md.samp_rz[hi] - md.samp_rz[lo]);
}

// Band b's photometry of line l (maggies): F R_b(lam_obs) lam_obs / Z_b.
__device__ __forceinline__ float line_in_band(const ModelDev& md, const GridDev& g, const RowScal& rs, int b, int l,
                                             float F) {
  const float x = g.line_att4[l].w / rs.inv1pz;   // observed wavelength, Angstrom
  float rz, drz;
  line_band_resp(md, b, x, rz, drz);
  return F * rz * x;
}

// Line-catalogue entry k's lnL term (FP64): model = the blend's summed line
// fluxes; the one-sided residual of an upper limit (Eq. app_line_chi2_UL);
// 0 for an entry outside the mask.
__device__ __forceinline__ double lcat_term(const ModelDev& md, int k, const float* F_s) {
  const double is = md.lcat_isig[k];
  if (is == 0.0) return 0.0;
  float m = 0.f;
  for (int j = md.lcat_start[k]; j < md.lcat_start[k + 1]; ++j) m += F_s[md.lcat_line[j]];
  const double d = md.lcat_d[k];
  double r = (d - (double)m) * is;
  if (md.lcat_ul && md.lcat_ul[k] && (double)m <= d) r = 0.0;
  return -0.5 * r * r + md.lcat_nlog[k];
}


}  // namespace sed
