// Attenuated rest-frame spectrum of one node (Sec. 2.4, App. C, Eq. app_attn),
// shared by the forward epilogue and its adjoint so that both evaluate the
// same FP32 arithmetic:
//   F = e^{-tau_d} [ e^{-tau_BC} (Y + neb) + O ]
//   tau_BC = tau_pow (lam/5500)^alpha_pow
//   tau_d  = tau_diff (lam/5500)^delta                        (power law), or
//            tau_diff [k'(lam) + E_b(delta) D(lam)]/4.05 (lam/5500)^delta  (Kriek & Conroy 2013)
//   neb    = Q_young 10^(bilinear log10 template)
// With an escape geometry (Sec. frac_obrun) and runaway fraction f, the
// nebular ages' ionising continuum Y_ion (nodes below 912 A, kept in Y) is
// split off, Y_s = Y - Y_ion, and
//   runaway_bc (Eq. runaway_mix):
//     F = e^{-tau_d} [ T (Y_s + (1-f) neb) + f Y_ion + O ],  T = (1-f) e^{-tau_BC} + f
//   picket:
//     F = f Y + e^{-tau_d} [ (1-f) e^{-tau_BC} (Y_s + neb) + O ]
#pragma once
#include "sed_internal.cuh"

namespace sed {

// 2^x by the hardware's approximate base-2 exponential (relative error below 2^-22)
__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__device__ __forceinline__ float dust_shape(const ModelDev& md, const float4& c, float eb, float pw) {
  return md.dust_law == SED_DUST_POWER_LAW ? pw : (c.y + eb * c.z) * pw;
}

__device__ __forceinline__ float neb_log10(const RowScal& rs, const float* tab, int k) {
  return rs.neb_w[0] * tab[rs.neb_off[0] + k] + rs.neb_w[1] * tab[rs.neb_off[1] + k] +
         rs.neb_w[2] * tab[rs.neb_off[2] + k] + rs.neb_w[3] * tab[rs.neb_off[3] + k];
}

// Nebular emission at node k (device units): Q_young 10^template, or with a
// nebular age axis (App. C) the sum over the nebular SSP ages of q_a 10^(the
// cube at that age), qa the row's q_a (NULL without an axis).
__device__ __forceinline__ float neb_emission(const RowScal& rs, const GridDev& g, const float* qa, int k) {
  if (qa) {
    const size_t plane = (size_t)g.neb_nu * g.neb_nz * g.n_lam;
    float acc = 0.f;
    for (int i = 0; i < g.neb_na; ++i) {
      const float q = qa[i];
      if (q != 0.f) acc = fmaf(q, ex2_approx(3.3219280948873623f * neb_log10(rs, g.neb_tab + i * plane, k)), acc);
    }
    return acc;
  }
  return ex2_approx(rs.log2_qy + 3.3219280948873623f * neb_log10(rs, g.neb_tab, k));
}

// c = {ln(lam/5500), k'/4.05, Drude/4.05, 1/lam^2}; eb = 0.85 - 1.9 delta
__device__ __forceinline__ float attenuated(const ModelDev& md, const RowScal& rs, const float4& c, float eb, float y,
                                           float o, const GridDev& g, const float* qa, int k) {
  const float tbc = rs.tau_bc * __expf(rs.alpha_bc * c.x);
  const float pw = __expf(rs.delta * c.x);
  const float td = rs.tau_d * dust_shape(md, c, eb, pw);
  if (md.fesc_geom == SED_FESC_NONE) {
    if (md.use_neb) y += neb_emission(rs, g, qa, k);
    return __expf(-td) * (__expf(-tbc) * y + o);
  }
  const float nb = md.use_neb ? neb_emission(rs, g, qa, k) : 0.f;
  const bool lyc = md.use_neb && k < md.n_lyc;
  const float ys = lyc ? 0.f : y, f = rs.fob, ed = __expf(-td), ebc = __expf(-tbc);
  if (md.fesc_geom == SED_FESC_PICKET) return f * y + ed * ((1.f - f) * ebc * (ys + nb) + o);
  const float T = (1.f - f) * ebc + f;
  return ed * (T * (ys + (1.f - f) * nb) + (lyc ? f * y : 0.f) + o);
}

// Age-binned attenuation (App. dust_attn, Eq. app_tau_bin, Eq. app_attn):
// attenuated block s of the young part (its ages share one row of the
// age-to-bin matrix) sees tau_s = sum_b M_sb kappa_b with kappa_b = tau_b
// shape_b(lam) of bin b's law; the nebular emission of each block's ages
// (Q_s 10^template) is attenuated with its block, and the ages outside every
// bin see the diffuse screen only:
//   F = e^{-tau_d} [ sum_s e^{-tau_s} (Y_s + Q_s neb) + O + Q_rest neb ]
__device__ __forceinline__ float bin_shape(int law, const float4& c, float slope) {
  const float pw = __expf(slope * c.x);
  return law == SED_DUST_POWER_LAW ? pw : (c.y + (0.85f - 1.9f * slope) * c.z) * pw;
}

__device__ __forceinline__ float attenuated_bins(const ModelDev& md, const RowScal& rs, const float4& c, float eb,
                                                const float* y, float o, const float* neb_tab, int k) {
  float kap[MAX_DUST_BIN];
#pragma unroll
  for (int b = 0; b < MAX_DUST_BIN; ++b)
    kap[b] = b < md.n_bin ? rs.bin_tau[b] * bin_shape(md.bin_law[b], c, rs.bin_slope[b]) : 0.f;
  const float lg = md.use_neb ? 3.3219280948873623f * neb_log10(rs, neb_tab, k) : 0.f;
  float acc = o;
  if (md.use_neb) acc += ex2_approx(rs.log2_qs[MAX_SEG] + lg);
#pragma unroll
  for (int sg = 0; sg < MAX_SEG; ++sg) {
    if (sg >= md.n_seg) break;
    float tau = 0.f;
#pragma unroll
    for (int b = 0; b < MAX_DUST_BIN; ++b) tau = fmaf(md.seg_M[sg][b], kap[b], tau);
    const float v = md.use_neb ? y[sg] + ex2_approx(rs.log2_qs[sg] + lg) : y[sg];
    acc = fmaf(__expf(-tau), v, acc);
  }
  const float td = rs.tau_d * dust_shape(md, c, eb, __expf(rs.delta * c.x));
  return __expf(-td) * acc;
}

}  // namespace sed
