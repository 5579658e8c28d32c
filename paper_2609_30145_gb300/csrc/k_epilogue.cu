// Fused epilogue: attenuation + nebular, observer-frame scaling, photometric
// and spectral projections and the Gaussian log-likelihood.  One CTA per
// parameter row; the attenuated rest-frame spectrum of the row is staged in
// shared memory once and every projection gathers from it.
//
//  F(lam) = e^{-tau_d(lam)} [ e^{-tau_BC(lam)} (Y(lam) + neb(lam)) + O(lam) ]
//     tau_BC = tau_pow (lam/5500)^alpha_pow (birth cloud, Sec. 2.4)
//     tau_d  = diffuse power law, or Kriek & Conroy 2013 (Sec. 2.4)
//     neb    = Q_young 10^(bilinear log10 template)        (App. C)
//  photometry (App. D, Eq. app_phot_T): m_b = P sum_j w_j lerp(F/lam^2)(lam_j/(1+z))
//  spectrum (App. E, Eq. app_response): m_i = s sum_j w_ij F_j / sum_j w_ij,
//     Gaussian in ln(lam) truncated at 5 sigma, linear interpolation for
//     kernels narrower than half a model log-pixel
//  lnL (Eq. total_lnlike): sum over included data of -r^2/2 - ln(2 pi sigma^2)/2
//     (r = (d - m)/sigma, min(r, 0) for a band that is an upper limit, Eq.
//     app_line_chi2_UL), with sigma_eff for sigma under the optional noise
//     floor (App. sys_floor) and the marginalised calibration polynomial's
//     terms (App. E); spectral residuals in FP32 on the host's d/sigma and
//     1/sigma, the bands' terms and every sum across threads in FP64
//  emission lines (App. C, App. line_proj): F_l = Q_young 10^(bilinear log10
//     cube) x the nebular attenuation at lam_l x s / (1+z); photometry
//     + F_l R_b(lam_obs) lam_obs / Z_b; spectrum + F_l (lam_i/c) N(ln lam_i;
//     ln lam_obs, s_l), s_l = sqrt(sigma_gas^2 + sigma_inst^2(lam_obs))/c
//     (Eq. app_line_profile); line catalogue: blends of F_l, one-sided upper
//     limits (Eq. app_line_chi2_det, Eq. app_line_chi2_UL)
//
// All reductions run in a fixed order, so the result is bitwise reproducible.
#include "sed_internal.cuh"
#include "locate.cuh"
#include "atten.cuh"
#include "calib.cuh"
#include "floor.cuh"
#include "igm.cuh"
#include "lines.cuh"

namespace sed {

// 128 threads per row and a small shared-memory window keep every row of a
// paper-scale batch resident at once (7 CTAs per SM, 1064 rows on 152 SMs):
// the kernel is bound by the latency of its gathers, so rows in flight is what
// sets its speed, and the 72 registers that 7 CTAs leave a thread (against 64
// at 8) keep more of each thread's loads in flight (measured 0.0988 against
// 0.1029 ms per 1024-row step).
constexpr int EPI_THREADS = 128;
constexpr int EPI_WARPS = EPI_THREADS / 32;
constexpr int MAX_BANDS = 128;

// dynamic shared memory: {lam, F/lam^2} and F over the row's window, the
// included pixels' mu/sigma for the calibration moments, and, with emission
// lines, per line ln(lam_obs) (an FP32 pair), F_l, A_l and 1/s_l
size_t epilogue_lines_off(const EpiArgs& a) {   // in floats, even (float2 alignment)
  const int np = a.row_model ? a.smem_pix : a.md.n_pix;
  const size_t W = (size_t)(a.row_model ? a.smem_win : a.md.win_max);
  const bool calib = a.row_model || a.md.calib_n > 0;
  const size_t f = 2 * W + (np > 0 ? W : 0) + (calib ? (size_t)np : 0);
  return (f + 1) & ~(size_t)1;
}
size_t epilogue_smem(const EpiArgs& a) {
  const bool lines = a.row_model ? a.g.n_line > 0 : a.md.use_lines != 0;
  return (epilogue_lines_off(a) + (lines ? (size_t)5 * a.g.n_line : 0)) * sizeof(float);
}

// MULTI: rows of several fits (serving), row r reads model mtab[row_model[r]];
// otherwise every row reads the model in the kernel parameters.  LINES: an
// instance with the emission lines (the one without keeps its code free of them).
// VAR: 1 the age-binned attenuation (one Y per attenuated block), 2 the
// nebular age axis (per-age ionising weights); 0 neither.
template <bool MULTI, bool LINES, int VAR = 0>
__global__ void __launch_bounds__(EPI_THREADS, 7) k_epilogue(const __grid_constant__ EpiArgs a) {
  pdl_enter();
  const int r = blockIdx.x;
  const ModelDev& md = MULTI ? a.mtab[a.row_model[a.rs[r].orig]] : a.md;
  const GridDev& g = a.g;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int N = g.n_lam;
  // shared memory holds the row's node window [k_lo, k_hi] only (at most
  // md.win_max nodes); the pointers below are offset so that they are indexed
  // by the global node k
  extern __shared__ float4 smem4[];
  const int WIN = MULTI ? a.smem_win : md.win_max;
  __shared__ float mb_s[MAX_BANDS];
  __shared__ double red[EPI_WARPS];
  __shared__ float cal_part[EPI_WARPS][CAL_NV];    // per-warp calibration sums
  __shared__ float cal_L[SED_MAX_CALIB * SED_MAX_CALIB], cal_D[SED_MAX_CALIB], cal_c[SED_MAX_CALIB];  // M = L L^T, 1/L_ii, c*
  __shared__ double cal_fix;                       // the row's lnL terms that do not sum over pixels

  if (a.win_reset && r == 0) empty_windows(a.win_reset, a.win_mt);
  RowScal rs = a.rs[r];
  if (a.err && *a.err) rs.status |= SED_ROW_DEVICE_TIMEOUT;
  const int ro = rs.orig;   // the caller's row index
  if (rs.status) {
    for (int b = tid; b < md.n_filt; b += blockDim.x)
      if (a.phot_out) a.phot_out[(size_t)ro * md.n_filt + b] = 0.f;
    for (int i = tid; i < md.n_pix; i += blockDim.x)
      if (a.spec_out) a.spec_out[(size_t)ro * md.n_pix + i] = 0.f;
    if (LINES && a.lines_out)
      for (int l = tid; l < g.n_line; l += blockDim.x) a.lines_out[(size_t)ro * g.n_line + l] = 0.f;
    if (tid == 0) {
      if (a.lnl) a.lnl[ro] = -INFINITY;
      if (a.status) a.status[ro] = rs.status;
    }
    return;
  }

  // ---- attenuated rest-frame spectrum of the row's node window into shared memory
  const float* Yr = a.Y + (size_t)r * a.ldn;
  const float* Or = a.O + (size_t)r * a.ldn;
  const float* O2r = a.O2 && a.split && *a.split ? a.O2 + (size_t)r * a.ldn : nullptr;
  const float eb = 0.85f - 1.9f * rs.delta;
  const float opz = 1.f / rs.inv1pz;
  // nebular age axis: the row's Q-weighted weight of each nebular SSP age
  __shared__ float qa_s[MAX_NEB_AGE];
  const float* qa = nullptr;
  if constexpr (VAR == 2) {
    for (int i = tid; i < g.neb_na; i += blockDim.x) qa_s[i] = a.qneb[(size_t)r * MAX_NEB_AGE + i];
    __syncthreads();
    qa = qa_s;
  }
  const bool spec = md.n_pix > 0;
  const int k_lo = rs.k_lo, k_hi = min(rs.k_hi, rs.k_lo + WIN - 1);   // nodes [k_lo, k_hi] are the only ones read below
  float2* LG = reinterpret_cast<float2*>(smem4) - k_lo;               // {rest-frame lambda, F / lam^2}
  float* Fs = reinterpret_cast<float*>(reinterpret_cast<float2*>(smem4) + WIN) - k_lo;   // F (spectral arm only)
  float* mu_s = reinterpret_cast<float*>(reinterpret_cast<float2*>(smem4) + WIN) + WIN;  // calibration: included pixels' mu/sigma (0 elsewhere)
  // not unrolled: measured faster than unrolling by 2, 4 or 8 (1024-row
  // photometric step 0.0892 against 0.0906, 0.0927 and 0.0947 ms)
#pragma unroll 1
  for (int k = k_lo + tid; k <= k_hi; k += EPI_THREADS) {
    const float4 c = g.att4[k];
    const float ys = a.lam8 ? rs.y_scale * a.lam8[k] : 1.f;
    const float o = O2r ? Or[k] + O2r[k] : Or[k];
    float F;
    if constexpr (VAR == 1) {
      float yv[MAX_SEG];
#pragma unroll
      for (int sg = 0; sg < MAX_SEG; ++sg) yv[sg] = sg < md.n_seg ? Yr[sg * a.seg_stride + k] * ys : 0.f;
      F = attenuated_bins(md, rs, c, eb, yv, o * ys, g.neb_tab, k);
    } else {
      F = attenuated(md, rs, c, eb, Yr[k] * ys, o * ys, g, qa, k);
    }
    if (md.use_igm && c.w < IGM_LYA) {   // the IGM transmission at the node's observed wavelength
      float tau, dtau;
      igm_madau(c.w, opz, tau, dtau);
      F *= __expf(-rs.igm_f * tau);
    }
    if (spec) Fs[k] = F;
    LG[k] = make_float2(c.w, __fdividef(F, c.w * c.w));
  }
  // emission lines: ln(lam_obs) pairs, fluxes F_l, profile peaks A_l = F_l /
  // (sqrt(2 pi) s_l) and 1/s_l in the tail of the dynamic shared memory
  const int NLn = LINES && md.use_lines ? g.n_line : 0;
  float2* ln_x = reinterpret_cast<float2*>(reinterpret_cast<float*>(smem4) + a.lines_off);
  float* ln_F = reinterpret_cast<float*>(ln_x + NLn);
  float* ln_A = ln_F + NLn;
  float* ln_is = ln_A + NLn;
  for (int l = tid; l < NLn; l += EPI_THREADS) line_setup(md, g, rs, eb, l, ln_F, ln_A, ln_is, ln_x);
  __syncthreads();
  if (LINES && a.lines_out) {   // the lines' fluxes only (sed_line_fluxes)
    for (int l = tid; l < NLn; l += EPI_THREADS) a.lines_out[(size_t)ro * NLn + l] = ln_F[l];
    if (!a.lnl && !a.phot_out && !a.spec_out) return;
  }

  // ---- photometry, one band per warp.  Consecutive lanes take consecutive
  //      filter samples (coalesced loads, eight in flight per lane); each
  //      sample's bracket starts from the index table over ln(lambda) at the
  //      sample's rest-frame wavelength and is corrected by a walk within the
  //      row's window in shared memory (any start gives the same bracket, so a
  //      fast logarithm serves).  Lane-strided sums and a fixed shuffle tree
  //      keep the order of the band sum fixed.
  const float lam0 = g.lam_f[0], lamN = g.lam_f[N - 1];
  {
    const int kmin = k_lo, kmax = k_hi - 1;
    for (int b = warp; b < md.n_filt; b += EPI_WARPS) {
      const int j1 = md.band_start[b + 1];
      float acc = 0.f;
      for (int j0 = md.band_start[b] + lane; j0 < j1; j0 += 256) {
        float2 sp[8];   // {lambda_obs, weight}; past the band's end x = 0 < lam0
        int kg[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) sp[u] = j0 + 32 * u < j1 ? md.samp2[j0 + 32 * u] : make_float2(0.f, 0.f);
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          int q = (int)((__logf(fmaxf(sp[u].x * rs.inv1pz, lam0)) - g.lut_x0) * g.lut_inv_h);
          q = q < 0 ? 0 : (q >= g.lut_n ? g.lut_n - 1 : q);
          kg[u] = g.lut[q];
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const float x = sp[u].x * rs.inv1pz;
          if (x >= lam0 && x <= lamN) {
            int kc = min(max(kg[u], kmin), kmax);
#pragma unroll 1
            while (kc < kmax && LG[kc + 1].x <= x) ++kc;
#pragma unroll 1
            while (kc > kmin && LG[kc].x > x) --kc;
            const float2 p0 = LG[kc], p1 = LG[kc + 1];
            const float t = __fdividef(x - p0.x, p1.x - p0.x);
            acc = fmaf(sp[u].y, p0.y + t * (p1.y - p0.y), acc);
          }
        }
      }
#pragma unroll
      for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
      // the lines in this band, one line per lane
      float lsum = 0.f;
      if (LINES && NLn) {
        for (int l = lane; l < NLn; l += 32) lsum += line_in_band(md, g, rs, b, l, ln_F[l]);
#pragma unroll
        for (int o = 16; o; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
      }
      if (lane == 0) {
        const float mb = LINES && NLn ? fmaf(rs.p_phot, acc, lsum) : rs.p_phot * acc;
        if (a.phot_out) a.phot_out[(size_t)ro * md.n_filt + b] = mb;
        mb_s[b] = mb;
      }
    }
  }

  // ---- spectrum: one thread per pixel
  // per-pixel terms in FP32 on the normalised residual (d - mu)/sigma; the
  // constants -1/2 ln(2 pi sigma^2) in FP64
  double part = 0.0;
  float chi = 0.f;
  const float ll0 = g.lnl_hi[0], llN = g.lnl_hi[N - 1];
  for (int i = tid; i < md.n_pix; i += blockDim.x) {
    float xh, xl;
    ln_rest(md.pix_ln2[i], rs.ln1pz_hi, rs.ln1pz_lo, xh, xl);
    float v = 0.f;
    bool valid = false;
    if (xh >= ll0 && xh <= llN) {
      // total dispersion: fixed, or sigma_fix composed with the row's sigma_gal (Eq. one_kernel)
      const float s = md.sample_sgal ? sqrtf(md.pix_fix2[i] + rs.sg_ln * rs.sg_ln) : md.pix_s[i];
      const int k = locate_ln(g, xh, g.lnl_hi);
      const float dln = (g.lnl_hi[k + 1] - g.lnl_hi[k]) + (g.lnl_lo[k + 1] - g.lnl_lo[k]);
      if (s < 0.5f * dln) {
        const float t = ((xh - g.lnl_hi[k]) + (xl - g.lnl_lo[k])) / dln;
        v = Fs[k] + t * (Fs[k + 1] - Fs[k]);
        valid = true;
      } else {
        // the nodes within 5 dispersions: a superset of them from the index
        // table alone (each entry within one node of the exact bracket; the
        // margins cover that), clamped to the row's window, which holds every
        // node within 5 dispersions of a pixel; a node past 5 dispersions
        // weighs exactly 0, so the sums are those over the nodes inside, in
        // the same order, and the loop carries no branch (its loads pipeline)
        const float inv_s = 1.f / s;
        int qa = (int)((fmaxf(xh - 5.f * s, ll0) - g.lut_x0) * g.lut_inv_h);
        int qb = (int)((fminf(xh + 5.f * s, llN) - g.lut_x0) * g.lut_inv_h);
        qa = min(max(qa, 0), g.lut_n - 1);
        qb = min(max(qb, 0), g.lut_n - 1);
        const int jlo = max(g.lut[qa] - 1, k_lo), jhi = min(g.lut[qb] + 3, k_hi);
        float sw = 0.f, sf = 0.f;
#pragma unroll 4
        for (int j = jlo; j <= jhi; ++j) {
          const float d = (g.lnl_hi[j] - xh) + (g.lnl_lo[j] - xl);
          const float u = d * inv_s;
          const float w = fabsf(u) <= 5.f ? __expf(-0.5f * u * u) : 0.f;
          sw += w;
          sf = fmaf(w, Fs[j], sf);
        }
        if (sw > 0.f) { v = sf / sw; valid = true; }
      }
    }
    const float mi = LINES && NLn ? fmaf(rs.s_spec, v, lines_at_pixel(md, i, NLn, ln_A, ln_is, ln_x)) : rs.s_spec * v;
    if (a.spec_out) a.spec_out[(size_t)ro * md.n_pix + i] = mi;
    const float isf = md.spec_isf[i];
    const bool inc = valid && isf != 0.f;
    const float ms = inc ? mi * isf : 0.f;   // mu / sigma
    if (inc) {
      const float dn = md.spec_dn[i], rn = dn - ms;   // (d - mu) / sigma
      if (md.floor_bits[1]) {                         // sigma_eff of Eq. app_noise_floor
        const float q = floor_q(rs.fl[1], ms, dn, rs.fl[1][3] * isf);
        chi -= 0.5f * (rn * rn / q + logf(q));
      } else {
        chi = fmaf(-0.5f * rn, rn, chi);
      }
      part += md.spec_nlog[i];
    }
    if (md.calib_n) mu_s[i] = ms;
  }
  part += (double)chi;
  // calibration moments over this thread's own pixels (no barrier needed),
  // in three blocks of sums (S_0..12, S_13..24, b_0..12), each summed per warp
  if (md.calib_n) {
    calib_block<0, 0, EPI_THREADS>(md, mu_s, cal_c, tid, lane, warp, &cal_part[0][0]);
    calib_block<SED_MAX_CALIB, 0, EPI_THREADS>(md, mu_s, cal_c, tid, lane, warp, &cal_part[0][0]);
    calib_block<0, 1, EPI_THREADS>(md, mu_s, cal_c, tid, lane, warp, &cal_part[0][0]);
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
  if (lane == 0) red[warp] = part;
  __syncthreads();
  if (md.calib_n) {
    // sum the warps' moments in warp order into row 0, factor M and solve for
    // c*; refine c* once from the pixels' calibrated residuals; then each
    // included pixel's change of its term under the polynomial p = A c*
    if (warp == 0) {
      const double f = calib_first_solve(md, &cal_part[0][0], EPI_WARPS, cal_L, cal_D, cal_c, lane);
      if (lane == 0) cal_fix = f;
    }
    __syncthreads();
    calib_block<0, 2, EPI_THREADS>(md, mu_s, cal_c, tid, lane, warp, &cal_part[0][0]);
    __syncthreads();
    if (warp == 0) {
      const double f = calib_refine(md, &cal_part[0][0], EPI_WARPS, cal_L, cal_D, cal_c, lane);
      if (lane == 0) cal_fix += f;
    }
    __syncthreads();
    float cpf = 0.f;
    for (int i = tid; i < md.n_pix; i += EPI_THREADS) {
      const float ms = mu_s[i];
      if (ms == 0.f) continue;
      cpf += calib_pixel_term(md.spec_dn[i] - ms, ms, calib_poly(cal_c, md.calib_n, md.pix_cx[i]));
    }
    double cp = (double)cpf;
#pragma unroll
    for (int o = 16; o; o >>= 1) cp += __shfl_xor_sync(0xffffffffu, cp, o);
    if (lane == 0) red[warp] += cp;
    __syncthreads();
  }
  // photometric terms in FP64, one band per lane of warp 0 (GB300's FP64 pipe
  // is narrow: one warp instruction serves all bands)
  if (warp == 0) {
    double pv = 0.0;
    for (int b = lane; b < md.n_filt; b += 32) {
      if (md.phot_isig[b] != 0.0) {
        const double is = md.phot_isig[b], mn = (double)mb_s[b] * is, dn = md.phot_d[b] * is;
        const double rr = phot_resid(md, b, dn, mn);
        if (md.floor_bits[0]) {   // sigma_eff of Eq. app_noise_floor
          const double q = floor_q(rs.fl[0], mn, dn, (double)rs.fl[0][3] * is);
          pv += -0.5 * (rr * rr / q + log(q)) + md.phot_nlog[b];
        } else {
          pv += -0.5 * rr * rr + md.phot_nlog[b];
        }
      }
    }
    // the line catalogue (Sec. 3.3), one entry per lane in FP64
    if (LINES)
      for (int k = lane; k < md.n_lcat; k += 32) pv += lcat_term(md, k, ln_F);
#pragma unroll
    for (int o = 16; o; o >>= 1) pv += __shfl_xor_sync(0xffffffffu, pv, o);
    if (lane == 0) {
      double tot = pv;
      for (int w = 0; w < EPI_WARPS; ++w) tot += red[w];
      if (md.calib_n) tot += cal_fix;
      uint32_t st = 0;
      if (!isfinite(tot)) { st = SED_ROW_NONFINITE; tot = -INFINITY; }
      if (a.lnl) a.lnl[ro] = tot;
      if (a.status) a.status[ro] = st;
    }
  }
}

cudaError_t launch_epilogue(const EpiArgs& a_in, cudaStream_t s) {
  EpiArgs a = a_in;
  a.lines_off = (int)epilogue_lines_off(a);
  const size_t smem = epilogue_smem(a);
  static DynSmemCache set_for[6];
  const bool lines = a.row_model ? a.g.n_line > 0 : a.md.use_lines != 0;
  // age-binned dust and the nebular age axis: neither served nor with lines
  const bool bins = !a.row_model && a.md.n_bin > 0, axis = !a.row_model && a.qneb;
  const int m = bins ? 4 : axis ? 5 : (a.row_model ? 1 : 0) + (lines ? 2 : 0);
  auto k = m == 0 ? k_epilogue<false, false>
         : m == 1 ? k_epilogue<true, false>
         : m == 2 ? k_epilogue<false, true>
         : m == 3 ? k_epilogue<true, true>
         : m == 4 ? k_epilogue<false, false, 1> : k_epilogue<false, false, 2>;
  cudaError_t e = ensure_dyn_smem(k, smem, &set_for[m]);
  if (e != cudaSuccess) return e;
  return launch_pdl(k, dim3(a.n), dim3(EPI_THREADS), smem, s, a);
}

}  // namespace sed
