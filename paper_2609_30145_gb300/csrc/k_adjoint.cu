// Adjoint of the epilogue and of the contraction (the reverse pass of
// sed_loglike_grad).  The paper obtains its gradients by automatic
// differentiation of the forward model (Sec. 4); here each step is
// differentiated by hand, in reverse order:
//
//   lnL (Eq. total_lnlike)          u_b = dlnL/dm_b = (d_b - m_b)/sigma_b^2 (with
//                                   the noise floor's sigma_eff and its f_calib
//                                   dependence on m, App. sys_floor; with the
//                                   calibration polynomial, App. E)
//   photometry (App. D)             dlnL/dF_k from the interpolation weights of
//                                   every filter sample that touches node k
//   spectrum (Eq. app_response)     dlnL/dF_k from every pixel whose Gaussian
//                                   row reaches node k
//   dust + nebular (Sec. 2.4, App. C)
//                                   dlnL/dY, dlnL/dO and the sums over lambda
//                                   giving d/dtau_BC, d/dalpha_BC, d/dtau_d,
//                                   d/ddelta, d/dQ_young, d/dlogU, d/dlogZ_gas
//   observer frame (Sec. 2.6)       d/dlogmass and the part of d/dz that comes
//                                   from the flux scale and the redshift gather
//   emission lines (App. C, App. line_proj, Eq. app_line_profile), line catalogue
//                                   dlnL/dF_l, d/d ln(lam_obs), d/ds_l of each
//                                   line from the pixels, bands and catalogue
//                                   entries it enters, then through the line's
//                                   flux and width to the dust, nebular, mass,
//                                   redshift and gas-dispersion parameters
//   contraction (Eq. csp_sum_main)  dlnL/dW = [G_Y SSP_young^T | G_O SSP_old^T]
//                                   (k_dw_simt here, or the tcgen05 kernel)
//
// k_epi_bwd takes one CTA per parameter row, recomputes the row's attenuated
// spectrum from Y and O (the forward's contraction output) instead of storing
// it, and accumulates dlnL/dF in shared memory.  Every sum runs in a fixed
// order (node-owned gathers, no atomics), so the gradient is bitwise
// reproducible.
#include "atten.cuh"
#include "calib.cuh"
#include "floor.cuh"
#include "igm.cuh"
#include "lines.cuh"
#include "locate.cuh"
#include "sed_internal.cuh"

namespace sed {

constexpr int EB_THREADS = 256;
constexpr int EB_WARPS = EB_THREADS / 32;
constexpr int EB_MAX_BANDS = 128;
constexpr int EB_NRED = 19;   // per-warp partial sums: 17 FP32 sums, then lnL and d lnL/d ln(mass) in FP64
constexpr int EB_NREDF = 17;
constexpr int EB_NREDB = 2 * MAX_DUST_BIN + MAX_SEG + 1;   // age-binned dust: d/d(tau_b, slope_b), d/dQ of each block

__device__ __forceinline__ float tf32_rna_dev(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

__device__ __forceinline__ void put_g(const EpiBwdArgs& a, float* hi, float* lo, size_t o, float v) {
  if (a.split) {
    const float h = tf32_rna_dev(v);
    hi[o] = h;
    lo[o] = v - h;
  } else {
    hi[o] = v;
  }
}

// Shared memory of one row: F and dlnL/dF over the row's node window, then a
// union of the filter samples' brackets (photometry) and the pixels' node
// ranges and positions (spectrum).
// bytes of the calibration scratch: per-warp sums, the Cholesky factor, its
// inverse diagonal and c* as floats
constexpr size_t EB_CAL_BYTES = (size_t)EB_WARPS * CAL_NV * sizeof(float) +
                                (size_t)(SED_MAX_CALIB * SED_MAX_CALIB + 2 * SED_MAX_CALIB) * sizeof(float);

size_t epi_bwd_lines_off(const EpiBwdArgs& a) {   // bytes, 8-aligned
  const size_t W = (size_t)a.md.win_max;
  const size_t samp = (size_t)a.md.n_samp * 8;    // node index + interpolation weight
  // 4 floats + node range; with a calibration polynomial also mu/sigma, dmu/dx, dmu/ds, 1/sum w
  const size_t pix = (size_t)a.md.n_pix * (a.md.calib_n ? 36 : 20);
  const size_t u = ((samp > pix ? samp : pix) + 7) & ~(size_t)7;
  return ((((2 * W + 3) & ~(size_t)3) * sizeof(float) + u + (a.md.calib_n ? EB_CAL_BYTES : 0)) + 7) & ~(size_t)7;
}
// with emission lines: per line ln(lam_obs) (FP32 pair), F_l, A_l, 1/s_l; per
// pixel dlnL/dmu (the line part of mu/sigma until the calibration solve); per
// catalogue entry dlnL/dm
size_t epi_bwd_smem(const EpiBwdArgs& a) {
  const size_t lines = a.md.use_lines
                           ? (size_t)a.g.n_line * 20 + (size_t)a.md.n_pix * 4 + (size_t)a.md.n_lcat * 4 : 0;
  return epi_bwd_lines_off(a) + lines;
}

// LINES: an instance with the emission lines (the one without keeps its code free of them);
// VAR: 1 the age-binned attenuation (one Y and one dlnL/dY per attenuated
// block), 2 the nebular age axis (per-age ionising weights); 0 neither
template <bool LINES, int VAR = 0>
__global__ void __launch_bounds__(EB_THREADS, 4) k_epi_bwd(const __grid_constant__ EpiBwdArgs a) {
  pdl_enter();
  const ModelDev& md = a.md;
  const GridDev& g = a.g;
  const int r = blockIdx.x;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int N = g.n_lam;
  extern __shared__ __align__(16) float smem[];
  __shared__ float ubp[EB_MAX_BANDS], mbp[EB_MAX_BANDS];
  __shared__ int bk0[EB_MAX_BANDS], bk1[EB_MAX_BANDS];
  __shared__ float mlb[EB_MAX_BANDS], ubm[EB_MAX_BANDS];   // lines: each band's line part, dlnL/dm_b
  __shared__ double red[EB_WARPS][EB_NRED + EB_NREDB];

  if (a.win_reset && r == 0) empty_windows(a.win_reset, a.win_mt);
  const size_t ro = (size_t)r * a.ldn;
  RowScal rs = a.rs[r];
  if (a.err && *a.err) rs.status |= SED_ROW_DEVICE_TIMEOUT;
  if (rs.status) {
    for (int k = tid; k < a.ldn; k += EB_THREADS) {
      for (int sg = 0; sg < (VAR == 1 ? md.n_seg : 1); ++sg) {
        a.gy_hi[sg * a.seg_stride + ro + k] = 0.f;
        if (a.split) a.gy_lo[sg * a.seg_stride + ro + k] = 0.f;
      }
      a.go_hi[ro + k] = 0.f;
      if (a.split) a.go_lo[ro + k] = 0.f;
    }
    if (tid < RGRAD) a.rgrad[(size_t)r * RGRAD + tid] = 0.0;
    if (tid == 0) {
      if (a.lnl) a.lnl[rs.orig] = -INFINITY;
      if (a.status) a.status[rs.orig] = rs.status;
    }
    return;
  }
  // the row's node window: F is read and dlnL/dF is non-zero only there
  const int WIN = md.win_max;
  const int k_lo = rs.k_lo, k_hi = min(rs.k_hi, rs.k_lo + WIN - 1);
  float* Fs = smem - k_lo;                // attenuated rest-frame spectrum F
  float* phi = smem + WIN - k_lo;         // dlnL/dF
  void* U = smem + ((2 * WIN + 3) & ~3);  // union: filter samples, then spectrum pixels
  int* sk = reinterpret_cast<int*>(U);
  float* st = reinterpret_cast<float*>(sk + md.n_samp);
  // per pixel {x_hi, x_lo, c, t}: position ln(lambda_obs/(1+z)) in two floats, its
  // weight in dlnL/dF, and for a linear row its weight t (within rounding of
  // [0, 1]; a pixel on a node can give t = -1e-9) or for a Gaussian row
  // -1 - 1/sigma (below -1): the two never meet, whatever the rounding
  float4* px4 = reinterpret_cast<float4*>(U);
  int* prg = reinterpret_cast<int*>(px4 + md.n_pix);   // node range lo | hi << 16
  // calibration polynomial (App. E): per pixel mu/sigma (0 when excluded), dv/dx, dv/ds,
  // 1/sum w, then the per-warp moments, the Cholesky factor and c*
  float* mu_s = reinterpret_cast<float*>(prg + md.n_pix);
  float* dv_s = mu_s + md.n_pix;
  float* dvs_s = dv_s + md.n_pix;
  float* cw_s = dvs_s + md.n_pix;
  float *cal_part = nullptr, *cal_Lf = nullptr, *cal_Df = nullptr, *cal_cf = nullptr;
  if (md.calib_n) {
    const size_t samp = (size_t)md.n_samp * 8, pix = (size_t)md.n_pix * 36;
    const size_t u = ((samp > pix ? samp : pix) + 7) & ~(size_t)7;
    cal_part = reinterpret_cast<float*>(reinterpret_cast<char*>(U) + u);
    cal_Lf = reinterpret_cast<float*>(cal_part + EB_WARPS * CAL_NV);
    cal_Df = cal_Lf + SED_MAX_CALIB * SED_MAX_CALIB;   // after L
    cal_cf = cal_Df + SED_MAX_CALIB;
  }
  // emission lines: per line ln(lam_obs), F_l, A_l, 1/s_l; per pixel dlnL/dmu;
  // per catalogue entry dlnL/dm
  const int NLn = LINES && md.use_lines ? g.n_line : 0;
  float2* ln_x = reinterpret_cast<float2*>(reinterpret_cast<char*>(smem) + a.lines_off);
  float* ln_F = reinterpret_cast<float*>(ln_x + NLn);
  float* ln_A = ln_F + NLn;
  float* ln_is = ln_A + NLn;
  float* upx = ln_is + NLn;
  float* ulc = upx + (NLn ? md.n_pix : 0);
  // each thread owns a contiguous run of CH window nodes (CH odd: the runs of a
  // warp fall in distinct shared-memory banks) for the node-owned gathers
  const int nw = k_hi - k_lo + 1;
  const int CH = ((nw + EB_THREADS - 1) / EB_THREADS) | 1;
  const int kr0 = k_lo + tid * CH, kr1 = min(kr0 + CH, k_hi + 1);   // this thread's nodes [kr0, kr1)
  const float* Yr = a.Y + ro;
  const float* Or = a.O + ro;
  const float* O2r = a.O2 && a.o2_split && *a.o2_split ? a.O2 + ro : nullptr;
  const float eb_kc = 0.85f - 1.9f * rs.delta;
  const float opz = 1.f / rs.inv1pz;
  // nebular age axis: the row's Q-weighted weight of each nebular SSP age, and
  // dlnL/dq of each (the second pass after the node loop)
  __shared__ float qa_s[MAX_NEB_AGE], gqa_s[MAX_NEB_AGE];
  const float* qa = nullptr;
  if constexpr (VAR == 2) {
    for (int i = tid; i < g.neb_na; i += EB_THREADS) qa_s[i] = a.qneb[(size_t)r * MAX_NEB_AGE + i];
    __syncthreads();
    qa = qa_s;
  }

  // ---- forward: attenuated spectrum in the window (the forward epilogue's
  //      arithmetic); phi holds the window's wavelengths until the photometric
  //      gather starts
#pragma unroll 1
  for (int k = k_lo + tid; k <= k_hi; k += EB_THREADS) {
    if constexpr (VAR == 1) {
      float yv[MAX_SEG];
#pragma unroll
      for (int sg = 0; sg < MAX_SEG; ++sg) yv[sg] = sg < md.n_seg ? Yr[sg * a.seg_stride + k] : 0.f;
      Fs[k] = attenuated_bins(md, rs, g.att4[k], eb_kc, yv, O2r ? Or[k] + O2r[k] : Or[k], g.neb_tab, k);
    } else {
      Fs[k] = attenuated(md, rs, g.att4[k], eb_kc, Yr[k], O2r ? Or[k] + O2r[k] : Or[k], g, qa, k);
    }
    if (md.use_igm && g.lam_f[k] < IGM_LYA) {   // the IGM transmission (the forward epilogue's)
      float tau, dtau;
      igm_madau(g.att4[k].w, opz, tau, dtau);
      Fs[k] *= __expf(-rs.igm_f * tau);
    }
    phi[k] = g.lam_f[k];
  }
  for (int l = tid; l < NLn; l += EB_THREADS) line_setup(md, g, rs, eb_kc, l, ln_F, ln_A, ln_is, ln_x);
  __syncthreads();
  // the catalogue entries' sigma dlnL/dm = (d - m)/sigma, 0 for a respected
  // upper limit or an entry outside the mask (Eq. app_line_chi2_det,
  // app_line_chi2_UL)
  for (int k = tid; k < md.n_lcat; k += EB_THREADS) {
    const double is = md.lcat_isig[k];
    float m = 0.f;
    for (int j = md.lcat_start[k]; j < md.lcat_start[k + 1]; ++j) m += ln_F[md.lcat_line[j]];
    const double d = md.lcat_d[k];
    double u = (d - (double)m) * is;
    if (md.lcat_ul && md.lcat_ul[k] && (double)m <= d) u = 0.0;
    ulc[k] = (float)u;
  }

  // ---- photometry forward (warp per band, four samples in flight per lane),
  //      the sample brackets, u_b and the gather part of dlnL/dz (the sample
  //      positions lam_j/(1+z) move with z).  Brackets start from the index
  //      table over ln(lambda) (fast logarithm: the walk within the window
  //      ends on the same node from any start).
  const float lam0 = g.lam_f[0], lamN = g.lam_f[N - 1];
  const int kmin = k_lo, kmax = k_hi - 1;
  const float* lam_s = phi;
  float gz_gather = 0.f;
  for (int b = warp; b < md.n_filt; b += EB_WARPS) {
    const int js = md.band_start[b], je = md.band_start[b + 1];
    float acc = 0.f, gzb = 0.f;
    int bmin = 0x7fffffff, bmax = -1;
    for (int j0 = js + lane; j0 < je; j0 += 128) {
      float2 sp[4];   // {lambda_obs, weight}
      int kg[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) sp[u] = j0 + 32 * u < je ? md.samp2[j0 + 32 * u] : make_float2(0.f, 0.f);
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        int q = (int)((__logf(fmaxf(sp[u].x * rs.inv1pz, lam0)) - g.lut_x0) * g.lut_inv_h);
        q = q < 0 ? 0 : (q >= g.lut_n ? g.lut_n - 1 : q);
        kg[u] = g.lut[q];
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int j = j0 + 32 * u;
        if (j >= je) continue;
        const float x = sp[u].x * rs.inv1pz;
        float v = 0.f, t = 0.f;
        int k;
        if (x < lam0) {
          k = -2;
        } else if (x > lamN) {
          k = N;
        } else {
          k = min(max(kg[u], kmin), kmax);
#pragma unroll 1
          while (k < kmax && lam_s[k + 1] <= x) ++k;
#pragma unroll 1
          while (k > kmin && lam_s[k] > x) --k;
          const float la = lam_s[k], lb = lam_s[k + 1];
          t = (x - la) / (lb - la);
          const float G0 = __fdividef(Fs[k], la * la), G1 = __fdividef(Fs[k + 1], lb * lb);
          v = G0 + t * (G1 - G0);
          gzb += sp[u].y * ((G1 - G0) / (lb - la)) * (-x * rs.inv1pz);
          bmin = min(bmin, k);
          bmax = max(bmax, k);
        }
        sk[j] = k;
        st[j] = t;
        acc = fmaf(sp[u].y, v, acc);
      }
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
      acc += __shfl_xor_sync(0xffffffffu, acc, o);
      bmin = min(bmin, __shfl_xor_sync(0xffffffffu, bmin, o));
      bmax = max(bmax, __shfl_xor_sync(0xffffffffu, bmax, o));
    }
    float lsum = 0.f;   // the band's lines (maggies), one line per lane as in the forward
    if (LINES && NLn) {
      for (int l = lane; l < NLn; l += 32) lsum += line_in_band(md, g, rs, b, l, ln_F[l]);
#pragma unroll
      for (int o = 16; o; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
    }
    const float mc = rs.p_phot * acc;   // the continuum part
    const float mb = LINES && NLn ? fmaf(rs.p_phot, acc, lsum) : mc;
    // d lnL / d(band flux) = (d - m)/sigma^2, formed in FP32 from the normalised
    // datum and 1/sigma (0 for a masked band); times p_phot it weighs F
    const float isf = md.phot_isf[b];
    float wb = phot_resid(md, b, md.phot_dn[b], mb * isf);   // (d - m)/sigma; with a noise floor sigma d term / d m
    if (md.floor_bits[0] && isf != 0.f) {
      const float mn = mb * isf, dn = md.phot_dn[b], q = floor_q(rs.fl[0], mn, dn, rs.fl[0][3] * isf);
      wb = floor_dm(rs.fl[0], wb, q, floor_gq(wb, q), mn);
    }
    const float c_b = wb * (isf * rs.p_phot);
    if (lane == 0) {
      mbp[b] = mc;
      mlb[b] = mb - mc;
      ubm[b] = wb;   // sigma_b dlnL/dm_b
      ubp[b] = c_b;
      bk0[b] = bmin;
      bk1[b] = bmax;
    }
    gz_gather += c_b * gzb;
  }
  __syncthreads();

  // ---- dlnL/dF from the photometry: node k gathers the samples bracketed by
  //      [k-1, k] (weight t) and [k, k+1] (weight 1-t), band by band in order
  //      and in sample order within a band.  Each thread owns a run of nodes and
  //      walks the samples that reach it once per band, from one binary search
  //      over the band's (ascending) brackets, with four sample weights in flight.
  for (int k = kr0; k < kr1; ++k) phi[k] = 0.f;
  for (int b = 0; b < md.n_filt; ++b) {
    const float cb = ubp[b];
    const int lo = max(bk0[b], kr0), hi = min(bk1[b] + 1, kr1 - 1);
    if (cb == 0.f || lo > hi) continue;
    const int je = md.band_start[b + 1];
    int j = md.band_start[b], j1 = je;
    while (j < j1) {
      const int mid = (j + j1) >> 1;
      if (sk[mid] < lo - 1) j = mid + 1; else j1 = mid;
    }
    for (; j < je && sk[j] <= hi; j += 4) {
      int kk[4];
      float ww[4], tt[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const bool ok = j + u < je;
        kk[u] = ok ? sk[j + u] : 0x7fffffff;
        ww[u] = ok ? md.samp2[j + u].y : 0.f;
        tt[u] = ok ? st[j + u] : 0.f;
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int k = kk[u];
        if (k > hi) continue;   // brackets ascend: the later samples lie beyond the run too
        const float c = cb * ww[u];
        if (k >= lo) phi[k] += c * (1.f - tt[u]);
        if (k + 1 >= lo && k + 1 <= hi) phi[k + 1] += c * tt[u];
      }
    }
  }
  for (int k = kr0; k < kr1; ++k) phi[k] *= g.inv_lam2[k];
  __syncthreads();

  // ---- spectrum forward (thread per pixel): m_i, u_i, each pixel's node range.
  //      A Gaussian row's range comes from the index table alone (a superset of
  //      the nodes within 5 sigma, clamped to the window): the |u| <= 5 test
  //      decides which nodes enter the sums.
  //      Per-pixel terms in FP32 on the normalised residual (d - mu)/sigma and
  //      model mu/sigma; the constants -1/2 ln(2 pi sigma^2) in FP64.
  double l_spec = 0.0, um_spec = 0.0;
  float chi = 0.f, um_f = 0.f, gz_spec = 0.f, g_sgal = 0.f;
  float gfs[4] = {0.f, 0.f, 0.f, 0.f};   // d lnL / d log10 of the spectral noise-floor terms
  const float ll0 = g.lnl_hi[0], llN = g.lnl_hi[N - 1];
  for (int i = tid; i < md.n_pix; i += EB_THREADS) {
    float xh, xl;
    ln_rest(md.pix_ln2[i], rs.ln1pz_hi, rs.ln1pz_lo, xh, xl);
    // total dispersion: fixed, or sigma_fix composed with the row's sigma_gal (Eq. one_kernel)
    const float s = md.sample_sgal ? sqrtf(md.pix_fix2[i] + rs.sg_ln * rs.sg_ln) : md.pix_s[i];
    float v = 0.f, dv = 0.f, dvs = 0.f, cw = 0.f, tl = 0.f;
    // node range of the pixel; outside the grid a one-node range at the
    // window's edge keeps the ranges in pixel order (the pixel has c = 0)
    int jlo = xh < ll0 ? k_lo : k_hi, jhi = jlo;
    bool valid = false;
    if (xh >= ll0 && xh <= llN) {
      const int k = locate_ln(g, xh, g.lnl_hi);
      const float dln = (g.lnl_hi[k + 1] - g.lnl_hi[k]) + (g.lnl_lo[k + 1] - g.lnl_lo[k]);
      if (s < 0.5f * dln) {
        const float t = ((xh - g.lnl_hi[k]) + (xl - g.lnl_lo[k])) / dln;
        v = Fs[k] + t * (Fs[k + 1] - Fs[k]);
        dv = (Fs[k + 1] - Fs[k]) / dln;
        valid = true;
        jlo = k; jhi = k + 1; tl = t; cw = 1.f;
      } else {
        const float inv_s = 1.f / s;
        int qa = (int)((fmaxf(xh - 5.f * s, ll0) - g.lut_x0) * g.lut_inv_h);
        int qb = (int)((fminf(xh + 5.f * s, llN) - g.lut_x0) * g.lut_inv_h);
        qa = min(max(qa, 0), g.lut_n - 1);
        qb = min(max(qb, 0), g.lut_n - 1);
        jlo = max(g.lut[qa] - 1, k_lo);
        jhi = min(g.lut[qb] + 3, k_hi);
        // a node past 5 dispersions weighs exactly 0 (its terms add zeros), so
        // the loop carries no branch and its loads pipeline
        float sw = 0.f, sf = 0.f, swd = 0.f, sfd = 0.f, sws = 0.f, sfs = 0.f;
        if (md.sample_sgal) {
#pragma unroll 4
          for (int j = jlo; j <= jhi; ++j) {
            const float d = (g.lnl_hi[j] - xh) + (g.lnl_lo[j] - xl);
            const float u = d * inv_s;
            const float w = fabsf(u) <= 5.f ? __expf(-0.5f * u * u) : 0.f;
            const float wd = w * u * inv_s;   // dw/dx
            const float ws = wd * u;          // dw/ds = w u^2 / s
            const float f = Fs[j];
            sw += w;
            sf = fmaf(w, f, sf);
            swd += wd;
            sfd = fmaf(wd, f, sfd);
            sws += ws;
            sfs = fmaf(ws, f, sfs);
          }
        } else {
#pragma unroll 4
          for (int j = jlo; j <= jhi; ++j) {
            const float d = (g.lnl_hi[j] - xh) + (g.lnl_lo[j] - xl);
            const float u = d * inv_s;
            const float w = fabsf(u) <= 5.f ? __expf(-0.5f * u * u) : 0.f;
            const float wd = w * u * inv_s;   // dw/dx
            const float f = Fs[j];
            sw += w;
            sf = fmaf(w, f, sf);
            swd += wd;
            sfd = fmaf(wd, f, sfd);
          }
        }
        tl = -1.f - inv_s;
        if (sw > 0.f) {
          v = sf / sw;
          dv = (sfd * sw - sf * swd) / (sw * sw);
          dvs = (sfs * sw - sf * sws) / (sw * sw);
          valid = true;
          cw = 1.f / sw;
        }
      }
    }
    const float mline = LINES && NLn ? lines_at_pixel(md, i, NLn, ln_A, ln_is, ln_x) : 0.f;
    const float mi = LINES && NLn ? fmaf(rs.s_spec, v, mline) : rs.s_spec * v;
    float ci = 0.f;
    const float isf = md.spec_isf[i];
    const bool inc = valid && isf != 0.f;
    const float ms = inc ? mi * isf : 0.f;   // mu / sigma
    const float lms = inc ? mline * isf : 0.f;   // its line part
    const float rn = md.spec_dn[i] - ms;     // (d - mu) / sigma where included
    float wsn = rn;                          // sigma d term / d mu
    if (inc) {
      if (md.floor_bits[1]) {                // sigma_eff of Eq. app_noise_floor
        const float dn = md.spec_dn[i], jn = rs.fl[1][3] * isf, q = floor_q(rs.fl[1], ms, dn, jn);
        const float gq = floor_gq(rn, q);
        chi -= 0.5f * (rn * rn / q + logf(q));
        wsn = floor_dm(rs.fl[1], rn, q, gq, ms);
        floor_dparam(rs.fl[1], gq, ms, dn, jn, gfs);
      } else {
        chi = fmaf(-0.5f * rn, rn, chi);
      }
      l_spec += md.spec_nlog[i];
    }
    if (md.calib_n) {
      // the weights need the whole row's calibration solve: keep what they use
      mu_s[i] = ms;
      dv_s[i] = dv;
      dvs_s[i] = dvs;
      cw_s[i] = cw;
      if (NLn) upx[i] = lms;
    } else if (inc) {
      // d lnL / d mu_i = r_i / sigma_i^2 (wsn / sigma_i with a noise floor);
      // d lnL / d v_i = that x s_spec (mu = s_spec v); the mass derivative
      // takes the continuum part (the lines' is in their own pass)
      um_f = fmaf(wsn, ms - lms, um_f);
      const float us = wsn * (isf * rs.s_spec);
      gz_spec += us * dv * (-rs.inv1pz);
      // s = sqrt(sigma_fix^2 + sigma_gal^2) / c: ds/dsigma_gal = (sigma_gal / c) / (s c)
      if (md.sample_sgal && s > 0.f) g_sgal += us * dvs * (rs.sg_ln / (s * (float)C_KMS));
      ci = us * cw;
    }
    if (NLn && !md.calib_n) upx[i] = inc ? wsn : 0.f;   // sigma_i d lnL / d mu_i
    prg[i] = (jlo & 0xffff) | (jhi << 16);
    px4[i] = make_float4(xh, xl, ci, tl);   // x_hi ascending in i: the pixels' wavelengths are strictly increasing
  }
  if (md.calib_n) {
    // ---- marginalised calibration (App. E): moments over this thread's own
    //      pixels, one solve per row, then each included pixel's lnL change
    //      (calib_pixel_term) and
    //      d lnL / d mu_i = [(d_i - mu_i (1 + p_i)) (1 + p_i) - mu_i q_i] / sigma_i^2
    //      (all in FP32 on the normalised values),
    //      p = A c*, q_i = |L^-1 T(x_i)|^2 (M = L L^T)
    calib_block<0, 0, EB_THREADS>(md, mu_s, cal_cf, tid, lane, warp, cal_part);
    calib_block<SED_MAX_CALIB, 0, EB_THREADS>(md, mu_s, cal_cf, tid, lane, warp, cal_part);
    calib_block<0, 1, EB_THREADS>(md, mu_s, cal_cf, tid, lane, warp, cal_part);
    __syncthreads();
    if (warp == 0) {
      const double f = calib_first_solve(md, cal_part, EB_WARPS, cal_Lf, cal_Df, cal_cf, lane);
      if (lane == 0) l_spec += f;
    }
    __syncthreads();
    // one refinement of c* from the pixels' calibrated residuals (the gradient
    // takes c* at first order)
    calib_block<0, 2, EB_THREADS>(md, mu_s, cal_cf, tid, lane, warp, cal_part);
    __syncthreads();
    if (warp == 0) {
      const double f = calib_refine(md, cal_part, EB_WARPS, cal_Lf, cal_Df, cal_cf, lane);
      if (lane == 0) l_spec += f;
    }
    __syncthreads();
    const int n = md.calib_n;
    for (int i = tid; i < md.n_pix; i += EB_THREADS) {
      const float m = mu_s[i];
      if (m == 0.f) {
        if (NLn) upx[i] = 0.f;
        continue;
      }
      const float x = md.pix_cx[i];
      float T[SED_MAX_CALIB], y[SED_MAX_CALIB];
      float p = 0.f, q = 0.f, tp = 1.f, tc = x;
#pragma unroll
      for (int a = 0; a < SED_MAX_CALIB; ++a) {
        T[a] = a == 0 ? 1.f : tc;
        if (a > 0) { const float tn = 2.f * x * tc - tp; tp = tc; tc = tn; }
      }
#pragma unroll
      for (int a = 0; a < SED_MAX_CALIB; ++a) {
        if (a < n) {
          p = fmaf(cal_cf[a], T[a], p);
          if (!md.calib_opt) {   // the optimised polynomial has no ln|M| term
            float v = T[a];
#pragma unroll
            for (int k = 0; k < a; ++k) v -= cal_Lf[a * n + k] * y[k];
            y[a] = v * cal_Df[a];
            q = fmaf(y[a], y[a], q);
          }
        }
      }
      // sigma_i d lnL / d mu_i = (r_i - mu_i p_i)(1 + p_i)/sigma_i - (mu_i/sigma_i) q_i
      const float rn = md.spec_dn[i] - m;
      chi += calib_pixel_term(rn, m, p);
      const float ws = fmaf(rn - m * p, 1.f + p, -m * q);
      um_f = fmaf(ws, NLn ? m - upx[i] : m, um_f);
      if (NLn) upx[i] = ws;   // sigma_i d lnL / d mu_i
      const float us = ws * (md.spec_isf[i] * rs.s_spec);
      gz_spec += us * dv_s[i] * (-rs.inv1pz);
      if (md.sample_sgal) {
        const float s = sqrtf(md.pix_fix2[i] + rs.sg_ln * rs.sg_ln);
        if (s > 0.f) g_sgal += us * dvs_s[i] * (rs.sg_ln / (s * (float)C_KMS));
      }
      px4[i].z = us * cw_s[i];
    }
  }
  l_spec += (double)chi;
  um_spec += (double)um_f;
  __syncthreads();

  // ---- dlnL/dF from the spectrum: node k gathers, in pixel order, every
  //      pixel whose node range holds k.  When the ranges' ends ascend with the
  //      pixel (the usual case: wavelengths ascend and the dispersion varies
  //      slowly), those pixels are exactly [first p with hi_p >= k, last p with
  //      lo_p <= k], two binary searches.  Otherwise they lie within R of
  //      ln(lam_k) in ln(lambda) (R = 5 sigma_max for Gaussian rows, one node
  //      spacing for linear ones), a run of the ascending pixel positions that is
  //      tested pixel by pixel.  Neighbouring threads take neighbouring nodes, so
  //      the searches and scans of a warp read nearby pixels.
  if (md.n_pix > 0) {
    const int P = md.n_pix;
    int mono = 1;
    for (int i = tid + 1; i < P; i += EB_THREADS) {
      const int r0 = prg[i - 1], r1 = prg[i];
      if ((r1 & 0xffff) < (r0 & 0xffff) || (r1 >> 16) < (r0 >> 16)) mono = 0;
    }
    mono = __syncthreads_and(mono);
    const float R = 5.f * md.pix_s_max * 1.0001f + g.dln_max * 1.0001f + 1e-6f;
    for (int k = k_lo + tid; k <= k_hi; k += EB_THREADS) {
      const float lh = g.lnl_hi[k], ll = g.lnl_lo[k];
      float acc = 0.f;
      if (mono) {
        int pa = 0, pe = P;
        while (pa < pe) {
          const int mid = (pa + pe) >> 1;
          if ((prg[mid] >> 16) < k) pa = mid + 1; else pe = mid;
        }
        int pb = pa;
        pe = P;
        while (pb < pe) {
          const int mid = (pb + pe) >> 1;
          if ((prg[mid] & 0xffff) <= k) pb = mid + 1; else pe = mid;
        }
        // lo_p <= k <= hi_p for every p here; a pixel with c = 0 (excluded)
        // adds an exact zero, so the loop carries no branch
#pragma unroll 4
        for (int p = pa; p < pb; ++p) {
          const float4 q = px4[p];
          const float d = (lh - q.x) + (ll - q.y);
          const float u = d * (-1.f - q.w);   // Gaussian row: 1/sigma = -1 - q.w
          const float wg = fabsf(u) <= 5.f ? __expf(-0.5f * u * u) : 0.f;
          const float wl = k == (prg[p] & 0xffff) ? 1.f - q.w : q.w;   // linear row: q.w = t in [0, 1]
          acc = fmaf(q.z, q.w > -0.5f ? wl : wg, acc);
        }
      } else {
        int p = 0, p1 = P;
        while (p < p1) {
          const int mid = (p + p1) >> 1;
          if (px4[mid].x < lh - R) p = mid + 1; else p1 = mid;
        }
        for (; p < P; ++p) {
          const float4 q = px4[p];
          if (q.x >= lh + R) break;
          const int rg = prg[p], lo = rg & 0xffff, hi = rg >> 16;
          if (q.z == 0.f || k < lo || k > hi) continue;
          float w;
          if (q.w > -0.5f) {   // linear row
            w = k == lo ? 1.f - q.w : q.w;
          } else {              // Gaussian row, 1/sigma = -1 - q.w
            const float d = (lh - q.x) + (ll - q.y);
            const float u = d * (-1.f - q.w);
            w = fabsf(u) <= 5.f ? __expf(-0.5f * u * u) : 0.f;
          }
          acc = fmaf(q.z, w, acc);
        }
      }
      phi[k] += acc;
    }
  }
  __syncthreads();

  // ---- dust and nebular: dlnL/dY, dlnL/dO and the parameter sums over lambda
  float g_tbc = 0.f, g_abc = 0.f, g_td = 0.f, g_dl = 0.f, g_qy = 0.f, g_lu = 0.f, g_lz = 0.f, g_fob = 0.f;
  float g_sgas = 0.f, g_lm = 0.f;   // lines: d/dsigma_gas (sampled), d/dln F summed over lines (mass)
  float g_igm = 0.f;                // d/digm_factor (the IGM's redshift derivative joins gz_spec)

  // ---- emission lines, thread per line.  F_l = Q fac_l B_l with Q = Q_young
  //      (device units), fac_l the attenuation factor and B_l = 10^(lg_l)
  //      s_spec/(1+z) the flux per unit of both.  The derivatives are gathered
  //      per unit of B_l from the normalised ones of the data (sigma dlnL/dm
  //      times m's sensitivity over sigma), which stay within FP32's range:
  //      G = B dlnL/dF, Gx and Gs the centre's and width's (per unit of Q fac)
  //      from the pixels within 5 s_l (pixel order), every band (in order) and
  //      the catalogue entries naming the line; then to the parameters
  for (int l = tid; l < NLn; l += EB_THREADS) {
    const float is = ln_is[l];
    const float2 xlp = ln_x[l];
    const float4 c = g.line_att4[l];
    const float lam_obs = c.w / rs.inv1pz;
    float lg = 0.f, su = 0.f, sz = 0.f;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float tv = g.line_tab[(rs.neb_off[q] / N) * g.n_line + l];
      lg = fmaf(rs.neb_w[q], tv, lg);
      su = fmaf(rs.neb_dwu[q], tv, su);
      sz = fmaf(rs.neb_dwz[q], tv, sz);
    }
    float B = ex2_approx(3.3219280948873623f * lg) * rs.s_spec * rs.inv1pz;
    float ltau = 0.f, ldtau = 0.f;   // the IGM at the line (B carries its transmission)
    if (md.use_igm && c.w < IGM_LYA) {
      igm_madau(c.w, opz, ltau, ldtau);
      B *= __expf(-rs.igm_f * ltau);
    }
    float G = 0.f, Gx = 0.f, Gs = 0.f, Gzp = 0.f;
    if (md.n_pix > 0 && is > 0.f) {
      const float sw = 5.0001f / is;
      int i = 0, i1 = md.n_pix;
      while (i < i1) {   // first pixel with ln(lambda) >= x - 5 s
        const int mid = (i + i1) >> 1;
        if (md.pix_ln2[mid].x < xlp.x - sw) i = mid + 1; else i1 = mid;
      }
      for (; i < md.n_pix && md.pix_ln2[i].x <= xlp.x + sw; ++i) {
        const float up = upx[i];
        if (up == 0.f) continue;
        const float2 p = md.pix_ln2[i];
        const float u = ((p.x - xlp.x) + (p.y - xlp.y)) * is;
        if (fabsf(u) > 5.f) continue;
        // B dmu_i/dF_l / sigma_i: the profile at the pixel per unit of Q fac, normalised
        const float eb = md.spec_isf[i] * md.pix_lamc[i] * B * (__expf(-0.5f * u * u) * is * 0.3989422804014327f);
        const float w = up * eb;
        G += w;
        Gx = fmaf(w, u * is, Gx);                 // dmu / d ln(lam_obs) = F e u / s
        Gs = fmaf(w, fmaf(u, u, -1.f) * is, Gs);  // dmu / ds = F e (u^2 - 1) / s
      }
    }
    for (int b = 0; b < md.n_filt; ++b) {
      const float ub = ubm[b];
      if (ub == 0.f) continue;
      float rz, drz;
      line_band_resp(md, b, lam_obs, rz, drz);
      const float wb = ub * (md.phot_isf[b] * B);
      G = fmaf(wb, rz * lam_obs, G);
      Gzp = fmaf(wb, fmaf(lam_obs, drz, rz) * c.w, Gzp);   // d(rz x)/dx, dx/dz = lam_l
    }
    for (int k = 0; k < md.n_lcat; ++k)
      for (int j = md.lcat_start[k]; j < md.lcat_start[k + 1]; ++j)
        if (md.lcat_line[j] == l) G = fmaf(ulc[k], (float)(md.lcat_isig[k] * (double)B), G);
    // attenuation factor of the line (atten.cuh's factor of the nebular emission)
    const float pa = __expf(rs.alpha_bc * c.x), tbc = rs.tau_bc * pa;
    const float pw = __expf(rs.delta * c.x), shape = dust_shape(md, c, eb_kc, pw);
    const float dshape = md.dust_law == SED_DUST_POWER_LAW ? pw * c.x : -1.9f * c.z * pw + shape * c.x;
    const float ed = __expf(-rs.tau_d * shape), ebc = __expf(-tbc), f = rs.fob;
    float fac, dfac_tbc, dfac_f;
    if (md.fesc_geom == SED_FESC_PICKET) {
      fac = ed * (1.f - f) * ebc;
      dfac_tbc = -fac;
      dfac_f = -ed * ebc;
    } else {
      const float T = (1.f - f) * ebc + f;
      fac = ed * T * (1.f - f);
      dfac_tbc = -ed * (1.f - f) * (1.f - f) * ebc;
      dfac_f = ed * fmaf(1.f - ebc, 1.f - f, -T);
    }
    const float Q = ex2_approx(rs.log2_qy);
    const float gfac = G * Q;          // dlnL / dfac
    const float gF = gfac * fac;       // dlnL / d ln F_l
    g_tbc = fmaf(gfac * dfac_tbc, pa, g_tbc);
    g_abc = fmaf(gfac * dfac_tbc, tbc * c.x, g_abc);
    const float gtd = -gF;             // dlnL / dtau_d(lam_l)
    g_td = fmaf(gtd, shape, g_td);
    g_dl = fmaf(gtd, rs.tau_d * dshape, g_dl);
    if (md.fesc_geom) g_fob = fmaf(gfac, dfac_f, g_fob);
    g_qy = fmaf(G, fac, g_qy);        // dlnL / dQ_young
    g_lu = fmaf(gF * 2.302585092994046f, su, g_lu);
    g_lz = fmaf(gF * 2.302585092994046f, sz, g_lz);
    g_lm += gF;
    // redshift: the flux factor s_spec/(1+z), the profile's centre on the
    // pixels, its width through sigma_inst(lam_obs), the bands' response
    const float qf = Q * fac;
    float gzl = gF * (rs.dlns_dz - rs.inv1pz - rs.igm_f * ldtau) + qf * (Gx * rs.inv1pz + Gzp);
    g_igm = fmaf(-gF, ltau, g_igm);
    if (md.n_pix > 0 && is > 0.f) {
      float si, dsi;
      line_sigma_inst(md, xlp.x, lam_obs, si, dsi);
      const float kc2 = (float)(1.0 / (C_KMS * C_KMS));
      const float gs = qf * Gs;
      gzl = fmaf(gs, si * dsi * c.w * is * kc2, gzl);        // ds/dz = sigma_inst sigma_inst' lam_l / (c^2 s)
      const float gsg = gs * rs.sgas * is * kc2;              // ds/dsigma_gas = sigma_gas / (c^2 s)
      if (md.gas_mode == SED_GAS_SIGMA_SAMPLED) g_sgas += gsg;
      else if (md.gas_mode == SED_GAS_SIGMA_TIED && md.sample_sgal) g_sgal += gsg;
    }
    gz_spec += gzl;
  }
  // age-binned dust: d/d(tau_b, slope_b) of each bin, d/dQ of each block
  float g_bin[2 * MAX_DUST_BIN] = {}, g_qs[MAX_SEG + 1] = {};
  if constexpr (VAR == 1) {
    // F = e^{-tau_d} [ sum_s A_s (Y_s + Q_s neb) + O + Q_rest neb ], A_s = e^{-tau_s},
    // tau_s = sum_b M_sb tau_b shape_b (atten.cuh's attenuated_bins)
    for (int k = tid; k < a.ldn; k += EB_THREADS) {
      if (k < k_lo || k > k_hi) {
        for (int sg = 0; sg < md.n_seg; ++sg) put_g(a, a.gy_hi, a.gy_lo, sg * a.seg_stride + ro + k, 0.f);
        put_g(a, a.go_hi, a.go_lo, ro + k, 0.f);
        continue;
      }
      const float4 c = g.att4[k];
      const float pw = __expf(rs.delta * c.x);
      const float shape = dust_shape(md, c, eb_kc, pw);
      const float dshape = md.dust_law == SED_DUST_POWER_LAW ? pw * c.x : -1.9f * c.z * pw + shape * c.x;
      const float ed = __expf(-rs.tau_d * shape);
      float lg = 0.f, nbu = 0.f;   // log10 and value of the nebular template per unit Q
      if (md.use_neb) {
        lg = neb_log10(rs, g.neb_tab, k);
        nbu = ex2_approx(3.3219280948873623f * lg);
      }
      // with the IGM, F = T F0: dlnL/dF0 = T dlnL/dF, and ln T = -f tau moves with f and z
      float T = 1.f, F0 = Fs[k];
      if (md.use_igm && c.w < IGM_LYA) {
        float tau, dtau;
        igm_madau(c.w, opz, tau, dtau);
        T = __expf(-rs.igm_f * tau);
        const float gl = phi[k] * Fs[k];   // dlnL / d ln T
        g_igm = fmaf(-gl, tau, g_igm);
        gz_spec = fmaf(-gl * rs.igm_f, dtau, gz_spec);
        F0 = T > 0.f ? Fs[k] / T : 0.f;
      }
      const float gF = phi[k] * T;
      const float gtd = -gF * F0;
      const float go = gF * ed;
      put_g(a, a.go_hi, a.go_lo, ro + k, go);
      float shp[MAX_DUST_BIN], dsh[MAX_DUST_BIN], kap[MAX_DUST_BIN], gk[MAX_DUST_BIN];
#pragma unroll
      for (int b = 0; b < MAX_DUST_BIN; ++b) {
        shp[b] = dsh[b] = kap[b] = gk[b] = 0.f;
        if (b < md.n_bin) {
          const float sl = rs.bin_slope[b], pb = __expf(sl * c.x);
          shp[b] = md.bin_law[b] == SED_DUST_POWER_LAW ? pb : (c.y + (0.85f - 1.9f * sl) * c.z) * pb;
          dsh[b] = md.bin_law[b] == SED_DUST_POWER_LAW ? pb * c.x : -1.9f * c.z * pb + shp[b] * c.x;
          kap[b] = rs.bin_tau[b] * shp[b];
        }
      }
      float gneb = 0.f;   // dlnL / d(neb per unit Q) summed over the blocks, times Q
      if (md.use_neb) {
        const float qr = ex2_approx(rs.log2_qs[MAX_SEG]);
        g_qs[MAX_SEG] = fmaf(go, nbu, g_qs[MAX_SEG]);
        gneb = go * qr;
      }
#pragma unroll
      for (int sg = 0; sg < MAX_SEG; ++sg) {
        if (sg >= md.n_seg) break;
        float tau = 0.f;
#pragma unroll
        for (int b = 0; b < MAX_DUST_BIN; ++b) tau = fmaf(md.seg_M[sg][b], kap[b], tau);
        const float gys = go * __expf(-tau);
        put_g(a, a.gy_hi, a.gy_lo, sg * a.seg_stride + ro + k, gys);
        const float qs = md.use_neb ? ex2_approx(rs.log2_qs[sg]) : 0.f;
        const float gtau = -gys * fmaf(qs, nbu, Yr[sg * a.seg_stride + k]);
#pragma unroll
        for (int b = 0; b < MAX_DUST_BIN; ++b) gk[b] = fmaf(gtau, md.seg_M[sg][b], gk[b]);
        if (md.use_neb) {
          g_qs[sg] = fmaf(gys, nbu, g_qs[sg]);
          gneb = fmaf(gys, qs, gneb);
        }
      }
#pragma unroll
      for (int b = 0; b < MAX_DUST_BIN; ++b) {
        g_bin[2 * b] = fmaf(gk[b], shp[b], g_bin[2 * b]);
        g_bin[2 * b + 1] = fmaf(gk[b] * rs.bin_tau[b], dsh[b], g_bin[2 * b + 1]);
      }
      g_td += gtd * shape;
      g_dl += gtd * rs.tau_d * dshape;
      if (md.use_neb) {
        const float glg = gneb * nbu * 2.302585092994046f;
        float su = 0.f, sz = 0.f;
#pragma unroll
        for (int cc = 0; cc < 4; ++cc) {
          const float tv = g.neb_tab[rs.neb_off[cc] + k];
          su += rs.neb_dwu[cc] * tv;
          sz += rs.neb_dwz[cc] * tv;
        }
        g_lu += glg * su;
        g_lz += glg * sz;
      }
    }
  } else
  for (int k = tid; k < a.ldn; k += EB_THREADS) {
    if (k < k_lo || k > k_hi) {
      put_g(a, a.gy_hi, a.gy_lo, ro + k, 0.f);
      put_g(a, a.go_hi, a.go_lo, ro + k, 0.f);
      continue;
    }
    const float4 c = g.att4[k];
    const float lnp = c.x;
    const float pa = __expf(rs.alpha_bc * lnp);
    const float tbc = rs.tau_bc * pa;
    const float pw = __expf(rs.delta * lnp);
    const float shape = dust_shape(md, c, eb_kc, pw);
    const float dshape = md.dust_law == SED_DUST_POWER_LAW ? pw * lnp : -1.9f * c.z * pw + shape * lnp;
    const float td = rs.tau_d * shape;
    const float ed = __expf(-td), eb = __expf(-tbc);
    const float y = Yr[k];
    float lg = 0.f, nb = 0.f;
    if (md.use_neb) {
      if (qa) {
        nb = neb_emission(rs, g, qa, k);
      } else {
        lg = neb_log10(rs, g.neb_tab, k);
        nb = ex2_approx(rs.log2_qy + 3.3219280948873623f * lg);
      }
    }
    // with the IGM, F = T F0: dlnL/dF0 = T dlnL/dF, and ln T = -f tau moves with f and z
    float T = 1.f, F0 = Fs[k];
    if (md.use_igm && c.w < IGM_LYA) {
      float tau, dtau;
      igm_madau(c.w, opz, tau, dtau);
      T = __expf(-rs.igm_f * tau);
      const float gl = phi[k] * Fs[k];   // dlnL / d ln T
      g_igm = fmaf(-gl, tau, g_igm);
      gz_spec = fmaf(-gl * rs.igm_f, dtau, gz_spec);
      F0 = T > 0.f ? Fs[k] / T : 0.f;
    }
    const float gF = phi[k] * T;
    // dF/dY, dF/dtau_BC (as gtbc), dF/dneb and dF/df of the node (atten.cuh's F)
    float gy, gtbc, gnb;
    float gtd = -gF * F0;
    if (md.fesc_geom == SED_FESC_NONE) {
      gy = gF * ed * eb;
      gtbc = -gy * (y + nb);
      gnb = gy;
    } else {
      const float f = rs.fob, c = (md.use_neb && k < md.n_lyc) ? 0.f : 1.f;
      if (md.fesc_geom == SED_FESC_PICKET) {
        const float b = c * y + nb, se = ed * (1.f - f) * eb;
        gy = gF * (f + se * c);
        gtbc = -gF * se * b;
        gnb = gF * se;
        g_fob += gF * (y - ed * eb * b);
        gtd = -gF * (F0 - f * y);   // the escaping light crosses no screen
      } else {
        const float T = (1.f - f) * eb + f, av = c * y + (1.f - f) * nb;
        gy = gF * ed * (T * c + f * (1.f - c));
        gtbc = -gF * ed * (1.f - f) * eb * av;
        gnb = gF * ed * T * (1.f - f);
        g_fob += gF * ed * ((1.f - eb) * av - T * nb + (1.f - c) * y);
      }
    }
    const float go = gF * ed;
    put_g(a, a.gy_hi, a.gy_lo, ro + k, gy);
    put_g(a, a.go_hi, a.go_lo, ro + k, go);
    g_tbc += gtbc * pa;
    g_abc += gtbc * tbc * lnp;
    g_td += gtd * shape;
    g_dl += gtd * rs.tau_d * dshape;
    if (md.use_neb && qa) {
      phi[k] = gnb;   // dlnL / d(nebular emission) of the node, for the per-age pass below
    } else if (md.use_neb) {
      g_qy += gnb * ex2_approx(3.3219280948873623f * lg);
      const float glg = gnb * nb * 2.302585092994046f;
      float su = 0.f, sz = 0.f;
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const float tv = g.neb_tab[rs.neb_off[c] + k];
        su += rs.neb_dwu[c] * tv;
        sz += rs.neb_dwz[c] * tv;
      }
      g_lu += glg * su;
      g_lz += glg * sz;
    }
  }
  if (qa) {
    // nebular age axis: warp per nebular SSP age, lanes over the window's
    // nodes (node order, fixed shuffle tree): dlnL/dq_a = sum_k g_k e_a(k) and
    // the (log U, log Z_gas) derivative of each age's plane, g_k = dlnL/d(neb)
    // at node k (phi), e_a(k) = 10^(the cube at age a)
    __syncthreads();
    const size_t plane = (size_t)g.neb_nu * g.neb_nz * N;
    for (int i = warp; i < g.neb_na; i += EB_WARPS) {
      const float q = qa[i];
      const float* tb = g.neb_tab + i * plane;
      float sq = 0.f;
      for (int k = k_lo + lane; k <= k_hi; k += 32) {
        float lgi = 0.f, su = 0.f, sz = 0.f;
#pragma unroll
        for (int cc = 0; cc < 4; ++cc) {
          const float tv = tb[rs.neb_off[cc] + k];
          lgi = fmaf(rs.neb_w[cc], tv, lgi);
          su = fmaf(rs.neb_dwu[cc], tv, su);
          sz = fmaf(rs.neb_dwz[cc], tv, sz);
        }
        const float e = ex2_approx(3.3219280948873623f * lgi);
        const float gn = phi[k];
        sq = fmaf(gn, e, sq);
        const float glg = gn * q * e * 2.302585092994046f;
        g_lu = fmaf(glg, su, g_lu);
        g_lz = fmaf(glg, sz, g_lz);
      }
#pragma unroll
      for (int o = 16; o; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
      if (lane == 0) gqa_s[i] = sq;
    }
  }

  // ---- fixed-order reductions of the per-thread pieces: the FP32 sums within
  //      the warp in FP32, lnL and d lnL/d ln(mass) in FP64; across the warps
  //      in FP64, one column per lane of warp 0
  float vf[EB_NREDF] = {g_tbc, g_abc, g_td, g_dl, g_lz, g_lu, gz_gather + gz_spec, g_qy, g_sgal,
                        gfs[0], gfs[1], gfs[2], gfs[3], g_fob, g_sgas, g_lm, g_igm};
#pragma unroll
  for (int q = 0; q < EB_NREDF; ++q) {
#pragma unroll
    for (int o = 16; o; o >>= 1) vf[q] += __shfl_xor_sync(0xffffffffu, vf[q], o);
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    l_spec += __shfl_xor_sync(0xffffffffu, l_spec, o);
    um_spec += __shfl_xor_sync(0xffffffffu, um_spec, o);
  }
  if constexpr (VAR == 1) {
#pragma unroll
    for (int q = 0; q < 2 * MAX_DUST_BIN; ++q)
#pragma unroll
      for (int o = 16; o; o >>= 1) g_bin[q] += __shfl_xor_sync(0xffffffffu, g_bin[q], o);
#pragma unroll
    for (int q = 0; q <= MAX_SEG; ++q)
#pragma unroll
      for (int o = 16; o; o >>= 1) g_qs[q] += __shfl_xor_sync(0xffffffffu, g_qs[q], o);
  }
  if (lane == 0) {
#pragma unroll
    for (int q = 0; q < EB_NREDF; ++q) red[warp][q] = (double)vf[q];
    red[warp][EB_NREDF] = l_spec;
    red[warp][EB_NREDF + 1] = um_spec;
    if constexpr (VAR == 1) {
#pragma unroll
      for (int q = 0; q < 2 * MAX_DUST_BIN; ++q) red[warp][EB_NRED + q] = (double)g_bin[q];
#pragma unroll
      for (int q = 0; q <= MAX_SEG; ++q) red[warp][EB_NRED + 2 * MAX_DUST_BIN + q] = (double)g_qs[q];
    }
  }
  __syncthreads();
  if (warp == 0) {
    double col = 0.0;
    if (lane < (VAR == 1 ? EB_NRED + EB_NREDB : EB_NRED))
      for (int w = 0; w < EB_WARPS; ++w) col += red[w][lane];
    // the photometric lnL terms and d lnL/d ln(mass) pieces in FP64, one band per lane
    double bl = 0.0, bu = 0.0, gfp[4] = {0.0, 0.0, 0.0, 0.0};
    for (int b = lane; b < md.n_filt; b += 32) {
      if (md.phot_isig[b] != 0.0) {
        // the band's model (continuum + lines) for lnL; its continuum part for
        // the mass derivative (the lines' runs through their own pass)
        const double is = md.phot_isig[b], mc = (double)mbp[b] * is;
        const double mn = NLn ? (double)(mbp[b] + mlb[b]) * is : mc, dn = md.phot_d[b] * is;
        const double rr = phot_resid(md, b, dn, mn);
        if (md.floor_bits[0]) {   // sigma_eff of Eq. app_noise_floor
          const double jn = (double)rs.fl[0][3] * is, q = floor_q(rs.fl[0], mn, dn, jn), gq = floor_gq(rr, q);
          bl += -0.5 * (rr * rr / q + log(q)) + md.phot_nlog[b];
          bu += floor_dm(rs.fl[0], rr, q, gq, mn) * mc;
          floor_dparam(rs.fl[0], gq, mn, dn, jn, gfp);
        } else {
          bl += -0.5 * rr * rr + md.phot_nlog[b];
          bu += rr * mc;
        }
      }
    }
    if (LINES)
      for (int k = lane; k < md.n_lcat; k += 32) bl += lcat_term(md, k, ln_F);   // the line catalogue
#pragma unroll
    for (int o = 16; o; o >>= 1) {
      bl += __shfl_xor_sync(0xffffffffu, bl, o);
      bu += __shfl_xor_sync(0xffffffffu, bu, o);
      if (md.floor_bits[0])
        for (int k = 0; k < 4; ++k) gfp[k] += __shfl_xor_sync(0xffffffffu, gfp[k], o);
    }
    double s[EB_NRED + EB_NREDB];
#pragma unroll
    for (int q = 0; q < EB_NRED + EB_NREDB; ++q) s[q] = __shfl_sync(0xffffffffu, col, q);
    if (lane == 0) {
      double lnl = s[EB_NREDF] + bl, um_phot = bu;
      const double um_sp = s[EB_NREDF + 1];
      double* rg = a.rgrad + (size_t)r * RGRAD;
      uint32_t stt = 0;
      if (!isfinite(lnl)) { stt = SED_ROW_NONFINITE; lnl = -INFINITY; }
      rg[RG_TAU_BC] = s[0];
      rg[RG_ALPHA_BC] = s[1];
      rg[RG_TAU_D] = s[2];
      rg[RG_DELTA] = s[3];
      rg[RG_GAS_LOGZ] = s[4];
      rg[RG_GAS_LOGU] = s[5];
      rg[RG_LOGMASS] = 2.302585092994046 * (um_phot + um_sp + s[15]);
      rg[RG_Z] = um_phot * (double)rs.dlnp_dz + um_sp * (double)rs.dlns_dz + s[6];
      rg[RG_QY] = s[7];
      rg[RG_SIGMA_GAL] = s[8];
      rg[RG_FOB] = s[13];
      rg[RG_SIGMA_GAS] = s[14];
      rg[RG_IGM] = s[16];
      if (qa)
        for (int i = 0; i < g.neb_na; ++i) rg[RG_QAGE + i] = (double)gqa_s[i];
      for (int k = 0; k < 4; ++k) {
        rg[RG_FLOOR + k] = gfp[k];
        rg[RG_FLOOR + 4 + k] = s[9 + k];
      }
      if constexpr (VAR == 1) {
        for (int q = 0; q < 2 * MAX_DUST_BIN; ++q) rg[RG_BIN + q] = s[EB_NRED + q];
        for (int q = 0; q <= MAX_SEG; ++q) rg[RG_QSEG + q] = s[EB_NRED + 2 * MAX_DUST_BIN + q];
        rg[RG_QY] = s[EB_NRED + 2 * MAX_DUST_BIN];
      }
      rg[RG_BAD] = stt ? 1.0 : 0.0;
      if (a.lnl) a.lnl[rs.orig] = lnl;
      if (a.status) a.status[rs.orig] = stt;
    }
  }
}

cudaError_t launch_epilogue_bwd(const EpiBwdArgs& a_in, size_t* smem_needed, cudaStream_t s) {
  EpiBwdArgs a = a_in;
  a.lines_off = (int)epi_bwd_lines_off(a);
  const size_t smem = epi_bwd_smem(a);
  if (smem_needed) *smem_needed = smem;
  static DynSmemCache set_for[4];
  const int m = a.md.n_bin > 0 ? 2 : a.qneb ? 3 : (a.md.use_lines ? 1 : 0);
  auto k = m == 3 ? k_epi_bwd<false, 2> : m == 2 ? k_epi_bwd<false, 1> : (m == 1 ? k_epi_bwd<true> : k_epi_bwd<false>);
  cudaError_t e = ensure_dyn_smem(k, smem, &set_for[m]);
  if (e != cudaSuccess) return e;
  return launch_pdl(k, dim3(a.n), dim3(EB_THREADS), smem, s, a);
}

// ---------------------------------------------------------------------------
// CUDA-core adjoint contraction (FP32-SIMT precision):
//   dW[r][k] = sum_lam G[r][lam] SSP[k][lam],  G = dlnL/dY (k young) or dlnL/dO (k old).
// 128 x 64 tile per CTA, 8 x 4 outputs per thread, lambda in steps of 8.
constexpr int DS_M = 128, DS_N = 64, DS_K = 8;

__global__ void __launch_bounds__(256) k_dw_simt(const DwSimtArgs a) {
  pdl_enter();
  __shared__ __align__(16) float As[DS_K][DS_M];
  __shared__ __align__(16) float Bs[DS_K][DS_N];
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int m0 = blockIdx.y * DS_M, n0 = blockIdx.x * DS_N;
  const float* G = n0 < a.Ky_pad ? a.gy : a.go;
  for (int sg = 1; sg < a.n_seg; ++sg)   // age-binned dust: the attenuated block of these columns
    if (n0 >= a.seg_k0[sg] && n0 < a.Ky_pad) G = a.gy + sg * a.seg_stride;
  // the reduction runs over the union of the tile's row windows (G vanishes outside)
  __shared__ int s_klo, s_khi;
  if (tid == 0) { s_klo = 0x7fffffff; s_khi = -1; }
  __syncthreads();
  if (tid < DS_M && m0 + tid < a.n) {
    const RowScal& q = a.rs[m0 + tid];
    if (q.status == 0) { atomicMin(&s_klo, q.k_lo); atomicMax(&s_khi, q.k_hi); }
  }
  __syncthreads();
  if (s_khi < 0) return;
  const int l_begin = s_klo / DS_K * DS_K, l_end = min(a.ldk, (s_khi / DS_K + 1) * DS_K);
  const int lrow = tid >> 1, lk = (tid & 1) * 4;
  float acc[8][4];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
  for (int l0 = l_begin; l0 < l_end; l0 += DS_K) {
    float4 va = make_float4(0.f, 0.f, 0.f, 0.f);
    if (m0 + lrow < a.n) va = *reinterpret_cast<const float4*>(G + (size_t)(m0 + lrow) * a.ldg + l0 + lk);
    As[lk + 0][lrow] = va.x; As[lk + 1][lrow] = va.y; As[lk + 2][lrow] = va.z; As[lk + 3][lrow] = va.w;
    if (tid < 2 * DS_N) {
      const float4 vb = *reinterpret_cast<const float4*>(a.sspK + (size_t)(n0 + lrow) * a.ldk + l0 + lk);
      Bs[lk + 0][lrow] = vb.x; Bs[lk + 1][lrow] = vb.y; Bs[lk + 2][lrow] = vb.z; Bs[lk + 3][lrow] = vb.w;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < DS_K; ++kk) {
      const float4 a0 = *reinterpret_cast<const float4*>(&As[kk][ty * 4]);
      const float4 a1 = *reinterpret_cast<const float4*>(&As[kk][ty * 4 + 64]);
      const float4 b0 = *reinterpret_cast<const float4*>(&Bs[kk][tx * 4]);
      const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      const float bv[4] = {b0.x, b0.y, b0.z, b0.w};
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int gm = m0 + ty * 4 + (i & 3) + (i >> 2) * 64;
    if (gm >= a.n) continue;
    *reinterpret_cast<float4*>(a.dW + (size_t)gm * a.Kpad + n0 + tx * 4) =
        make_float4(acc[i][0], acc[i][1], acc[i][2], acc[i][3]);
  }
}

cudaError_t launch_dw_simt(const DwSimtArgs& a, cudaStream_t s) {
  dim3 grid(a.Kpad / DS_N, (a.n + DS_M - 1) / DS_M);
  return launch_pdl(k_dw_simt, grid, dim3(256), 0, s, a);
}

}  // namespace sed
