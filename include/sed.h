/*
 * sed.h -- C ABI of the GB300 (sm_103a) batched SED forward model and
 * Gaussian log-likelihood.
 *
 * The library evaluates, for a batch of parameter rows theta (the live points
 * of a nested sampler, or any batch), the stellar-population forward model of
 * the paper and its log-likelihood:
 *
 *   SFH + [Fe/H] (+[a/Fe]) history -> SSP weights W      (Sec. 2.2, App. B, Sec. 5.4)
 *   young / old contraction of W with the SSP grid        (Eq. csp_sum_main, Eq. app_attn)
 *   + nebular template scaled by the ionising photons     (App. C, Eq. app_q)
 *   two-component dust attenuation                        (Sec. 2.4)
 *   mass, luminosity distance and (1+z) scaling           (Sec. 2.6)
 *   photometric projection through filter curves         (App. D, Eq. app_phot_row/app_phot_T)
 *   spectral projection with a Gaussian LSF               (Eq. one_kernel, App. E, Eq. app_response)
 *   diagonal Gaussian log-likelihood, normalisation kept  (Eq. total_lnlike, Eq. app_spec_lndiag)
 *
 * Conventions for every entry point:
 *  - Arguments that can be checked on the host are checked before anything is
 *    launched; a failed check returns SED_EINVAL (or SED_ERANGE/SED_EUNSUPPORTED)
 *    and nothing runs.  sed_last_error() then holds a one-line reason.
 *  - Hot-path calls (sed_forward, sed_loglike, sed_loglike_grad) take DEVICE
 *    pointers and a CUDA stream (cudaStream_t passed as void*; NULL = legacy
 *    default stream).  They only enqueue work and return SED_OK; results are
 *    ready when the stream reaches that point.  sed_loglike_host takes HOST
 *    buffers, copies in, runs and copies out, and returns when done.
 *  - Per-row problems found on the device (non-finite parameter, z outside
 *    [0, zf), oldest SFH edge not older than 10 Myr, non-finite model) set the
 *    row's bits in row_status (SED_ROW_*) and write lnL = -INFINITY for it;
 *    the call itself still returns SED_OK.
 *  - Ownership: host arrays passed in descriptors are copied; the caller keeps
 *    ownership and may free them after the call returns.  Device memory owned
 *    by the context (grids, models, per-stream workspaces) is freed by
 *    sed_destroy_model / sed_destroy.  Output buffers belong to the caller.
 *  - Threading: one context may be used from several host threads as long as
 *    each thread uses its own CUDA stream.  The first call on a stream (or with
 *    a larger batch than before on that stream) allocates that stream's
 *    workspace with cudaMalloc, which synchronises the device.
 *  - Memory budget: allocations beyond hbm_budget_bytes return SED_ENOMEM.
 */
#ifndef SED_H
#define SED_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  SED_OK = 0,
  SED_EINVAL = 1,       /* invalid argument or descriptor */
  SED_ENOMEM = 2,       /* HBM budget or cudaMalloc exhausted */
  SED_ECUDA = 3,        /* a CUDA runtime/driver call failed */
  SED_ERANGE = 4,       /* a size exceeds a supported maximum */
  SED_ENONFINITE = 5,   /* non-finite value in a host input */
  SED_EBUSY = 6,        /* object still in use */
  SED_ETIMEOUT = 7,     /* a bounded device wait gave up */
  SED_EUNSUPPORTED = 8  /* feature/precision not available for this model */
} sed_status;

/* Contraction precision (argument `precision`). */
enum {
  SED_PREC_FP32 = 0,      /* tcgen05 tensor cores, 3xTF32 split (FP32-grade) */
  SED_PREC_FP32_SIMT = 1, /* CUDA-core FP32 FFMA (independent cross-check) */
  SED_PREC_BF16 = 2,      /* tcgen05 tensor cores, BF16 operands, FP32 accumulate */
  SED_PREC_FP8 = 3        /* tcgen05 tensor cores, FP8 E4M3 operands with power-of-two scales
                             per SSP column (age, [Fe/H], [a/Fe]) and per row, FP32 accumulate */
};

/* Diffuse dust law (Sec. 2.4). */
enum { SED_DUST_POWER_LAW = 0, SED_DUST_KC13 = 1 };

/* Line-spread-function units (Eq. app_modes). */
enum {
  SED_LSF_R_FWHM = 0, SED_LSF_R_SIGMA = 1, SED_LSF_FWHM_AA = 2,
  SED_LSF_SIGMA_AA = 3, SED_LSF_SIGMA_KMS = 4, SED_LSF_FWHM_KMS = 5
};

/* Row status bits. */
#define SED_ROW_BAD_THETA 1u  /* a parameter is not finite */
#define SED_ROW_BAD_Z 2u      /* zred < 0 or zred >= zf */
#define SED_ROW_BAD_TMAX 4u   /* t_univ(z) - t_univ(zf) <= 10 Myr */
#define SED_ROW_NONFINITE 16u /* model or log-likelihood not finite */
#define SED_ROW_DEVICE_TIMEOUT 32u /* a bounded wait inside a kernel gave up: the call's results are invalid */

/* Parameter keys (paper names, Fig. "ceridwen_flow"); index into the offsets
 * returned by sed_model_layout. */
enum {
  SED_KEY_SFH = 0,            /* N_T formed-mass fractions, bin 0 = most recent (step scheme), or
                                 N_T + 1 SFRs (Msun/yr) at the bin edges, edge 0 = today (linear scheme) */
  SED_KEY_LOGZSOL = 1,        /* N_T per-bin [Fe/H] (zmode 0) or 1 constant (zmode 1) */
  SED_KEY_AFE = 2,            /* [a/Fe] (used when use_afe) */
  SED_KEY_LOGMASS = 3,        /* log10 total formed mass / Msun */
  SED_KEY_ZRED = 4,           /* redshift */
  SED_KEY_TAU_POW = 5,        /* birth-cloud optical depth at 5500 A */
  SED_KEY_ALPHA_POW = 6,      /* birth-cloud power-law slope */
  SED_KEY_DIFFUSE_TAU = 7,    /* diffuse optical depth at 5500 A */
  SED_KEY_DIFFUSE_INDEX = 8,  /* diffuse slope delta (power-law index or KC13 delta) */
  SED_KEY_GAS_LOGZ = 9,       /* log10 Z_gas/Zsun (used when use_nebular) */
  SED_KEY_GAS_LOGU = 10,      /* log10 U (used when use_nebular) */
  SED_KEY_SIGMA_GAL = 11,     /* stellar velocity dispersion, km/s (a column only when sample_sigma_gal) */
  /* systematic noise floor (App. sys_floor, Eq. app_noise_floor), log10 of each
   * term, a column only when the model switches that term on for that arm */
  SED_KEY_LOG_ERR_SCALE_PHOT = 12,  /* s: scale of the formal errors */
  SED_KEY_LOG_F_CALIB_PHOT = 13,    /* f_calib: fraction of |model| */
  SED_KEY_LOG_F_DATA_PHOT = 14,     /* f_data: fraction of |datum| */
  SED_KEY_LOG_JITTER_PHOT = 15,     /* j: additive, in the photometric data's units */
  SED_KEY_LOG_ERR_SCALE_SPEC = 16,
  SED_KEY_LOG_F_CALIB_SPEC = 17,
  SED_KEY_LOG_F_DATA_SPEC = 18,
  SED_KEY_LOG_JITTER_SPEC = 19,     /* j in the spectral data's units */
  SED_KEY_FRAC_OBRUN = 20,    /* runaway fraction f_ob in [0, 1] (a column only with an escape geometry) */
  SED_KEY_SIGMA_GAS = 21,     /* gas velocity dispersion of the emission lines, km/s (a column only when
                                 gas_sigma_mode = SED_GAS_SIGMA_SAMPLED) */
  SED_KEY_DUST_BINS = 22,     /* age-binned attenuation: 2 dust_n_bin columns, each bin's optical depth at
                                 5500 A then its slope (power-law index or KC13 delta) */
  SED_KEY_IGM_FACTOR = 23,    /* scaling of the IGM optical depth (a column only with use_igm) */
  SED_NKEYS = 24
};

typedef struct sed_ctx sed_ctx;
typedef int32_t sed_grid_id;
typedef int32_t sed_model_id;

/*
 * SSP grid (Sec. 2.1): spectra on (age, [Fe/H], [a/Fe]) nodes and a common
 * rest-frame wavelength axis.  All axes strictly increasing, fluxes finite and
 * >= 0.  Copied to the device once (FP32 master, TF32 split and BF16 copies).
 */
typedef struct {
  int n_age, n_feh, n_afe, n_lam;  /* n_afe = 1 for a 3-D grid */
  const double *log_age_yr;        /* [n_age] log10 age / yr */
  const double *feh;               /* [n_feh] log10 Z/Zsun */
  const double *afe;               /* [n_afe] [a/Fe] nodes (NULL allowed when n_afe = 1) */
  const double *lam_aa;            /* [n_lam] rest-frame Angstrom */
  const double *flux;              /* [n_afe][n_feh][n_age][n_lam] Lsun/Hz per Msun formed */
  const double *sigma_lib_kms;     /* [n_lam] documented library LSF, or NULL (Eq. app_siglib) */
  int neb_n_logu, neb_n_logz;      /* nebular template axes (0 = no nebular) */
  const double *neb_logu, *neb_logz;
  const double *neb_log10_lnu_per_q; /* [n_logu][n_logz][n_lam] log10(L_nu/Q), (Lsun/Hz)/(photon/s) */
  /* Operand copies of the grid to keep on the device, as SED_GRID_COPY_* bits
   * (one per precision; 0 = the default: the 3xTF32, FP32 and BF16 copies at
   * load, the FP8 copy on the first FP8 call).  With a mask, only the named
   * precisions are available -- a call in another one returns
   * SED_EUNSUPPORTED -- and a requested FP8 copy is built at load.  Per
   * layout the copies take 8 (3xTF32), 4 (FP32), 2 (BF16) and 1 (FP8) bytes
   * x Kpad x n_lam: a server that runs BF16 only keeps a fifth of the default
   * footprint.  The gradient needs the copy of its precision (3xTF32 or FP32). */
  unsigned precision_mask;
  /* Emission-line cube of the nebular grid (App. C): line luminosity per
   * ionising photon on the same (log U, log Z_gas) axes as the continuum
   * template, kept apart from the continuum (Sec. 2.5): 0 lines = none. */
  int neb_n_line;
  const double *neb_line_lam_aa;       /* [n_line] rest-frame wavelengths, Angstrom */
  const double *neb_log10_line_per_q;  /* [n_logu][n_logz][n_line] log10(L_line/Q), Lsun/(photon/s) */
  /* Nebular age axis (App. C): neb_n_age > 0 gives the continuum cube an
   * ionising-source age axis, neb_log10_lnu_per_q then being
   * [neb_n_age][n_logu][n_logz][n_lam] on the increasing log10 ages
   * neb_log_age_yr.  The cube is queried at each SSP age inside its tabulated
   * ages (linear in log age between its planes, bilinear in log U and
   * log Z_gas): those SSP ages, at most 32 and all within a model's
   * birth-cloud ages (else SED_EUNSUPPORTED at model creation), power the
   * nebular emission with their own Q.  Not combined with a line cube
   * (SED_EUNSUPPORTED), nor, in a model, with an escape geometry or
   * age-binned dust; not served by sed_server_* or sed_loglike_noalloc. */
  int neb_n_age;
  const double *neb_log_age_yr;
} sed_grid_desc;

#define SED_GRID_COPY_FP32 (1u << SED_PREC_FP32)           /* TF32 hi/lo parts (3xTF32 path) */
#define SED_GRID_COPY_FP32_SIMT (1u << SED_PREC_FP32_SIMT) /* exact FP32 (FFMA path) */
#define SED_GRID_COPY_BF16 (1u << SED_PREC_BF16)
#define SED_GRID_COPY_FP8 (1u << SED_PREC_FP8)

/*
 * One fit: model choices, observations and their uncertainties (Sec. 2, 3, 4.1).
 * Filters are concatenated: band b has filt_len[b] samples (Angstrom, observed
 * frame) with transmission filt_trans.  Photometric data and uncertainties are
 * in maggies; spectral data in cgs F_nu on observed-frame pixels spec_lam_aa.
 * n_filt or n_pix may be 0 (arm absent).  Masks may be NULL (all included).
 */
typedef struct {
  sed_grid_id grid;
  int n_sfh;                  /* N_T >= 3: edges 0, 5 Myr, 10 Myr, log-uniform to t_univ(z)-t_univ(zf) */
  double zf;                  /* formation redshift of the oldest edge */
  int zmode;                  /* 0: one [Fe/H] per SFH bin; 1: one constant [Fe/H] */
  int use_afe;                /* interpolate the [a/Fe] axis (else [a/Fe] = 0) */
  int use_nebular;            /* add the nebular template (grid must carry one) */
  int dust_law;               /* SED_DUST_POWER_LAW or SED_DUST_KC13 (diffuse component) */
  double bc_edge_log_age_yr;  /* birth-cloud edge; paper default log10(age/Gyr) = -1.97 -> 7.03 */
  double H0, Om0;             /* flat LCDM, km/s/Mpc */
  int n_filt;
  const int *filt_len;
  const double *filt_lam_aa, *filt_trans;
  const double *phot_d, *phot_sigma;
  const uint8_t *phot_mask;
  int n_pix;
  const double *spec_lam_aa, *spec_d, *spec_sigma;
  const uint8_t *spec_mask;
  int lsf_mode;               /* SED_LSF_* */
  const double *lsf_value;    /* [n_pix] value in the unit of lsf_mode */
  double sigma_gal_kms;       /* fixed stellar dispersion folded into the LSF kernel */
  double z_ref;               /* reference redshift of the projector (Eq. app_sigeff) */
  /* Sampled stellar dispersion (Sec. 2.7 kinematics; App. E): with
   * sample_sigma_gal = 1 each parameter row carries sigma_gal (km/s) in column
   * offsets[SED_KEY_SIGMA_GAL] instead of the fixed sigma_gal_kms; a row whose
   * value lies outside [0, sigma_gal_max_kms] gets SED_ROW_BAD_THETA.  The
   * maximum bounds the spectral kernels' reach (shared-memory window sizes). */
  int sample_sigma_gal;
  double sigma_gal_max_kms;
  /* Marginalised calibration polynomial (App. E, Eq. app_polymarg): the
   * spectrum's model is mu_i (1 + sum_m c_m T_m(x_i)), T_m Chebyshev
   * polynomials of the pixel wavelengths mapped linearly onto [-1, 1] (first
   * and last pixel), with c_m ~ N(0, calib_sigma[m]^2) integrated out of lnL in
   * closed form.  calib_n = number of coefficients (0: none, at most
   * SED_MAX_CALIB); calib_sigma [calib_n] > 0.  Needs a spectrum.  Model
   * spectra returned by sed_forward stay uncalibrated (mu). */
  int calib_n;
  const double *calib_sigma;
  /* Systematic noise floor (App. sys_floor, Eq. app_noise_floor), per arm: each
   * datum's variance becomes sigma_eff^2 = s^2 sigma^2 + (f_calib |m|)^2 +
   * (f_data |d|)^2 + j^2 and its lnL term -r^2/(2 sigma_eff^2) -
   * ln(2 pi sigma_eff^2)/2, with m the model and d the datum.  A SED_FLOOR_*
   * bit switches a term on and gives it a parameter column (key
   * SED_KEY_LOG_*_PHOT / _SPEC) holding log10 of its value; a term that is off
   * leaves s = 1, the others 0.  0 = the plain Gaussian (the default).  A
   * spectral floor needs a spectrum and no calibration polynomial
   * (SED_EUNSUPPORTED); a photometric one needs filters. */
  int noise_floor_phot, noise_floor_spec;
  /* SFH -> SSP age weights (App. B): SED_SFH_STEP (0, the default) spreads
   * each bin's mass m_i over the age nodes by linear-time Voronoi overlap;
   * SED_SFH_LINEAR (1) takes the SFR linear in lookback time across each bin
   * through per-edge rates psi_0..psi_NT and integrates it against the nodes'
   * log-age tents (Eq. tent_integral), pieces clipped at 0 and each bin scaled
   * to its trapezoidal mass max(0, (psi_i + psi_{i+1}) dT_i / 2).  The linear
   * scheme has N_T + 1 SFH columns, and sed_loglike_grad returns d lnL / d psi
   * for each edge. */
  int sfh_scheme;
  /* Photometric upper limits (Sec. 4.1 likelihood, App. line_lik, Eq.
   * app_line_chi2_UL): [n_filt], nonzero marks phot_d[b] as an upper limit.
   * Such a band adds ((d - m)/sigma_eff)^2 to chi^2 only while its model m
   * exceeds the limit d and nothing while m <= d; its -1/2 ln(2 pi
   * sigma_eff^2) stays in lnL, with sigma_eff of the noise floor when one is
   * on.  NULL = no limits (the default).  Copied; a band the mask excludes
   * stays out of lnL whatever its flag. */
  const uint8_t *phot_upper;
  /* Ionising-photon escape (Sec. frac_obrun): SED_FESC_NONE (0, the default),
   * SED_FESC_RUNAWAY_BC (Eq. runaway_mix: the young light, stellar and
   * nebular continuum, crosses (1 - f_ob) e^{-tau_BC} + f_ob, then the
   * diffuse screen) or SED_FESC_PICKET (a fraction f_ob of the young stellar
   * light escapes both screens, the rest crosses both).  Either way only the
   * covered fraction 1 - f_ob powers the nebular continuum, and the fraction
   * f_ob of the nebular ages' ionising continuum (below 912 A) escapes instead
   * of being absorbed, bypassing the birth cloud.  A geometry adds the column
   * SED_KEY_FRAC_OBRUN; a row whose f_ob lies outside [0, 1] gets
   * SED_ROW_BAD_THETA.  With f_ob = 0 the model is the one without a geometry. */
  int fesc_geometry;
  /* Fixed and sampled keys (the paper's parameter dictionary, Sec. 4: each
   * key is either sampled or fixed at a value): fixed[k] != 0 fixes key k at
   * fixed_val[k] for every row, and the key then has no column in the
   * parameter rows (sed_model_layout gives it zero width) and no gradient.
   * Only one-column keys can be fixed: logzsol with one constant [Fe/H]
   * (zmode 1), afe, logmass, zred, the dust and gas keys, and sigma_gal, the
   * noise-floor terms and f_ob where the model samples them; SED_EINVAL
   * otherwise, or for a non-finite value.  A fixed value goes through the same
   * per-row checks as a column (e.g. zred outside [0, zf) marks every row).
   * All zero (the default) = every key sampled. */
  int fixed[SED_NKEYS];
  double fixed_val[SED_NKEYS];
  /* How the calibration polynomial (calib_n > 0) enters lnL (App. E):
   * SED_CALIB_MARGINAL (0, the default) integrates the coefficients out
   * (Eq. app_polymarg); SED_CALIB_OPTIMISED (1) takes at every evaluation the
   * coefficients that maximise the spectrum's lnL plus their log prior (the
   * weighted least-squares fit regularised by 1/calib_sigma; very wide
   * calib_sigma give the unregularised fit), i.e. lnL gains b^T M^-1 b / 2
   * and not the Occam terms -ln|M|/2 - ln|Lambda|/2. */
  int calib_mode;
  /* Emission lines (App. C, App. line_proj; needs use_nebular and a grid with
   * a line cube): each line's flux, L = Q_young 10^(bilinear log10 cube) through
   * the nebular attenuation at its wavelength, times 10^logmass Lsun /
   * (4 pi D_L^2), enters the photometry as F R_b(lam_obs) lam_obs / Z_b and
   * the spectrum as a unit-area Gaussian in ln(lambda) of width
   * sqrt(sigma_gas^2 + sigma_inst^2(lam_obs)) / c sampled at the pixels
   * (Eq. app_line_profile; sigma_inst interpolated linearly in wavelength
   * between the pixels' LSF).  sigma_gas: SED_GAS_SIGMA_TIED to the stellar
   * sigma_gal (fixed or sampled), SED_GAS_SIGMA_FIXED at sigma_gas_kms, or
   * SED_GAS_SIGMA_SAMPLED as the column SED_KEY_SIGMA_GAS in
   * [0, sigma_gas_max_kms] (else SED_ROW_BAD_THETA). */
  int use_lines;
  int gas_sigma_mode;
  double sigma_gas_kms, sigma_gas_max_kms;
  /* Line catalogue arm (Sec. 3.3 "Lines", App. line_lik; needs use_lines):
   * n_lcat entries, entry k the blend of lcat_len[k] grid lines listed in
   * lcat_line (concatenated), observed integrated flux lcat_d[k] and error
   * lcat_sigma[k] in erg/s/cm^2; the model is the blend's summed flux (no
   * profile); detections add -((d - m)/sigma)^2/2 - ln(2 pi sigma^2)/2, an
   * entry flagged in lcat_upper (may be NULL) adds the residual only while
   * m > d (Eq. app_line_chi2_UL); lcat_mask (may be NULL) excludes entries. */
  int n_lcat;
  const int *lcat_len, *lcat_line;
  const double *lcat_d, *lcat_sigma;
  const uint8_t *lcat_mask, *lcat_upper;
  /* Age-binned attenuation (App. dust_attn, Eq. app_tau_bin): dust_n_bin > 0
   * replaces the birth-cloud power law by dust_n_bin laws over the SSP age
   * axis.  dust_bin_M [n_age][dust_n_bin] is the age-to-bin matrix: each row
   * in [0, 1] summing to 1 (a node in one bin, or shared between overlapping
   * bins) or all zero (no bin: the node sees the diffuse screen only); the
   * optical depth at age node a is tau_a = sum_b M_ab kappa_b(lambda), with
   * kappa_b of law dust_bin_law[b] (SED_DUST_POWER_LAW: tau_b (lam/5500)^s_b;
   * SED_DUST_KC13: the Kriek & Conroy form of the diffuse component with
   * delta = s_b), and it attenuates the node's stellar and nebular light before
   * the diffuse screen.  The columns SED_KEY_DUST_BINS hold (tau_b, s_b) per
   * bin; tau_pow and alpha_pow keep their columns and are not read.  The ages
   * sharing one non-zero row form one of the contraction's attenuated blocks
   * (at most SED_MAX_DUST_SEG distinct non-zero rows).  Not combined with emission
   * lines or an escape geometry (SED_EUNSUPPORTED), nor served by sed_server_*
   * or sed_loglike_noalloc. */
  int dust_n_bin;
  const double *dust_bin_M;
  const int *dust_bin_law;
  /* IGM transmission (Sec. 2.6): SED_IGM_MADAU multiplies the rest-frame model
   * at each node, and each emission line, by exp(-f tau(lam_obs, z)), tau the
   * Madau (1995) mean optical depth (Lyman-series blanketing, Ly-alpha to
   * Ly-delta, and Lyman-limit photoelectric absorption), f the column
   * SED_KEY_IGM_FACTOR (fix it at 1 for the plain prescription).  Applied to
   * the nodes before the spectral kernel. */
  int use_igm;
} sed_model_desc;

#define SED_IGM_NONE 0
#define SED_IGM_MADAU 1

#define SED_MAX_DUST_BIN 4
#define SED_MAX_DUST_SEG 4

#define SED_GAS_SIGMA_TIED 0
#define SED_GAS_SIGMA_FIXED 1
#define SED_GAS_SIGMA_SAMPLED 2

#define SED_CALIB_MARGINAL 0
#define SED_CALIB_OPTIMISED 1

#define SED_MAX_CALIB 13
#define SED_FESC_NONE 0
#define SED_FESC_RUNAWAY_BC 1
#define SED_FESC_PICKET 2
#define SED_SFH_STEP 0
#define SED_SFH_LINEAR 1
#define SED_FLOOR_ERR_SCALE 1
#define SED_FLOOR_F_CALIB 2
#define SED_FLOOR_F_DATA 4
#define SED_FLOOR_JITTER 8

/* Context on one CUDA device; hbm_budget_bytes = 0 means no limit. */
sed_status sed_create(sed_ctx **out, int device, size_t hbm_budget_bytes);
sed_status sed_destroy(sed_ctx *ctx);
const char *sed_status_string(sed_status s);
/* One-line description of the last error on this context (never NULL). */
const char *sed_last_error(const sed_ctx *ctx);
/* Device bytes currently held by the context. */
sed_status sed_memory_used(const sed_ctx *ctx, size_t *bytes);
/* How the last sed_loglike_host call on this context ran: bit 0 set = theta
 * was read in place, bit 1 set = lnl_out was written in place (both
 * page-locked and device-mapped), 0 = both were staged; bit 2 set = the call
 * replayed a CUDA graph of its launches.  Only valid once such a call has
 * returned SED_OK. */
sed_status sed_last_host_path(const sed_ctx *ctx, int *mapped);

sed_status sed_load_grid(sed_ctx *ctx, const sed_grid_desc *desc, sed_grid_id *out);

sed_status sed_create_model(sed_ctx *ctx, const sed_model_desc *desc, sed_model_id *out);
/* n_param: columns a parameter row needs; offsets[SED_NKEYS]: first column of each key (a key
 * without a column -- unused option or fixed -- has the next key's offset, i.e. zero width). */
sed_status sed_model_layout(const sed_ctx *ctx, sed_model_id model, int *n_param, int *offsets);
/* Replace the observed data/uncertainties of a model (host arrays, copied).  Data and
 * sigma come in pairs (both or neither, else SED_EINVAL); a pair passed as NULL keeps
 * its last value, and a block never given stays out of lnL.  Every datum is checked
 * before anything changes (SED_EINVAL: sigma <= 0 or a non-finite value; spectral
 * 1/sigma and d/sigma outside FP32's normal range, which the kernels work in). */
sed_status sed_set_data(sed_ctx *ctx, sed_model_id model, const double *phot_d,
                        const double *phot_sigma, const double *spec_d, const double *spec_sigma);
sed_status sed_destroy_model(sed_ctx *ctx, sed_model_id model);

/*
 * Forward model: photometry phot_out [n][n_filt] in maggies and/or the
 * projected spectrum spec_out [n][n_pix] in cgs F_nu (either may be NULL).
 * theta: device, row-major [n][ld] FP32 with ld >= n_param.  0 <= n.
 */
sed_status sed_forward(sed_ctx *ctx, sed_model_id model, const float *theta, int n, int ld,
                       float *phot_out, float *spec_out, int precision, void *stream);

/*
 * Log-likelihood lnl_out [n] (FP64, device) and optional row_status [n]
 * (device, may be NULL).  Eq. total_lnlike with the normalisation term kept.
 */
sed_status sed_loglike(sed_ctx *ctx, sed_model_id model, const float *theta, int n, int ld,
                       double *lnl_out, uint32_t *row_status, int precision, void *stream);

/*
 * Log-likelihood and its gradient with respect to every parameter column:
 * grad_out [n][ld] (FP32, device; columns >= n_param are zeroed).  Columns the
 * model does not use (e.g. gas_* without nebular, afe without use_afe) get 0;
 * rows with a non-zero row_status get an all-zero gradient row.
 * The gradient is the analytic derivative of the forward model (the paper
 * differentiates it automatically, Sec. 4): a hand-written reverse pass that
 * recomputes the per-row spectrum from the contraction output, forms
 * dlnL/dY and dlnL/dO, contracts them with the SSP grid for dlnL/dW (the
 * transpose of Eq. csp_sum_main) and maps dlnL/dW back through the step-scheme
 * weights, the metallicity / [a/Fe] splits and the SFH edges (App. B) to the
 * parameters.  At a kink (an interpolation node, a bracket node, a Voronoi
 * cell edge) the one-sided derivative of the branch the forward took is
 * returned.
 * precision: SED_PREC_FP32 (3xTF32 tensor-core contractions) or
 * SED_PREC_FP32_SIMT; SED_PREC_BF16 and SED_PREC_FP8 return SED_EUNSUPPORTED.
 * The first gradient call on a grid layout builds its lambda-major copies
 * (host work and synchronous copies to the device, ~3 x 4 x Kpad x n_lam
 * bytes); later calls only enqueue kernels.  SED_ERANGE when the adjoint
 * epilogue's shared-memory staging (8 n_lam + max(8 filter samples, 20 n_pix)
 * bytes) exceeds 227 KB.
 */
sed_status sed_loglike_grad(sed_ctx *ctx, sed_model_id model, const float *theta, int n, int ld,
                            double *lnl_out, float *grad_out, uint32_t *row_status,
                            int precision, void *stream);

/*
 * Observer-frame integrated fluxes of the grid's emission lines (App. C, App.
 * line_proj), erg/s/cm^2, for a model with use_lines: flux_out is a DEVICE
 * buffer [n][neb_n_line] (row-major, the grid's line order), the quantities
 * the line catalogue's entries sum (Sec. 3.3).  Rows with a non-zero status
 * get zeros.  SED_EUNSUPPORTED for a model without lines; otherwise as
 * sed_forward (asynchronous on `stream`).
 */
sed_status sed_line_fluxes(sed_ctx *ctx, sed_model_id model, const float *theta, int n, int ld, float *flux_out,
                           int precision, void *stream);

/*
 * sed_loglike with HOST buffers: theta [n][ld] FP32, lnl_out [n], row_status
 * [n] or NULL.  Runs on `stream` and synchronises the stream before
 * returning.  A page-locked host buffer that the device can address (memory
 * from cudaHostAlloc / cudaMallocHost, or cudaHostRegister'ed, on a 64-bit
 * unified-address system) is used in place: the kernels read theta and write
 * lnl_out / row_status over the host link (NVLink-C2C on a Grace host), so no
 * separate copy sits on the call's critical path.  Any other buffer is staged
 * through device memory with an asynchronous copy.  With every buffer used in
 * place and a non-NULL stream (not while profiling), the second call with the
 * same model, buffers, n, ld and precision captures the call's launches into
 * a CUDA graph, kept with the stream's workspace, and later such calls replay
 * it; the buffers' contents and the model's data may change between calls.
 * The result is the same on every path, bit for bit.  ld <= 1024.
 */
sed_status sed_loglike_host(sed_ctx *ctx, sed_model_id model, const float *theta, int n, int ld,
                            double *lnl_out, uint32_t *row_status, int precision, void *stream);

/*
 * sed_loglike without any device allocation by the library.  (An addition of
 * this library; the paper has no counterpart.)
 *
 * For callers that cannot let the library call cudaMalloc during a call: a
 * host framework whose own allocator already owns the GPU's memory, a
 * sampler loop that cannot absorb the device synchronisation a cudaMalloc
 * may cause, or a deployment that must fix the library's device footprint
 * when it is loaded.  Same arguments, row-status semantics and kernels as
 * sed_loglike (device pointers, asynchronous on `stream`; the same row
 * order, wavelength windows and contraction schedule, so the same results),
 * but every intermediate buffer comes from one fixed array of
 * SED_NOALLOC_SCRATCH_BYTES in device global memory that each device loading
 * the library holds until the process exits; no cudaMalloc, cudaFree or
 * allocating library routine is called.
 *  - Precisions: SED_PREC_FP32, SED_PREC_FP32_SIMT and SED_PREC_BF16.
 *    SED_PREC_FP8 returns SED_EUNSUPPORTED: its copy of the grid is built by
 *    an allocation on the first FP8 call of sed_loglike.
 *  - Limit: the scratch a call needs grows with n: per row 3 x 4 x ldn bytes
 *    for SED_PREC_FP32 (2 x 4 x ldn otherwise; ldn = n_lam rounded up to
 *    256) plus 8 x Kpad (FP32), 2 x Kpad (BF16) or 4 x Kpad (FP32_SIMT) and
 *    about 250 bytes of row scalars -- about 390 rows of a 107 x 12 x 6000
 *    grid in FP32, thousands for small grids.  A call needing more than
 *    SED_NOALLOC_SCRATCH_BYTES returns SED_ERANGE with the sizes in
 *    sed_last_error() and launches nothing.  Split larger batches.
 *  - The array is shared by all calls and keeps the contents of the last
 *    one: calls that can overlap on the GPU (other streams or threads) race
 *    on it and must be serialised by the caller.
 *  - The first call on a device looks up the array's device address
 *    (cudaGetSymbolAddress); make that first call before any stream capture.
 */
#define SED_NOALLOC_SCRATCH_BYTES (32u * 1024u * 1024u)
sed_status sed_loglike_noalloc(sed_ctx *ctx, sed_model_id model, const float *theta, int n, int ld,
                               double *lnl_out, uint32_t *row_status, int precision, void *stream);

/*
 * Continuous-batching server of log-likelihood calls (the serving pattern of
 * the library; the paper runs one fit per GPU).  Many fits -- each a model
 * created with sed_create_model, i.e. its own filters, spectrum, data and SFH
 * layout -- share one HBM-resident SSP grid.  A fit owns a device buffer of
 * live points (max_rows x n_param FP32).  Clients submit calls (the first n
 * rows of a fit) at any time; a scheduler thread packs the pending calls of
 * all fits, first come first served, into launches of up to max_launch_rows
 * rows, with up to n_slots launches in flight on their own streams, so calls
 * that arrive while others run are taken into the next free slot and their
 * work overlaps on the device.  Each row reads its own fit's model in the
 * kernels, and no row's arithmetic depends on the other rows of a launch: a
 * call's result equals sed_loglike on the same rows, alone or in any mix.
 *  - sed_server_create: all fits must use the grid layout of `model_layout`
 *    (same grid, birth-cloud edge and nebular setting).  Allocates the
 *    launch buffers of every slot up front; SED_ENOMEM on failure.
 *  - sed_server_open_fit: admission by device memory: reserves the fit's
 *    live-point buffer against fit_budget_bytes (0 = no server limit; the
 *    context budget still applies) and returns SED_EBUSY when it does not
 *    fit now (retry after another fit closes).  max_rows <= max_launch_rows.
 *  - sed_server_submit: copies n host rows (stride ld >= n_param) into the
 *    fit's live points and queues the call; the caller may reuse its buffer
 *    at once.  sed_server_submit_device queues a call on the live points
 *    already in the fit's device buffer (sed_server_fit_theta; writes to it
 *    must be complete, e.g. their stream synchronised, before the submit).
 *    One call per fit at a time (SED_EBUSY otherwise).
 *  - sed_server_wait: blocks until the call is done (timeout_ms < 0: no
 *    limit; SED_ETIMEOUT otherwise) and copies lnL [n] / row status [n] to
 *    host buffers (either may be NULL); latency_ms (may be NULL) receives the
 *    time from submit to the results being on the host.  Each ticket is
 *    waited for once.
 *  - sed_server_close_fit waits for the fit's call in flight, then releases
 *    its buffers; sed_server_destroy lets the launches in flight finish.
 * Thread-safe: submit / wait / open / close may be called from many threads.
 */
typedef struct sed_server sed_server;
typedef struct {
  sed_grid_id grid;
  sed_model_id model_layout;  /* a model whose grid layout every fit shares */
  int precision;              /* SED_PREC_* of every launch */
  int max_launch_rows;        /* rows packed into one launch */
  int n_slots;                /* launches in flight at once, 1..8 */
  size_t fit_budget_bytes;    /* device memory for the fits' live points (0 = no limit) */
} sed_server_desc;
typedef struct {
  uint64_t calls, launches, rows;  /* completed calls, issued launches and their rows */
  int fits_open;
  size_t fit_bytes;                /* device bytes held by open fits */
} sed_server_stats;
sed_status sed_server_create(sed_ctx *ctx, const sed_server_desc *desc, sed_server **out);
sed_status sed_server_destroy(sed_server *server);
sed_status sed_server_open_fit(sed_server *server, sed_model_id model, int max_rows, int *fit);
sed_status sed_server_close_fit(sed_server *server, int fit);
float *sed_server_fit_theta(sed_server *server, int fit);
sed_status sed_server_submit(sed_server *server, int fit, const float *theta_host, int n, int ld,
                             uint64_t *ticket);
sed_status sed_server_submit_device(sed_server *server, int fit, int n, uint64_t *ticket);
sed_status sed_server_wait(sed_server *server, uint64_t ticket, double *lnl_host, uint32_t *status_host,
                           int timeout_ms, double *latency_ms);
sed_status sed_server_get_stats(sed_server *server, sed_server_stats *out);

/*
 * Per-stage timing and work counters of the last hot-path call on a stream.
 * With profiling on, each hot-path call records CUDA events on its stream
 * before and after each of its kernels (preparation, contraction, epilogue;
 * for sed_loglike_grad the epilogue is the adjoint epilogue, followed by the
 * dW contraction and the weights' reverse pass); sed_last_stats synchronises
 * on the last event and reads them.  nnz_w is the number of non-zero SSP
 * weights of the call's rows (the contraction's algorithmic work is
 * 2 * nnz_w * n_lam FLOPs).
 */
typedef struct {
  float ms_prep, ms_contract, ms_epilogue;
  double nnz_w;          /* sum over rows of the non-zero weights W[theta][k] */
  double dense_k;        /* padded K of the contraction (young + old) */
  double issued_flop;    /* tensor (or FFMA) FLOPs the contraction issued over its computed tiles
                            (x3 for the 3xTF32 split) */
  int n_rows, n_lam, ldn, precision;
  int is_grad;           /* 1 if the call was sed_loglike_grad */
  float ms_dw, ms_prep_bwd;  /* gradient calls: dW = G SSP^T contraction, weights / edges / cosmology reverse pass */
} sed_stage_stats;

sed_status sed_set_profiling(sed_ctx *ctx, int on);
sed_status sed_last_stats(sed_ctx *ctx, void *stream, sed_stage_stats *out);

/*
 * Nested slice sampling (Sec. 4.3): a nested-sampling run (Skilling 2006) on
 * the GPU whose likelihood is sed_loglike of one model.  The live points start
 * uniform in a box prior (one interval per parameter column: lo[j] < hi[j]);
 * each iteration removes the n_replace live points of lowest lnL and replaces
 * them by as many hit-and-run slice chains, run in parallel, each started at a
 * random surviving live point with lnL above the removed ones and making
 * n_slice_steps slice steps inside the likelihood contour (stepping out, then
 * shrinking) along directions drawn from the surviving live points'
 * covariance.  Every chain's proposals of one round go through one
 * sed_loglike call; the proposals, the contour, the covariance and its
 * Cholesky factor, the evidence sums and the stop test run in the library's
 * kernels, the host only sequences the rounds.  Random numbers: Philox4x32-10
 * keyed by seed.  The prior volume after removing the j-th of the n live
 * points of lowest lnL shrinks by exp(-1 / (n - j)) (the expectation of the log
 * shrinkage); the removed point's weight is X_before - X_after.  The run stops
 * when ln(Z_live / Z) < stop_dlnz, Z_live = X * mean(L_live) (the paper: -5),
 * or after max_iter iterations; the final live points are then added with
 * weight X / n each.
 */
typedef struct {
  int n_live;              /* live points, 2 <= n_live <= 4096 */
  int n_replace;           /* live points replaced per iteration, 1 <= n_replace <= n_live / 2 */
  int n_slice_steps;       /* slice steps per replacement chain, >= 1 */
  int max_iter;            /* iteration limit, >= 1 */
  double stop_dlnz;        /* stop when ln(Z_live / Z) < stop_dlnz */
  double slice_width;      /* initial slice bracket, in units of the live points' spread along the
                              direction (0 = sqrt(n_param + 2)) */
  uint64_t seed;
  int precision;           /* SED_PREC_* of the likelihood calls */
  const double *lo, *hi;   /* [n_param] HOST: the box prior of each parameter column */
} sed_nss_desc;

typedef struct {
  double lnz;              /* ln of the evidence (the mean likelihood over the box prior) */
  double info_h;           /* information H = sum_i p_i ln(L_i / Z), nats; ln Z's spread is ~ sqrt(H / n_live) */
  int n_iter;              /* iterations run */
  int n_dead;              /* points returned: every removed point, then the final live points */
  int converged;           /* 1: the stop test was met; 0: max_iter was reached */
  int64_t n_like;          /* likelihood evaluations of proposals */
  int64_t n_rows;          /* rows sent through sed_loglike (idle chains included) */
} sed_nss_result;

/*
 * Runs nested slice sampling for `model` on `stream` and waits for it.  The
 * host buffers (each may be NULL) receive, for max_dead points at most, in
 * the order of removal and then the final live points in increasing lnL: the
 * parameter rows dead_theta [max_dead][n_param], their lnL dead_lnl, their
 * log posterior weights dead_logw (ln(L_i w_i / Z), summing to 1 in exp), and
 * ins_rank [max_dead] the insertion rank of each replacement among the live
 * points that survived its iteration (n_iter * n_replace entries; uniform on
 * 0..n_live - n_replace for a correct constrained sampler).  SED_ERANGE when
 * max_dead is below the points the run produced (the run's results are still
 * in *out); SED_EINVAL for a bad descriptor; the library allocates and frees
 * the run's device buffers.
 */
sed_status sed_nss_run(sed_ctx *ctx, sed_model_id model, const sed_nss_desc *desc, float *dead_theta,
                       double *dead_lnl, double *dead_logw, int32_t *ins_rank, int max_dead,
                       sed_nss_result *out, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* SED_H */
