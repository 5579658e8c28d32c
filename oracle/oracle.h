/*
 * FP64 CPU oracle of the batched SED forward model and Gaussian log-likelihood.
 *
 * TEST INFRASTRUCTURE ONLY.  This code is the independent reference that the
 * GPU library is checked against.  It shares no code, header, table or
 * constant with the library; only the test suite, the smoke check and the CPU
 * baseline of the benchmark may load it.  The product path never calls it.
 *
 * Each function follows the paper's definitions directly, in the plainest loop
 * order, in double precision:
 *   cosmology            Sec. 2.6 (flat LCDM luminosity distance, age of the Universe)
 *   SFH -> SSP weights   Sec. 2.2, App. B (step scheme, Voronoi cells in linear time; linear
 *                        scheme, Eq. "tent_integral"),
 *                        App. B metallicity split, Sec. 5.4 [a/Fe] axis
 *   ionising photons     App. C, Eq. "app_q"
 *   contraction          Eq. "csp_sum_main", Eq. "app_attn" (two age bins)
 *   nebular              App. C (template interpolated in log10, scaled by Q)
 *   dust                 Sec. 2.4 (birth-cloud power law + diffuse law)
 *   observer frame       Sec. 2.6 (mass, flux factor (1+z)(10pc/D_L)^2)
 *   photometry           App. D, Eqs. "app_phot_row", "app_phot_T"
 *   spectrum             Eq. "one_kernel", App. E, Eqs. "app_siglib", "app_sigeff", "app_response"
 *   likelihood           Eq. "total_lnlike", Eq. "app_spec_lndiag", the optional
 *                        noise floor of App. "sys_floor", Eq. "app_noise_floor"
 *   gradient             the chain rule through all of the above (the paper takes its
 *                        gradients by automatic differentiation, Sec. 4)
 */
#ifndef SED_ORACLE_H
#define SED_ORACLE_H
#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  int n_age, n_feh, n_afe, n_lam;
  const double *log_age_yr, *feh, *afe, *lam; /* lam: rest frame, Angstrom */
  const double *flux;          /* [n_afe][n_feh][n_age][n_lam], Lsun/Hz per Msun formed */
  const double *sigma_lib_kms; /* [n_lam] documented library LSF, or NULL */
  int neb_n_logu, neb_n_logz;
  const double *neb_logu, *neb_logz;
  const double *neb_tab;       /* [n_logu][n_logz][n_lam] log10(L_nu/Q), or NULL */
  int neb_n_line;              /* emission lines of the nebular grid (App. C), 0: none */
  const double *neb_line_lam;  /* [n_line] rest-frame wavelength, Angstrom */
  const double *neb_line_tab;  /* [n_logu][n_logz][n_line] log10(L_line/Q), Lsun / (photon/s) */
  int neb_n_age;               /* nebular age axis (App. C), 0: none; with one, neb_tab is
                                  [n_age][n_logu][n_logz][n_lam] on the ionising-source ages neb_log_age */
  const double *neb_log_age;   /* [neb_n_age] log10 age / yr, increasing */
} orc_grid;

typedef struct {
  int n_sfh;                   /* SFH bins N_T (>= 3) */
  double zf;                   /* formation redshift of the oldest edge */
  int zmode;                   /* 0: one [Fe/H] per bin, 1: one constant [Fe/H] */
  int use_afe, use_nebular;
  int dust_law;                /* diffuse law: 0 power law, 1 Kriek & Conroy 2013 */
  double bc_edge_log_age_yr;   /* ages <= this are in the birth cloud */
  double H0, Om0;              /* flat LCDM, H0 in km/s/Mpc */
  int n_filt;
  const int *filt_len;
  const double *filt_lam, *filt_trans;      /* concatenated, Angstrom */
  const double *phot_d, *phot_sigma;        /* maggies */
  const unsigned char *phot_mask;
  int n_pix;
  const double *spec_lam, *spec_d, *spec_sigma; /* observed frame, cgs F_nu */
  const unsigned char *spec_mask;
  int lsf_mode;                /* 0 R_fwhm, 1 R_sigma, 2 fwhm_aa, 3 sigma_aa, 4 sigma_kms, 5 fwhm_kms */
  const double *lsf_value;     /* [n_pix] */
  double sigma_gal_kms, z_ref;  /* fixed stellar dispersion (when not sampled), projector redshift */
  int sample_sigma_gal;        /* 1: sigma_gal (km/s) is a parameter column (Sec. 2.7 kinematics) */
  double sigma_gal_max_kms;    /* sampled sigma_gal must lie in [0, this] */
  int calib_n;                 /* coefficients of the marginalised calibration polynomial (0: none) */
  const double *calib_sigma;   /* [calib_n] prior widths s_m of the coefficients (App. E) */
  int sfh_scheme;              /* 0 step (per-bin masses m_i, N_T columns), 1 linear (per-edge SFRs psi_i,
                                  N_T + 1 columns; App. B, Eq. "tent_integral") */
  int floor_phot, floor_spec;  /* systematic noise floor of each arm (App. "sys_floor"): ORC_FLOOR_* bits;
                                  each term on adds a parameter column holding log10 of its value */
  const unsigned char *phot_upper; /* [n_filt] nonzero: phot_d[b] is an upper limit (Sec. 4.1 likelihood,
                                      Eq. "app_line_chi2_UL"), or NULL (none) */
  int fesc_geometry;           /* ionising-photon escape (Sec. "frac_obrun"): ORC_FESC_*; with a geometry the
                                  row's last column is the runaway fraction f_ob in [0, 1] */
  int calib_mode;              /* ORC_CALIB_MARGINAL (Eq. "app_polymarg") or ORC_CALIB_OPTIMISED (the
                                  polynomial optimised at each call, Sec. 3.2 / App. E) */
  int use_lines;               /* 1: the grid's emission lines (App. C, App. "line_proj") enter the
                                  photometry and the spectrum (needs use_nebular) */
  int gas_sigma_mode;          /* ORC_GAS_SIGMA_*: the gas dispersion sigma_gas of the line profiles */
  double sigma_gas_kms;        /* ORC_GAS_SIGMA_FIXED: its value */
  double sigma_gas_max_kms;    /* ORC_GAS_SIGMA_SAMPLED: the column must lie in [0, this] */
  int n_lcat;                  /* entries of the line-catalogue arm (Sec. 3.3 "Lines"), 0: none */
  const int *lcat_start;       /* [n_lcat + 1]: entry k is the blend of grid lines
                                  lcat_line[lcat_start[k] .. lcat_start[k + 1]) */
  const int *lcat_line;
  const double *lcat_d, *lcat_sigma;   /* observed integrated fluxes and errors, erg/s/cm^2 */
  const unsigned char *lcat_mask;      /* [n_lcat] or NULL (all included) */
  const unsigned char *lcat_upper;     /* [n_lcat] nonzero: lcat_d[k] is an upper limit, or NULL */
  int dust_n_bin;              /* age-binned attenuation (App. "dust_attn"): 0 = the birth-cloud power law;
                                  n > 0 replaces it by n laws over the age axis, each with two columns
                                  (optical depth at 5500 A, slope) after every other key of the row */
  const double *dust_bin_M;    /* [n_age][n_bin] age-to-bin matrix, rows summing to 1 or all zero */
  const int *dust_bin_law;     /* [n_bin] 0 power law, 1 Kriek & Conroy 2013 */
  int use_igm;                 /* 1: the Madau (1995) IGM transmission (Sec. 2.6), scaled by the row's last
                                  column igm_factor: T = exp(-igm_factor tau_IGM(lam_obs, z)) */
} orc_model;
#define ORC_MAX_DUST_BIN 4
/* Madau (1995) effective IGM optical depth at the rest wavelengths lam_rest[n] (Angstrom) of a source
 * at redshift z (factor 1) */
void orc_igm_tau(const double *lam_rest, int n, double z, double *tau);
/* The gas velocity dispersion of the emission lines (Sec. 2.7): tied to the
 * stellar sigma_gal (the paper's default), a fixed value, or a parameter
 * column (the last one of the row). */
#define ORC_GAS_SIGMA_TIED 0
#define ORC_GAS_SIGMA_FIXED 1
#define ORC_GAS_SIGMA_SAMPLED 2
/* The calibration polynomial of the spectrum, App. E.  MARGINAL integrates the
 * coefficients out under their Gaussian prior (Eq. "app_polymarg").  OPTIMISED
 * takes, at every evaluation, the coefficients that maximise the spectrum's
 * lnL plus their log prior (the weighted least-squares solve regularised by
 * 1/s_m, whose solution is the mean M^-1 b of the marginal form): lnL gains
 * b^T M^-1 b / 2 and no Occam terms. */
#define ORC_CALIB_MARGINAL 0
#define ORC_CALIB_OPTIMISED 1

/* Escape geometries of the young light, Sec. "frac_obrun" */
#define ORC_FESC_NONE 0
#define ORC_FESC_RUNAWAY_BC 1   /* Eq. "runaway_mix": T_BC -> (1 - f_ob) e^{-tau_BC} + f_ob */
#define ORC_FESC_PICKET 2       /* f_ob of the young light escapes both dust components */

/* Terms of the noise floor, Eq. "app_noise_floor":
 * sigma_eff^2 = s^2 sigma^2 + (f_calib |m|)^2 + (f_data |d|)^2 + j^2.  Their
 * columns follow sigma_gal (when sampled), photometry first, each arm in this
 * bit order; the jitter j is in the arm's data units. */
#define ORC_FLOOR_ERR_SCALE 1   /* log10 s */
#define ORC_FLOOR_F_CALIB 2     /* log10 f_calib (model-anchored) */
#define ORC_FLOOR_F_DATA 4      /* log10 f_data (data-anchored) */
#define ORC_FLOOR_JITTER 8      /* log10 j */

/* Row status bits (shared meaning with the library by documentation only). */
#define ORC_BAD_THETA 1   /* non-finite parameter, or a sampled sigma_gal outside [0, max] */
#define ORC_BAD_Z 2       /* z < 0 or z >= zf */
#define ORC_BAD_TMAX 4    /* oldest edge not older than 10 Myr */
#define ORC_NONFINITE 16  /* non-finite model or likelihood */

int orc_n_param(const orc_model *md);

/* Cosmology: out[0] = D_L [cm] (not floored), out[1] = t_univ(z) [yr],
 * out[2] = comoving distance [cm].  Adaptive Simpson quadrature. */
void orc_cosmology(double H0, double Om0, double z, double *out);

/* SFH edges (N_T + 1 values, yr). */
void orc_sfh_edges(int n_sfh, double tmax_yr, double *T);

/* Weights W[n][m][a] for one parameter row; returns row status. */
int orc_weights(const orc_grid *g, const orc_model *md, const double *theta, double *W);

/* Ionising photon rate per SSP node, Q[n][m][a] (photons/s per Msun). */
void orc_q(const orc_grid *g, double *Q);

/* Optical depth tau(lam) of a law (0 power law, 1 KC13). */
void orc_dust_tau(int law, const double *lam, int n, double tau, double index, double *out);

/* Photometric projection of an observer-frame F_nu given on the rest grid. */
void orc_photometry(const orc_model *md, const double *lam_rest, int n_lam, double z,
                    const double *fnu_obs, double *maggies);

/* Spectral projection; valid[i] = 0 where the pixel has no model node. */
void orc_spectrum(const orc_grid *g, const orc_model *md, const double *lam_rest, int n_lam,
                  double z, double sigma_gal_kms, const double *fnu_obs, double *pix, unsigned char *valid);

/* Per-row intermediates: Y, O (young / old sums), F (attenuated rest-frame),
 * fnu (observer frame, cgs) each [n_lam]; scal[0..5] = D_L cm, t_univ yr,
 * T_max yr, Q_young, flux scale, lnL.  Any output may be NULL. Returns status. */
int orc_row(const orc_grid *g, const orc_model *md, const double *theta, double *W,
            double *Y, double *O, double *F, double *fnu, double *phot, double *spec,
            double *scal);

/* Batched evaluation: phot_out [n][n_filt], spec_out [n][n_pix], lnl_out [n],
 * status_out [n]; outputs may be NULL.  nthreads <= 0: all OpenMP threads. */
void orc_eval(const orc_grid *g, const orc_model *md, const double *theta, int n, int ld,
              double *phot_out, double *spec_out, double *lnl_out, int *status_out,
              int nthreads);

/* Observer-frame integrated flux of every grid line (erg/s/cm^2, App.
 * "line_proj"), out [n][neb_n_line]; zeros for rows with a nonzero status. */
void orc_line_fluxes(const orc_grid *g, const orc_model *md, const double *theta, int n, int ld, double *out);
/* Central finite-difference gradient of lnL (FP64), step h_j = h_rel*max(|x_j|, 1). */
void orc_grad_fd(const orc_grid *g, const orc_model *md, const double *theta, int n, int ld,
                 double h_rel, double *grad_out, int nthreads);

/* Analytic gradient of lnL (FP64 reverse pass through the same definitions):
 * grad[n_param] for one row; returns the row status, lnL in *lnl. */
int orc_row_grad(const orc_grid *g, const orc_model *md, const double *theta, double *grad, double *lnl);

/* Batched analytic gradient: grad_out [n][ld] (columns >= n_param untouched),
 * lnl_out [n], status_out [n] (either may be NULL). */
void orc_grad(const orc_grid *g, const orc_model *md, const double *theta, int n, int ld, double *lnl_out,
              double *grad_out, int *status_out, int nthreads);

#ifdef __cplusplus
}
#endif
#endif
