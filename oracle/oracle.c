/*
 * FP64 CPU oracle of the batched SED forward model and Gaussian log-likelihood.
 *
 * TEST INFRASTRUCTURE ONLY: the independent reference the GPU library is
 * checked against.  Only the test suite, the smoke check and the CPU-baseline
 * leg of the benchmark load it.  It shares no code with the library.
 *
 * Plain double precision, plainest loop order, one function per step of the
 * paper's method (section and equation named at each function).
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Physical constants (cgs unless noted). */
static const double O_LSUN = 3.839e33;            /* erg/s, value adopted in Sec. 2.6 */
static const double O_H = 6.62607015e-27;         /* erg s */
static const double O_C_AA = 2.99792458e18;       /* Angstrom/s */
static const double O_C_KMS = 299792.458;         /* km/s */
static const double O_AB = 3.631e-20;             /* erg/s/cm^2/Hz, AB zero point, App. D */
static const double O_PC_CM = 3.0856775814913673e18;
static const double O_MPC_KM = 3.0856775814913673e19;
static const double O_YR_S = 3.15576e7;           /* Julian year */
static const double O_LYMAN = 912.0;              /* Angstrom, App. C */
static const double O_FWHM_SIG = 2.3548200450309493; /* 2 sqrt(2 ln 2), Eq. "app_fwhm" */

/* ------------------------------------------------------------------ */
/* Adaptive Simpson quadrature                                          */
/* ------------------------------------------------------------------ */
typedef double (*orc_fn)(double, const double *);

static double simpson_step(orc_fn f, const double *p, double a, double b, double fa, double fm,
                           double fb, double whole, double eps, int depth) {
  double m = 0.5 * (a + b), lm = 0.5 * (a + m), rm = 0.5 * (m + b);
  double flm = f(lm, p), frm = f(rm, p);
  double left = (m - a) / 6.0 * (fa + 4.0 * flm + fm);
  double right = (b - m) / 6.0 * (fm + 4.0 * frm + fb);
  double delta = left + right - whole;
  if (depth <= 0 || fabs(delta) <= 15.0 * eps) return left + right + delta / 15.0;
  return simpson_step(f, p, a, m, fa, flm, fm, left, 0.5 * eps, depth - 1) +
         simpson_step(f, p, m, b, fm, frm, fb, right, 0.5 * eps, depth - 1);
}

static double integrate(orc_fn f, const double *p, double a, double b, double rel) {
  if (b == a) return 0.0;
  /* coarse estimate sets the absolute tolerance */
  double s = 0.0;
  int n = 64;
  double h = (b - a) / n;
  for (int i = 0; i <= n; i++) {
    double w = (i == 0 || i == n) ? 1.0 : ((i & 1) ? 4.0 : 2.0);
    s += w * f(a + i * h, p);
  }
  s *= h / 3.0;
  double eps = rel * fabs(s) + 1e-300;
  double total = 0.0;
  for (int i = 0; i < n; i++) { /* 64 panels, each adaptive */
    double x0 = a + i * h, x1 = x0 + h, xm = 0.5 * (x0 + x1);
    double f0 = f(x0, p), f1 = f(x1, p), fm = f(xm, p);
    double whole = h / 6.0 * (f0 + 4.0 * fm + f1);
    total += simpson_step(f, p, x0, x1, f0, fm, f1, whole, eps / n, 40);
  }
  return total;
}

/* ------------------------------------------------------------------ */
/* Cosmology, Sec. 2.6: flat LCDM without radiation                     */
/* ------------------------------------------------------------------ */
static double inv_E(double z, const double *p) { /* p[0] = Om */
  double zp = 1.0 + z;
  return 1.0 / sqrt(p[0] * zp * zp * zp + 1.0 - p[0]);
}
/* t = int_0^a da'/(a' H(a')), with a' = u^2: integrand 2u^2/sqrt(Om + OL u^6) (units 1/H0) */
static double age_integrand(double u, const double *p) {
  double u2 = u * u;
  return 2.0 * u2 / sqrt(p[0] + (1.0 - p[0]) * u2 * u2 * u2);
}

void orc_cosmology(double H0, double Om0, double z, double *out) {
  double p[1] = {Om0};
  double dh_cm = O_C_KMS / H0 * 1e6 * O_PC_CM;          /* c/H0 in cm */
  double th_yr = O_MPC_KM / H0 / O_YR_S;                 /* 1/H0 in yr */
  double dc = dh_cm * integrate(inv_E, p, 0.0, z, 1e-13);
  double umax = 1.0 / sqrt(1.0 + z);
  double t = th_yr * integrate(age_integrand, p, 0.0, umax, 1e-13);
  out[0] = (1.0 + z) * dc;
  out[1] = t;
  out[2] = dc;
}

/* ------------------------------------------------------------------ */
/* SFH edges: 0, 5 Myr, 10 Myr, then log-uniform to T_max (Sec. 5, App. B) */
/* ------------------------------------------------------------------ */
void orc_sfh_edges(int n_sfh, double tmax_yr, double *T) {
  T[0] = 0.0;
  T[1] = 5e6;
  T[2] = 1e7;
  for (int i = 3; i <= n_sfh; i++)
    T[i] = 1e7 * pow(tmax_yr / 1e7, (double)(i - 2) / (double)(n_sfh - 2));
}

/* Linear interpolation weights between the bracketing nodes, clamped to the
 * end nodes outside the axis (App. B: "linear interpolation in log10(Z/Zsun)"). */
static void bracket(const double *x, int n, double v, int *j0, double *w0, int *j1, double *w1) {
  if (n == 1) { *j0 = *j1 = 0; *w0 = 1.0; *w1 = 0.0; return; }
  if (v <= x[0]) { *j0 = 0; *j1 = 1; *w0 = 1.0; *w1 = 0.0; return; }
  if (v >= x[n - 1]) { *j0 = n - 2; *j1 = n - 1; *w0 = 0.0; *w1 = 1.0; return; }
  int j = 0;
  while (!(x[j] <= v && v < x[j + 1])) j++;
  double t = (v - x[j]) / (x[j + 1] - x[j]);
  *j0 = j; *j1 = j + 1; *w0 = 1.0 - t; *w1 = t;
}

static int n_floor(int bits) {
  int c = 0;
  for (int k = 0; k < 4; k++) c += (bits >> k) & 1;
  return c;
}

/* columns of the SFH key: N_T bin masses (step scheme) or N_T + 1 edge SFRs (linear scheme) */
static int sfh_cols(const orc_model *md) { return md->n_sfh + (md->sfh_scheme == 1 ? 1 : 0); }

int orc_n_param(const orc_model *md) {
  return sfh_cols(md) + (md->zmode == 0 ? md->n_sfh : 1) + 9 + (md->sample_sigma_gal ? 1 : 0) +
         n_floor(md->floor_phot) + n_floor(md->floor_spec) + (md->fesc_geometry ? 1 : 0) +
         (md->gas_sigma_mode == ORC_GAS_SIGMA_SAMPLED ? 1 : 0) + 2 * md->dust_n_bin + (md->use_igm ? 1 : 0);
}

/* parameter row decoding (layout: sfh[N_T], logzsol[N_T or 1], afe, logmass,
 * zred, tau_pow, alpha_pow, diffuse_tau_kc, diffuse_dust_index, gas_logz, gas_logu,
 * then sigma_gal when the model samples it) */
typedef struct {
  const double *m, *zeta;
  double afe, logmass, z, tau_bc, alpha_bc, tau_d, delta, gas_logz, gas_logu, sigma_gal;
  double fl[2][4];   /* noise floor {s, f_calib, f_data, j} of photometry [0] and spectrum [1] */
  int fl_col[2][4];  /* column of each term in the row, -1 when the term is off */
  double fob;        /* runaway fraction f_ob (0 without an escape geometry) */
  double sigma_gas;  /* gas dispersion of the emission lines, km/s */
  double bin_tau[ORC_MAX_DUST_BIN], bin_slope[ORC_MAX_DUST_BIN];   /* age-binned laws' parameters */
  double igm_f;      /* scaling of the IGM optical depth (1 without a column) */
} orc_theta;

static void decode_theta(const orc_model *md, const double *th, orc_theta *o) {
  int nz = md->zmode == 0 ? md->n_sfh : 1, ns = sfh_cols(md);
  const double *s = th + ns + nz;
  o->m = th;
  o->zeta = th + ns;
  o->afe = s[0]; o->logmass = s[1]; o->z = s[2]; o->tau_bc = s[3]; o->alpha_bc = s[4];
  o->tau_d = s[5]; o->delta = s[6]; o->gas_logz = s[7]; o->gas_logu = s[8];
  o->sigma_gal = md->sample_sigma_gal ? s[9] : md->sigma_gal_kms;
  /* App. "sys_floor": a term that is off leaves s = 1 and the others 0 */
  int col = ns + nz + 9 + (md->sample_sigma_gal ? 1 : 0);
  for (int arm = 0; arm < 2; arm++) {
    int bits = arm == 0 ? md->floor_phot : md->floor_spec;
    for (int k = 0; k < 4; k++) {
      o->fl[arm][k] = k == 0 ? 1.0 : 0.0;
      o->fl_col[arm][k] = -1;
      if ((bits >> k) & 1) {
        o->fl[arm][k] = pow(10.0, th[col]);
        o->fl_col[arm][k] = col++;
      }
    }
  }
  o->fob = md->fesc_geometry ? th[col++] : 0.0;
  o->sigma_gas = md->gas_sigma_mode == ORC_GAS_SIGMA_SAMPLED ? th[col++]
               : (md->gas_sigma_mode == ORC_GAS_SIGMA_FIXED ? md->sigma_gas_kms : o->sigma_gal);
  for (int b = 0; b < md->dust_n_bin && b < ORC_MAX_DUST_BIN; b++) {
    o->bin_tau[b] = th[col++];
    o->bin_slope[b] = th[col++];
  }
  o->igm_f = md->use_igm ? th[col++] : 1.0;
}

/* Madau (1995) mean IGM optical depth seen at the observed wavelength
 * lam_obs = lam_rest (1 + z) from a source at z (Sec. 2.6 names the
 * prescription): line blanketing by the Lyman series, A_j (lam_obs/lam_j)^3.46
 * for each line j with lam_j < lam_obs < lam_j (1 + z) (Ly-alpha to Ly-delta,
 * A_j = 3.6e-3, 1.7e-3, 1.1846e-3, 9.316e-4), plus photoelectric absorption by
 * Lyman-limit systems for lam_obs < lam_L (1 + z), lam_L = 911.75 A, with
 * x_c = lam_obs / lam_L (not below 1) and x_e = 1 + z:
 *   0.25 x_c^3 (x_e^0.46 - x_c^0.46) + 9.4 x_c^1.5 (x_e^0.18 - x_c^0.18)
 *   - 0.7 x_c^3 (x_c^-1.32 - x_e^-1.32) - 0.023 (x_e^1.68 - x_c^1.68). */
static double igm_madau_tau(double lam_rest, double z) {
  static const double lj[4] = {1215.67, 1025.72, 972.537, 949.743};
  static const double aj[4] = {3.6e-3, 1.7e-3, 1.1846e-3, 9.316e-4};
  const double lo = lam_rest * (1.0 + z);
  double tau = 0.0;
  for (int j = 0; j < 4; j++)
    if (lam_rest < lj[j] && lo > lj[j]) tau += aj[j] * pow(lo / lj[j], 3.46);
  if (lam_rest < 911.75) {
    double xc = lo / 911.75, xe = 1.0 + z;
    if (xc < 1.0) xc = 1.0;
    tau += 0.25 * xc * xc * xc * (pow(xe, 0.46) - pow(xc, 0.46)) + 9.4 * pow(xc, 1.5) * (pow(xe, 0.18) - pow(xc, 0.18)) -
           0.7 * xc * xc * xc * (pow(xc, -1.32) - pow(xe, -1.32)) - 0.023 * (pow(xe, 1.68) - pow(xc, 1.68));
  }
  return tau;
}

void orc_igm_tau(const double *lam_rest, int n, double z, double *tau) {
  for (int k = 0; k < n; k++) tau[k] = igm_madau_tau(lam_rest[k], z);
}

/* Eq. "app_noise_floor": the effective variance of a datum with formal error
 * sigma, model m and datum d under the floor fl = {s, f_calib, f_data, j}. */
static double eff_var(const double *fl, double sigma, double m, double d) {
  return fl[0] * fl[0] * sigma * sigma + fl[1] * fl[1] * m * m + fl[2] * fl[2] * d * d + fl[3] * fl[3];
}

/* Derivatives of one datum's term -r^2/(2v) - ln(2 pi v)/2 (r = d - m, v its
 * effective variance): returns d term / d m (v depends on m through the
 * model-anchored f_calib), and adds d term / d log10 of each floor term,
 * dv/dlog10 x = 2 ln(10) x^2 (sigma^2, m^2, d^2, 1 for s, f_calib, f_data, j). */
static double floor_terms_grad(const double *fl, double v, double r, double sigma, double m, double d,
                               double *g) {
  const double gv = 0.5 * r * r / (v * v) - 0.5 / v;   /* d term / d v */
  const double l10 = log(10.0);
  g[0] += gv * 2.0 * l10 * fl[0] * fl[0] * sigma * sigma;
  g[1] += gv * 2.0 * l10 * fl[1] * fl[1] * m * m;
  g[2] += gv * 2.0 * l10 * fl[2] * fl[2] * d * d;
  g[3] += gv * 2.0 * l10 * fl[3] * fl[3];
  return r / v + gv * 2.0 * fl[1] * fl[1] * m;
}

/* The residual d - m of photometric band b in Eq. "total_lnlike".  A band
 * flagged as an upper limit (Sec. 4.1, Eq. "app_line_chi2_UL") costs nothing
 * while the model stays at or below the limit d (residual 0) and the Gaussian
 * residual against d once it exceeds it; its normalisation term stays. */
static double phot_residual(const orc_model *md, int b, double d, double m) {
  if (md->phot_upper && md->phot_upper[b] && m <= d) return 0.0;
  return d - m;
}

static int theta_status(const orc_model *md, const double *th, double *tmax_out, double *cos_out) {
  int np = orc_n_param(md);
  for (int j = 0; j < np; j++)
    if (!isfinite(th[j])) return ORC_BAD_THETA;
  orc_theta t;
  decode_theta(md, th, &t);
  if (md->sample_sigma_gal && !(t.sigma_gal >= 0.0 && t.sigma_gal <= md->sigma_gal_max_kms)) return ORC_BAD_THETA;
  if (md->fesc_geometry && !(t.fob >= 0.0 && t.fob <= 1.0)) return ORC_BAD_THETA;
  if (md->gas_sigma_mode == ORC_GAS_SIGMA_SAMPLED && !(t.sigma_gas >= 0.0 && t.sigma_gas <= md->sigma_gas_max_kms))
    return ORC_BAD_THETA;
  if (t.z < 0.0 || t.z >= md->zf) return ORC_BAD_Z;
  double cz[3], cf[3];
  orc_cosmology(md->H0, md->Om0, t.z, cz);
  orc_cosmology(md->H0, md->Om0, md->zf, cf);
  double tmax = cz[1] - cf[1];
  if (cos_out) { cos_out[0] = cz[0]; cos_out[1] = cz[1]; }
  if (tmax_out) *tmax_out = tmax;
  if (!(tmax > 1e7)) return ORC_BAD_TMAX;
  return 0;
}

/* App. B step scheme: A_ia = m_i |[T_i,T_{i+1}] ∩ cell_a| / dT_i with cell_a the
 * linear-time Voronoi cell of age node a (midpoints to its neighbours, first
 * cell from 0, last cell to infinity); then the metallicity split of each bin
 * and the [a/Fe] split (Sec. 5.4), W[n][m][a] = sum_i A_ia w_m(zeta_i) w_n(afe). */
/* App. B linear scheme, Eq. "tent_integral": the SFR is linear in lookback
 * time across the bin [T0, T1], from psi0 at T0 to psi1 at T1, and the mass an
 * SSP age node receives is the integral of the SFR against that node's tent,
 * the linear interpolation in log(age) between neighbouring nodes (a_j(t) =
 * ln(t_{j+1}/t) / ln(t_{j+1}/t_j) on [t_j, t_{j+1}], b_{j+1} = 1 - a_j).  The
 * bin is cut at the nodes and each piece integrated in closed form with the
 * antiderivatives of psi(t) and psi(t) ln t; ages below the youngest node go
 * to it, ages above the oldest to that one.  Negative pieces are clipped to 0,
 * then the bin's masses are scaled to sum to its trapezoidal mass
 * (psi0 + psi1)(T1 - T0)/2, itself clipped at 0.  A[NA] receives the bin's
 * mass per node. */
static void linear_bin_masses(const orc_grid *g, double T0, double T1, double psi0, double psi1, double *A) {
  int NA = g->n_age;
  for (int a = 0; a < NA; a++) A[a] = 0.0;
  double dT = T1 - T0;
  if (!(dT > 0.0)) return;
  double beta = (psi1 - psi0) / dT, alpha = psi0 - beta * T0;   /* psi(t) = alpha + beta t */
  /* P = antiderivative of psi, Q = antiderivative of psi ln t */
#define LIN_P(x) (alpha * (x) + 0.5 * beta * (x) * (x))
#define LIN_Q(x) (alpha * ((x) * log(x) - (x)) + beta * (0.5 * (x) * (x) * log(x) - 0.25 * (x) * (x)))
  double t_first = pow(10.0, g->log_age_yr[0]), t_last = pow(10.0, g->log_age_yr[NA - 1]);
  /* below the youngest node and above the oldest: wholly to the end node */
  if (T0 < t_first) {
    double hi = T1 < t_first ? T1 : t_first, m = LIN_P(hi) - LIN_P(T0);
    A[0] += m > 0.0 ? m : 0.0;
  }
  if (T1 > t_last) {
    double lo = T0 > t_last ? T0 : t_last, m = LIN_P(T1) - LIN_P(lo);
    A[NA - 1] += m > 0.0 ? m : 0.0;
  }
  for (int j = 0; j + 1 < NA; j++) {
    double tj = pow(10.0, g->log_age_yr[j]), tj1 = pow(10.0, g->log_age_yr[j + 1]);
    double x0 = T0 > tj ? T0 : tj, x1 = T1 < tj1 ? T1 : tj1;
    if (!(x1 > x0)) continue;
    double mass = LIN_P(x1) - LIN_P(x0), mlog = LIN_Q(x1) - LIN_Q(x0);
    double lj = log(tj), lj1 = log(tj1), d = lj1 - lj;
    double to_j = (lj1 * mass - mlog) / d, to_j1 = (mlog - lj * mass) / d;
    A[j] += to_j > 0.0 ? to_j : 0.0;
    A[j + 1] += to_j1 > 0.0 ? to_j1 : 0.0;
  }
#undef LIN_P
#undef LIN_Q
  double s = 0.0, target = 0.5 * (psi0 + psi1) * dT;
  if (target < 0.0) target = 0.0;   /* a bin whose rates average below 0 forms nothing */
  for (int a = 0; a < NA; a++) s += A[a];
  if (s > 0.0)
    for (int a = 0; a < NA; a++) A[a] *= target / s;
}

/* One piece of the linear scheme's bin: the integral over [x0, x1] of the rate
 * alpha + beta t against the weight of its kind (0: 1, the end pieces; 1: the
 * tent of node j, (l1 - ln t)/(l1 - l0); 2: the tent of node j + 1,
 * (ln t - l0)/(l1 - l0)), with l0 = ln t_j, l1 = ln t_{j+1}. */
static double lin_piece(double alpha, double beta, double x0, double x1, int kind, double l0, double l1) {
  double mass = alpha * (x1 - x0) + 0.5 * beta * (x1 * x1 - x0 * x0);
  if (kind == 0) return mass;
  double mlog = alpha * (x1 * log(x1) - x1 - x0 * log(x0) + x0) +
                beta * (0.5 * x1 * x1 * log(x1) - 0.25 * x1 * x1 - 0.5 * x0 * x0 * log(x0) + 0.25 * x0 * x0);
  double d = l1 - l0;
  return kind == 1 ? (l1 * mass - mlog) / d : (mlog - l0 * mass) / d;
}

static double lin_weight(double x, int kind, double l0, double l1) {
  if (kind == 0) return 1.0;
  return kind == 1 ? (l1 - log(x)) / (l1 - l0) : (log(x) - l0) / (l1 - l0);
}

/* Reverse of linear_bin_masses.  Given gA[a] = dL/dA[a] for the bin's node
 * masses, returns d4 = dL/d{psi0, psi1, T0, T1}.  Each piece is linear in the
 * rate: its derivative in psi0 (psi1) is the same piece for the unit rate
 * falling from 1 to 0 (rising from 0 to 1) across the bin.  An edge moves a
 * piece through the integral's limit (minus or plus the integrand there, when
 * the piece starts or ends at that edge) and through the rate itself:
 * dpsi/dT0 = c (t - T1) and dpsi/dT1 = -c (t - T0), c = (psi1 - psi0)/dT^2,
 * both again linear rates.  A clipped piece carries no derivative.  The scale
 * to the trapezoidal mass enters by the quotient rule. */
static void linear_bin_grad(const orc_grid *g, double T0, double T1, double psi0, double psi1,
                            const double *gA, double *d4) {
  int NA = g->n_age;
  d4[0] = d4[1] = d4[2] = d4[3] = 0.0;
  double dT = T1 - T0;
  if (!(dT > 0.0)) return;
  double c = (psi1 - psi0) / (dT * dT);
  /* rates (alpha, beta): the row's psi, d/dpsi0, d/dpsi1, d/dT0, d/dT1 */
  double rb[5] = {(psi1 - psi0) / dT, -1.0 / dT, 1.0 / dT, c, -c};
  double ra[5] = {psi0 - rb[0] * T0, 1.0 - rb[1] * T0, -rb[2] * T0, -c * T1, c * T0};
  double *raw = (double *)calloc(NA, sizeof(double));
  double *dr = (double *)calloc((size_t)4 * NA, sizeof(double));
  double t_first = pow(10.0, g->log_age_yr[0]), t_last = pow(10.0, g->log_age_yr[NA - 1]);
  /* the pieces in the forward's order: (node, kind, x0, x1, l0, l1) */
  for (int j = -1; j < NA; j++) {
    int nodes[2], kinds[2], np_ = 0;
    double x0, x1, l0 = 0.0, l1 = 0.0;
    if (j == -1) {                 /* below the youngest node */
      if (!(T0 < t_first)) continue;
      x0 = T0; x1 = T1 < t_first ? T1 : t_first;
      nodes[0] = 0; kinds[0] = 0; np_ = 1;
    } else if (j == NA - 1) {      /* above the oldest node */
      if (!(T1 > t_last)) continue;
      x0 = T0 > t_last ? T0 : t_last; x1 = T1;
      nodes[0] = NA - 1; kinds[0] = 0; np_ = 1;
    } else {
      double tj = pow(10.0, g->log_age_yr[j]), tj1 = pow(10.0, g->log_age_yr[j + 1]);
      x0 = T0 > tj ? T0 : tj; x1 = T1 < tj1 ? T1 : tj1;
      if (!(x1 > x0)) continue;
      l0 = log(tj); l1 = log(tj1);
      nodes[0] = j; kinds[0] = 1; nodes[1] = j + 1; kinds[1] = 2; np_ = 2;
    }
    if (np_ == 1 && !(x1 > x0)) continue;
    for (int q = 0; q < np_; q++) {
      int a = nodes[q], kd = kinds[q];
      double v = lin_piece(ra[0], rb[0], x0, x1, kd, l0, l1);
      if (!(v > 0.0)) continue;   /* clipped */
      raw[a] += v;
      dr[4 * a + 0] += lin_piece(ra[1], rb[1], x0, x1, kd, l0, l1);
      dr[4 * a + 1] += lin_piece(ra[2], rb[2], x0, x1, kd, l0, l1);
      dr[4 * a + 2] += lin_piece(ra[3], rb[3], x0, x1, kd, l0, l1) - (x0 == T0 ? psi0 * lin_weight(T0, kd, l0, l1) : 0.0);
      dr[4 * a + 3] += lin_piece(ra[4], rb[4], x0, x1, kd, l0, l1) + (x1 == T1 ? psi1 * lin_weight(T1, kd, l0, l1) : 0.0);
    }
  }
  double sum = 0.0, ds[4] = {0, 0, 0, 0};
  for (int a = 0; a < NA; a++) {
    sum += raw[a];
    for (int p = 0; p < 4; p++) ds[p] += dr[4 * a + p];
  }
  double target = 0.5 * (psi0 + psi1) * dT, dtg[4] = {0, 0, 0, 0};
  if (target > 0.0) {
    dtg[0] = 0.5 * dT; dtg[1] = 0.5 * dT; dtg[2] = -0.5 * (psi0 + psi1); dtg[3] = 0.5 * (psi0 + psi1);
  } else {
    target = 0.0;
  }
  if (sum > 0.0)
    for (int a = 0; a < NA; a++)
      for (int p = 0; p < 4; p++)
        d4[p] += gA[a] * (dr[4 * a + p] * target / sum + raw[a] * (dtg[p] * sum - target * ds[p]) / (sum * sum));
  free(raw); free(dr);
}

int orc_weights(const orc_grid *g, const orc_model *md, const double *theta, double *W) {
  double tmax;
  int st = theta_status(md, theta, &tmax, NULL);
  size_t nW = (size_t)g->n_afe * g->n_feh * g->n_age;
  memset(W, 0, nW * sizeof(double));
  if (st) return st;
  orc_theta t;
  decode_theta(md, theta, &t);
  int NT = md->n_sfh, NA = g->n_age;
  double *T = (double *)malloc((NT + 1) * sizeof(double));
  double *cm = (double *)malloc(NA * sizeof(double));
  double *cp = (double *)malloc(NA * sizeof(double));
  orc_sfh_edges(NT, tmax, T);
  for (int a = 0; a < NA; a++) {
    double ta = pow(10.0, g->log_age_yr[a]);
    cm[a] = (a == 0) ? 0.0 : 0.5 * (pow(10.0, g->log_age_yr[a - 1]) + ta);
    cp[a] = (a == NA - 1) ? INFINITY : 0.5 * (ta + pow(10.0, g->log_age_yr[a + 1]));
  }
  int n0, n1;
  double wn0, wn1;
  double afe = md->use_afe ? t.afe : 0.0;
  bracket(g->afe, g->n_afe, afe, &n0, &wn0, &n1, &wn1);
  double *A = (double *)malloc(NA * sizeof(double));
  for (int i = 0; i < NT; i++) {
    double dT = T[i + 1] - T[i];
    double zeta = t.zeta[md->zmode == 0 ? i : 0];
    int m0, m1;
    double wm0, wm1;
    bracket(g->feh, g->n_feh, zeta, &m0, &wm0, &m1, &wm1);
    /* the mass bin i gives each age node */
    if (md->sfh_scheme == 1) {
      linear_bin_masses(g, T[i], T[i + 1], t.m[i], t.m[i + 1], A);
    } else {
      for (int a = 0; a < NA; a++) {
        double lo = T[i] > cm[a] ? T[i] : cm[a];
        double hi = T[i + 1] < cp[a] ? T[i + 1] : cp[a];
        double ov = hi - lo;
        A[a] = ov > 0.0 ? t.m[i] * ov / dT : 0.0;
      }
    }
    for (int a = 0; a < NA; a++) {
      if (A[a] == 0.0) continue;
      W[((size_t)n0 * g->n_feh + m0) * NA + a] += A[a] * wm0 * wn0;
      W[((size_t)n0 * g->n_feh + m1) * NA + a] += A[a] * wm1 * wn0;
      W[((size_t)n1 * g->n_feh + m0) * NA + a] += A[a] * wm0 * wn1;
      W[((size_t)n1 * g->n_feh + m1) * NA + a] += A[a] * wm1 * wn1;
    }
  }
  free(T); free(cm); free(cp); free(A);
  return 0;
}

/* App. C, Eq. "app_q": Q = (Lsun/h) int_0^912 f(lam)/lam dlam, trapezoid over the
 * nodes below 912 A plus the linearly interpolated piece up to 912 A. */
void orc_q(const orc_grid *g, double *Q) {
  size_t nsp = (size_t)g->n_afe * g->n_feh * g->n_age;
  const double *lam = g->lam;
  for (size_t s = 0; s < nsp; s++) {
    const double *f = g->flux + s * g->n_lam;
    double acc = 0.0;
    for (int k = 0; k + 1 < g->n_lam; k++) {
      if (lam[k] >= O_LYMAN) break;
      double x1 = lam[k + 1], f1 = f[k + 1];
      if (x1 > O_LYMAN) {
        f1 = f[k] + (f[k + 1] - f[k]) * (O_LYMAN - lam[k]) / (lam[k + 1] - lam[k]);
        x1 = O_LYMAN;
      }
      acc += 0.5 * (f[k] / lam[k] + f1 / x1) * (x1 - lam[k]);
    }
    Q[s] = O_LSUN / O_H * acc;
  }
}

/* Calzetti et al. (2000) k'(lam), R_V = 4.05, lam in micron; the UV branch is
 * used below 0.63 micron (also below 0.12 micron); clamped at zero. */
static double calzetti_kprime(double lum) {
  double k;
  if (lum >= 0.63)
    k = 2.659 * (-1.857 + 1.040 / lum) + 4.05;
  else
    k = 2.659 * (-2.156 + 1.509 / lum - 0.198 / (lum * lum) + 0.011 / (lum * lum * lum)) + 4.05;
  return k > 0.0 ? k : 0.0;
}

/* Sec. 2.4: Kriek & Conroy (2013) diffuse law, tau(lam) = tau [k'(lam) +
 * D(lam)] / 4.05 (lam/5500)^delta with a Drude bump of central wavelength
 * 2175 A, width 350 A and strength E_b = 0.85 - 1.9 delta; power law:
 * tau(lam) = tau (lam/5500)^index. */
void orc_dust_tau(int law, const double *lam, int n, double tau, double index, double *out) {
  for (int k = 0; k < n; k++) {
    double p = pow(lam[k] / 5500.0, index);
    if (law == 0) {
      out[k] = tau * p;
    } else {
      double eb = 0.85 - 1.9 * index;
      double x = lam[k] * 350.0;
      double d = lam[k] * lam[k] - 2175.0 * 2175.0;
      double drude = eb * x * x / (d * d + x * x);
      out[k] = tau * (calzetti_kprime(lam[k] * 1e-4) + drude) / 4.05 * p;
    }
  }
}

/* App. D: m_b = sum_j R_b(l_j) l_j dl_j f_lam(l_j) / Z_b, with f_lam the linear
 * interpolation (in observed wavelength) of c F_nu/lam_obs^2 over the redshifted
 * model grid (zero outside it), dl_j the local spacing (half-interval at the
 * ends) and Z_b = trapz_j l_j R_b(l_j) c 3.631e-20 / l_j^2. */
void orc_photometry(const orc_model *md, const double *lam_rest, int n_lam, double z,
                    const double *fnu_obs, double *maggies) {
  double zp = 1.0 + z;
  double lo = zp * lam_rest[0], hi = zp * lam_rest[n_lam - 1];
  int off = 0;
  for (int b = 0; b < md->n_filt; b++) {
    int n = md->filt_len[b];
    const double *L = md->filt_lam + off, *R = md->filt_trans + off;
    off += n;
    double zb = 0.0;
    for (int j = 0; j + 1 < n; j++) {
      double g0 = L[j] * R[j] * O_C_AA * O_AB / (L[j] * L[j]);
      double g1 = L[j + 1] * R[j + 1] * O_C_AA * O_AB / (L[j + 1] * L[j + 1]);
      zb += 0.5 * (g0 + g1) * (L[j + 1] - L[j]);
    }
    double acc = 0.0;
    for (int j = 0; j < n; j++) {
      double dl;
      if (n == 1) dl = 0.0;
      else if (j == 0) dl = 0.5 * (L[1] - L[0]);
      else if (j == n - 1) dl = 0.5 * (L[n - 1] - L[n - 2]);
      else dl = 0.5 * (L[j + 1] - L[j - 1]);
      double x = L[j], flam = 0.0;
      if (x >= lo && x <= hi) {
        int k = 0, kh = n_lam - 1; /* binary search: zp*lam[k] <= x <= zp*lam[k+1] */
        while (kh - k > 1) {
          int mid = (k + kh) / 2;
          if (zp * lam_rest[mid] <= x) k = mid; else kh = mid;
        }
        double xa = zp * lam_rest[k], xb = zp * lam_rest[k + 1];
        double ga = O_C_AA * fnu_obs[k] / (xa * xa), gb = O_C_AA * fnu_obs[k + 1] / (xb * xb);
        flam = ga + (gb - ga) * (x - xa) / (xb - xa);
      }
      acc += R[j] * x * dl * flam;
    }
    maggies[b] = acc / zb;
  }
}

/* Eq. "app_siglib" two-pixel floor at the grid nodes, max with the documented
 * library LSF when given. */
static void siglib_nodes(const orc_grid *g, double *out) {
  int n = g->n_lam;
  const double *L = g->lam;
  for (int k = 0; k < n; k++) {
    double dl;
    if (k == 0) dl = L[1] - L[0];
    else if (k == n - 1) dl = L[n - 1] - L[n - 2];
    else dl = 0.5 * (L[k + 1] - L[k - 1]);
    double s = O_C_KMS / O_FWHM_SIG * 2.0 * dl / L[k];
    if (g->sigma_lib_kms && g->sigma_lib_kms[k] > s) s = g->sigma_lib_kms[k];
    out[k] = s;
  }
}

/* Eq. "app_modes": instrumental velocity dispersion at an observed pixel. */
static double sigma_inst_kms(int mode, double v, double lam_obs) {
  switch (mode) {
    case 0: return O_C_KMS / (O_FWHM_SIG * v);
    case 1: return O_C_KMS / v;
    case 2: return O_C_KMS * v / (O_FWHM_SIG * lam_obs);
    case 3: return O_C_KMS * v / lam_obs;
    case 4: return v;
    default: return v / O_FWHM_SIG;
  }
}

/* Per-pixel total dispersion in ln(lam): Eq. "app_sigeff" (fixed part at the
 * projector's reference redshift) composed in quadrature with the row's
 * sigma_gal (Eq. "one_kernel"; the paper's Fourier stage for sigma_gal and the
 * banded sigma_fix response compose to this one Gaussian, App. E). */
static void spec_widths(const orc_grid *g, const orc_model *md, double sigma_gal_kms, double *s_ln) {
  double *sl = (double *)malloc(g->n_lam * sizeof(double));
  siglib_nodes(g, sl);
  for (int i = 0; i < md->n_pix; i++) {
    double lo = md->spec_lam[i];
    double si = sigma_inst_kms(md->lsf_mode, md->lsf_value[i], lo);
    double lr = lo / (1.0 + md->z_ref), slib;
    if (lr <= g->lam[0]) slib = sl[0];
    else if (lr >= g->lam[g->n_lam - 1]) slib = sl[g->n_lam - 1];
    else {
      int k = 0;
      while (!(g->lam[k] <= lr && lr < g->lam[k + 1])) k++;
      slib = sl[k] + (sl[k + 1] - sl[k]) * (lr - g->lam[k]) / (g->lam[k + 1] - g->lam[k]);
    }
    double fix2 = si * si - slib * slib;
    if (fix2 < 0.0) fix2 = 0.0;
    s_ln[i] = sqrt(fix2 + sigma_gal_kms * sigma_gal_kms) / O_C_KMS;
  }
  free(sl);
}

/* Eq. "app_response": Gaussian rows in ln(lam) centred on each pixel shifted
 * by ln(1+z), truncated at five dispersions, normalised to unit sum; rows
 * narrower than half a model log-pixel are linear interpolation in ln(lam). */
void orc_spectrum(const orc_grid *g, const orc_model *md, const double *lam_rest, int n_lam,
                  double z, double sigma_gal_kms, const double *fnu_obs, double *pix, unsigned char *valid) {
  double *s_ln = (double *)malloc(md->n_pix * sizeof(double));
  double *ll = (double *)malloc(n_lam * sizeof(double));
  spec_widths(g, md, sigma_gal_kms, s_ln);
  for (int k = 0; k < n_lam; k++) ll[k] = log(lam_rest[k]);
  double lz = log(1.0 + z);
  for (int i = 0; i < md->n_pix; i++) {
    double x = log(md->spec_lam[i]) - lz, s = s_ln[i];
    pix[i] = 0.0;
    valid[i] = 0;
    if (x < ll[0] || x > ll[n_lam - 1]) continue;
    int k = 0;
    while (k + 2 < n_lam && !(ll[k] <= x && x < ll[k + 1])) k++;
    double dln = ll[k + 1] - ll[k];
    if (s < 0.5 * dln) {
      double t = (x - ll[k]) / dln;
      pix[i] = (1.0 - t) * fnu_obs[k] + t * fnu_obs[k + 1];
      valid[i] = 1;
      continue;
    }
    double sw = 0.0, sf = 0.0;
    for (int j = 0; j < n_lam; j++) {
      double u = (ll[j] - x) / s;
      if (fabs(u) > 5.0) continue;
      double w = exp(-0.5 * u * u);
      sw += w;
      sf += w * fnu_obs[j];
    }
    if (sw > 0.0) { pix[i] = sf / sw; valid[i] = 1; }
  }
  free(s_ln);
  free(ll);
}

/* App. E, marginalised calibration polynomial (Eq. app_polymarg).  The
 * calibrated model is mu_i (1 + sum_m c_m T_m(x_i)), T_m the Chebyshev
 * polynomials of the pixel wavelengths mapped linearly onto [-1, 1] (first and
 * last pixel at -1 and 1); with the prior c ~ N(0, Lambda), Lambda = diag(s_m^2),
 * the coefficients integrate out and lnL gains
 *   b^T M^-1 b / 2 - ln|M| / 2 - ln|Lambda| / 2,
 *   M = D^T C^-1 D + Lambda^-1,  b = D^T C^-1 r,  D = diag(mu) A,  A_im = T_m(x_i),
 * r = d - mu, C = diag(sigma^2), over the included pixels inc[i] != 0.  With
 * the polynomial optimised instead (calib_mode ORC_CALIB_OPTIMISED) the gain is
 * b^T M^-1 b / 2 alone: the maximum over c of lnL_diag(r - D c) - c^T
 * Lambda^-1 c / 2, reached at c = M^-1 b.  Returns these terms; minv [n][n] =
 * M^-1 and cstar [n] = M^-1 b when non-NULL. */
static void cheb_row(double x, int n, double *T) {
  T[0] = 1.0;
  if (n > 1) T[1] = x;
  for (int m = 2; m < n; m++) T[m] = 2.0 * x * T[m - 1] - T[m - 2];
}
static double cheb_x(const orc_model *md, int i) {
  double lo = md->spec_lam[0], hi = md->spec_lam[md->n_pix - 1];
  return md->n_pix > 1 ? (2.0 * md->spec_lam[i] - (lo + hi)) / (hi - lo) : 0.0;
}
static double calib_terms(const orc_model *md, const double *mu, const unsigned char *inc, double *minv,
                          double *cstar) {
  int n = md->calib_n;
  double *M = (double *)calloc((size_t)n * n, sizeof(double));
  double *L = (double *)calloc((size_t)n * n, sizeof(double));
  double *b = (double *)calloc(n, sizeof(double));
  double *c = (double *)calloc(n, sizeof(double));
  double *T = (double *)malloc(n * sizeof(double));
  for (int i = 0; i < md->n_pix; i++) {
    if (!inc[i]) continue;
    cheb_row(cheb_x(md, i), n, T);
    double w = 1.0 / (md->spec_sigma[i] * md->spec_sigma[i]), r = md->spec_d[i] - mu[i];
    for (int a = 0; a < n; a++) {
      b[a] += mu[i] * T[a] * w * r;
      for (int e = 0; e < n; e++) M[a * n + e] += mu[i] * T[a] * w * mu[i] * T[e];
    }
  }
  double logdet_lam = 0.0;
  for (int a = 0; a < n; a++) {
    M[a * n + a] += 1.0 / (md->calib_sigma[a] * md->calib_sigma[a]);
    logdet_lam += log(md->calib_sigma[a] * md->calib_sigma[a]);
  }
  /* Cholesky M = L L^T */
  double logdet = 0.0;
  int ok = 1;
  for (int j = 0; j < n && ok; j++) {
    double d = M[j * n + j];
    for (int k = 0; k < j; k++) d -= L[j * n + k] * L[j * n + k];
    if (!(d > 0.0)) { ok = 0; break; }
    L[j * n + j] = sqrt(d);
    logdet += log(d);
    for (int i = j + 1; i < n; i++) {
      double v = M[i * n + j];
      for (int k = 0; k < j; k++) v -= L[i * n + k] * L[j * n + k];
      L[i * n + j] = v / L[j * n + j];
    }
  }
  double out = NAN;
  if (ok) {
    /* c = M^-1 b by forward and back substitution */
    for (int i = 0; i < n; i++) {
      double v = b[i];
      for (int k = 0; k < i; k++) v -= L[i * n + k] * c[k];
      c[i] = v / L[i * n + i];
    }
    for (int i = n - 1; i >= 0; i--) {
      double v = c[i];
      for (int k = i + 1; k < n; k++) v -= L[k * n + i] * c[k];
      c[i] = v / L[i * n + i];
    }
    double quad = 0.0;
    for (int a = 0; a < n; a++) quad += b[a] * c[a];
    /* optimised polynomial: max over c of lnL_diag(r - D c) - c^T Lambda^-1 c / 2
     * = lnL_diag(r) + b^T M^-1 b / 2; marginalised: minus the Occam terms */
    out = md->calib_mode == ORC_CALIB_OPTIMISED ? 0.5 * quad : 0.5 * quad - 0.5 * logdet - 0.5 * logdet_lam;
    if (cstar) memcpy(cstar, c, n * sizeof(double));
    if (minv) {
      double *e = (double *)malloc(n * sizeof(double));
      for (int col = 0; col < n; col++) {
        for (int i = 0; i < n; i++) {
          double v = i == col ? 1.0 : 0.0;
          for (int k = 0; k < i; k++) v -= L[i * n + k] * e[k];
          e[i] = v / L[i * n + i];
        }
        for (int i = n - 1; i >= 0; i--) {
          double v = e[i];
          for (int k = i + 1; k < n; k++) v -= L[k * n + i] * e[k];
          e[i] = v / L[i * n + i];
        }
        for (int i = 0; i < n; i++) minv[i * n + col] = e[i];
      }
      free(e);
    }
  }
  free(M); free(L); free(b); free(c); free(T);
  return out;
}

/* ---- emission lines (App. C, App. "line_proj", Eq. "app_line_profile") ---- */

/* App. D normalisation of band b (samples from off): Z_b, the trapezoid of
 * lam R c AB / lam^2, as in orc_photometry. */
static double band_norm(const orc_model *md, int b, int off) {
  int n = md->filt_len[b];
  const double *L = md->filt_lam + off, *R = md->filt_trans + off;
  double zb = 0.0;
  for (int j = 0; j + 1 < n; j++) {
    double g0 = L[j] * R[j] * O_C_AA * O_AB / (L[j] * L[j]);
    double g1 = L[j + 1] * R[j + 1] * O_C_AA * O_AB / (L[j + 1] * L[j + 1]);
    zb += 0.5 * (g0 + g1) * (L[j + 1] - L[j]);
  }
  return zb;
}

/* Transmission of band b at observed wavelength x: linear between its
 * samples, zero outside them. */
static double band_trans(const orc_model *md, int b, int off, double x) {
  int n = md->filt_len[b];
  const double *L = md->filt_lam + off, *R = md->filt_trans + off;
  if (!(x >= L[0] && x <= L[n - 1])) return 0.0;
  for (int j = 0; j + 1 < n; j++)
    if (x >= L[j] && x <= L[j + 1]) return R[j] + (R[j + 1] - R[j]) * (x - L[j]) / (L[j + 1] - L[j]);
  return 0.0;
}

/* Instrumental dispersion (km/s) at observed wavelength x: the spectrum's LSF
 * at its pixels, linear in wavelength between them, constant past the ends. */
static double sigma_inst_at(const orc_model *md, double x) {
  int n = md->n_pix;
  if (x <= md->spec_lam[0]) return sigma_inst_kms(md->lsf_mode, md->lsf_value[0], md->spec_lam[0]);
  if (x >= md->spec_lam[n - 1]) return sigma_inst_kms(md->lsf_mode, md->lsf_value[n - 1], md->spec_lam[n - 1]);
  int i = 0;
  while (i + 2 < n && md->spec_lam[i + 1] <= x) i++;
  double a = sigma_inst_kms(md->lsf_mode, md->lsf_value[i], md->spec_lam[i]);
  double b = sigma_inst_kms(md->lsf_mode, md->lsf_value[i + 1], md->spec_lam[i + 1]);
  return a + (b - a) * (x - md->spec_lam[i]) / (md->spec_lam[i + 1] - md->spec_lam[i]);
}

/* Observer-frame integrated flux of every grid line, erg/s/cm^2 (App.
 * "line_proj"): L = Q_young 10^(bilinear log10 line table at (log U, log
 * Z_gas)) (App. C, the same interpolation as the nebular continuum), through
 * the attenuation the nebular continuum meets at the line's wavelength
 * (birth cloud and diffuse screen, Eq. "app_attn"; with an escape geometry
 * the covered fraction 1 - f_ob as in Sec. "frac_obrun"), times
 * scale = 10^logmass Lsun / (4 pi D_L^2): the flux factor of Sec. 2.6 without
 * its (1+z), since an integrated flux has no bandwidth. */
static void line_fluxes(const orc_grid *g, const orc_model *md, const orc_theta *t, double qy, double scale,
                        double *Fl) {
  int u0, u1, z0, z1;
  double wu0, wu1, wz0, wz1;
  bracket(g->neb_logu, g->neb_n_logu, t->gas_logu, &u0, &wu0, &u1, &wu1);
  bracket(g->neb_logz, g->neb_n_logz, t->gas_logz, &z0, &wz0, &z1, &wz1);
  int NLn = g->neb_n_line, NZg = g->neb_n_logz;
  for (int l = 0; l < NLn; l++) {
    double lg = wu0 * wz0 * g->neb_line_tab[((size_t)u0 * NZg + z0) * NLn + l] +
                wu0 * wz1 * g->neb_line_tab[((size_t)u0 * NZg + z1) * NLn + l] +
                wu1 * wz0 * g->neb_line_tab[((size_t)u1 * NZg + z0) * NLn + l] +
                wu1 * wz1 * g->neb_line_tab[((size_t)u1 * NZg + z1) * NLn + l];
    double lam = g->neb_line_lam[l], td = 0.0;
    orc_dust_tau(md->dust_law, &lam, 1, t->tau_d, t->delta, &td);
    double ed = exp(-td), eb = exp(-t->tau_bc * pow(lam / 5500.0, t->alpha_bc)), f = t->fob, fac;
    if (md->fesc_geometry == ORC_FESC_PICKET) fac = ed * (1.0 - f) * eb;
    else fac = ed * ((1.0 - f) * eb + f) * (1.0 - f);
    Fl[l] = qy * pow(10.0, lg) * fac * scale;
  }
}

/* Whether SSP age node a powers the nebular emission (App. C): a birth-cloud
 * age, and with a nebular age axis one inside the cube's tabulated ages. */
static int nebular_age(const orc_grid *g, const orc_model *md, int a) {
  if (!md->use_nebular || !g->neb_tab) return 0;
  const double la = g->log_age_yr[a];
  if (la > md->bc_edge_log_age_yr) return 0;
  if (g->neb_n_age <= 0) return 1;
  return la >= g->neb_log_age[0] && la <= g->neb_log_age[g->neb_n_age - 1];
}

/* One parameter row through the whole forward model and likelihood. */
int orc_row(const orc_grid *g, const orc_model *md, const double *theta, double *W_out,
            double *Y_out, double *O_out, double *F_out, double *fnu_out, double *phot,
            double *spec, double *scal) {
  int NA = g->n_age, NL = g->n_lam, NZ = g->n_feh, NAF = g->n_afe;
  size_t nsp = (size_t)NAF * NZ * NA;
  double *W = (double *)malloc(nsp * sizeof(double));
  double *Q = (double *)malloc(nsp * sizeof(double));
  double *Y = (double *)calloc(NL, sizeof(double));
  double *O = (double *)calloc(NL, sizeof(double));
  double *F = (double *)malloc(NL * sizeof(double));
  double *YL = (double *)calloc(NL, sizeof(double)); /* young ionising continuum (nebular ages, < 912 A) */
  double *N = (double *)calloc(NL, sizeof(double));  /* nebular continuum */
  double *fnu = (double *)malloc(NL * sizeof(double));
  double *tbc = (double *)malloc(NL * sizeof(double));
  double *td = (double *)malloc(NL * sizeof(double));
  double cosm[2] = {0, 0}, tmax = 0;
  int st = theta_status(md, theta, &tmax, cosm);
  int st_w = orc_weights(g, md, theta, W);
  if (!st) st = st_w;
  double lnl = -INFINITY;
  orc_theta t;
  decode_theta(md, theta, &t);
  if (!st) {
    orc_q(g, Q);
    double qy = 0.0;
    double *qa = (double *)calloc(NA, sizeof(double));   /* Q-weighted weight of each nebular age */
    if (md->dust_n_bin > 0) {
      /* App. "dust_attn": per age node a the optical depth tau_a = sum_b M_ab
       * kappa_b(lam; theta_b) (Eq. "app_tau_bin"), applied to the node's
       * stellar plus nebular light inside the contraction and followed by the
       * diffuse screen (Eq. "app_attn"); nebular ages lose their stellar flux
       * below 912 A and carry Q_ma 10^(bilinear log10 template) instead */
      const int nb = md->dust_n_bin;
      double *kap = (double *)malloc((size_t)nb * NL * sizeof(double));
      double *shp = (double *)malloc(NL * sizeof(double));
      double *att = (double *)malloc(NL * sizeof(double));
      for (int b = 0; b < nb; b++) orc_dust_tau(md->dust_bin_law[b], g->lam, NL, t.bin_tau[b], t.bin_slope[b], kap + (size_t)b * NL);
      const int has_neb = md->use_nebular && g->neb_tab;
      if (has_neb) {
        int u0, u1, z0, z1;
        double wu0, wu1, wz0, wz1;
        bracket(g->neb_logu, g->neb_n_logu, t.gas_logu, &u0, &wu0, &u1, &wu1);
        bracket(g->neb_logz, g->neb_n_logz, t.gas_logz, &z0, &wz0, &z1, &wz1);
        const double *t00 = g->neb_tab + ((size_t)u0 * g->neb_n_logz + z0) * NL;
        const double *t01 = g->neb_tab + ((size_t)u0 * g->neb_n_logz + z1) * NL;
        const double *t10 = g->neb_tab + ((size_t)u1 * g->neb_n_logz + z0) * NL;
        const double *t11 = g->neb_tab + ((size_t)u1 * g->neb_n_logz + z1) * NL;
        for (int k = 0; k < NL; k++)
          shp[k] = pow(10.0, wu0 * wz0 * t00[k] + wu0 * wz1 * t01[k] + wu1 * wz0 * t10[k] + wu1 * wz1 * t11[k]);
      }
      for (int k = 0; k < NL; k++) F[k] = 0.0;
      for (int a = 0; a < NA; a++) {
        for (int k = 0; k < NL; k++) {
          double tau = 0.0;
          for (int b = 0; b < nb; b++) tau += md->dust_bin_M[(size_t)a * nb + b] * kap[(size_t)b * NL + k];
          att[k] = exp(-tau);
        }
        const int neb = has_neb && g->log_age_yr[a] <= md->bc_edge_log_age_yr;
        for (int n = 0; n < NAF; n++)
          for (int m = 0; m < NZ; m++) {
            size_t s = ((size_t)n * NZ + m) * NA + a;
            double w = W[s];
            if (w == 0.0) continue;
            const double *f = g->flux + s * NL;
            for (int k = 0; k < NL; k++) {
              double v = (neb && g->lam[k] < O_LYMAN) ? 0.0 : f[k];
              if (neb) v += Q[s] * shp[k];
              F[k] += w * v * att[k];
              (g->log_age_yr[a] <= md->bc_edge_log_age_yr ? Y : O)[k] += w * v;
            }
            if (g->log_age_yr[a] <= md->bc_edge_log_age_yr) qy += w * Q[s];
          }
      }
      orc_dust_tau(md->dust_law, g->lam, NL, t.tau_d, t.delta, td);
      for (int k = 0; k < NL; k++) F[k] *= exp(-td[k]);
      free(kap); free(shp); free(att);
    } else {
    /* contraction, Eq. "csp_sum_main" split into birth-cloud (young) and
     * older ages (Eq. "app_attn" with a two-bin age-to-bin matrix); the
     * stellar flux below 912 A of nebular ages is removed (App. A, Fig. flow) */
    for (int n = 0; n < NAF; n++)
      for (int m = 0; m < NZ; m++)
        for (int a = 0; a < NA; a++) {
          size_t s = ((size_t)n * NZ + m) * NA + a;
          double w = W[s];
          if (w == 0.0) continue; /* exact zero contributes nothing */
          const double *f = g->flux + s * NL;
          int young = g->log_age_yr[a] <= md->bc_edge_log_age_yr;
          int neb = nebular_age(g, md, a);
          double *acc = young ? Y : O;
          for (int k = 0; k < NL; k++) {
            if (neb && g->lam[k] < O_LYMAN) YL[k] += w * f[k];
            else acc[k] += w * f[k];
          }
          if (g->neb_n_age > 0 ? neb : young) qy += w * Q[s];
          if (neb) qa[a] += w * Q[s];
        }
    /* nebular continuum, App. C: Q_young * 10^(bilinear log10 template); with
     * an age axis, each nebular SSP age a contributes Q_a 10^(the cube
     * interpolated trilinearly: bilinear in (log U, log Z_gas) on the two
     * planes of ionising-source age bracketing the node's age, linear in log
     * age between them) */
    if (md->use_nebular && g->neb_tab && g->neb_n_age > 0) {
      int u0, u1, z0, z1;
      double wu0, wu1, wz0, wz1;
      bracket(g->neb_logu, g->neb_n_logu, t.gas_logu, &u0, &wu0, &u1, &wu1);
      bracket(g->neb_logz, g->neb_n_logz, t.gas_logz, &z0, &wz0, &z1, &wz1);
      const size_t plane = (size_t)g->neb_n_logu * g->neb_n_logz * NL;
      for (int a = 0; a < NA; a++) {
        if (qa[a] == 0.0) continue;
        int i0, i1;
        double wa0, wa1;
        bracket(g->neb_log_age, g->neb_n_age, g->log_age_yr[a], &i0, &wa0, &i1, &wa1);
        for (int k = 0; k < NL; k++) {
          double lg = 0.0;
          for (int e = 0; e < 2; e++) {
            const double we = e ? wa1 : wa0;
            if (we == 0.0) continue;
            const double *b = g->neb_tab + (size_t)(e ? i1 : i0) * plane;
            lg += we * (wu0 * wz0 * b[((size_t)u0 * g->neb_n_logz + z0) * NL + k] +
                        wu0 * wz1 * b[((size_t)u0 * g->neb_n_logz + z1) * NL + k] +
                        wu1 * wz0 * b[((size_t)u1 * g->neb_n_logz + z0) * NL + k] +
                        wu1 * wz1 * b[((size_t)u1 * g->neb_n_logz + z1) * NL + k]);
          }
          N[k] += qa[a] * pow(10.0, lg);
        }
      }
    } else if (md->use_nebular && g->neb_tab) {
      int u0, u1, z0, z1;
      double wu0, wu1, wz0, wz1;
      bracket(g->neb_logu, g->neb_n_logu, t.gas_logu, &u0, &wu0, &u1, &wu1);
      bracket(g->neb_logz, g->neb_n_logz, t.gas_logz, &z0, &wz0, &z1, &wz1);
      const double *t00 = g->neb_tab + ((size_t)u0 * g->neb_n_logz + z0) * NL;
      const double *t01 = g->neb_tab + ((size_t)u0 * g->neb_n_logz + z1) * NL;
      const double *t10 = g->neb_tab + ((size_t)u1 * g->neb_n_logz + z0) * NL;
      const double *t11 = g->neb_tab + ((size_t)u1 * g->neb_n_logz + z1) * NL;
      for (int k = 0; k < NL; k++) {
        double lg = wu0 * wz0 * t00[k] + wu0 * wz1 * t01[k] + wu1 * wz0 * t10[k] + wu1 * wz1 * t11[k];
        N[k] = qy * pow(10.0, lg);
      }
    }
    /* two-component dust (Sec. 2.4) */
    for (int k = 0; k < NL; k++) tbc[k] = t.tau_bc * pow(g->lam[k] / 5500.0, t.alpha_bc);
    orc_dust_tau(md->dust_law, g->lam, NL, t.tau_d, t.delta, td);
    /* Eq. "app_attn" with the escape geometries of Sec. "frac_obrun".  The
     * covered fraction 1 - f_ob powers the nebular continuum; the ionising
     * continuum of the nebular ages is absorbed except for the fraction f_ob
     * that escapes, which bypasses the birth cloud.  runaway_bc: the young
     * array (stellar + nebular continuum) crosses T = (1 - f_ob) e^{-tau_BC} +
     * f_ob, then everything the diffuse screen.  picket: f_ob of the young
     * stellar light, ionising continuum included, escapes both screens; the
     * rest crosses both.  f_ob = 0 (or no geometry) is Eq. "app_attn". */
    const double fob = t.fob;
    for (int k = 0; k < NL; k++) {
      const double ed = exp(-td[k]), eb = exp(-tbc[k]);
      if (md->fesc_geometry == ORC_FESC_PICKET) {
        F[k] = fob * (Y[k] + YL[k]) + ed * ((1.0 - fob) * eb * (Y[k] + N[k]) + O[k]);
      } else {
        const double T = (1.0 - fob) * eb + fob;
        F[k] = ed * (T * (Y[k] + (1.0 - fob) * N[k]) + fob * YL[k] + O[k]);
      }
      Y[k] += N[k];   /* Y_out: young stellar flux (ionising continuum removed) plus nebular */
    }
    }
    free(qa);
    /* observer frame, Sec. 2.6 */
    double dl = cosm[0] > 10.0 * O_PC_CM ? cosm[0] : 10.0 * O_PC_CM;
    double scale = pow(10.0, t.logmass) * O_LSUN * (1.0 + t.z) / (4.0 * M_PI * dl * dl);
    for (int k = 0; k < NL; k++) fnu[k] = scale * F[k];
    /* the IGM transmission at each node's observed wavelength (Sec. 2.6) */
    if (md->use_igm)
      for (int k = 0; k < NL; k++) fnu[k] *= exp(-t.igm_f * igm_madau_tau(g->lam[k], t.z));
    /* the grid's emission lines, App. "line_proj" (through the same IGM transmission) */
    const int nline = (md->use_lines && md->use_nebular && g->neb_line_tab) ? g->neb_n_line : 0;
    double *Fl = (double *)calloc(nline > 0 ? nline : 1, sizeof(double));
    if (nline) line_fluxes(g, md, &t, qy, pow(10.0, t.logmass) * O_LSUN / (4.0 * M_PI * dl * dl), Fl);
    if (nline && md->use_igm)
      for (int l = 0; l < nline; l++) Fl[l] *= exp(-t.igm_f * igm_madau_tau(g->neb_line_lam[l], t.z));
    /* projections + likelihood, Eq. "total_lnlike" */
    double *ph = (double *)malloc((md->n_filt > 0 ? md->n_filt : 1) * sizeof(double));
    double *sp = (double *)malloc((md->n_pix > 0 ? md->n_pix : 1) * sizeof(double));
    unsigned char *vd = (unsigned char *)malloc(md->n_pix > 0 ? md->n_pix : 1);
    lnl = 0.0;
    if (md->n_filt > 0) {
      orc_photometry(md, g->lam, NL, t.z, fnu, ph);
      /* a line in a band: its integrated flux at its observed wavelength
       * through the band's photon-counting response, F R_b(lam_obs) lam_obs / Z_b
       * (App. D; the limit of a line much narrower than the band) */
      for (int b = 0, off = 0; b < md->n_filt; off += md->filt_len[b], b++)
        for (int l = 0; l < nline; l++) {
          double xo = g->neb_line_lam[l] * (1.0 + t.z);
          ph[b] += Fl[l] * band_trans(md, b, off, xo) * xo / band_norm(md, b, off);
        }
      for (int b = 0; b < md->n_filt; b++) {
        if (phot) phot[b] = ph[b];
        if (md->phot_d && (!md->phot_mask || md->phot_mask[b])) {
          /* Eq. "total_lnlike" with sigma_eff of Eq. "app_noise_floor" (= sigma without a floor) */
          double v = eff_var(t.fl[0], md->phot_sigma[b], ph[b], md->phot_d[b]);
          double r = phot_residual(md, b, md->phot_d[b], ph[b]);
          lnl += -0.5 * r * r / v - 0.5 * log(2.0 * M_PI * v);
        }
      }
    }
    if (md->n_pix > 0) {
      orc_spectrum(g, md, g->lam, NL, t.z, t.sigma_gal, fnu, sp, vd);
      /* Eq. "app_line_profile": each line a unit-area Gaussian in ln(lambda) of
       * width s = sqrt(sigma_gas^2 + sigma_inst^2(lam_obs)) / c, sampled at the
       * pixel centres (truncated at 5 s, not renormalised), as a flux density
       * per unit frequency through lambda / c */
      for (int l = 0; l < nline; l++) {
        double xo = g->neb_line_lam[l] * (1.0 + t.z), si = sigma_inst_at(md, xo);
        double s = sqrt(t.sigma_gas * t.sigma_gas + si * si) / O_C_KMS;
        if (!(s > 0.0)) continue;
        for (int i = 0; i < md->n_pix; i++) {
          double u = (log(md->spec_lam[i]) - log(xo)) / s;
          if (fabs(u) > 5.0) continue;
          sp[i] += Fl[l] * (md->spec_lam[i] / O_C_AA) * exp(-0.5 * u * u) / (sqrt(2.0 * M_PI) * s);
        }
      }
      unsigned char *inc = (unsigned char *)calloc(md->n_pix, 1);
      for (int i = 0; i < md->n_pix; i++) {
        if (spec) spec[i] = sp[i];
        if (md->spec_d && vd[i] && (!md->spec_mask || md->spec_mask[i])) {
          double v = eff_var(t.fl[1], md->spec_sigma[i], sp[i], md->spec_d[i]), r = md->spec_d[i] - sp[i];
          lnl += -0.5 * r * r / v - 0.5 * log(2.0 * M_PI * v);
          inc[i] = 1;
        }
      }
      if (md->calib_n > 0 && md->spec_d) lnl += calib_terms(md, sp, inc, NULL, NULL);
      free(inc);
    }
    /* the line-catalogue arm (Sec. 3.3, App. "line_lik"): a blend's model is the
     * sum of its grid lines' fluxes; detections by Eq. "app_line_chi2_det",
     * upper limits by the one-sided Eq. "app_line_chi2_UL" (residual 0 while
     * the model stays at or below the limit); the normalisation of every
     * included entry is kept, as in Eq. "total_lnlike" */
    for (int k = 0; k < md->n_lcat; k++) {
      double m = 0.0;
      for (int j = md->lcat_start[k]; j < md->lcat_start[k + 1]; j++) m += nline ? Fl[md->lcat_line[j]] : 0.0;
      if (md->lcat_mask && !md->lcat_mask[k]) continue;
      double d = md->lcat_d[k], sg = md->lcat_sigma[k];
      double r = (md->lcat_upper && md->lcat_upper[k] && m <= d) ? 0.0 : d - m;
      lnl += -0.5 * r * r / (sg * sg) - 0.5 * log(2.0 * M_PI * sg * sg);
    }
    if (!isfinite(lnl)) { st = ORC_NONFINITE; lnl = -INFINITY; }
    if (scal) { scal[0] = cosm[0]; scal[1] = cosm[1]; scal[2] = tmax; scal[3] = qy; scal[4] = scale; }
    free(ph); free(sp); free(vd); free(Fl);
  }
  if (st) {
    if (phot) for (int b = 0; b < md->n_filt; b++) phot[b] = 0.0;
    if (spec) for (int i = 0; i < md->n_pix; i++) spec[i] = 0.0;
  }
  if (scal) scal[5] = lnl;
  if (W_out) memcpy(W_out, W, nsp * sizeof(double));
  if (Y_out) memcpy(Y_out, Y, NL * sizeof(double));
  if (O_out) memcpy(O_out, O, NL * sizeof(double));
  if (F_out) memcpy(F_out, F, NL * sizeof(double));
  if (fnu_out) memcpy(fnu_out, fnu, NL * sizeof(double));
  free(W); free(Q); free(Y); free(O); free(F); free(YL); free(N); free(fnu); free(tbc); free(td);
  return st;
}

void orc_eval(const orc_grid *g, const orc_model *md, const double *theta, int n, int ld,
              double *phot_out, double *spec_out, double *lnl_out, int *status_out,
              int nthreads) {
#ifdef _OPENMP
  int nt = nthreads > 0 ? nthreads : omp_get_max_threads();
#pragma omp parallel for num_threads(nt) schedule(dynamic, 1)
#endif
  for (int r = 0; r < n; r++) {
    double scal[6];
    int st = orc_row(g, md, theta + (size_t)r * ld, NULL, NULL, NULL, NULL, NULL,
                     phot_out ? phot_out + (size_t)r * md->n_filt : NULL,
                     spec_out ? spec_out + (size_t)r * md->n_pix : NULL, scal);
    if (lnl_out) lnl_out[r] = st ? -INFINITY : scal[5];
    if (status_out) status_out[r] = st;
  }
  (void)nthreads;
}

void orc_line_fluxes(const orc_grid *g, const orc_model *md, const double *theta, int n, int ld, double *out) {
  int nl = g->neb_n_line > 0 ? g->neb_n_line : 0;
  for (int r = 0; r < n; r++) {
    const double *th = theta + (size_t)r * ld;
    double scal[6];
    int st = orc_row(g, md, th, NULL, NULL, NULL, NULL, NULL, NULL, NULL, scal);
    double *o = out + (size_t)r * nl;
    for (int l = 0; l < nl; l++) o[l] = 0.0;
    if (st || !nl || !g->neb_line_tab || !md->use_nebular) continue;
    orc_theta t;
    decode_theta(md, th, &t);
    double dl = scal[0] > 10.0 * O_PC_CM ? scal[0] : 10.0 * O_PC_CM;
    line_fluxes(g, md, &t, scal[3], pow(10.0, t.logmass) * O_LSUN / (4.0 * M_PI * dl * dl), o);
    if (md->use_igm)
      for (int l = 0; l < nl; l++) o[l] *= exp(-t.igm_f * igm_madau_tau(g->neb_line_lam[l], t.z));
  }
}

void orc_grad_fd(const orc_grid *g, const orc_model *md, const double *theta, int n, int ld,
                 double h_rel, double *grad_out, int nthreads) {
  int np = orc_n_param(md);
#ifdef _OPENMP
  int nt = nthreads > 0 ? nthreads : omp_get_max_threads();
#pragma omp parallel for num_threads(nt) schedule(dynamic, 1) collapse(2)
#endif
  for (int r = 0; r < n; r++) {
    for (int j = 0; j < np; j++) {
      double *x = (double *)malloc(np * sizeof(double));
      memcpy(x, theta + (size_t)r * ld, np * sizeof(double));
      double x0 = x[j];
      double h = h_rel * (fabs(x0) > 1.0 ? fabs(x0) : 1.0);
      double sp[6], sm[6];
      x[j] = x0 + h;
      int a = orc_row(g, md, x, NULL, NULL, NULL, NULL, NULL, NULL, NULL, sp);
      x[j] = x0 - h;
      int b = orc_row(g, md, x, NULL, NULL, NULL, NULL, NULL, NULL, NULL, sm);
      grad_out[(size_t)r * ld + j] = (a || b) ? NAN : (sp[5] - sm[5]) / (2.0 * h);
      free(x);
    }
  }
  (void)nthreads;
}

/* ------------------------------------------------------------------ */
/* Analytic gradient of lnL with respect to every parameter (FP64).     */
/* ------------------------------------------------------------------ */
/* Bracket of v on the node array x with the derivatives of the two weights
 * with respect to v (zero where the value is clamped or the axis has one node). */
static void bracket_d(const double *x, int n, double v, int *j0, double *w0, double *d0, int *j1,
                      double *w1, double *d1) {
  bracket(x, n, v, j0, w0, j1, w1);
  *d0 = *d1 = 0.0;
  if (n > 1 && v > x[0] && v < x[n - 1]) {
    double h = x[*j1] - x[*j0];
    *d0 = -1.0 / h;
    *d1 = 1.0 / h;
  }
}

/* Reverse pass of orc_row: the derivative of lnL (Eq. "total_lnlike") with
 * respect to each parameter column, by the chain rule taken step by step
 * backwards through the same definitions (likelihood -> projections -> observer
 * frame -> dust and nebular -> contraction -> weights -> SFH edges -> cosmology).
 * Everything is piecewise smooth; at a kink (a bracket node, a Voronoi cell
 * edge, an interpolation node) the one-sided derivative of the branch the
 * forward pass took is returned.  grad[n_param]; returns the row status
 * (grad = 0 when it is not 0) and lnL in *lnl. */
int orc_row_grad(const orc_grid *g, const orc_model *md, const double *theta, double *grad, double *lnl) {
  int NA = g->n_age, NL = g->n_lam, NZ = g->n_feh, NAF = g->n_afe, NT = md->n_sfh;
  int np = orc_n_param(md);
  for (int j = 0; j < np; j++) grad[j] = 0.0;
  *lnl = -INFINITY;
  double cz[3], cf[3], tmax;
  int st = theta_status(md, theta, &tmax, NULL);
  if (st) return st;
  orc_theta t;
  decode_theta(md, theta, &t);
  orc_cosmology(md->H0, md->Om0, t.z, cz);
  orc_cosmology(md->H0, md->Om0, md->zf, cf);
  double zp = 1.0 + t.z;
  size_t nsp = (size_t)NAF * NZ * NA;

  /* ---------------- forward, keeping what the reverse pass needs */
  double *T = (double *)malloc((NT + 1) * sizeof(double));
  double *cm = (double *)malloc(NA * sizeof(double));
  double *cp = (double *)malloc(NA * sizeof(double));
  double *A = (double *)calloc((size_t)NT * NA, sizeof(double));
  int *zm0 = (int *)malloc(NT * sizeof(int)), *zm1 = (int *)malloc(NT * sizeof(int));
  double *wz0 = (double *)malloc(NT * sizeof(double)), *wz1 = (double *)malloc(NT * sizeof(double));
  double *dz0 = (double *)malloc(NT * sizeof(double)), *dz1 = (double *)malloc(NT * sizeof(double));
  double *W = (double *)calloc(nsp, sizeof(double));
  double *Q = (double *)malloc(nsp * sizeof(double));
  double *Y = (double *)calloc(NL, sizeof(double)), *O = (double *)calloc(NL, sizeof(double));
  double *neb = (double *)calloc(NL, sizeof(double)), *lg = (double *)calloc(NL, sizeof(double));
  double *YL = (double *)calloc(NL, sizeof(double)); /* young ionising continuum (nebular ages, < 912 A) */
  double *tbc = (double *)malloc(NL * sizeof(double)), *td = (double *)malloc(NL * sizeof(double));
  double *F = (double *)malloc(NL * sizeof(double)), *fnu = (double *)malloc(NL * sizeof(double));
  double *gfnu = (double *)calloc(NL, sizeof(double));
  double *gW = (double *)calloc(nsp, sizeof(double));

  orc_sfh_edges(NT, tmax, T);
  for (int a = 0; a < NA; a++) {
    double ta = pow(10.0, g->log_age_yr[a]);
    cm[a] = (a == 0) ? 0.0 : 0.5 * (pow(10.0, g->log_age_yr[a - 1]) + ta);
    cp[a] = (a == NA - 1) ? INFINITY : 0.5 * (ta + pow(10.0, g->log_age_yr[a + 1]));
  }
  int an0, an1;
  double wa0, wa1, da0, da1;
  bracket_d(g->afe, NAF, md->use_afe ? t.afe : 0.0, &an0, &wa0, &da0, &an1, &wa1, &da1);
  if (!md->use_afe) da0 = da1 = 0.0;
  for (int i = 0; i < NT; i++) {
    double dT = T[i + 1] - T[i];
    bracket_d(g->feh, NZ, t.zeta[md->zmode == 0 ? i : 0], &zm0[i], &wz0[i], &dz0[i], &zm1[i], &wz1[i], &dz1[i]);
    if (md->sfh_scheme == 1) linear_bin_masses(g, T[i], T[i + 1], t.m[i], t.m[i + 1], A + (size_t)i * NA);
    for (int a = 0; a < NA; a++) {
      double Aia;
      if (md->sfh_scheme == 1) {
        Aia = A[(size_t)i * NA + a];
        if (Aia == 0.0) continue;
      } else {
        double lo = T[i] > cm[a] ? T[i] : cm[a];
        double hi = T[i + 1] < cp[a] ? T[i + 1] : cp[a];
        if (hi - lo <= 0.0) continue;
        Aia = t.m[i] * (hi - lo) / dT;
        A[(size_t)i * NA + a] = Aia;
      }
      W[((size_t)an0 * NZ + zm0[i]) * NA + a] += Aia * wz0[i] * wa0;
      W[((size_t)an0 * NZ + zm1[i]) * NA + a] += Aia * wz1[i] * wa0;
      W[((size_t)an1 * NZ + zm0[i]) * NA + a] += Aia * wz0[i] * wa1;
      W[((size_t)an1 * NZ + zm1[i]) * NA + a] += Aia * wz1[i] * wa1;
    }
  }
  orc_q(g, Q);
  double qy = 0.0;
  int has_neb = md->use_nebular && g->neb_tab;
  for (size_t s = 0; s < nsp; s++) {
    int a = (int)(s % NA);
    int young = g->log_age_yr[a] <= md->bc_edge_log_age_yr;
    if (W[s] == 0.0) continue;
    const double *f = g->flux + s * NL;
    for (int k = 0; k < NL; k++) {
      if (young && has_neb && g->lam[k] < O_LYMAN) YL[k] += W[s] * f[k];
      else (young ? Y : O)[k] += W[s] * f[k];
    }
    if (young) qy += W[s] * Q[s];
  }
  int u0 = 0, u1 = 0, zz0 = 0, zz1 = 0;
  double wu0 = 0, wu1 = 0, du0 = 0, du1 = 0, wg0 = 0, wg1 = 0, dg0 = 0, dg1 = 0;
  const double *t00 = NULL, *t01 = NULL, *t10 = NULL, *t11 = NULL;
  if (has_neb) {
    bracket_d(g->neb_logu, g->neb_n_logu, t.gas_logu, &u0, &wu0, &du0, &u1, &wu1, &du1);
    bracket_d(g->neb_logz, g->neb_n_logz, t.gas_logz, &zz0, &wg0, &dg0, &zz1, &wg1, &dg1);
    t00 = g->neb_tab + ((size_t)u0 * g->neb_n_logz + zz0) * NL;
    t01 = g->neb_tab + ((size_t)u0 * g->neb_n_logz + zz1) * NL;
    t10 = g->neb_tab + ((size_t)u1 * g->neb_n_logz + zz0) * NL;
    t11 = g->neb_tab + ((size_t)u1 * g->neb_n_logz + zz1) * NL;
    for (int k = 0; k < NL; k++) {
      lg[k] = wu0 * wg0 * t00[k] + wu0 * wg1 * t01[k] + wu1 * wg0 * t10[k] + wu1 * wg1 * t11[k];
      neb[k] = qy * pow(10.0, lg[k]);
    }
  }
  for (int k = 0; k < NL; k++) tbc[k] = t.tau_bc * pow(g->lam[k] / 5500.0, t.alpha_bc);
  orc_dust_tau(md->dust_law, g->lam, NL, t.tau_d, t.delta, td);
  /* Eq. "app_attn" with the escape geometry of Sec. "frac_obrun" (as in orc_row) */
  const double fob = t.fob;
  for (int k = 0; k < NL; k++) {
    const double ed = exp(-td[k]), eb = exp(-tbc[k]);
    if (md->fesc_geometry == ORC_FESC_PICKET)
      F[k] = fob * (Y[k] + YL[k]) + ed * ((1.0 - fob) * eb * (Y[k] + neb[k]) + O[k]);
    else
      F[k] = ed * (((1.0 - fob) * eb + fob) * (Y[k] + (1.0 - fob) * neb[k]) + fob * YL[k] + O[k]);
  }
  double dl = cz[0], ddl = cz[2] + zp * (O_C_KMS / md->H0 * 1e6 * O_PC_CM) * inv_E(t.z, &md->Om0);
  if (dl < 10.0 * O_PC_CM) { dl = 10.0 * O_PC_CM; ddl = 0.0; }
  double scale = pow(10.0, t.logmass) * O_LSUN * zp / (4.0 * M_PI * dl * dl);
  double dlns_dz = 1.0 / zp - 2.0 * ddl / dl;
  for (int k = 0; k < NL; k++) fnu[k] = scale * F[k];

  /* ---------------- likelihood and its derivative with respect to the model */
  double L = 0.0, gscale = 0.0, gz = 0.0, g_sgal = 0.0;
  /* noise floor (Eq. "app_noise_floor"): d lnL / d log10 of each term, per arm */
  double gfl[2][4] = {{0, 0, 0, 0}, {0, 0, 0, 0}};
  if (md->n_filt > 0) {
    double *ph = (double *)malloc(md->n_filt * sizeof(double));
    orc_photometry(md, g->lam, NL, t.z, fnu, ph);
    int off = 0;
    for (int b = 0; b < md->n_filt; b++) {
      int n = md->filt_len[b];
      const double *Lf = md->filt_lam + off, *R = md->filt_trans + off;
      off += n;
      double ub = 0.0;
      if (md->phot_d && (!md->phot_mask || md->phot_mask[b])) {
        double d = md->phot_d[b], m = ph[b], sg = md->phot_sigma[b];
        double v = eff_var(t.fl[0], sg, m, d), r = phot_residual(md, b, d, m);
        L += -0.5 * r * r / v - 0.5 * log(2.0 * M_PI * v);
        ub = floor_terms_grad(t.fl[0], v, r, sg, m, d, gfl[0]);
      }
      if (ub == 0.0) continue;
      /* m_b = sum_j R_j x_j dl_j flam(x_j) / Z_b (App. D), as in orc_photometry */
      double zb = 0.0;
      for (int j = 0; j + 1 < n; j++) {
        double g0 = Lf[j] * R[j] * O_C_AA * O_AB / (Lf[j] * Lf[j]);
        double g1 = Lf[j + 1] * R[j + 1] * O_C_AA * O_AB / (Lf[j + 1] * Lf[j + 1]);
        zb += 0.5 * (g0 + g1) * (Lf[j + 1] - Lf[j]);
      }
      double lo = zp * g->lam[0], hi = zp * g->lam[NL - 1];
      for (int j = 0; j < n; j++) {
        double dlj;
        if (n == 1) dlj = 0.0;
        else if (j == 0) dlj = 0.5 * (Lf[1] - Lf[0]);
        else if (j == n - 1) dlj = 0.5 * (Lf[n - 1] - Lf[n - 2]);
        else dlj = 0.5 * (Lf[j + 1] - Lf[j - 1]);
        double x = Lf[j];
        if (!(x >= lo && x <= hi)) continue;
        int k = 0, kh = NL - 1;
        while (kh - k > 1) {
          int mid = (k + kh) / 2;
          if (zp * g->lam[mid] <= x) k = mid; else kh = mid;
        }
        double xa = zp * g->lam[k], xb = zp * g->lam[k + 1];
        double tt = (x - xa) / (xb - xa);
        double ga = O_C_AA * fnu[k] / (xa * xa), gb = O_C_AA * fnu[k + 1] / (xb * xb);
        double c = ub * R[j] * x * dlj / zb;
        gfnu[k] += c * (1.0 - tt) * O_C_AA / (xa * xa);
        gfnu[k + 1] += c * tt * O_C_AA / (xb * xb);
        /* the gather position moves with z: xa, xb = (1+z) lam */
        double dflam = (1.0 - tt) * (-2.0 * ga / zp) + tt * (-2.0 * gb / zp) +
                       (gb - ga) * (-x / (zp * zp * (g->lam[k + 1] - g->lam[k])));
        gz += c * dflam;
      }
    }
    free(ph);
  }
  if (md->n_pix > 0) {
    double *sp = (double *)malloc(md->n_pix * sizeof(double));
    unsigned char *vd = (unsigned char *)malloc(md->n_pix);
    double *s_ln = (double *)malloc(md->n_pix * sizeof(double));
    double *ll = (double *)malloc(NL * sizeof(double));
    orc_spectrum(g, md, g->lam, NL, t.z, t.sigma_gal, fnu, sp, vd);
    spec_widths(g, md, t.sigma_gal, s_ln);
    for (int k = 0; k < NL; k++) ll[k] = log(g->lam[k]);
    double lz = log(zp);
    /* marginalised calibration polynomial: its lnL terms, and for every pixel
     * d lnL / d mu_i = [(d_i - mu_i (1 + p_i)) (1 + p_i) - mu_i q_i] / sigma_i^2
     * with p_i = sum_m c*_m T_m(x_i) (c* = M^-1 b) and q_i = T(x_i)^T M^-1 T(x_i) */
    int nc = (md->calib_n > 0 && md->spec_d) ? md->calib_n : 0;
    double *minv = NULL, *cst = NULL, *T = NULL, l_calib = 0.0;
    if (nc) {
      unsigned char *inc = (unsigned char *)calloc(md->n_pix, 1);
      for (int i = 0; i < md->n_pix; i++) inc[i] = vd[i] && (!md->spec_mask || md->spec_mask[i]);
      minv = (double *)malloc((size_t)nc * nc * sizeof(double));
      cst = (double *)malloc(nc * sizeof(double));
      T = (double *)malloc(nc * sizeof(double));
      l_calib = calib_terms(md, sp, inc, minv, cst);   /* added after the pixel sum, as in orc_row */
      free(inc);
    }
    for (int i = 0; i < md->n_pix; i++) {
      if (!(md->spec_d && vd[i] && (!md->spec_mask || md->spec_mask[i]))) continue;
      double s = md->spec_sigma[i];
      double v = eff_var(t.fl[1], s, sp[i], md->spec_d[i]), r = md->spec_d[i] - sp[i];
      L += -0.5 * r * r / v - 0.5 * log(2.0 * M_PI * v);
      double ui = floor_terms_grad(t.fl[1], v, r, s, sp[i], md->spec_d[i], gfl[1]);
      if (nc) {
        cheb_row(cheb_x(md, i), nc, T);
        double p = 0.0, q = 0.0;
        for (int a = 0; a < nc; a++) {
          p += cst[a] * T[a];
          for (int e = 0; e < nc; e++) q += T[a] * minv[a * nc + e] * T[e];
        }
        /* the optimised polynomial has no ln|M| term: c* is stationary, so only
         * the explicit dependence on mu_i remains (q_i comes from -ln|M|/2) */
        if (md->calib_mode == ORC_CALIB_OPTIMISED) q = 0.0;
        ui = ((md->spec_d[i] - sp[i] * (1.0 + p)) * (1.0 + p) - sp[i] * q) / (s * s);
      }
      /* Eq. "app_response" row of pixel i, as in orc_spectrum */
      double x = log(md->spec_lam[i]) - lz, sg = s_ln[i];
      int k = 0;
      while (k + 2 < NL && !(ll[k] <= x && x < ll[k + 1])) k++;
      double dln = ll[k + 1] - ll[k];
      if (sg < 0.5 * dln) {
        double tt = (x - ll[k]) / dln;
        gfnu[k] += ui * (1.0 - tt);
        gfnu[k + 1] += ui * tt;
        gz += ui * (fnu[k + 1] - fnu[k]) / dln * (-1.0 / zp);
        continue;
      }
      double sw = 0.0, sf = 0.0, swd = 0.0, sfd = 0.0, sws = 0.0, sfs = 0.0;
      for (int j = 0; j < NL; j++) {
        double u = (ll[j] - x) / sg;
        if (fabs(u) > 5.0) continue;
        double w = exp(-0.5 * u * u), wd = w * u / sg; /* d w / d x */
        double ws = w * u * u / sg;                     /* d w / d s */
        sw += w; sf += w * fnu[j]; swd += wd; sfd += wd * fnu[j]; sws += ws; sfs += ws * fnu[j];
      }
      /* width of the row: s = sqrt(sigma_fix^2 + sigma_gal^2) / c, so
       * ds/dsigma_gal = sigma_gal / (c^2 s) */
      g_sgal += ui * (sfs * sw - sf * sws) / (sw * sw) * t.sigma_gal / (O_C_KMS * O_C_KMS * sg);
      for (int j = 0; j < NL; j++) {
        double u = (ll[j] - x) / sg;
        if (fabs(u) > 5.0) continue;
        gfnu[j] += ui * exp(-0.5 * u * u) / sw;
      }
      gz += ui * (sfd * sw - sf * swd) / (sw * sw) * (-1.0 / zp);
    }
    if (nc) L += l_calib;
    free(sp); free(vd); free(s_ln); free(ll);
    free(minv); free(cst); free(T);
  }
  *lnl = L;
  if (!isfinite(L)) {
    st = ORC_NONFINITE;
    *lnl = -INFINITY;
  } else {
    /* ---------------- observer frame: fnu = scale F */
    for (int k = 0; k < NL; k++) gscale += gfnu[k] * F[k];
    double gl_mass = gscale * scale * log(10.0);
    gz += gscale * scale * dlns_dz;
    /* ---------------- dust and nebular (Sec. 2.4, App. C) */
    double g_taubc = 0, g_alpha = 0, g_taud = 0, g_delta = 0, g_qy = 0, g_lu = 0, g_lz = 0, g_fob = 0;
    double *gY = (double *)malloc(NL * sizeof(double)), *gO = (double *)malloc(NL * sizeof(double));
    double *gYL = (double *)malloc(NL * sizeof(double)), *gN = (double *)malloc(NL * sizeof(double));
    for (int k = 0; k < NL; k++) {
      double gF = gfnu[k] * scale;
      double ed = exp(-td[k]), eb = exp(-tbc[k]);
      /* derivatives of F with respect to Y (young stellar, ionising continuum
       * apart), YL (that continuum), O, the birth-cloud depth and the nebular
       * continuum, under the row's escape geometry */
      double gtbc, gtd = -gF * F[k];
      gO[k] = gF * ed;
      if (md->fesc_geometry == ORC_FESC_PICKET) {
        const double b = Y[k] + neb[k];
        gY[k] = gF * (fob + ed * (1.0 - fob) * eb);
        gYL[k] = gF * fob;
        gtbc = -gF * ed * (1.0 - fob) * eb * b;
        gN[k] = gF * ed * (1.0 - fob) * eb;
        gtd = -gF * (F[k] - fob * (Y[k] + YL[k]));
        g_fob += gF * (Y[k] + YL[k] - ed * eb * b);
      } else {
        const double T = (1.0 - fob) * eb + fob, av = Y[k] + (1.0 - fob) * neb[k];
        gY[k] = gF * ed * T;
        gYL[k] = gF * ed * fob;
        gtbc = -gF * ed * (1.0 - fob) * eb * av;
        gN[k] = gF * ed * T * (1.0 - fob);
        g_fob += gF * ed * ((1.0 - eb) * av - T * neb[k] + YL[k]);
      }
      double lp = log(g->lam[k] / 5500.0);
      g_taubc += gtbc * pow(g->lam[k] / 5500.0, t.alpha_bc);
      g_alpha += gtbc * tbc[k] * lp;
      double p = pow(g->lam[k] / 5500.0, t.delta);
      double shape, dshape;
      if (md->dust_law == 0) {
        shape = p;
        dshape = p * lp;
      } else {
        double xx = g->lam[k] * 350.0, dd = g->lam[k] * g->lam[k] - 2175.0 * 2175.0;
        double drude = xx * xx / (dd * dd + xx * xx);
        double kp = calzetti_kprime(g->lam[k] * 1e-4);
        shape = (kp + (0.85 - 1.9 * t.delta) * drude) / 4.05 * p;
        dshape = (-1.9 * drude) / 4.05 * p + shape * lp;
      }
      g_taud += gtd * shape;
      g_delta += gtd * t.tau_d * dshape;
      if (has_neb) {
        double gneb = gN[k];
        g_qy += gneb * pow(10.0, lg[k]);
        double glg = gneb * neb[k] * log(10.0);
        g_lu += glg * (du0 * wg0 * t00[k] + du0 * wg1 * t01[k] + du1 * wg0 * t10[k] + du1 * wg1 * t11[k]);
        g_lz += glg * (wu0 * dg0 * t00[k] + wu0 * dg1 * t01[k] + wu1 * dg0 * t10[k] + wu1 * dg1 * t11[k]);
      }
    }
    /* ---------------- contraction (Eq. csp_sum_main / app_attn) and Q_young */
    for (size_t s = 0; s < nsp; s++) {
      int a = (int)(s % NA);
      int young = g->log_age_yr[a] <= md->bc_edge_log_age_yr;
      const double *f = g->flux + s * NL;
      double acc = 0.0;
      for (int k = 0; k < NL; k++) {
        if (young && has_neb && g->lam[k] < O_LYMAN) acc += gYL[k] * f[k];
        else acc += (young ? gY : gO)[k] * f[k];
      }
      if (young) acc += g_qy * Q[s];
      gW[s] = acc;
    }
    /* ---------------- weights (App. B step scheme, metallicity and [a/Fe] splits) */
    double *gT = (double *)calloc(NT + 1, sizeof(double));
    double g_afe = 0.0;
    int nz = md->zmode == 0 ? NT : 1;
    const int offz = sfh_cols(md), offs = offz + nz;
    double *gAl = (double *)malloc(NA * sizeof(double));
    for (int i = 0; i < NT; i++) {
      double dT = T[i + 1] - T[i];
      if (md->sfh_scheme == 1) {   /* linear scheme: node masses from the edge rates */
        for (int a = 0; a < NA; a++) {
          double Aia = A[(size_t)i * NA + a];
          double g00 = gW[((size_t)an0 * NZ + zm0[i]) * NA + a], g01 = gW[((size_t)an0 * NZ + zm1[i]) * NA + a];
          double g10 = gW[((size_t)an1 * NZ + zm0[i]) * NA + a], g11 = gW[((size_t)an1 * NZ + zm1[i]) * NA + a];
          gAl[a] = g00 * wz0[i] * wa0 + g01 * wz1[i] * wa0 + g10 * wz0[i] * wa1 + g11 * wz1[i] * wa1;
          if (Aia == 0.0) continue;
          grad[offz + (md->zmode == 0 ? i : 0)] +=
              Aia * (g00 * dz0[i] * wa0 + g01 * dz1[i] * wa0 + g10 * dz0[i] * wa1 + g11 * dz1[i] * wa1);
          g_afe += Aia * (g00 * wz0[i] * da0 + g01 * wz1[i] * da0 + g10 * wz0[i] * da1 + g11 * wz1[i] * da1);
        }
        double d4[4];
        linear_bin_grad(g, T[i], T[i + 1], t.m[i], t.m[i + 1], gAl, d4);
        grad[i] += d4[0];
        grad[i + 1] += d4[1];
        gT[i] += d4[2];
        gT[i + 1] += d4[3];
        continue;
      }
      for (int a = 0; a < NA; a++) {
        double Aia = A[(size_t)i * NA + a];
        double lo = T[i] > cm[a] ? T[i] : cm[a];
        double hi = T[i + 1] < cp[a] ? T[i + 1] : cp[a];
        if (hi - lo <= 0.0) continue;
        double g00 = gW[((size_t)an0 * NZ + zm0[i]) * NA + a], g01 = gW[((size_t)an0 * NZ + zm1[i]) * NA + a];
        double g10 = gW[((size_t)an1 * NZ + zm0[i]) * NA + a], g11 = gW[((size_t)an1 * NZ + zm1[i]) * NA + a];
        double gA = g00 * wz0[i] * wa0 + g01 * wz1[i] * wa0 + g10 * wz0[i] * wa1 + g11 * wz1[i] * wa1;
        grad[offz + (md->zmode == 0 ? i : 0)] +=
            Aia * (g00 * dz0[i] * wa0 + g01 * dz1[i] * wa0 + g10 * dz0[i] * wa1 + g11 * dz1[i] * wa1);
        g_afe += Aia * (g00 * wz0[i] * da0 + g01 * wz1[i] * da0 + g10 * wz0[i] * da1 + g11 * wz1[i] * da1);
        /* A = m_i (hi - lo) / dT */
        grad[i] += gA * (hi - lo) / dT;
        double ov = hi - lo;
        gT[i + 1] += gA * t.m[i] * ((T[i + 1] < cp[a] ? 1.0 : 0.0) / dT - ov / (dT * dT));
        gT[i] += gA * t.m[i] * (-(T[i] > cm[a] ? 1.0 : 0.0) / dT + ov / (dT * dT));
      }
    }
    /* SFH edges: T_i = 1e7 (T_max/1e7)^((i-2)/(N_T-2)) for i >= 3; T_max = t(z) - t(z_f) */
    double g_tmax = 0.0;
    for (int i = 3; i <= NT; i++) g_tmax += gT[i] * T[i] * (double)(i - 2) / ((double)(NT - 2) * tmax);
    double th_yr = O_MPC_KM / md->H0 / O_YR_S;
    gz += g_tmax * (-th_yr * inv_E(t.z, &md->Om0) / zp);
    grad[offs + 0] = md->use_afe ? g_afe : 0.0;
    grad[offs + 1] = gl_mass;
    grad[offs + 2] = gz;
    grad[offs + 3] = g_taubc;
    grad[offs + 4] = g_alpha;
    grad[offs + 5] = g_taud;
    grad[offs + 6] = g_delta;
    grad[offs + 7] = has_neb ? g_lz : 0.0;
    grad[offs + 8] = has_neb ? g_lu : 0.0;
    if (md->sample_sigma_gal) grad[offs + 9] = g_sgal;
    for (int arm = 0; arm < 2; arm++)
      for (int k = 0; k < 4; k++)
        if (t.fl_col[arm][k] >= 0) grad[t.fl_col[arm][k]] = gfl[arm][k];
    if (md->fesc_geometry) grad[np - 1] = g_fob;
    free(gT); free(gY); free(gO); free(gYL); free(gN); free(gAl);
  }
  if (st) for (int j = 0; j < np; j++) grad[j] = 0.0;
  free(T); free(cm); free(cp); free(A); free(zm0); free(zm1); free(wz0); free(wz1); free(dz0); free(dz1);
  free(W); free(Q); free(Y); free(O); free(neb); free(lg); free(YL); free(tbc); free(td); free(F); free(fnu);
  free(gfnu); free(gW);
  (void)cf;
  return st;
}

void orc_grad(const orc_grid *g, const orc_model *md, const double *theta, int n, int ld, double *lnl_out,
              double *grad_out, int *status_out, int nthreads) {
#ifdef _OPENMP
  int nt = nthreads > 0 ? nthreads : omp_get_max_threads();
#pragma omp parallel for num_threads(nt) schedule(dynamic, 1)
#endif
  for (int r = 0; r < n; r++) {
    double l;
    int st = orc_row_grad(g, md, theta + (size_t)r * ld, grad_out + (size_t)r * ld, &l);
    if (lnl_out) lnl_out[r] = l;
    if (status_out) status_out[r] = st;
  }
  (void)nthreads;
}
