// Internal declarations of the GB300 SED library (not part of the ABI).
#pragma once
#include <utility>

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "sed.h"

namespace sed {

// ---------------------------------------------------------------------------
// Tiling constants of the contraction.
// K is tiled in 32 FP32 / 64 BF16 elements (128 bytes, one 128B-swizzle row).
constexpr int KT = 64;           // K granule of the layouts: one 128-byte BF16 row, two FP32 rows
constexpr int MAX_AGE = 256;
constexpr int MAX_FEH = 64;
constexpr int MAX_AFE = 16;
constexpr int MAX_SFH = 512;
constexpr int MAX_LAM = 24576;   // rest-frame nodes an epilogue row can stage in shared memory
constexpr int COSMO_TAB = 4096;  // intervals of the cosmology table on [0, zf]
constexpr int COSMO_COLS = 8;    // value / derivative pairs of D_C, t_univ, ln(1+z), 1/(1+z)
// K-tile occupancy masks of the contraction: one bit per K tile of the
// precision's operand layout (32 FP32 / 64 BF16 / 128 FP8 columns), one row of
// KMASK_WORDS words per 128-row tile; grids with more K tiles run unmasked
constexpr int KMASK_WORDS = 8;
constexpr int MAX_LINES = 128;   // emission lines of a nebular grid
constexpr int MAX_DUST_BIN = SED_MAX_DUST_BIN;   // age-binned attenuation laws
constexpr int MAX_SEG = SED_MAX_DUST_SEG;        // attenuated K blocks (runs of ages with one non-zero row of M)
constexpr int MAX_NEB_AGE = 32;  // SSP ages a nebular age axis spans

// Physical constants (cgs unless noted).
constexpr double LSUN = 3.839e33;              // erg/s (Sec. 2.6)
constexpr double HPLANCK = 6.62607015e-27;     // erg s
constexpr double C_AA = 2.99792458e18;         // Angstrom/s
constexpr double C_KMS = 299792.458;
constexpr double AB_FNU = 3.631e-20;           // erg/s/cm^2/Hz (App. D)
constexpr double PC_CM = 3.0856775814913673e18;
constexpr double MPC_KM = 3.0856775814913673e19;
constexpr double YR_S = 3.15576e7;
constexpr double LYMAN_AA = 912.0;
constexpr double FWHM_PER_SIGMA = 2.3548200450309493;

// ---------------------------------------------------------------------------
// Per-row scalars produced by the preparation kernel and read by the epilogue
// and the adjoint kernels.
struct RowScal {
  float p_phot;     // c * s * 2^-E / (1+z)^2 : maggie prefactor of sum_j w_j lerp(F/lam^2)
  float s_spec;     // s * 2^-E : cgs F_nu per unit of device-scaled flux
  float inv1pz;     // 1/(1+z)
  float ln1pz_hi;   // ln(1+z) split in two floats
  float ln1pz_lo;
  float tau_bc, alpha_bc, tau_d, delta;
  float log2_qy;    // log2(Q_young, device units) (-inf when Q_young = 0)
  float neb_w[4];   // bilinear weights of the nebular template corners
  int neb_off[4];   // corner offsets (rows of the template)
  float neb_dwu[4]; // d neb_w / d gas_logu (adjoint)
  float neb_dwz[4]; // d neb_w / d gas_logz (adjoint)
  float dlnp_dz;    // d ln(p_phot)/dz (adjoint)
  float dlns_dz;    // d ln(s_spec)/dz (adjoint)
  float dtmax_dz;   // dT_max/dz in yr (adjoint)
  float tmax;       // yr
  float lrat;       // ln(T_max / 10 Myr) as used for the SFH edges
  uint32_t status;
  int k_lo, k_hi;   // rest-frame node window this row needs
  float y_scale;    // FP8 path: the row's power of two folded out of W (Y, O are multiplied by it); else 1
  int orig;         // the caller's index of this row (rows are processed in redshift order)
  int nnz;          // non-zero weights of the row
  float sg_ln;      // sampled sigma_gal / c (ln-lambda units); 0 with a fixed sigma_gal
  float fl[2][4];   // noise floor {s, f_calib, f_data, j} of photometry [0] and spectrum [1]
  float fob;        // runaway fraction f_ob (0 without an escape geometry)
  float sgas;       // gas velocity dispersion of the emission lines, km/s
  // age-binned attenuation (App. dust_attn): each bin's optical depth and slope,
  // and log2 of Q (device units) of each attenuated block, then of the block
  // outside every bin (-inf when zero)
  float bin_tau[MAX_DUST_BIN], bin_slope[MAX_DUST_BIN];
  float log2_qs[MAX_SEG + 1];
  float igm_f;      // scaling of the IGM optical depth (with use_igm)
};

// Cosmology and observer-frame scalars of one row (computed at the start of k_prep).
struct CosmoRow {
  double tmax_d;    // T_max = t_univ(z) - t_univ(zf), yr
  float p_phot, s_spec, inv1pz, ln1pz_hi, ln1pz_lo, dlnp_dz, dlns_dz, dtmax_dz, lrat;
  uint32_t status;  // SED_ROW_BAD_THETA (z or logmass), SED_ROW_BAD_Z, SED_ROW_BAD_TMAX or 0
};

// ---------------------------------------------------------------------------
// Kernel-parameter views (plain data, device pointers only).
struct GridDev {
  int n_age, n_feh, n_afe, n_lam;
  const float* lam_f;      // lambda (A)
  const float4* att4;      // per node: ln(lambda/5500), k'/4.05, Drude/4.05, lambda
  const float* inv_lam2;   // 1/lambda^2
  const float* inv_dlam;   // 1/(lambda[k+1] - lambda[k]) (0 at the last node)
  const float* lnp;        // ln(lambda/5500)
  const float* kprime;     // Calzetti k'(lambda), R_V = 4.05, clamped >= 0
  const float* drude;      // Drude profile with E_b = 1
  const float* lnl_hi;     // ln(lambda) split in two floats
  const float* lnl_lo;
  const int* lut;          // lut[q] = last node with ln(lambda) <= x0 + q/inv_h
  int lut_n;
  float lut_x0, lut_inv_h;
  float dln_max;           // largest ln(lambda[k+1] / lambda[k])
  const float* cell_lo;    // linear-time Voronoi cell of each age node (yr)
  const float* cell_hi;
  const float* age_t;      // age of each node (yr), for the linear SFH scheme's tents
  const float* age_dl;     // ln(t_{a+1} / t_a) (last entry unused)
  const float* neb_tab;    // [nu][nz][n_lam] log10 template + device-unit offset; with an age axis
                           // [neb_na][nu][nz][n_lam], plane i the cube at SSP age neb_a0 + i
  int neb_nu, neb_nz;
  int neb_a0, neb_na;      // nebular age axis: the SSP ages [neb_a0, neb_a0 + neb_na) (neb_na = 0: none)
  // emission-line cube: per line {ln(lam/5500), k'/4.05, Drude/4.05, lam},
  // ln(lam) as an FP32 pair, and [nu][nz][n_line] log10(L/Q) + device-unit offset
  int n_line;
  const float4* line_att4;
  const float2* line_ln2;
  const float* line_tab;
};

struct LayoutDev {
  int n_young, neb_cut, Ky, Ko, Ky_pad, Kpad;
  const float* q_s;        // [Kpad]
  const int* k_code;       // [Kpad]
  int Ky_pad8, Kpad8;      // FP8 layout: each block padded to 128 (one 128-byte K tile)
  const float* col8;       // [Kpad] 2^-e_k, the FP8 column scale folded into W (0 for empty columns)
  int neb_a0;              // nebular ages: [neb_a0, n_young)
  int n_seg;               // attenuated blocks in [0, Ky_pad): block s = columns [seg_k0[s], seg_k0[s+1])
  int seg_k0[MAX_SEG + 1];
  const int4* age_col;     // [n_age] column of (afe n, feh m, age a) = x + (n n_feh + m) y; z = a's block
                           // (MAX_SEG: outside every attenuated block)
};

struct ModelDev {
  int n_sfh, zmode, use_afe, use_neb, dust_law, n_param;
  int offs[SED_NKEYS];
  double zf, t_zf_yr, dh_cm, th_yr, Om0;
  double lsun_c;           // Lsun 2^-f_log2 / (4 pi)
  const double* ctab;      // cosmology table [n_ctab + 1][COSMO_COLS] on z = i ctab_h: D_C (cm), dD_C/dz,
                           // t_univ (yr), dt/dz, ln(1+z), 1/(1+z), 1/(1+z), -1/(1+z)^2
  int n_ctab;
  double ctab_h, ctab_inv_h;
  double f_log2, q_log2;
  int n_feh, n_afe;
  float feh[MAX_FEH];
  float afe[MAX_AFE];
  int neb_nu, neb_nz;
  float neb_logu[32], neb_logz[32];
  // photometry (samples band-major)
  int n_filt, n_samp;
  const int* band_start;   // [n_filt + 1]
  const float2* samp2;     // [n_samp] {observed-frame lambda (A), weight R lam dlam / Z_b}
  const double* phot_d;    // [n_filt]
  const double* phot_isig; // [n_filt] 1/sigma (0 when masked out)
  const double* phot_nlog; // [n_filt] -1/2 ln(2 pi sigma^2) (0 when masked out)
  const float* phot_dn;    // [n_filt] d/sigma and 1/sigma in FP32 (0 when masked out), for the
  const float* phot_isf;   //   adjoint's per-band weights
  const uint8_t* phot_ul;  // [n_filt] 1: the datum is an upper limit (Eq. app_line_chi2_UL); NULL: none
  float samp_lam_min, samp_lam_max;
  // spectrum
  int n_pix;
  const float2* pix_ln2;   // [n_pix] ln(lambda_obs) as an FP32 pair {hi, lo}, hi + lo to 2^-48
  const float* pix_s;      // [n_pix] total dispersion in ln(lambda) (fixed sigma_gal)
  const float* pix_fix2;   // [n_pix] sigma_fix^2 / c^2 (sampled sigma_gal; NULL otherwise)
  // marginalised calibration polynomial (App. E): calib_n coefficients, prior
  // 1/s_m^2, ln|Lambda| = sum ln s_m^2, per-pixel Chebyshev coordinate in [-1, 1]
  int calib_n;
  int calib_opt;           // 1: the polynomial optimised at each call (no Occam terms), 0: marginalised
  double calib_isig2[SED_MAX_CALIB];
  double calib_logdet_lam;
  const float* pix_cx;
  int floor_bits[2];       // noise-floor terms on (SED_FLOOR_* bits) of photometry [0] and spectrum [1]
  int sfh_linear;          // 1: SFH key = N_T + 1 per-edge SFRs, linear scheme (App. B, Eq. tent_integral)
  int fesc_geom;           // SED_FESC_*: escape geometry of the young light (Sec. frac_obrun)
  int n_lyc;               // rest-frame nodes below 912 A (the ionising continuum)
  int sample_sgal;         // 1: each row carries sigma_gal (km/s), joined in quadrature per pixel
  float sgal_max_kms;      // sampled sigma_gal range [0, sgal_max_kms]
  // spectral data, normalised per pixel so that the per-pixel terms stay in FP32
  // (GB300's FP64 pipe issues a warp instruction every 16 SM cycles): d/sigma
  // and 1/sigma (both 0 where the pixel is excluded), -1/2 ln(2 pi sigma^2)
  const float* spec_dn;
  const float* spec_isf;
  const double* spec_nlog;
  double pix_ln_min, pix_ln_max;
  float pix_s_max;         // largest total dispersion a row can have (ln units)
  int win_max;             // most rest-frame nodes one row's window can span (any redshift)
  // fixed keys (sed_model_desc.fixed): the caller's rows have n_param columns;
  // fixed key j is read from column n_param + j of the row as the kernels stage
  // it (offs[] points there), filled from fixed_v[j]
  int n_fixed;
  float fixed_v[SED_NKEYS];
  // emission lines (App. C, App. line_proj, Eq. app_line_profile)
  int use_lines, gas_mode;   // SED_GAS_SIGMA_*
  float sgas_fix_kms, sgas_max_kms, sgal_fix_kms;
  const float* samp_rz;      // [n_samp] filter transmission R_j / Z_b (the photometry of a line)
  const float* pix_sinst;    // [n_pix] instrumental dispersion, km/s
  const float* pix_lamc;     // [n_pix] lambda_obs / c, s
  // line catalogue (Sec. 3.3): entry k sums the lines lcat_line[lcat_start[k] .. lcat_start[k+1])
  int n_lcat;
  const int* lcat_start;
  const int* lcat_line;
  const double* lcat_d;      // datum, 1/sigma (0 when masked out), -ln(2 pi sigma^2)/2 (0 when masked out)
  const double* lcat_isig;
  const double* lcat_nlog;
  const uint8_t* lcat_ul;    // 1: an upper limit (Eq. app_line_chi2_UL); NULL: none
  // age-binned attenuation (App. dust_attn, Eq. app_tau_bin): n_bin laws
  // (SED_DUST_*), n_seg attenuated K blocks; block s sees tau_s = sum_b
  // seg_M[s][b] kappa_b.  n_bin = 0: the birth-cloud power law
  int n_bin, n_seg;
  int bin_law[MAX_DUST_BIN];
  float seg_M[MAX_SEG][MAX_DUST_BIN];
  int use_igm;             // SED_IGM_MADAU: the Madau (1995) IGM transmission (Sec. 2.6)
};

// Value of column `col` of a parameter row in the kernels' layout: a caller's
// column, or a fixed key's value past the caller's columns.
__host__ __device__ __forceinline__ float theta_col(const ModelDev& md, const float* row, int col) {
  return col < md.n_param ? row[col] : md.fixed_v[col - md.n_param];
}

// ---------------------------------------------------------------------------
// Device copy of a grid in one K order: [young block | old block], each block
// ordered (afe n, feh m, age a) with age fastest, each block padded to KT.
struct Layout {
  int n_young = 0;    // nebular ages [neb_a0, n_young) (<= birth-cloud edge): Q and the 912 A cut
  int neb_a0 = 0;
  int neb_cut = 0;    // 1: stellar flux below 912 A removed for nebular ages
  // the attenuated blocks: age a is in block blk[a] (0 .. n_seg - 1) or, for
  // -1, in the block after them (no age-dependent attenuation); without
  // age-binned dust there is one block, the birth-cloud ages
  std::vector<int> blk;
  int n_seg = 1;
  int seg_k0[MAX_SEG + 1] = {};
  int Ky = 0, Ko = 0, Ky_pad = 0, Kpad = 0;
  float* sspT_f32 = nullptr;         // [n_lam][Kpad] scaled flux, exact FP32
  float* sspT_hi = nullptr;          // [n_lam][Kpad] TF32-rounded high part
  float* sspT_lo = nullptr;          // [n_lam][Kpad] low part (x - hi)
  __nv_bfloat16* sspT_bf16 = nullptr;
  // adjoint copies, lambda-major: [Kpad][ldn] with ldn = n_lam rounded up to 256
  // (zero beyond n_lam); built on the first gradient call
  int ldn = 0;
  float* sspK_f32 = nullptr;
  float* sspK_hi = nullptr;
  float* sspK_lo = nullptr;
  // FP8 copy (built on the first FP8 call): [n_lam][Kpad8], E4M3 of SSP * 2^e_k, with
  // the old block starting at Ky_pad8; col8[k] = 2^-e_k
  int Ky_pad8 = 0, Kpad8 = 0;
  uint8_t* sspT_f8 = nullptr;
  float* col8 = nullptr;
  float* lam8 = nullptr;             // [n_lam] 2^-f_l, the FP8 wavelength scale undone in the epilogue
  float* q_s = nullptr;              // [Kpad] scaled Q for young k, 0 elsewhere
  int4* age_col = nullptr;           // [n_age] see LayoutDev
  int* k_code = nullptr;             // [Kpad] packed (n<<24 | m<<16 | a), -1 for padding
  std::vector<int> code_h;           // host copy of k_code
  double q_log2 = 0.0;               // Q_dev = Q * 2^-q_log2
  bool have_tmaps = false;
  CUtensorMap tm_hi, tm_lo, tm_bf16;
  LayoutDev dv() const {
    LayoutDev d{n_young, neb_cut, Ky, Ko, Ky_pad, Kpad, q_s, k_code, Ky_pad8, Kpad8, col8, neb_a0, n_seg, {}, age_col};
    for (int s = 0; s <= MAX_SEG; ++s) d.seg_k0[s] = seg_k0[s];
    return d;
  }
};

struct Grid {
  int n_age = 0, n_feh = 0, n_afe = 0, n_lam = 0;
  int n_line = 0;          // emission lines of the nebular grid
  unsigned copies = 0;     // SED_GRID_COPY_* bits built with each layout
  unsigned avail = 0;      // precisions a call may use (FP8 built on first use when not in `copies`)
  std::vector<double> log_age, feh, afe, lam, flux;  // host master copy (FP64)
  std::vector<double> siglib_kms;                    // Eq. app_siglib at the nodes
  double f_log2 = 0.0;                               // f_dev = f * 2^f_log2
  double f_scale = 1.0;                              // 2^f_log2
  double q_log2 = 0.0;                               // Q_dev = Q * 2^-q_log2
  std::vector<double> q;                             // [n_afe][n_feh][n_age] Eq. app_q
  GridDev dv{};
  int neb_nu = 0, neb_nz = 0;
  int neb_a0 = 0, neb_na = 0;  // nebular age axis: the SSP ages it spans (neb_na = 0: none)
  std::vector<double> neb_logu, neb_logz;
  std::vector<Layout*> layouts;
  std::vector<void*> allocs;
  size_t bytes = 0;
};

struct Model {
  int grid = -1;
  int offs_caller[SED_NKEYS] = {};   // first column of each key in the caller's rows (sed_model_layout)
  Grid* g = nullptr;
  Layout* L = nullptr;
  ModelDev dv{};
  double bc_edge = 7.03, H0 = 0;
  std::vector<uint8_t> phot_mask_h, spec_mask_h;
  // the data as last set (sed_set_data keeps a pair passed as NULL); empty
  // until set, and a block never set stays out of lnL
  std::vector<double> phot_d_h, phot_s_h, spec_d_h, spec_s_h;
  std::vector<void*> allocs;
  size_t bytes = 0;
};

// Operand tensor maps of one tensor-core contraction.
struct TcMaps {
  CUtensorMap a_hi, a_lo, b_hi, b_lo;
};
// Operand maps of the adjoint contraction (A: dlnL/dY, dlnL/dO; B: SSP [k][lam]).
struct DwMaps {
  CUtensorMap gy_hi, gy_lo, go_hi, go_lo, s_hi, s_lo;
};

// Per-row scalar gradient pieces written by the adjoint epilogue.
enum {
  RG_TAU_BC = 0, RG_ALPHA_BC, RG_TAU_D, RG_DELTA, RG_GAS_LOGZ, RG_GAS_LOGU, RG_LOGMASS, RG_Z, RG_QY,
  RG_BAD,   // non-zero: the row's likelihood is not finite (gradient row written as zeros)
  RG_SIGMA_GAL,   // dlnL/dsigma_gal (km/s) of a sampled sigma_gal
  RG_FLOOR,       // 8 slots: dlnL/dlog10 of the noise-floor terms, photometry then spectrum
  RG_FOB = RG_FLOOR + 8,   // dlnL/df_ob
  RG_SIGMA_GAS,            // dlnL/dsigma_gas (km/s) of a sampled gas dispersion
  RG_BIN,                  // 2 MAX_DUST_BIN slots: dlnL/dtau_b, dlnL/dslope_b of each attenuation bin
  RG_QSEG = RG_BIN + 2 * MAX_DUST_BIN,   // MAX_SEG + 1 slots: dlnL/dQ of each attenuated block, then
                                        // of the block outside every bin
  RG_IGM = RG_QSEG + MAX_SEG + 1,       // dlnL/digm_factor
  RG_QAGE,                              // MAX_NEB_AGE slots: dlnL/dQ of each SSP age of a nebular age axis
  RGRAD = RG_QAGE + MAX_NEB_AGE + 4
};

// Per-stream scratch.
struct Workspace {
  int cap_rows = 0;
  size_t cap_k = 0, cap_n = 0;
  int cap_seg = 1;               // attenuated blocks Y and G hold (slabs of [cap_rows][ldn])
  float* W = nullptr;            // [rows][Kpad]  exact FP32 weights (also the TF32 hi part source)
  float* W_hi = nullptr;         // [rows][Kpad]
  float* W_lo = nullptr;
  int* perm = nullptr;           // [rows] processing order
  int* tile_win = nullptr;       // [2][ceil(rows/128)] per-tile node windows
  uint32_t* kmask = nullptr;     // [ceil(rows/128)][KMASK_WORDS] per-tile K-tile occupancy
  int kmask_w_call = 0;          // words per tile of the current call's masks (0: the call has none)
  // The K tiles of W_hi/W_lo row p that may hold non-zeros (bit set), for the
  // layout of row stride wmask_kpad (0: unknown -- every bit set first): a
  // K-tile-masked 3xTF32 call writes only its rows' touched tiles and zeros
  // over the tiles the row at that position touched before
  uint32_t* wmask = nullptr;     // [rows][KMASK_WORDS]
  int wmask_kpad = 0;
  __nv_bfloat16* W_bf16 = nullptr;
  uint8_t* W_f8 = nullptr;       // [rows][Kpad8] E4M3
  float* Y = nullptr;            // [cap_seg][cap_rows][ldn]: one slab per attenuated block
  float* O = nullptr;
  float* O2 = nullptr;           // [rows][ldn] second half of the old part (a split 3xTF32 launch)
  RowScal* rs = nullptr;
  int* err = nullptr;            // device error word of bounded waits (err[0]); err[8]: the 3xTF32
                                 // launch's split choice
  float* theta_h = nullptr;      // host-path staging (device)
  double* lnl_h = nullptr;
  uint32_t* st_h = nullptr;
  int ldn = 0;
  // adjoint
  float* G_hi = nullptr;         // [rows][ldn] dlnL/dY (TF32 high part, or exact for FP32-SIMT)
  float* G_lo = nullptr;         // [rows][ldn] low part
  float* GO_hi = nullptr;        // [rows][ldn] dlnL/dO
  float* GO_lo = nullptr;
  float* dW = nullptr;           // [rows][Kpad] dlnL/dW
  double* rgrad = nullptr;       // [rows][RGRAD] per-row scalar gradient pieces
  float* qneb = nullptr;         // [rows][MAX_NEB_AGE] nebular age axis: Q-weighted weight of each nebular age
  bool dw_maps_valid = false;
  const void* dw_maps_for = nullptr;
  int dw_maps_n = -1;
  const void* dw_maps_g = nullptr;
  size_t bytes = 0;
  bool tmap_valid = false;
  const void* tmap_for = nullptr;
  int tmap_n = -1, tmap_prec = -1;
  const void* tmap_a = nullptr;
  TcMaps maps;
  DwMaps dw_maps;
  // profiling: events before/after prep, contraction, epilogue of the last call
  cudaEvent_t ev[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};  // prep, contract, epilogue, end,
                                                                               // adjoint epilogue end, dW end
  bool last_grad = false;
  int last_n = 0, last_prec = 0, last_kpad = 0, last_nlam = 0;
  int last_kmask_w = 0, last_kt_shift = 0;   // the last call's K-tile masks (0 words: unmasked)
  bool have_stats = false;
  // sed_loglike_host on buffers used in place: the call's launches as a CUDA
  // graph, captured when the same call repeats and replayed after that (the
  // graph holds this workspace's buffers, so it goes when they are reallocated)
  struct HostKey {
    int model = -1;
    const void *mp = nullptr, *th = nullptr, *lnl = nullptr, *st = nullptr;
    int n = 0, ld = 0, prec = -1;
    bool operator==(const HostKey& o) const {
      return model == o.model && mp == o.mp && th == o.th && lnl == o.lnl && st == o.st && n == o.n && ld == o.ld &&
             prec == o.prec;
    }
  };
  cudaGraphExec_t host_exec = nullptr;
  HostKey host_key, host_seen;
};

}  // namespace sed

struct sed_ctx {
  int device = 0;
  size_t budget = 0;
  std::atomic<size_t> used{0};   // device bytes held; changed only through sed::budget_reserve / budget_release
  std::mutex mu;
  std::string last_error = "ok";
  std::vector<sed::Grid*> grids;
  std::vector<sed::Model*> models;
  std::map<void*, sed::Workspace*> ws;
  void* encode_fn = nullptr;   // cuTensorMapEncodeTiled
  int profiling = 0;
  int tc_ok = -1;              // tcgen05 path usable on this device (sm_103)
  int last_host_mapped = 0;    // sed_last_host_path
};

namespace sed {
// Device-memory accounting of a context against its budget.  The context's
// allocations (grids, models, per-stream workspaces) and the server's (launch
// slots, fits' live points) can run on different host threads under different
// locks, so the count is atomic and a reservation is one compare-exchange:
// either the whole amount fits under the budget and is added, or nothing is.
inline bool budget_reserve(sed_ctx* ctx, size_t bytes) {
  size_t cur = ctx->used.load(std::memory_order_relaxed);
  do {
    if (ctx->budget && cur + bytes > ctx->budget) return false;
  } while (!ctx->used.compare_exchange_weak(cur, cur + bytes, std::memory_order_relaxed));
  return true;
}
inline void budget_release(sed_ctx* ctx, size_t bytes) {
  size_t cur = ctx->used.load(std::memory_order_relaxed);
  while (!ctx->used.compare_exchange_weak(cur, cur - std::min(cur, bytes), std::memory_order_relaxed)) {
  }
}
}  // namespace sed

// ---------------------------------------------------------------------------
// Kernel launchers (defined in the .cu files).
namespace sed {

struct PrepArgs {
  const float* theta; int n, ld;
  ModelDev md; GridDev g; LayoutDev L;
  const ModelDev* mtab;    // rows from several fits (serving): model of row r = mtab[row_model[r]];
  const int* row_model;    // NULL: every row uses md
  float* W; float* W_hi; float* W_lo; __nv_bfloat16* W_bf16;
  uint8_t* W_f8;       // FP8 path: [n][Kpad8]
  RowScal* rs;
  int* err;            // device error word of the contraction, cleared by the prep kernel
  int* perm;           // [n] scratch: processing order (rows sorted by redshift), or NULL = caller's order
  int* tile_win;       // [2][ceil(n/128)] union of the row windows of each 128-row tile (launch_prep
                       // starts them empty: lo 0x7f7f7f7f, hi -1), or NULL
  uint32_t* kmask;     // [ceil(n/128)][kmask_w] K tiles that some row of each 128-row tile touches
                       // (launch_prep clears them), or NULL
  int kmask_w;         // words per 128-row tile (<= KMASK_WORDS)
  int kt_shift;        // log2 of the columns of one K tile of the contraction's layout (5, 6 or 7)
  uint32_t* wmask;     // with kmask and W_hi: [n][KMASK_WORDS] K tiles of each W row that may hold
                       // non-zeros from before (read) and that hold them now (written); the row's
                       // other tiles are zeros and are not written.  NULL: every column written
  float* qneb;         // nebular age axis: [n][MAX_NEB_AGE] Q-weighted weight of each nebular SSP age, or NULL
  int self_order;      // 1: the prep kernel finds each row's place in the redshift order itself (no
                       // k_order launch) where launch_prep allows it: one fit, no K-tile masks, a
                       // redshift column, n <= SELF_ORDER_MAX, theta in device memory (each CTA
                       // reads every row's redshift), and tile_win already empty
};
// Per-tile windows (lo, hi) of the contraction back to empty (lo 0x7f7f7f7f,
// hi -1) once their reader has finished, by one CTA, so that the next call's
// prep kernel can fill them without an ordering kernel or memsets before it.
__device__ __forceinline__ void empty_windows(int* win, int mt) {
  for (int i = threadIdx.x; i < mt; i += blockDim.x) {
    win[i] = 0x7f7f7f7f;
    win[mt + i] = -1;
  }
}
// A pixel's rest-frame ln(lambda) = ln(lambda_obs) - ln(1+z), both given as
// FP32 pairs {hi, lo}, returned as an FP32 pair: the high parts' difference is
// made exact by Knuth's two-sum (s + e = p.hi - z_hi), the low parts join its
// error term, and a final fast two-sum renormalises.  FP32 only (the FP64 pipe
// is the scarce one).
__device__ __forceinline__ void ln_rest(float2 p, float z_hi, float z_lo, float& x_hi, float& x_lo) {
  const float s = p.x - z_hi;
  const float bv = s - p.x;
  const float e = (p.x - (s - bv)) + (-z_hi - bv);
  const float t = e + (p.y - z_lo);
  x_hi = s + t;
  x_lo = t - (x_hi - s);
}

// Programmatic dependent launch.  Every kernel of the library begins with
// pdl_enter(): it waits until the kernel before it on the stream has completed
// and its writes are visible, then lets the next kernel be scheduled.  Launched
// directly on a stream, a kernel carries programmatic stream serialisation, so
// its launch and scheduling overlap the previous kernel's work; results are
// those of plain stream order.  Under stream capture the attribute is left off:
// a graph replay already launches back to back, and measured slower with it.
// Without the attribute the wait returns at once.
__device__ __forceinline__ void pdl_enter() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                       Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cap) != cudaSuccess) cap = cudaStreamCaptureStatusNone;
  cfg.attrs = at;
  cfg.numAttrs = cap == cudaStreamCaptureStatusNone ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// Raises a kernel's dynamic shared-memory limit once its static plus dynamic
// shared memory passes the 48 KB default.  The attribute belongs to the
// current device, so the largest size set is cached per device; one lock
// orders the updates of every cache (a launch on another thread never sees a
// limit lowered under it).  cudaErrorInvalidConfiguration if the total passes
// the 227 KB a CTA can have.
constexpr int MAX_DEVICES = 64;
struct DynSmemCache {
  size_t v[MAX_DEVICES] = {};
};
inline std::mutex& dyn_smem_mutex() {
  static std::mutex m;
  return m;
}
template <typename K>
cudaError_t ensure_dyn_smem(K* kernel, size_t dyn, DynSmemCache* cache) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= MAX_DEVICES) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(dyn_smem_mutex());
  if (dyn <= cache->v[dev]) return cudaSuccess;
  cudaFuncAttributes fa;
  e = cudaFuncGetAttributes(&fa, kernel);
  if (e != cudaSuccess) return e;
  if (dyn + fa.sharedSizeBytes > 227 * 1024) return cudaErrorInvalidConfiguration;
  if (dyn + fa.sharedSizeBytes > 48 * 1024) {
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
    if (e != cudaSuccess) return e;
  }
  cache->v[dev] = dyn;
  return cudaSuccess;
}

// Streaming multiprocessors of the current device (cached per device).
inline int device_sm_count() {
  static std::atomic<int> n_sm[MAX_DEVICES];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) return 1;
  int v = n_sm[dev].load(std::memory_order_relaxed);
  if (v > 0) return v;
  if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) return 1;
  n_sm[dev].store(v, std::memory_order_relaxed);
  return v;
}

cudaError_t launch_prep(const PrepArgs& a, cudaStream_t s);

struct ContractArgs {
  const RowScal* rs;   // per-row node windows: tiles outside every row's window are skipped
  int n;               // rows (theta)
  int n_lam, ldn;
  int Ky_pad, Kpad;
  const float* W;      // [n][Kpad]
  const float* sspT;   // [n_lam][Kpad]
  float* Y; float* O;  // [n][ldn]
  int n_seg;           // attenuated blocks: columns [seg_k0[s], seg_k0[s+1]) into Y + s seg_stride
  int seg_k0[MAX_SEG + 1];
  size_t seg_stride;
};
cudaError_t launch_contract_simt(const ContractArgs& a, cudaStream_t s);

struct TcArgs {
  const RowScal* rs;   // per-row node windows: tiles outside every row's window are skipped
  int n, n_lam, ldn, Ky_pad, Kpad, prec;   // prec: SED_PREC_FP32, SED_PREC_BF16 or SED_PREC_FP8
                                          // (for FP8, Ky_pad/Kpad are the FP8 layout's Ky_pad8/Kpad8)
  const TcMaps* maps;
  float* Y; float* O; int* err;
  float* O2;           // 3xTF32: second half of the old part if the launch splits its tiles, or NULL
  int* split_out;      // the launch's choice (1: the old part is O + O2), or NULL
  const int* tile_win; // non-NULL (and <= 64 M tiles): persistent schedule over the computed tiles
  const uint32_t* kmask; int kmask_w;   // K tiles some row of each 128-row tile touches (NULL: all)
  int n_seg;           // attenuated blocks of the young part (0 or 1: one), block s of the main layout's
  int seg_k0[MAX_SEG + 1];   // columns [seg_k0[s], seg_k0[s+1]) into Y + s seg_stride
  size_t seg_stride;
};
// encodes the four operand maps; returns 0 on success
int tc_encode_maps(void* encode_fn, TcMaps* out, int prec, const void* a_hi, const void* a_lo,
                   const void* b_hi, const void* b_lo, int n, int n_lam, int kpad);
cudaError_t launch_contract_tc(const TcArgs& a, cudaStream_t s);
// wavelength width of the forward tensor-core tile for a precision and padded K
int tc_bn_for(int prec, int kpad);
int tc_max_m_tiles();   // 128-row tiles of the largest launch that runs the persistent schedule

// Adjoint contraction dW = [G_Y SSP_young^T | G_O SSP_old^T] (3xTF32 on tcgen05).
// G rows have stride ldg; SSP rows [Kpad][ldk] (ldk <= ldg is the reduction length).
int tc_encode_dw_maps(void* encode_fn, DwMaps* out, const float* gy_hi, const float* gy_lo, const float* go_hi,
                      const float* go_lo, const float* sk_hi, const float* sk_lo, int n, int n_gy, int ldg, int ldk,
                      int kpad);
struct DwArgs {
  const RowScal* rs;   // per-row node windows bound the reduction over lambda
  const uint32_t* kmask; int kmask_w;   // 32-column K tiles some row of each 128-row tile touches (NULL: all);
                                        // output tiles of dW no row touches are not computed
  int n, ldk, Ky_pad, Kpad;
  const DwMaps* maps;
  float* dW; int* err;
  int n_seg, seg_rows;       // attenuated blocks: dW columns [seg_k0[s], seg_k0[s+1]) read dlnL/dY of block s
  int seg_k0[MAX_SEG + 1];   // (rows s seg_rows + m of the dlnL/dY map)
};
cudaError_t launch_dw_tc(const DwArgs& a, cudaStream_t s);

struct EpiArgs {
  int n; int ldn;
  const float* Y; const float* O;
  const float* O2;       // second half of the old part, added to O where *split is 1 (NULL: none)
  const int* split;      // the contraction's choice (written by it before this kernel runs), or NULL
  const RowScal* rs;
  ModelDev md; GridDev g;
  const ModelDev* mtab;    // as in PrepArgs; with row_model set, smem_samp / smem_pix give the
  const int* row_model;    // largest n_samp / n_pix of the launch's models
  int smem_samp, smem_pix, smem_win;
  float* phot_out; float* spec_out;
  float* lines_out;    // [n][n_line] observer-frame line fluxes (erg/s/cm^2), or NULL
  double* lnl; uint32_t* status;
  const int* err;      // device error word of the contraction (row status SED_ROW_DEVICE_TIMEOUT)
  const float* lam8;   // FP8 path: [n_lam] 2^-f_l multiplying Y and O; NULL otherwise
  int lines_off;       // set by launch_epilogue: float offset of the emission lines' shared arrays
  size_t seg_stride;   // age-binned dust: Y of attenuated block s at Y + s seg_stride
  const float* qneb;   // nebular age axis: [n][MAX_NEB_AGE] (k_prep's), or NULL
  int* win_reset;      // [2][win_mt] per-tile windows set back to empty by CTA 0 (the contraction,
  int win_mt;          // their reader, has finished), or NULL
};
cudaError_t launch_epilogue(const EpiArgs& a, cudaStream_t s);

// ---- adjoint
struct EpiBwdArgs {
  int n; int ldn;
  const float* Y; const float* O;
  const float* O2;       // as in EpiArgs
  const int* o2_split;
  const RowScal* rs;
  ModelDev md; GridDev g;
  int split;            // 1: write G as TF32 hi/lo parts (3xTF32), 0: exact FP32 into *_hi
  float* gy_hi; float* gy_lo; float* go_hi; float* go_lo;
  double* rgrad;
  double* lnl; uint32_t* status;
  const int* err;
  int lines_off;        // set by launch_epilogue_bwd: byte offset of the emission lines' shared arrays
  size_t seg_stride;    // age-binned dust: Y and dlnL/dY of attenuated block s at + s seg_stride
  const float* qneb;    // nebular age axis: [n][MAX_NEB_AGE] (k_prep's), or NULL
  int* win_reset;       // as in EpiArgs
  int win_mt;
};
cudaError_t launch_epilogue_bwd(const EpiBwdArgs& a, size_t* smem_needed, cudaStream_t s);

struct DwSimtArgs {
  const RowScal* rs;
  int n, ldg, ldk, Ky_pad, Kpad;
  int n_seg;                          // attenuated blocks: columns [seg_k0[s], seg_k0[s+1]) read gy + s seg_stride
  int seg_k0[MAX_SEG + 1];
  size_t seg_stride;
  const float* gy; const float* go;   // [n][ldg]
  const float* sspK;                  // [Kpad][ldk], ldk <= ldg: the reduction length
  float* dW;                          // [n][Kpad]
};
cudaError_t launch_dw_simt(const DwSimtArgs& a, cudaStream_t s);

struct PrepBwdArgs {
  const float* theta; int n, ld;
  ModelDev md; GridDev g; LayoutDev L;
  const RowScal* rs;
  const float* dW; const double* rgrad;
  float* grad;          // [n][ld]
};
cudaError_t launch_prep_bwd(const PrepBwdArgs& a, cudaStream_t s);

// Build the FP8 copy of a layout (caller holds ctx->mu).
sed_status ensure_f8_layout_shared(sed_ctx* ctx, Grid* g, Layout* L);

}  // namespace sed
