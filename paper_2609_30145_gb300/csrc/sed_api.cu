// Host side of the C ABI declared in include/sed.h: validation, grid and
// model set-up (all static precomputation in FP64 on the host), per-stream
// workspaces and the dispatch of the hot-path kernels.
#include <cudaTypedefs.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <cfloat>
#include <cmath>

#include "sed_internal.cuh"

using namespace sed;

namespace {

sed_status fail(sed_ctx* ctx, sed_status st, const char* fmt, ...) {
  if (ctx) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    ctx->last_error = buf;
  }
  return st;
}

#define CK(call)                                                                          \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess) return fail(ctx, SED_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

struct DevGuard {
  int prev = -1;
  explicit DevGuard(int d) {
    cudaGetDevice(&prev);
    if (prev != d) cudaSetDevice(d);
  }
  ~DevGuard() {
    int cur = -1;
    cudaGetDevice(&cur);
    if (prev >= 0 && cur != prev) cudaSetDevice(prev);
  }
};

sed_status dalloc(sed_ctx* ctx, void** p, size_t bytes, std::vector<void*>* owner, size_t* acct) {
  *p = nullptr;
  if (bytes == 0) bytes = 16;
  bytes = (bytes + 255) & ~(size_t)255;
  if (!budget_reserve(ctx, bytes))
    return fail(ctx, SED_ENOMEM, "HBM budget exceeded (%zu + %zu > %zu bytes)", ctx->used.load(), bytes, ctx->budget);
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    budget_release(ctx, bytes);
    return fail(ctx, SED_ENOMEM, "cudaMalloc(%zu): %s", bytes, cudaGetErrorString(e));
  }
  if (acct) *acct += bytes;
  if (owner) owner->push_back(*p);
  return SED_OK;
}

template <class T>
sed_status upload(sed_ctx* ctx, T** dst, const T* src, size_t n, std::vector<void*>* owner, size_t* acct) {
  sed_status st = dalloc(ctx, (void**)dst, n * sizeof(T), owner, acct);
  if (st) return st;
  if (n) CK(cudaMemcpy(*dst, src, n * sizeof(T), cudaMemcpyHostToDevice));
  return SED_OK;
}

void free_all(sed_ctx* ctx, std::vector<void*>& v, size_t& acct) {
  for (void* p : v) cudaFree(p);
  v.clear();
  budget_release(ctx, acct);
  acct = 0;
}

bool strictly_increasing(const double* x, int n) {
  for (int i = 0; i < n; i++)
    if (!std::isfinite(x[i]) || (i && !(x[i] > x[i - 1]))) return false;
  return true;
}

float tf32_rna_host(float x) {
  uint32_t u;
  memcpy(&u, &x, 4);
  if ((u & 0x7f800000u) == 0x7f800000u) return x;
  u += 0x1000u;
  u &= 0xffffe000u;
  float r;
  memcpy(&r, &u, 4);
  return r;
}

double calzetti_kprime(double lum) {  // Calzetti et al. 2000, R_V = 4.05, UV branch below 0.63 um
  double k;
  if (lum >= 0.63)
    k = 2.659 * (-1.857 + 1.040 / lum) + 4.05;
  else
    k = 2.659 * (-2.156 + 1.509 / lum - 0.198 / (lum * lum) + 0.011 / (lum * lum * lum)) + 4.05;
  return k > 0.0 ? k : 0.0;
}

sed::Workspace* get_ws(sed_ctx* ctx, void* stream, int rows, int kpad, int ldn, bool grad, sed_status* st,
                       int nseg = 1);
sed_status ensure_f8_layout(sed_ctx* ctx, Grid* g, Layout* L);

}  // namespace

namespace sed {
sed_status ensure_f8_layout_shared(sed_ctx* ctx, Grid* g, Layout* L) { return ensure_f8_layout(ctx, g, L); }
}  // namespace sed

// ===========================================================================
extern "C" {

const char* sed_status_string(sed_status s) {
  switch (s) {
    case SED_OK: return "ok";
    case SED_EINVAL: return "invalid argument";
    case SED_ENOMEM: return "out of device memory or budget";
    case SED_ECUDA: return "CUDA error";
    case SED_ERANGE: return "size out of supported range";
    case SED_ENONFINITE: return "non-finite input";
    case SED_EBUSY: return "busy";
    case SED_ETIMEOUT: return "device wait timed out";
    case SED_EUNSUPPORTED: return "unsupported";
  }
  return "unknown status";
}

const char* sed_last_error(const sed_ctx* ctx) { return ctx ? ctx->last_error.c_str() : "null context"; }

sed_status sed_create(sed_ctx** out, int device, size_t budget) {
  if (!out) return SED_EINVAL;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return SED_EINVAL;
  }
  sed_ctx* ctx = new sed_ctx();
  ctx->device = device;
  ctx->budget = budget;
  DevGuard dg(device);
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) {
    delete ctx;
    return SED_ECUDA;
  }
  ctx->tc_ok = (prop.major == 10 && prop.minor == 3) ? 1 : 0;
  void* fn = nullptr;
  cudaDriverEntryPointQueryResult q;
  if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) == cudaSuccess &&
      q == cudaDriverEntryPointSuccess)
    ctx->encode_fn = fn;
  else
    ctx->tc_ok = 0;
  *out = ctx;
  return SED_OK;
}

sed_status sed_destroy_model(sed_ctx* ctx, sed_model_id id);

sed_status sed_destroy(sed_ctx* ctx) {
  if (!ctx) return SED_EINVAL;
  {
    DevGuard dg(ctx->device);
    cudaDeviceSynchronize();
    for (size_t i = 0; i < ctx->models.size(); i++)
      if (ctx->models[i]) sed_destroy_model(ctx, (sed_model_id)i);
    for (Grid* g : ctx->grids) {
      if (!g) continue;
      for (Layout* L : g->layouts) delete L;
      free_all(ctx, g->allocs, g->bytes);
      delete g;
    }
    for (auto& kv : ctx->ws) {
      Workspace* w = kv.second;
      std::vector<void*> v = {w->perm, w->tile_win, w->kmask, w->W, w->W_hi, w->W_lo, w->W_bf16, w->W_f8, w->Y, w->O, w->O2, w->rs, w->err,
                              w->wmask, w->theta_h, w->lnl_h, w->st_h, w->G_hi, w->G_lo, w->GO_hi, w->GO_lo,
                              w->dW, w->rgrad, w->qneb};
      for (void* p : v)
        if (p) cudaFree(p);
      for (cudaEvent_t e : w->ev)
        if (e) cudaEventDestroy(e);
      if (w->host_exec) cudaGraphExecDestroy(w->host_exec);
      delete w;
    }
  }
  delete ctx;
  return SED_OK;
}

sed_status sed_last_host_path(const sed_ctx* ctx, int* mapped) {
  if (!ctx || !mapped) return SED_EINVAL;
  *mapped = ctx->last_host_mapped;
  return SED_OK;
}

sed_status sed_memory_used(const sed_ctx* ctx, size_t* bytes) {
  if (!ctx || !bytes) return SED_EINVAL;
  *bytes = ctx->used.load();
  return SED_OK;
}

// ---------------------------------------------------------------------------
sed_status sed_load_grid(sed_ctx* ctx, const sed_grid_desc* d, sed_grid_id* out) {
  if (!ctx || !d || !out) return fail(ctx, SED_EINVAL, "null argument");
  std::lock_guard<std::mutex> lk(ctx->mu);
  DevGuard dg(ctx->device);
  if (d->n_age < 2 || d->n_feh < 1 || d->n_afe < 1 || d->n_lam < 4)
    return fail(ctx, SED_EINVAL, "grid needs n_age >= 2, n_feh >= 1, n_afe >= 1, n_lam >= 4");
  if (d->n_age > MAX_AGE || d->n_feh > MAX_FEH || d->n_afe > MAX_AFE || d->n_lam > MAX_LAM)
    return fail(ctx, SED_ERANGE, "grid axis too long (max age %d feh %d afe %d lam %d)", MAX_AGE, MAX_FEH, MAX_AFE, MAX_LAM);
  if (!d->log_age_yr || !d->feh || !d->lam_aa || !d->flux || (d->n_afe > 1 && !d->afe))
    return fail(ctx, SED_EINVAL, "grid axis or flux pointer is NULL");
  if (!strictly_increasing(d->log_age_yr, d->n_age) || !strictly_increasing(d->feh, d->n_feh) ||
      (d->afe && !strictly_increasing(d->afe, d->n_afe)) || !strictly_increasing(d->lam_aa, d->n_lam) ||
      !(d->lam_aa[0] > 0))
    return fail(ctx, SED_EINVAL, "grid axes must be finite and strictly increasing (lam > 0)");
  const size_t nsp = (size_t)d->n_afe * d->n_feh * d->n_age, nl = d->n_lam;
  double fmax = 0.0;
  for (size_t i = 0; i < nsp * nl; i++) {
    double v = d->flux[i];
    if (!std::isfinite(v) || v < 0.0) return fail(ctx, SED_EINVAL, "flux must be finite and >= 0 (index %zu)", i);
    fmax = std::max(fmax, v);
  }
  if (!(fmax > 0)) return fail(ctx, SED_EINVAL, "flux is identically zero");
  if (d->precision_mask > 15u) return fail(ctx, SED_EINVAL, "precision_mask has bits other than SED_GRID_COPY_*");
  const bool neb = d->neb_n_logu > 0 && d->neb_n_logz > 0 && d->neb_log10_lnu_per_q;
  if (neb) {
    if (d->neb_n_logu > 32 || d->neb_n_logz > 32) return fail(ctx, SED_ERANGE, "nebular axes longer than 32");
    if (!d->neb_logu || !d->neb_logz || !strictly_increasing(d->neb_logu, d->neb_n_logu) ||
        !strictly_increasing(d->neb_logz, d->neb_n_logz))
      return fail(ctx, SED_EINVAL, "nebular axes must be strictly increasing");
    if (d->neb_n_age < 0 || d->neb_n_age > 64) return fail(ctx, SED_ERANGE, "neb_n_age must be in [0, 64]");
    if (d->neb_n_age > 0) {
      if (!d->neb_log_age_yr || !strictly_increasing(d->neb_log_age_yr, d->neb_n_age))
        return fail(ctx, SED_EINVAL, "the nebular age axis must be finite and strictly increasing");
      if (d->neb_n_line > 0) return fail(ctx, SED_EUNSUPPORTED, "a line cube with a nebular age axis is not supported");
    }
    size_t nt = (size_t)std::max(d->neb_n_age, 1) * d->neb_n_logu * d->neb_n_logz * nl;
    for (size_t i = 0; i < nt; i++)
      if (!std::isfinite(d->neb_log10_lnu_per_q[i])) return fail(ctx, SED_EINVAL, "nebular template not finite");
  }
  // the SSP ages inside a nebular age axis's tabulated ages
  int neb_a0 = 0, neb_na = 0;
  if (neb && d->neb_n_age > 0) {
    const double lo = d->neb_log_age_yr[0], hi = d->neb_log_age_yr[d->neb_n_age - 1];
    while (neb_a0 < d->n_age && d->log_age_yr[neb_a0] < lo) neb_a0++;
    while (neb_a0 + neb_na < d->n_age && d->log_age_yr[neb_a0 + neb_na] <= hi) neb_na++;
    if (neb_na == 0) return fail(ctx, SED_EINVAL, "no SSP age lies inside the nebular age axis");
    if (neb_na > MAX_NEB_AGE) return fail(ctx, SED_ERANGE, "the nebular age axis spans more than %d SSP ages", MAX_NEB_AGE);
  }
  if (d->neb_n_line < 0 || d->neb_n_line > MAX_LINES)
    return fail(ctx, SED_ERANGE, "neb_n_line must be in [0, %d]", MAX_LINES);
  if (d->neb_n_line > 0) {
    if (!neb) return fail(ctx, SED_EINVAL, "an emission-line cube needs the nebular template and its axes");
    if (!d->neb_line_lam_aa || !d->neb_log10_line_per_q) return fail(ctx, SED_EINVAL, "line cube pointer is NULL");
    for (int l = 0; l < d->neb_n_line; l++)
      if (!(d->neb_line_lam_aa[l] > 0 && std::isfinite(d->neb_line_lam_aa[l])))
        return fail(ctx, SED_EINVAL, "line wavelength %d must be finite and > 0", l);
    const size_t nt = (size_t)d->neb_n_logu * d->neb_n_logz * d->neb_n_line;
    for (size_t i = 0; i < nt; i++)
      if (!std::isfinite(d->neb_log10_line_per_q[i])) return fail(ctx, SED_EINVAL, "line cube not finite");
  }

  Grid* g = new Grid();
  g->n_age = d->n_age; g->n_feh = d->n_feh; g->n_afe = d->n_afe; g->n_lam = d->n_lam;
  g->copies = d->precision_mask ? d->precision_mask : (SED_GRID_COPY_FP32 | SED_GRID_COPY_FP32_SIMT | SED_GRID_COPY_BF16);
  g->avail = d->precision_mask ? d->precision_mask : 15u;
  g->log_age.assign(d->log_age_yr, d->log_age_yr + d->n_age);
  g->feh.assign(d->feh, d->feh + d->n_feh);
  if (d->afe) g->afe.assign(d->afe, d->afe + d->n_afe); else g->afe.assign(1, 0.0);
  g->lam.assign(d->lam_aa, d->lam_aa + nl);
  g->flux.assign(d->flux, d->flux + nsp * nl);
  g->f_log2 = -std::ceil(std::log2(fmax));
  g->f_scale = std::exp2(g->f_log2);

  // Eq. app_q: Q = (Lsun/h) int_0^912 f/lam dlam (trapezoid to the last node
  // below 912 A plus the linearly interpolated piece up to 912 A)
  g->q.assign(nsp, 0.0);
  double qmax = 0.0;
  for (size_t s = 0; s < nsp; s++) {
    const double* f = d->flux + s * nl;
    double acc = 0.0;
    for (size_t k = 0; k + 1 < nl && g->lam[k] < LYMAN_AA; k++) {
      double x1 = g->lam[k + 1], f1 = f[k + 1];
      if (x1 > LYMAN_AA) {
        f1 = f[k] + (f[k + 1] - f[k]) * (LYMAN_AA - g->lam[k]) / (g->lam[k + 1] - g->lam[k]);
        x1 = LYMAN_AA;
      }
      acc += 0.5 * (f[k] / g->lam[k] + f1 / x1) * (x1 - g->lam[k]);
    }
    g->q[s] = LSUN / HPLANCK * acc;
    qmax = std::max(qmax, g->q[s]);
  }
  g->q_log2 = qmax > 0 ? std::ceil(std::log2(qmax)) : 0.0;

  // per-node constants
  std::vector<float> lam_f(nl), inv_lam2(nl), lnp(nl), kp(nl), dr(nl), lh(nl), lo(nl), idl(nl, 0.f);
  g->siglib_kms.resize(nl);
  double hmin = 1e300, hmax = 0.0;
  for (size_t k = 0; k < nl; k++) {
    const double L = g->lam[k];
    lam_f[k] = (float)L;
    inv_lam2[k] = (float)(1.0 / (L * L));
    if (k + 1 < nl) idl[k] = (float)(1.0 / (g->lam[k + 1] - L));
    lnp[k] = (float)std::log(L / 5500.0);
    kp[k] = (float)calzetti_kprime(L * 1e-4);
    const double x = L * 350.0, dd = L * L - 2175.0 * 2175.0;
    dr[k] = (float)(x * x / (dd * dd + x * x));
    const double ll = std::log(L);
    lh[k] = (float)ll;
    lo[k] = (float)(ll - (double)lh[k]);
    double dl = (k == 0) ? g->lam[1] - g->lam[0]
                         : (k == nl - 1 ? g->lam[nl - 1] - g->lam[nl - 2] : 0.5 * (g->lam[k + 1] - g->lam[k - 1]));
    double sl = C_KMS / FWHM_PER_SIGMA * 2.0 * dl / L;  // Eq. app_siglib two-pixel floor
    if (d->sigma_lib_kms && d->sigma_lib_kms[k] > sl) sl = d->sigma_lib_kms[k];
    g->siglib_kms[k] = sl;
    if (k + 1 < nl) {
      hmin = std::min(hmin, std::log(g->lam[k + 1]) - ll);
      hmax = std::max(hmax, std::log(g->lam[k + 1]) - ll);
    }
  }
  // index LUT over ln(lambda): cells of width h <= smallest log spacing
  const double x0 = (double)lh[0];
  const double h = hmin * 0.5;
  const int lut_n = (int)std::ceil(((double)lh[nl - 1] - x0) / h) + 2;
  if (lut_n > (1 << 24)) {
    delete g;
    return fail(ctx, SED_ERANGE, "wavelength axis too unevenly spaced for the index table");
  }
  std::vector<int> lut(lut_n);
  {
    size_t k = 0;
    for (int q = 0; q < lut_n; q++) {
      const double xq = x0 + q * h;
      while (k + 1 < nl && (double)lh[k + 1] <= xq) k++;
      lut[q] = (int)k;
    }
  }
  // linear-time Voronoi cells (App. B step scheme)
  std::vector<float> clo(d->n_age), chi(d->n_age), at(d->n_age), adl(d->n_age, 0.f);
  for (int a = 0; a < d->n_age; a++) {
    at[a] = (float)std::pow(10.0, g->log_age[a]);
    if (a + 1 < d->n_age) adl[a] = (float)((g->log_age[a + 1] - g->log_age[a]) * std::log(10.0));
  }
  for (int a = 0; a < d->n_age; a++) {
    const double ta = std::pow(10.0, g->log_age[a]);
    clo[a] = a == 0 ? 0.f : (float)(0.5 * (std::pow(10.0, g->log_age[a - 1]) + ta));
    chi[a] = a == d->n_age - 1 ? INFINITY : (float)(0.5 * (ta + std::pow(10.0, g->log_age[a + 1])));
  }

  sed_status st = SED_OK;
  GridDev& dv = g->dv;
  dv.n_age = g->n_age; dv.n_feh = g->n_feh; dv.n_afe = g->n_afe; dv.n_lam = g->n_lam;
  float* p;
  int* pi;
#define UPF(field, vec)                                                   \
  if (!st) { st = upload(ctx, &p, vec.data(), vec.size(), &g->allocs, &g->bytes); dv.field = p; }
  UPF(lam_f, lam_f) UPF(inv_lam2, inv_lam2) UPF(inv_dlam, idl) UPF(lnp, lnp) UPF(kprime, kp) UPF(drude, dr)
  UPF(lnl_hi, lh) UPF(lnl_lo, lo) UPF(cell_lo, clo) UPF(cell_hi, chi) UPF(age_t, at) UPF(age_dl, adl)
#undef UPF
  if (!st) { st = upload(ctx, &pi, lut.data(), lut.size(), &g->allocs, &g->bytes); dv.lut = pi; }
  if (!st) {
    std::vector<float4> a4(nl);
    for (size_t k = 0; k < nl; k++)
    {
      const double L = g->lam[k], x = L * 350.0, dd = L * L - 2175.0 * 2175.0;
      a4[k] = make_float4(lnp[k], (float)(calzetti_kprime(L * 1e-4) / 4.05), (float)(x * x / (dd * dd + x * x) / 4.05),
                          lam_f[k]);
    }
    float4* p4;
    st = upload(ctx, &p4, a4.data(), nl, &g->allocs, &g->bytes);
    dv.att4 = p4;
  }
  dv.lut_n = lut_n;
  dv.lut_x0 = (float)x0;
  dv.lut_inv_h = (float)(1.0 / h);
  dv.dln_max = (float)hmax;
  if (neb && !st) {
    g->neb_nu = d->neb_n_logu; g->neb_nz = d->neb_n_logz;
    g->neb_logu.assign(d->neb_logu, d->neb_logu + g->neb_nu);
    g->neb_logz.assign(d->neb_logz, d->neb_logz + g->neb_nz);
    const size_t plane = (size_t)g->neb_nu * g->neb_nz * nl;
    const double off = (g->f_log2 + g->q_log2) * std::log10(2.0);
    std::vector<float> tab(plane * std::max(neb_na, 1));
    if (neb_na == 0) {
      for (size_t i = 0; i < plane; i++) tab[i] = (float)(d->neb_log10_lnu_per_q[i] + off);
    } else {
      // the cube at each SSP age inside it: linear in log age between the two
      // planes bracketing the age (App. C's trilinear interpolation; the bilinear
      // part in log U and log Z_gas is the row's)
      const int na = d->neb_n_age;
      for (int i = 0; i < neb_na; i++) {
        const double la = d->log_age_yr[neb_a0 + i];
        int j = 0;
        while (j + 2 < na && la >= d->neb_log_age_yr[j + 1]) j++;
        const double t = na == 1 ? 0.0 : std::min(std::max((la - d->neb_log_age_yr[j]) /
                                                            (d->neb_log_age_yr[j + 1] - d->neb_log_age_yr[j]), 0.0), 1.0);
        const double* c0 = d->neb_log10_lnu_per_q + (size_t)j * plane;
        const double* c1 = d->neb_log10_lnu_per_q + (size_t)(na == 1 ? j : j + 1) * plane;
        for (size_t q = 0; q < plane; q++) tab[(size_t)i * plane + q] = (float)((1.0 - t) * c0[q] + t * c1[q] + off);
      }
    }
    st = upload(ctx, &p, tab.data(), tab.size(), &g->allocs, &g->bytes);
    dv.neb_tab = p;
    dv.neb_nu = g->neb_nu; dv.neb_nz = g->neb_nz;
    g->neb_a0 = dv.neb_a0 = neb_a0;
    g->neb_na = dv.neb_na = neb_na;
    // emission-line cube: per line the constants of the attenuation at its
    // wavelength, ln(lambda) as an FP32 pair, and log10(L/Q) with the same
    // device-unit offset as the continuum template
    if (!st && d->neb_n_line > 0) {
      const int NLn = d->neb_n_line;
      g->n_line = NLn;
      std::vector<float4> a4(NLn);
      std::vector<float2> l2(NLn);
      for (int l = 0; l < NLn; l++) {
        const double L = d->neb_line_lam_aa[l], x = L * 350.0, dd = L * L - 2175.0 * 2175.0;
        a4[l] = make_float4((float)std::log(L / 5500.0), (float)(calzetti_kprime(L * 1e-4) / 4.05),
                            (float)(x * x / (dd * dd + x * x) / 4.05), (float)L);
        const double ll = std::log(L);
        l2[l].x = (float)ll;
        l2[l].y = (float)(ll - (double)l2[l].x);
      }
      const size_t ntl = (size_t)g->neb_nu * g->neb_nz * NLn;
      std::vector<float> lt(ntl);
      for (size_t i = 0; i < ntl; i++) lt[i] = (float)(d->neb_log10_line_per_q[i] + off);
      float4* p4;
      float2* p2;
      st = upload(ctx, &p4, a4.data(), NLn, &g->allocs, &g->bytes);
      dv.line_att4 = p4;
      if (!st) { st = upload(ctx, &p2, l2.data(), NLn, &g->allocs, &g->bytes); dv.line_ln2 = p2; }
      if (!st) { st = upload(ctx, &p, lt.data(), ntl, &g->allocs, &g->bytes); dv.line_tab = p; }
      dv.n_line = NLn;
    }
  }
  if (st) {
    free_all(ctx, g->allocs, g->bytes);
    delete g;
    return st;
  }
  ctx->grids.push_back(g);
  *out = (sed_grid_id)(ctx->grids.size() - 1);
  return SED_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
namespace {

// Device-scaled SSP flux of layout column k at node l (0 for padding columns
// and, with nebular emission, for young ages below 912 A).
float ssp_value(const Grid* g, const Layout* L, int k, int l) {
  const int c = L->code_h[k];
  if (c < 0) return 0.f;
  const int n = c >> 24, m = (c >> 16) & 0xff, a = c & 0xffff;
  if (L->neb_cut && a >= L->neb_a0 && a < L->n_young && g->lam[l] < LYMAN_AA) return 0.f;
  return (float)(g->flux[(((size_t)n * g->n_feh + m) * g->n_age + a) * g->n_lam + l] * g->f_scale);
}

// Lambda-major copies of a layout for the adjoint contraction: [Kpad][ldn].
sed_status ensure_grad_layout(sed_ctx* ctx, Grid* g, Layout* L, int ldn) {
  if (L->sspK_f32) return SED_OK;
  const int Kpad = L->Kpad, NL = g->n_lam;
  std::vector<float> f32((size_t)Kpad * ldn, 0.f), hi((size_t)Kpad * ldn, 0.f), lo((size_t)Kpad * ldn, 0.f);
  for (int k = 0; k < Kpad; k++)
    for (int l = 0; l < NL; l++) {
      const float v = ssp_value(g, L, k, l);
      const size_t o = (size_t)k * ldn + l;
      f32[o] = v;
      hi[o] = tf32_rna_host(v);
      lo[o] = v - hi[o];
    }
  float *a = nullptr, *b = nullptr, *c = nullptr;
  sed_status st = upload(ctx, &a, f32.data(), f32.size(), &g->allocs, &g->bytes);
  if (!st) st = upload(ctx, &b, hi.data(), hi.size(), &g->allocs, &g->bytes);
  if (!st) st = upload(ctx, &c, lo.data(), lo.size(), &g->allocs, &g->bytes);
  if (st) return st;
  L->ldn = ldn;
  L->sspK_f32 = a;
  L->sspK_hi = b;
  L->sspK_lo = c;
  return SED_OK;
}

// FP8 copy of a layout.  E4M3 has a 3-bit mantissa and covers 2^-9..448, while
// the SSP fluxes span ~1e-6..1 across ages and further decades across
// wavelength, so the matrix is balanced by powers of two before rounding:
// SSP[k][l] 2^(e_k + f_l), with e_k (per column k = age, [Fe/H], [a/Fe]) and
// f_l (per wavelength) chosen by alternating passes so that every column and
// every wavelength row peaks in [120, 240].  e_k is folded into W by the prep
// kernel, f_l is undone in the epilogue (Y and O times 2^-f_l).  The young and
// old blocks are each padded to 128 columns (one 128-byte K tile).
sed_status ensure_f8_layout(sed_ctx* ctx, Grid* g, Layout* L) {
  if (L->sspT_f8) return SED_OK;
  const int NL = g->n_lam, Kpad = L->Kpad;
  const int Ky_pad8 = (L->Ky_pad + 127) / 128 * 128;
  const int Kpad8 = Ky_pad8 + (Kpad - L->Ky_pad + 127) / 128 * 128;
  std::vector<float> v((size_t)Kpad * NL);
  for (int k = 0; k < Kpad; k++)
    for (int l = 0; l < NL; l++) v[(size_t)k * NL + l] = ssp_value(g, L, k, l);
  std::vector<int> ek(Kpad, 0), fl(NL, 0);
  std::vector<double> sk(Kpad, 1.0), sl(NL, 1.0);   // 2^e_k, 2^f_l
  std::vector<char> live(Kpad, 0);
  for (int it = 0; it < 4; it++) {
    for (int k = 0; k < Kpad; k++) {
      double m = 0.0;
      const float* vk = v.data() + (size_t)k * NL;
      for (int l = 0; l < NL; l++) m = std::max(m, (double)vk[l] * sl[l]);
      live[k] = m > 0.0;
      if (m > 0.0) { ek[k] = (int)std::floor(std::log2(240.0 / m)); sk[k] = std::ldexp(1.0, ek[k]); }
    }
    std::vector<double> ml(NL, 0.0);
    for (int k = 0; k < Kpad; k++) {
      if (!live[k]) continue;
      const float* vk = v.data() + (size_t)k * NL;
      for (int l = 0; l < NL; l++) ml[l] = std::max(ml[l], (double)vk[l] * sk[k]);
    }
    for (int l = 0; l < NL; l++)
      if (ml[l] > 0.0) { fl[l] = (int)std::floor(std::log2(240.0 / ml[l])); sl[l] = std::ldexp(1.0, fl[l]); }
  }
  std::vector<float> col(Kpad, 0.f), lsc(NL);
  for (int k = 0; k < Kpad; k++) col[k] = live[k] ? (float)(1.0 / sk[k]) : 0.f;
  for (int l = 0; l < NL; l++) lsc[l] = (float)(1.0 / sl[l]);
  std::vector<uint8_t> f8((size_t)NL * Kpad8, 0);
  for (int p = 0; p < Kpad8; p++) {
    const int k = p < L->Ky_pad ? p : (p < Ky_pad8 ? -1 : p - (Ky_pad8 - L->Ky_pad));
    if (k < 0 || k >= Kpad || !live[k]) continue;
    for (int l = 0; l < NL; l++)
      f8[(size_t)l * Kpad8 + p] = (uint8_t)__nv_cvt_float_to_fp8(
          (float)((double)v[(size_t)k * NL + l] * sk[k] * sl[l]), __NV_SATFINITE, __NV_E4M3);
  }
  uint8_t* a = nullptr;
  float *c = nullptr, *d = nullptr;
  sed_status st = upload(ctx, &a, f8.data(), f8.size(), &g->allocs, &g->bytes);
  if (!st) st = upload(ctx, &c, col.data(), col.size(), &g->allocs, &g->bytes);
  if (!st) st = upload(ctx, &d, lsc.data(), lsc.size(), &g->allocs, &g->bytes);
  if (st) return st;
  L->Ky_pad8 = Ky_pad8;
  L->Kpad8 = Kpad8;
  L->sspT_f8 = a;
  L->col8 = c;
  L->lam8 = d;
  return SED_OK;
}

// Layout of the grid for a block assignment of the ages and 912 A removal:
// the attenuated blocks (age a in block blk[a] >= 0), then the ages outside
// every block (blk[a] = -1), each block ordered (afe n, feh m, age a) with age
// fastest.  One attenuated block is padded to KT; several are padded to 128
// columns each, so that every precision's K tiles (32, 64 and 128 columns)
// and the adjoint's 128-column output tiles lie within one block.  Nebular
// ages (the first n_neb) carry Q and, with neb_cut, lose their flux below 912 A.
sed_status get_layout(sed_ctx* ctx, Grid* g, const std::vector<int>& blk, int neb0, int n_neb, int neb_cut,
                      Layout** out) {
  for (Layout* L : g->layouts)
    if (L->blk == blk && L->neb_a0 == neb0 && L->n_young == n_neb && L->neb_cut == neb_cut) { *out = L; return SED_OK; }
  Layout* L = new Layout();
  L->blk = blk;
  L->neb_a0 = neb0;
  L->n_young = n_neb;
  L->neb_cut = neb_cut;
  const int NA = g->n_age, NZ = g->n_feh, NAF = g->n_afe, NL = g->n_lam;
  int n_seg = 0;
  for (int a = 0; a < NA; a++) n_seg = std::max(n_seg, blk[a] + 1);
  n_seg = std::max(n_seg, 1);
  L->n_seg = n_seg;
  // ages of each block in age order (block n_seg: outside every bin)
  std::vector<std::vector<int>> ages(n_seg + 1);
  for (int a = 0; a < NA; a++) ages[blk[a] >= 0 ? blk[a] : n_seg].push_back(a);
  const int pad = n_seg > 1 ? 128 : KT;
  int k0 = 0;
  for (int s = 0; s < n_seg; s++) {
    L->seg_k0[s] = k0;
    k0 += ((int)(NAF * NZ * ages[s].size()) + pad - 1) / pad * pad;
  }
  for (int s = n_seg; s <= MAX_SEG; s++) L->seg_k0[s] = k0;
  L->Ky_pad = k0;
  L->Ky = n_seg > 1 ? k0 : NAF * NZ * (int)ages[0].size();
  L->Ko = NAF * NZ * (int)ages[n_seg].size();
  L->Kpad = L->Ky_pad + (L->Ko + KT - 1) / KT * KT;
  const int Kpad = L->Kpad;
  std::vector<int> code(Kpad, -1);
  std::vector<float> qs(Kpad, 0.f);
  std::vector<int4> acol(NA);
  for (int s = 0; s <= n_seg; s++) {
    const int base = s < n_seg ? L->seg_k0[s] : L->Ky_pad, len = (int)ages[s].size();
    for (int i = 0; i < len; i++) acol[ages[s][i]] = make_int4(base + i, len, s < n_seg ? s : MAX_SEG, 0);
    for (int n = 0; n < NAF; n++)
      for (int m = 0; m < NZ; m++)
        for (int i = 0; i < len; i++) {
          const int a = ages[s][i];
          const int k = base + (n * NZ + m) * len + i;
          code[k] = (n << 24) | (m << 16) | a;
          if (a >= neb0 && a < n_neb) qs[k] = (float)(g->q[((size_t)n * NZ + m) * NA + a] * std::exp2(-g->q_log2));
        }
  }
  L->q_log2 = g->q_log2;
  sed_status st = upload(ctx, &L->k_code, code.data(), Kpad, &g->allocs, &g->bytes);
  if (!st) st = upload(ctx, &L->age_col, acol.data(), NA, &g->allocs, &g->bytes);
  if (!st) st = upload(ctx, &L->q_s, qs.data(), Kpad, &g->allocs, &g->bytes);
  // SSP^T [lam][k], scaled by 2^f_log2, in FP32, TF32 hi/lo and BF16 (the
  // copies the grid keeps; FP8 below when it is asked for at load)
  L->code_h = code;
  const bool c_hl = g->copies & SED_GRID_COPY_FP32, c_f = g->copies & SED_GRID_COPY_FP32_SIMT,
             c_b = g->copies & SED_GRID_COPY_BF16;
  const size_t NE = (size_t)NL * Kpad;
  std::vector<float> f32(c_f ? NE : 0), hi(c_hl ? NE : 0), lo(c_hl ? NE : 0);
  std::vector<__nv_bfloat16> bf(c_b ? NE : 0);
  for (int k = 0; k < Kpad; k++) {
    for (int l = 0; l < NL; l++) {
      const float v = ssp_value(g, L, k, l);
      const size_t o = (size_t)l * Kpad + k;
      if (c_f) f32[o] = v;
      if (c_hl) {
        const float h = tf32_rna_host(v);
        hi[o] = h;
        lo[o] = v - h;
      }
      if (c_b) bf[o] = __float2bfloat16_rn(v);
    }
  }
  if (!st && c_f) st = upload(ctx, &L->sspT_f32, f32.data(), f32.size(), &g->allocs, &g->bytes);
  if (!st && c_hl) st = upload(ctx, &L->sspT_hi, hi.data(), hi.size(), &g->allocs, &g->bytes);
  if (!st && c_hl) st = upload(ctx, &L->sspT_lo, lo.data(), lo.size(), &g->allocs, &g->bytes);
  if (!st && c_b) st = upload(ctx, &L->sspT_bf16, bf.data(), bf.size(), &g->allocs, &g->bytes);
  if (!st && (g->copies & SED_GRID_COPY_FP8)) st = ensure_f8_layout(ctx, g, L);
  if (st) {
    delete L;
    return st;
  }
  g->layouts.push_back(L);
  *out = L;
  return SED_OK;
}

double sigma_inst_kms(int mode, double v, double lam_obs) {  // Eq. app_modes
  switch (mode) {
    case SED_LSF_R_FWHM: return C_KMS / (FWHM_PER_SIGMA * v);
    case SED_LSF_R_SIGMA: return C_KMS / v;
    case SED_LSF_FWHM_AA: return C_KMS * v / (FWHM_PER_SIGMA * lam_obs);
    case SED_LSF_SIGMA_AA: return C_KMS * v / lam_obs;
    case SED_LSF_SIGMA_KMS: return v;
    default: return v / FWHM_PER_SIGMA;
  }
}

// t_univ(z) in yr, closed form for flat LCDM without radiation
double t_univ_yr(double th_yr, double Om, double z) {
  const double OL = 1.0 - Om;
  return th_yr * 2.0 / (3.0 * std::sqrt(OL)) * std::asinh(std::sqrt(OL / Om) * std::pow(1.0 + z, -1.5));
}

// Cosmology table of a model (flat LCDM without radiation, Sec. 2.6): at
// z_i = i zf / n, D_C(z_i) = (c/H0) int_0^z_i dz/E by 16-point Gauss-Legendre
// on each interval (FP64, accumulated), its derivative c/(H0 E), the age of
// the Universe t(z_i) in closed form and dt/dz = -1/(H0 (1+z) E), and
// ln(1+z) and 1/(1+z) with their derivatives.
void cosmo_table(double H0, double Om, double zf, int n, std::vector<double>* out) {
  static const double x16[8] = {0.0950125098376374, 0.2816035507792589, 0.4580167776572274, 0.6178762444026438,
                                0.7554044083550030, 0.8656312023878318, 0.9445750230732326, 0.9894009349916499};
  static const double w16[8] = {0.1894506104550685, 0.1826034150449236, 0.1691565193950025, 0.1495959888165767,
                                0.1246289712555339, 0.0951585116824928, 0.0622535239386479, 0.0271524594117541};
  const double OL = 1.0 - Om, dh = C_KMS / H0 * 1e6 * PC_CM, thy = MPC_KM / H0 / YR_S, h = zf / n;
  auto E = [&](double z) { const double zp = 1.0 + z; return std::sqrt(Om * zp * zp * zp + OL); };
  out->assign((size_t)(n + 1) * COSMO_COLS, 0.0);
  double dc = 0.0;
  for (int i = 0; i <= n; i++) {
    const double z = i * h;
    if (i > 0) {
      const double a = z - h, mid = a + 0.5 * h, hw = 0.5 * h;
      double acc = 0.0;
      for (int k = 0; k < 8; k++) acc += w16[k] * (1.0 / E(mid - hw * x16[k]) + 1.0 / E(mid + hw * x16[k]));
      dc += dh * hw * acc;
    }
    double* t = out->data() + COSMO_COLS * (size_t)i;
    t[0] = dc;
    t[1] = dh / E(z);
    t[2] = t_univ_yr(thy, Om, z);
    t[3] = -thy / ((1.0 + z) * E(z));
    t[4] = std::log1p(z);
    t[5] = 1.0 / (1.0 + z);
    t[6] = 1.0 / (1.0 + z);
    t[7] = -1.0 / ((1.0 + z) * (1.0 + z));
  }
}

// The device address of a page-locked, device-mapped host buffer, or NULL
// (pageable or unknown memory).
void* mapped_host(const void* p) {
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return at.type == cudaMemoryTypeHost ? at.devicePointer : nullptr;
}

sed_status set_data_dev(sed_ctx* ctx, Model* M, const double* pd, const double* ps, const double* sd,
                        const double* ss) {
  ModelDev& dv = M->dv;
  // a pair passed as NULL keeps its last value; one never set stays out of lnL
  // (its device arrays hold zeros).  Copies first (a caller's array may be the
  // kept one), then every datum checked before anything is uploaded: the call
  // changes all or nothing
  const bool ph = pd || ps || !M->phot_d_h.empty(), sp = sd || ss || !M->spec_d_h.empty();
  const int nb = ph ? dv.n_filt : 0, np = sp ? dv.n_pix : 0;
  // (sed_create_model may give data without sigma: sigma 1 then)
  auto pick = [](const double* given, const std::vector<double>& kept, int n, double dflt) {
    if (given) return std::vector<double>(given, given + n);
    if (kept.size() == (size_t)n) return kept;
    return std::vector<double>(n, dflt);
  };
  std::vector<double> pdv = pick(pd, M->phot_d_h, nb, 0.0), psv = pick(ps, M->phot_s_h, nb, 1.0);
  std::vector<double> sdv = pick(sd, M->spec_d_h, np, 0.0), ssv = pick(ss, M->spec_s_h, np, 1.0);
  std::vector<double> p_d(nb), p_isig(nb), p_nlog(nb);
  std::vector<float> p_dn(nb), p_isf(nb);
  for (int b = 0; b < nb; b++) {
    const bool on = M->phot_mask_h.empty() || M->phot_mask_h[b];
    const double s = psv[b], dv_ = pdv[b];
    if (on && !(std::isfinite(s) && s > 0 && std::isfinite(dv_)))
      return fail(ctx, SED_EINVAL, "photometric datum %d: sigma must be > 0 and data finite", b);
    const double is = 1.0 / s, dn_ = dv_ * is;
    if (on && !(is >= (double)FLT_MIN && is <= (double)FLT_MAX && std::fabs(dn_) <= (double)FLT_MAX))
      return fail(ctx, SED_EINVAL, "photometric datum %d: 1/sigma and d/sigma must lie in FP32's normal range", b);
    p_d[b] = on ? dv_ : 0.0;
    p_isig[b] = on ? is : 0.0;
    p_nlog[b] = on ? -0.5 * std::log(2.0 * M_PI * s * s) : 0.0;
    p_dn[b] = on ? (float)dn_ : 0.f;
    p_isf[b] = on ? (float)is : 0.f;
  }
  std::vector<float> s_dn(np), s_isf(np);
  std::vector<double> s_nlog(np);
  for (int i = 0; i < np; i++) {
    const bool on = M->spec_mask_h.empty() || M->spec_mask_h[i];
    const double s = ssv[i], dv_ = sdv[i];
    if (on && !(std::isfinite(s) && s > 0 && std::isfinite(dv_)))
      return fail(ctx, SED_EINVAL, "spectral datum %d: sigma must be > 0 and data finite", i);
    // the kernels take d/sigma and 1/sigma in FP32: both must be finite there
    // and 1/sigma a normal number
    const double is = 1.0 / s, dn_ = dv_ * is;
    if (on && !(is >= (double)FLT_MIN && is <= (double)FLT_MAX && std::fabs(dn_) <= (double)FLT_MAX))
      return fail(ctx, SED_EINVAL, "spectral datum %d: 1/sigma and d/sigma must lie in FP32's normal range", i);
    s_dn[i] = on ? (float)dn_ : 0.f;
    s_isf[i] = on ? (float)is : 0.f;
    s_nlog[i] = on ? -0.5 * std::log(2.0 * M_PI * s * s) : 0.0;
  }
  if (nb) {
    CK(cudaMemcpy((void*)dv.phot_d, p_d.data(), nb * 8, cudaMemcpyHostToDevice));
    CK(cudaMemcpy((void*)dv.phot_isig, p_isig.data(), nb * 8, cudaMemcpyHostToDevice));
    CK(cudaMemcpy((void*)dv.phot_nlog, p_nlog.data(), nb * 8, cudaMemcpyHostToDevice));
    CK(cudaMemcpy((void*)dv.phot_dn, p_dn.data(), nb * 4, cudaMemcpyHostToDevice));
    CK(cudaMemcpy((void*)dv.phot_isf, p_isf.data(), nb * 4, cudaMemcpyHostToDevice));
  }
  if (np) {
    CK(cudaMemcpy((void*)dv.spec_dn, s_dn.data(), np * 4, cudaMemcpyHostToDevice));
    CK(cudaMemcpy((void*)dv.spec_isf, s_isf.data(), np * 4, cudaMemcpyHostToDevice));
    CK(cudaMemcpy((void*)dv.spec_nlog, s_nlog.data(), np * 8, cudaMemcpyHostToDevice));
  }
  if (ph) {
    M->phot_d_h.swap(pdv);
    M->phot_s_h.swap(psv);
  }
  if (sp) {
    M->spec_d_h.swap(sdv);
    M->spec_s_h.swap(ssv);
  }
  return SED_OK;
}

}  // namespace

extern "C" {

sed_status sed_create_model(sed_ctx* ctx, const sed_model_desc* d, sed_model_id* out) {
  if (!ctx || !d || !out) return fail(ctx, SED_EINVAL, "null argument");
  std::lock_guard<std::mutex> lk(ctx->mu);
  DevGuard dg(ctx->device);
  if (d->grid < 0 || d->grid >= (int)ctx->grids.size() || !ctx->grids[d->grid])
    return fail(ctx, SED_EINVAL, "unknown grid id %d", d->grid);
  Grid* g = ctx->grids[d->grid];
  if (d->n_sfh < 3 || d->n_sfh > MAX_SFH) return fail(ctx, SED_ERANGE, "n_sfh must be in [3, %d]", MAX_SFH);
  if (!(d->zf > 0 && std::isfinite(d->zf))) return fail(ctx, SED_EINVAL, "zf must be > 0");
  if (d->zmode != 0 && d->zmode != 1) return fail(ctx, SED_EINVAL, "zmode must be 0 or 1");
  if (d->dust_law != SED_DUST_POWER_LAW && d->dust_law != SED_DUST_KC13) return fail(ctx, SED_EINVAL, "bad dust_law");
  if (!(d->H0 > 0) || !(d->Om0 > 0 && d->Om0 < 1)) return fail(ctx, SED_EINVAL, "need H0 > 0 and 0 < Om0 < 1");
  if (d->use_nebular && g->neb_nu == 0) return fail(ctx, SED_EINVAL, "use_nebular needs a grid with a nebular template");
  if (d->use_afe && g->n_afe < 2) return fail(ctx, SED_EINVAL, "use_afe needs a grid with an [a/Fe] axis");
  if (d->n_filt < 0 || d->n_filt > 128) return fail(ctx, SED_ERANGE, "n_filt must be in [0, 128]");
  if (d->n_pix < 0) return fail(ctx, SED_EINVAL, "n_pix < 0");
  if (d->n_filt == 0 && d->n_pix == 0 && d->n_lcat <= 0) return fail(ctx, SED_EINVAL, "model has no observation");
  if (!std::isfinite(d->bc_edge_log_age_yr)) return fail(ctx, SED_EINVAL, "bc edge not finite");
  if (d->n_filt && (!d->filt_len || !d->filt_lam_aa || !d->filt_trans))
    return fail(ctx, SED_EINVAL, "filter arrays are NULL");
  if (d->n_pix && (!d->spec_lam_aa || !d->lsf_value)) return fail(ctx, SED_EINVAL, "spectrum arrays are NULL");
  if (d->n_pix && (d->lsf_mode < 0 || d->lsf_mode > 5)) return fail(ctx, SED_EINVAL, "bad lsf_mode");
  if (d->n_pix && !(d->sigma_gal_kms >= 0 && d->z_ref >= 0)) return fail(ctx, SED_EINVAL, "sigma_gal, z_ref must be >= 0");
  if (d->sample_sigma_gal != 0 && d->sample_sigma_gal != 1) return fail(ctx, SED_EINVAL, "sample_sigma_gal must be 0 or 1");
  if (d->calib_mode != SED_CALIB_MARGINAL && d->calib_mode != SED_CALIB_OPTIMISED)
    return fail(ctx, SED_EINVAL, "calib_mode must be SED_CALIB_MARGINAL or SED_CALIB_OPTIMISED");
  if (d->calib_n < 0 || d->calib_n > SED_MAX_CALIB)
    return fail(ctx, SED_EINVAL, "calib_n must be in [0, %d]", SED_MAX_CALIB);
  if (d->calib_n > 0) {
    if (!d->n_pix) return fail(ctx, SED_EINVAL, "a calibration polynomial needs a spectrum");
    if (!d->calib_sigma) return fail(ctx, SED_EINVAL, "calib_sigma is NULL");
    for (int m = 0; m < d->calib_n; m++)
      if (!(d->calib_sigma[m] > 0 && std::isfinite(d->calib_sigma[m])))
        return fail(ctx, SED_EINVAL, "calib_sigma[%d] must be finite and > 0", m);
  }
  if (d->sample_sigma_gal && !(d->sigma_gal_max_kms > 0 && d->sigma_gal_max_kms < 1e5))
    return fail(ctx, SED_EINVAL, "sigma_gal_max_kms must be in (0, 1e5) when sigma_gal is sampled");
  if (d->sfh_scheme != SED_SFH_STEP && d->sfh_scheme != SED_SFH_LINEAR)
    return fail(ctx, SED_EINVAL, "sfh_scheme must be SED_SFH_STEP or SED_SFH_LINEAR");
  if (d->fesc_geometry < SED_FESC_NONE || d->fesc_geometry > SED_FESC_PICKET)
    return fail(ctx, SED_EINVAL, "fesc_geometry must be SED_FESC_NONE, SED_FESC_RUNAWAY_BC or SED_FESC_PICKET");
  if (d->noise_floor_phot < 0 || d->noise_floor_phot > 15 || d->noise_floor_spec < 0 || d->noise_floor_spec > 15)
    return fail(ctx, SED_EINVAL, "noise_floor_phot / noise_floor_spec must be SED_FLOOR_* bits (0..15)");
  if (d->noise_floor_phot && d->n_filt <= 0) return fail(ctx, SED_EINVAL, "a photometric noise floor needs filters");
  if (d->noise_floor_spec && d->n_pix <= 0) return fail(ctx, SED_EINVAL, "a spectral noise floor needs a spectrum");
  if (d->noise_floor_spec && d->calib_n > 0)
    return fail(ctx, SED_EUNSUPPORTED, "a spectral noise floor with the calibration polynomial is not supported");
  if (d->use_lines != 0 && d->use_lines != 1) return fail(ctx, SED_EINVAL, "use_lines must be 0 or 1");
  if (d->use_lines && (!d->use_nebular || g->n_line == 0))
    return fail(ctx, SED_EINVAL, "emission lines need use_nebular and a grid with a line cube");
  if (d->gas_sigma_mode < SED_GAS_SIGMA_TIED || d->gas_sigma_mode > SED_GAS_SIGMA_SAMPLED)
    return fail(ctx, SED_EINVAL, "gas_sigma_mode must be SED_GAS_SIGMA_TIED, _FIXED or _SAMPLED");
  if (d->use_lines && d->gas_sigma_mode == SED_GAS_SIGMA_FIXED && !(d->sigma_gas_kms >= 0 && d->sigma_gas_kms < 1e5))
    return fail(ctx, SED_EINVAL, "sigma_gas_kms must be in [0, 1e5)");
  if (d->use_lines && d->gas_sigma_mode == SED_GAS_SIGMA_SAMPLED &&
      !(d->sigma_gas_max_kms > 0 && d->sigma_gas_max_kms < 1e5))
    return fail(ctx, SED_EINVAL, "sigma_gas_max_kms must be in (0, 1e5) when sigma_gas is sampled");
  if (d->n_lcat < 0 || d->n_lcat > 1024) return fail(ctx, SED_ERANGE, "n_lcat must be in [0, 1024]");
  if (d->n_lcat > 0) {
    if (!d->use_lines) return fail(ctx, SED_EINVAL, "a line catalogue needs use_lines");
    if (!d->lcat_len || !d->lcat_line || !d->lcat_d || !d->lcat_sigma)
      return fail(ctx, SED_EINVAL, "line catalogue arrays are NULL");
    int c = 0;
    for (int k = 0; k < d->n_lcat; k++) {
      if (d->lcat_len[k] < 1 || d->lcat_len[k] > MAX_LINES) return fail(ctx, SED_EINVAL, "lcat_len[%d] out of range", k);
      for (int j = 0; j < d->lcat_len[k]; j++, c++)
        if (d->lcat_line[c] < 0 || d->lcat_line[c] >= g->n_line)
          return fail(ctx, SED_EINVAL, "line catalogue entry %d names line %d of %d", k, d->lcat_line[c], g->n_line);
      if (!std::isfinite(d->lcat_d[k]) || !(d->lcat_sigma[k] > 0 && std::isfinite(d->lcat_sigma[k])))
        return fail(ctx, SED_EINVAL, "line catalogue entry %d: datum not finite or sigma <= 0", k);
    }
  }
  if (d->use_nebular && g->neb_na > 0) {
    if (d->fesc_geometry || d->dust_n_bin > 0 || d->use_lines)
      return fail(ctx, SED_EUNSUPPORTED, "a nebular age axis is not combined with an escape geometry, age-binned "
                                         "dust or emission lines");
    if (g->log_age[g->neb_a0 + g->neb_na - 1] > d->bc_edge_log_age_yr)
      return fail(ctx, SED_EUNSUPPORTED, "the nebular age axis reaches past the birth-cloud edge");
  }
  if (d->use_igm != SED_IGM_NONE && d->use_igm != SED_IGM_MADAU)
    return fail(ctx, SED_EINVAL, "use_igm must be SED_IGM_NONE or SED_IGM_MADAU");
  if (d->dust_n_bin < 0 || d->dust_n_bin > MAX_DUST_BIN)
    return fail(ctx, SED_EINVAL, "dust_n_bin must be in [0, %d]", MAX_DUST_BIN);
  // age-binned attenuation: the ages with one non-zero row of M form one
  // attenuated block
  std::vector<int> blk(g->n_age, -1);
  std::vector<std::vector<double>> seg_rows;
  if (d->dust_n_bin > 0) {
    const int nb = d->dust_n_bin;
    if (!d->dust_bin_M || !d->dust_bin_law) return fail(ctx, SED_EINVAL, "dust_bin_M / dust_bin_law is NULL");
    if (d->use_lines || d->fesc_geometry)
      return fail(ctx, SED_EUNSUPPORTED, "age-binned dust is not combined with emission lines or an escape geometry");
    for (int b = 0; b < nb; b++)
      if (d->dust_bin_law[b] != SED_DUST_POWER_LAW && d->dust_bin_law[b] != SED_DUST_KC13)
        return fail(ctx, SED_EINVAL, "dust_bin_law[%d] must be SED_DUST_POWER_LAW or SED_DUST_KC13", b);
    for (int a = 0; a < g->n_age; a++) {
      const double* row = d->dust_bin_M + (size_t)a * nb;
      double sum = 0.0;
      for (int b = 0; b < nb; b++) {
        if (!(row[b] >= 0.0 && row[b] <= 1.0)) return fail(ctx, SED_EINVAL, "dust_bin_M[%d][%d] not in [0, 1]", a, b);
        sum += row[b];
      }
      if (sum == 0.0) continue;
      if (std::fabs(sum - 1.0) > 1e-9) return fail(ctx, SED_EINVAL, "row %d of dust_bin_M sums to %g (not 0 or 1)", a, sum);
      std::vector<double> r(row, row + nb);
      int s = 0;
      while (s < (int)seg_rows.size() && seg_rows[s] != r) s++;
      if (s == (int)seg_rows.size()) {
        if (s == MAX_SEG)
          return fail(ctx, SED_EUNSUPPORTED, "dust_bin_M has more than %d distinct non-zero rows", MAX_SEG);
        seg_rows.push_back(r);
      }
      blk[a] = s;
    }
  }

  Model* M = new Model();
  M->grid = d->grid;
  M->g = g;
  M->bc_edge = d->bc_edge_log_age_yr;
  M->H0 = d->H0;
  ModelDev& dv = M->dv;
  memset(&dv, 0, sizeof dv);
  dv.n_sfh = d->n_sfh; dv.zmode = d->zmode; dv.use_afe = d->use_afe; dv.use_neb = d->use_nebular;
  dv.dust_law = d->dust_law;
  const int nz = d->zmode == 0 ? d->n_sfh : 1;
  int o = 0;
  dv.sfh_linear = d->sfh_scheme == SED_SFH_LINEAR ? 1 : 0;
  dv.offs[SED_KEY_SFH] = o; o += d->n_sfh + dv.sfh_linear;   // bin masses, or edge SFRs (one more)
  dv.offs[SED_KEY_LOGZSOL] = o; o += nz;
  for (int k = SED_KEY_AFE; k <= SED_KEY_GAS_LOGU; k++) dv.offs[k] = o++;
  dv.offs[SED_KEY_SIGMA_GAL] = o;
  o += d->sample_sigma_gal ? 1 : 0;
  // noise-floor terms (App. sys_floor): photometry then spectrum, in SED_FLOOR_* bit order
  dv.floor_bits[0] = d->noise_floor_phot;
  dv.floor_bits[1] = d->noise_floor_spec;
  for (int arm = 0; arm < 2; arm++)
    for (int k = 0; k < 4; k++) {
      dv.offs[SED_KEY_LOG_ERR_SCALE_PHOT + 4 * arm + k] = o;
      o += (dv.floor_bits[arm] >> k) & 1;
    }
  // runaway fraction of an escape geometry (Sec. frac_obrun)
  dv.fesc_geom = d->fesc_geometry;
  dv.offs[SED_KEY_FRAC_OBRUN] = o;
  o += d->fesc_geometry ? 1 : 0;
  // gas dispersion of the emission lines when sampled (Sec. 2.7)
  dv.use_lines = d->use_lines;
  dv.gas_mode = d->use_lines ? d->gas_sigma_mode : SED_GAS_SIGMA_FIXED;
  dv.sgas_fix_kms = (float)d->sigma_gas_kms;
  dv.sgas_max_kms = (float)d->sigma_gas_max_kms;
  dv.sgal_fix_kms = (float)d->sigma_gal_kms;
  dv.offs[SED_KEY_SIGMA_GAS] = o;
  o += dv.gas_mode == SED_GAS_SIGMA_SAMPLED ? 1 : 0;
  // age-binned attenuation (App. dust_attn): (tau_b, slope_b) per bin
  dv.n_bin = d->dust_n_bin;
  dv.n_seg = d->dust_n_bin > 0 ? std::max((int)seg_rows.size(), 1) : 1;
  for (int b = 0; b < dv.n_bin; b++) dv.bin_law[b] = d->dust_bin_law[b];
  for (int s = 0; s < (int)seg_rows.size(); s++)
    for (int b = 0; b < dv.n_bin; b++) dv.seg_M[s][b] = (float)seg_rows[s][b];
  dv.offs[SED_KEY_DUST_BINS] = o;
  o += 2 * d->dust_n_bin;
  // the IGM transmission's scaling (Sec. 2.6)
  dv.use_igm = d->use_igm;
  dv.offs[SED_KEY_IGM_FACTOR] = o;
  o += d->use_igm ? 1 : 0;
  // fixed keys (Sec. 4 parameter dictionary): a fixed one-column key leaves the
  // caller's rows; the kernels read it past the caller's columns
  {
    int width[SED_NKEYS];
    for (int k = 0; k < SED_NKEYS; k++) width[k] = (k + 1 < SED_NKEYS ? dv.offs[k + 1] : o) - dv.offs[k];
    for (int k = 0; k < SED_NKEYS; k++) {
      if (!d->fixed[k]) continue;
      if (k == SED_KEY_SFH || width[k] != 1) {
        delete M;
        return fail(ctx, SED_EINVAL, "key %d cannot be fixed (only keys with one column in this model)", k);
      }
      if (!std::isfinite(d->fixed_val[k])) {
        delete M;
        return fail(ctx, SED_EINVAL, "fixed_val[%d] is not finite", k);
      }
    }
    int c = 0, nf = 0;
    int in_off[SED_NKEYS];
    for (int k = 0; k < SED_NKEYS; k++) {
      M->offs_caller[k] = c;
      in_off[k] = c;
      if (!d->fixed[k]) c += width[k];
    }
    for (int k = 0; k < SED_NKEYS; k++) {
      if (d->fixed[k]) {
        in_off[k] = c + nf;
        dv.fixed_v[nf++] = (float)d->fixed_val[k];
      }
      dv.offs[k] = in_off[k];
    }
    o = c;
    dv.n_fixed = nf;
  }
  dv.n_param = o;
  dv.zf = d->zf;
  dv.Om0 = d->Om0;
  dv.dh_cm = C_KMS / d->H0 * 1e6 * PC_CM;
  dv.th_yr = MPC_KM / d->H0 / YR_S;
  dv.t_zf_yr = t_univ_yr(dv.th_yr, d->Om0, d->zf);
  dv.lsun_c = LSUN * std::exp2(-g->f_log2) / (4.0 * M_PI);
  dv.f_log2 = g->f_log2;
  dv.q_log2 = g->q_log2;
  dv.n_feh = g->n_feh; dv.n_afe = g->n_afe;
  for (int i = 0; i < g->n_feh; i++) dv.feh[i] = (float)g->feh[i];
  for (int i = 0; i < g->n_afe; i++) dv.afe[i] = (float)g->afe[i];
  dv.neb_nu = g->neb_nu; dv.neb_nz = g->neb_nz;
  for (int i = 0; i < g->neb_nu; i++) dv.neb_logu[i] = (float)g->neb_logu[i];
  for (int i = 0; i < g->neb_nz; i++) dv.neb_logz[i] = (float)g->neb_logz[i];

  int n_young = 0;
  while (n_young < g->n_age && g->log_age[n_young] <= d->bc_edge_log_age_yr) n_young++;
  // the young ages' flux below 912 A is removed from the SSP copy when the
  // nebular emission absorbs all of it; with an escape geometry the copy keeps
  // it and the epilogues split it off (nodes below n_lyc)
  while (dv.n_lyc < g->n_lam && g->lam[dv.n_lyc] < LYMAN_AA) dv.n_lyc++;
  if (d->dust_n_bin == 0)
    for (int a = 0; a < g->n_age; a++) blk[a] = a < n_young ? 0 : -1;
  // the nebular ages: the birth-cloud ages, or those a nebular age axis spans
  const bool axis = d->use_nebular && g->neb_na > 0;
  sed_status st = get_layout(ctx, g, blk, axis ? g->neb_a0 : 0, axis ? g->neb_a0 + g->neb_na : n_young,
                             d->use_nebular && !d->fesc_geometry ? 1 : 0, &M->L);
  if (!st) {
    std::vector<double> tab;
    cosmo_table(d->H0, d->Om0, d->zf, COSMO_TAB, &tab);
    double* pd;
    st = upload(ctx, &pd, tab.data(), tab.size(), &M->allocs, &M->bytes);
    dv.ctab = pd;
    dv.n_ctab = COSMO_TAB;
    dv.ctab_h = d->zf / COSMO_TAB;
    dv.ctab_inv_h = COSMO_TAB / d->zf;
  }

  // ---- photometry: App. D weights R lam dlam / Z_b, band-major samples
  if (!st && d->n_filt) {
    dv.n_filt = d->n_filt;
    std::vector<int> bs(d->n_filt + 1, 0);
    for (int b = 0; b < d->n_filt; b++) {
      if (d->filt_len[b] < 2) { st = fail(ctx, SED_EINVAL, "filter %d has < 2 samples", b); break; }
      bs[b + 1] = bs[b] + d->filt_len[b];
    }
    const int S = st ? 0 : bs[d->n_filt];
    std::vector<float> sl(S), sw(S), srz(S);
    double lmin = 1e300, lmax = 0;
    for (int b = 0; !st && b < d->n_filt; b++) {
      const double* L = d->filt_lam_aa + bs[b];
      const double* R = d->filt_trans + bs[b];
      const int n = d->filt_len[b];
      if (!strictly_increasing(L, n) || !(L[0] > 0)) { st = fail(ctx, SED_EINVAL, "filter %d wavelengths", b); break; }
      double zb = 0.0;
      for (int j = 0; j < n; j++)
        if (!std::isfinite(R[j]) || R[j] < 0) { st = fail(ctx, SED_EINVAL, "filter %d transmission", b); break; }
      for (int j = 0; j + 1 < n; j++) {
        const double g0 = L[j] * R[j] * C_AA * AB_FNU / (L[j] * L[j]);
        const double g1 = L[j + 1] * R[j + 1] * C_AA * AB_FNU / (L[j + 1] * L[j + 1]);
        zb += 0.5 * (g0 + g1) * (L[j + 1] - L[j]);
      }
      if (!st && !(zb > 0)) st = fail(ctx, SED_EINVAL, "filter %d has zero throughput", b);
      for (int j = 0; !st && j < n; j++) {
        const double dl = j == 0 ? 0.5 * (L[1] - L[0])
                                 : (j == n - 1 ? 0.5 * (L[n - 1] - L[n - 2]) : 0.5 * (L[j + 1] - L[j - 1]));
        sl[bs[b] + j] = (float)L[j];
        sw[bs[b] + j] = (float)(R[j] * L[j] * dl / zb);
        srz[bs[b] + j] = (float)(R[j] / zb);
        lmin = std::min(lmin, L[j]);
        lmax = std::max(lmax, L[j]);
      }
    }
    dv.n_samp = S;
    dv.samp_lam_min = (float)lmin;
    dv.samp_lam_max = (float)lmax;
    int* pi;
    double* pd;
    if (!st) { st = upload(ctx, &pi, bs.data(), bs.size(), &M->allocs, &M->bytes); dv.band_start = pi; }
    std::vector<float2> s2(S);
    for (int j = 0; j < S; j++) s2[j] = make_float2(sl[j], sw[j]);
    float2* p2;
    if (!st) { st = upload(ctx, &p2, s2.data(), s2.size(), &M->allocs, &M->bytes); dv.samp2 = p2; }
    if (!st && d->use_lines) {   // a line's photometry: R / Z_b at the samples
      float* pr;
      st = upload(ctx, &pr, srz.data(), srz.size(), &M->allocs, &M->bytes);
      dv.samp_rz = pr;
    }
    std::vector<double> zeros(d->n_filt, 0.0);
    if (!st) { st = upload(ctx, &pd, zeros.data(), zeros.size(), &M->allocs, &M->bytes); dv.phot_d = pd; }
    if (!st) { st = upload(ctx, &pd, zeros.data(), zeros.size(), &M->allocs, &M->bytes); dv.phot_isig = pd; }
    if (!st) { st = upload(ctx, &pd, zeros.data(), zeros.size(), &M->allocs, &M->bytes); dv.phot_nlog = pd; }
    std::vector<float> zf(d->n_filt, 0.f);
    float* pz;
    if (!st) { st = upload(ctx, &pz, zf.data(), zf.size(), &M->allocs, &M->bytes); dv.phot_dn = pz; }
    if (!st) { st = upload(ctx, &pz, zf.data(), zf.size(), &M->allocs, &M->bytes); dv.phot_isf = pz; }
    if (d->phot_mask) M->phot_mask_h.assign(d->phot_mask, d->phot_mask + d->n_filt);
    // upper-limit flags (Eq. app_line_chi2_UL): uploaded only when a band has one
    if (!st && d->phot_upper) {
      std::vector<uint8_t> ul(d->n_filt);
      bool any = false;
      for (int b = 0; b < d->n_filt; b++) any |= (ul[b] = d->phot_upper[b] ? 1 : 0) != 0;
      uint8_t* pu;
      if (any) { st = upload(ctx, &pu, ul.data(), ul.size(), &M->allocs, &M->bytes); dv.phot_ul = pu; }
    }
  }
  // ---- spectrum: per-pixel dispersion, Eq. app_sigeff + fixed sigma_gal (Eq. one_kernel);
  //      with a sampled sigma_gal the fixed part sigma_fix^2 / c^2 per pixel, the
  //      row's sigma_gal joining it in the kernels, and the widest reach bounded
  //      by sigma_gal_max
  dv.sample_sgal = d->sample_sigma_gal;
  dv.sgal_max_kms = (float)d->sigma_gal_max_kms;
  if (!st && d->n_pix) {
    const int np = d->n_pix;
    dv.n_pix = np;
    if (!strictly_increasing(d->spec_lam_aa, np) || !(d->spec_lam_aa[0] > 0))
      st = fail(ctx, SED_EINVAL, "spectrum wavelengths must be strictly increasing and > 0");
    std::vector<double> pl(np);
    std::vector<float> ps(np), pf2(np), psi(np), plc(np);
    double smax = 0;
    const double sg = d->sample_sigma_gal ? d->sigma_gal_max_kms : d->sigma_gal_kms;
    for (int i = 0; !st && i < np; i++) {
      const double lo_ = d->spec_lam_aa[i];
      if (!(d->lsf_value[i] > 0 && std::isfinite(d->lsf_value[i]))) { st = fail(ctx, SED_EINVAL, "lsf_value[%d] must be > 0", i); break; }
      const double si = sigma_inst_kms(d->lsf_mode, d->lsf_value[i], lo_);
      psi[i] = (float)si;
      plc[i] = (float)(lo_ / C_AA);
      const double lr = lo_ / (1.0 + d->z_ref);
      double slib;
      const auto& L = g->lam;
      if (lr <= L[0]) slib = g->siglib_kms[0];
      else if (lr >= L.back()) slib = g->siglib_kms.back();
      else {
        size_t k = std::upper_bound(L.begin(), L.end(), lr) - L.begin() - 1;
        slib = g->siglib_kms[k] + (g->siglib_kms[k + 1] - g->siglib_kms[k]) * (lr - L[k]) / (L[k + 1] - L[k]);
      }
      double fix2 = si * si - slib * slib;
      if (fix2 < 0) fix2 = 0;
      const double s = std::sqrt(fix2 + d->sigma_gal_kms * d->sigma_gal_kms) / C_KMS;
      pl[i] = std::log(lo_);
      ps[i] = (float)s;
      pf2[i] = (float)(fix2 / (C_KMS * C_KMS));
      smax = std::max(smax, std::sqrt(fix2 + sg * sg) / C_KMS);
    }
    dv.pix_ln_min = pl.empty() ? 0 : pl.front();
    dv.pix_ln_max = pl.empty() ? 0 : pl.back();
    dv.pix_s_max = (float)smax;
    double* pd;
    float* pf;
    std::vector<float2> pl2(np);
    for (int i = 0; i < np; i++) {
      pl2[i].x = (float)pl[i];
      pl2[i].y = (float)(pl[i] - (double)pl2[i].x);
    }
    if (!st) {
      float2* p2;
      st = upload(ctx, &p2, pl2.data(), pl2.size(), &M->allocs, &M->bytes);
      dv.pix_ln2 = p2;
    }
    if (!st) { st = upload(ctx, &pf, ps.data(), ps.size(), &M->allocs, &M->bytes); dv.pix_s = pf; }
    if (!st && d->sample_sigma_gal) {
      st = upload(ctx, &pf, pf2.data(), pf2.size(), &M->allocs, &M->bytes);
      dv.pix_fix2 = pf;
    }
    if (!st && d->use_lines) {   // the line profiles: instrumental dispersion and lambda / c per pixel
      st = upload(ctx, &pf, psi.data(), np, &M->allocs, &M->bytes);
      dv.pix_sinst = pf;
      if (!st) { st = upload(ctx, &pf, plc.data(), np, &M->allocs, &M->bytes); dv.pix_lamc = pf; }
    }
    // calibration polynomial: Chebyshev coordinate of each pixel, prior terms
    if (!st && d->calib_n > 0) {
      std::vector<float> cx(np);
      const double l0 = d->spec_lam_aa[0], l1 = d->spec_lam_aa[np - 1];
      for (int i = 0; i < np; i++) cx[i] = np > 1 ? (float)((2.0 * d->spec_lam_aa[i] - (l0 + l1)) / (l1 - l0)) : 0.f;
      st = upload(ctx, &pf, cx.data(), cx.size(), &M->allocs, &M->bytes);
      dv.pix_cx = pf;
      dv.calib_n = d->calib_n;
      dv.calib_opt = d->calib_mode == SED_CALIB_OPTIMISED ? 1 : 0;
      dv.calib_logdet_lam = 0.0;
      for (int m = 0; m < d->calib_n; m++) {
        dv.calib_isig2[m] = 1.0 / (d->calib_sigma[m] * d->calib_sigma[m]);
        dv.calib_logdet_lam += std::log(d->calib_sigma[m] * d->calib_sigma[m]);
      }
    }
    std::vector<double> zeros(np, 0.0);
    std::vector<float> zerof(np, 0.f);
    if (!st) { st = upload(ctx, &pf, zerof.data(), np, &M->allocs, &M->bytes); dv.spec_dn = pf; }
    if (!st) { st = upload(ctx, &pf, zerof.data(), np, &M->allocs, &M->bytes); dv.spec_isf = pf; }
    if (!st) { st = upload(ctx, &pd, zeros.data(), np, &M->allocs, &M->bytes); dv.spec_nlog = pd; }
    if (d->spec_mask) M->spec_mask_h.assign(d->spec_mask, d->spec_mask + np);
  }
  // ---- line catalogue (Sec. 3.3): blends, data in FP64, masked entries out of lnL
  if (!st && d->n_lcat > 0) {
    const int nk = d->n_lcat;
    std::vector<int> start(nk + 1, 0);
    for (int k = 0; k < nk; k++) start[k + 1] = start[k] + d->lcat_len[k];
    std::vector<int> lines(d->lcat_line, d->lcat_line + start[nk]);
    std::vector<double> ld(nk), li(nk), ln(nk);
    std::vector<uint8_t> ul(nk, 0);
    bool any_ul = false;
    for (int k = 0; k < nk; k++) {
      const bool inc = !d->lcat_mask || d->lcat_mask[k];
      ld[k] = d->lcat_d[k];
      li[k] = inc ? 1.0 / d->lcat_sigma[k] : 0.0;
      ln[k] = inc ? -0.5 * std::log(2.0 * M_PI * d->lcat_sigma[k] * d->lcat_sigma[k]) : 0.0;
      any_ul |= (ul[k] = d->lcat_upper && d->lcat_upper[k] ? 1 : 0) != 0;
    }
    int* pi;
    double* pd;
    st = upload(ctx, &pi, start.data(), start.size(), &M->allocs, &M->bytes);
    dv.lcat_start = pi;
    if (!st) { st = upload(ctx, &pi, lines.data(), lines.size(), &M->allocs, &M->bytes); dv.lcat_line = pi; }
    if (!st) { st = upload(ctx, &pd, ld.data(), nk, &M->allocs, &M->bytes); dv.lcat_d = pd; }
    if (!st) { st = upload(ctx, &pd, li.data(), nk, &M->allocs, &M->bytes); dv.lcat_isig = pd; }
    if (!st) { st = upload(ctx, &pd, ln.data(), nk, &M->allocs, &M->bytes); dv.lcat_nlog = pd; }
    if (!st && any_ul) {
      uint8_t* pu;
      st = upload(ctx, &pu, ul.data(), nk, &M->allocs, &M->bytes);
      dv.lcat_ul = pu;
    }
    dv.n_lcat = nk;
  }
  // widest rest-frame window a row can need: the observed span of the filter
  // samples and spectral pixels (5 dispersions out) is a fixed wavelength ratio
  // at every redshift; count the most nodes that ratio covers from any node,
  // plus the kernels' margins
  if (!st) {
    double lo = 1e300, hi = 0.0;
    if (dv.n_filt) { lo = std::min(lo, (double)dv.samp_lam_min); hi = std::max(hi, (double)dv.samp_lam_max); }
    if (dv.n_pix) {
      lo = std::min(lo, std::exp(dv.pix_ln_min - 5.0 * dv.pix_s_max));
      hi = std::max(hi, std::exp(dv.pix_ln_max + 5.0 * dv.pix_s_max));
    }
    const double ratio = hi / lo * (1.0 + 1e-6);
    const auto& Lg = g->lam;
    int wmax = 1;
    for (size_t k0 = 0; k0 < Lg.size(); k0++) {
      const size_t k1 = std::upper_bound(Lg.begin(), Lg.end(), Lg[k0] * ratio) - Lg.begin();
      wmax = std::max(wmax, (int)(k1 - k0));
    }
    dv.win_max = std::min(g->n_lam, wmax + 16);
  }
  if (!st && (d->phot_d || d->phot_sigma || d->spec_d || d->spec_sigma))
    st = set_data_dev(ctx, M, d->phot_d, d->phot_sigma, d->spec_d, d->spec_sigma);
  if (st) {
    free_all(ctx, M->allocs, M->bytes);
    delete M;
    return st;
  }
  ctx->models.push_back(M);
  *out = (sed_model_id)(ctx->models.size() - 1);
  return SED_OK;
}

static Model* find_model(const sed_ctx* ctx, sed_model_id id) {
  if (!ctx || id < 0 || id >= (int)ctx->models.size()) return nullptr;
  return ctx->models[id];
}

sed_status sed_model_layout(const sed_ctx* ctx, sed_model_id id, int* n_param, int* offsets) {
  Model* M = find_model(ctx, id);
  if (!M) return SED_EINVAL;
  if (n_param) *n_param = M->dv.n_param;
  if (offsets)
    for (int k = 0; k < SED_NKEYS; k++) offsets[k] = M->offs_caller[k];
  return SED_OK;
}

sed_status sed_set_data(sed_ctx* ctx, sed_model_id id, const double* pd, const double* ps, const double* sd,
                        const double* ss) {
  if (!ctx) return SED_EINVAL;
  std::lock_guard<std::mutex> lk(ctx->mu);
  DevGuard dg(ctx->device);
  Model* M = find_model(ctx, id);
  if (!M) return fail(ctx, SED_EINVAL, "unknown model id %d", id);
  if ((pd == nullptr) != (ps == nullptr) || (sd == nullptr) != (ss == nullptr))
    return fail(ctx, SED_EINVAL, "data and sigma must be given together");
  return set_data_dev(ctx, M, pd, ps, sd, ss);
}

sed_status sed_destroy_model(sed_ctx* ctx, sed_model_id id) {
  Model* M = find_model(ctx, id);
  if (!M) return fail(ctx, SED_EINVAL, "unknown model id %d", id);
  DevGuard dg(ctx->device);
  cudaDeviceSynchronize();
  free_all(ctx, M->allocs, M->bytes);
  delete M;
  ctx->models[id] = nullptr;
  return SED_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
namespace {

sed::Workspace* get_ws(sed_ctx* ctx, void* stream, int rows, int kpad, int ldn, bool grad, sed_status* st,
                       int nseg) {
  *st = SED_OK;
  std::lock_guard<std::mutex> lk(ctx->mu);
  Workspace*& w = ctx->ws[stream];
  if (!w) w = new Workspace();
  const bool need = rows > w->cap_rows || (size_t)kpad > w->cap_k || (size_t)ldn > w->cap_n || (grad && !w->dW) ||
                    nseg > w->cap_seg;
  if (!need) return w;
  // grow: free and reallocate everything (the stream's previous work must finish first)
  cudaStreamSynchronize((cudaStream_t)stream);
  std::vector<void*> old = {w->perm, w->tile_win, w->kmask, w->W, w->W_hi, w->W_lo, w->W_bf16, w->W_f8, w->Y, w->O, w->O2, w->rs, w->err,
                            w->wmask, w->theta_h, w->lnl_h, w->st_h, w->G_hi, w->G_lo, w->GO_hi, w->GO_lo,
                            w->dW, w->rgrad, w->qneb};
  for (void* p : old)
    if (p) cudaFree(p);
  budget_release(ctx, w->bytes);
  const bool had_grad = w->dW != nullptr;
  const int seg = std::max(nseg, w->cap_seg);
  if (w->host_exec) cudaGraphExecDestroy(w->host_exec);   // it holds the old buffers
  *w = Workspace();
  const int R = std::max(rows, 1);
  const size_t K = std::max<size_t>(kpad, 1), N = std::max<size_t>(ldn, 1);
  w->cap_rows = R;
  w->cap_k = K;
  w->cap_n = N;
  w->cap_seg = std::max(seg, 1);
  w->ldn = (int)N;
  std::vector<void*>* no = nullptr;
  sed_status s = SED_OK;
#define AL(ptr, nb) if (!s) s = dalloc(ctx, (void**)&w->ptr, nb, no, &w->bytes)
  AL(perm, R * 4); AL(tile_win, 2 * ((R + 127) / 128) * 4); AL(kmask, ((R + 127) / 128) * KMASK_WORDS * 4); AL(W, R * K * 4); AL(W_hi, R * K * 4); AL(W_lo, R * K * 4); AL(W_bf16, R * K * 2); AL(W_f8, R * (K + 128));
  AL(Y, R * N * 4 * w->cap_seg); AL(O, R * N * 4); AL(O2, R * N * 4); AL(wmask, R * KMASK_WORDS * 4); AL(rs, R * sizeof(RowScal)); AL(err, 64);
  AL(theta_h, R * 1024 * 4); AL(lnl_h, R * 8); AL(st_h, R * 4); AL(qneb, R * MAX_NEB_AGE * 4);
  if (grad || had_grad) {
    AL(G_hi, R * N * 4 * w->cap_seg); AL(G_lo, R * N * 4 * w->cap_seg); AL(GO_hi, R * N * 4); AL(GO_lo, R * N * 4);
    AL(dW, R * K * 4); AL(rgrad, R * RGRAD * 8);
  }
#undef AL
  if (!s) {   // the error words cleared, the per-tile windows empty (k_prep's self-ordered launches expect it)
    cudaError_t e = cudaMemset(w->err, 0, 64);
    const size_t mt = (R + 127) / 128;
    if (e == cudaSuccess) e = cudaMemset(w->tile_win, 0x7f, mt * sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(w->tile_win + mt, 0xff, mt * sizeof(int));
    if (e != cudaSuccess) s = fail(ctx, SED_ECUDA, "cudaMemset: %s", cudaGetErrorString(e));
  }
  *st = s;
  return s ? nullptr : w;
}

sed_status check_hot_args(sed_ctx* ctx, Model* M, const float* theta, int n, int ld, int precision) {
  if (!M) return fail(ctx, SED_EINVAL, "unknown model");
  if (n < 0) return fail(ctx, SED_EINVAL, "n < 0");
  if (n > 0 && !theta) return fail(ctx, SED_EINVAL, "theta is NULL");
  if (ld < M->dv.n_param) return fail(ctx, SED_EINVAL, "ld (%d) < n_param (%d)", ld, M->dv.n_param);
  if (precision != SED_PREC_FP32 && precision != SED_PREC_FP32_SIMT && precision != SED_PREC_BF16 &&
      precision != SED_PREC_FP8)
    return fail(ctx, SED_EINVAL, "unknown precision %d", precision);
  if (n > (1 << 22)) return fail(ctx, SED_ERANGE, "batch larger than 4M rows");
  if (!(M->g->avail & (1u << precision)))
    return fail(ctx, SED_EUNSUPPORTED, "precision %d: its copy of the grid was not kept (precision_mask)", precision);
  return SED_OK;
}

sed_status prof_mark(sed_ctx* ctx, Workspace* w, int i, cudaStream_t s) {
  if (!ctx->profiling) return SED_OK;
  if (!w->ev[i]) CK(cudaEventCreate(&w->ev[i]));
  CK(cudaEventRecord(w->ev[i], s));
  return SED_OK;
}

// prep + contraction into ws->Y / ws->O; theta_dev: theta is device memory
// (not a mapped host buffer), so the prep kernel may order the rows itself
sed_status run_forward_core(sed_ctx* ctx, Model* M, Workspace* w, const float* theta, int n, int ld,
                            int precision, cudaStream_t s, bool theta_dev = true) {
  Grid* g = M->g;
  Layout* L = M->L;
  if (ctx->profiling) {
    w->last_n = n; w->last_prec = precision; w->last_nlam = g->n_lam;
    w->last_kpad = precision == SED_PREC_FP8 ? L->Ky_pad8 == 0 ? L->Kpad : L->Kpad8 : L->Kpad;
    w->have_stats = true;
    w->last_grad = false;
  }
  if (sed_status ps = prof_mark(ctx, w, 0, s)) return ps;
  PrepArgs pa{};
  pa.theta = theta; pa.n = n; pa.ld = ld;
  pa.md = M->dv; pa.g = g->dv; pa.L = L->dv();
  pa.W = precision == SED_PREC_FP32_SIMT ? w->W : nullptr;   // only the CUDA-core contraction reads FP32 W
  pa.W_hi = precision == SED_PREC_FP32 ? w->W_hi : nullptr;
  pa.W_lo = precision == SED_PREC_FP32 ? w->W_lo : nullptr;
  pa.W_bf16 = precision == SED_PREC_BF16 ? w->W_bf16 : nullptr;
  pa.W_f8 = precision == SED_PREC_FP8 ? w->W_f8 : nullptr;
  if (precision == SED_PREC_FP8) {
    sed_status fs;
    {
      std::lock_guard<std::mutex> lk(ctx->mu);
      fs = ensure_f8_layout(ctx, g, L);
    }
    if (fs) return fs;
    pa.L = L->dv();
  }
  pa.rs = w->rs;
  pa.err = w->err;
  pa.perm = w->perm;
  pa.qneb = M->dv.use_neb && g->neb_na > 0 ? w->qneb : nullptr;
  pa.tile_win = w->tile_win;
  pa.self_order = theta_dev ? 1 : 0;
  // K-tile masks for the tensor-core contractions (32 / 64 / 128 columns per tile)
  {
    const int shift = precision == SED_PREC_FP8 ? 7 : (precision == SED_PREC_BF16 ? 6 : 5);
    const int kp = precision == SED_PREC_FP8 ? L->Kpad8 : L->Kpad;
    const int kw = ((kp >> shift) + 31) / 32;
    // skipping pays where the rows' weights sit in few (a/Fe, Fe/H) blocks
    // (one constant [Fe/H] per row) and the K tiles are narrowest (3xTF32):
    // measured, the wider BF16 / FP8 tiles lose more to the looser redshift
    // windows of the bracket-pair row order than they save
    const int pairs = std::max(g->n_feh - 1, 1) * (M->dv.use_afe ? std::max(g->n_afe - 1, 1) : 1);
    const bool use = precision == SED_PREC_FP32 && M->dv.zmode == 1 && pairs > 1 && kw <= KMASK_WORDS;
    pa.kmask = use ? w->kmask : nullptr;
    pa.kmask_w = use ? kw : 0;
    // the masked 3xTF32 fit writes only its rows' touched K tiles of W (and
    // zeros where the row at the same position had non-zeros); other writes of
    // W_hi/W_lo are dense and leave the tracked tiles unknown
    pa.wmask = nullptr;
    if (use && pa.W_hi) {
      if (w->wmask_kpad != L->Kpad) {
        CK(cudaMemsetAsync(w->wmask, 0xff, (size_t)w->cap_rows * KMASK_WORDS * sizeof(uint32_t), s));
        w->wmask_kpad = L->Kpad;
      }
      pa.wmask = w->wmask;
    } else if (pa.W_hi) {
      w->wmask_kpad = 0;
    }
    pa.kt_shift = shift;
    w->kmask_w_call = pa.kmask_w;
    if (ctx->profiling) { w->last_kmask_w = pa.kmask_w; w->last_kt_shift = shift; }
  }
  CK(launch_prep(pa, s));
  if (sed_status ps = prof_mark(ctx, w, 1, s)) return ps;
  if (precision == SED_PREC_FP32_SIMT) {
    ContractArgs ca{};
    ca.n = n; ca.n_lam = g->n_lam; ca.ldn = w->ldn; ca.Ky_pad = L->Ky_pad; ca.Kpad = L->Kpad;
    ca.W = w->W; ca.sspT = L->sspT_f32; ca.Y = w->Y; ca.O = w->O; ca.rs = w->rs;
    ca.n_seg = L->n_seg; ca.seg_stride = (size_t)w->cap_rows * w->ldn;
    for (int sg = 0; sg <= MAX_SEG; ++sg) ca.seg_k0[sg] = L->seg_k0[sg];
    CK(launch_contract_simt(ca, s));
    return prof_mark(ctx, w, 2, s);
  }
  if (ctx->tc_ok != 1)
    return fail(ctx, SED_EUNSUPPORTED, "tensor-core precisions need an sm_103 device and cuTensorMapEncodeTiled");
  const bool f32 = precision == SED_PREC_FP32, f8 = precision == SED_PREC_FP8;
  TcMaps* maps = &w->maps;
  const void* key = f32 ? (const void*)L->sspT_hi : (f8 ? (const void*)L->sspT_f8 : (const void*)L->sspT_bf16);
  const void* a_op = f32 ? (const void*)w->W_hi : (f8 ? (const void*)w->W_f8 : (const void*)w->W_bf16);
  if (!w->tmap_valid || w->tmap_for != key || w->tmap_n != n || w->tmap_prec != precision || w->tmap_a != a_op) {
    int e = tc_encode_maps(ctx->encode_fn, maps, precision, a_op, w->W_lo, key, L->sspT_lo, n, g->n_lam,
                           f8 ? L->Kpad8 : L->Kpad);
    if (e) return fail(ctx, SED_ECUDA, "cuTensorMapEncodeTiled failed (operand %d)", e);
    w->tmap_valid = true;
    w->tmap_for = key;
    w->tmap_n = n;
    w->tmap_prec = precision;
    w->tmap_a = a_op;
  }
  TcArgs ta{};
  ta.n = n; ta.n_lam = g->n_lam; ta.ldn = w->ldn; ta.prec = precision;
  ta.Ky_pad = f8 ? L->Ky_pad8 : L->Ky_pad;
  ta.Kpad = f8 ? L->Kpad8 : L->Kpad;
  ta.maps = maps; ta.Y = w->Y; ta.O = w->O; ta.err = w->err; ta.rs = w->rs;
  ta.O2 = w->O2; ta.split_out = w->err + 8;   // err[8]: the launch records whether it split its tiles
  ta.tile_win = w->tile_win;
  ta.kmask = pa.kmask; ta.kmask_w = pa.kmask_w;
  ta.n_seg = L->n_seg; ta.seg_stride = (size_t)w->cap_rows * w->ldn;
  for (int sg = 0; sg <= MAX_SEG; ++sg) ta.seg_k0[sg] = L->seg_k0[sg];
  CK(launch_contract_tc(ta, s));
  return prof_mark(ctx, w, 2, s);
}

int ldn_for(const Grid* g) { return (g->n_lam + 255) / 256 * 256; }

}  // namespace

extern "C" {

sed_status sed_forward(sed_ctx* ctx, sed_model_id id, const float* theta, int n, int ld, float* phot_out,
                       float* spec_out, int precision, void* stream) {
  if (!ctx) return SED_EINVAL;
  Model* M = find_model(ctx, id);
  sed_status st = check_hot_args(ctx, M, theta, n, ld, precision);
  if (st) return st;
  if (n == 0) return SED_OK;
  DevGuard dg(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  Workspace* w = get_ws(ctx, stream, n, M->L->Kpad, ldn_for(M->g), false, &st, M->L->n_seg);
  if (!w) return st;
  st = run_forward_core(ctx, M, w, theta, n, ld, precision, s);
  if (st) return st;
  EpiArgs ea{};
  ea.n = n; ea.ldn = w->ldn; ea.Y = w->Y; ea.O = w->O; ea.rs = w->rs;
  ea.O2 = w->O2; ea.split = precision == SED_PREC_FP32 ? w->err + 8 : nullptr;   // the 3xTF32 launch's split choice
  ea.md = M->dv; ea.g = M->g->dv;
  ea.seg_stride = (size_t)w->cap_rows * w->ldn;
  ea.qneb = M->dv.use_neb && M->g->neb_na > 0 ? w->qneb : nullptr;
  ea.win_reset = w->tile_win; ea.win_mt = (n + 127) / 128;   // read by the contraction, emptied for the next call
  ea.lam8 = precision == SED_PREC_FP8 ? M->L->lam8 : nullptr;
  ea.phot_out = M->dv.n_filt ? phot_out : nullptr;
  ea.spec_out = M->dv.n_pix ? spec_out : nullptr;
  ea.lnl = nullptr; ea.status = nullptr; ea.err = w->err;
  CK(launch_epilogue(ea, s));
  return prof_mark(ctx, w, 3, s);
}

sed_status sed_line_fluxes(sed_ctx* ctx, sed_model_id id, const float* theta, int n, int ld, float* flux_out,
                           int precision, void* stream) {
  if (!ctx) return SED_EINVAL;
  Model* M = find_model(ctx, id);
  sed_status st = check_hot_args(ctx, M, theta, n, ld, precision);
  if (st) return st;
  if (!M->dv.use_lines) return fail(ctx, SED_EUNSUPPORTED, "the model has no emission lines");
  if (n > 0 && !flux_out) return fail(ctx, SED_EINVAL, "flux_out is NULL");
  if (n == 0) return SED_OK;
  DevGuard dg(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  Workspace* w = get_ws(ctx, stream, n, M->L->Kpad, ldn_for(M->g), false, &st, M->L->n_seg);
  if (!w) return st;
  st = run_forward_core(ctx, M, w, theta, n, ld, precision, s);
  if (st) return st;
  EpiArgs ea{};
  ea.n = n; ea.ldn = w->ldn; ea.Y = w->Y; ea.O = w->O; ea.rs = w->rs;
  ea.O2 = w->O2; ea.split = precision == SED_PREC_FP32 ? w->err + 8 : nullptr;   // the 3xTF32 launch's split choice
  ea.md = M->dv; ea.g = M->g->dv;
  ea.seg_stride = (size_t)w->cap_rows * w->ldn;
  ea.qneb = M->dv.use_neb && M->g->neb_na > 0 ? w->qneb : nullptr;
  ea.win_reset = w->tile_win; ea.win_mt = (n + 127) / 128;   // read by the contraction, emptied for the next call
  ea.lam8 = precision == SED_PREC_FP8 ? M->L->lam8 : nullptr;
  ea.lines_out = flux_out;
  ea.err = w->err;
  CK(launch_epilogue(ea, s));
  return prof_mark(ctx, w, 3, s);
}

// sed_loglike; theta_dev false for a mapped host theta (sed_loglike_host)
static sed_status loglike_impl(sed_ctx* ctx, sed_model_id id, const float* theta, int n, int ld, double* lnl_out,
                               uint32_t* row_status, int precision, void* stream, bool theta_dev) {
  if (!ctx) return SED_EINVAL;
  Model* M = find_model(ctx, id);
  sed_status st = check_hot_args(ctx, M, theta, n, ld, precision);
  if (st) return st;
  if (n > 0 && !lnl_out) return fail(ctx, SED_EINVAL, "lnl_out is NULL");
  if (n == 0) return SED_OK;
  DevGuard dg(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  Workspace* w = get_ws(ctx, stream, n, M->L->Kpad, ldn_for(M->g), false, &st, M->L->n_seg);
  if (!w) return st;
  st = run_forward_core(ctx, M, w, theta, n, ld, precision, s, theta_dev);
  if (st) return st;
  EpiArgs ea{};
  ea.n = n; ea.ldn = w->ldn; ea.Y = w->Y; ea.O = w->O; ea.rs = w->rs;
  ea.O2 = w->O2; ea.split = precision == SED_PREC_FP32 ? w->err + 8 : nullptr;   // the 3xTF32 launch's split choice
  ea.md = M->dv; ea.g = M->g->dv;
  ea.seg_stride = (size_t)w->cap_rows * w->ldn;
  ea.qneb = M->dv.use_neb && M->g->neb_na > 0 ? w->qneb : nullptr;
  ea.win_reset = w->tile_win; ea.win_mt = (n + 127) / 128;   // read by the contraction, emptied for the next call
  ea.lnl = lnl_out; ea.status = row_status; ea.err = w->err;
  ea.lam8 = precision == SED_PREC_FP8 ? M->L->lam8 : nullptr;
  CK(launch_epilogue(ea, s));
  return prof_mark(ctx, w, 3, s);
}

sed_status sed_loglike(sed_ctx* ctx, sed_model_id id, const float* theta, int n, int ld, double* lnl_out,
                       uint32_t* row_status, int precision, void* stream) {
  return loglike_impl(ctx, id, theta, n, ld, lnl_out, row_status, precision, stream, true);
}

sed_status sed_loglike_host(sed_ctx* ctx, sed_model_id id, const float* theta, int n, int ld, double* lnl_out,
                            uint32_t* row_status, int precision, void* stream) {
  if (!ctx) return SED_EINVAL;
  Model* M = find_model(ctx, id);
  sed_status st = check_hot_args(ctx, M, theta, n, ld, precision);
  if (st) return st;
  if (n > 0 && !lnl_out) return fail(ctx, SED_EINVAL, "lnl_out is NULL");
  if (ld > 1024) return fail(ctx, SED_ERANGE, "host path supports ld <= 1024");
  if (n == 0) return SED_OK;
  DevGuard dg(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  Workspace* w = get_ws(ctx, stream, n, M->L->Kpad, ldn_for(M->g), false, &st, M->L->n_seg);
  if (!w) return st;
  // page-locked, device-mapped host buffers are used in place: the kernels
  // read theta and write lnL / status over the host link (NVLink-C2C on a
  // Grace host), so no copy sits on the critical path; other buffers are
  // staged through device memory
  const float* th_d = (const float*)mapped_host(theta);
  double* lnl_d = (double*)mapped_host(lnl_out);
  uint32_t* st_d = row_status ? (uint32_t*)mapped_host(row_status) : nullptr;
  // all buffers in place, on a caller's stream (capture is not possible on the
  // legacy default stream), not profiling: the second identical call captures
  // its launches into a CUDA graph, later ones replay it (one launch instead of
  // two memsets and four kernels)
  if (th_d && lnl_d && (!row_status || st_d) && stream && !ctx->profiling) {
    Workspace::HostKey k;
    k.model = id; k.mp = M; k.th = th_d; k.lnl = lnl_d; k.st = st_d; k.n = n; k.ld = ld; k.prec = precision;
    if (!(w->host_exec && w->host_key == k)) {
      if (w->host_seen == k) {
        if (w->host_exec) {
          cudaGraphExecDestroy(w->host_exec);
          w->host_exec = nullptr;
        }
        cudaGraph_t gr = nullptr;
        sed_status cs = SED_OK;
        cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
          cs = loglike_impl(ctx, id, th_d, n, ld, lnl_d, st_d, precision, stream, false);
          e = cudaStreamEndCapture(s, &gr);
        }
        if (e == cudaSuccess && cs == SED_OK && gr) e = cudaGraphInstantiate(&w->host_exec, gr, 0);
        if (gr) cudaGraphDestroy(gr);
        if (e != cudaSuccess || cs != SED_OK) {
          cudaGetLastError();   // no graph: the direct launches below serve this key
          if (w->host_exec) cudaGraphExecDestroy(w->host_exec);
          w->host_exec = nullptr;
          w->host_seen = Workspace::HostKey();
        } else {
          w->host_key = k;
        }
      } else {
        w->host_seen = k;
      }
    }
    if (w->host_exec && w->host_key == k) {
      CK(cudaGraphLaunch(w->host_exec, s));
      CK(cudaStreamSynchronize(s));
      ctx->last_host_mapped = 1 | 2 | 4;
      return SED_OK;
    }
  }
  if (!th_d) {
    CK(cudaMemcpyAsync(w->theta_h, theta, (size_t)n * ld * 4, cudaMemcpyHostToDevice, s));
    th_d = w->theta_h;
  }
  st = loglike_impl(ctx, id, th_d, n, ld, lnl_d ? lnl_d : w->lnl_h, row_status && !st_d ? w->st_h : st_d,
                    precision, stream, th_d == w->theta_h);
  if (st) return st;
  if (!lnl_d) CK(cudaMemcpyAsync(lnl_out, w->lnl_h, (size_t)n * 8, cudaMemcpyDeviceToHost, s));
  if (row_status && !st_d) CK(cudaMemcpyAsync(row_status, w->st_h, (size_t)n * 4, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  ctx->last_host_mapped = (th_d != w->theta_h ? 1 : 0) | (lnl_d ? 2 : 0);
  return SED_OK;
}

sed_status sed_loglike_grad(sed_ctx* ctx, sed_model_id id, const float* theta, int n, int ld, double* lnl_out,
                            float* grad_out, uint32_t* row_status, int precision, void* stream) {
  if (!ctx) return SED_EINVAL;
  Model* M = find_model(ctx, id);
  sed_status st = check_hot_args(ctx, M, theta, n, ld, precision);
  if (st) return st;
  if (precision == SED_PREC_BF16 || precision == SED_PREC_FP8)
    return fail(ctx, SED_EUNSUPPORTED, "the gradient is available for SED_PREC_FP32 and SED_PREC_FP32_SIMT");
  if (n > 0 && (!lnl_out || !grad_out)) return fail(ctx, SED_EINVAL, "lnl_out or grad_out is NULL");
  if (n == 0) return SED_OK;
  DevGuard dg(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  Grid* g = M->g;
  Layout* L = M->L;
  const int ldn = ldn_for(g);
  {
    std::lock_guard<std::mutex> lk(ctx->mu);
    st = ensure_grad_layout(ctx, g, L, ldn);
  }
  if (st) return st;
  Workspace* w = get_ws(ctx, stream, n, L->Kpad, ldn, true, &st, L->n_seg);
  if (!w) return st;
  st = run_forward_core(ctx, M, w, theta, n, ld, precision, s);
  if (st) return st;
  if (ctx->profiling) w->last_grad = true;
  const bool f32 = precision == SED_PREC_FP32;
  EpiBwdArgs eb{};
  eb.n = n; eb.ldn = w->ldn; eb.Y = w->Y; eb.O = w->O; eb.rs = w->rs;
  eb.O2 = w->O2; eb.o2_split = precision == SED_PREC_FP32 ? w->err + 8 : nullptr;
  eb.md = M->dv; eb.g = g->dv; eb.split = f32 ? 1 : 0;
  eb.gy_hi = w->G_hi; eb.gy_lo = w->G_lo; eb.go_hi = w->GO_hi; eb.go_lo = w->GO_lo;
  eb.rgrad = w->rgrad; eb.lnl = lnl_out; eb.status = row_status; eb.err = w->err;
  eb.seg_stride = (size_t)w->cap_rows * w->ldn;
  eb.qneb = M->dv.use_neb && g->neb_na > 0 ? w->qneb : nullptr;
  eb.win_reset = w->tile_win; eb.win_mt = (n + 127) / 128;   // read by the contraction, emptied for the next call
  size_t smem = 0;
  cudaError_t e = launch_epilogue_bwd(eb, &smem, s);
  if (e == cudaErrorInvalidConfiguration)
    return fail(ctx, SED_ERANGE, "adjoint epilogue needs %zu bytes of dynamic shared memory (227 KB per CTA in all)", smem);
  CK(e);
  if (sed_status ps = prof_mark(ctx, w, 4, s)) return ps;
  if (f32) {
    if (!w->dw_maps_valid || w->dw_maps_for != (const void*)L || w->dw_maps_n != n || w->dw_maps_g != w->G_hi) {
      // dlnL/dY of the attenuated blocks: slab s at rows s cap_rows + m of one map
      const int n_gy = (L->n_seg - 1) * w->cap_rows + n;
      int ee = tc_encode_dw_maps(ctx->encode_fn, &w->dw_maps, w->G_hi, w->G_lo, w->GO_hi, w->GO_lo, L->sspK_hi,
                                 L->sspK_lo, n, n_gy, w->ldn, L->ldn, L->Kpad);
      if (ee) return fail(ctx, SED_ECUDA, "cuTensorMapEncodeTiled failed (adjoint operand %d)", ee);
      w->dw_maps_valid = true;
      w->dw_maps_for = L;
      w->dw_maps_n = n;
      w->dw_maps_g = w->G_hi;
    }
    DwArgs da{};
    da.n = n; da.ldk = L->ldn; da.Ky_pad = L->Ky_pad; da.Kpad = L->Kpad;
    da.maps = &w->dw_maps; da.dW = w->dW; da.err = w->err; da.rs = w->rs;
    // the forward's K-tile masks (3xTF32: 32-column tiles), when it had any,
    // select dW's output tiles
    da.kmask = w->kmask_w_call > 0 ? w->kmask : nullptr;
    da.kmask_w = w->kmask_w_call;
    da.n_seg = L->n_seg; da.seg_rows = w->cap_rows;
    for (int sg = 0; sg <= MAX_SEG; ++sg) da.seg_k0[sg] = L->seg_k0[sg];
    CK(launch_dw_tc(da, s));
  } else {
    DwSimtArgs da{};
    da.n = n; da.ldg = w->ldn; da.ldk = L->ldn; da.Ky_pad = L->Ky_pad; da.Kpad = L->Kpad;
    da.gy = w->G_hi; da.go = w->GO_hi; da.sspK = L->sspK_f32; da.dW = w->dW; da.rs = w->rs;
    da.n_seg = L->n_seg; da.seg_stride = (size_t)w->cap_rows * w->ldn;
    for (int sg = 0; sg <= MAX_SEG; ++sg) da.seg_k0[sg] = L->seg_k0[sg];
    CK(launch_dw_simt(da, s));
  }
  if (sed_status ps = prof_mark(ctx, w, 5, s)) return ps;
  PrepBwdArgs pb{};
  pb.theta = theta; pb.n = n; pb.ld = ld;
  pb.md = M->dv; pb.g = g->dv; pb.L = L->dv();
  pb.rs = w->rs; pb.dW = w->dW; pb.rgrad = w->rgrad; pb.grad = grad_out;
  CK(launch_prep_bwd(pb, s));
  return prof_mark(ctx, w, 3, s);
}

sed_status sed_set_profiling(sed_ctx* ctx, int on) {
  if (!ctx) return SED_EINVAL;
  ctx->profiling = on ? 1 : 0;
  return SED_OK;
}

sed_status sed_last_stats(sed_ctx* ctx, void* stream, sed_stage_stats* out) {
  if (!ctx || !out) return fail(ctx, SED_EINVAL, "null argument");
  Workspace* w = nullptr;
  {
    std::lock_guard<std::mutex> lk(ctx->mu);
    auto it = ctx->ws.find(stream);
    if (it != ctx->ws.end()) w = it->second;
  }
  if (!w || !w->have_stats || !w->ev[3]) return fail(ctx, SED_EINVAL, "no profiled call on this stream");
  DevGuard dg(ctx->device);
  CK(cudaEventSynchronize(w->ev[3]));
  memset(out, 0, sizeof *out);
  CK(cudaEventElapsedTime(&out->ms_prep, w->ev[0], w->ev[1]));
  CK(cudaEventElapsedTime(&out->ms_contract, w->ev[1], w->ev[2]));
  if (w->last_grad) {
    CK(cudaEventElapsedTime(&out->ms_epilogue, w->ev[2], w->ev[4]));
    CK(cudaEventElapsedTime(&out->ms_dw, w->ev[4], w->ev[5]));
    CK(cudaEventElapsedTime(&out->ms_prep_bwd, w->ev[5], w->ev[3]));
    out->is_grad = 1;
  } else {
    CK(cudaEventElapsedTime(&out->ms_epilogue, w->ev[2], w->ev[3]));
  }
  std::vector<RowScal> rs(w->last_n);
  CK(cudaMemcpy(rs.data(), w->rs, rs.size() * sizeof(RowScal), cudaMemcpyDeviceToHost));
  double nnz = 0;
  for (const RowScal& r : rs) nnz += r.nnz;
  out->nnz_w = nnz;
  out->dense_k = w->last_kpad;
  // tensor work actually issued
  {
    const bool simt = w->last_prec == SED_PREC_FP32_SIMT;
    const int bn = simt ? 128 : tc_bn_for(w->last_prec, w->last_kpad);
    // K columns each 128-row tile multiplies: its touched K tiles when the call skipped the others
    std::vector<double> kcols((rs.size() + 127) / 128, (double)w->last_kpad);
    if (w->last_kmask_w > 0 && !simt) {
      std::vector<uint32_t> km(kcols.size() * w->last_kmask_w);
      CK(cudaMemcpy(km.data(), w->kmask, km.size() * 4, cudaMemcpyDeviceToHost));
      for (size_t t = 0; t < kcols.size(); ++t) {
        int bits = 0;
        for (int j = 0; j < w->last_kmask_w; ++j) bits += __builtin_popcount(km[t * w->last_kmask_w + j]);
        kcols[t] = (double)bits * (1 << w->last_kt_shift);
      }
    }
    // wavelength tiles of each 128-row tile's window union x its K columns; the
    // persistent tensor-core schedule starts a tile's run at the window's first
    // node rounded down to 16 columns, the grid schedules at a whole tile
    const bool unaligned = !simt && kcols.size() <= (size_t)tc_max_m_tiles();
    double issued = 0;
    for (size_t m0 = 0; m0 < rs.size(); m0 += 128) {
      int lo = 0x7fffffff, hi = -1;
      for (size_t r = m0; r < std::min(rs.size(), m0 + 128); ++r)
        if (rs[r].status == 0) { lo = std::min(lo, rs[r].k_lo); hi = std::max(hi, rs[r].k_hi); }
      if (hi < 0) continue;
      const int tiles = unaligned ? (std::min(hi, w->ldn - 1) - (lo & ~15)) / bn + 1 : hi / bn - lo / bn + 1;
      issued += tiles * kcols[m0 / 128];
    }
    out->issued_flop = issued * 2.0 * 128.0 * bn * (w->last_prec == SED_PREC_FP32 ? 3.0 : 1.0);
  }
  out->n_rows = w->last_n;
  out->n_lam = w->last_nlam;
  out->ldn = w->ldn;
  out->precision = w->last_prec;
  return SED_OK;
}

}  // extern "C"
