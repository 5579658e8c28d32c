// Per-row preparation: cosmology, SFH edges, SSP weights, Q_young and the
// per-row scalars of the epilogue.  One CTA per parameter row.
//
//  - cosmology (Sec. 2.6): comoving distance and age of the Universe from a
//    per-model FP64 table (cubic Hermite), luminosity distance floored at 10 pc;
//  - SFH edges 0, 5 Myr, 10 Myr, then log-uniform to T_max = t(z) - t(zf),
//    so the grid follows the sampled redshift and the bin masses are kept
//    (Sec. 2.2, Sec. 2.6);
//  - step-scheme weights (App. B): each age node owns its linear-time Voronoi
//    cell, A_ia = m_i |bin_i ∩ cell_a| / dT_i; each bin's mass is split between
//    the two bracketing [Fe/H] nodes linearly in log Z (App. B), and over the
//    two bracketing [a/Fe] nodes (Sec. 5.4).  A thread owns one age node and
//    sums the bins overlapping its cell in order, so W is deterministic;
//  - Q_young = sum over birth-cloud ages of W Q (App. C, Eq. app_q).
#include <algorithm>

#include "sed_internal.cuh"
#include "locate.cuh"

namespace sed {

__device__ __forceinline__ float tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// clamped linear bracket on a small node array in registers/param space
__device__ __forceinline__ void bracket_f(const float* x, int n, float v, int& j0, float& w0,
                                          int& j1, float& w1) {
  if (n == 1) { j0 = j1 = 0; w0 = 1.f; w1 = 0.f; return; }
  if (v <= x[0]) { j0 = 0; j1 = 1; w0 = 1.f; w1 = 0.f; return; }
  if (v >= x[n - 1]) { j0 = n - 2; j1 = n - 1; w0 = 0.f; w1 = 1.f; return; }
  int j = 0;
  while (j + 2 < n && !(v < x[j + 1])) j++;
  float t = (v - x[j]) / (x[j + 1] - x[j]);
  j0 = j; j1 = j + 1; w0 = 1.f - t; w1 = t;
}

// derivatives of the two bracket weights with respect to v (0 when clamped)
__device__ __forceinline__ void bracket_df(const float* x, int n, float v, int j0, int j1, float& d0, float& d1) {
  d0 = d1 = 0.f;
  if (n > 1 && v > x[0] && v < x[n - 1]) {
    const float h = x[j1] - x[j0];
    d0 = -1.f / h;
    d1 = 1.f / h;
  }
}

// SFH edges of one row (FP32): 0, 5 Myr, 10 Myr, then log-uniform to T_max.
__device__ __forceinline__ float sfh_edge(int i, int NT, double tmax, float lrat) {
  if (i == 0) return 0.f;
  if (i == 1) return 5e6f;
  if (i == 2) return 1e7f;
  if (i == NT) return (float)tmax;
  return 1e7f * expf(lrat * (float)(i - 2) / (float)(NT - 2));
}

// Cosmology and observer-frame scalars of one row (Sec. 2.6).  D_C(z),
// t_univ(z), ln(1+z) and 1/(1+z) are cubic Hermite interpolants (FP64) of a
// table the host fills once per model with FP64 values and their exact
// derivatives (c/H0/E, -1/(H0 (1+z) E), 1/(1+z), -1/(1+z)^2); the
// interpolation error is below 1e-10 relative.  GB300's FP64 pipe is narrow
// (a warp instruction every 16 SM cycles, whatever the active lanes), so FP64
// is kept to the interpolation, T_max, ln(1+z) (hi + lo floats for the
// spectral positions) and a five-term product for the flux scale; 1/D_L, the
// power of ten and the derivative factors used only by the adjoint are FP32.
//  D_L = (1+z) D_C, floored at 10 pc;  T_max = t(z) - t(zf);
//  s = 10^logmass Lsun (1+z) / (4 pi D_L^2) in device flux units, with
//  10^logmass = 2^n 2^f from an exact FP32 split of logmass log2(10) and an
//  FP32 exp2 of the fraction (FP32-grade).
// App. B linear scheme (Eq. tent_integral).  Across an SFH bin [T0, T1] the
// SFR is psi(t) = psi0 + g (t - T0); the piece [x0, x1] of the bin between age
// nodes t_j < t_{j+1} (dl = ln(t_{j+1}/t_j)) gives node j+1 the share
// int psi(t) ln(t/t_j) dt / dl of its mass M and node j the rest, each
// clipped at 0.  With t = x0 (1 + u), r = (x1 - x0)/x0,
//   int psi ln(t/t_j) dt = ln(x0/t_j) M + x0 [psi(x0) F1(r) + g x0 F2(r)],
//   F1 = (1 + r) log1p(r) - r,   F2 = (r^2 - 1) log1p(r)/2 - r^2/4 + r/2,
// all in FP32: F1 and F2 are formed from quantities of the size of r, so the
// rounding of a share stays relative to M.
__device__ __forceinline__ float lin_mass(float x0, float x1, float psi0, float g, float T0) {
  return 0.5f * (fmaf(g, x0 - T0, psi0) + fmaf(g, x1 - T0, psi0)) * (x1 - x0);
}
// unclipped shares (linear in psi0 and g)
__device__ __forceinline__ void tent_piece_raw(float x0, float x1, float tj, float dl, float psi0, float g, float T0,
                                               float& lo, float& hi) {
  const float p0 = fmaf(g, x0 - T0, psi0);
  const float M = lin_mass(x0, x1, psi0, g, T0);
  const float r = (x1 - x0) / x0, L = log1pf(r);
  const float F1 = fmaf(1.f + r, L, -r);
  const float F2 = fmaf(0.5f * (r * r - 1.f), L, r * (0.5f - 0.25f * r));
  const float lx = x0 > tj ? logf(x0 / tj) : 0.f;
  hi = fmaf(lx, M, x0 * fmaf(p0, F1, g * x0 * F2)) / dl;
  lo = M - hi;
}
__device__ __forceinline__ void tent_piece(float x0, float x1, float tj, float dl, float psi0, float g, float T0,
                                           float& lo, float& hi) {
  tent_piece_raw(x0, x1, tj, dl, psi0, g, T0, lo, hi);
  lo = fmaxf(lo, 0.f);
  hi = fmaxf(hi, 0.f);
}

// Reverse pass of the linear scheme for bin [T0, T1] with edge rates psi0,
// psi1: the bin's masses per node are W_a = sc S_a, S_a the clipped shares and
// sc = target / sum_a S_a.  Given G_a = dlnL/dW_a (from the node's gradient
// row split by the bin's [Fe/H], gsel), returns dlnL/d{psi0, psi1, T0, T1} and
// dlnL/dzeta of the bin.  A share depends on the rates linearly (unit-rate
// shares), on an edge through the integral's limit (-+psi tau at the edge) and
// through psi(t) = psi0 + (psi1 - psi0)(t - T0)/(T1 - T0) (the shares of the
// linear functions dpsi/dT0, dpsi/dT1); a clipped share carries no derivative.
struct LinGrad {
  float p0, p1, t0, t1, zeta;
};
template <typename GFn>
__device__ LinGrad lin_bin_grad(const GridDev& g, float T0, float T1, float psi0, float psi1, GFn gsel) {
  const int NA = g.n_age;
  const float D = T1 - T0, gr = (psi1 - psi0) / D;
  const float t_first = g.age_t[0], t_last = g.age_t[NA - 1];
  // accumulators: sum S, its derivatives, and the same weighted by G
  float S = 0.f, SP0 = 0.f, SP1 = 0.f, ST0 = 0.f, ST1 = 0.f;
  float GS = 0.f, GP0 = 0.f, GP1 = 0.f, GT0 = 0.f, GT1 = 0.f, GZ = 0.f;
  const float hT0_0 = -gr, hT0_g = gr / D;      // dpsi/dT0 = (psi1-psi0)(t - T1)/D^2: value at T0, slope
  const float hT1_g = -gr / D;                  // dpsi/dT1 = -(psi1-psi0)(t - T0)/D^2: 0 at T0
  auto add = [&](int a, float s, float dp0, float dp1, float dt0, float dt1) {
    if (!(s > 0.f)) return;   // clipped: no mass, no derivative
    float G, Gz;
    gsel(a, G, Gz);
    S += s; SP0 += dp0; SP1 += dp1; ST0 += dt0; ST1 += dt1;
    GS += G * s; GP0 += G * dp0; GP1 += G * dp1; GT0 += G * dt0; GT1 += G * dt1; GZ += Gz * s;
  };
  // ages beyond the axis: the piece's mass goes to the end node (tau = 1)
  if (T0 < t_first) {
    const float x1 = fminf(T1, t_first);
    const float m = lin_mass(T0, x1, psi0, gr, T0);
    const float dp0 = lin_mass(T0, x1, 1.f, -1.f / D, T0), dp1 = lin_mass(T0, x1, 0.f, 1.f / D, T0);
    const float dt0 = -psi0 + lin_mass(T0, x1, hT0_0, hT0_g, T0);
    const float dt1 = (T1 < t_first ? psi1 : 0.f) + lin_mass(T0, x1, 0.f, hT1_g, T0);
    add(0, m, dp0, dp1, dt0, dt1);
  }
  if (T1 > t_last) {
    const float x0 = fmaxf(T0, t_last);
    const float m = lin_mass(x0, T1, psi0, gr, T0);
    const float dp0 = lin_mass(x0, T1, 1.f, -1.f / D, T0), dp1 = lin_mass(x0, T1, 0.f, 1.f / D, T0);
    const float dt0 = (T0 > t_last ? -psi0 : 0.f) + lin_mass(x0, T1, hT0_0, hT0_g, T0);
    const float dt1 = psi1 + lin_mass(x0, T1, 0.f, hT1_g, T0);
    add(NA - 1, m, dp0, dp1, dt0, dt1);
  }
  int j = 0, jh = NA - 1;
  while (j < jh) {
    const int mid = (j + jh) >> 1;
    if (g.age_t[mid + 1] > T0) jh = mid; else j = mid + 1;
  }
  for (; j + 1 < NA && g.age_t[j] < T1; ++j) {
    const float tj = g.age_t[j], tj1 = g.age_t[j + 1], dl = g.age_dl[j];
    const float x0 = fmaxf(T0, tj), x1 = fminf(T1, tj1);
    if (!(x1 > x0)) continue;
    float lo, hi, lp0, hp0, lp1, hp1, lt0, ht0, lt1, ht1;
    tent_piece_raw(x0, x1, tj, dl, psi0, gr, T0, lo, hi);
    tent_piece_raw(x0, x1, tj, dl, 1.f, -1.f / D, T0, lp0, hp0);
    tent_piece_raw(x0, x1, tj, dl, 0.f, 1.f / D, T0, lp1, hp1);
    tent_piece_raw(x0, x1, tj, dl, hT0_0, hT0_g, T0, lt0, ht0);
    tent_piece_raw(x0, x1, tj, dl, 0.f, hT1_g, T0, lt1, ht1);
    // moving limits: the piece starts at T0 / ends at T1 when the edge lies inside the interval
    if (T0 > tj) {
      const float tau = logf(T0 / tj) / dl;
      ht0 -= psi0 * tau;
      lt0 -= psi0 * (1.f - tau);
    }
    if (T1 < tj1) {
      const float tau = logf(T1 / tj) / dl;
      ht1 += psi1 * tau;
      lt1 += psi1 * (1.f - tau);
    }
    add(j, lo, lp0, lp1, lt0, lt1);
    add(j + 1, hi, hp0, hp1, ht0, ht1);
  }
  LinGrad out{0.f, 0.f, 0.f, 0.f, 0.f};
  if (!(S > 0.f)) return out;
  const float tgt = 0.5f * (psi0 + psi1) * D;
  const bool on = tgt > 0.f;
  const float target = on ? tgt : 0.f, sc = target / S;
  // dsc/dx = (dtarget/dx - sc dS/dx) / S
  const float tP = on ? 0.5f * D : 0.f, tT0 = on ? -0.5f * (psi0 + psi1) : 0.f, tT1 = -tT0;
  out.p0 = sc * GP0 + GS * (tP - sc * SP0) / S;
  out.p1 = sc * GP1 + GS * (tP - sc * SP1) / S;
  out.t0 = sc * GT0 + GS * (tT0 - sc * ST0) / S;
  out.t1 = sc * GT1 + GS * (tT1 - sc * ST1) / S;
  out.zeta = sc * GZ;
  return out;
}

// Linear scheme, pass 1: the factor that scales bin [T0, T1]'s clipped tent
// shares to its trapezoidal mass max(0, (psi0 + psi1)(T1 - T0)/2).
__device__ float lin_bin_scale(const GridDev& g, float T0, float T1, float psi0, float psi1) {
  const int NA = g.n_age;
  const float t_first = g.age_t[0], t_last = g.age_t[NA - 1], gr = (psi1 - psi0) / (T1 - T0);
  float sum = 0.f;
  if (T0 < t_first) sum += fmaxf(lin_mass(T0, fminf(T1, t_first), psi0, gr, T0), 0.f);
  if (T1 > t_last) sum += fmaxf(lin_mass(fmaxf(T0, t_last), T1, psi0, gr, T0), 0.f);
  int j = 0, jh = NA - 1;   // first node interval [t_j, t_{j+1}] reaching above T0
  while (j < jh) {
    const int mid = (j + jh) >> 1;
    if (g.age_t[mid + 1] > T0) jh = mid; else j = mid + 1;
  }
  for (; j + 1 < NA && g.age_t[j] < T1; ++j) {
    const float x0 = fmaxf(T0, g.age_t[j]), x1 = fminf(T1, g.age_t[j + 1]);
    if (!(x1 > x0)) continue;
    float lo, hi;
    tent_piece(x0, x1, g.age_t[j], g.age_dl[j], psi0, gr, T0, lo, hi);
    sum += lo + hi;
  }
  const float target = fmaxf(0.5f * (psi0 + psi1) * (T1 - T0), 0.f);
  return sum > 0.f ? target / sum : 0.f;
}

// Linear scheme, pass 2: node ag gathers the tent shares of the bins over its
// support [t_{a-1}, t_{a+1}] (and the ages beyond the axis at the end nodes),
// scaled by each bin's factor sc[i] and split by the bin's [Fe/H] (zb, zt),
// into row[NZ].
__device__ void lin_node_fill(const GridDev& g, int ag, int NT, const float* T, const float* m, const float* sc,
                              const int* zb, const float* zt, float* row, int NZ) {
  const int NA = g.n_age;
  const float t_first = g.age_t[0], t_last = g.age_t[NA - 1];
  const float lo_s = ag == 0 ? 0.f : g.age_t[ag - 1];
  const float hi_s = ag == NA - 1 ? INFINITY : g.age_t[ag + 1];
  int i0 = 0, i1 = NT;
  while (i0 < i1) {
    const int mid = (i0 + i1) >> 1;
    if (T[mid + 1] > lo_s) i1 = mid; else i0 = mid + 1;
  }
  for (int i = i0; i < NT && T[i] < hi_s; ++i) {
    if (sc[i] == 0.f) continue;
    const float T0 = T[i], T1 = T[i + 1], psi0 = m[i], gr = (m[i + 1] - psi0) / (T1 - T0);
    float A = 0.f, lo, hi;
    if (ag == 0 && T0 < t_first) A += fmaxf(lin_mass(T0, fminf(T1, t_first), psi0, gr, T0), 0.f);
    if (ag == NA - 1 && T1 > t_last) A += fmaxf(lin_mass(fmaxf(T0, t_last), T1, psi0, gr, T0), 0.f);
    if (ag > 0) {
      const float x0 = fmaxf(T0, g.age_t[ag - 1]), x1 = fminf(T1, g.age_t[ag]);
      if (x1 > x0) {
        tent_piece(x0, x1, g.age_t[ag - 1], g.age_dl[ag - 1], psi0, gr, T0, lo, hi);
        A += hi;
      }
    }
    if (ag + 1 < NA) {
      const float x0 = fmaxf(T0, g.age_t[ag]), x1 = fminf(T1, g.age_t[ag + 1]);
      if (x1 > x0) {
        tent_piece(x0, x1, g.age_t[ag], g.age_dl[ag], psi0, gr, T0, lo, hi);
        A += lo;
      }
    }
    A *= sc[i];
    row[zb[i]] += A * (1.f - zt[i]);
    if (NZ > 1) row[zb[i] + 1] += A * zt[i];
  }
}

// Cubic Hermite interpolant (FP64) of column pair c of the cosmology table
// (value, derivative) at redshift zd.
__device__ __forceinline__ double cosmo_interp(const ModelDev& md, double zd, int c) {
  const double q = zd * md.ctab_inv_h;
  const int i = min((int)q, md.n_ctab - 1);
  const double u = q - (double)i, v = 1.0 - u;
  const double* t0 = md.ctab + COSMO_COLS * (size_t)i + 2 * c;
  const double* t1 = t0 + COSMO_COLS;
  const double h00 = (1.0 + 2.0 * u) * v * v, h10 = u * v * v * md.ctab_h;
  const double h01 = u * u * (3.0 - 2.0 * u), h11 = -u * u * v * md.ctab_h;
  return h00 * t0[0] + h10 * t0[1] + h01 * t1[0] + h11 * t1[1];
}

// T_max = t_univ(z) - t_univ(z_f) and ln(T_max / 10 Myr) alone, with the
// row's redshift status: the SFH edges wait for it, the rest of the row's
// cosmology (row_cosmo) does not.
struct TmaxRow {
  double tmax;
  float lrat;
  uint32_t status;   // SED_ROW_BAD_THETA (z or logmass), SED_ROW_BAD_Z, SED_ROW_BAD_TMAX or 0
};
__device__ TmaxRow row_tmax(const ModelDev& md, float z, float lm) {
  TmaxRow t{0.0, 0.f, 0u};
  if (!isfinite(z) || !isfinite(lm)) {
    t.status = SED_ROW_BAD_THETA;
  } else if (!(z >= 0.f && (double)z < md.zf)) {
    t.status = SED_ROW_BAD_Z;
  } else {
    t.tmax = cosmo_interp(md, (double)z, 1) - md.t_zf_yr;
    t.lrat = t.tmax > 1e7 ? logf((float)(t.tmax * 1e-7)) : 0.f;
    t.status = t.tmax > 1e7 ? 0u : SED_ROW_BAD_TMAX;
  }
  return t;
}

__device__ CosmoRow row_cosmo(const ModelDev& md, float z, float lm, int lane) {
  // All 32 lanes of a warp call it with the same z and lm; lane 0's result is
  // complete.  Lanes 0-3 each evaluate one of the four interpolants in the same
  // FP64 instructions (lane & 3 picks the column pair), the others follow by
  // shuffles: a quarter of the FP64 work of one lane doing all four.
  CosmoRow c{};
  if (!isfinite(z) || !isfinite(lm)) {
    c.status = SED_ROW_BAD_THETA;
  } else if (!(z >= 0.f && (double)z < md.zf)) {
    c.status = SED_ROW_BAD_Z;
  } else {
    const double zd = (double)z, zp = 1.0 + zd;
    const double val = cosmo_interp(md, zd, lane & 3);
    const double dc = __shfl_sync(0xffffffffu, val, 0), tu = __shfl_sync(0xffffffffu, val, 1);
    const double l1 = __shfl_sync(0xffffffffu, val, 2), izp = __shfl_sync(0xffffffffu, val, 3);
    const double tmax = tu - md.t_zf_yr;
    double dl = zp * dc;
    const bool floor10 = dl < 10.0 * PC_CM;
    if (floor10) dl = 10.0 * PC_CM;
    // 1/D_L: the FP32 reciprocal and one Newton step in FP64 (two FMAs instead
    // of an FP64 division); the flux scale s carries no rounding of it that the
    // likelihood of a well-fitting row would amplify
    const float idlf = 1.f / (float)dl;
    const double idl0 = (double)idlf, idl = fma(idl0, fma(-dl, idl0, 1.0), idl0);
    // 2^(lm log2 10) from an exact FP32 split: e2 = hi + lo with hi the rounded
    // product, floor(hi) as the binary exponent, exp2f of the small remainder
    constexpr float L2T_HI = 3.32192802429199219f;                 // log2(10) rounded to FP32
    constexpr float L2T_LO = (float)(3.32192809488736234787 - 3.32192802429199218750);  // the rest, 7.06e-8
    const float hi = lm * L2T_HI;
    const float lo = fmaf(lm, L2T_HI, -hi) + lm * L2T_LO;
    const float en = floorf(hi);
    const float m2 = exp2f((hi - en) + lo);
    const double sc = (double)ldexpf(m2, (int)en) * md.lsun_c * zp * idl * idl;
    const float izf = (float)izp;
    c.s_spec = (float)sc;
    c.p_phot = (float)(C_AA * sc) * izf * izf;
    c.inv1pz = izf;
    c.ln1pz_hi = (float)l1;
    c.ln1pz_lo = (float)(l1 - (double)c.ln1pz_hi);
    // adjoint factors (FP32): dlnD_L/dz = (D_C + (1+z) c/(H0 E)) / D_L, dt/dz = -1/(H0 (1+z) E)
    const float zpf = 1.f + z, ezf = sqrtf((float)md.Om0 * zpf * zpf * zpf + (1.f - (float)md.Om0));
    const float dlnd = floor10 ? 0.f : ((float)dc + zpf * (float)md.dh_cm / ezf) * idlf;
    c.dlns_dz = izf - 2.f * dlnd;
    c.dlnp_dz = -izf - 2.f * dlnd;
    c.dtmax_dz = -(float)md.th_yr * izf / ezf;
    c.tmax_d = tmax;
    c.lrat = tmax > 1e7 ? logf((float)(tmax * 1e-7)) : 0.f;
    c.status = tmax > 1e7 ? 0u : SED_ROW_BAD_TMAX;
  }
  return c;
}

struct PrepKernelArgs {
  PrepArgs p;
};

// Processing order: rows grouped by redshift within chunks of ORDER_CHUNK rows
// (one CTA per chunk, counting sort into ORDER_BINS bins; rows with an invalid
// redshift go last).  Rows that are close in redshift need the same
// rest-frame wavelengths, so a 128-row tile of grouped rows spans a narrow node
// window and the contraction skips the wavelength tiles no row of the tile
// reads.  With one constant [Fe/H] (and [a/Fe]) per row, a row's weights sit
// in the four (a/Fe, Fe/H) blocks of its bracket pair: the rows are then
// grouped by that pair first and by redshift within it, so a 128-row tile
// touches few K tiles and the contraction skips the rest (K-tile masks).
// The order within a bin follows shared-memory atomics and may change from
// call to call; no row's result depends on the order or on which rows share
// its tile.
constexpr int ORDER_CHUNK = 4096;
constexpr int ORDER_THREADS = 1024;
constexpr int ORDER_BINS = 1024;

struct OrderArgs {
  const float* theta;
  int n, ld;
  int* perm;
  ModelDev md;
  const ModelDev* mtab;   // rows of several fits (serving): row r's model is mtab[row_model[r]]
  const int* row_model;   // NULL: every row uses md
  int by_pair;       // 1: two redshift halves, bracket pair, then redshift
  int n_pairs;       // bracket pairs (by_pair)
  int* tile_win;     // set to empty windows by CTA 0 (lo = 0x7f7f7f7f, hi = -1), or NULL
  uint32_t* kmask;   // cleared by CTA 0, or NULL
  int mt, kmask_w;   // 128-row tiles; mask words per tile
};

__global__ void __launch_bounds__(ORDER_THREADS) k_order(const __grid_constant__ OrderArgs oa) {
  pdl_enter();
  // the per-tile windows and K-tile masks the preparation kernel accumulates
  // into start empty (done here rather than by separate memsets)
  if (blockIdx.x == 0) {
    for (int i = threadIdx.x; i < oa.mt && oa.tile_win; i += ORDER_THREADS) {
      oa.tile_win[i] = 0x7f7f7f7f;
      oa.tile_win[oa.mt + i] = -1;
    }
    for (int i = threadIdx.x; i < oa.mt * oa.kmask_w && oa.kmask; i += ORDER_THREADS) oa.kmask[i] = 0u;
  }
  __shared__ int cnt[ORDER_BINS + 1];
  __shared__ int wsum[ORDER_THREADS / 32];
  const ModelDev& md = oa.md;
  const int base = blockIdx.x * ORDER_CHUNK;
  const int m = min(ORDER_CHUNK, oa.n - base);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  __shared__ int s_zlo, s_zhi;   // redshift range of the chunk's valid rows (float bits: z >= 0)
  for (int b = tid; b <= ORDER_BINS; b += ORDER_THREADS) cnt[b] = 0;
  if (tid == 0) { s_zlo = 0x7f7fffff; s_zhi = 0; }
  __syncthreads();
  constexpr int PER = ORDER_CHUNK / ORDER_THREADS;
  int bin[PER];
  float zv[PER];
#pragma unroll
  for (int u = 0; u < PER; ++u) {
    const int i = tid + u * ORDER_THREADS;
    zv[u] = -1.f;
    if (i < m) {
      // the row's own model (serving: fits with their own layouts and z_f); a
      // fixed redshift is read past the caller's columns
      const ModelDev& mr = oa.row_model ? oa.mtab[oa.row_model[base + i]] : md;
      const int zoff = mr.offs[SED_KEY_ZRED];
      const float z = zoff < mr.n_param ? oa.theta[(size_t)(base + i) * oa.ld + zoff] : mr.fixed_v[zoff - mr.n_param];
      if (z >= 0.f && z < (float)mr.zf) zv[u] = z;
    }
  }
  {
    // range of the valid redshifts (z >= 0: their float bits order like ints),
    // one shared atomic per warp
    int lo = 0x7f7fffff, hi = 0;
#pragma unroll
    for (int u = 0; u < PER; ++u)
      if (zv[u] >= 0.f) { lo = min(lo, __float_as_int(zv[u])); hi = max(hi, __float_as_int(zv[u])); }
    lo = __reduce_min_sync(0xffffffffu, lo);
    hi = __reduce_max_sync(0xffffffffu, hi);
    if (lane == 0) { atomicMin(&s_zlo, lo); atomicMax(&s_zhi, hi); }
  }
  __syncthreads();
  // bins over the chunk's own redshift range: by_pair, two halves of it, the
  // bracket pair, then fine redshift bins; else fine redshift bins only
  const float zlo = __int_as_float(s_zlo), zr = fmaxf(__int_as_float(s_zhi) - zlo, 1e-6f);
  const int nf = oa.by_pair ? ORDER_BINS / (2 * oa.n_pairs) : ORDER_BINS;
  const float fscale = (float)nf / zr;
#pragma unroll
  for (int u = 0; u < PER; ++u) {
    const int i = tid + u * ORDER_THREADS;
    bin[u] = -1;
    if (i < m) {
      const float z = zv[u];
      if (z >= 0.f) {
        int b = min(nf - 1, (int)((z - zlo) * fscale));
        if (oa.by_pair) {
          const float* row = oa.theta + (size_t)(base + i) * oa.ld;
          int j0, j1, n0 = 0, n1;
          float w0, w1;
          bracket_f(md.feh, md.n_feh, theta_col(md, row, md.offs[SED_KEY_LOGZSOL]), j0, w0, j1, w1);
          if (md.use_afe && md.n_afe > 1) bracket_f(md.afe, md.n_afe, theta_col(md, row, md.offs[SED_KEY_AFE]), n0, w0, n1, w1);
          const int half = (z - zlo) * 2.f >= zr ? 1 : 0;
          b += (half * oa.n_pairs + n0 * max(md.n_feh - 1, 1) + j0) * nf;
        }
        bin[u] = b;
      } else {
        bin[u] = ORDER_BINS;
      }
      atomicAdd(&cnt[bin[u]], 1);
    }
  }
  __syncthreads();
  // exclusive scan of the bin counts (one bin per thread, plus the invalid bin)
  int v = tid < ORDER_BINS ? cnt[tid] : 0;
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) wsum[warp] = x;
  __syncthreads();
  if (warp == 0) {
    int w = wsum[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    wsum[lane] = w;
  }
  __syncthreads();
  const int total_valid = wsum[ORDER_THREADS / 32 - 1];
  const int excl = x - v + (warp ? wsum[warp - 1] : 0);
  __syncthreads();
  if (tid < ORDER_BINS) cnt[tid] = excl;
  if (tid == 0) cnt[ORDER_BINS] = total_valid;
  __syncthreads();
#pragma unroll
  for (int u = 0; u < PER; ++u) {
    const int i = tid + u * ORDER_THREADS;
    if (i < m) oa.perm[base + atomicAdd(&cnt[bin[u]], 1)] = base + i;
  }
}

constexpr int PREP_THREADS = 128;
constexpr int PREP_KWARPS = PREP_THREADS / 32 - 1;   // warps writing W; the last one assembles the row's scalars
// Largest launch that orders itself (PrepArgs::self_order): each CTA reads
// every row's redshift, so the cost grows with n^2
constexpr int SELF_ORDER_MAX = 1024;
static_assert(SELF_ORDER_MAX <= 2 * MAX_SFH + 1, "the redshifts are staged in the edge and rate arrays");

// Row p of the launch processes the caller's row r = perm[p] and records r in
// RowScal::orig; every later kernel indexes by p and writes results to r.
// Self-ordered (a.self_order): CTA b processes the caller's row r = b, and its
// last warp finds p, the row's place in the order k_order would give by
// counting the rows whose (redshift bin, index) key is below its own (stable
// counting sort over the same bins; every CTA forms the same keys).
template <bool MULTI>
__global__ void __launch_bounds__(PREP_THREADS) k_prep(const __grid_constant__ PrepKernelArgs ka) {
  const PrepArgs& a = ka.p;
  pdl_enter();
  const int b = blockIdx.x;
  const int r = a.self_order ? b : (a.perm ? a.perm[b] : b);
  const ModelDev& md = MULTI ? a.mtab[a.row_model[r]] : a.md;
  const GridDev& g = a.g;
  const LayoutDev& L = a.L;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const float* th = a.theta + (size_t)r * a.ld;
  const int NT = md.n_sfh, NA = g.n_age, NZ = g.n_feh;
  if (b == 0 && tid == 0 && a.err) *a.err = 0;

  extern __shared__ float smem[];
  float* Ws = smem;                     // [NA][NZ]
  // the row's parameters, read once (coalesced) into the tail of the dynamic
  // shared memory: theta may be the caller's pinned host buffer, read in place
  float* th_s = smem + (size_t)NA * NZ + (a.W_f8 ? L.Kpad : 0);
  // edges T[0..NT] and rates m_i / dT_i; before them (self-ordered launch) the
  // launch's redshifts
  __shared__ float s_trate[2 * MAX_SFH + 1];
  float* T = s_trate;
  float* rate = s_trate + MAX_SFH + 1;
  __shared__ int s_pos;
  __shared__ int zb[MAX_SFH];
  __shared__ float zt[MAX_SFH];
  __shared__ float s_red[PREP_THREADS / 32];
  __shared__ float s_redq[MAX_SEG + 1][PREP_THREADS / 32];   // age-binned dust: Q of each block
  __shared__ float s_red8[PREP_THREADS / 32];
  __shared__ int s_nnz[PREP_THREADS / 32];
  // K tiles the row touches: [Fe/H] nodes that bracket some bin, ages whose
  // cell (or tent) reaches below T_max, and both [a/Fe] nodes of the bracket
  __shared__ unsigned long long s_mpart[PREP_THREADS / 32];   // per warp
  __shared__ int s_alim;
  __shared__ uint32_t s_km[KMASK_WORDS];
  __shared__ uint32_t s_wprev[KMASK_WORDS];   // K tiles of this W row that may hold non-zeros from before
  if (tid == 0) s_alim = 0;
  if (tid < KMASK_WORDS) s_km[tid] = 0u;

  // ---- in the shadow of the row's loads: finiteness of the whole row; T_max
  //      (warp 0: the SFH edges wait for it); the bins' [Fe/H] brackets and the
  //      cleared weight table (the other warps).  The rest of the row's
  //      cosmology waits for the last warp, beside the writes of W.
  __shared__ double s_tmax;
  __shared__ float s_lrat;
  __shared__ uint32_t s_zst;
  int bad = 0;
  for (int j = tid; j < md.n_param; j += blockDim.x) {
    const float v = th[j];
    th_s[j] = v;
    bad |= !isfinite(v);
  }
  for (int j = tid; j < md.n_fixed; j += blockDim.x) th_s[md.n_param + j] = md.fixed_v[j];   // fixed keys
  unsigned long long mpart = 0ull;
  const bool rank_warp = a.self_order && warp == PREP_THREADS / 32 - 1;
  if (warp == 0) {
    const TmaxRow t = row_tmax(md, theta_col(md, th, md.offs[SED_KEY_ZRED]), theta_col(md, th, md.offs[SED_KEY_LOGMASS]));
    if (lane == 0) { s_tmax = t.tmax; s_lrat = t.lrat; s_zst = t.status; }
  } else if (rank_warp) {
    // the row's place in the redshift order: the valid redshifts (z in
    // [0, z_f), others -1) and their range, then the keys of k_order's bins
    // over that range (invalid rows in the last bin) and the count of rows
    // whose (key, index) is below this row's
    float* zs = s_trate;
    const int zoff = md.offs[SED_KEY_ZRED];
    int lo = 0x7f7fffff, hi = 0;
#pragma unroll 8
    for (int j = lane; j < a.n; j += 32) {
      const float z = a.theta[(size_t)j * a.ld + zoff];
      const float zv = z >= 0.f && z < (float)md.zf ? z : -1.f;
      zs[j] = zv;
      if (zv >= 0.f) { lo = min(lo, __float_as_int(zv)); hi = max(hi, __float_as_int(zv)); }
    }
    lo = __reduce_min_sync(0xffffffffu, lo);
    hi = __reduce_max_sync(0xffffffffu, hi);
    __syncwarp();
    const float zlo = __int_as_float(lo), zr = fmaxf(__int_as_float(hi) - zlo, 1e-6f);
    const float fscale = (float)ORDER_BINS / zr;
    auto key = [&](float z) { return z >= 0.f ? min(ORDER_BINS - 1, (int)((z - zlo) * fscale)) : ORDER_BINS; };
    const int kb = key(zs[b]);
    int below = 0;
    for (int j = lane; j < a.n; j += 32) {
      const int kj = key(zs[j]);
      below += kj < kb || (kj == kb && j < b);
    }
    below = __reduce_add_sync(0xffffffffu, below);
    if (lane == 0) s_pos = below;
  } else {
    const int NB = PREP_THREADS - 32 - (a.self_order ? 32 : 0);
    for (int j = tid - 32; j < NA * NZ; j += NB) Ws[j] = 0.f;
    for (int i = tid - 32; i < NT; i += NB) {
      int j0, j1;
      float w0, w1;
      bracket_f(md.feh, md.n_feh, theta_col(md, th, md.offs[SED_KEY_LOGZSOL] + (md.zmode == 0 ? i : 0)), j0, w0, j1, w1);
      zb[i] = j0;
      zt[i] = w1;   // weight of j0 + 1 (0 when n_feh == 1)
      mpart |= (1ull << j0) | (1ull << j1);
    }
  }
  for (int o = 16; o; o >>= 1) mpart |= __shfl_xor_sync(0xffffffffu, mpart, o);
  if (lane == 0) s_mpart[warp] = mpart;
  bad = __syncthreads_or(bad);
  th = th_s;
  const int p = a.self_order ? s_pos : b;   // the row's place in the launch's order
  if (tid < KMASK_WORDS) s_wprev[tid] = a.wmask ? a.wmask[(size_t)p * KMASK_WORDS + tid] : 0xffffffffu;
  uint32_t status = bad ? SED_ROW_BAD_THETA : 0u;
  // a sampled sigma_gal outside the model's declared range [0, max]
  if (!status && md.sample_sgal) {
    const float sg = th[md.offs[SED_KEY_SIGMA_GAL]];
    if (!(sg >= 0.f && sg <= md.sgal_max_kms)) status = SED_ROW_BAD_THETA;
  }
  // a runaway fraction outside [0, 1] (Sec. frac_obrun)
  if (!status && md.fesc_geom) {
    const float f = th[md.offs[SED_KEY_FRAC_OBRUN]];
    if (!(f >= 0.f && f <= 1.f)) status = SED_ROW_BAD_THETA;
  }
  // a sampled gas dispersion outside its declared range [0, max]
  if (!status && md.gas_mode == SED_GAS_SIGMA_SAMPLED) {
    const float sg = th[md.offs[SED_KEY_SIGMA_GAS]];
    if (!(sg >= 0.f && sg <= md.sgas_max_kms)) status = SED_ROW_BAD_THETA;
  }
  if (!status) status = s_zst;
  const double tmax = status ? 0.0 : s_tmax;

  RowScal* out = a.rs + p;
  const int Kpad = L.Kpad;
  if (status) {
    for (int k = tid; k < Kpad; k += blockDim.x) {
      size_t o = (size_t)p * Kpad + k;
      if (a.W) a.W[o] = 0.f;
      if (a.W_hi) { a.W_hi[o] = 0.f; a.W_lo[o] = 0.f; }
      if (a.W_bf16) a.W_bf16[o] = __float2bfloat16_rn(0.f);
    }
    if (a.W_f8)
      for (int k = tid; k < L.Kpad8; k += blockDim.x) a.W_f8[(size_t)p * L.Kpad8 + k] = 0;
    if (a.wmask && tid < KMASK_WORDS) a.wmask[(size_t)p * KMASK_WORDS + tid] = 0u;   // the row is all zeros now
    if (tid == 0) {
      RowScal rs{};
      rs.status = status;
      rs.k_lo = 0;
      rs.k_hi = 0;
      rs.orig = r;
      *out = rs;
    }
    return;
  }

  // ---- SFH edges (FP32) and per-bin rates: thread i forms both edges of bin
  //      i (the same function of i, so neighbours agree on the shared edge)
  const float* m = th + md.offs[SED_KEY_SFH];
  const float lrat = s_lrat;
  for (int i = tid; i < NT; i += blockDim.x) {
    const float t0 = sfh_edge(i, NT, tmax, lrat), t1 = sfh_edge(i + 1, NT, tmax, lrat);
    T[i] = t0;
    if (i == NT - 1) T[NT] = t1;
    // linear scheme, pass 1: the factor scaling the bin's tent shares
    rate[i] = md.sfh_linear ? lin_bin_scale(g, t0, t1, m[i], m[i + 1]) : m[i] / (t1 - t0);
  }
  if (a.kmask) {
    const float tn = sfh_edge(NT, NT, tmax, lrat);
    for (int ag = tid; ag < NA; ag += blockDim.x)
      if (g.cell_lo[ag] < tn) atomicMax(&s_alim, ag + 1);
  }
  __syncthreads();

  // ---- weights on (age, feh): thread per age node, by the warps that write W
  //      (a named barrier joins them); the last warp goes straight on to the
  //      row's cosmology and scalars, which do not read the weights
  constexpr int NKT = PREP_KWARPS * 32;
  if (warp < PREP_KWARPS) {
  if (md.sfh_linear) {
    // linear scheme, pass 2: node a gathers the tent shares of the bins over
    // its support [t_{a-1}, t_{a+1}] (and the ages beyond the axis at the end
    // nodes), scaled by each bin's factor and split by the bin's [Fe/H]
    for (int ag = tid; ag < NA; ag += NKT) lin_node_fill(g, ag, NT, T, m, rate, zb, zt, Ws + ag * NZ, NZ);
  } else
  for (int ag = tid; ag < NA; ag += NKT) {
    const float lo = g.cell_lo[ag], hi = g.cell_hi[ag];
    // first bin whose upper edge is above the cell's lower edge
    int i0 = 0, i1 = NT;
    while (i0 < i1) {
      int mid = (i0 + i1) >> 1;
      if (T[mid + 1] > lo) i1 = mid; else i0 = mid + 1;
    }
    float* row = Ws + ag * NZ;
    for (int i = i0; i < NT && T[i] < hi; ++i) {
      float ov = fminf(T[i + 1], hi) - fmaxf(T[i], lo);
      if (ov <= 0.f) continue;
      float A = rate[i] * ov;
      int j = zb[i];
      float t = zt[i];
      row[j] += A * (1.f - t);
      if (NZ > 1) row[j + 1] += A * t;
    }
  }
  asm volatile("bar.sync 1, %0;" ::"r"(NKT) : "memory");
  }

  // ---- [a/Fe] split and the K-ordered row of W; Q_young
  int n0 = 0, n1 = 0;
  float wn0 = 1.f, wn1 = 0.f;
  if (md.n_afe > 1) {
    const float afe = md.use_afe ? th[md.offs[SED_KEY_AFE]] : 0.f;
    bracket_f(md.afe, md.n_afe, afe, n0, wn0, n1, wn1);
  }
  float qpart = 0.f;
  int nnz = 0;
  float* Vs = smem + NA * NZ;           // FP8 path: W_k 2^-e_k
  // the row's scalars, assembled by the last warp while the others write W
  static_assert(sizeof(RowScal) % 4 == 0, "RowScal is cleared and copied as words");
  __shared__ RowScal s_rs;
  if (warp < PREP_KWARPS) {
    // touched columns: the bracket nodes (also where a weight is 0 at a node:
    // the adjoint reads their derivative) and one age past the last cell below
    // T_max (the linear scheme's tents reach one node further)
    unsigned long long mset = 0ull;
    for (int w = 0; w < PREP_THREADS / 32; ++w) mset |= s_mpart[w];
    const int alim = s_alim + 1;
    const int f8_shift = L.Ky_pad8 - L.Ky_pad;
    // four consecutive columns per lane (one int4 of column codes, vector
    // stores); a warp step spans 128 columns, so the loop is uniform per warp
    // and the K-tile mask needs no partial-warp ballot
    // the column codes and Q of the next step are loaded before this step's
    // work (the loop's latency is these loads, not its arithmetic)
    constexpr int KSTEP = PREP_KWARPS * 128;
    auto load_cols = [&](int kb, int4& cd, float4& qs) {
      const int k4 = kb + 4 * lane;
      cd = make_int4(-1, -1, -1, -1);
      qs = make_float4(0.f, 0.f, 0.f, 0.f);
      if (k4 < Kpad) {
        cd = __ldg(reinterpret_cast<const int4*>(L.k_code + k4));
        if (k4 < L.Ky_pad) qs = __ldg(reinterpret_cast<const float4*>(L.q_s + k4));
      }
    };
    int4 cd_next;
    float4 qs_next;
    load_cols(warp * 128, cd_next, qs_next);
    for (int kb = warp * 128; kb < Kpad; kb += KSTEP) {
      const int k4 = kb + 4 * lane;
      const bool in = k4 < Kpad;   // Kpad is a multiple of 32, so a lane's four columns are all in or all out
      const int4 cd = cd_next;
      const float4 qs = qs_next;
      if (kb + KSTEP < Kpad) load_cols(kb + KSTEP, cd_next, qs_next);
      const int cc[4] = {cd.x, cd.y, cd.z, cd.w};
      const float qq[4] = {qs.x, qs.y, qs.z, qs.w};
      float v[4];
      bool touched = false;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        v[j] = 0.f;
        const int code = cc[j];
        if (code >= 0) {
          const int n = code >> 24, mm = (code >> 16) & 0xff, ag = code & 0xffff;
          const float wn = (n == n0 ? wn0 : 0.f) + (n == n1 && n1 != n0 ? wn1 : 0.f);
          v[j] = wn * Ws[ag * NZ + mm];
          touched |= (n == n0 || (n == n1 && (md.use_afe || wn1 != 0.f))) && ((mset >> mm) & 1ull) && ag < alim;
        }
        qpart = fmaf(v[j], qq[j], qpart);   // q_s is 0 past the young block
        nnz += v[j] != 0.f;
      }
      bool store = in;
      if (a.kmask) {
        // one K tile holds 32, 64 or 128 columns, i.e. 8, 16 or 32 lanes' quads:
        // the lowest lane of each tile's group sets its bit
        const int q = a.W_f8 ? (k4 < L.Ky_pad ? k4 : k4 + f8_shift) : k4;
        const int t = q >> a.kt_shift;
        // 32-column tiles (3xTF32) are the quads of lanes 8g..8g+7 (a warp step
        // starts on a 128-column boundary); other layouts group by tile
        const unsigned grp = a.kt_shift == 5 && !a.W_f8 ? 0xffu << (lane & ~7) : __match_any_sync(0xffffffffu, t);
        const unsigned tb = __ballot_sync(0xffffffffu, touched && in);
        if ((tb & grp) && lane == __ffs(grp) - 1) atomicOr(&s_km[t >> 5], 1u << (t & 31));
        // a tile this row does not touch holds zeros: written only where the
        // row at this position may have left non-zeros
        if (a.wmask) store = in && ((tb & grp) != 0u || ((s_wprev[t >> 5] >> (t & 31)) & 1u));
      }
      if (!store) continue;
      const size_t o = (size_t)p * Kpad + k4;
      if (a.W) *reinterpret_cast<float4*>(a.W + o) = make_float4(v[0], v[1], v[2], v[3]);
      if (a.W_hi) {
        const float4 h = make_float4(tf32_rna(v[0]), tf32_rna(v[1]), tf32_rna(v[2]), tf32_rna(v[3]));
        *reinterpret_cast<float4*>(a.W_hi + o) = h;
        *reinterpret_cast<float4*>(a.W_lo + o) = make_float4(v[0] - h.x, v[1] - h.y, v[2] - h.z, v[3] - h.w);
      }
      if (a.W_bf16) {
        const __nv_bfloat162 b01 = __floats2bfloat162_rn(v[0], v[1]), b23 = __floats2bfloat162_rn(v[2], v[3]);
        uint2 u;
        u.x = *reinterpret_cast<const uint32_t*>(&b01);
        u.y = *reinterpret_cast<const uint32_t*>(&b23);
        *reinterpret_cast<uint2*>(a.W_bf16 + o) = u;
      }
      if (a.W_f8) {
        const float4 c8 = __ldg(reinterpret_cast<const float4*>(L.col8 + k4));
        Vs[k4] = v[0] * c8.x;
        Vs[k4 + 1] = v[1] * c8.y;
        Vs[k4 + 2] = v[2] * c8.z;
        Vs[k4 + 3] = v[3] * c8.w;
      }
    }
    for (int o = 16; o; o >>= 1) {
      qpart += __shfl_xor_sync(0xffffffffu, qpart, o);
      nnz += __shfl_xor_sync(0xffffffffu, nnz, o);
    }
  } else {
    // ---- the row's cosmology and observer-frame scalars (FP64 interpolants;
    //      measured slower when run beside T_max at the start: the two warps
    //      then share the SM's FP64 pipe on the critical path)
    const CosmoRow cr = row_cosmo(md, th[md.offs[SED_KEY_ZRED]], th[md.offs[SED_KEY_LOGMASS]], lane);
    // ---- rest-frame node window the epilogue reads: the redshifted filter
    //      samples and the spectral pixels with 5 dispersions on either side.
    //      Lanes 0-3 look up its four candidate ends in the index table over
    //      ln(lambda) (each entry lies within one node of the exact bracket);
    //      the margins cover that slack and the interpolation's k + 1.
    const int N = g.n_lam;
    const float lam0 = g.lam_f[0], lamN = g.lam_f[N - 1];
    int lo = N - 1, hi = 0;
    float xl = 0.f;
    bool use = false;
    if (lane < 2 && md.n_filt > 0) {
      xl = __logf(fminf(fmaxf((lane == 0 ? md.samp_lam_min : md.samp_lam_max) * cr.inv1pz, lam0), lamN));
      use = true;
    } else if (lane >= 2 && lane < 4 && md.n_pix > 0) {
      const double l1 = (double)cr.ln1pz_hi + (double)cr.ln1pz_lo;
      const float ll0 = g.lnl_hi[0], llN = g.lnl_hi[N - 1];
      xl = lane == 2 ? fminf(fmaxf((float)(md.pix_ln_min - l1) - 5.f * md.pix_s_max, ll0), llN)
                     : fminf(fmaxf((float)(md.pix_ln_max - l1) + 5.f * md.pix_s_max, ll0), llN);
      use = true;
    }
    if (use) {
      int q = (int)((xl - g.lut_x0) * g.lut_inv_h);
      q = q < 0 ? 0 : (q >= g.lut_n ? g.lut_n - 1 : q);
      const int k = g.lut[q];
      if ((lane & 1) == 0) lo = k; else hi = k;
    }
    for (int o = 2; o; o >>= 1) {
      lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
      hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    const int win_lo = max(lo - 3, 0);
    const int win_hi = min(max(hi + 4, win_lo + 1), N - 1);
    for (int i = lane; i < (int)(sizeof(RowScal) / 4); i += 32) reinterpret_cast<uint32_t*>(&s_rs)[i] = 0u;
    __syncwarp();
    if (lane == 0) {
      RowScal& rs = s_rs;   // fields set in place (shared memory; no local copy)
      rs.p_phot = cr.p_phot;
      rs.s_spec = cr.s_spec;
      rs.inv1pz = cr.inv1pz;
      rs.ln1pz_hi = cr.ln1pz_hi;
      rs.ln1pz_lo = cr.ln1pz_lo;
      rs.tau_bc = th[md.offs[SED_KEY_TAU_POW]];
      rs.alpha_bc = th[md.offs[SED_KEY_ALPHA_POW]];
      rs.tau_d = th[md.offs[SED_KEY_DIFFUSE_TAU]];
      rs.delta = th[md.offs[SED_KEY_DIFFUSE_INDEX]];
      // noise-floor terms (App. sys_floor): 10^column for a term that is on
      for (int arm = 0; arm < 2; ++arm)
        for (int k = 0; k < 4; ++k)
          rs.fl[arm][k] = ((md.floor_bits[arm] >> k) & 1) ? exp10f(th[md.offs[SED_KEY_LOG_ERR_SCALE_PHOT + 4 * arm + k]])
                                                          : (k == 0 ? 1.f : 0.f);
      if (md.use_neb) {
        int u0, u1, z0, z1;
        float wu0, wu1, wz0, wz1;
        bracket_f(md.neb_logu, md.neb_nu, th[md.offs[SED_KEY_GAS_LOGU]], u0, wu0, u1, wu1);
        bracket_f(md.neb_logz, md.neb_nz, th[md.offs[SED_KEY_GAS_LOGZ]], z0, wz0, z1, wz1);
        const int nl = g.n_lam;
        rs.neb_w[0] = wu0 * wz0; rs.neb_off[0] = (u0 * md.neb_nz + z0) * nl;
        rs.neb_w[1] = wu0 * wz1; rs.neb_off[1] = (u0 * md.neb_nz + z1) * nl;
        rs.neb_w[2] = wu1 * wz0; rs.neb_off[2] = (u1 * md.neb_nz + z0) * nl;
        rs.neb_w[3] = wu1 * wz1; rs.neb_off[3] = (u1 * md.neb_nz + z1) * nl;
        float du0, du1, dz0, dz1;
        bracket_df(md.neb_logu, md.neb_nu, th[md.offs[SED_KEY_GAS_LOGU]], u0, u1, du0, du1);
        bracket_df(md.neb_logz, md.neb_nz, th[md.offs[SED_KEY_GAS_LOGZ]], z0, z1, dz0, dz1);
        rs.neb_dwu[0] = du0 * wz0; rs.neb_dwu[1] = du0 * wz1; rs.neb_dwu[2] = du1 * wz0; rs.neb_dwu[3] = du1 * wz1;
        rs.neb_dwz[0] = wu0 * dz0; rs.neb_dwz[1] = wu0 * dz1; rs.neb_dwz[2] = wu1 * dz0; rs.neb_dwz[3] = wu1 * dz1;
      }
      rs.dlns_dz = cr.dlns_dz;
      rs.dlnp_dz = cr.dlnp_dz;
      rs.dtmax_dz = cr.dtmax_dz;
      rs.tmax = (float)tmax;
      rs.lrat = lrat;
      rs.status = 0;
      rs.orig = r;
      rs.y_scale = 1.f;
      rs.sg_ln = md.sample_sgal ? th[md.offs[SED_KEY_SIGMA_GAL]] / (float)C_KMS : 0.f;
      rs.fob = md.fesc_geom ? th[md.offs[SED_KEY_FRAC_OBRUN]] : 0.f;
      // the emission lines' gas dispersion (km/s): a column, a fixed value, or
      // tied to the stellar dispersion (the row's sampled sigma_gal, else the fixed one)
      rs.sgas = md.gas_mode == SED_GAS_SIGMA_SAMPLED ? th[md.offs[SED_KEY_SIGMA_GAS]]
              : md.gas_mode == SED_GAS_SIGMA_FIXED ? md.sgas_fix_kms
              : (md.sample_sgal ? th[md.offs[SED_KEY_SIGMA_GAL]] : md.sgal_fix_kms);
      rs.igm_f = md.use_igm ? th[md.offs[SED_KEY_IGM_FACTOR]] : 0.f;
      rs.k_lo = win_lo;
      rs.k_hi = win_hi;
      if (md.n_bin > 0)   // age-binned dust (App. dust_attn): each bin's law parameters
        for (int b = 0; b < md.n_bin; ++b) {
          rs.bin_tau[b] = th[md.offs[SED_KEY_DUST_BINS] + 2 * b];
          rs.bin_slope[b] = th[md.offs[SED_KEY_DUST_BINS] + 2 * b + 1];
        }
      if (a.tile_win) {   // union of the windows of this row's 128-row tile
        const int mt = (a.n + 127) >> 7;
        atomicMin(&a.tile_win[p >> 7], win_lo);
        atomicMax(&a.tile_win[mt + (p >> 7)], win_hi);
      }
    }
  }
  // the passes below read the weights with every warp
  if (md.n_bin > 0 || (a.qneb && g.neb_na > 0)) __syncthreads();
  if (md.n_bin > 0) {
    // age-binned dust: Q of each attenuated block and of the ages outside
    // every block, from the nebular ages' weights (W_k = w_n Ws[a][m] with the
    // [a/Fe] bracket weights w_n)
    float qb[MAX_SEG + 1] = {};
    for (int j = tid + L.neb_a0 * NZ; j < L.n_young * NZ; j += blockDim.x) {
      const int ag = j / NZ, mm = j - ag * NZ;
      const int4 ac = L.age_col[ag];
      const float wv = Ws[ag * NZ + mm];
      float q = wn0 * wv * __ldg(L.q_s + ac.x + (n0 * NZ + mm) * ac.y);
      if (n1 != n0) q += wn1 * wv * __ldg(L.q_s + ac.x + (n1 * NZ + mm) * ac.y);
#pragma unroll
      for (int jj = 0; jj <= MAX_SEG; ++jj) qb[jj] += ac.z == jj ? q : 0.f;
    }
#pragma unroll
    for (int jj = 0; jj <= MAX_SEG; ++jj) {
      for (int o = 16; o; o >>= 1) qb[jj] += __shfl_xor_sync(0xffffffffu, qb[jj], o);
      if (lane == 0) s_redq[jj][warp] = qb[jj];
    }
  }
  if (a.qneb && g.neb_na > 0) {
    // nebular age axis: the Q-weighted weight of each nebular SSP age (the
    // epilogue weights each age's plane of the nebular cube by it)
    for (int i = tid; i < g.neb_na; i += blockDim.x) {
      const int ag = g.neb_a0 + i;
      const int4 ac = L.age_col[ag];
      float q = 0.f;
      for (int mm = 0; mm < NZ; ++mm) {
        const float wv = Ws[ag * NZ + mm];
        q += wn0 * wv * __ldg(L.q_s + ac.x + (n0 * NZ + mm) * ac.y);
        if (n1 != n0) q += wn1 * wv * __ldg(L.q_s + ac.x + (n1 * NZ + mm) * ac.y);
      }
      a.qneb[(size_t)p * MAX_NEB_AGE + i] = q;
    }
  }
  if (lane == 0) { s_red[warp] = qpart; s_nnz[warp] = nnz; }   // 0 from the last warp
  __syncthreads();
  if (a.kmask && tid < a.kmask_w && s_km[tid]) atomicOr(&a.kmask[(size_t)(p >> 7) * a.kmask_w + tid], s_km[tid]);
  if (a.wmask && tid < KMASK_WORDS) a.wmask[(size_t)p * KMASK_WORDS + tid] = s_km[tid];   // the tiles written now

  // ---- FP8 operand: E4M3 of W_k 2^-e_k 2^-y, with the row's power of two 2^y
  //      chosen so that its largest entry maps to at most 240 (< 448, the E4M3
  //      maximum); the epilogue multiplies Y and O back by 2^y
  float y_scale = 1.f;
  if (a.W_f8) {
    float m = 0.f;
    for (int k = tid; k < Kpad; k += blockDim.x) m = fmaxf(m, fabsf(Vs[k]));
    for (int o = 16; o; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0) s_red8[warp] = m;
    __syncthreads();
    m = 0.f;
    for (int w = 0; w < PREP_THREADS / 32; ++w) m = fmaxf(m, s_red8[w]);
    const float e = m > 0.f ? ceilf(log2f(m / 240.f)) : 0.f;
    y_scale = exp2f(e);
    const float inv = exp2f(-e);
    const int shift = L.Ky_pad8 - L.Ky_pad;
    uint8_t* w8 = a.W_f8 + (size_t)p * L.Kpad8;
    for (int q = tid; q < L.Kpad8; q += blockDim.x) {
      int k = q < L.Ky_pad ? q : (q < L.Ky_pad8 ? -1 : q - shift);
      const float v = (k >= 0 && k < Kpad) ? Vs[k] * inv : 0.f;
      w8[q] = (uint8_t)__nv_cvt_float_to_fp8(v, __NV_SATFINITE, __NV_E4M3);
    }
  }

  // ---- the sums over warps, then the row's scalars to global memory (one word per thread)
  if (tid == 0) {
    float qy = 0.f;
    int nz = 0;
    for (int w = 0; w < PREP_THREADS / 32; ++w) {
      qy += s_red[w];
      nz += s_nnz[w];
    }
    s_rs.log2_qy = qy > 0.f ? log2f(qy) : -INFINITY;
    s_rs.nnz = nz;
    s_rs.y_scale = y_scale;
    if (md.n_bin > 0)   // log2 of Q of each attenuated block
      for (int j = 0; j <= MAX_SEG; ++j) {
        float q = 0.f;
        for (int w = 0; w < PREP_THREADS / 32; ++w) q += s_redq[j][w];
        s_rs.log2_qs[j] = q > 0.f ? log2f(q) : -INFINITY;
      }
  }
  __syncthreads();
  for (int i = tid; i < (int)(sizeof(RowScal) / 4); i += blockDim.x)
    reinterpret_cast<uint32_t*>(out)[i] = reinterpret_cast<const uint32_t*>(&s_rs)[i];
}

// ---------------------------------------------------------------------------
// Adjoint of the weights (App. B step scheme, metallicity and [a/Fe] splits)
// and assembly of the gradient row.  One CTA per row.  Input: dlnL/dW from the
// adjoint contraction, dlnL/dQ_young and the other per-row scalar pieces from
// the adjoint epilogue.  W_k = w_n(afe) Ws[a][m], Ws[a][m] = sum_i A_ia w_m(zeta_i),
// A_ia = m_i |bin_i ∩ cell_a| / dT_i, with the edges T_i (i >= 3) following T_max(z).
constexpr int PREP_BWD_THREADS = 128;

// LINEAR: the weights' reverse pass of the linear SFH scheme (a separate
// instance, so the step scheme's keeps its registers and shared memory)
template <bool LINEAR>
__global__ void __launch_bounds__(PREP_BWD_THREADS) k_prep_bwd(const __grid_constant__ PrepBwdArgs a) {
  pdl_enter();
  const ModelDev& md = a.md;
  const GridDev& g = a.g;
  const LayoutDev& L = a.L;
  const int r = blockIdx.x;                 // processing order (dW, rgrad, RowScal)
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const RowScal rs = a.rs[r];
  const float* th = a.theta + (size_t)rs.orig * a.ld;
  float* out = a.grad + (size_t)rs.orig * a.ld;
  const int NT = md.n_sfh, NA = g.n_age, NZ = g.n_feh;
  if (rs.status || a.rgrad[(size_t)r * RGRAD + RG_BAD] != 0.0) {
    for (int j = tid; j < a.ld; j += blockDim.x) out[j] = 0.f;
    return;
  }
  extern __shared__ float smem[];
  float* Ws = smem;               // [NA][NZ] forward Ws
  float* gWs = smem + NA * NZ;    // [NA][NZ] dlnL/dWs
  __shared__ float T[MAX_SFH + 1];
  __shared__ int zb[MAX_SFH];
  __shared__ float zt[MAX_SFH], zd0[MAX_SFH], zd1[MAX_SFH];
  __shared__ float gTlo[MAX_SFH], gThi[MAX_SFH], gzeta[MAX_SFH];
  __shared__ float lin_buf[LINEAR ? 3 * MAX_SFH : 1];   // linear scheme: bin scales, d/dpsi of each bin's edges
  float* lin_sc = lin_buf;
  float* gps0 = lin_buf + (LINEAR ? MAX_SFH : 0);
  float* gps1 = lin_buf + (LINEAR ? 2 * MAX_SFH : 0);
  __shared__ double red[PREP_BWD_THREADS / 32];
  __shared__ double s_tmax_part[PREP_BWD_THREADS / 32];

  const float* m = th + md.offs[SED_KEY_SFH];
  const float* zeta = th + md.offs[SED_KEY_LOGZSOL];
  const double tmax = (double)rs.tmax;
  const float lrat = rs.lrat;   // the forward's edges, bit for bit
  for (int i = tid; i <= NT; i += blockDim.x) T[i] = sfh_edge(i, NT, tmax, lrat);
  for (int j = tid; j < NA * NZ; j += blockDim.x) Ws[j] = 0.f;
  __syncthreads();
  for (int i = tid; i < NT; i += blockDim.x) {
    int j0, j1;
    float w0, w1, d0, d1;
    const float v = md.zmode == 0 ? zeta[i] : theta_col(md, th, md.offs[SED_KEY_LOGZSOL]);
    bracket_f(md.feh, md.n_feh, v, j0, w0, j1, w1);
    bracket_df(md.feh, md.n_feh, v, j0, j1, d0, d1);
    zb[i] = j0;
    zt[i] = w1;
    zd0[i] = d0;
    zd1[i] = d1;
    if constexpr (LINEAR) lin_sc[i] = lin_bin_scale(g, T[i], T[i + 1], m[i], m[i + 1]);
  }
  __syncthreads();
  // forward Ws (needed for the [a/Fe] derivative), thread per age node as in k_prep
  if constexpr (LINEAR) {
    for (int ag = tid; ag < NA; ag += blockDim.x) lin_node_fill(g, ag, NT, T, m, lin_sc, zb, zt, Ws + ag * NZ, NZ);
  } else
  for (int ag = tid; ag < NA; ag += blockDim.x) {
    const float lo = g.cell_lo[ag], hi = g.cell_hi[ag];
    int i0 = 0, i1 = NT;
    while (i0 < i1) {
      int mid = (i0 + i1) >> 1;
      if (T[mid + 1] > lo) i1 = mid; else i0 = mid + 1;
    }
    float* row = Ws + ag * NZ;
    for (int i = i0; i < NT && T[i] < hi; ++i) {
      float ov = fminf(T[i + 1], hi) - fmaxf(T[i], lo);
      if (ov <= 0.f) continue;
      float A = m[i] / (T[i + 1] - T[i]) * ov;
      row[zb[i]] += A * (1.f - zt[i]);
      if (NZ > 1) row[zb[i] + 1] += A * zt[i];
    }
  }
  // [a/Fe] bracket
  int n0 = 0, n1 = 0;
  float wn0 = 1.f, wn1 = 0.f, dn0 = 0.f, dn1 = 0.f;
  if (md.n_afe > 1) {
    const float afe = md.use_afe ? theta_col(md, th, md.offs[SED_KEY_AFE]) : 0.f;
    bracket_f(md.afe, md.n_afe, afe, n0, wn0, n1, wn1);
    if (md.use_afe) bracket_df(md.afe, md.n_afe, afe, n0, n1, dn0, dn1);
  }
  __syncthreads();
  // dlnL/dWs[a][m] and the [a/Fe] derivative; column k of (n, m, a) in the layout
  const float* dW = a.dW + (size_t)r * L.Kpad;
  const float gqy = (float)a.rgrad[(size_t)r * RGRAD + RG_QY];
  float gqb[MAX_SEG + 1];   // age-binned dust: dlnL/dQ of each block
#pragma unroll
  for (int j = 0; j <= MAX_SEG; ++j) gqb[j] = md.n_bin > 0 ? (float)a.rgrad[(size_t)r * RGRAD + RG_QSEG + j] : 0.f;
  // dW holds values only in the columns the forward's rows touched (the
  // contraction skips the others): the second [a/Fe] node's block only when it
  // carries weight or the [a/Fe] derivative, and only (age, [Fe/H]) pairs with
  // Ws != 0 enter the [a/Fe] derivative
  const bool use_n1 = n1 != n0 && (md.use_afe || wn1 != 0.f);
  float gafe = 0.f;
  for (int j = tid; j < NA * NZ; j += blockDim.x) {
    const int ag = j / NZ, mm = j % NZ;
    const bool young = ag >= L.neb_a0 && ag < L.n_young;   // a nebular age: Q enters through it
    const int4 ac = L.age_col[ag];
    float gq = gqy;
    if (g.neb_na > 0 && md.use_neb && young)   // nebular age axis: this age's own dlnL/dQ
      gq = (float)a.rgrad[(size_t)r * RGRAD + RG_QAGE + (ag - g.neb_a0)];
    if (md.n_bin > 0) {
#pragma unroll
      for (int jj = 0; jj <= MAX_SEG; ++jj) gq = ac.z == jj ? gqb[jj] : gq;
    }
    float gv[2] = {0.f, 0.f};
    const int nn[2] = {n0, n1};
    for (int q = 0; q < (use_n1 ? 2 : 1); ++q) {
      const int k = ac.x + (nn[q] * NZ + mm) * ac.y;
      gv[q] = dW[k] + (young ? gq * L.q_s[k] : 0.f);
    }
    gWs[j] = use_n1 ? gv[0] * wn0 + gv[1] * wn1 : gv[0] * wn0;
    if (use_n1 && Ws[j] != 0.f) gafe += Ws[j] * (gv[0] * dn0 + gv[1] * dn1);
  }
  __syncthreads();
  // thread per SFH bin: dlnL/dm_i (linear scheme: d/dpsi of its two edges),
  // dlnL/dzeta_i and the edge derivatives
  if constexpr (LINEAR) {
    for (int i = tid; i < NT; i += blockDim.x) {
      const int j0 = zb[i];
      const float t = zt[i], d0 = zd0[i], d1 = zd1[i];
      const LinGrad lg = lin_bin_grad(g, T[i], T[i + 1], m[i], m[i + 1], [&](int ag, float& G, float& Gz) {
        const float g0 = gWs[ag * NZ + j0], g1 = NZ > 1 ? gWs[ag * NZ + j0 + 1] : 0.f;
        G = g0 * (1.f - t) + g1 * t;
        Gz = g0 * d0 + g1 * d1;
      });
      gps0[i] = lg.p0;
      gps1[i] = lg.p1;
      gzeta[i] = lg.zeta;
      gTlo[i] = lg.t0;
      gThi[i] = lg.t1;
    }
    __syncthreads();
    for (int k = tid; k <= NT; k += blockDim.x)
      out[md.offs[SED_KEY_SFH] + k] = (k < NT ? gps0[k] : 0.f) + (k > 0 ? gps1[k - 1] : 0.f);
  } else
  for (int i = tid; i < NT; i += blockDim.x) {
    const float Ti = T[i], Ti1 = T[i + 1], dT = Ti1 - Ti;
    // first age whose cell reaches above T_i
    int a0 = 0, a1 = NA;
    while (a0 < a1) {
      int mid = (a0 + a1) >> 1;
      if (g.cell_hi[mid] > Ti) a1 = mid; else a0 = mid + 1;
    }
    float gm = 0.f, gz = 0.f, glo = 0.f, ghi = 0.f;
    const int j0 = zb[i];
    const float t = zt[i];
    for (int ag = a0; ag < NA && g.cell_lo[ag] < Ti1; ++ag) {
      const float lo = g.cell_lo[ag], hi = g.cell_hi[ag];
      const float ov = fminf(Ti1, hi) - fmaxf(Ti, lo);
      if (ov <= 0.f) continue;
      const float A = m[i] / dT * ov;
      const float g0 = gWs[ag * NZ + j0];
      const float g1 = NZ > 1 ? gWs[ag * NZ + j0 + 1] : 0.f;
      const float gA = g0 * (1.f - t) + g1 * t;
      gz += A * (g0 * zd0[i] + g1 * zd1[i]);
      gm += gA * ov / dT;
      ghi += gA * m[i] * ((Ti1 < hi ? 1.f : 0.f) / dT - ov / (dT * dT));
      glo += gA * m[i] * (-(Ti > lo ? 1.f : 0.f) / dT + ov / (dT * dT));
    }
    out[md.offs[SED_KEY_SFH] + i] = gm;
    gzeta[i] = gz;
    gTlo[i] = glo;
    gThi[i] = ghi;
  }
  __syncthreads();
  // T_max(z) path: dT_i/dT_max = T_i (i-2) / ((N_T-2) T_max) for i >= 3
  double part = 0.0;
  const double inv_den = 1.0 / ((double)(NT - 2) * tmax);   // one FP64 division per row, not per edge
  for (int i = 3 + tid; i <= NT; i += blockDim.x) {
    const float gT = gThi[i - 1] + (i < NT ? gTlo[i] : 0.f);
    part += (double)gT * (double)T[i] * (double)(i - 2) * inv_den;
  }
  double ga = (double)gafe;
  // one [Fe/H] for every bin: its derivative sums the bins' (thread-strided,
  // then a fixed tree)
  double gzp = 0.0;
  if (md.zmode == 1)
    for (int i = tid; i < NT; i += blockDim.x) gzp += (double)gzeta[i];
  for (int o = 16; o; o >>= 1) {
    part += __shfl_xor_sync(0xffffffffu, part, o);
    ga += __shfl_xor_sync(0xffffffffu, ga, o);
    gzp += __shfl_xor_sync(0xffffffffu, gzp, o);
  }
  __shared__ double s_zeta_part[PREP_BWD_THREADS / 32];
  if (lane == 0) { s_tmax_part[warp] = part; red[warp] = ga; s_zeta_part[warp] = gzp; }
  __syncthreads();
  if (tid == 0) {
    double gtmax = 0.0, gafe_t = 0.0, gzs = 0.0;
    for (int w = 0; w < PREP_BWD_THREADS / 32; ++w) { gtmax += s_tmax_part[w]; gafe_t += red[w]; gzs += s_zeta_part[w]; }
    // a fixed key has no column in the caller's rows (and no gradient)
    auto put = [&](int key, float v) {
      if (md.offs[key] < md.n_param) out[md.offs[key]] = v;
    };
    const double* rg = a.rgrad + (size_t)r * RGRAD;
    if (md.zmode == 1) put(SED_KEY_LOGZSOL, (float)gzs);
    put(SED_KEY_AFE, md.use_afe ? (float)gafe_t : 0.f);
    put(SED_KEY_LOGMASS, (float)rg[RG_LOGMASS]);
    put(SED_KEY_ZRED, (float)(rg[RG_Z] + gtmax * (double)rs.dtmax_dz));
    put(SED_KEY_TAU_POW, (float)rg[RG_TAU_BC]);
    put(SED_KEY_ALPHA_POW, (float)rg[RG_ALPHA_BC]);
    put(SED_KEY_DIFFUSE_TAU, (float)rg[RG_TAU_D]);
    put(SED_KEY_DIFFUSE_INDEX, (float)rg[RG_DELTA]);
    put(SED_KEY_GAS_LOGZ, md.use_neb ? (float)rg[RG_GAS_LOGZ] : 0.f);
    put(SED_KEY_GAS_LOGU, md.use_neb ? (float)rg[RG_GAS_LOGU] : 0.f);
    put(SED_KEY_IGM_FACTOR, md.use_igm ? (float)rg[RG_IGM] : 0.f);
    for (int b = 0; b < md.n_bin; ++b) {   // age-binned dust: (tau_b, slope_b), never fixed
      out[md.offs[SED_KEY_DUST_BINS] + 2 * b] = (float)rg[RG_BIN + 2 * b];
      out[md.offs[SED_KEY_DUST_BINS] + 2 * b + 1] = (float)rg[RG_BIN + 2 * b + 1];
    }
    if (md.sample_sgal) put(SED_KEY_SIGMA_GAL, (float)rg[RG_SIGMA_GAL]);
    if (md.fesc_geom) put(SED_KEY_FRAC_OBRUN, (float)rg[RG_FOB]);
    if (md.gas_mode == SED_GAS_SIGMA_SAMPLED) put(SED_KEY_SIGMA_GAS, (float)rg[RG_SIGMA_GAS]);
    for (int arm = 0; arm < 2; ++arm)
      for (int k = 0; k < 4; ++k)
        if ((md.floor_bits[arm] >> k) & 1)
          put(SED_KEY_LOG_ERR_SCALE_PHOT + 4 * arm + k, (float)rg[RG_FLOOR + 4 * arm + k]);
  }
  if (md.zmode == 0)
    for (int i = tid; i < NT; i += blockDim.x) out[md.offs[SED_KEY_LOGZSOL] + i] = gzeta[i];
  for (int j = md.n_param + tid; j < a.ld; j += blockDim.x) out[j] = 0.f;
}

cudaError_t launch_prep_bwd(const PrepBwdArgs& p, cudaStream_t s) {
  const size_t smem = (size_t)2 * p.g.n_age * p.g.n_feh * sizeof(float);
  static DynSmemCache set_for;
  static DynSmemCache set_for_lin;
  if (p.md.sfh_linear) {
    const cudaError_t e = ensure_dyn_smem(k_prep_bwd<true>, smem, &set_for_lin);
    if (e != cudaSuccess) return e;
    return launch_pdl(k_prep_bwd<true>, dim3(p.n), dim3(PREP_BWD_THREADS), smem, s, p);
  }
  const cudaError_t e = ensure_dyn_smem(k_prep_bwd<false>, smem, &set_for);
  if (e != cudaSuccess) return e;
  return launch_pdl(k_prep_bwd<false>, dim3(p.n), dim3(PREP_BWD_THREADS), smem, s, p);
}

cudaError_t launch_prep(const PrepArgs& p, cudaStream_t s) {
  cudaError_t e = cudaSuccess;
  // a fixed redshift (no column) needs no redshift order: the caller's order is kept
  const bool z_col = p.md.offs[SED_KEY_ZRED] < p.md.n_param;
  const int mt = (p.n + 127) / 128;
  // a small single-fit launch without K-tile masks orders itself; its windows
  // start empty because the last kernel of every call that filled them (the
  // epilogue) empties them again, and the workspace starts them empty
  const bool self = p.self_order && z_col && !p.row_model && !p.kmask && p.n <= SELF_ORDER_MAX;
  const bool order = !self && p.perm && (p.row_model || z_col);
  if (!order && !self) {   // no ordering kernel to start the windows and masks empty
    if (p.tile_win) {
      e = cudaMemsetAsync(p.tile_win, 0x7f, mt * sizeof(int), s);
      if (e == cudaSuccess) e = cudaMemsetAsync(p.tile_win + mt, 0xff, mt * sizeof(int), s);
    }
    if (e == cudaSuccess && p.kmask) e = cudaMemsetAsync(p.kmask, 0, (size_t)mt * p.kmask_w * sizeof(uint32_t), s);
    if (e != cudaSuccess) return e;
  }
  if (order) {
    OrderArgs oa;
    oa.theta = p.theta; oa.n = p.n; oa.ld = p.ld; oa.perm = p.perm; oa.md = p.md;
    oa.mtab = p.mtab; oa.row_model = p.row_model;
    // bracket pair major when the contraction skips K tiles (the host gives
    // masks only to models with one [Fe/H], and [a/Fe], per row)
    const int pairs = std::max(p.md.n_feh - 1, 1) * (p.md.use_afe ? std::max(p.md.n_afe - 1, 1) : 1);
    oa.by_pair = !p.row_model && p.kmask && pairs > 1 && pairs <= ORDER_BINS / 4;
    oa.n_pairs = pairs;
    oa.tile_win = p.tile_win;
    oa.kmask = p.kmask;
    oa.mt = mt;
    oa.kmask_w = p.kmask ? p.kmask_w : 0;
    e = launch_pdl(k_order, dim3((p.n + ORDER_CHUNK - 1) / ORDER_CHUNK), dim3(ORDER_THREADS), 0, s, oa);
    if (e != cudaSuccess) return e;
  }
  PrepKernelArgs ka;
  ka.p = p;
  ka.p.self_order = self ? 1 : 0;
  if (self || (!p.row_model && !z_col)) ka.p.perm = nullptr;
  // Ws [n_age][n_feh], the FP8 row scratch, the row's parameters (n_param <= ld
  // and n_param <= 2 MAX_SFH + SED_NKEYS + 2 MAX_DUST_BIN for every model)
  // (+ the fixed keys' values past the caller's columns)
  const size_t npar = (size_t)std::min(p.ld, 2 * MAX_SFH + SED_NKEYS + 2 * MAX_DUST_BIN) + SED_NKEYS;
  const size_t smem = ((size_t)p.g.n_age * p.g.n_feh + (p.W_f8 ? (size_t)p.L.Kpad : 0) + npar) * sizeof(float);
  static DynSmemCache set_for[2];
  e = p.row_model ? ensure_dyn_smem(k_prep<true>, smem, &set_for[1]) : ensure_dyn_smem(k_prep<false>, smem, &set_for[0]);
  if (e != cudaSuccess) return e;
  return p.row_model ? launch_pdl(k_prep<true>, dim3(p.n), dim3(PREP_THREADS), smem, s, ka)
                     : launch_pdl(k_prep<false>, dim3(p.n), dim3(PREP_THREADS), smem, s, ka);
}

}  // namespace sed
