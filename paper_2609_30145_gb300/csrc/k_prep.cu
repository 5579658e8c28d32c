// Per-row preparation: cosmology, SFH edges, SSP weights, Q_young and the
// per-row scalars of the epilogue.  One CTA per parameter row.
//
//  - cosmology (Sec. 2.6): comoving distance by 32-node Gauss-Legendre in FP64
//    on u = sqrt(a) (smooth integrand 2/sqrt(Om + OL u^6)), age of the
//    Universe by its closed form, luminosity distance floored at 10 pc;
//  - SFH edges 0, 5 Myr, 10 Myr, then log-uniform to T_max = t(z) - t(zf),
//    so the grid follows the sampled redshift and the bin masses are kept
//    (Sec. 2.2, Sec. 2.6);
//  - step-scheme weights (App. B): each age node owns its linear-time Voronoi
//    cell, A_ia = m_i |bin_i ∩ cell_a| / dT_i; each bin's mass is split between
//    the two bracketing [Fe/H] nodes linearly in log Z (App. B), and over the
//    two bracketing [a/Fe] nodes (Sec. 5.4).  A thread owns one age node and
//    sums the bins overlapping its cell in order, so W is deterministic;
//  - Q_young = sum over birth-cloud ages of W Q (App. C, Eq. app_q).
#include "sed_internal.cuh"

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

struct PrepKernelArgs {
  PrepArgs p;
  double gl_x[GL_NODES];
  double gl_w[GL_NODES];
};

constexpr int PREP_THREADS = 128;

__global__ void __launch_bounds__(PREP_THREADS) k_prep(const __grid_constant__ PrepKernelArgs ka) {
  const PrepArgs& a = ka.p;
  const ModelDev& md = a.md;
  const GridDev& g = a.g;
  const LayoutDev& L = a.L;
  const int r = blockIdx.x;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const float* th = a.theta + (size_t)r * a.ld;
  const int NT = md.n_sfh, NA = g.n_age, NZ = g.n_feh;
  if (r == 0 && tid == 0 && a.err) *a.err = 0;

  extern __shared__ float smem[];
  float* Ws = smem;                     // [NA][NZ]
  __shared__ float T[MAX_SFH + 1];      // edges
  __shared__ float rate[MAX_SFH];       // m_i / dT_i
  __shared__ int zb[MAX_SFH];
  __shared__ float zt[MAX_SFH];
  __shared__ double s_cos[4];
  __shared__ float s_red[PREP_THREADS / 32];
  __shared__ int s_nnz[PREP_THREADS / 32];

  // ---- finiteness of the whole row
  int bad = 0;
  for (int j = tid; j < md.n_param; j += blockDim.x) bad |= !isfinite(th[j]);
  bad = __syncthreads_or(bad);
  const float z = th[md.offs[SED_KEY_ZRED]];
  uint32_t status = bad ? SED_ROW_BAD_THETA : 0u;
  if (!status && !(z >= 0.f && (double)z < md.zf)) status = SED_ROW_BAD_Z;

  // ---- cosmology in FP64 (warp 0)
  if (!status && warp == 0) {
    const double zp = 1.0 + (double)z;
    const double Om = md.Om0, OL = 1.0 - md.Om0;
    const double u0 = 1.0 / sqrt(zp);
    const double half = 0.5 * (1.0 - u0), mid = 0.5 * (1.0 + u0);
    double acc = 0.0;
    for (int i = lane; i < GL_NODES; i += 32) {
      double u = mid + half * ka.gl_x[i];
      double u2 = u * u;
      acc += ka.gl_w[i] * 2.0 / sqrt(Om + OL * u2 * u2 * u2);
    }
    for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) {
      const double dc = md.dh_cm * half * acc;
      const double ez = sqrt(Om * zp * zp * zp + OL);
      const double t = md.th_yr * 2.0 / (3.0 * sqrt(OL)) * asinh(sqrt(OL / Om) * pow(zp, -1.5));
      double dl = zp * dc;
      double ddl = dc + zp * md.dh_cm / ez;  // dD_L/dz
      if (dl < 10.0 * PC_CM) { dl = 10.0 * PC_CM; ddl = 0.0; }
      s_cos[0] = dl;
      s_cos[1] = t - md.t_zf_yr;                  // T_max
      s_cos[2] = ddl / dl;                        // dlnD_L/dz
      s_cos[3] = -md.th_yr / (zp * ez);           // dt/dz
    }
  }
  __syncthreads();
  const double tmax = status ? 0.0 : s_cos[1];
  if (!status && !(tmax > 1e7)) status = SED_ROW_BAD_TMAX;

  RowScal* out = a.rs + r;
  const int Kpad = L.Kpad;
  if (status) {
    for (int k = tid; k < Kpad; k += blockDim.x) {
      size_t o = (size_t)r * Kpad + k;
      if (a.W) a.W[o] = 0.f;
      if (a.W_hi) { a.W_hi[o] = 0.f; a.W_lo[o] = 0.f; }
      if (a.W_bf16) a.W_bf16[o] = __float2bfloat16_rn(0.f);
    }
    if (tid == 0) {
      RowScal rs{};
      rs.status = status;
      rs.k_lo = 0;
      rs.k_hi = 0;
      *out = rs;
    }
    return;
  }

  // ---- SFH edges (FP32) and per-bin quantities
  const float* m = th + md.offs[SED_KEY_SFH];
  const float* zeta = th + md.offs[SED_KEY_LOGZSOL];
  const float lrat = (float)log(tmax / 1e7);
  for (int i = tid; i <= NT; i += blockDim.x) {
    float v;
    if (i == 0) v = 0.f;
    else if (i == 1) v = 5e6f;
    else if (i == 2) v = 1e7f;
    else if (i == NT) v = (float)tmax;
    else v = 1e7f * expf(lrat * (float)(i - 2) / (float)(NT - 2));
    T[i] = v;
  }
  for (int j = tid; j < NA * NZ; j += blockDim.x) Ws[j] = 0.f;
  __syncthreads();
  for (int i = tid; i < NT; i += blockDim.x) {
    rate[i] = m[i] / (T[i + 1] - T[i]);
    int j0, j1;
    float w0, w1;
    bracket_f(md.feh, md.n_feh, zeta[md.zmode == 0 ? i : 0], j0, w0, j1, w1);
    zb[i] = j0;
    zt[i] = w1;   // weight of j0 + 1 (0 when n_feh == 1)
  }
  __syncthreads();

  // ---- weights on (age, feh): thread per age node
  for (int ag = tid; ag < NA; ag += blockDim.x) {
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
  __syncthreads();

  // ---- [a/Fe] split and the K-ordered row of W; Q_young
  int n0 = 0, n1 = 0;
  float wn0 = 1.f, wn1 = 0.f;
  if (md.n_afe > 1) {
    const float afe = md.use_afe ? th[md.offs[SED_KEY_AFE]] : 0.f;
    bracket_f(md.afe, md.n_afe, afe, n0, wn0, n1, wn1);
  }
  float qpart = 0.f;
  int nnz = 0;
  for (int k = tid; k < Kpad; k += blockDim.x) {
    const int code = L.k_code[k];
    float v = 0.f;
    if (code >= 0) {
      const int n = code >> 24, mm = (code >> 16) & 0xff, ag = code & 0xffff;
      const float wn = (n == n0 ? wn0 : 0.f) + (n == n1 && n1 != n0 ? wn1 : 0.f);
      v = wn * Ws[ag * NZ + mm];
    }
    if (k < L.Ky_pad) qpart += v * L.q_s[k];
    nnz += v != 0.f;
    const size_t o = (size_t)r * Kpad + k;
    if (a.W) a.W[o] = v;
    if (a.W_hi) {
      const float h = tf32_rna(v);
      a.W_hi[o] = h;
      a.W_lo[o] = v - h;
    }
    if (a.W_bf16) a.W_bf16[o] = __float2bfloat16_rn(v);
  }
  for (int o = 16; o; o >>= 1) {
    qpart += __shfl_xor_sync(0xffffffffu, qpart, o);
    nnz += __shfl_xor_sync(0xffffffffu, nnz, o);
  }
  if (lane == 0) { s_red[warp] = qpart; s_nnz[warp] = nnz; }
  __syncthreads();

  if (tid == 0) {
    float qy = 0.f;
    for (int w = 0; w < PREP_THREADS / 32; ++w) qy += s_red[w];
    const double zp = 1.0 + (double)z;
    const double logmass = (double)th[md.offs[SED_KEY_LOGMASS]];
    const double dl = s_cos[0];
    // s = 10^logmass Lsun (1+z) / (4 pi D_L^2), in device flux units (x 2^-f_log2)
    const double ls = logmass * 3.321928094887362 + log2(LSUN * zp / (4.0 * M_PI)) - 2.0 * log2(dl) - md.f_log2;
    const double s = exp2(ls);
    RowScal rs{};
    rs.p_phot = (float)(C_AA * s / (zp * zp));
    rs.s_spec = (float)s;
    rs.inv1pz = (float)(1.0 / zp);
    const double l1 = log1p((double)z);
    rs.ln1pz_hi = (float)l1;
    rs.ln1pz_lo = (float)(l1 - (double)rs.ln1pz_hi);
    rs.tau_bc = th[md.offs[SED_KEY_TAU_POW]];
    rs.alpha_bc = th[md.offs[SED_KEY_ALPHA_POW]];
    rs.tau_d = th[md.offs[SED_KEY_DIFFUSE_TAU]];
    rs.delta = th[md.offs[SED_KEY_DIFFUSE_INDEX]];
    rs.log2_qy = qy > 0.f ? log2f(qy) : -INFINITY;
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
    }
    rs.dlns_dz = (float)(1.0 / zp - 2.0 * s_cos[2]);
    rs.dlnp_dz = (float)(-1.0 / zp - 2.0 * s_cos[2]);
    rs.dtmax_dz = (float)s_cos[3];
    rs.tmax = (float)tmax;
    rs.status = 0;
    rs.k_lo = 0;
    rs.k_hi = g.n_lam;
    rs.nnz = 0;
    for (int w = 0; w < PREP_THREADS / 32; ++w) rs.nnz += s_nnz[w];
    *out = rs;
  }
}

cudaError_t launch_prep(const PrepArgs& p, cudaStream_t s) {
  static double gx[GL_NODES], gw[GL_NODES];
  static bool init = false;
  if (!init) {  // Gauss-Legendre nodes by Newton iteration on P_n
    const int n = GL_NODES;
    for (int i = 0; i < n; i++) {
      double x = cos(M_PI * (i + 0.75) / (n + 0.5)), dp = 0;
      for (int it = 0; it < 100; it++) {
        double p0 = 1.0, p1 = x;
        for (int k = 2; k <= n; k++) {
          double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
          p0 = p1; p1 = p2;
        }
        dp = n * (x * p1 - p0) / (x * x - 1.0);
        double dx = p1 / dp;
        x -= dx;
        if (fabs(dx) < 1e-16) break;
      }
      gx[i] = x;
      gw[i] = 2.0 / ((1.0 - x * x) * dp * dp);
    }
    init = true;
  }
  PrepKernelArgs ka;
  ka.p = p;
  for (int i = 0; i < GL_NODES; i++) { ka.gl_x[i] = gx[i]; ka.gl_w[i] = gw[i]; }
  const size_t smem = (size_t)p.g.n_age * p.g.n_feh * sizeof(float);
  k_prep<<<p.n, PREP_THREADS, smem, s>>>(ka);
  return cudaGetLastError();
}

}  // namespace sed
