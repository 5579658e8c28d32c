// Marginalised calibration polynomial (App. E, Eq. app_polymarg), shared by
// the forward epilogue and its adjoint.  The spectrum's model is
// mu_i (1 + sum_m c_m T_m(x_i)) with c ~ N(0, diag(s_m^2)); integrating c out,
//   lnL += b^T M^-1 b / 2 - ln|M| / 2 - ln|Lambda| / 2,
//   M_ab = sum_i w_i mu_i^2 T_a(x_i) T_b(x_i) + delta_ab / s_a^2,
//   b_a  = sum_i w_i mu_i r_i T_a(x_i),   w_i = 1/sigma_i^2,  r_i = d_i - mu_i,
// over the included pixels.  With T_a T_b = (T_{a+b} + T_{|a-b|}) / 2 the
// Gram matrix needs only the 2n-1 moments S_k = sum_i w_i mu_i^2 T_k(x_i).
//
// The kernels evaluate it through the equivalent form at the optimum
// c* = M^-1 b (ridge least squares):
//   lnL_diag(r) + b^T M^-1 b / 2 = sum_i -((r_i - mu_i p_i) / sigma_i)^2 / 2 + const
//                                  - c*^T Lambda^-1 c* / 2,   p_i = sum_m c*_m T_m(x_i),
// which is stationary in c*, so rounding in c* enters lnL only at second
// order; the gradient takes c* at first order.  Everything runs in FP32 on the
// normalised values m_i = mu_i/sigma_i and r_i/sigma_i (of the order of the
// S/N; GB300 issues FP64 at a small fraction of the FP32 rate): c* from the
// FP32 moments, then one step of iterative refinement whose residual
//   b - M c = sum_i T(x_i) m_i (r_i/sigma_i - m_i p_i) - Lambda^-1 c
// is summed pixel by pixel, from each pixel's calibrated residual, so that it
// carries no rounding of M (which the condition number of M would amplify).
#pragma once
#include "sed_internal.cuh"

namespace sed {

constexpr int CAL_NS = 2 * SED_MAX_CALIB - 1;   // moments S_k
constexpr int CAL_NV = CAL_NS + SED_MAX_CALIB;  // S_k then b_a (or the refinement residual)

// One pixel's share of a block of NK consecutive sums: moments k = K0 .. K0+NK-1
// of coef * T_k(x), up to k < kmax.  The sums are taken in blocks of
// SED_MAX_CALIB to keep few of them live at a time.
template <int K0, int NK>
__device__ __forceinline__ void calib_accumulate(float x, float coef, int kmax, float (&v)[NK]) {
  float tp = 1.f, tc = x;   // T_{k-1}, T_k for k = 1
  if (K0 == 0) v[0] += coef;
#pragma unroll
  for (int k = 1; k < K0 + NK; ++k) {
    if (k >= K0 && k < kmax) v[k - K0] += coef * tc;
    const float tn = 2.f * x * tc - tp;
    tp = tc;
    tc = tn;
  }
}

// p = sum_m c_m T_m(x) for one pixel (n terms)
__device__ __forceinline__ float calib_poly(const float* c, int n, float x) {
  float p = c[0], tp = 1.f, tc = x;
#pragma unroll
  for (int a = 1; a < SED_MAX_CALIB; ++a) {
    if (a < n) p = fmaf(c[a], tc, p);
    const float tn = 2.f * x * tc - tp;
    tp = tc;
    tc = tn;
  }
  return p;
}

// One block of calibration sums over the thread's own pixels, from m_i in ms_s
// (0 for an excluded pixel) and the normalised datum d_i/sigma_i:
//   B = 0: the moments S_K0 .. S_K0+12 of m^2,
//   B = 1: the vector b of m r/sigma,
//   B = 2: the refinement's pixel sums of m (r/sigma - m p), p from c.
// Per-warp FP32 totals into part[warp][...] (B > 0: from index CAL_NS).
template <int K0, int B, int NT>
__device__ __forceinline__ void calib_block(const ModelDev& md, const float* ms_s, const float* c, int tid,
                                            int lane, int warp, float* part) {
  constexpr int NK = SED_MAX_CALIB;
  float v[NK];
#pragma unroll
  for (int q = 0; q < NK; ++q) v[q] = 0.f;
  const int n = md.calib_n;
  const int kmax = B ? n : 2 * n - 1;
  for (int i = tid; i < md.n_pix; i += NT) {
    const float m = ms_s[i];
    if (m == 0.f) continue;
    const float x = md.pix_cx[i];
    float coef;
    if (B == 0) coef = m * m;
    else if (B == 1) coef = m * (md.spec_dn[i] - m);
    else coef = m * fmaf(-m, calib_poly(c, n, x), md.spec_dn[i] - m);
    calib_accumulate<K0, NK>(x, coef, kmax, v);
  }
  const int base = B ? CAL_NS : K0;
#pragma unroll
  for (int q = 0; q < NK; ++q) {
    if (base + q >= (B ? CAL_NV : CAL_NS)) break;
    float x = v[q];
#pragma unroll
    for (int o = 16; o; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if (lane == 0) part[warp * CAL_NV + base + q] = x;
  }
}

// The small solves run on one warp, lane i owning row i of M (n <= 13 <= 32),
// the matrix in shared memory.  They run once per row between long phases of
// other code, so they are written as short runtime loops (a fully unrolled
// form measured several times slower there, fetching its instructions cold):
// the Cholesky factor is left-looking, one column per step with a dot product
// per lane, one reciprocal square root and a warp barrier; the inverse
// diagonal is kept so that the substitutions only multiply; ln|M| comes from
// the pivots at the end, one logarithm per lane.  All 32 lanes of the warp
// must call them together.

// Sum of the per-warp partials into row 0, in warp order, of entries [q0, q1).
__device__ __forceinline__ void calib_sum_warps(float* part, int nwarps, int q0, int q1, int lane) {
  for (int q = q0 + lane; q < q1; q += 32) {
    float v = part[q];
    for (int w = 1; w < nwarps; ++w) v += part[w * CAL_NV + q];
    part[q] = v;
  }
  __syncwarp();
}

// M from the moments S (row 0 of the partials), factored into its Cholesky
// factor L, written to the lower triangle of the row-major n x n array L, and
// 1/L_ii to Dinv.  Returns -ln|M| / 2 - ln|Lambda| / 2 (0 for the optimised
// polynomial, which has no Occam terms), or NaN when M is not positive
// definite (every lane).
static __device__ __noinline__ double calib_factor(const ModelDev& md, const float* S, float* L, float* Dinv, int lane) {
  const int n = md.calib_n, i = lane;
  if (i < n) {
    const float isg = (float)md.calib_isig2[i];
    for (int k = 0; k <= i; ++k) L[i * n + k] = 0.5f * (S[i + k] + S[i - k]) + (i == k ? isg : 0.f);
  }
  __syncwarp();
  float dii = 1.f, iii = 1.f;   // this lane's pivot L_ii^2 and 1/L_ii
  for (int j = 0; j < n; ++j) {
    // s_i = M_ij - sum_{k<j} L_ik L_jk for the rows i >= j
    float s = 0.f;
    if (i >= j && i < n) {
      s = L[i * n + j];
      for (int k = 0; k < j; ++k) s = fmaf(-L[i * n + k], L[j * n + k], s);
    }
    const float d = __shfl_sync(0xffffffffu, s, j);
    const float inv = rsqrtf(d);
    if (i == j) { dii = d; iii = inv; }
    if (i >= j && i < n) L[i * n + j] = i == j ? d * inv : s * inv;
    __syncwarp();
  }
  if (i < n) Dinv[i] = iii;
  float lg = i < n ? logf(dii) : 0.f;   // ln L_ii^2
  int bad = i < n && !(dii > 0.f);
  for (int o = 16; o; o >>= 1) {
    lg += __shfl_xor_sync(0xffffffffu, lg, o);
    bad |= __shfl_xor_sync(0xffffffffu, bad, o);
  }
  __syncwarp();
  if (bad) return (double)NAN;
  return md.calib_opt ? 0.0 : -0.5 * (double)lg - 0.5 * md.calib_logdet_lam;
}

// x = (L L^T)^-1 rhs with rhs_i in lane i; returns x_i in lane i (0 for i >= n).
static __device__ __noinline__ float calib_subst(const float* L, const float* Dinv, int n, float rhs, int lane) {
  const int i = lane;
  const float di = i < n ? Dinv[i] : 0.f;
  float v = rhs, y = 0.f;   // forward: L y = rhs
  for (int k = 0; k < n; ++k) {
    const float yk = __shfl_sync(0xffffffffu, v * di, k);
    if (i == k) y = yk;
    if (i > k && i < n) v = fmaf(-L[i * n + k], yk, v);
  }
  float w = y, x = 0.f;     // back: L^T x = y
  for (int k = n - 1; k >= 0; --k) {
    const float xk = __shfl_sync(0xffffffffu, w * di, k);
    if (i == k) x = xk;
    if (i < k) w = fmaf(-L[k * n + i], xk, w);
  }
  return i < n ? x : 0.f;
}

// c* from the first solve: the moments summed, M factored, c = M^-1 b written
// to c; returns the calib_factor value (every lane).
__device__ inline double calib_first_solve(const ModelDev& md, float* part, int nwarps, float* L, float* Dinv,
                                           float* c, int lane) {
  const int n = md.calib_n;
  calib_sum_warps(part, nwarps, 0, CAL_NV, lane);
  const double f = calib_factor(md, part, L, Dinv, lane);
  const float x = calib_subst(L, Dinv, n, lane < n ? part[CAL_NS + lane] : 0.f, lane);
  if (lane < n) c[lane] = x;
  __syncwarp();
  return f;
}

// The refinement: residual b - M c from the pixel sums (partials from index
// CAL_NS) minus Lambda^-1 c, its correction added to c, and the prior term
// -c^T Lambda^-1 c / 2 of the refined c returned (every lane).
__device__ inline double calib_refine(const ModelDev& md, float* part, int nwarps, const float* L,
                                      const float* Dinv, float* c, int lane) {
  const int n = md.calib_n;
  calib_sum_warps(part, nwarps, CAL_NS, CAL_NV, lane);
  const float isg = lane < n ? (float)md.calib_isig2[lane] : 0.f;
  const float ca = lane < n ? c[lane] : 0.f;
  const float r = lane < n ? fmaf(-isg, ca, part[CAL_NS + lane]) : 0.f;
  const float cn = ca + calib_subst(L, Dinv, n, r, lane);
  if (lane < n) c[lane] = cn;
  float pr = cn * cn * isg;
#pragma unroll
  for (int o = 16; o; o >>= 1) pr += __shfl_xor_sync(0xffffffffu, pr, o);
  __syncwarp();
  return -0.5 * (double)pr;
}

// one included pixel's change of its diagonal lnL term under the calibration,
// ((r/sigma)^2 - ((r - mu p)/sigma)^2) / 2 = m p (r/sigma - m p / 2), m = mu/sigma,
// from rn = r/sigma
__device__ __forceinline__ float calib_pixel_term(float rn, float m, float p) {
  const float mp = m * p;
  return mp * fmaf(-0.5f, mp, rn);
}

}  // namespace sed
