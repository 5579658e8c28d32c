// Nested slice sampling (Sec. 4.3) on the GPU, around sed_loglike.
//
// Nested sampling (Skilling 2006) keeps n live points drawn from the prior
// inside a rising likelihood contour.  Each iteration here removes the k live
// points of lowest lnL, adds them to the evidence sum, and replaces them by k
// hit-and-run slice chains run side by side: a chain starts at a random
// surviving live point above the contour and makes a fixed number of slice
// steps (Neal 2003: a bracket placed at random around the point, stepped out
// until both ends leave the contour, then shrunk towards the point until a
// proposal lands inside) along directions drawn from the surviving live
// points' covariance.  All chains advance together in rounds: a round kernel
// consumes the last round's likelihoods, moves every chain's state machine on
// to its next proposal and writes the proposals as parameter rows, and one
// sed_loglike call evaluates them.  Proposals that leave the unit cube of the
// box prior are outside the contour without an evaluation.
//
// Prior volume: removing the j-th lowest of n live points shrinks the volume
// by exp(-1 / (n - j)), the expectation of its log shrinkage; the removed
// point's weight is the volume it leaves behind.  Evidence and information
// are accumulated in FP64 by one thread in removal order (Skilling's
// recurrence for H), so a run is deterministic for a given seed.
#include <math.h>
#include <string.h>

#include <vector>

#include "sed_internal.cuh"

using namespace sed;

namespace {

constexpr int NSS_MAX_D = 1024;      // parameter columns of a row
constexpr int NSS_FULL_COV = 128;    // full covariance up to this many columns, its diagonal above
constexpr int NSS_MAX_LIVE = 4096;
constexpr int MAXOUT = 16;           // stepping-out moves per side and slice step
constexpr int MAXSHRINK = 48;        // shrinking proposals per slice step (then the step keeps its point)
constexpr int ROUNDS = 16;           // rounds queued between two checks by the host
constexpr int CHAINS_PER_BLOCK = 4;  // one warp per chain

enum Phase : int { PH_NEW = 0, PH_LEFT = 1, PH_RIGHT = 2, PH_SHRINK = 3, PH_DONE = 4 };
enum Tag : uint32_t { TAG_INIT = 1, TAG_START = 2, TAG_DIR = 3, TAG_SLICE = 4 };

struct NssState {
  double lnX, lnZ, H, lstar;
  unsigned long long n_like;
  int n_dead, stop, n_above, pad;
  int active[2];
};

struct Chains {
  float* x0;        // [k][d] current point (unit cube)
  float* v;         // [k][d] direction of the current slice step
  double* lnl0;     // [k] lnL at x0
  float *tL, *tR, *t;
  int *phase, *step, *nl, *nr, *ns, *pend;
  uint32_t* draw;   // per-chain counter of random draws within the iteration
};

struct Live {
  float* U;         // [n][d] unit-cube coordinates
  float* TH;        // [n][d] parameter rows
  double* lnl;      // [n]
  int* order;       // [n] indices in increasing lnL (ties by index)
};

struct Dead {
  float* TH;        // [cap][d]
  double* lnl;      // [cap]
  double* lnw;      // [cap] ln prior weight, turned into the ln posterior weight at the end
  int* rank;        // [cap] insertion ranks
  int cap;
};

// ---- Philox4x32-10 (Salmon, Moraes, Dror & Shaw 2011), counter -> 4 words
__device__ __forceinline__ uint4 philox(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return c;
}
// uniform in (0, 1) from the top 24 bits
__device__ __forceinline__ float u01(uint32_t x) { return ((float)(x >> 8) + 0.5f) * (1.0f / 16777216.0f); }

__device__ __forceinline__ double lae(double a, double b) {   // ln(e^a + e^b)
  if (a == -INFINITY) return b;
  if (b == -INFINITY) return a;
  const double m = fmax(a, b);
  return m + log1p(exp(-fabs(a - b)));
}

// Skilling's update of ln Z and H for one removed point of weight ln w.
__device__ __forceinline__ void add_point(NssState* st, double lnl, double lnw) {
  if (lnl == -INFINITY) return;
  const double lz = lae(st->lnZ, lnw + lnl);
  const double h = exp(lnw + lnl - lz) * lnl + (st->lnZ == -INFINITY ? 0.0 : exp(st->lnZ - lz) * (st->H + st->lnZ)) - lz;
  st->H = h;
  st->lnZ = lz;
}

__global__ void k_nss_init(int n, int d, const double* lo, const double* hi, Live lv, NssState* st, uint32_t k0,
                           uint32_t k1) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0) {
    st->lnX = 0.0; st->lnZ = -INFINITY; st->H = 0.0; st->lstar = -INFINITY;
    st->n_like = 0; st->n_dead = 0; st->stop = 0; st->n_above = 0;
    st->active[0] = st->active[1] = 0;
  }
  if (i >= n * d) return;
  const int p = i / d, j = i - p * d;
  const uint4 r = philox(make_uint4((uint32_t)p, (uint32_t)(j >> 2), 0u, TAG_INIT), k0, k1);
  const uint32_t w = (j & 3) == 0 ? r.x : (j & 3) == 1 ? r.y : (j & 3) == 2 ? r.z : r.w;
  const float u = u01(w);
  lv.U[i] = u;
  lv.TH[i] = (float)(lo[j] + (double)u * (hi[j] - lo[j]));
}

// Ranks of lnL (ascending, ties broken by index) into ord[], one CTA.
__device__ void rank_live(int n, const double* lnl_s, int* ord) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double a = lnl_s[i];
    int r = 0;
    for (int j = 0; j < n; ++j) {
      const double b = lnl_s[j];
      r += (b < a) || (b == a && j < i);
    }
    ord[r] = i;
  }
}

// One CTA: remove the k lowest live points (evidence, dead records), start the
// chains, and factor the survivors' covariance for the directions.
__global__ void __launch_bounds__(1024) k_nss_select(int n, int k, int d, int iter, Live lv, Dead dd, Chains ch,
                                                     float* chol, NssState* st, uint32_t k0, uint32_t k1) {
  extern __shared__ __align__(16) uint8_t smem[];
  double* lnl_s = reinterpret_cast<double*>(smem);
  int* ord = reinterpret_cast<int*>(lnl_s + n);
  float* mu = reinterpret_cast<float*>(ord + n);
  float* A = mu + d;                          // [d][d] covariance, then its Cholesky factor (full mode)
  __shared__ int s_above, s_nd0;
  const bool full = d <= NSS_FULL_COV;
  const int tid = threadIdx.x;
  for (int i = tid; i < n; i += blockDim.x) lnl_s[i] = lv.lnl[i];
  if (tid == 0) {
    s_above = 0;
    s_nd0 = st->n_dead;
    st->active[0] = st->active[1] = 0;
  }
  __syncthreads();
  rank_live(n, lnl_s, ord);
  __syncthreads();
  const double lstar = lnl_s[ord[k - 1]];
  int cnt = 0;
  for (int i = tid; i < n; i += blockDim.x) cnt += lnl_s[i] > lstar;
  cnt = __reduce_add_sync(0xffffffffu, cnt);
  if ((tid & 31) == 0 && cnt) atomicAdd(&s_above, cnt);
  for (int i = tid; i < n; i += blockDim.x) lv.order[i] = ord[i];
  __syncthreads();
  const int n_above = s_above;
  const int nd0 = s_nd0;
  // dead records: the removed rows, in increasing lnL
  for (int q = tid; q < k * d; q += blockDim.x) {
    const int j = q / d, c = q - j * d;
    if (nd0 + j < dd.cap) dd.TH[(size_t)(nd0 + j) * d + c] = lv.TH[(size_t)ord[j] * d + c];
  }
  if (tid == 0) {
    double lnX = st->lnX;
    for (int j = 0; j < k; ++j) {
      const double step = 1.0 / (double)(n - j);
      const double lnw = lnX + log(-expm1(-step));
      lnX -= step;
      const double l = lnl_s[ord[j]];
      add_point(st, l, lnw);
      if (nd0 + j < dd.cap) {
        dd.lnl[nd0 + j] = l;
        dd.lnw[nd0 + j] = lnw;
      }
    }
    st->lnX = lnX;
    st->lstar = lstar;
    st->n_above = n_above;
    st->n_dead = nd0 + k;
    if (n_above == 0) st->stop = 2;   // every survivor sits on the contour: nothing left to climb
  }
  // chains: start at a random survivor strictly above the contour
  for (int c = tid; c < k; c += blockDim.x) {
    const uint4 r = philox(make_uint4((uint32_t)iter, (uint32_t)c, 0u, TAG_START), k0, k1);
    int src = ord[n - 1];
    if (n_above > 0) src = ord[n - n_above + min((int)(u01(r.x) * n_above), n_above - 1)];
    ch.lnl0[c] = lnl_s[src];
    ch.phase[c] = n_above > 0 ? PH_NEW : PH_DONE;
    ch.step[c] = 0; ch.pend[c] = 0; ch.draw[c] = 0;
    ch.nl[c] = 0; ch.nr[c] = 0; ch.ns[c] = 0;
  }
  for (int q = tid; q < k * d; q += blockDim.x) {
    const int c = q / d, j = q - c * d;
    const uint4 r = philox(make_uint4((uint32_t)iter, (uint32_t)c, 0u, TAG_START), k0, k1);
    int src = ord[n - 1];
    if (n_above > 0) src = ord[n - n_above + min((int)(u01(r.x) * n_above), n_above - 1)];
    ch.x0[q] = lv.U[(size_t)src * d + j];
  }
  // covariance of the survivors (all live points but the k removed), unit-cube coordinates
  const int m = n - k;
  for (int j = tid; j < d; j += blockDim.x) {
    float s = 0.f;
    for (int q = 0; q < m; ++q) s += lv.U[(size_t)ord[k + q] * d + j];
    mu[j] = s / (float)m;
  }
  __syncthreads();
  const float inv = 1.f / (float)max(m - 1, 1);
  if (!full) {
    for (int j = tid; j < d; j += blockDim.x) {
      float s = 0.f;
      for (int q = 0; q < m; ++q) {
        const float x = lv.U[(size_t)ord[k + q] * d + j] - mu[j];
        s = fmaf(x, x, s);
      }
      chol[j] = sqrtf(s * inv + 1e-14f);
    }
    return;
  }
  for (int e = tid; e < d * d; e += blockDim.x) {
    const int i = e / d, j = e - i * d;
    if (j > i) continue;
    float s = 0.f;
    for (int q = 0; q < m; ++q) {
      const float* u = lv.U + (size_t)ord[k + q] * d;
      s = fmaf(u[i] - mu[i], u[j] - mu[j], s);
    }
    A[i * d + j] = s * inv;
  }
  __syncthreads();
  for (int j = tid; j < d; j += blockDim.x) mu[j] = A[j * d + j];   // the variances, for the pivot floor
  __syncthreads();
  // right-looking Cholesky in shared memory; a pivot below 1e-7 of its column's
  // variance (a direction the survivors do not span) is raised to that floor
  for (int j = 0; j < d; ++j) {
    if (tid == 0) {
      const float a = A[j * d + j];
      A[j * d + j] = sqrtf(fmaxf(a, 1e-7f * mu[j] + 1e-14f));
    }
    __syncthreads();
    const float pj = A[j * d + j];
    for (int i = j + 1 + tid; i < d; i += blockDim.x) A[i * d + j] /= pj;
    __syncthreads();
    const int rem = d - j - 1;
    for (int e = tid; e < rem * rem; e += blockDim.x) {
      const int i = j + 1 + e / rem, p = j + 1 + e % rem;
      if (p <= i) A[i * d + p] -= A[i * d + j] * A[p * d + j];
    }
    __syncthreads();
  }
  for (int e = tid; e < d * d; e += blockDim.x) {
    const int i = e / d, j = e - i * d;
    chol[e] = j <= i ? A[e] : 0.f;
  }
}

struct RoundArgs {
  int k, d, m_steps, round, iter;
  float w;
  const double *lo, *hi;
  const float* chol;       // [d][d] lower factor (full) or [d] standard deviations
  int full;
  Chains ch;
  const double* lnl_b;     // [k] last round's lnL
  const uint32_t* st_b;    // [k] last round's row status
  float* th_b;             // [k][d] this round's proposals
  NssState* st;
  uint32_t k0, k1;
};

__device__ __forceinline__ void write_row(const RoundArgs& a, int c, const float* x, int lane) {
  for (int j = lane; j < a.d; j += 32)
    a.th_b[(size_t)c * a.d + j] = (float)(a.lo[j] + (double)x[j] * (a.hi[j] - a.lo[j]));
}

// One warp per chain: consume the chain's last likelihood, advance its slice
// state machine to its next proposal (proposals outside the unit cube are
// decided without an evaluation) and write it as a parameter row.
__global__ void __launch_bounds__(CHAINS_PER_BLOCK * 32) k_nss_round(RoundArgs a) {
  extern __shared__ float zsh[];                       // [CHAINS_PER_BLOCK][d] normals, then x
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int c = blockIdx.x * CHAINS_PER_BLOCK + warp;
  if (blockIdx.x == 0 && threadIdx.x == 0) a.st->active[(a.round + 1) & 1] = 0;
  if (c >= a.k) return;
  float* z = zsh + (size_t)warp * 2 * a.d;
  float* x = z + a.d;
  const int d = a.d;
  float* x0 = a.ch.x0 + (size_t)c * d;
  float* v = a.ch.v + (size_t)c * d;
  int ph = a.ch.phase[c], s = a.ch.step[c], nl = a.ch.nl[c], nr = a.ch.nr[c], ns = a.ch.ns[c];
  float tL = a.ch.tL[c], tR = a.ch.tR[c], t = a.ch.t[c];
  uint32_t draw = a.ch.draw[c];
  const double lstar = a.st->lstar;
  bool have = a.ch.pend[c] != 0;
  double lc = have ? a.lnl_b[c] : -INFINITY;
  bool inside = have && a.st_b[c] == 0 && lc > lstar;
  bool wrote = false;
  for (int it = 0; it < 4 * (2 * MAXOUT + MAXSHRINK) && ph != PH_DONE; ++it) {
    if (have) {   // the outcome of the last proposal at t
      have = false;
      if (ph == PH_LEFT) {
        if (inside && nl < MAXOUT) { tL -= a.w; ++nl; } else ph = PH_RIGHT;
      } else if (ph == PH_RIGHT) {
        if (inside && nr < MAXOUT) { tR += a.w; ++nr; } else ph = PH_SHRINK;
      } else if (ph == PH_SHRINK) {
        if (inside) {
          for (int j = lane; j < d; j += 32) x0[j] = fmaf(t, v[j], x0[j]);
          if (lane == 0) a.ch.lnl0[c] = lc;
          ++s;
          ph = PH_NEW;
        } else {
          if (t < 0.f) tL = t; else tR = t;
          if (++ns >= MAXSHRINK) { ++s; ph = PH_NEW; }
        }
      }
      __syncwarp();
    }
    if (ph == PH_NEW) {
      if (s >= a.m_steps) { ph = PH_DONE; break; }
      // direction: v = L z / |z| with z standard normal (Box-Muller on Philox words)
      float zz = 0.f;
      for (int j0 = 0; j0 < d; j0 += 128) {
        const int j = j0 + 4 * lane;
        if (j < d) {
          const uint4 r = philox(make_uint4((uint32_t)a.iter, (uint32_t)c, draw, TAG_DIR | ((uint32_t)(j >> 2) << 8)),
                                 a.k0, a.k1);
          float s0, c0, s1, c1;
          const float r0 = sqrtf(-2.f * logf(u01(r.x))), r1 = sqrtf(-2.f * logf(u01(r.z)));
          sincospif(2.f * u01(r.y), &s0, &c0);
          sincospif(2.f * u01(r.w), &s1, &c1);
          const float g[4] = {r0 * c0, r0 * s0, r1 * c1, r1 * s1};
#pragma unroll
          for (int q = 0; q < 4; ++q)
            if (j + q < d) { z[j + q] = g[q]; zz = fmaf(g[q], g[q], zz); }
        }
      }
      ++draw;
#pragma unroll
      for (int o = 16; o; o >>= 1) zz += __shfl_xor_sync(0xffffffffu, zz, o);
      const float rz = rsqrtf(zz);
      __syncwarp();
      for (int i = lane; i < d; i += 32) {
        float acc = 0.f;
        if (a.full) {
          const float* Li = a.chol + (size_t)i * d;
          for (int j = 0; j <= i; ++j) acc = fmaf(Li[j], z[j], acc);
        } else {
          acc = a.chol[i] * z[i];
        }
        v[i] = acc * rz;
      }
      const uint4 r = philox(make_uint4((uint32_t)a.iter, (uint32_t)c, draw++, TAG_SLICE), a.k0, a.k1);
      tL = -u01(r.x) * a.w;
      tR = tL + a.w;
      nl = nr = ns = 0;
      ph = PH_LEFT;
      __syncwarp();
    }
    if (ph == PH_LEFT) t = tL;
    else if (ph == PH_RIGHT) t = tR;
    else {
      const uint4 r = philox(make_uint4((uint32_t)a.iter, (uint32_t)c, draw++, TAG_SLICE), a.k0, a.k1);
      t = tL + u01(r.x) * (tR - tL);
    }
    bool out = false;
    for (int j = lane; j < d; j += 32) {
      const float xj = fmaf(t, v[j], x0[j]);
      x[j] = xj;
      out |= !(xj >= 0.f && xj <= 1.f);
    }
    out = __any_sync(0xffffffffu, out);
    __syncwarp();
    if (out) {   // outside the box prior: outside the contour, no evaluation
      have = true;
      inside = false;
      continue;
    }
    write_row(a, c, x, lane);
    wrote = true;
    break;
  }
  if (!wrote) write_row(a, c, x0, lane);   // an idle row (done chain): evaluated, not used
  if (lane == 0) {
    a.ch.phase[c] = ph; a.ch.step[c] = s; a.ch.nl[c] = nl; a.ch.nr[c] = nr; a.ch.ns[c] = ns;
    a.ch.tL[c] = tL; a.ch.tR[c] = tR; a.ch.t[c] = t; a.ch.draw[c] = draw;
    a.ch.pend[c] = wrote ? 1 : 0;
    if (wrote) atomicAdd(&a.st->n_like, 1ull);
    if (ph != PH_DONE) atomicAdd(&a.st->active[a.round & 1], 1);
  }
}

// One CTA: the chains' end points replace the removed live points; insertion
// ranks among the survivors; the stop test ln(Z_live / Z) < stop_dlnz.
__global__ void __launch_bounds__(1024) k_nss_replace(int n, int k, int d, int iter, const double* lo,
                                                      const double* hi, Live lv, Dead dd, Chains ch, NssState* st,
                                                      double stop_dlnz, int last) {
  __shared__ double red[32];
  const int tid = threadIdx.x;
  const int nd0 = st->n_dead - k;   // first dead record of this iteration
  for (int c = tid; c < k; c += blockDim.x) {
    const double l = ch.lnl0[c];
    int r = 0;
    for (int q = k; q < n; ++q) r += lv.lnl[lv.order[q]] < l;
    if (nd0 + c < dd.cap && dd.rank) dd.rank[nd0 + c] = r;
  }
  __syncthreads();
  for (int q = tid; q < k * d; q += blockDim.x) {
    const int c = q / d, j = q - c * d;
    const int slot = lv.order[c];
    const float u = ch.x0[q];
    lv.U[(size_t)slot * d + j] = u;
    lv.TH[(size_t)slot * d + j] = (float)(lo[j] + (double)u * (hi[j] - lo[j]));
  }
  for (int c = tid; c < k; c += blockDim.x) lv.lnl[lv.order[c]] = ch.lnl0[c];
  __syncthreads();
  // ln Z_live = ln X + ln(mean L_live)
  double mx = -INFINITY;
  for (int i = tid; i < n; i += blockDim.x) mx = fmax(mx, lv.lnl[i]);
#pragma unroll
  for (int o = 16; o; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((tid & 31) == 0) red[tid >> 5] = mx;
  __syncthreads();
  if (tid < 32) {
    double v = tid < (int)(blockDim.x >> 5) ? red[tid] : -INFINITY;
#pragma unroll
    for (int o = 16; o; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    if (tid == 0) red[0] = v;
  }
  __syncthreads();
  mx = red[0];
  __syncthreads();
  double sm = 0.0;
  if (mx > -INFINITY)
    for (int i = tid; i < n; i += blockDim.x) sm += exp(lv.lnl[i] - mx);
#pragma unroll
  for (int o = 16; o; o >>= 1) sm += __shfl_xor_sync(0xffffffffu, sm, o);
  if ((tid & 31) == 0) red[tid >> 5] = sm;
  __syncthreads();
  if (tid == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    const double lz_live = mx == -INFINITY ? -INFINITY : st->lnX + mx + log(t) - log((double)n);
    if (st->lnZ > -INFINITY && lz_live - st->lnZ < stop_dlnz) st->stop = 1;
    if (last && !st->stop) st->stop = 3;
  }
}

// One CTA: the final live points join the evidence (weight X / n each, in
// increasing lnL) and the records' weights become ln posterior weights.
__global__ void __launch_bounds__(1024) k_nss_final(int n, int d, Live lv, Dead dd, NssState* st) {
  extern __shared__ __align__(16) uint8_t smem[];
  double* lnl_s = reinterpret_cast<double*>(smem);
  int* ord = reinterpret_cast<int*>(lnl_s + n);
  __shared__ int s_nd0;
  const int tid = threadIdx.x;
  for (int i = tid; i < n; i += blockDim.x) lnl_s[i] = lv.lnl[i];
  if (tid == 0) s_nd0 = st->n_dead;
  __syncthreads();
  rank_live(n, lnl_s, ord);
  __syncthreads();
  const int nd0 = s_nd0;
  for (int q = tid; q < n * d; q += blockDim.x) {
    const int j = q / d, c = q - j * d;
    if (nd0 + j < dd.cap) dd.TH[(size_t)(nd0 + j) * d + c] = lv.TH[(size_t)ord[j] * d + c];
  }
  if (tid == 0) {
    const double lnw = st->lnX - log((double)n);
    for (int j = 0; j < n; ++j) {
      const double l = lnl_s[ord[j]];
      add_point(st, l, lnw);
      if (nd0 + j < dd.cap) {
        dd.lnl[nd0 + j] = l;
        dd.lnw[nd0 + j] = lnw;
      }
    }
    st->n_dead = nd0 + n;
  }
  __syncthreads();
  const double lz = st->lnZ;
  const int nrec = min(st->n_dead, dd.cap);
  for (int i = tid; i < nrec; i += blockDim.x) dd.lnw[i] = dd.lnl[i] + dd.lnw[i] - lz;
}

}  // namespace

extern "C" {

sed_status sed_nss_run(sed_ctx* ctx, sed_model_id model, const sed_nss_desc* desc, float* dead_theta,
                       double* dead_lnl, double* dead_logw, int32_t* ins_rank, int max_dead, sed_nss_result* out,
                       void* stream) {
  if (!ctx || !desc || !out) return SED_EINVAL;
  memset(out, 0, sizeof *out);
  if (model < 0 || model >= (int)ctx->models.size() || !ctx->models[model]) return SED_EINVAL;
  Model* M = ctx->models[model];
  const int d = M->dv.n_param, n = desc->n_live, k = desc->n_replace;
  if (d < 1 || d > NSS_MAX_D) return SED_EINVAL;
  if (n < 2 || n > NSS_MAX_LIVE || k < 1 || k > n / 2 || desc->n_slice_steps < 1 || desc->max_iter < 1)
    return SED_EINVAL;
  if (!desc->lo || !desc->hi || !(desc->stop_dlnz == desc->stop_dlnz) || desc->slice_width < 0.0) return SED_EINVAL;
  for (int j = 0; j < d; ++j)
    if (!(desc->lo[j] < desc->hi[j]) || !isfinite(desc->lo[j]) || !isfinite(desc->hi[j])) return SED_EINVAL;
  if (max_dead < 0) return SED_EINVAL;
  const bool want = dead_theta || dead_lnl || dead_logw || ins_rank;
  const int cap = want ? max_dead : 0;
  const bool full = d <= NSS_FULL_COV;
  int prev = -1;
  cudaGetDevice(&prev);
  cudaSetDevice(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;

  // one device allocation, carved into the run's buffers
  size_t off = 0;
  auto take = [&](size_t bytes) { const size_t o = off; off += (bytes + 255) / 256 * 256; return o; };
  const size_t o_lo = take(8 * d), o_hi = take(8 * d), o_st = take(sizeof(NssState));
  const size_t o_U = take(4ull * n * d), o_TH = take(4ull * n * d), o_lnl = take(8ull * n), o_ord = take(4ull * n);
  const size_t o_x0 = take(4ull * k * d), o_v = take(4ull * k * d), o_l0 = take(8ull * k);
  const size_t o_f = take(4ull * 3 * k), o_i = take(4ull * 7 * k);
  const size_t o_thb = take(4ull * k * d), o_lb = take(8ull * k), o_sb = take(4ull * k);
  const size_t o_ch = take(full ? 4ull * d * d : 4ull * d);
  const size_t o_dth = take(4ull * cap * d), o_dl = take(8ull * cap), o_dw = take(8ull * cap), o_dr = take(4ull * cap);
  const size_t total = off;
  if (!budget_reserve(ctx, total)) {
    cudaSetDevice(prev);
    return SED_ENOMEM;
  }
  uint8_t* base = nullptr;
  if (cudaMalloc(&base, total) != cudaSuccess) {
    budget_release(ctx, total);
    cudaSetDevice(prev);
    return SED_ENOMEM;
  }
  NssState* st_h = nullptr;
  cudaHostAlloc((void**)&st_h, sizeof(NssState), cudaHostAllocDefault);
  sed_status ret = SED_OK;
  auto F = [&](size_t o) { return base + o; };
  double* lo_d = (double*)F(o_lo);
  double* hi_d = (double*)F(o_hi);
  NssState* st = (NssState*)F(o_st);
  Live lv{(float*)F(o_U), (float*)F(o_TH), (double*)F(o_lnl), (int*)F(o_ord)};
  Chains ch{};
  ch.x0 = (float*)F(o_x0); ch.v = (float*)F(o_v); ch.lnl0 = (double*)F(o_l0);
  float* fb = (float*)F(o_f);
  ch.tL = fb; ch.tR = fb + k; ch.t = fb + 2 * k;
  int* ib = (int*)F(o_i);
  ch.phase = ib; ch.step = ib + k; ch.nl = ib + 2 * k; ch.nr = ib + 3 * k; ch.ns = ib + 4 * k; ch.pend = ib + 5 * k;
  ch.draw = (uint32_t*)(ib + 6 * k);
  float* th_b = (float*)F(o_thb);
  double* lnl_b = (double*)F(o_lb);
  uint32_t* st_b = (uint32_t*)F(o_sb);
  float* chol = (float*)F(o_ch);
  Dead dd{(float*)F(o_dth), (double*)F(o_dl), (double*)F(o_dw), (int*)F(o_dr), cap};
  const uint32_t k0 = (uint32_t)desc->seed, k1 = (uint32_t)(desc->seed >> 32);
  const float w = desc->slice_width > 0.0 ? (float)desc->slice_width : sqrtf((float)d + 2.f);
  const size_t sel_smem = 12ull * n + 4ull * d + (full ? 4ull * d * d : 0);
  const size_t fin_smem = 12ull * n;
  const size_t round_smem = 4ull * CHAINS_PER_BLOCK * 2 * d;
  static DynSmemCache a_sel, a_fin, a_round;
  const long long max_rounds = (long long)desc->n_slice_steps * (2 * MAXOUT + MAXSHRINK) + 4;
  long long n_rows = n;
  int iter = 0;
  auto CKE = [&](cudaError_t e) {
    if (e != cudaSuccess && !ret) {
      ctx->last_error = std::string("nss: ") + cudaGetErrorString(e);
      ret = SED_ECUDA;
    }
    return e == cudaSuccess;
  };
  CKE(cudaMemcpyAsync(lo_d, desc->lo, 8 * d, cudaMemcpyHostToDevice, s));
  CKE(cudaMemcpyAsync(hi_d, desc->hi, 8 * d, cudaMemcpyHostToDevice, s));
  CKE(cudaMemsetAsync(ib, 0, 4ull * 7 * k, s));
  CKE(ensure_dyn_smem(k_nss_select, sel_smem, &a_sel));
  CKE(ensure_dyn_smem(k_nss_final, fin_smem, &a_fin));
  CKE(ensure_dyn_smem(k_nss_round, round_smem, &a_round));
  if (!ret) {
    k_nss_init<<<(n * d + 255) / 256, 256, 0, s>>>(n, d, lo_d, hi_d, lv, st, k0, k1);
    CKE(cudaGetLastError());
  }
  if (!ret) ret = sed_loglike(ctx, model, lv.TH, n, d, lv.lnl, nullptr, desc->precision, stream);
  for (; !ret && iter < desc->max_iter; ++iter) {
    k_nss_select<<<1, 1024, sel_smem, s>>>(n, k, d, iter, lv, dd, ch, chol, st, k0, k1);
    if (!CKE(cudaGetLastError())) break;
    RoundArgs ra{};
    ra.k = k; ra.d = d; ra.m_steps = desc->n_slice_steps; ra.iter = iter; ra.w = w;
    ra.lo = lo_d; ra.hi = hi_d; ra.chol = chol; ra.full = full; ra.ch = ch;
    ra.lnl_b = lnl_b; ra.st_b = st_b; ra.th_b = th_b; ra.st = st; ra.k0 = k0; ra.k1 = k1;
    long long r = 0;
    bool done = false;
    while (!done && !ret) {
      for (int q = 0; q < ROUNDS && !ret; ++q, ++r) {
        ra.round = (int)(r & 1);
        k_nss_round<<<(k + CHAINS_PER_BLOCK - 1) / CHAINS_PER_BLOCK, CHAINS_PER_BLOCK * 32, round_smem, s>>>(ra);
        if (!CKE(cudaGetLastError())) break;
        ret = sed_loglike(ctx, model, th_b, k, d, lnl_b, st_b, desc->precision, stream);
        n_rows += k;
      }
      if (ret) break;
      CKE(cudaMemcpyAsync(st_h, st, sizeof(NssState), cudaMemcpyDeviceToHost, s));
      CKE(cudaStreamSynchronize(s));
      if (ret) break;
      done = st_h->active[(int)((r - 1) & 1)] == 0;
      if (!done && r > max_rounds) {
        ctx->last_error = "nss: slice chains did not finish";
        ret = SED_ECUDA;
      }
    }
    if (ret) break;
    k_nss_replace<<<1, 1024, 0, s>>>(n, k, d, iter, lo_d, hi_d, lv, dd, ch, st, desc->stop_dlnz,
                                     iter + 1 == desc->max_iter);
    CKE(cudaGetLastError());
    CKE(cudaMemcpyAsync(st_h, st, sizeof(NssState), cudaMemcpyDeviceToHost, s));
    CKE(cudaStreamSynchronize(s));
    if (!ret && st_h->stop) {
      ++iter;
      break;
    }
  }
  if (!ret) {
    k_nss_final<<<1, 1024, fin_smem, s>>>(n, d, lv, dd, st);
    CKE(cudaGetLastError());
    CKE(cudaMemcpyAsync(st_h, st, sizeof(NssState), cudaMemcpyDeviceToHost, s));
    CKE(cudaStreamSynchronize(s));
  }
  if (!ret) {
    out->lnz = st_h->lnZ;
    out->info_h = st_h->H;
    out->n_iter = iter;
    out->n_dead = st_h->n_dead;
    out->converged = st_h->stop == 1 || st_h->stop == 2;
    out->n_like = (int64_t)st_h->n_like;
    out->n_rows = n_rows;
    const int nrec = std::min(st_h->n_dead, cap);
    if (dead_theta) CKE(cudaMemcpy(dead_theta, dd.TH, 4ull * nrec * d, cudaMemcpyDeviceToHost));
    if (dead_lnl) CKE(cudaMemcpy(dead_lnl, dd.lnl, 8ull * nrec, cudaMemcpyDeviceToHost));
    if (dead_logw) CKE(cudaMemcpy(dead_logw, dd.lnw, 8ull * nrec, cudaMemcpyDeviceToHost));
    if (ins_rank) CKE(cudaMemcpy(ins_rank, dd.rank, 4ull * std::min(nrec, iter * k), cudaMemcpyDeviceToHost));
    if (!ret && want && st_h->n_dead > cap) {
      ctx->last_error = "nss: max_dead below the points of the run";
      ret = SED_ERANGE;
    }
  }
  cudaStreamSynchronize(s);
  cudaFree(base);
  budget_release(ctx, total);
  if (st_h) cudaFreeHost(st_h);
  cudaSetDevice(prev);
  return ret;
}

}  // extern "C"
