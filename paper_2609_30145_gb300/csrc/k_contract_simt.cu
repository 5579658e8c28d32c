// CUDA-core FP32 contraction (precision SED_PREC_FP32_SIMT): the weighted sum
// of Eq. csp_sum_main evaluated separately over the young (birth-cloud) and the
// old K blocks, Y = W[:, young] SSP[young, :], O = W[:, old] SSP[old, :]
// (Eq. app_attn with the two-bin age split), the young part per attenuated
// block with age-binned dust.  Plain register-tiled SGEMM,
// 128x128 tile, 8x8 outputs per thread.  Kept as an independent FFMA
// cross-check of the tensor-core paths.
#include "sed_internal.cuh"

namespace sed {

constexpr int SB_M = 128, SB_N = 128, SB_K = 8;

__global__ void __launch_bounds__(256) k_contract_simt(const ContractArgs a) {
  pdl_enter();
  __shared__ __align__(16) float As[SB_K][SB_M];
  __shared__ __align__(16) float Bs[SB_K][SB_N];
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int m0 = blockIdx.y * SB_M, n0 = blockIdx.x * SB_N;
  const int lrow = tid >> 1, lk = (tid & 1) * 4;
  // skip wavelength tiles outside the union of the tile's row windows
  if (a.rs) {
    __shared__ int s_klo, s_khi;
    if (tid == 0) { s_klo = 0x7fffffff; s_khi = -1; }
    __syncthreads();
    if (tid < SB_M && m0 + tid < a.n) {
      const RowScal& q = a.rs[m0 + tid];
      if (q.status == 0) { atomicMin(&s_klo, q.k_lo); atomicMax(&s_khi, q.k_hi); }
    }
    __syncthreads();
    if (s_khi < 0 || n0 > s_khi || n0 + SB_N - 1 < s_klo) return;
  }

  // the attenuated blocks of the young part (one without age-binned dust), then the old part
  const int nseg = a.n_seg > 0 ? a.n_seg : 1;
  for (int part = 0; part <= nseg; ++part) {
    const bool old = part == nseg;
    const int kb = old ? a.Ky_pad : (part == 0 ? 0 : a.seg_k0[part]);
    const int ke = old ? a.Kpad : (part + 1 == nseg ? a.Ky_pad : a.seg_k0[part + 1]);
    float acc[8][8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;

    for (int k0 = kb; k0 < ke; k0 += SB_K) {
      float4 va = make_float4(0.f, 0.f, 0.f, 0.f), vb = va;
      if (m0 + lrow < a.n)
        va = *reinterpret_cast<const float4*>(a.W + (size_t)(m0 + lrow) * a.Kpad + k0 + lk);
      if (n0 + lrow < a.n_lam)
        vb = *reinterpret_cast<const float4*>(a.sspT + (size_t)(n0 + lrow) * a.Kpad + k0 + lk);
      As[lk + 0][lrow] = va.x; As[lk + 1][lrow] = va.y; As[lk + 2][lrow] = va.z; As[lk + 3][lrow] = va.w;
      Bs[lk + 0][lrow] = vb.x; Bs[lk + 1][lrow] = vb.y; Bs[lk + 2][lrow] = vb.z; Bs[lk + 3][lrow] = vb.w;
      __syncthreads();
#pragma unroll
      for (int kk = 0; kk < SB_K; ++kk) {
        const float4 a0 = *reinterpret_cast<const float4*>(&As[kk][ty * 4]);
        const float4 a1 = *reinterpret_cast<const float4*>(&As[kk][ty * 4 + 64]);
        const float4 b0 = *reinterpret_cast<const float4*>(&Bs[kk][tx * 4]);
        const float4 b1 = *reinterpret_cast<const float4*>(&Bs[kk][tx * 4 + 64]);
        const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
        const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
          for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
      }
      __syncthreads();
    }
    float* out = old ? a.O : a.Y + part * a.seg_stride;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int gm = m0 + ty * 4 + (i & 3) + (i >> 2) * 64;
      if (gm >= a.n) continue;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int gn = n0 + tx * 4 + h * 64;
        if (gn >= a.ldn) continue;
        *reinterpret_cast<float4*>(out + (size_t)gm * a.ldn + gn) =
            make_float4(acc[i][h * 4 + 0], acc[i][h * 4 + 1], acc[i][h * 4 + 2], acc[i][h * 4 + 3]);
      }
    }
  }
}

cudaError_t launch_contract_simt(const ContractArgs& a, cudaStream_t s) {
  dim3 grid((a.ldn + SB_N - 1) / SB_N, (a.n + SB_M - 1) / SB_M);
  return launch_pdl(k_contract_simt, grid, dim3(256), 0, s, a);
}

}  // namespace sed
