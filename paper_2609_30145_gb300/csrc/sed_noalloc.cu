// sed_loglike_noalloc: the log-likelihood entry point for callers that must
// not have the library allocate device memory during a call.
//
// sed_loglike keeps a per-stream workspace that it grows with cudaMalloc the
// first time a stream is used or a batch outgrows it.  Some callers cannot
// accept that: a host framework that has already handed all of the GPU's
// memory to its own allocator (so a cudaMalloc from this library fails or
// fragments its pool), a sampler loop that cannot tolerate the implicit
// device synchronisation a cudaMalloc may cause in the middle of a step, or
// a deployment that must know the library's device footprint exactly at load
// time.  This entry point runs the same three kernels as sed_loglike but
// takes every intermediate buffer from one fixed array in device global
// memory, declared below, and calls no cudaMalloc, cudaFree or allocating
// library routine.
//
// The array is SED_NOALLOC_SCRATCH_BYTES long and lives for the life of the
// process on every device that loads the library.  All calls share it:
// calls whose kernels can overlap on the GPU (different streams, or
// different host threads) race on it and must be serialised by the caller.
// Each call overwrites what it uses; the one word that must start at zero
// (the device error word of the contraction) is cleared by the first kernel
// of every call.
#include <stdarg.h>
#include <stdio.h>

#include <mutex>

#include "sed_internal.cuh"

namespace {

// Scratch of sed_loglike_noalloc.  In host code this name is only a handle
// of the symbol, not a device address: the address used by the kernels is
// obtained once per device with cudaGetSymbolAddress (noalloc_scratch_ptr).
static __device__ __align__(256) unsigned char g_noalloc_scratch[SED_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_ptr[kMaxDevices] = {};

sed_status na_fail(sed_ctx* ctx, sed_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  ctx->last_error = buf;
  return st;
}

// Device address of the scratch on the current device (set up once per device).
sed_status noalloc_scratch_ptr(sed_ctx* ctx, void** out) {
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (ctx->device < 0 || ctx->device >= kMaxDevices) return na_fail(ctx, SED_ERANGE, "device index too large");
  if (!g_noalloc_ptr[ctx->device]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
      return na_fail(ctx, SED_ECUDA, "cudaGetSymbolAddress(scratch): %s", cudaGetErrorString(e));
    g_noalloc_ptr[ctx->device] = p;
  }
  *out = g_noalloc_ptr[ctx->device];
  return SED_OK;
}

size_t up256(size_t b) { return (b + 255) & ~(size_t)255; }

}  // namespace

extern "C" sed_status sed_loglike_noalloc(sed_ctx* ctx, sed_model_id id, const float* theta, int n, int ld,
                                          double* lnl_out, uint32_t* row_status, int precision, void* stream) {
  using namespace sed;
  if (!ctx) return SED_EINVAL;
  if (id < 0 || id >= (int)ctx->models.size() || !ctx->models[id]) return na_fail(ctx, SED_EINVAL, "unknown model");
  Model* M = ctx->models[id];
  if (n < 0) return na_fail(ctx, SED_EINVAL, "n < 0");
  if (n > 0 && (!theta || !lnl_out)) return na_fail(ctx, SED_EINVAL, "theta or lnl_out is NULL");
  if (ld < M->dv.n_param) return na_fail(ctx, SED_EINVAL, "ld (%d) < n_param (%d)", ld, M->dv.n_param);
  if (precision != SED_PREC_FP32 && precision != SED_PREC_FP32_SIMT && precision != SED_PREC_BF16)
    return na_fail(ctx, SED_EINVAL, "unknown precision %d", precision);
  if (precision != SED_PREC_FP32_SIMT && ctx->tc_ok != 1)
    return na_fail(ctx, SED_EUNSUPPORTED, "tensor-core precisions need an sm_103 device");
  if (n == 0) return SED_OK;

  const Grid* g = M->g;
  const Layout* L = M->L;
  const int kpad = L->Kpad;
  const int ldn = (g->n_lam + 255) / 256 * 256;
  const bool f32 = precision == SED_PREC_FP32, bf = precision == SED_PREC_BF16;
  // carve the scratch: err | RowScal | W | W_hi | W_lo | W_bf16 | Y | O
  const size_t nn = (size_t)n;
  size_t off[8], need = 0;
  const size_t sz[8] = {256, nn * sizeof(RowScal), nn * kpad * 4, f32 ? nn * kpad * 4 : 0, f32 ? nn * kpad * 4 : 0,
                        bf ? nn * kpad * 2 : 0, nn * ldn * 4, nn * ldn * 4};
  for (int i = 0; i < 8; i++) {
    off[i] = need;
    need += up256(sz[i]);
  }
  if (need > (size_t)SED_NOALLOC_SCRATCH_BYTES)
    return na_fail(ctx, SED_ERANGE,
                   "sed_loglike_noalloc: %d rows need %zu bytes of scratch, the fixed maximum is %zu bytes",
                   n, need, (size_t)SED_NOALLOC_SCRATCH_BYTES);

  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != ctx->device) cudaSetDevice(ctx->device);
  struct Restore {
    int d;
    ~Restore() { if (d >= 0) cudaSetDevice(d); }
  } restore{prev != ctx->device ? prev : -1};

  void* base = nullptr;
  if (sed_status st = noalloc_scratch_ptr(ctx, &base)) return st;
  unsigned char* b = static_cast<unsigned char*>(base);
  int* err = reinterpret_cast<int*>(b + off[0]);
  RowScal* rs = reinterpret_cast<RowScal*>(b + off[1]);
  float* W = reinterpret_cast<float*>(b + off[2]);
  float* W_hi = f32 ? reinterpret_cast<float*>(b + off[3]) : nullptr;
  float* W_lo = f32 ? reinterpret_cast<float*>(b + off[4]) : nullptr;
  __nv_bfloat16* W_bf = bf ? reinterpret_cast<__nv_bfloat16*>(b + off[5]) : nullptr;
  float* Y = reinterpret_cast<float*>(b + off[6]);
  float* O = reinterpret_cast<float*>(b + off[7]);
  cudaStream_t s = static_cast<cudaStream_t>(stream);

  PrepArgs pa{};
  pa.theta = theta; pa.n = n; pa.ld = ld;
  pa.md = M->dv; pa.g = g->dv; pa.L = L->dv();
  pa.W = precision == SED_PREC_FP32_SIMT ? W : nullptr;   // only the CUDA-core contraction reads FP32 W
  pa.W_hi = W_hi; pa.W_lo = W_lo; pa.W_bf16 = W_bf;
  pa.rs = rs; pa.err = err;
  cudaError_t e = launch_prep(pa, s);
  if (e == cudaSuccess) {
    if (precision == SED_PREC_FP32_SIMT) {
      ContractArgs ca{};
      ca.n = n; ca.n_lam = g->n_lam; ca.ldn = ldn; ca.Ky_pad = L->Ky_pad; ca.Kpad = kpad;
      ca.W = W; ca.sspT = L->sspT_f32; ca.Y = Y; ca.O = O;
      e = launch_contract_simt(ca, s);
    } else {
      TcMaps maps;
      if (tc_encode_maps(ctx->encode_fn, &maps, precision, f32 ? (const void*)W_hi : (const void*)W_bf, W_lo,
                         f32 ? (const void*)L->sspT_hi : (const void*)L->sspT_bf16, L->sspT_lo, n, g->n_lam,
                         kpad) != 0)
        return na_fail(ctx, SED_ECUDA, "cuTensorMapEncodeTiled failed");
      TcArgs ta{};
      ta.n = n; ta.n_lam = g->n_lam; ta.ldn = ldn; ta.Ky_pad = L->Ky_pad; ta.Kpad = kpad; ta.prec = precision;
      ta.maps = &maps; ta.Y = Y; ta.O = O; ta.err = err;
      e = launch_contract_tc(ta, s);
    }
  }
  if (e == cudaSuccess) {
    EpiArgs ea{};
    ea.n = n; ea.ldn = ldn; ea.Y = Y; ea.O = O; ea.rs = rs;
    ea.md = M->dv; ea.g = g->dv;
    ea.lnl = lnl_out; ea.status = row_status; ea.err = err;
    e = launch_epilogue(ea, s);
  }
  if (e != cudaSuccess) return na_fail(ctx, SED_ECUDA, "kernel launch: %s", cudaGetErrorString(e));
  return SED_OK;
}
