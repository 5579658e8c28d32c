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
// time.  This entry point runs the same kernels as sed_loglike, in the same
// order and with the same schedule (the redshift row order, the per-tile
// wavelength windows, the three-way split of the 3xTF32 contraction), so its
// results equal sed_loglike's bit for bit, but it takes every intermediate
// buffer from one fixed array in device global memory, declared below, and
// calls no cudaMalloc, cudaFree or allocating library routine.
//
// The array is SED_NOALLOC_SCRATCH_BYTES long and lives for the life of the
// process on every device that loads the library.  All calls share it:
// calls whose kernels can overlap on the GPU (different streams, or
// different host threads) race on it and must be serialised by the caller.
// Each call overwrites what it uses.  What must start from a known value is
// set on the call's stream before its kernels: the per-tile window bounds
// (two memsets, as in sed_loglike); the device error word of the
// contraction is cleared by the first kernel of every call.
//
// FP8 is refused (SED_EUNSUPPORTED): its operand copy of the grid is built
// with cudaMalloc on the first FP8 call of sed_loglike, so an allocation-free
// call cannot rely on it.
#include <stdarg.h>
#include <stdio.h>

#include <algorithm>
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
  if (M->dv.n_bin > 0) return na_fail(ctx, SED_EUNSUPPORTED, "age-binned dust needs sed_loglike (one slab per block)");
  if (M->dv.use_neb && M->g->neb_na > 0)
    return na_fail(ctx, SED_EUNSUPPORTED, "a nebular age axis needs sed_loglike (per-age weights)");
  if (n < 0) return na_fail(ctx, SED_EINVAL, "n < 0");
  if (n > 0 && (!theta || !lnl_out)) return na_fail(ctx, SED_EINVAL, "theta or lnl_out is NULL");
  if (ld < M->dv.n_param) return na_fail(ctx, SED_EINVAL, "ld (%d) < n_param (%d)", ld, M->dv.n_param);
  if (precision == SED_PREC_FP8)
    return na_fail(ctx, SED_EUNSUPPORTED,
                   "sed_loglike_noalloc: FP8 needs the grid's FP8 copy, which sed_loglike allocates on first use");
  if (precision != SED_PREC_FP32 && precision != SED_PREC_FP32_SIMT && precision != SED_PREC_BF16)
    return na_fail(ctx, SED_EINVAL, "unknown precision %d", precision);
  if (precision != SED_PREC_FP32_SIMT && ctx->tc_ok != 1)
    return na_fail(ctx, SED_EUNSUPPORTED, "tensor-core precisions need an sm_103 device");
  if (!(M->g->avail & (1u << precision)))
    return na_fail(ctx, SED_EUNSUPPORTED, "precision %d: its copy of the grid was not kept (precision_mask)", precision);
  if (n > (1 << 22)) return na_fail(ctx, SED_ERANGE, "batch larger than 4M rows");
  if (n == 0) return SED_OK;

  const Grid* g = M->g;
  const Layout* L = M->L;
  const int kpad = L->Kpad;
  const int ldn = (g->n_lam + 255) / 256 * 256;
  const bool f32 = precision == SED_PREC_FP32, bf = precision == SED_PREC_BF16, simt = !f32 && !bf;
  // K-tile masks of the tensor-core contraction, as in sed_loglike
  const int kt_shift = bf ? 6 : 5;
  const int kmask_w = ((kpad >> kt_shift) + 31) / 32;
  const int pairs = std::max(g->n_feh - 1, 1) * (M->dv.use_afe ? std::max(g->n_afe - 1, 1) : 1);
  const bool use_km = f32 && M->dv.zmode == 1 && pairs > 1 && kmask_w <= KMASK_WORDS;
  // carve the scratch: err | perm | tile windows | K-tile masks | RowScal | W (FFMA) | W_hi | W_lo | W_bf16 |
  // Y | O
  const size_t nn = (size_t)n, mt = (nn + 127) / 128;
  constexpr int NB = 11;
  size_t off[NB], need = 0;
  const size_t sz[NB] = {256, nn * 4, 2 * mt * 4, use_km ? mt * kmask_w * 4 : 0, nn * sizeof(RowScal),
                         simt ? nn * kpad * 4 : 0, f32 ? nn * kpad * 4 : 0, f32 ? nn * kpad * 4 : 0,
                         bf ? nn * kpad * 2 : 0, nn * ldn * 4, nn * ldn * 4};
  for (int i = 0; i < NB; i++) {
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
  auto at = [&](int i) { return sz[i] ? static_cast<void*>(b + off[i]) : nullptr; };
  int* err = static_cast<int*>(at(0));
  int* perm = static_cast<int*>(at(1));
  int* tile_win = static_cast<int*>(at(2));
  uint32_t* kmask = static_cast<uint32_t*>(at(3));
  RowScal* rs = static_cast<RowScal*>(at(4));
  float* W = static_cast<float*>(at(5));
  float* W_hi = static_cast<float*>(at(6));
  float* W_lo = static_cast<float*>(at(7));
  __nv_bfloat16* W_bf = static_cast<__nv_bfloat16*>(at(8));
  float* Y = static_cast<float*>(at(9));
  float* O = static_cast<float*>(at(10));
  cudaStream_t s = static_cast<cudaStream_t>(stream);

  cudaError_t e = cudaSuccess;   // launch_prep starts the per-tile windows and masks empty
  PrepArgs pa{};
  pa.theta = theta; pa.n = n; pa.ld = ld;
  pa.md = M->dv; pa.g = g->dv; pa.L = L->dv();
  pa.W = W; pa.W_hi = W_hi; pa.W_lo = W_lo; pa.W_bf16 = W_bf;
  pa.rs = rs; pa.err = err; pa.perm = perm; pa.tile_win = tile_win;
  pa.kmask = use_km ? kmask : nullptr; pa.kmask_w = use_km ? kmask_w : 0; pa.kt_shift = kt_shift;
  if (e == cudaSuccess) e = launch_prep(pa, s);
  if (e == cudaSuccess) {
    if (simt) {
      ContractArgs ca{};
      ca.n = n; ca.n_lam = g->n_lam; ca.ldn = ldn; ca.Ky_pad = L->Ky_pad; ca.Kpad = kpad;
      ca.W = W; ca.sspT = L->sspT_f32; ca.Y = Y; ca.O = O; ca.rs = rs;
      e = launch_contract_simt(ca, s);
    } else {
      TcMaps maps;
      if (tc_encode_maps(ctx->encode_fn, &maps, precision, f32 ? (const void*)W_hi : (const void*)W_bf, W_lo,
                         f32 ? (const void*)L->sspT_hi : (const void*)L->sspT_bf16, L->sspT_lo, n, g->n_lam,
                         kpad) != 0)
        return na_fail(ctx, SED_ECUDA, "cuTensorMapEncodeTiled failed");
      TcArgs ta{};
      ta.n = n; ta.n_lam = g->n_lam; ta.ldn = ldn; ta.Ky_pad = L->Ky_pad; ta.Kpad = kpad; ta.prec = precision;
      ta.maps = &maps; ta.Y = Y; ta.O = O; ta.err = err; ta.rs = rs; ta.tile_win = tile_win;
      ta.kmask = pa.kmask; ta.kmask_w = pa.kmask_w;
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
