// Continuous-batching server of log-likelihood calls (include/sed.h, sed_server_*).
//
// Many fits (each a model: its filters, spectrum and data, plus a device buffer
// of live points) share one HBM-resident SSP grid.  Clients submit calls (a
// batch of parameter rows of one fit) as they arrive; a scheduler thread packs
// the pending calls of all fits, first come first served, into one launch of up
// to max_launch_rows rows, and keeps up to n_slots launches in flight on their
// own streams, so a call that arrives while others run is taken into the next
// free slot and its work overlaps theirs on the device.  Every row of a launch
// carries its fit's model index: the preparation and epilogue kernels read
// that row's model (filters, spectrum, data, SFH layout) from a device table,
// and the contraction is shared by all rows (one grid layout per server).
// Each row's arithmetic does not depend on the other rows of the launch, so a
// call's result is the same alone and in a mix.
//
// Fit admission is by device memory: open_fit reserves the fit's live-point
// buffer against fit_budget_bytes and returns SED_EBUSY when it does not fit.
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <chrono>
#include <condition_variable>
#include <deque>
#include <thread>
#include <unordered_map>

#include "sed_internal.cuh"

using namespace sed;

namespace {

constexpr int SRV_LD = 1048;          // row pitch of the packed launch buffer (a multiple of 4 floats)
// the widest parameter row: SFH (one more column with the linear scheme) and
// per-bin [Fe/H] (2 MAX_SFH + 1), 9 scalars, sigma_gal, 8 noise-floor terms and
// f_ob = 2 MAX_SFH + SED_NKEYS - 2 + 1
static_assert(SRV_LD >= 2 * MAX_SFH + SED_NKEYS - 1, "server row pitch below the widest parameter row");
constexpr int SRV_MAX_MODELS = 4096;  // entries of the device model table
constexpr int SRV_MAX_SLOTS = 8;

struct SrvCall {
  uint64_t ticket = 0;
  int fit = -1, n = 0;
  bool done = false;
  std::chrono::steady_clock::time_point t_submit;
  double latency_ms = 0.0;
  std::vector<double> lnl;
  std::vector<uint32_t> status;
};

struct SrvFit {
  bool open = false, busy = false;
  int model = -1, max_rows = 0, ld = 0;
  float* theta_d = nullptr;     // [max_rows][ld] live points on the device
  float* stage_h = nullptr;     // [max_rows][ld] pinned staging of host submissions
  cudaEvent_t uploaded = nullptr;
  size_t bytes = 0;
};

struct SrvSlot {
  cudaStream_t s = nullptr;
  cudaEvent_t done = nullptr;
  // launch buffers (device)
  float* theta = nullptr;       // [max_rows][SRV_LD]
  int* rowm = nullptr;          // [max_rows]
  int* perm = nullptr;          // [max_rows] processing order (rows grouped by redshift)
  int* tile_win = nullptr;      // [2][ceil(max_rows/128)] node windows of the 128-row tiles
  double* lnl = nullptr;
  uint32_t* st = nullptr;
  float *W = nullptr, *W_hi = nullptr, *W_lo = nullptr, *Y = nullptr, *O = nullptr, *O2 = nullptr;
  __nv_bfloat16* W_bf16 = nullptr;
  uint8_t* W_f8 = nullptr;
  RowScal* rs = nullptr;
  int* err = nullptr;
  // pinned host mirrors
  int* rowm_h = nullptr;
  double* lnl_h = nullptr;
  uint32_t* st_h = nullptr;
  TcMaps maps;
  int maps_n = -1;
  // the launch in flight
  bool busy = false, launched = false;
  std::vector<SrvCall*> calls;
  std::vector<int> offs;
  int rows = 0;
  std::thread th;
  std::vector<void*> dev;
  std::vector<void*> host;
};

}  // namespace

struct sed_server {
  sed_ctx* ctx = nullptr;
  Grid* g = nullptr;
  Layout* L = nullptr;
  int prec = 0, max_rows = 0, n_slots = 0, ldn = 0;
  size_t budget = 0, used = 0;
  ModelDev* mtab = nullptr;
  std::vector<char> mtab_loaded;
  int max_samp = 0, max_pix = 0, max_win = 1;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<SrvCall*> pending;
  std::unordered_map<uint64_t, SrvCall*> calls;
  std::vector<SrvFit> fits;
  SrvSlot slots[SRV_MAX_SLOTS];
  std::thread sched;
  cudaStream_t up = nullptr;    // uploads of host submissions
  bool stop = false;
  uint64_t next_ticket = 1;
  sed_server_stats stats{};
  std::vector<void*> dev;
  std::string err;
};

namespace {

sed_status sfail(sed_server* sv, sed_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (sv) {
    sv->ctx->last_error = buf;
  }
  return st;
}

template <class T>
bool dmalloc(sed_server* sv, std::vector<void*>& own, T** p, size_t bytes) {
  bytes = (bytes + 255) & ~(size_t)255;
  if (!budget_reserve(sv->ctx, bytes)) return false;
  if (cudaMalloc((void**)p, bytes) != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    budget_release(sv->ctx, bytes);
    return false;
  }
  own.push_back(*p);
  return true;
}

template <class T>
bool hmalloc(std::vector<void*>& own, T** p, size_t bytes) {
  if (cudaMallocHost((void**)p, bytes) != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return false;
  }
  own.push_back(*p);
  return true;
}

// Enqueue one packed launch on the slot's stream (server lock held by the caller).
cudaError_t issue_launch(sed_server* sv, SrvSlot& sl) {
  cudaStream_t s = sl.s;
  const int n = sl.rows;
  cudaError_t e = cudaSuccess;
  // gather the calls' live points into the packed buffer, and their model indices
  for (size_t c = 0; c < sl.calls.size() && e == cudaSuccess; ++c) {
    SrvFit& f = sv->fits[sl.calls[c]->fit];
    e = cudaStreamWaitEvent(s, f.uploaded, 0);
    if (e == cudaSuccess)
      e = cudaMemcpy2DAsync(sl.theta + (size_t)sl.offs[c] * SRV_LD, SRV_LD * sizeof(float), f.theta_d,
                            f.ld * sizeof(float), f.ld * sizeof(float), sl.calls[c]->n, cudaMemcpyDeviceToDevice, s);
    for (int i = 0; i < sl.calls[c]->n; ++i) sl.rowm_h[sl.offs[c] + i] = f.model;
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(sl.rowm, sl.rowm_h, n * sizeof(int), cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return e;
  const Grid* g = sv->g;
  const Layout* L = sv->L;
  const bool f32 = sv->prec == SED_PREC_FP32, bf = sv->prec == SED_PREC_BF16, f8 = sv->prec == SED_PREC_FP8;
  PrepArgs pa{};
  pa.theta = sl.theta; pa.n = n; pa.ld = SRV_LD;
  pa.g = g->dv; pa.L = L->dv();
  pa.mtab = sv->mtab; pa.row_model = sl.rowm;
  pa.W = sv->prec == SED_PREC_FP32_SIMT ? sl.W : nullptr;   // only the CUDA-core contraction reads FP32 W
  pa.W_hi = f32 ? sl.W_hi : nullptr;
  pa.W_lo = f32 ? sl.W_lo : nullptr;
  pa.W_bf16 = bf ? sl.W_bf16 : nullptr;
  pa.W_f8 = f8 ? sl.W_f8 : nullptr;
  pa.rs = sl.rs;
  pa.err = sl.err;
  // rows grouped by redshift (each row's own model) and each 128-row tile's
  // node window, as sed_loglike does: the contraction then computes only the
  // wavelength tiles its rows read, on the persistent schedule
  pa.perm = sl.perm;
  pa.tile_win = sl.tile_win;   // launch_prep starts its windows empty
  e = launch_prep(pa, s);
  if (e != cudaSuccess) return e;
  if (sv->prec == SED_PREC_FP32_SIMT) {
    ContractArgs ca{};
    ca.n = n; ca.n_lam = g->n_lam; ca.ldn = sv->ldn; ca.Ky_pad = L->Ky_pad; ca.Kpad = L->Kpad;
    ca.W = sl.W; ca.sspT = L->sspT_f32; ca.Y = sl.Y; ca.O = sl.O; ca.rs = sl.rs;
    e = launch_contract_simt(ca, s);
  } else {
    // the operand maps are encoded once per slot, over its max_launch_rows rows:
    // rows past a launch's n are read by its last M tile but never stored
    if (sl.maps_n != sv->max_rows) {
      const void* a_op = f32 ? (const void*)sl.W_hi : (f8 ? (const void*)sl.W_f8 : (const void*)sl.W_bf16);
      const void* b_op = f32 ? (const void*)L->sspT_hi : (f8 ? (const void*)L->sspT_f8 : (const void*)L->sspT_bf16);
      if (tc_encode_maps(sv->ctx->encode_fn, &sl.maps, sv->prec, a_op, sl.W_lo, b_op, L->sspT_lo, sv->max_rows,
                         g->n_lam, f8 ? L->Kpad8 : L->Kpad))
        return cudaErrorInvalidValue;
      sl.maps_n = sv->max_rows;
    }
    TcArgs ta{};
    ta.n = n; ta.n_lam = g->n_lam; ta.ldn = sv->ldn; ta.prec = sv->prec;
    ta.Ky_pad = f8 ? L->Ky_pad8 : L->Ky_pad;
    ta.Kpad = f8 ? L->Kpad8 : L->Kpad;
    ta.maps = &sl.maps; ta.Y = sl.Y; ta.O = sl.O; ta.err = sl.err; ta.rs = sl.rs;
    ta.tile_win = sl.tile_win;
    ta.O2 = sl.O2; ta.split_out = sl.err + 8;   // err[8]: the launch records whether it split its tiles
    e = launch_contract_tc(ta, s);
  }
  if (e != cudaSuccess) return e;
  EpiArgs ea{};
  ea.n = n; ea.ldn = sv->ldn; ea.Y = sl.Y; ea.O = sl.O; ea.rs = sl.rs;
  ea.O2 = sl.O2; ea.split = sv->prec == SED_PREC_FP32 ? sl.err + 8 : nullptr;   // same choice as sed_loglike
  ea.g = g->dv;
  ea.mtab = sv->mtab; ea.row_model = sl.rowm;
  ea.smem_samp = sv->max_samp; ea.smem_pix = sv->max_pix; ea.smem_win = sv->max_win;
  ea.lnl = sl.lnl; ea.status = sl.st; ea.err = sl.err;
  ea.lam8 = f8 ? L->lam8 : nullptr;
  e = launch_epilogue(ea, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(sl.lnl_h, sl.lnl, n * sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(sl.st_h, sl.st, n * sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaEventRecord(sl.done, s);
  return e;
}

void scheduler_main(sed_server* sv) {
  cudaSetDevice(sv->ctx->device);
  std::unique_lock<std::mutex> lk(sv->mu);
  for (;;) {
    int slot = -1;
    sv->cv.wait(lk, [&] {
      if (sv->stop) return true;
      if (sv->pending.empty()) return false;
      for (int i = 0; i < sv->n_slots; ++i)
        if (!sv->slots[i].busy) { slot = i; return true; }
      return false;
    });
    if (sv->stop) break;
    SrvSlot& sl = sv->slots[slot];
    sl.calls.clear();
    sl.offs.clear();
    sl.rows = 0;
    // first come, first served, while the rows fit in one launch
    while (!sv->pending.empty() && sl.rows + sv->pending.front()->n <= sv->max_rows) {
      SrvCall* c = sv->pending.front();
      sv->pending.pop_front();
      sl.offs.push_back(sl.rows);
      sl.calls.push_back(c);
      sl.rows += c->n;
    }
    sl.busy = true;
    cudaError_t e = issue_launch(sv, sl);
    if (e != cudaSuccess) {
      cudaGetLastError();
      for (SrvCall* c : sl.calls) {
        c->lnl.assign(c->n, -INFINITY);
        c->status.assign(c->n, SED_ROW_DEVICE_TIMEOUT);
        c->done = true;
        sv->fits[c->fit].busy = false;
      }
      sv->err = std::string("launch failed: ") + cudaGetErrorString(e);
      sl.busy = false;
      sv->cv.notify_all();
      continue;
    }
    sv->stats.launches++;
    sv->stats.rows += (uint64_t)sl.rows;
    sl.launched = true;
    sv->cv.notify_all();
  }
}

void slot_main(sed_server* sv, int i) {
  cudaSetDevice(sv->ctx->device);
  SrvSlot& sl = sv->slots[i];
  std::unique_lock<std::mutex> lk(sv->mu);
  for (;;) {
    sv->cv.wait(lk, [&] { return sv->stop || sl.launched; });
    if (sv->stop && !sl.launched) break;
    lk.unlock();
    cudaEventSynchronize(sl.done);   // the kernels' own waits are bounded, so this returns
    const auto now = std::chrono::steady_clock::now();
    lk.lock();
    for (size_t c = 0; c < sl.calls.size(); ++c) {
      SrvCall* call = sl.calls[c];
      call->lnl.assign(sl.lnl_h + sl.offs[c], sl.lnl_h + sl.offs[c] + call->n);
      call->status.assign(sl.st_h + sl.offs[c], sl.st_h + sl.offs[c] + call->n);
      call->latency_ms = std::chrono::duration<double, std::milli>(now - call->t_submit).count();
      call->done = true;
      sv->fits[call->fit].busy = false;
      sv->stats.calls++;
    }
    sl.calls.clear();
    sl.launched = false;
    sl.busy = false;
    sv->cv.notify_all();
  }
}

}  // namespace

extern "C" {

sed_status sed_server_create(sed_ctx* ctx, const sed_server_desc* d, sed_server** out) {
  if (!ctx || !d || !out) return SED_EINVAL;
  *out = nullptr;
  if (d->grid < 0 || d->grid >= (int)ctx->grids.size() || !ctx->grids[d->grid])
    return SED_EINVAL;
  if (d->precision < SED_PREC_FP32 || d->precision > SED_PREC_FP8) return SED_EINVAL;
  if (d->precision != SED_PREC_FP32_SIMT && ctx->tc_ok != 1) return SED_EUNSUPPORTED;
  if (!(ctx->grids[d->grid]->avail & (1u << d->precision))) return SED_EUNSUPPORTED;   // copy not kept
  if (d->max_launch_rows < 1 || d->max_launch_rows > (1 << 20)) return SED_ERANGE;
  if (d->n_slots < 1 || d->n_slots > SRV_MAX_SLOTS) return SED_ERANGE;
  if (d->model_layout < 0 || d->model_layout >= (int)ctx->models.size() || !ctx->models[d->model_layout])
    return SED_EINVAL;
  sed::Model* M0 = ctx->models[d->model_layout];
  if (M0->grid != d->grid) return SED_EINVAL;
  if (M0->dv.n_bin > 0) return SED_EUNSUPPORTED;   // age-binned dust is not served
  if (M0->dv.use_neb && M0->g->neb_na > 0) return SED_EUNSUPPORTED;   // nor a nebular age axis
  int prev = -1;
  cudaGetDevice(&prev);
  cudaSetDevice(ctx->device);
  sed_server* sv = new sed_server();
  sv->ctx = ctx;
  sv->g = ctx->grids[d->grid];
  sv->L = M0->L;
  sv->prec = d->precision;
  sv->max_rows = d->max_launch_rows;
  sv->n_slots = d->n_slots;
  sv->budget = d->fit_budget_bytes;
  sv->ldn = (sv->g->n_lam + 255) / 256 * 256;
  bool ok = true;
  if (sv->prec == SED_PREC_FP8) {
    std::lock_guard<std::mutex> lk(ctx->mu);
    ok = ensure_f8_layout_shared(ctx, sv->g, sv->L) == SED_OK;
  }
  ok = ok && cudaStreamCreateWithFlags(&sv->up, cudaStreamNonBlocking) == cudaSuccess;
  ok = ok && dmalloc(sv, sv->dev, &sv->mtab, sizeof(ModelDev) * SRV_MAX_MODELS);
  sv->mtab_loaded.assign(SRV_MAX_MODELS, 0);
  const size_t R = (size_t)sv->max_rows, K = (size_t)sv->L->Kpad, N = (size_t)sv->ldn;
  for (int i = 0; ok && i < sv->n_slots; ++i) {
    SrvSlot& sl = sv->slots[i];
    ok = cudaStreamCreateWithFlags(&sl.s, cudaStreamNonBlocking) == cudaSuccess &&
         cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming) == cudaSuccess;
    ok = ok && dmalloc(sv, sl.dev, &sl.theta, R * SRV_LD * 4) && dmalloc(sv, sl.dev, &sl.rowm, R * 4) &&
         dmalloc(sv, sl.dev, &sl.lnl, R * 8) && dmalloc(sv, sl.dev, &sl.st, R * 4) &&
         dmalloc(sv, sl.dev, &sl.W, R * K * 4) && dmalloc(sv, sl.dev, &sl.Y, R * N * 4) &&
         dmalloc(sv, sl.dev, &sl.O, R * N * 4) && dmalloc(sv, sl.dev, &sl.O2, R * N * 4) &&
         dmalloc(sv, sl.dev, &sl.rs, R * sizeof(RowScal)) &&
         dmalloc(sv, sl.dev, &sl.err, 256) && dmalloc(sv, sl.dev, &sl.perm, R * 4) &&
         dmalloc(sv, sl.dev, &sl.tile_win, 2 * ((R + 127) / 128) * 4);
    if (ok && sv->prec == SED_PREC_FP32)
      ok = dmalloc(sv, sl.dev, &sl.W_hi, R * K * 4) && dmalloc(sv, sl.dev, &sl.W_lo, R * K * 4);
    if (ok && sv->prec == SED_PREC_BF16) ok = dmalloc(sv, sl.dev, &sl.W_bf16, R * K * 2);
    if (ok && sv->prec == SED_PREC_FP8) ok = dmalloc(sv, sl.dev, &sl.W_f8, R * (K + 128));
    ok = ok && hmalloc(sl.host, &sl.rowm_h, R * 4) && hmalloc(sl.host, &sl.lnl_h, R * 8) &&
         hmalloc(sl.host, &sl.st_h, R * 4);
    ok = ok && cudaMemset(sl.err, 0, 256) == cudaSuccess;
  }
  if (!ok) {
    cudaGetLastError();
    sv->stop = true;
    sed_server_destroy(sv);
    if (prev >= 0) cudaSetDevice(prev);
    return SED_ENOMEM;
  }
  sv->sched = std::thread(scheduler_main, sv);
  for (int i = 0; i < sv->n_slots; ++i) sv->slots[i].th = std::thread(slot_main, sv, i);
  if (prev >= 0) cudaSetDevice(prev);
  *out = sv;
  return SED_OK;
}

sed_status sed_server_destroy(sed_server* sv) {
  if (!sv) return SED_EINVAL;
  int prev = -1;
  cudaGetDevice(&prev);
  cudaSetDevice(sv->ctx->device);
  {
    // let the launches in flight finish, then stop the threads
    std::unique_lock<std::mutex> lk(sv->mu);
    sv->cv.wait(lk, [&] {
      for (int i = 0; i < sv->n_slots; ++i)
        if (sv->slots[i].busy) return false;
      return true;
    });
    sv->stop = true;
  }
  sv->cv.notify_all();
  if (sv->sched.joinable()) sv->sched.join();
  for (int i = 0; i < SRV_MAX_SLOTS; ++i) {
    SrvSlot& sl = sv->slots[i];
    if (sl.th.joinable()) sl.th.join();
    for (void* p : sl.dev) cudaFree(p);
    for (void* p : sl.host) cudaFreeHost(p);
    if (sl.done) cudaEventDestroy(sl.done);
    if (sl.s) cudaStreamDestroy(sl.s);
  }
  for (SrvFit& f : sv->fits) {
    if (f.theta_d) cudaFree(f.theta_d);
    if (f.stage_h) cudaFreeHost(f.stage_h);
    if (f.uploaded) cudaEventDestroy(f.uploaded);
  }
  for (void* p : sv->dev) cudaFree(p);
  if (sv->up) cudaStreamDestroy(sv->up);
  for (auto& kv : sv->calls) delete kv.second;   // pending calls are in this map too
  delete sv;
  if (prev >= 0) cudaSetDevice(prev);
  return SED_OK;
}

sed_status sed_server_open_fit(sed_server* sv, sed_model_id model, int max_rows, int* fit) {
  if (!sv || !fit) return SED_EINVAL;
  sed_ctx* ctx = sv->ctx;
  if (model < 0 || model >= (int)ctx->models.size() || !ctx->models[model])
    return sfail(sv, SED_EINVAL, "unknown model %d", model);
  if (model >= SRV_MAX_MODELS) return sfail(sv, SED_ERANGE, "model id beyond the server's table (%d)", SRV_MAX_MODELS);
  sed::Model* M = ctx->models[model];
  if (M->L != sv->L) return sfail(sv, SED_EINVAL, "model %d uses another grid layout than the server", model);
  if (M->dv.n_bin > 0) return sfail(sv, SED_EUNSUPPORTED, "model %d has age-binned dust (not served)", model);
  if (M->dv.use_neb && M->g->neb_na > 0)
    return sfail(sv, SED_EUNSUPPORTED, "model %d has a nebular age axis (not served)", model);
  if (max_rows < 1 || max_rows > sv->max_rows)
    return sfail(sv, SED_ERANGE, "max_rows must be in [1, %d]", sv->max_rows);
  const int ld = M->dv.n_param;
  const size_t need = ((size_t)max_rows * ld * 4 + 255) & ~(size_t)255;
  std::lock_guard<std::mutex> lk(sv->mu);
  if (sv->budget && sv->used + need > sv->budget)
    return sfail(sv, SED_EBUSY, "fit needs %zu bytes, %zu of %zu in use", need, sv->used, sv->budget);
  int prev = -1;
  cudaGetDevice(&prev);
  cudaSetDevice(ctx->device);
  SrvFit f;
  f.open = true;
  f.model = model;
  f.max_rows = max_rows;
  f.ld = ld;
  f.bytes = need;
  sed_status st = SED_OK;
  const bool reserved = budget_reserve(ctx, need);
  if (!reserved) st = SED_ENOMEM;
  if (!st && cudaMalloc((void**)&f.theta_d, need) != cudaSuccess) st = SED_ENOMEM;
  if (!st && cudaMallocHost((void**)&f.stage_h, (size_t)max_rows * ld * 4) != cudaSuccess) st = SED_ENOMEM;
  if (!st && cudaEventCreateWithFlags(&f.uploaded, cudaEventDisableTiming) != cudaSuccess) st = SED_ECUDA;
  if (!st && !sv->mtab_loaded[model]) {
    if (cudaMemcpy(sv->mtab + model, &M->dv, sizeof(ModelDev), cudaMemcpyHostToDevice) != cudaSuccess) st = SED_ECUDA;
    else sv->mtab_loaded[model] = 1;
  }
  if (!st && cudaEventRecord(f.uploaded, sv->up) != cudaSuccess) st = SED_ECUDA;
  if (st) {
    cudaGetLastError();
    if (f.theta_d) cudaFree(f.theta_d);
    if (f.stage_h) cudaFreeHost(f.stage_h);
    if (f.uploaded) cudaEventDestroy(f.uploaded);
    if (reserved) budget_release(ctx, need);
    if (prev >= 0) cudaSetDevice(prev);
    return sfail(sv, st, "could not allocate the fit's buffers");
  }
  sv->used += need;
  sv->max_samp = std::max(sv->max_samp, M->dv.n_samp);
  sv->max_pix = std::max(sv->max_pix, M->dv.n_pix);
  sv->max_win = std::max(sv->max_win, M->dv.win_max);
  int id = -1;
  for (size_t i = 0; i < sv->fits.size(); ++i)
    if (!sv->fits[i].open && !sv->fits[i].theta_d) { id = (int)i; break; }
  if (id < 0) { id = (int)sv->fits.size(); sv->fits.push_back(f); }
  else sv->fits[id] = f;
  sv->stats.fits_open++;
  sv->stats.fit_bytes = sv->used;
  if (prev >= 0) cudaSetDevice(prev);
  *fit = id;
  return SED_OK;
}

sed_status sed_server_close_fit(sed_server* sv, int fit) {
  if (!sv) return SED_EINVAL;
  std::unique_lock<std::mutex> lk(sv->mu);
  if (fit < 0 || fit >= (int)sv->fits.size() || !sv->fits[fit].open) return sfail(sv, SED_EINVAL, "unknown fit %d", fit);
  sv->cv.wait(lk, [&] { return !sv->fits[fit].busy; });
  SrvFit& f = sv->fits[fit];
  int prev = -1;
  cudaGetDevice(&prev);
  cudaSetDevice(sv->ctx->device);
  cudaEventSynchronize(f.uploaded);
  cudaFree(f.theta_d);
  cudaFreeHost(f.stage_h);
  cudaEventDestroy(f.uploaded);
  budget_release(sv->ctx, f.bytes);
  sv->used -= std::min(sv->used, f.bytes);
  f = SrvFit();
  sv->stats.fits_open--;
  sv->stats.fit_bytes = sv->used;
  if (prev >= 0) cudaSetDevice(prev);
  return SED_OK;
}

float* sed_server_fit_theta(sed_server* sv, int fit) {
  if (!sv) return nullptr;
  std::lock_guard<std::mutex> lk(sv->mu);
  if (fit < 0 || fit >= (int)sv->fits.size() || !sv->fits[fit].open) return nullptr;
  return sv->fits[fit].theta_d;
}

static sed_status submit_impl(sed_server* sv, int fit, const float* theta, int n, int ld, uint64_t* ticket) {
  if (!sv || !ticket) return SED_EINVAL;
  std::unique_lock<std::mutex> lk(sv->mu);
  if (fit < 0 || fit >= (int)sv->fits.size() || !sv->fits[fit].open) return sfail(sv, SED_EINVAL, "unknown fit %d", fit);
  SrvFit& f = sv->fits[fit];
  if (n < 1 || n > f.max_rows) return sfail(sv, SED_ERANGE, "n must be in [1, %d]", f.max_rows);
  if (f.busy) return sfail(sv, SED_EBUSY, "fit %d has a call in flight", fit);
  if (theta) {
    if (ld < f.ld) return sfail(sv, SED_EINVAL, "ld (%d) < n_param (%d)", ld, f.ld);
    for (int r = 0; r < n; ++r) memcpy(f.stage_h + (size_t)r * f.ld, theta + (size_t)r * ld, f.ld * sizeof(float));
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(sv->ctx->device);
    cudaStream_t s = sv->up;
    cudaError_t e = cudaMemcpyAsync(f.theta_d, f.stage_h, (size_t)n * f.ld * sizeof(float), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaEventRecord(f.uploaded, s);
    if (prev >= 0) cudaSetDevice(prev);
    if (e != cudaSuccess) return sfail(sv, SED_ECUDA, "upload: %s", cudaGetErrorString(e));
  }
  SrvCall* c = new SrvCall();
  c->ticket = sv->next_ticket++;
  c->fit = fit;
  c->n = n;
  c->t_submit = std::chrono::steady_clock::now();
  f.busy = true;
  sv->calls[c->ticket] = c;
  sv->pending.push_back(c);
  *ticket = c->ticket;
  sv->cv.notify_all();
  return SED_OK;
}

sed_status sed_server_submit(sed_server* sv, int fit, const float* theta_host, int n, int ld, uint64_t* ticket) {
  if (!theta_host) return SED_EINVAL;
  return submit_impl(sv, fit, theta_host, n, ld, ticket);
}

sed_status sed_server_submit_device(sed_server* sv, int fit, int n, uint64_t* ticket) {
  return submit_impl(sv, fit, nullptr, n, 0, ticket);
}

sed_status sed_server_wait(sed_server* sv, uint64_t ticket, double* lnl_host, uint32_t* status_host, int timeout_ms,
                           double* latency_ms) {
  if (!sv) return SED_EINVAL;
  std::unique_lock<std::mutex> lk(sv->mu);
  auto it = sv->calls.find(ticket);
  if (it == sv->calls.end()) return sfail(sv, SED_EINVAL, "unknown ticket %llu", (unsigned long long)ticket);
  SrvCall* c = it->second;
  const auto pred = [&] { return c->done; };
  if (timeout_ms < 0) sv->cv.wait(lk, pred);
  else if (!sv->cv.wait_for(lk, std::chrono::milliseconds(timeout_ms), pred)) return SED_ETIMEOUT;
  if (lnl_host) memcpy(lnl_host, c->lnl.data(), c->n * sizeof(double));
  if (status_host) memcpy(status_host, c->status.data(), c->n * sizeof(uint32_t));
  if (latency_ms) *latency_ms = c->latency_ms;
  sv->calls.erase(it);
  delete c;
  return SED_OK;
}

sed_status sed_server_get_stats(sed_server* sv, sed_server_stats* out) {
  if (!sv || !out) return SED_EINVAL;
  std::lock_guard<std::mutex> lk(sv->mu);
  *out = sv->stats;
  return SED_OK;
}

}  // extern "C"
