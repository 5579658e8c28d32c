"""Python binding of the C ABI (include/sed.h): argument marshalling only.

Every step of the forward model and likelihood runs in the CUDA library; this
module converts numpy/torch arguments into the pointers, sizes and streams
the C functions take.  PyTorch supplies device memory and streams.
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import _ffi
from ._ffi import KEYS, NKEYS

PREC = {"fp32": _ffi.PREC_FP32, "fp32_simt": _ffi.PREC_FP32_SIMT, "bf16": _ffi.PREC_BF16, "fp8": _ffi.PREC_FP8}


class SedError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{status}: {msg}")
        self.status = status


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a):
    return None if a is None else a.ctypes.data


def _stream_handle(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _prec(p):
    return PREC[p] if isinstance(p, str) else int(p)


class Context:
    """One library context on one CUDA device."""

    def __init__(self, device: int = 0, hbm_budget_bytes: int = 0):
        self._lib = _ffi.load()
        self.device = int(device)
        h = C.c_void_p()
        st = self._lib.sed_create(C.byref(h), self.device, C.c_size_t(int(hbm_budget_bytes)))
        if st:
            raise SedError(st, "sed_create failed")
        self._h = h
        self._grids = []

    def _check(self, st):
        if st:
            raise SedError(st, self._lib.sed_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None):
            self._lib.sed_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_profiling(self, on: bool):
        self._check(self._lib.sed_set_profiling(self._h, 1 if on else 0))

    def last_stats(self, stream=None):
        """Stage times (ms) and work counters of the last profiled call on `stream`."""
        st = _ffi.StageStats()
        self._check(self._lib.sed_last_stats(self._h, _stream_handle(stream), C.byref(st)))
        return {f: getattr(st, f) for f, _ in st._fields_}

    def last_host_path(self):
        """Bits of the last loglike_host call: 1 = theta read in place, 2 = lnL
        written in place (page-locked, device-mapped host buffers)."""
        v = C.c_int()
        self._check(self._lib.sed_last_host_path(self._h, C.byref(v)))
        return v.value

    def memory_used(self):
        v = C.c_size_t()
        self._check(self._lib.sed_memory_used(self._h, C.byref(v)))
        return v.value

    # ------------------------------------------------------------------
    def load_grid(self, grid, precision_mask=0) -> int:
        """grid: object with log_age_yr, feh, afe, lam_aa, flux[n_afe][n_feh][n_age][n_lam]
        and optionally neb_logu, neb_logz, neb_tab, sigma_lib_kms."""
        keep = [_f64(grid.log_age_yr), _f64(grid.feh), _f64(grid.afe), _f64(grid.lam_aa), _f64(grid.flux)]
        d = _ffi.GridDesc()
        d.n_afe, d.n_feh, d.n_age, d.n_lam = grid.flux.shape
        d.log_age_yr, d.feh, d.afe, d.lam_aa, d.flux = (_ptr(a) for a in keep)
        sl = _f64(getattr(grid, "sigma_lib_kms", None))
        keep.append(sl)
        d.sigma_lib_kms = _ptr(sl)
        if getattr(grid, "neb_tab", None) is not None:
            nu, nz, nt = _f64(grid.neb_logu), _f64(grid.neb_logz), _f64(grid.neb_tab)
            keep += [nu, nz, nt]
            na = getattr(grid, "neb_log_age", None)
            if na is not None:   # nebular age axis: neb_tab [n_age][n_logu][n_logz][n_lam]
                na = _f64(na)
                keep.append(na)
                d.neb_n_age, d.neb_log_age_yr = na.size, _ptr(na)
                d.neb_n_logu, d.neb_n_logz = nt.shape[1:3]
            else:
                d.neb_n_logu, d.neb_n_logz = nt.shape[:2]
            d.neb_logu, d.neb_logz, d.neb_log10_lnu_per_q = _ptr(nu), _ptr(nz), _ptr(nt)
            if getattr(grid, "line_tab", None) is not None:
                ll, lt = _f64(grid.line_lam), _f64(grid.line_tab)
                keep += [ll, lt]
                d.neb_n_line = ll.size
                d.neb_line_lam_aa, d.neb_log10_line_per_q = _ptr(ll), _ptr(lt)
        d.precision_mask = int(precision_mask)
        gid = C.c_int32()
        self._check(self._lib.sed_load_grid(self._h, C.byref(d), C.byref(gid)))
        self.__dict__.setdefault("_grid_lines", {})[gid.value] = int(d.neb_n_line)
        return gid.value

    def create_model(self, grid_id, n_sfh, zf, zmode, *, use_afe=0, use_nebular=0, dust_law=0,
                     bc_edge_log_age_yr=7.03, H0=67.66, Om0=0.3097, filters=None,
                     phot_d=None, phot_sigma=None, phot_mask=None, spec_lam=None, spec_d=None,
                     spec_sigma=None, spec_mask=None, lsf_mode=0, lsf_value=None,
                     sigma_gal_kms=0.0, z_ref=0.0, sample_sigma_gal=0, sigma_gal_max_kms=1000.0,
                     calib_sigma=None, noise_floor_phot=0, noise_floor_spec=0, sfh_scheme=0,
                     phot_upper=None, fesc_geometry=0, fixed=None, calib_mode=0, use_lines=0,
                     gas_sigma_mode=0, sigma_gas_kms=300.0, sigma_gas_max_kms=1000.0, lcat=None,
                     dust_bins=None, use_igm=0) -> "Model":
        """fixed: optional {key name: value} of keys fixed for every row (no
        column in the parameter rows, no gradient); key names as in _ffi.KEYS.
        lcat: optional line catalogue (blends: list of lists of grid-line
        indices, data, sigma, mask or None, upper-limit flags or None).
        dust_bins: optional age-binned attenuation (M [n_age][n_bin] age-to-bin
        matrix, laws [n_bin] of DUST_POWER_LAW / DUST_KC13)."""
        d = _ffi.ModelDesc()
        d.grid, d.n_sfh, d.zf, d.zmode = grid_id, n_sfh, zf, zmode
        d.use_afe, d.use_nebular, d.dust_law = use_afe, use_nebular, dust_law
        d.bc_edge_log_age_yr, d.H0, d.Om0 = bc_edge_log_age_yr, H0, Om0
        keep = []
        if filters is not None:
            lens, lam, tr = filters
            lens = np.ascontiguousarray(lens, dtype=np.int32)
            lam, tr = _f64(lam), _f64(tr)
            keep += [lens, lam, tr]
            d.n_filt = len(lens)
            d.filt_len, d.filt_lam_aa, d.filt_trans = _ptr(lens), _ptr(lam), _ptr(tr)
            pd, ps = _f64(phot_d), _f64(phot_sigma)
            pm = None if phot_mask is None else np.ascontiguousarray(phot_mask, dtype=np.uint8)
            pu = None if phot_upper is None else np.ascontiguousarray(phot_upper, dtype=np.uint8)
            keep += [pd, ps, pm, pu]
            d.phot_d, d.phot_sigma, d.phot_mask = _ptr(pd), _ptr(ps), _ptr(pm)
            d.phot_upper = _ptr(pu)
        if spec_lam is not None:
            sl, sd, ss, lv = _f64(spec_lam), _f64(spec_d), _f64(spec_sigma), _f64(lsf_value)
            sm = None if spec_mask is None else np.ascontiguousarray(spec_mask, dtype=np.uint8)
            keep += [sl, sd, ss, lv, sm]
            d.n_pix = sl.size
            d.spec_lam_aa, d.spec_d, d.spec_sigma, d.spec_mask = _ptr(sl), _ptr(sd), _ptr(ss), _ptr(sm)
            d.lsf_mode, d.lsf_value = lsf_mode, _ptr(lv)
            d.sigma_gal_kms, d.z_ref = sigma_gal_kms, z_ref
        d.sample_sigma_gal, d.sigma_gal_max_kms = int(sample_sigma_gal), float(sigma_gal_max_kms)
        if calib_sigma is not None:
            cs = _f64(calib_sigma)
            keep.append(cs)
            d.calib_n, d.calib_sigma = cs.size, _ptr(cs)
        d.calib_mode = int(calib_mode)
        d.use_igm = int(use_igm)
        if dust_bins is not None:
            bm, bl = dust_bins
            bm = np.ascontiguousarray(bm, dtype=np.float64)
            bl = np.ascontiguousarray(bl, dtype=np.int32)
            keep += [bm, bl]
            d.dust_n_bin = bm.shape[1]
            d.dust_bin_M, d.dust_bin_law = _ptr(bm), _ptr(bl)
        d.use_lines, d.gas_sigma_mode = int(use_lines), int(gas_sigma_mode)
        d.sigma_gas_kms, d.sigma_gas_max_kms = float(sigma_gas_kms), float(sigma_gas_max_kms)
        if lcat is not None:
            blends, ld, ls, lm, lu = lcat
            lens = np.ascontiguousarray([len(b) for b in blends], dtype=np.int32)
            lines = np.ascontiguousarray(np.concatenate([np.asarray(b, dtype=np.int32) for b in blends]), dtype=np.int32)
            ld, ls = _f64(ld), _f64(ls)
            lm = None if lm is None else np.ascontiguousarray(lm, dtype=np.uint8)
            lu = None if lu is None else np.ascontiguousarray(lu, dtype=np.uint8)
            keep += [lens, lines, ld, ls, lm, lu]
            d.n_lcat = len(blends)
            d.lcat_len, d.lcat_line, d.lcat_d, d.lcat_sigma = _ptr(lens), _ptr(lines), _ptr(ld), _ptr(ls)
            d.lcat_mask, d.lcat_upper = _ptr(lm), _ptr(lu)
        d.noise_floor_phot, d.noise_floor_spec = int(noise_floor_phot), int(noise_floor_spec)
        d.sfh_scheme = int(sfh_scheme)
        d.fesc_geometry = int(fesc_geometry)
        for k, v in (fixed or {}).items():
            i = KEYS.index(k)
            d.fixed[i] = 1
            d.fixed_val[i] = float(v)
        mid = C.c_int32()
        self._check(self._lib.sed_create_model(self._h, C.byref(d), C.byref(mid)))
        self.__dict__.setdefault("_n_line", {})[mid.value] = self.__dict__.get("_grid_lines", {}).get(grid_id, 0)
        return Model(self, mid.value, n_filt=d.n_filt, n_pix=d.n_pix)


class Model:
    """One fit (model description + observations) inside a Context."""

    def __init__(self, ctx: Context, mid: int, n_filt: int, n_pix: int):
        self.ctx, self.id, self.n_filt, self.n_pix = ctx, mid, n_filt, n_pix
        n = C.c_int()
        offs = (C.c_int * NKEYS)()
        ctx._check(ctx._lib.sed_model_layout(ctx._h, mid, C.byref(n), offs))
        self.n_param = n.value
        self.offsets = dict(zip(KEYS, list(offs)))

    def pack(self, d, dtype=np.float32):
        """Parameter rows in this model's column layout from a dict of arrays."""
        n = np.asarray(d["sfh"]).shape[0]
        out = np.zeros((n, self.n_param), dtype=np.float64)
        bounds = list(self.offsets.values()) + [self.n_param]
        for i, k in enumerate(KEYS):
            w = bounds[i + 1] - bounds[i]
            if w == 0:      # key without a column in this model (e.g. a fixed sigma_gal)
                continue
            out[:, bounds[i]:bounds[i] + w] = np.asarray(d[k], dtype=np.float64).reshape(n, w)
        return out.astype(dtype)

    def close(self):
        """Release the model's device memory (sed_destroy_model)."""
        if self.id is not None and getattr(self.ctx, "_h", None):
            self.ctx._check(self.ctx._lib.sed_destroy_model(self.ctx._h, self.id))
        self.id = None

    def set_data(self, phot_d=None, phot_sigma=None, spec_d=None, spec_sigma=None):
        a = [_f64(phot_d), _f64(phot_sigma), _f64(spec_d), _f64(spec_sigma)]
        self.ctx._check(self.ctx._lib.sed_set_data(self.ctx._h, self.id, *(_ptr(x) for x in a)))

    def _theta(self, theta):
        if not (theta.is_cuda and theta.dtype == torch.float32 and theta.dim() == 2 and theta.stride(1) == 1):
            raise ValueError("theta must be a CUDA float32 [n, ld] tensor with unit column stride")
        return theta.shape[0], theta.stride(0)

    def forward(self, theta: torch.Tensor, precision="fp32", stream=None):
        n, ld = self._theta(theta)
        dev = theta.device
        phot = torch.empty((n, self.n_filt), dtype=torch.float32, device=dev) if self.n_filt else None
        spec = torch.empty((n, self.n_pix), dtype=torch.float32, device=dev) if self.n_pix else None
        st = self.ctx._lib.sed_forward(self.ctx._h, self.id, C.c_void_p(theta.data_ptr()), n, ld,
                                       None if phot is None else C.c_void_p(phot.data_ptr()),
                                       None if spec is None else C.c_void_p(spec.data_ptr()),
                                       _prec(precision), _stream_handle(stream))
        self.ctx._check(st)
        return phot, spec

    def loglike(self, theta: torch.Tensor, precision="fp32", stream=None, out=None, status=None):
        n, ld = self._theta(theta)
        lnl = out if out is not None else torch.empty(n, dtype=torch.float64, device=theta.device)
        stt = status if status is not None else torch.empty(n, dtype=torch.int32, device=theta.device)
        st = self.ctx._lib.sed_loglike(self.ctx._h, self.id, C.c_void_p(theta.data_ptr()), n, ld,
                                       C.c_void_p(lnl.data_ptr()), C.c_void_p(stt.data_ptr()),
                                       _prec(precision), _stream_handle(stream))
        self.ctx._check(st)
        return lnl, stt

    def line_fluxes(self, theta: torch.Tensor, precision="fp32", stream=None):
        """Observer-frame fluxes of the grid's emission lines, erg/s/cm^2, as a
        CUDA float32 tensor [n, n_line] (sed_line_fluxes)."""
        n, ld = self._theta(theta)
        n_line = self.ctx.__dict__.get("_n_line", {}).get(self.id)
        if n_line is None:
            raise ValueError("line_fluxes needs the model's grid line count (create the model through Context)")
        out = torch.empty((n, n_line), dtype=torch.float32, device=theta.device)
        st = self.ctx._lib.sed_line_fluxes(self.ctx._h, self.id, C.c_void_p(theta.data_ptr()), n, ld,
                                           C.c_void_p(out.data_ptr()), _prec(precision), _stream_handle(stream))
        self.ctx._check(st)
        return out

    def loglike_noalloc(self, theta: torch.Tensor, precision="fp32", stream=None, out=None, status=None):
        """sed_loglike_noalloc: the same lnL and row status as loglike, with every
        intermediate buffer taken from the library's fixed device scratch array
        (no device allocation by the library; calls on different streams must
        not overlap)."""
        n, ld = self._theta(theta)
        lnl = out if out is not None else torch.empty(n, dtype=torch.float64, device=theta.device)
        stt = status if status is not None else torch.empty(n, dtype=torch.int32, device=theta.device)
        st = self.ctx._lib.sed_loglike_noalloc(self.ctx._h, self.id, C.c_void_p(theta.data_ptr()), n, ld,
                                               C.c_void_p(lnl.data_ptr()), C.c_void_p(stt.data_ptr()),
                                               _prec(precision), _stream_handle(stream))
        self.ctx._check(st)
        return lnl, stt

    def loglike_grad(self, theta: torch.Tensor, precision="fp32", stream=None, out=None):
        """lnL [n] (FP64), dlnL/dtheta [n, ld] (FP32) and row status [n]; `out` may
        give the three output tensors."""
        n, ld = self._theta(theta)
        if out is not None:
            lnl, grad, stt = out
        else:
            lnl = torch.empty(n, dtype=torch.float64, device=theta.device)
            grad = torch.empty((n, ld), dtype=torch.float32, device=theta.device)
            stt = torch.empty(n, dtype=torch.int32, device=theta.device)
        st = self.ctx._lib.sed_loglike_grad(self.ctx._h, self.id, C.c_void_p(theta.data_ptr()), n, ld,
                                            C.c_void_p(lnl.data_ptr()), C.c_void_p(grad.data_ptr()),
                                            C.c_void_p(stt.data_ptr()), _prec(precision),
                                            _stream_handle(stream))
        self.ctx._check(st)
        return lnl, grad, stt

    def loglike_host(self, theta: np.ndarray, precision="fp32", stream=None, out=None, status=None):
        """theta: host float32 [n, ld] (pinned memory recommended); returns host arrays."""
        th = np.ascontiguousarray(theta, dtype=np.float32) if not isinstance(theta, torch.Tensor) else theta
        if isinstance(th, torch.Tensor):
            n, ld = th.shape[0], th.stride(0)
            tp = th.data_ptr()
        else:
            n, ld = th.shape
            tp = th.ctypes.data
        lnl = out if out is not None else np.empty(n, dtype=np.float64)
        stt = status if status is not None else np.empty(n, dtype=np.uint32)
        lp = lnl.data_ptr() if isinstance(lnl, torch.Tensor) else lnl.ctypes.data
        sp = stt.data_ptr() if isinstance(stt, torch.Tensor) else stt.ctypes.data
        st = self.ctx._lib.sed_loglike_host(self.ctx._h, self.id, C.c_void_p(tp), n, ld, C.c_void_p(lp),
                                            C.c_void_p(sp), _prec(precision), _stream_handle(stream))
        self.ctx._check(st)
        return lnl, stt

    def nss(self, lo, hi, n_live=300, n_replace=64, n_slice_steps=40, max_iter=20000, stop_dlnz=-5.0,
            slice_width=0.0, seed=1, precision="fp32", max_dead=None, stream=None):
        """Nested slice sampling of this model's likelihood over the box prior
        [lo, hi] of each parameter column (sed_nss_run).  Returns a dict with
        lnz, info_h, n_iter, converged, n_like, n_rows, and the dead points
        (removed points, then the final live points): theta [n_dead, n_param],
        lnl, logw (ln posterior weights) and ins_rank (insertion ranks of the
        replacements)."""
        lo, hi = _f64(lo), _f64(hi)
        if lo.size != self.n_param or hi.size != self.n_param:
            raise ValueError(f"lo/hi need {self.n_param} entries")
        d = _ffi.NssDesc()
        d.n_live, d.n_replace, d.n_slice_steps, d.max_iter = n_live, n_replace, n_slice_steps, max_iter
        d.stop_dlnz, d.slice_width, d.seed, d.precision = stop_dlnz, slice_width, seed, _prec(precision)
        d.lo, d.hi = _ptr(lo), _ptr(hi)
        cap = int(max_dead) if max_dead is not None else n_live + max_iter * n_replace
        th = np.empty((cap, self.n_param), dtype=np.float32)
        lnl = np.empty(cap, dtype=np.float64)
        logw = np.empty(cap, dtype=np.float64)
        rank = np.empty(cap, dtype=np.int32)
        res = _ffi.NssResult()
        st = self.ctx._lib.sed_nss_run(self.ctx._h, self.id, C.byref(d), C.c_void_p(th.ctypes.data),
                                       C.c_void_p(lnl.ctypes.data), C.c_void_p(logw.ctypes.data),
                                       C.c_void_p(rank.ctypes.data), cap, C.byref(res), _stream_handle(stream))
        self.ctx._check(st)
        nd = res.n_dead
        return dict(lnz=res.lnz, info_h=res.info_h, n_iter=res.n_iter, converged=bool(res.converged),
                    n_like=res.n_like, n_rows=res.n_rows, theta=th[:nd], lnl=lnl[:nd], logw=logw[:nd],
                    ins_rank=rank[:res.n_iter * n_replace])


class Server:
    """Continuous-batching server of log-likelihood calls over many fits that
    share one grid (sed_server_* in include/sed.h)."""

    def __init__(self, ctx: Context, grid_id: int, layout_model: "Model", precision="bf16",
                 max_launch_rows=8192, n_slots=3, fit_budget_bytes=0):
        self.ctx = ctx
        self._lib = ctx._lib
        d = _ffi.ServerDesc(grid_id, layout_model.id, _prec(precision), int(max_launch_rows), int(n_slots),
                            int(fit_budget_bytes))
        h = C.c_void_p()
        ctx._check(self._lib.sed_server_create(ctx._h, C.byref(d), C.byref(h)))
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            self._lib.sed_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def open_fit(self, model: "Model", max_rows: int):
        """Fit id, or None when the fit budget is full (SED_EBUSY: retry later)."""
        f = C.c_int()
        st = self._lib.sed_server_open_fit(self._h, model.id, int(max_rows), C.byref(f))
        if st == _ffi.SED_EBUSY:
            return None
        self.ctx._check(st)
        return f.value

    def close_fit(self, fit: int):
        self.ctx._check(self._lib.sed_server_close_fit(self._h, int(fit)))

    def fit_theta_ptr(self, fit: int) -> int:
        return self._lib.sed_server_fit_theta(self._h, int(fit)) or 0

    def submit(self, fit: int, theta: np.ndarray) -> int:
        th = np.ascontiguousarray(theta, dtype=np.float32)
        t = C.c_uint64()
        self.ctx._check(self._lib.sed_server_submit(self._h, int(fit), C.c_void_p(th.ctypes.data), th.shape[0],
                                                    th.shape[1], C.byref(t)))
        return t.value

    def submit_device(self, fit: int, n: int) -> int:
        t = C.c_uint64()
        self.ctx._check(self._lib.sed_server_submit_device(self._h, int(fit), int(n), C.byref(t)))
        return t.value

    def wait(self, ticket: int, n: int, timeout_ms: int = -1):
        """(lnL [n] float64, row status [n] uint32, latency in ms)."""
        lnl = np.empty(n, dtype=np.float64)
        st = np.empty(n, dtype=np.uint32)
        lat = C.c_double()
        self.ctx._check(self._lib.sed_server_wait(self._h, C.c_uint64(ticket), C.c_void_p(lnl.ctypes.data),
                                                  C.c_void_p(st.ctypes.data), int(timeout_ms), C.byref(lat)))
        return lnl, st, lat.value

    def stats(self):
        s = _ffi.ServerStats()
        self.ctx._check(self._lib.sed_server_get_stats(self._h, C.byref(s)))
        return {f: getattr(s, f) for f, _ in s._fields_}


class SedLogLike(torch.autograd.Function):
    """lnL(theta) with the library's hand-written adjoint as the backward."""

    @staticmethod
    def forward(ctx, theta, model: Model, precision="fp32"):
        if theta.requires_grad:
            lnl, grad, st = model.loglike_grad(theta.detach().contiguous(), precision)
            ctx.save_for_backward(grad)
        else:
            lnl, st = model.loglike(theta.detach().contiguous(), precision)
            ctx.save_for_backward(None)
        return lnl

    @staticmethod
    def backward(ctx, g):
        (grad,) = ctx.saved_tensors
        return (g[:, None].to(grad.dtype) * grad, None, None)
