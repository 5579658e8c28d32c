"""FP64 CPU oracle of the SED forward model + Gaussian log-likelihood.

TEST INFRASTRUCTURE ONLY.  Only the test suite, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this package.  It shares no
code with the GPU library (``paper_2609_30145_gb300``); both consume the seeded
inputs of ``synth``.

``build()`` compiles ``oracle.c`` with gcc (OpenMP) into ``_build/liboracle.so``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_build", "liboracle.so")
_lib = None

BAD_THETA, BAD_Z, BAD_TMAX, NONFINITE = 1, 2, 4, 16


def build(force=False):
    src = os.path.join(_HERE, "oracle.c")
    if (not force and os.path.exists(_SO)
            and os.path.getmtime(_SO) >= max(os.path.getmtime(src),
                                              os.path.getmtime(os.path.join(_HERE, "oracle.h")))):
        return _SO
    os.makedirs(os.path.dirname(_SO), exist_ok=True)
    tmp = _SO + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared",
                           "-D_DEFAULT_SOURCE", "-o", tmp, src, "-lm"])
    os.replace(tmp, _SO)
    return _SO


class _Grid(C.Structure):
    _fields_ = [("n_age", C.c_int), ("n_feh", C.c_int), ("n_afe", C.c_int), ("n_lam", C.c_int),
                ("log_age_yr", C.c_void_p), ("feh", C.c_void_p), ("afe", C.c_void_p),
                ("lam", C.c_void_p), ("flux", C.c_void_p), ("sigma_lib_kms", C.c_void_p),
                ("neb_n_logu", C.c_int), ("neb_n_logz", C.c_int),
                ("neb_logu", C.c_void_p), ("neb_logz", C.c_void_p), ("neb_tab", C.c_void_p),
                ("neb_n_line", C.c_int), ("neb_line_lam", C.c_void_p), ("neb_line_tab", C.c_void_p),
                ("neb_n_age", C.c_int), ("neb_log_age", C.c_void_p)]


class _Model(C.Structure):
    _fields_ = [("n_sfh", C.c_int), ("zf", C.c_double), ("zmode", C.c_int),
                ("use_afe", C.c_int), ("use_nebular", C.c_int), ("dust_law", C.c_int),
                ("bc_edge_log_age_yr", C.c_double), ("H0", C.c_double), ("Om0", C.c_double),
                ("n_filt", C.c_int), ("filt_len", C.c_void_p), ("filt_lam", C.c_void_p),
                ("filt_trans", C.c_void_p), ("phot_d", C.c_void_p), ("phot_sigma", C.c_void_p),
                ("phot_mask", C.c_void_p), ("n_pix", C.c_int), ("spec_lam", C.c_void_p),
                ("spec_d", C.c_void_p), ("spec_sigma", C.c_void_p), ("spec_mask", C.c_void_p),
                ("lsf_mode", C.c_int), ("lsf_value", C.c_void_p),
                ("sigma_gal_kms", C.c_double), ("z_ref", C.c_double),
                ("sample_sigma_gal", C.c_int), ("sigma_gal_max_kms", C.c_double),
                ("calib_n", C.c_int), ("calib_sigma", C.c_void_p),
                ("sfh_scheme", C.c_int), ("floor_phot", C.c_int), ("floor_spec", C.c_int),
                ("phot_upper", C.c_void_p), ("fesc_geometry", C.c_int), ("calib_mode", C.c_int),
                ("use_lines", C.c_int), ("gas_sigma_mode", C.c_int), ("sigma_gas_kms", C.c_double),
                ("sigma_gas_max_kms", C.c_double), ("n_lcat", C.c_int), ("lcat_start", C.c_void_p),
                ("lcat_line", C.c_void_p), ("lcat_d", C.c_void_p), ("lcat_sigma", C.c_void_p),
                ("lcat_mask", C.c_void_p), ("lcat_upper", C.c_void_p), ("dust_n_bin", C.c_int),
                ("dust_bin_M", C.c_void_p), ("dust_bin_law", C.c_void_p), ("use_igm", C.c_int)]


def _load():
    global _lib
    if _lib is None:
        build()
        lib = C.CDLL(_SO)
        P = C.c_void_p
        lib.orc_cosmology.argtypes = [C.c_double, C.c_double, C.c_double, P]
        lib.orc_sfh_edges.argtypes = [C.c_int, C.c_double, P]
        lib.orc_weights.argtypes = [P, P, P, P]
        lib.orc_weights.restype = C.c_int
        lib.orc_q.argtypes = [P, P]
        lib.orc_dust_tau.argtypes = [C.c_int, P, C.c_int, C.c_double, C.c_double, P]
        lib.orc_photometry.argtypes = [P, P, C.c_int, C.c_double, P, P]
        lib.orc_spectrum.argtypes = [P, P, P, C.c_int, C.c_double, C.c_double, P, P, P]
        lib.orc_row.argtypes = [P, P, P, P, P, P, P, P, P, P, P]
        lib.orc_row.restype = C.c_int
        lib.orc_eval.argtypes = [P, P, P, C.c_int, C.c_int, P, P, P, P, C.c_int]
        lib.orc_line_fluxes.argtypes = [P, P, P, C.c_int, C.c_int, P]
        lib.orc_grad_fd.argtypes = [P, P, P, C.c_int, C.c_int, C.c_double, P, C.c_int]
        lib.orc_grad.argtypes = [P, P, P, C.c_int, C.c_int, P, P, P, C.c_int]
        lib.orc_n_param.argtypes = [P]
        lib.orc_igm_tau.argtypes = [P, C.c_int, C.c_double, P]
        lib.orc_n_param.restype = C.c_int
        _lib = lib
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


PHYS = dict(H0=67.66, Om0=0.3097, bc_edge_log_age_yr=7.03)


@dataclass
class Oracle:
    """Holds the grid and one model (fit) description; arrays are kept alive here."""

    grid: object
    n_sfh: int
    zf: float
    zmode: int
    use_afe: int = 0
    use_nebular: int = 0
    dust_law: int = 0
    filters: tuple | None = None     # (lens, lam, trans)
    phot_d: np.ndarray | None = None
    phot_sigma: np.ndarray | None = None
    phot_mask: np.ndarray | None = None
    phot_upper: np.ndarray | None = None   # nonzero: the band's datum is an upper limit (Eq. app_line_chi2_UL)
    spec_lam: np.ndarray | None = None
    spec_d: np.ndarray | None = None
    spec_sigma: np.ndarray | None = None
    spec_mask: np.ndarray | None = None
    lsf_mode: int = 0
    lsf_value: np.ndarray | None = None
    sigma_gal_kms: float = 0.0
    z_ref: float = 0.0
    sample_sigma_gal: int = 0           # 1: sigma_gal (km/s) is the last parameter column
    sigma_gal_max_kms: float = 1000.0   # sampled sigma_gal must lie in [0, this]
    calib_sigma: np.ndarray | None = None   # prior widths s_m of the calibration polynomial's coefficients
    calib_mode: int = 0                 # 0 marginalised (Eq. app_polymarg), 1 optimised at each call
    use_lines: int = 0                  # 1: the grid's emission lines enter photometry and spectrum (App. C)
    gas_sigma_mode: int = 0             # GAS_SIGMA_TIED (= sigma_gal), _FIXED (sigma_gas_kms) or _SAMPLED (last column)
    sigma_gas_kms: float = 300.0
    sigma_gas_max_kms: float = 1000.0
    lcat: tuple | None = None           # line catalogue (Sec. 3.3): (blends: list of lists of grid-line
                                        # indices, d, sigma, mask or None, upper or None), erg/s/cm^2
    sfh_scheme: int = 0                 # 0 step (N_T bin masses), 1 linear (N_T + 1 edge SFRs; App. B)
    use_igm: int = 0                    # 1: Madau (1995) IGM transmission, scaled by the last column (igm_factor)
    dust_bins: tuple | None = None      # age-binned attenuation (App. "dust_attn"): (M [n_age][n_bin], laws
                                        # [n_bin], 0 power law / 1 KC13); adds 2 n_bin columns at the row's end
    floor_phot: int = 0                 # noise-floor terms of each arm (App. sys_floor): FLOOR_* bits
    floor_spec: int = 0
    fesc_geometry: int = 0              # ionising-photon escape (Sec. frac_obrun): FESC_*; adds the frac_obrun column
    H0: float = PHYS["H0"]
    Om0: float = PHYS["Om0"]
    bc_edge_log_age_yr: float = PHYS["bc_edge_log_age_yr"]

    def __post_init__(self):
        self._lib = _load()
        g = self.grid
        self._keep = []

        def k(a, dt=np.float64):
            if a is None:
                return None
            a = np.ascontiguousarray(a, dtype=dt)
            self._keep.append(a)
            return a
        self._g = _Grid()
        self._g.n_afe, self._g.n_feh, self._g.n_age, self._g.n_lam = g.flux.shape
        self._g.log_age_yr = _p(k(g.log_age_yr))
        self._g.feh = _p(k(g.feh))
        self._g.afe = _p(k(g.afe))
        self._g.lam = _p(k(g.lam_aa))
        self._g.flux = _p(k(g.flux))
        self._g.sigma_lib_kms = _p(k(getattr(g, "sigma_lib_kms", None)))
        if g.neb_tab is not None:
            na = getattr(g, "neb_log_age", None)
            if na is not None:   # nebular age axis: neb_tab [n_age][n_logu][n_logz][n_lam]
                self._g.neb_n_age = len(na)
                self._g.neb_log_age = _p(k(na))
                self._g.neb_n_logu, self._g.neb_n_logz = g.neb_tab.shape[1:3]
            else:
                self._g.neb_n_logu, self._g.neb_n_logz = g.neb_tab.shape[:2]
            self._g.neb_logu = _p(k(g.neb_logu))
            self._g.neb_logz = _p(k(g.neb_logz))
            self._g.neb_tab = _p(k(g.neb_tab))
            if getattr(g, "line_tab", None) is not None:
                self._g.neb_n_line = g.line_tab.shape[2]
                self._g.neb_line_lam = _p(k(g.line_lam))
                self._g.neb_line_tab = _p(k(g.line_tab))
        self._rebuild_model()

    def _rebuild_model(self):
        def k(a, dt=np.float64):
            if a is None:
                return None
            a = np.ascontiguousarray(a, dtype=dt)
            self._keep.append(a)
            return a
        m = _Model()
        m.n_sfh, m.zf, m.zmode = self.n_sfh, self.zf, self.zmode
        m.use_afe, m.use_nebular, m.dust_law = self.use_afe, self.use_nebular, self.dust_law
        m.bc_edge_log_age_yr, m.H0, m.Om0 = self.bc_edge_log_age_yr, self.H0, self.Om0
        if self.filters is not None:
            lens, lam, tr = self.filters
            m.n_filt = len(lens)
            m.filt_len = _p(k(lens, np.int32))
            m.filt_lam = _p(k(lam))
            m.filt_trans = _p(k(tr))
            m.phot_d = _p(k(self.phot_d))
            m.phot_sigma = _p(k(self.phot_sigma))
            m.phot_mask = _p(k(self.phot_mask, np.uint8))
            m.phot_upper = _p(k(self.phot_upper, np.uint8))
        if self.spec_lam is not None:
            m.n_pix = len(self.spec_lam)
            m.spec_lam = _p(k(self.spec_lam))
            m.spec_d = _p(k(self.spec_d))
            m.spec_sigma = _p(k(self.spec_sigma))
            m.spec_mask = _p(k(self.spec_mask, np.uint8))
            m.lsf_mode = self.lsf_mode
            m.lsf_value = _p(k(self.lsf_value))
            m.sigma_gal_kms, m.z_ref = self.sigma_gal_kms, self.z_ref
        m.sample_sigma_gal, m.sigma_gal_max_kms = int(self.sample_sigma_gal), float(self.sigma_gal_max_kms)
        if self.calib_sigma is not None and self.spec_lam is not None:
            m.calib_n = len(self.calib_sigma)
            m.calib_sigma = _p(k(self.calib_sigma))
            if self.floor_spec:
                raise ValueError("a spectral noise floor with the marginalised calibration polynomial is not defined here")
        m.floor_phot, m.floor_spec = int(self.floor_phot), int(self.floor_spec)
        m.sfh_scheme = int(self.sfh_scheme)
        m.fesc_geometry = int(self.fesc_geometry)
        m.calib_mode = int(self.calib_mode)
        m.use_lines = int(self.use_lines)
        m.gas_sigma_mode = int(self.gas_sigma_mode)
        m.sigma_gas_kms, m.sigma_gas_max_kms = float(self.sigma_gas_kms), float(self.sigma_gas_max_kms)
        if self.lcat is not None:
            blends, d, s, mask, upper = self.lcat
            start = np.concatenate([[0], np.cumsum([len(b) for b in blends])]).astype(np.int32)
            m.n_lcat = len(blends)
            m.lcat_start = _p(k(start, np.int32))
            m.lcat_line = _p(k(np.concatenate([np.asarray(b, dtype=np.int32) for b in blends]), np.int32))
            m.lcat_d, m.lcat_sigma = _p(k(d)), _p(k(s))
            m.lcat_mask = _p(k(mask, np.uint8))
            m.lcat_upper = _p(k(upper, np.uint8))
        if self.dust_bins is not None:
            M, laws = self.dust_bins
            M = np.asarray(M, dtype=np.float64)
            if M.ndim != 2 or M.shape[0] != self.grid.flux.shape[2] or not 1 <= M.shape[1] <= 4:
                raise ValueError("dust_bins: M must be [n_age][n_bin], 1 <= n_bin <= 4")
            sums = M.sum(axis=1)
            if np.any(M < 0) or np.any(M > 1) or not np.all((np.abs(sums - 1) < 1e-9) | (sums == 0)):
                raise ValueError("dust_bins: rows of M in [0, 1] summing to 1 or all zero")
            if self.use_lines or self.fesc_geometry:
                raise ValueError("dust_bins: not combined with emission lines or an escape geometry")
            m.dust_n_bin = M.shape[1]
            m.dust_bin_M = _p(k(M))
            m.dust_bin_law = _p(k(np.asarray(laws), np.int32))
        m.use_igm = int(self.use_igm)
        na = getattr(self.grid, "neb_log_age", None)
        if na is not None and self.use_nebular:
            la = np.asarray(self.grid.log_age_yr)
            inside = (la >= na[0]) & (la <= na[-1])
            if np.any(la[inside] > self.bc_edge_log_age_yr):
                raise ValueError("nebular age axis: the cube's ages reach past the birth-cloud edge")
            if self.use_lines or self.fesc_geometry or self.dust_bins is not None:
                raise ValueError("nebular age axis: not combined with emission lines, an escape geometry or "
                                 "age-binned dust")
        self._m = m

    def set_data(self, phot_d=None, phot_sigma=None, spec_d=None, spec_sigma=None):
        if phot_d is not None:
            self.phot_d, self.phot_sigma = phot_d, phot_sigma
        if spec_d is not None:
            self.spec_d, self.spec_sigma = spec_d, spec_sigma
        self._rebuild_model()

    # ---------------------------------------------------------------
    @property
    def n_param(self):
        return self._lib.orc_n_param(C.byref(self._m))

    @property
    def n_filt(self):
        return self._m.n_filt

    @property
    def n_pix(self):
        return self._m.n_pix

    def eval(self, theta, nthreads=0):
        th = np.ascontiguousarray(theta, dtype=np.float64)
        n, ld = th.shape
        phot = np.zeros((n, max(self.n_filt, 1)))
        spec = np.zeros((n, max(self.n_pix, 1)))
        lnl = np.zeros(n)
        st = np.zeros(n, dtype=np.int32)
        self._lib.orc_eval(C.byref(self._g), C.byref(self._m), _p(th), n, ld,
                           _p(phot) if self.n_filt else None, _p(spec) if self.n_pix else None,
                           _p(lnl), _p(st), int(nthreads))
        return dict(phot=phot[:, :self.n_filt], spec=spec[:, :self.n_pix], lnl=lnl, status=st)

    def row(self, theta_row):
        th = np.ascontiguousarray(theta_row, dtype=np.float64)
        g = self.grid
        nsp = g.flux.shape[0] * g.flux.shape[1] * g.flux.shape[2]
        nl = g.flux.shape[3]
        W = np.zeros(nsp)
        Y, O, F, fnu = (np.zeros(nl) for _ in range(4))
        phot = np.zeros(max(self.n_filt, 1))
        spec = np.zeros(max(self.n_pix, 1))
        scal = np.zeros(6)
        st = self._lib.orc_row(C.byref(self._g), C.byref(self._m), _p(th), _p(W), _p(Y), _p(O),
                               _p(F), _p(fnu), _p(phot), _p(spec), _p(scal))
        return dict(status=st, W=W.reshape(g.flux.shape[:3]), Y=Y, O=O, F=F, fnu=fnu,
                    phot=phot[:self.n_filt], spec=spec[:self.n_pix], D_L=scal[0], t_univ=scal[1],
                    T_max=scal[2], Q_young=scal[3], scale=scal[4], lnl=scal[5])

    def weights(self, theta_row):
        th = np.ascontiguousarray(theta_row, dtype=np.float64)
        g = self.grid
        W = np.zeros(g.flux.shape[:3])
        st = self._lib.orc_weights(C.byref(self._g), C.byref(self._m), _p(th), _p(W))
        return st, W

    def q(self):
        g = self.grid
        Q = np.zeros(g.flux.shape[:3])
        self._lib.orc_q(C.byref(self._g), _p(Q))
        return Q

    def photometry(self, lam_rest, fnu_obs, z):
        lam_rest, fnu_obs = _f64(lam_rest), _f64(fnu_obs)
        out = np.zeros(self.n_filt)
        self._lib.orc_photometry(C.byref(self._m), _p(lam_rest), lam_rest.size, float(z),
                                 _p(fnu_obs), _p(out))
        return out

    def spectrum(self, lam_rest, fnu_obs, z, sigma_gal_kms=None):
        """App. E projection of an observer-frame F_nu sampled at rest-frame
        lam_rest onto the pixels; sigma_gal defaults to the model's fixed value."""
        lam_rest, fnu_obs = _f64(lam_rest), _f64(fnu_obs)
        out = np.zeros(self.n_pix)
        valid = np.zeros(self.n_pix, dtype=np.uint8)
        sg = self.sigma_gal_kms if sigma_gal_kms is None else sigma_gal_kms
        self._lib.orc_spectrum(C.byref(self._g), C.byref(self._m), _p(lam_rest), lam_rest.size,
                               float(z), float(sg), _p(fnu_obs), _p(out), _p(valid))
        return out, valid

    def line_fluxes(self, theta):
        """Observer-frame integrated flux of every grid line [n][n_line], erg/s/cm^2."""
        th = np.ascontiguousarray(theta, dtype=np.float64)
        n, ld = th.shape
        nl = self._g.neb_n_line
        out = np.zeros((n, max(nl, 1)))
        self._lib.orc_line_fluxes(C.byref(self._g), C.byref(self._m), _p(th), n, ld, _p(out))
        return out[:, :nl]

    def grad(self, theta, nthreads=0):
        """Analytic FP64 gradient of lnL: dict(lnl [n], grad [n][n_param], status [n])."""
        if (self.use_lines or self.lcat is not None or self.dust_bins is not None or self.use_igm
                or getattr(self.grid, "neb_log_age", None) is not None):
            raise NotImplementedError("the analytic gradient does not cover emission lines, age-binned dust or the "
                                      "IGM: use grad_fd")
        th = np.ascontiguousarray(theta, dtype=np.float64)
        n, ld = th.shape
        out = np.zeros((n, ld))
        lnl = np.zeros(n)
        st = np.zeros(n, dtype=np.int32)
        self._lib.orc_grad(C.byref(self._g), C.byref(self._m), _p(th), n, ld, _p(lnl), _p(out), _p(st),
                           int(nthreads))
        return dict(lnl=lnl, grad=out, status=st)

    def grad_fd(self, theta, h_rel=1e-6, nthreads=0):
        th = np.ascontiguousarray(theta, dtype=np.float64)
        n, ld = th.shape
        out = np.zeros((n, ld))
        self._lib.orc_grad_fd(C.byref(self._g), C.byref(self._m), _p(th), n, ld, float(h_rel),
                              _p(out), int(nthreads))
        return out


def cosmology(H0, Om0, z):
    lib = _load()
    out = np.zeros(3)
    lib.orc_cosmology(float(H0), float(Om0), float(z), _p(out))
    return dict(D_L=out[0], t_univ=out[1], D_C=out[2])


def sfh_edges(n_sfh, tmax_yr):
    lib = _load()
    T = np.zeros(n_sfh + 1)
    lib.orc_sfh_edges(int(n_sfh), float(tmax_yr), _p(T))
    return T


def dust_tau(law, lam, tau, index):
    lib = _load()
    lam = _f64(lam)
    out = np.zeros(lam.size)
    lib.orc_dust_tau(int(law), _p(lam), lam.size, float(tau), float(index), _p(out))
    return out


FLOOR_ERR_SCALE, FLOOR_F_CALIB, FLOOR_F_DATA, FLOOR_JITTER = 1, 2, 4, 8
FESC_NONE, FESC_RUNAWAY_BC, FESC_PICKET = 0, 1, 2
GAS_SIGMA_TIED, GAS_SIGMA_FIXED, GAS_SIGMA_SAMPLED = 0, 1, 2
FLOOR_NAMES = ("log_err_scale", "log_f_calib", "log_f_data", "log_jitter")


def igm_tau(lam_rest, z):
    """Madau (1995) IGM optical depth (factor 1) at the rest wavelengths lam_rest
    (Angstrom) of a source at redshift z."""
    lib = _load()
    lam = np.ascontiguousarray(lam_rest, dtype=np.float64)
    out = np.zeros(lam.size)
    lib.orc_igm_tau(_p(lam), lam.size, float(z), _p(out))
    return out


def floor_keys(floor_phot=0, floor_spec=0):
    """Column names of the noise-floor terms that are on, in the row's order."""
    return tuple(f"{FLOOR_NAMES[k]}_{arm}" for arm, bits in (("phot", floor_phot), ("spec", floor_spec))
                 for k in range(4) if (bits >> k) & 1)


def pack_theta(d, n_sfh, zmode, sample_sigma_gal=0, floor_phot=0, floor_spec=0, sfh_scheme=0, fesc_geometry=0,
               sample_sigma_gas=0, dust_n_bin=0, use_igm=0):
    """Parameter rows in the oracle's layout: sfh[N_T] (bin masses; N_T + 1 edge
    SFRs with the linear scheme), logzsol[N_T or 1], then
    afe, logmass, zred, tau_pow, alpha_pow, diffuse_tau_kc, diffuse_dust_index,
    gas_logz, gas_logu, sigma_gal when the model samples it, and the log10 of
    each noise-floor term that is on (photometry, then spectrum), and frac_obrun
    with an escape geometry, sigma_gas when the model samples the gas dispersion, and
    with age-binned dust the 2 n_bin columns of d["dust_bins"] (tau_b, slope_b of each bin), and
    with the IGM its scaling igm_factor."""
    nz = n_sfh if zmode == 0 else 1
    n = d["sfh"].shape[0]
    cols = [np.asarray(d["sfh"], dtype=np.float64).reshape(n, n_sfh + (1 if sfh_scheme == 1 else 0)),
            np.asarray(d["logzsol"], dtype=np.float64).reshape(n, nz)]
    for k in ("afe", "logmass", "zred", "tau_pow", "alpha_pow", "diffuse_tau_kc",
              "diffuse_dust_index", "gas_logz", "gas_logu") + (("sigma_gal",) if sample_sigma_gal else ()) + \
            floor_keys(floor_phot, floor_spec) + (("frac_obrun",) if fesc_geometry else ()) + \
            (("sigma_gas",) if sample_sigma_gas else ()):
        cols.append(np.asarray(d[k], dtype=np.float64).reshape(n, 1))
    if dust_n_bin:
        cols.append(np.asarray(d["dust_bins"], dtype=np.float64).reshape(n, 2 * dust_n_bin))
    if use_igm:
        cols.append(np.asarray(d["igm_factor"], dtype=np.float64).reshape(n, 1))
    return np.ascontiguousarray(np.concatenate(cols, axis=1))
