"""Seeded synthetic inputs for the SED forward model and likelihood.

This module produces *data only*: SSP grids, nebular templates, filter curves,
spectrum pixel grids with their resolution curves, parameter batches and noise
draws.  It holds none of the method's arithmetic (no weights, no contraction,
no attenuation, no projection, no likelihood), so both the CPU oracle and the
GPU library can consume its output without sharing any code of the method.

The real inputs of the paper (FSPS/BPASS/MIST/C3K SSP grids, the Byler et al.
nebular grids, sedpy/NIRCam filter curves, JADES catalogues) are not available
here.  The stand-ins below copy their *shapes*: grid sizes and axis ranges,
dynamic range of the SSP fluxes, filter widths and counts, spectrum lengths and
resolution curves, and the parameter ranges of the paper's priors.

Every generator takes an explicit integer seed and uses numpy's PCG64 bit
generator with `random()` / `standard_normal()` draws only.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

C_KMS = 299792.458

# Names of the scalar parameter columns that follow the SFH and metallicity
# blocks of a parameter row, in order (paper key names, Fig. "ceridwen_flow").
SCALAR_KEYS = ("afe", "logmass", "zred", "tau_pow", "alpha_pow",
               "diffuse_tau_kc", "diffuse_dust_index", "gas_logz", "gas_logu", "sigma_gal")


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


# --------------------------------------------------------------------------
# SSP grid
# --------------------------------------------------------------------------
@dataclass
class Grid:
    log_age_yr: np.ndarray          # [n_age] strictly increasing
    feh: np.ndarray                 # [n_feh]
    afe: np.ndarray                 # [n_afe] (length 1 for 3-D grids)
    lam_aa: np.ndarray              # [n_lam] rest-frame wavelengths, Angstrom
    flux: np.ndarray                # [n_afe][n_feh][n_age][n_lam] Lsun/Hz per Msun formed
    neb_logu: np.ndarray | None = None
    neb_logz: np.ndarray | None = None
    neb_tab: np.ndarray | None = None   # [n_logu][n_logz][n_lam] log10(L_nu/Q), (Lsun/Hz)/(photon/s)
    line_lam: np.ndarray | None = None  # [n_line] rest-frame wavelengths of the emission-line cube, Angstrom
    line_tab: np.ndarray | None = None  # [n_logu][n_logz][n_line] log10(L_line/Q), Lsun/(photon/s)
    neb_log_age: np.ndarray | None = None  # nebular age axis (log10 yr): neb_tab is then [n_age][n_logu][n_logz][n_lam]

    @property
    def shape(self):
        return self.flux.shape


def make_grid(n_age=16, log_age=(6.0, 10.1), feh=(-2.0, 0.2), n_feh=4,
              afe_nodes=None, n_lam=512, lam_um=(0.1, 5.0), nebular=None,
              seed=1) -> Grid:
    """Blackbody-like SSP spectra with lognormal amplitudes and absorption dips.

    f = 1e-11 * A_am * B_nu(lam; T_am) / max * prod_k (1 - d_k exp(-((lam-lam_k)/w_k)^2/2))
    with T_am = 3e4 K * 10^(-0.35 (log age - 6)) * (1 + 0.05 [Fe/H]) * (1 - 0.03 [a/Fe]),
    log10 A spanning 0 .. -6 from the youngest to the oldest age plus 0.1 dex
    scatter, d_k in [0.05, 0.2], w_k in [5, 50] Angstrom, six dips per spectrum.
    """
    rng = _rng(seed)
    log_age_yr = np.linspace(log_age[0], log_age[1], n_age)
    feh_v = np.linspace(feh[0], feh[1], n_feh)
    afe_v = np.array([0.0]) if afe_nodes is None else np.asarray(afe_nodes, dtype=np.float64)
    lam = np.geomspace(lam_um[0] * 1e4, lam_um[1] * 1e4, n_lam)
    n_afe = afe_v.size
    h_over_k = 6.62607015e-27 / 1.380649e-16          # s K
    nu = 2.99792458e18 / lam                            # Hz
    flux = np.empty((n_afe, n_feh, n_age, n_lam))
    age_frac = (log_age_yr - log_age_yr[0]) / max(log_age_yr[-1] - log_age_yr[0], 1e-12)
    scatter = rng.standard_normal((n_afe, n_feh, n_age))
    dip_c = rng.random((n_afe, n_feh, n_age, 6))
    dip_d = rng.random((n_afe, n_feh, n_age, 6))
    dip_w = rng.random((n_afe, n_feh, n_age, 6))
    lo_l, hi_l = math.log(lam[0]), math.log(lam[-1])
    for n in range(n_afe):
        for m in range(n_feh):
            for a in range(n_age):
                T = 3e4 * 10 ** (-0.35 * (log_age_yr[a] - 6.0)) * (1 + 0.05 * feh_v[m]) \
                    * (1 - 0.03 * afe_v[n])
                x = h_over_k * nu / T
                with np.errstate(over="ignore", under="ignore"):
                    bb = x ** 3 * np.exp(-x) / -np.expm1(-x)
                bb = bb / bb.max()
                logA = -6.0 * age_frac[a] + 0.1 * scatter[n, m, a]
                shape = bb.copy()
                for k in range(6):
                    lc = math.exp(lo_l + (0.15 + 0.7 * dip_c[n, m, a, k]) * (hi_l - lo_l))
                    depth = (0.05 + 0.15 * dip_d[n, m, a, k]) * (1 + 0.5 * afe_v[n])
                    w = 5.0 + 45.0 * dip_w[n, m, a, k]
                    shape *= 1.0 - depth * np.exp(-0.5 * ((lam - lc) / w) ** 2)
                flux[n, m, a] = 1e-11 * 10 ** logA * shape
    g = Grid(log_age_yr=log_age_yr, feh=feh_v, afe=afe_v, lam_aa=lam, flux=flux)
    if nebular is not None:
        n_cube = nebular.get("line_cube", 0)
        # with a separate line cube the continuum template carries no lines
        g.neb_logu, g.neb_logz, g.neb_tab = make_nebular(lam, seed=nebular.get("seed", 2),
                                                        n_logu=nebular.get("n_logu", 7),
                                                        n_logz=nebular.get("n_logz", 12),
                                                        n_lines=0 if n_cube else 30)
        if n_cube:
            g.line_lam, g.line_tab = make_line_cube(g.neb_logu, g.neb_logz, n_cube, seed=nebular.get("seed", 2) + 10)
        if nebular.get("age_axis"):
            g.neb_log_age, g.neb_tab = nebular_age_axis(g.neb_tab, g.neb_logu, lam, *nebular["age_axis"],
                                                        seed=nebular.get("seed", 2) + 20)
    return g


def nebular_age_axis(tab, logu, lam, n_age, lo, hi, seed=22):
    """A nebular cube with an ionising-source age axis: n_age planes at log10
    ages lo..hi (yr), plane i = the age-free template dimmed by 0.8 dex per dex
    of age (the ionising output fading with age), with a seeded slope that
    steepens towards high log U and a seeded wavelength ripple of 0.05 dex; -99
    below 912 Angstrom as in the template."""
    rng = _rng(seed)
    ages = np.linspace(lo, hi, n_age)
    du = (np.asarray(logu) + 2.5)[:, None, None]
    ripple = 0.05 * np.sin(np.log(lam) * rng.uniform(5.0, 15.0) + rng.uniform(0, 2 * np.pi))[None, None, :]
    out = np.empty((n_age,) + tab.shape)
    for i, t in enumerate(ages):
        dt = t - lo
        plane = tab - 0.8 * dt - 0.2 * dt * du + dt * ripple
        plane[:, :, lam < 912.0] = -99.0
        out[i] = plane
    return ages, out


def make_line_cube(logu, logz, n_lines, seed=12, lam_aa=(1000.0, 22000.0)):
    """Emission-line cube log10(L_line/Q) in Lsun/(photon/s) on the nebular
    (log U, log Z_gas) axes: `n_lines` seeded rest wavelengths, log-uniform in
    lam_aa, sorted, and strengths around 1e-46 Lsun per ionising photon per
    second (an H-beta-like line is ~1.2e-46) times 0.1..3, varying linearly
    with log U and log Z_gas."""
    rng = _rng(seed)
    lam = np.sort(np.exp(np.log(lam_aa[0]) + rng.random(n_lines) * (np.log(lam_aa[1]) - np.log(lam_aa[0]))))
    base = -46.0 + np.log10(0.1 + 2.9 * rng.random(n_lines))
    su = 0.3 * (rng.random(n_lines) - 0.5)
    sz = 0.4 * (rng.random(n_lines) - 0.5)
    lu, lz = np.asarray(logu), np.asarray(logz)
    tab = base[None, None, :] + su[None, None, :] * (lu[:, None, None] + 2.5) + sz[None, None, :] * (lz[None, :, None] + 0.5)
    return lam, tab


def make_nebular(lam, seed=2, n_logu=7, n_logz=12, logu=(-4.0, -1.0), logz=(-1.3, 0.3),
                 n_lines=30):
    """log10(L_nu/Q) template on the SSP wavelength grid, in (Lsun/Hz)/(photon/s).

    A smooth continuum (level ~1e-60, i.e. nebular L_nu of a few per cent of a
    young population's stellar L_nu for the amplitudes of `make_grid`) plus
    `n_lines` seeded emission lines, each a Gaussian two model pixels wide whose
    strength varies linearly with log U and log Z_gas.  Set to -99 (no emission)
    below 912 Angstrom.
    """
    rng = _rng(seed)
    lu = np.linspace(logu[0], logu[1], n_logu)
    lz = np.linspace(logz[0], logz[1], n_logz)
    ll = np.log(lam)
    dll = np.gradient(ll)
    cont = -60.3 - 0.4 * (np.log10(lam) - 3.7)
    line_c = np.exp(np.log(1000.0) + rng.random(n_lines) * (np.log(2.2e4) - np.log(1000.0)))
    line_a = 0.5 + 1.5 * rng.random(n_lines)
    line_su = rng.random(n_lines) - 0.5
    line_sz = rng.random(n_lines) - 0.5
    tab = np.empty((n_logu, n_logz, lam.size))
    for iu in range(n_logu):
        for iz in range(n_logz):
            lin = np.zeros(lam.size)
            for k in range(n_lines):
                amp = line_a[k] * (1 + line_su[k] * (lu[iu] + 2.5) / 1.5) * (1 + line_sz[k] * (lz[iz] + 0.5))
                kc = np.searchsorted(lam, line_c[k])
                kc = min(max(kc, 1), lam.size - 2)
                width = 2.0 * dll[kc]
                lin += max(amp, 0.0) * 30.0 * np.exp(-0.5 * ((ll - math.log(line_c[k])) / width) ** 2)
            lin_cont = 1.0 + 0.05 * (lu[iu] + 2.5) - 0.04 * lz[iz]
            val = np.log10(10 ** cont * lin_cont * (1.0 + lin))
            val[lam < 912.0] = -99.0
            tab[iu, iz] = val
    return lu, lz, tab


# --------------------------------------------------------------------------
# Filters
# --------------------------------------------------------------------------
def make_filters_gauss(n=8, lo_um=0.6, hi_um=4.5, fwhm_frac=0.2, n_samp=200):
    """Gaussian bands, centres log-spaced, FWHM = fwhm_frac * centre, `n_samp`
    samples over +-3 sigma, transmission shifted so that it is 0 at both ends."""
    out = []
    for lc in np.geomspace(lo_um * 1e4, hi_um * 1e4, n):
        sig = fwhm_frac * lc / 2.3548200450309493
        lam = np.linspace(lc - 3 * sig, lc + 3 * sig, n_samp)
        tr = np.exp(-0.5 * ((lam - lc) / sig) ** 2) - math.exp(-4.5)
        tr = np.clip(tr, 0.0, None)
        tr[0] = tr[-1] = 0.0
        out.append((lam, tr))
    return out


def make_filters_nircam_like(n_wide=8, n_medium=12, lo_um=0.6, hi_um=5.0, n_samp=200, seed=3):
    """Flat-topped bands shaped like broad (R~4) and medium (R~10) imaging
    filters: a super-Gaussian core with a few per cent of seeded ripple, zero at
    both sample ends.  Not the real curves."""
    rng = _rng(seed)
    out = []
    cw = np.geomspace(lo_um * 1e4 * 1.25, hi_um * 1e4 / 1.15, n_wide)
    cm = np.geomspace(lo_um * 1e4 * 1.08, hi_um * 1e4 / 1.06, n_medium)
    for lc, R in [(c, 4.0) for c in cw] + [(c, 10.0) for c in cm]:
        half = 0.5 * lc / R
        lam = np.linspace(lc - 1.6 * half, lc + 1.6 * half, n_samp)
        x = (lam - lc) / half
        ph = rng.random() * 6.283
        tr = np.exp(-0.5 * x ** 8) * (0.85 + 0.03 * np.sin(9 * x + ph))
        tr -= tr[[0, -1]].max()
        tr = np.clip(tr, 0.0, None)
        tr[0] = tr[-1] = 0.0
        out.append((lam, tr))
    return out


def pack_filters(filters):
    """Concatenate filter curves: (lengths int32, lam float64, trans float64)."""
    lens = np.array([f[0].size for f in filters], dtype=np.int32)
    lam = np.concatenate([f[0] for f in filters]).astype(np.float64)
    tr = np.concatenate([f[1] for f in filters]).astype(np.float64)
    return lens, lam, tr


# --------------------------------------------------------------------------
# Spectrum pixel grid
# --------------------------------------------------------------------------
def make_spectrum_pixels(n_pix=1500, lo_um=0.6, hi_um=5.3, r_lo=100.0, r_hi=1000.0):
    """Observed-frame pixel centres (Angstrom), log-spaced, and an R_fwhm curve
    rising linearly from r_lo to r_hi across the pixels."""
    lam = np.geomspace(lo_um * 1e4, hi_um * 1e4, n_pix)
    r = np.linspace(r_lo, r_hi, n_pix)
    return lam, r


# --------------------------------------------------------------------------
# Parameter batches
# --------------------------------------------------------------------------
def dirichlet1(rng, n_rows, n):
    """Dirichlet(1,...,1) rows from uniform draws (normalised exponentials)."""
    u = rng.random((n_rows, n))
    e = -np.log1p(-u)
    return e / e.sum(axis=1, keepdims=True)


def make_theta(n_rows, n_sfh, zmode, ranges, seed=4):
    """Parameter dictionary of `n_rows` draws.

    ranges: dict key -> (lo, hi) uniform range, or a float for a fixed value.
    'feh' gives the range of the per-bin (zmode 0) or constant (zmode 1) [Fe/H].
    The SFH masses are Dirichlet(1) over the bins (one solar mass formed).
    """
    rng = _rng(seed)
    out = {"sfh": dirichlet1(rng, n_rows, n_sfh)}
    nz = n_sfh if zmode == 0 else 1
    lo, hi = ranges["feh"]
    out["logzsol"] = lo + (hi - lo) * rng.random((n_rows, nz))
    for k in SCALAR_KEYS:
        r = ranges.get(k, 0.0)
        if isinstance(r, tuple):
            out[k] = r[0] + (r[1] - r[0]) * rng.random(n_rows)
        else:
            out[k] = np.full(n_rows, float(r))
    if ranges.get("tie_tau", False):
        out["tau_pow"] = out["diffuse_tau_kc"].copy()
    return out


def edge_sfr(n_rows, n_sfh, seed=4):
    """Per-edge SFRs (Msun/yr) for the linear SFH scheme: positive, varied
    (Gamma(1.5)), ~1e-10 so that a bin's mass is of order its width / 1e10 yr."""
    return 1e-10 * _rng(seed).gamma(1.5, 1.0, (n_rows, n_sfh + 1))


FLOOR_NAMES = ("log_err_scale", "log_f_calib", "log_f_data", "log_jitter")


def floor_theta(n_rows, floor_phot, floor_spec, phot_sigma=None, spec_sigma=None, seed=8):
    """log10 values of the noise-floor terms that are on, keyed like the
    library's columns: error scale in [-0.2, 0.3], fractions in [-2.5, -1], the
    jitter (in the data's units) within a decade below the median error."""
    rng = _rng(seed)
    out = {}
    for arm, bits, sg in (("phot", floor_phot, phot_sigma), ("spec", floor_spec, spec_sigma)):
        for k, name in enumerate(FLOOR_NAMES):
            if not (bits >> k) & 1:
                continue
            if k == 0:
                lo, hi = -0.2, 0.3
            elif k < 3:
                lo, hi = -2.5, -1.0
            else:
                m = float(np.log10(np.median(np.abs(sg))))
                lo, hi = m - 1.0, m
            out[f"{name}_{arm}"] = lo + (hi - lo) * rng.random(n_rows)
    return out


def noise(shape, seed=5):
    return _rng(seed).standard_normal(shape)


# --------------------------------------------------------------------------
# Workload shapes
# --------------------------------------------------------------------------
@dataclass
class Workload:
    name: str
    grid_kw: dict
    n_sfh: int
    zf: float
    zmode: int              # 0 = one [Fe/H] per SFH bin, 1 = one constant [Fe/H]
    use_afe: int
    use_nebular: int
    dust_law: int           # diffuse law: 0 = power law, 1 = Kriek & Conroy 2013
    filters: str            # 'gauss8' | 'nircam20'
    batch: int
    ranges: dict
    spectrum: dict | None = None
    z_ref: float = 0.0
    sigma_gal_kms: float = 0.0
    sample_sigma_gal: int = 0          # 1: sigma_gal (km/s) is a parameter, drawn from ranges["sigma_gal"]
    sigma_gal_max_kms: float = 1000.0
    sfh_scheme: int = 0                # 0 step (N_T bin masses), 1 linear (N_T + 1 edge SFRs)
    floor_phot: int = 0                # noise-floor terms on (bits: 1 err scale, 2 f_calib, 4 f_data, 8 jitter)
    floor_spec: int = 0
    extra: dict = field(default_factory=dict)


WORKLOADS = {
    # tiny FP64-parity photometric fit step
    "tiny_phot_16x4x512": Workload(
        name="tiny_phot_16x4x512",
        grid_kw=dict(n_age=16, log_age=(6.0, 10.1), feh=(-2.0, 0.2), n_feh=4, n_lam=512,
                     lam_um=(0.1, 5.0)),
        n_sfh=8, zf=10.0, zmode=0, use_afe=0, use_nebular=0, dust_law=0,
        filters="gauss8", batch=64,
        ranges=dict(feh=(-2.0, 0.2), logmass=(8.0, 11.0), zred=(0.5, 8.0),
                    diffuse_tau_kc=(0.0, 2.0), diffuse_dust_index=-0.7, alpha_pow=-1.0,
                    tie_tau=True, gas_logz=0.0, gas_logu=-2.0, afe=0.0)),
    # paper-scale photometric batch
    "phot_107x12x6000_b1024": Workload(
        name="phot_107x12x6000_b1024",
        grid_kw=dict(n_age=107, log_age=(5.5, 10.8), feh=(-2.5, 0.5), n_feh=12, n_lam=6000,
                     lam_um=(0.01, 6.0), nebular=dict(seed=2, n_logu=7, n_logz=12)),
        n_sfh=120, zf=30.0, zmode=0, use_afe=0, use_nebular=1, dust_law=1,
        filters="nircam20", batch=1024,
        ranges=dict(feh=(-2.5, 0.5), logmass=(8.0, 11.0), zred=(0.0, 12.0),
                    tau_pow=(0.0, 2.0), alpha_pow=-1.0, diffuse_tau_kc=(0.0, 2.0),
                    diffuse_dust_index=(-1.0, 0.4), gas_logz=(-1.3, 0.3), gas_logu=(-4.0, -1.0),
                    afe=0.0)),
    # spectro-photometric fit with [a/Fe] and gradients
    "specphot_afe_107x12x5x6000_b2048": Workload(
        name="specphot_afe_107x12x5x6000_b2048",
        grid_kw=dict(n_age=107, log_age=(5.5, 10.8), feh=(-2.5, 0.5), n_feh=12,
                     afe_nodes=(-0.2, 0.0, 0.2, 0.4, 0.6), n_lam=6000, lam_um=(0.01, 6.0)),
        n_sfh=120, zf=30.0, zmode=1, use_afe=1, use_nebular=0, dust_law=1,
        filters="nircam20", batch=2048,
        ranges=dict(feh=(-2.5, 0.5), afe=(-0.2, 0.6), logmass=(8.0, 11.0), zred=(0.0, 12.0),
                    tau_pow=(0.0, 2.0), alpha_pow=-1.0, diffuse_tau_kc=(0.0, 2.0),
                    diffuse_dust_index=(-1.0, 0.4), gas_logz=0.0, gas_logu=-2.0),
        spectrum=dict(n_pix=1500, lo_um=0.6, hi_um=5.3, r_lo=100.0, r_hi=1000.0, snr=20.0),
        z_ref=6.0, sigma_gal_kms=300.0),
}
# spectro-photometric fit with a sampled stellar velocity dispersion (Sec. 2.7:
# sigma_gal a parameter with its own prior; default 300 km/s, here U[50, 500])
_s = WORKLOADS["specphot_afe_107x12x5x6000_b2048"]
WORKLOADS["specphot_afe_sgal_107x12x5x6000_b2048"] = Workload(**{
    **_s.__dict__, "name": "specphot_afe_sgal_107x12x5x6000_b2048", "sample_sigma_gal": 1,
    "sigma_gal_max_kms": 600.0, "ranges": {**_s.ranges, "sigma_gal": (50.0, 500.0)}})
# the same fit with a marginalised 12th-order Chebyshev calibration polynomial
# on the spectrum (App. E; the paper's spectral demonstrations use 12th order)
WORKLOADS["specphot_afe_calib13_107x12x5x6000_b2048"] = Workload(**{
    **_s.__dict__, "name": "specphot_afe_calib13_107x12x5x6000_b2048",
    "extra": {"calib_sigma": [0.2] + [0.1] * 12}})
# the same fit with every term of the systematic noise floor on for both arms
# (App. sys_floor): error scale, model- and data-anchored fractions, jitter
WORKLOADS["specphot_afe_floor_107x12x5x6000_b2048"] = Workload(**{
    **_s.__dict__, "name": "specphot_afe_floor_107x12x5x6000_b2048", "floor_phot": 15, "floor_spec": 15})
# the paper-scale photometric fit with the linear SFH scheme (App. B, Eq.
# tent_integral): per-edge SFRs, N_T + 1 columns
WORKLOADS["phot_linsfh_107x12x6000_b1024"] = Workload(**{
    **WORKLOADS["phot_107x12x6000_b1024"].__dict__, "name": "phot_linsfh_107x12x6000_b1024", "sfh_scheme": 1})
# mixed-precision contraction: the paper-scale photometric batch at 4096 rows
_w = WORKLOADS["phot_107x12x6000_b1024"]
WORKLOADS["phot_107x12x6000_b4096"] = Workload(**{**_w.__dict__, "name": "phot_107x12x6000_b4096",
                                                  "batch": 4096})


# JADES-like spectro-photometric fit with the nebular grid's emission lines
# apart from its continuum (App. C): the paper-scale photometric grid with a
# 30-line cube, a 1500-pixel R = 100-1000 spectrum, 20 filters and a line
# catalogue (Sec. 3.3); sigma_gas sampled in U[50, 400] km/s (bound 600)
_p = WORKLOADS["phot_107x12x6000_b1024"]
WORKLOADS["specphot_lines_107x12x6000_b1024"] = Workload(**{
    **_p.__dict__, "name": "specphot_lines_107x12x6000_b1024",
    "grid_kw": dict(_p.grid_kw, nebular=dict(seed=2, n_logu=7, n_logz=12, line_cube=30)),
    "spectrum": dict(n_pix=1500, lo_um=0.6, hi_um=5.3, r_lo=100.0, r_hi=1000.0, snr=20.0),
    "z_ref": 6.0, "sigma_gal_kms": 300.0,
    "ranges": {**_p.ranges, "sigma_gas": (50.0, 400.0)},
    "extra": {"lines": dict(gas_sigma_mode=2, sigma_gas_max_kms=600.0, n_lcat=12)}})


def workload_filters(w: Workload):
    if w.filters == "gauss8":
        return make_filters_gauss(8, 0.6, 4.5, 0.2, 200)
    if w.filters == "nircam20":
        return make_filters_nircam_like(8, 12, 0.6, 5.0, 200, seed=3)
    raise ValueError(w.filters)


def shrink(w: Workload, n_age=None, n_feh=None, n_lam=None, batch=None, n_sfh=None, n_pix=None):
    """A smaller case of the same workload (same structure, fewer nodes)."""
    gk = dict(w.grid_kw)
    if n_age is not None:
        gk["n_age"] = n_age
    if n_feh is not None:
        gk["n_feh"] = n_feh
    if n_lam is not None:
        gk["n_lam"] = n_lam
    sp = None if w.spectrum is None else dict(w.spectrum)
    if sp is not None and n_pix is not None:
        sp["n_pix"] = n_pix
    d = dict(w.__dict__)
    d.update(grid_kw=gk, spectrum=sp, name=w.name + "_small")
    if batch is not None:
        d["batch"] = batch
    if n_sfh is not None:
        d["n_sfh"] = n_sfh
    return Workload(**d)
