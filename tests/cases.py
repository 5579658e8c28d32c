"""Test-side assembly of seeded cases: grid, filters, spectrum pixels,
parameter rows and mock data (data = oracle model at a true parameter row,
perturbed by Gaussian noise at S/N 20)."""
from __future__ import annotations

import dataclasses

import numpy as np

import oracle
import synth


def z_column(n_sfh, zmode, sfh_scheme=0):
    """Column of the redshift in the oracle's parameter layout: the SFH key (N_T
    masses, or N_T + 1 edge SFRs), logzsol (N_T or 1), afe, logmass, zred."""
    return n_sfh + (1 if sfh_scheme == 1 else 0) + (n_sfh if zmode == 0 else 1) + 2


def oracle_for(w: synth.Workload, grid=None, filters=None, with_data=True, seed_theta=4, lsf_r=None,
               spec_mask=None, sigma_gal_kms=None, calib_sigma=None, calib_mode=0):
    """lsf_r, spec_mask, sigma_gal_kms: optional replacements of the
    workload's R_fwhm curve, pixel mask and stellar dispersion; calib_sigma:
    prior widths of a calibration polynomial (App. E), marginalised
    (calib_mode 0) or optimised at each call (1)."""
    grid = grid if grid is not None else synth.make_grid(**w.grid_kw, seed=1)
    filt = filters if filters is not None else synth.pack_filters(synth.workload_filters(w))
    kw = dict(grid=grid, n_sfh=w.n_sfh, zf=w.zf, zmode=w.zmode, use_afe=w.use_afe,
              use_nebular=w.use_nebular, dust_law=w.dust_law, filters=filt,
              sample_sigma_gal=w.sample_sigma_gal, sigma_gal_max_kms=w.sigma_gal_max_kms,
              floor_phot=w.floor_phot, floor_spec=w.floor_spec, sfh_scheme=w.sfh_scheme)
    nb = len(filt[0])
    kw.update(phot_d=np.ones(nb), phot_sigma=np.ones(nb), phot_mask=np.ones(nb, np.uint8))
    if w.spectrum is not None:
        sp = w.spectrum
        lam, r = synth.make_spectrum_pixels(sp["n_pix"], sp["lo_um"], sp["hi_um"], sp["r_lo"], sp["r_hi"])
        kw.update(spec_lam=lam, spec_d=np.ones(lam.size), spec_sigma=np.ones(lam.size),
                  spec_mask=np.ones(lam.size, np.uint8) if spec_mask is None else spec_mask, lsf_mode=0,
                  lsf_value=r if lsf_r is None else lsf_r,
                  sigma_gal_kms=w.sigma_gal_kms if sigma_gal_kms is None else sigma_gal_kms, z_ref=w.z_ref,
                  calib_sigma=None if calib_sigma is None else np.asarray(calib_sigma, dtype=np.float64),
                  calib_mode=calib_mode)
    orc = oracle.Oracle(**kw)
    if with_data:
        d_true = synth.make_theta(1, w.n_sfh, w.zmode, w.ranges, seed=99)
        if w.sfh_scheme == 1:
            d_true["sfh"] = synth.edge_sfr(1, w.n_sfh, seed=99)
        th_true = oracle.pack_theta(d_true, w.n_sfh, w.zmode, w.sample_sigma_gal, sfh_scheme=w.sfh_scheme)
        if w.floor_phot or w.floor_spec:   # the truth row only makes the data: floors off for it
            orc.floor_phot, orc.floor_spec = 0, 0
            orc._rebuild_model()
        th_true[0, z_column(w.n_sfh, w.zmode, w.sfh_scheme)] = min(2.0, w.zf * 0.5)
        res = orc.eval(th_true)
        assert res["status"][0] == 0
        nz = synth.noise(res["phot"].shape[1] + res["spec"].shape[1], seed=5)
        ph = res["phot"][0]
        sp_ = res["spec"][0]
        snr = 20.0
        orc.set_data(phot_d=ph * (1 + nz[:ph.size] / snr), phot_sigma=np.abs(ph) / snr,
                     spec_d=(sp_ * (1 + nz[ph.size:] / snr)) if sp_.size else None,
                     spec_sigma=(np.abs(sp_) / snr) if sp_.size else None)
        if w.floor_phot or w.floor_spec:
            orc.floor_phot, orc.floor_spec = w.floor_phot, w.floor_spec
            orc._rebuild_model()
    return orc


def theta_dict(w: synth.Workload, n, seed=4, orc=None):
    """Parameter draws; with a noise floor, its columns too (the jitter's range
    follows the errors of the oracle `orc` holds)."""
    d = synth.make_theta(n, w.n_sfh, w.zmode, w.ranges, seed=seed)
    if w.sfh_scheme == 1:
        d["sfh"] = synth.edge_sfr(n, w.n_sfh, seed=seed)
    if w.floor_phot or w.floor_spec:
        d.update(synth.floor_theta(n, w.floor_phot, w.floor_spec,
                                   None if orc is None else orc.phot_sigma,
                                   None if orc is None else orc.spec_sigma, seed=seed + 1000))
    return d


def theta_rows(w: synth.Workload, n, seed=4, orc=None):
    return oracle.pack_theta(theta_dict(w, n, seed, orc), w.n_sfh, w.zmode, w.sample_sigma_gal,
                             w.floor_phot, w.floor_spec, w.sfh_scheme)


def gpu_model_for(ctx, orc, w: synth.Workload, with_spec_data=True, fixed=None):
    """A library model with exactly the oracle's inputs (grid loaded once per grid
    object); with_spec_data=False gives the spectrum's pixels but not its data;
    fixed: {key: value} of keys fixed for every row (no column)."""
    cache = ctx.__dict__.setdefault("_grid_ids", {})
    key = id(orc.grid)
    if key not in cache:
        cache[key] = (ctx.load_grid(orc.grid), orc.grid)
    gid = cache[key][0]
    kw = dict(use_afe=w.use_afe, use_nebular=w.use_nebular, dust_law=w.dust_law,
              sample_sigma_gal=orc.sample_sigma_gal, sigma_gal_max_kms=orc.sigma_gal_max_kms,
              noise_floor_phot=orc.floor_phot, noise_floor_spec=orc.floor_spec, sfh_scheme=orc.sfh_scheme,
              bc_edge_log_age_yr=orc.bc_edge_log_age_yr, H0=orc.H0, Om0=orc.Om0,
              filters=orc.filters, phot_d=orc.phot_d, phot_sigma=orc.phot_sigma,
              phot_mask=orc.phot_mask, phot_upper=orc.phot_upper, fesc_geometry=orc.fesc_geometry)
    if orc.spec_lam is not None:
        kw.update(spec_lam=orc.spec_lam, spec_d=orc.spec_d if with_spec_data else None,
                  spec_sigma=orc.spec_sigma if with_spec_data else None,
                  spec_mask=orc.spec_mask, lsf_mode=orc.lsf_mode, lsf_value=orc.lsf_value,
                  sigma_gal_kms=orc.sigma_gal_kms, z_ref=orc.z_ref, calib_sigma=orc.calib_sigma,
                  calib_mode=orc.calib_mode)
    kw.update(use_lines=orc.use_lines, gas_sigma_mode=orc.gas_sigma_mode, sigma_gas_kms=orc.sigma_gas_kms,
              sigma_gas_max_kms=orc.sigma_gas_max_kms, lcat=orc.lcat, dust_bins=orc.dust_bins,
              use_igm=orc.use_igm)
    return ctx.create_model(gid, w.n_sfh, w.zf, w.zmode, fixed=fixed, **kw)


def theta_pair(w: synth.Workload, n, seed=4, orc=None):
    """Parameter rows rounded to FP32 (library input) and the same values in FP64 (oracle input)."""
    th32 = theta_rows(w, n, seed, orc).astype(np.float32)
    return th32, th32.astype(np.float64)


def rel_err(a, b, floor=0.0):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return np.abs(a - b) / np.maximum(np.abs(b), floor)


def poison_rows(model, th32):
    """Rows that fill a call's workspace with other values: the same rows with
    their SFH mass fractions reversed in bin order (other weights, other
    contraction outputs, same redshifts).  A call on these just before the call
    under test leaves stale values of other rows in any output element the
    tested call would fail to write."""
    th = th32.copy()
    a = model.offsets["sfh"]
    b = model.offsets["logzsol"]
    th[:, a:b] = th32[:, a:b][:, ::-1]
    return th


def kink_rows(orc, th64, rel=2e-4):
    """Rows at which d lnL / dz has a kink that matters: a spectral pixel whose
    rest-frame position ln(lambda_obs / (1+z)) lies within rel node spacings
    of a model node.  There a linear-interpolation row switches brackets, and
    the GPU (which picks the bracket from FP32 positions, ~1e-4 node spacings
    apart at these grids) and the oracle (FP64) may each take the derivative
    of a different side: both valid one-sided derivatives of the same
    continuous function (the kink reading of the adjoint).  Filter samples
    also have kinks there, but one sample's share of a band sum is too small
    to show."""
    ll = np.log(np.asarray(orc.grid.lam_aa, dtype=np.float64))
    pos = np.log(np.asarray(orc.spec_lam, dtype=np.float64))
    jz = z_column(orc.n_sfh, orc.zmode, orc.sfh_scheme)
    out = np.zeros(th64.shape[0], bool)
    for r in range(th64.shape[0]):
        x = pos - np.log1p(th64[r, jz])
        k = np.clip(np.searchsorted(ll, x), 1, ll.size - 1)
        d = np.minimum(np.abs(x - ll[k - 1]), np.abs(ll[k] - x)) / (ll[k] - ll[k - 1])
        out[r] = bool((d < rel).any())
    return out


def calib_case(w: synth.Workload, calib_sigma, calib_mode=0):
    """Oracle of a workload with a calibration polynomial (marginalised, or
    optimised with calib_mode 1) and data carrying a smooth multiplicative
    distortion (1 + 0.08 x - 0.05 T_2(x)) over the spectrum's Chebyshev
    coordinate x, the kind the polynomial absorbs."""
    orc = oracle_for(w, calib_sigma=calib_sigma, calib_mode=calib_mode)
    lam = np.asarray(orc.spec_lam)
    x = (2.0 * lam - (lam[0] + lam[-1])) / (lam[-1] - lam[0])
    dist = 1.0 + 0.08 * x - 0.05 * (2 * x * x - 1)
    orc.set_data(phot_d=orc.phot_d, phot_sigma=orc.phot_sigma, spec_d=orc.spec_d * dist,
                 spec_sigma=orc.spec_sigma * dist)
    return orc


def lnl_scale(orc, ref):
    """Magnitude of the terms of lnL = -chi2/2 + C (C = -1/2 sum ln 2 pi sigma^2
    over included data): the FP64 sum's natural error scale.  lnL itself can
    cancel to ~0 while both terms are large."""
    c = 0.0
    if orc.phot_d is not None:
        m = np.ones(len(orc.phot_sigma), bool) if orc.phot_mask is None else orc.phot_mask.astype(bool)
        c += -0.5 * np.sum(np.log(2 * np.pi * orc.phot_sigma[m] ** 2))
    if orc.spec_d is not None:
        m = np.ones(len(orc.spec_sigma), bool) if orc.spec_mask is None else orc.spec_mask.astype(bool)
        c += -0.5 * np.sum(np.log(2 * np.pi * orc.spec_sigma[m] ** 2))
    half_chi2 = c - ref["lnl"]
    return np.maximum(np.abs(ref["lnl"]), half_chi2 + abs(c))


def with_upper_limits(orc):
    """The oracle `orc` with every other photometric band's datum taken as an
    upper limit (Sec. 4.1 likelihood, Eq. app_line_chi2_UL)."""
    return dataclasses.replace(orc, phot_upper=(np.arange(len(orc.phot_sigma)) % 2).astype(np.uint8))


def limit_regimes(orc, phot):
    """(limits the rows' models exceed, limits they respect), counted over the
    flagged bands of `orc` and the rows' band fluxes `phot`."""
    up = np.asarray(orc.phot_upper).astype(bool)
    d = np.asarray(orc.phot_d)[up]
    m = np.asarray(phot)[:, up]
    return int(np.sum(m > d)), int(np.sum(m <= d))


def escape_pair(w: synth.Workload, n, seed, geometry):
    """Parameter rows (FP32 and the same values in FP64) of a model with an
    escape geometry (Sec. frac_obrun): the workload's draws plus the runaway
    fraction f_ob ~ U[0.05, 0.95] in the last column."""
    d = theta_dict(w, n, seed)
    d["frac_obrun"] = np.random.default_rng(seed + 2000).uniform(0.05, 0.95, n)
    th32 = oracle.pack_theta(d, w.n_sfh, w.zmode, w.sample_sigma_gal, w.floor_phot, w.floor_spec,
                             w.sfh_scheme, geometry).astype(np.float32)
    return th32, th32.astype(np.float64)


def lines_case(w: synth.Workload, gas_sigma_mode=2, sigma_gas_kms=300.0, sigma_gas_max_kms=600.0, n_lcat=12,
               seed=7):
    """Oracle of a workload whose grid carries an emission-line cube, with the
    lines on (App. C, App. line_proj), the given gas dispersion mode, and a line
    catalogue of n_lcat entries (Sec. 3.3): single lines and blends of two or
    three neighbours, two upper limits (one exceeded at the truth, one not) and
    one masked entry.  Photometry, spectrum and catalogue data are the model
    of a true row (z = 2, sigma_gas = 150 km/s when sampled) with 5% noise."""
    orc = oracle_for(w, with_data=False)
    orc = dataclasses.replace(orc, use_lines=1, gas_sigma_mode=gas_sigma_mode, sigma_gas_kms=sigma_gas_kms,
                              sigma_gas_max_kms=sigma_gas_max_kms)
    d_true = synth.make_theta(1, w.n_sfh, w.zmode, w.ranges, seed=99)
    d_true["zred"][:] = min(2.0, w.zf * 0.5)
    sampled = gas_sigma_mode == 2
    if sampled:
        d_true["sigma_gas"] = np.array([150.0])
    th = oracle.pack_theta(d_true, w.n_sfh, w.zmode, w.sample_sigma_gal, sample_sigma_gas=int(sampled))
    res = orc.eval(th)
    assert res["status"][0] == 0
    fl = orc.line_fluxes(th)[0]
    nl = fl.size
    rng = np.random.default_rng(seed)
    blends, k = [], 0
    while len(blends) < n_lcat and k < nl:
        size = 1 + int(rng.integers(0, 3)) if len(blends) % 3 == 1 else 1
        blends.append(list(range(k, min(k + size, nl))))
        k += size
    m = np.array([fl[b].sum() for b in blends])
    nz = synth.noise(res["phot"].shape[1] + res["spec"].shape[1] + len(blends), seed=5)
    ph, sp_ = res["phot"][0], res["spec"][0]
    snr = 20.0
    ld = m * (1 + nz[-len(blends):] / snr)
    upper = np.zeros(len(blends), np.uint8)
    mask = np.ones(len(blends), np.uint8)
    if len(blends) >= 4:
        upper[1], ld[1] = 1, 0.5 * m[1]      # exceeded at the truth
        upper[2], ld[2] = 1, 3.0 * m[2]      # respected
        mask[3] = 0
    orc = dataclasses.replace(orc, lcat=(blends, ld, np.abs(m) / snr, mask, upper))
    orc.set_data(phot_d=ph * (1 + nz[:ph.size] / snr), phot_sigma=np.abs(ph) / snr,
                 spec_d=(sp_ * (1 + nz[ph.size:ph.size + sp_.size] / snr)) if sp_.size else None,
                 spec_sigma=(np.abs(sp_) / snr) if sp_.size else None)
    return orc


def lines_theta_pair(w: synth.Workload, orc, n, seed=4):
    """Parameter rows of a lines case: the workload's draws plus sigma_gas
    ~ U[50, 400] km/s in the last column when the model samples it."""
    d = theta_dict(w, n, seed)
    sampled = orc.gas_sigma_mode == 2
    if sampled:
        d["sigma_gas"] = np.random.default_rng(seed + 3000).uniform(50.0, 400.0, n)
    th32 = oracle.pack_theta(d, w.n_sfh, w.zmode, w.sample_sigma_gal, w.floor_phot, w.floor_spec, w.sfh_scheme,
                             sample_sigma_gas=int(sampled)).astype(np.float32)
    return th32, th32.astype(np.float64)
