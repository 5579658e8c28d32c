"""Pins of the oracle's emission lines (App. C line cube, App. "line_proj",
Eq. app_line_profile) and of the line-catalogue arm (Sec. 3.3, App.
"line_lik"), each against a quantity computed here independently with numpy:

- a line's observer-frame flux: Q_young 10^(line table) 10^logmass Lsun /
  (4 pi D_L^2) at a (log U, log Z_gas) node with no dust, from the oracle's own
  Q_young and D_L (App. "line_proj": the flux factor without (1+z));
- dust on a line: the ratio with / without dust is exp(-tau_d - tau_BC) of the
  power laws at the line's rest wavelength (Sec. 2.4);
- the spectrum: the line-only spectrum (with lines minus without) integrated
  over frequency returns every line's flux (unit-area profiles, Eq.
  app_line_profile), and an isolated line's second moment in ln(lambda) is
  (sigma_gas^2 + sigma_inst^2)/c^2 for a fixed, a tied and a sampled sigma_gas;
- the photometry: the line-only band fluxes are F R_b(lam_obs) lam_obs / Z_b
  with numpy's interpolation of the filter and trapezoid of Z_b (App. D);
- the catalogue: the lnL change equals the Gaussian terms of each entry, a
  blend's model is the sum of its lines, an upper limit costs nothing while
  the model stays below it (Eq. app_line_chi2_det, Eq. app_line_chi2_UL).
"""
import dataclasses
import math

import numpy as np
import pytest

import oracle
import synth
from tests import cases

C_AA, C_KMS, LSUN, AB = 2.99792458e18, 299792.458, 3.839e33, 3.631e-20
PC_CM = 3.0856775814913673e18


def _workload(n_pix=6000, r=300.0):
    w = synth.shrink(synth.WORKLOADS["phot_107x12x6000_b1024"], n_age=20, n_feh=4, n_lam=3000, n_sfh=10,
                     batch=8)
    w.grid_kw = dict(w.grid_kw, nebular=dict(seed=2, n_logu=7, n_logz=12, line_cube=12))
    w.dust_law = 0
    w.spectrum = dict(n_pix=n_pix, lo_um=0.3, hi_um=5.3, r_lo=r, r_hi=r, snr=20.0)
    w.sigma_gal_kms = 150.0
    w.z_ref = 1.0
    return w


@pytest.fixture(scope="module")
def base():
    w = _workload()
    orc = cases.oracle_for(w)      # the data come from the model without lines
    return w, orc


def _rows(w, n, seed, z=1.2, dust=True):
    d = cases.theta_dict(w, n, seed=seed)
    d["zred"][:] = z
    if not dust:
        d["tau_pow"][:] = 0.0
        d["diffuse_tau_kc"][:] = 0.0
    return oracle.pack_theta(d, w.n_sfh, w.zmode)


def test_line_flux_at_a_node_without_dust(base):
    w, orc0 = base
    orc = dataclasses.replace(orc0, use_lines=1)
    g = orc.grid
    th = _rows(w, 3, seed=81, dust=False)
    jz = cases.z_column(w.n_sfh, w.zmode)
    iu, iz = 3, 5
    th[:, jz + 5] = g.neb_logz[iz]        # gas_logz, gas_logu follow the dust keys
    th[:, jz + 6] = g.neb_logu[iu]
    fl = orc.line_fluxes(th)
    for r in range(th.shape[0]):
        row = orc.row(th[r])
        dl = max(row["D_L"], 10.0 * PC_CM)
        want = row["Q_young"] * 10.0 ** g.line_tab[iu, iz] * 10.0 ** th[r, jz - 1] * LSUN / (4 * math.pi * dl * dl)
        np.testing.assert_allclose(fl[r], want, rtol=1e-12)


def test_dust_on_a_line_is_the_power_law_screens(base):
    w, orc0 = base
    orc = dataclasses.replace(orc0, use_lines=1)
    lam = orc.grid.line_lam
    th = _rows(w, 3, seed=82)
    th0 = th.copy()
    jz = cases.z_column(w.n_sfh, w.zmode)
    th0[:, jz + 1] = 0.0     # tau_pow
    th0[:, jz + 3] = 0.0     # diffuse_tau_kc
    ratio = orc.line_fluxes(th) / orc.line_fluxes(th0)
    for r in range(th.shape[0]):
        tbc = th[r, jz + 1] * (lam / 5500.0) ** th[r, jz + 2]
        td = th[r, jz + 3] * (lam / 5500.0) ** th[r, jz + 4]
        np.testing.assert_allclose(ratio[r], np.exp(-tbc - td), rtol=1e-12)


@pytest.mark.parametrize("mode", ["fixed", "tied", "sampled"])
def test_spectral_lines_conserve_flux_and_compose_widths(base, mode):
    w, orc0 = base
    kw = dict(use_lines=1)
    if mode == "fixed":
        kw.update(gas_sigma_mode=oracle.GAS_SIGMA_FIXED, sigma_gas_kms=80.0)
    elif mode == "sampled":
        kw.update(gas_sigma_mode=oracle.GAS_SIGMA_SAMPLED, sigma_gas_max_kms=500.0)
    orc = dataclasses.replace(orc0, **kw)
    th = _rows(w, 2, seed=83)
    if mode == "sampled":
        th = np.concatenate([th, np.array([[120.0], [260.0]])], axis=1)
    th_nol = th[:, :orc0.n_param]
    sp = orc.eval(th)["spec"] - orc0.eval(th_nol)["spec"]
    fl = orc.line_fluxes(th)
    lam = np.asarray(orc.spec_lam)
    ll = np.log(lam)
    dll = np.gradient(ll)
    jz = cases.z_column(w.n_sfh, w.zmode)
    sig_inst = C_KMS / (2.3548200450309493 * np.asarray(orc.lsf_value))   # R_fwhm pixels
    for r in range(th.shape[0]):
        z = th[r, jz]
        lo = orc.grid.line_lam * (1 + z)
        inside = (lo > lam[0] * 1.05) & (lo < lam[-1] / 1.05)
        sg = {"fixed": 80.0, "tied": 150.0, "sampled": th[r, -1]}[mode]
        s = math.sqrt(sg ** 2 + sig_inst[0] ** 2) / C_KMS
        # integral over frequency, f_nu dnu = f_nu (c / lambda) dln(lambda): each
        # line's flux times the part of its profile (cut at 5 s) on the pixels
        tot = np.sum(sp[r] * C_AA / lam * dll)
        a_ = np.clip((ll[0] - np.log(lo)) / s, -5, 5)
        b_ = np.clip((ll[-1] - np.log(lo)) / s, -5, 5)
        cover = np.array([0.5 * (math.erf(y / math.sqrt(2)) - math.erf(x / math.sqrt(2))) for x, y in zip(a_, b_)])
        np.testing.assert_allclose(tot, np.sum(fl[r] * cover), rtol=1e-5)
        # the most isolated line: its second moment in ln(lambda)
        order = np.argsort(lo)
        gaps = np.diff(np.log(lo[order]))
        iso = [order[k] for k in range(len(order)) if inside[order[k]]
               and (k == 0 or gaps[k - 1] > 0.02) and (k == len(order) - 1 or gaps[k] > 0.02)]
        assert iso
        l = iso[0]
        win = np.abs(ll - math.log(lo[l])) < 0.01
        prof = sp[r, win] * C_AA / lam[win]          # flux per unit ln(lambda)
        x = ll[win] - math.log(lo[l])
        m2 = np.sum(prof * x * x * dll[win]) / np.sum(prof * dll[win])
        s2 = s * s
        assert m2 == pytest.approx(s2, rel=2e-3)


def test_photometric_lines_through_the_band_response(base):
    w, orc0 = base
    orc = dataclasses.replace(orc0, use_lines=1)
    th = _rows(w, 3, seed=84)
    dph = orc.eval(th)["phot"] - orc0.eval(th)["phot"]
    fl = orc.line_fluxes(th)
    lens, flam, ftr = orc.filters
    jz = cases.z_column(w.n_sfh, w.zmode)
    for r in range(th.shape[0]):
        lo = orc.grid.line_lam * (1 + th[r, jz])
        off = 0
        for b, n in enumerate(lens):
            L, R = flam[off:off + n], ftr[off:off + n]
            off += n
            zb = np.trapezoid(L * R * C_AA * AB / L ** 2, L)
            want = np.sum(fl[r] * np.interp(lo, L, R, left=0.0, right=0.0) * lo) / zb
            assert dph[r, b] == pytest.approx(want, rel=1e-9, abs=1e-12 * abs(orc0.eval(th)["phot"][r]).max())


def test_line_catalogue_detections_blends_and_upper_limits(base):
    w, orc0 = base
    orc = dataclasses.replace(orc0, use_lines=1)
    th = _rows(w, 3, seed=85)
    fl = orc.line_fluxes(th)
    blends = [[0], [1, 2], [4], [5], [7, 8, 9], [11]]
    m_ref = np.stack([fl[0, b].sum() for b in blends])
    d = m_ref * np.array([1.1, 0.9, 1.0, 1.05, 0.97, 1.0])
    d[3] = 0.5 * m_ref[3]      # an upper limit the model exceeds
    d[5] = 2.0 * m_ref[5]      # one it respects
    sig = 0.05 * np.abs(m_ref)
    upper = np.array([0, 0, 0, 1, 0, 1], np.uint8)
    mask = np.array([1, 1, 0, 1, 1, 1], np.uint8)   # entry 2 masked out
    cat = dataclasses.replace(orc, lcat=(blends, d, sig, mask, upper))
    base_l = orc.eval(th)["lnl"]
    got = cat.eval(th)["lnl"] - base_l
    for r in range(th.shape[0]):
        m = np.array([fl[r, b].sum() for b in blends])
        res = d - m
        res[(upper == 1) & (m <= d)] = 0.0
        want = np.sum((-0.5 * (res / sig) ** 2 - 0.5 * np.log(2 * np.pi * sig ** 2))[mask == 1])
        assert got[r] == pytest.approx(want, rel=1e-9, abs=1e-9 * abs(base_l[r]))
    # row 0: the respected limit adds only its normalisation
    m0 = np.array([fl[0, b].sum() for b in blends])
    assert m0[5] < d[5] and m0[3] > d[3]
