"""Pins of the oracle's sampled stellar velocity dispersion (Sec. 2.7
kinematics: sigma_gal may be a parameter with its own prior; App. E: the
continuum is broadened by sigma_gal and by the fixed kernel sigma_fix).

- The paper's own two-stage operator: sigma_gal applied as a Gaussian in
  Fourier space on a grid uniform in ln(lambda) (edge-padded), then the banded
  response of the fixed width alone.  numpy's FFT does the first stage here,
  independently of the oracle; the oracle's single kernel of width
  sqrt(sigma_fix^2 + sigma_gal^2) must give the same pixels.
- A sampled sigma_gal equal to a fixed one gives that fixed model exactly.
- A sampled sigma_gal outside [0, sigma_gal_max] marks the row invalid.
The analytic d lnL / d sigma_gal is pinned by central differences in
test_oracle_grad.py (workload shape "sgal_spec").
"""
import math

import numpy as np
import pytest

import oracle
import synth
from tests import cases

C_KMS = 299792.458
SGAL_W = synth.shrink(synth.WORKLOADS["specphot_afe_sgal_107x12x5x6000_b2048"], n_age=20, n_feh=4,
                      n_lam=1500, n_sfh=10, n_pix=240, batch=40)


def _spec_oracle(lam_grid, pix, sigma_inst_kms):
    g = synth.make_grid(n_age=3, log_age=(6.9, 8.3), n_feh=2, n_lam=lam_grid.size, seed=1)
    g.lam_aa = lam_grid
    g.flux = np.ones(g.flux.shape[:3] + (lam_grid.size,))
    return oracle.Oracle(grid=g, n_sfh=8, zf=10.0, zmode=1, spec_lam=pix, spec_d=np.ones(pix.size),
                         spec_sigma=np.ones(pix.size), lsf_mode=4,
                         lsf_value=np.full(pix.size, float(sigma_inst_kms)))


@pytest.mark.parametrize("sigma_gal", [80.0, 250.0])
def test_fourier_stage_then_fixed_response_equals_one_kernel(sigma_gal):
    # model grid uniform in ln(lambda) (the paper's stage-1 grid), a smooth
    # continuum with narrow absorption features
    lam = np.geomspace(4000.0, 8000.0, 6001)
    ll = np.log(lam)
    dln = ll[1] - ll[0]
    f = 1.0 + 0.3 * (ll - ll.mean())
    for c, d, w in ((4700.0, 0.4, 2.0e-4), (5300.0, 0.6, 3.5e-4), (6100.0, 0.3, 1.5e-4), (6900.0, 0.5, 5.0e-4)):
        f = f * (1.0 - d * np.exp(-0.5 * ((ll - math.log(c)) / w) ** 2))
    z = 0.2
    pix = np.geomspace(5200.0, 8800.0, 150)       # observed frame, inside the grid at z = 0.2
    orc = _spec_oracle(lam, pix, 90.0)
    # stage 1 (numpy): Gaussian of sigma_gal / c in ln(lambda) in Fourier space,
    # exp(-2 pi^2 s^2 nu^2) with nu conjugate to ln(lambda); buffer padded with
    # the edge values so the window edges are not darkened
    s = sigma_gal / C_KMS
    pad = int(12 * s / dln) + 1
    fp = np.concatenate([np.full(pad, f[0]), f, np.full(pad, f[-1])])
    nu = np.fft.rfftfreq(fp.size, d=dln)
    fs = np.fft.irfft(np.fft.rfft(fp) * np.exp(-2.0 * math.pi ** 2 * s ** 2 * nu ** 2), n=fp.size)[pad:-pad]
    # stage 2 (oracle): the banded response of the fixed width alone
    two_stage, v2 = orc.spectrum(lam, fs, z, sigma_gal_kms=0.0)
    # the oracle's single kernel of the composed width
    one, v1 = orc.spectrum(lam, f, z, sigma_gal_kms=sigma_gal)
    assert v1.all() and v2.all()
    np.testing.assert_allclose(one, two_stage, rtol=2e-6, atol=0)
    # and the broadening is not negligible at these widths
    plain, _ = orc.spectrum(lam, f, z, sigma_gal_kms=0.0)
    assert np.abs(one - plain).max() > 1e-3


def test_sampled_sigma_gal_equal_to_fixed_gives_the_fixed_model():
    orc_s = cases.oracle_for(SGAL_W)
    th = cases.theta_rows(SGAL_W, 12, seed=61)
    j = orc_s.n_param - 1
    th[:, j] = 300.0
    w_fixed = synth.Workload(**{**SGAL_W.__dict__, "sample_sigma_gal": 0, "sigma_gal_kms": 300.0})
    orc_f = cases.oracle_for(w_fixed)
    assert orc_f.n_param == orc_s.n_param - 1
    a = orc_s.eval(th)
    b = orc_f.eval(np.ascontiguousarray(th[:, :j]))
    assert np.array_equal(a["status"], b["status"])
    assert (a["status"] == 0).any()
    np.testing.assert_array_equal(a["spec"], b["spec"])
    np.testing.assert_array_equal(a["phot"], b["phot"])
    # the data of the two oracles differ only through their mock rows; compare
    # the projections above, and lnL against the same data
    orc_f.set_data(phot_d=orc_s.phot_d, phot_sigma=orc_s.phot_sigma, spec_d=orc_s.spec_d,
                   spec_sigma=orc_s.spec_sigma)
    np.testing.assert_array_equal(orc_f.eval(np.ascontiguousarray(th[:, :j]))["lnl"], a["lnl"])


def test_sigma_gal_outside_declared_range_marks_the_row():
    orc = cases.oracle_for(SGAL_W)
    th = cases.theta_rows(SGAL_W, 4, seed=62)
    j = orc.n_param - 1
    th[0, j] = -1.0
    th[1, j] = SGAL_W.sigma_gal_max_kms * 1.01
    th[2, j] = SGAL_W.sigma_gal_max_kms
    th[3, j] = 0.0
    st = orc.eval(th)["status"]
    assert list(st[:2]) == [1, 1]
    assert list(st[2:]) == [0, 0]
