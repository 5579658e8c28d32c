"""Pins of the oracle's marginalised calibration polynomial (App. E,
Eq. app_polymarg): the calibrated model mu_i (1 + sum_m c_m T_m(x_i)) with a
Gaussian prior on the coefficients, integrated out in closed form.

- The closed form against the integral itself, done numerically over the
  coefficients on a grid (one and two coefficients): the lnL of the spectrum
  with the calibration, exp(lnL_diag(d - mu (1 + c.T))) N(c; 0, Lambda),
  integrated by quadrature with numpy, plus the photometric terms.
- s_m -> 0 gives back the uncalibrated lnL (the paper states this limit).
- The gradient with the calibration on is pinned by central differences in
  test_oracle_grad.py (shapes "calib_spec" and "calib_opt_spec").
- The optimised polynomial (calib_mode 1; App. E: the mean of the marginal
  form is the optimised polynomial regularised by 1/s_m): lnL is the maximum
  over the coefficients from numpy's least-squares solver, and it exceeds the
  marginal lnL by exactly the Occam terms ln|M|/2 + ln|Lambda|/2.
"""
import math

import numpy as np
import pytest

import synth
from tests import cases

W_SMALL = synth.shrink(synth.WORKLOADS["specphot_afe_107x12x5x6000_b2048"], n_age=20, n_feh=4,
                       n_lam=1500, n_sfh=10, n_pix=20, batch=8)


def cheb(x, n):
    T = np.zeros((x.size, n))
    T[:, 0] = 1.0
    if n > 1:
        T[:, 1] = x
    for m in range(2, n):
        T[:, m] = 2.0 * x * T[:, m - 1] - T[:, m - 2]
    return T


@pytest.mark.parametrize("s", [[0.3], [0.3, 0.15]])
def test_closed_form_equals_numerical_integral_over_the_coefficients(s):
    orc_c = cases.oracle_for(W_SMALL, calib_sigma=s)
    orc_0 = cases.oracle_for(W_SMALL)
    th = cases.theta_rows(W_SMALL, 3, seed=71)
    a = orc_c.eval(th)
    b = orc_0.eval(th)
    assert np.array_equal(a["status"], b["status"]) and (a["status"] == 0).all()
    lam = np.asarray(orc_0.spec_lam)
    x = (2.0 * lam - (lam[0] + lam[-1])) / (lam[-1] - lam[0])
    A = cheb(x, len(s))
    d, sig = np.asarray(orc_0.spec_d), np.asarray(orc_0.spec_sigma)
    for r in range(th.shape[0]):
        mu = b["spec"][r]
        lnl_spec0 = np.sum(-0.5 * ((d - mu) / sig) ** 2 - 0.5 * np.log(2 * np.pi * sig ** 2))
        lnl_rest = b["lnl"][r] - lnl_spec0          # photometric terms, untouched by the calibration
        # the exponent is quadratic in c: find its peak and width, then integrate on a grid
        Dw = (mu[:, None] * A) / sig[:, None]
        rw = (d - mu) / sig
        H = Dw.T @ Dw + np.diag(1.0 / np.asarray(s) ** 2)
        c0 = np.linalg.solve(H, Dw.T @ rw)
        wid = np.sqrt(np.diag(np.linalg.inv(H)))
        grids = [c0[m] + wid[m] * np.linspace(-9, 9, 1201 if len(s) == 1 else 481) for m in range(len(s))]
        mesh = np.meshgrid(*grids, indexing="ij")
        C = np.stack([g.ravel() for g in mesh], axis=1)           # [npts][n]
        resid = (d[None, :] - mu[None, :] * (1.0 + C @ A.T)) / sig[None, :]
        log_like = np.sum(-0.5 * resid ** 2 - 0.5 * np.log(2 * np.pi * sig ** 2)[None, :], axis=1)
        log_prior = np.sum(-0.5 * (C / np.asarray(s)) ** 2 - 0.5 * np.log(2 * np.pi * np.asarray(s) ** 2), axis=1)
        f = log_like + log_prior
        fmax = f.max()
        vol = np.prod([g[1] - g[0] for g in grids])
        lnl_num = fmax + math.log(np.exp(f - fmax).sum() * vol) + lnl_rest
        assert abs(a["lnl"][r] - lnl_num) < 1e-6 * max(1.0, abs(lnl_num)), (r, a["lnl"][r], lnl_num)


def test_vanishing_prior_width_gives_the_uncalibrated_likelihood():
    orc_c = cases.oracle_for(W_SMALL, calib_sigma=[1e-9] * 6)
    orc_0 = cases.oracle_for(W_SMALL)
    th = cases.theta_rows(W_SMALL, 4, seed=72)
    a, b = orc_c.eval(th), orc_0.eval(th)
    np.testing.assert_allclose(a["lnl"], b["lnl"], rtol=1e-9, atol=1e-6)
    np.testing.assert_array_equal(a["spec"], b["spec"])


def test_calibration_raises_the_likelihood_of_a_miscalibrated_model():
    """Data carrying a smooth multiplicative distortion: the marginal lnL with a
    generous prior exceeds the uncalibrated one by a large margin (the gain term
    b^T M^-1 b / 2 dominates the Occam penalty)."""
    orc_0 = cases.oracle_for(W_SMALL)
    th = cases.theta_rows(W_SMALL, 1, seed=73)
    mu = orc_0.eval(th)["spec"][0]
    lam = np.asarray(orc_0.spec_lam)
    x = (2.0 * lam - (lam[0] + lam[-1])) / (lam[-1] - lam[0])
    d = mu * (1.0 + 0.3 * x - 0.1 * (2 * x * x - 1))
    sig = np.abs(mu) / 50.0
    orc_0.set_data(spec_d=d, spec_sigma=sig)
    orc_c = cases.oracle_for(W_SMALL, calib_sigma=[0.5, 0.5, 0.5])
    orc_c.set_data(phot_d=orc_0.phot_d, phot_sigma=orc_0.phot_sigma, spec_d=d, spec_sigma=sig)
    a, b = orc_c.eval(th)["lnl"][0], orc_0.eval(th)["lnl"][0]
    assert a > b + 100.0


def _lnl_parts(orc_0, th, r):
    """The spectrum's uncalibrated model, its data and the photometric lnL terms."""
    b = orc_0.eval(th)
    mu = b["spec"][r]
    d, sig = np.asarray(orc_0.spec_d), np.asarray(orc_0.spec_sigma)
    lnl_spec0 = np.sum(-0.5 * ((d - mu) / sig) ** 2 - 0.5 * np.log(2 * np.pi * sig ** 2))
    return mu, d, sig, b["lnl"][r] - lnl_spec0


@pytest.mark.parametrize("s", [[1e6] * 4, [0.3, 0.2, 0.1]])
def test_optimised_polynomial_is_the_regularised_least_squares_maximum(s):
    """The optimised polynomial (calib_mode 1): lnL is the maximum over the
    coefficients of lnL_diag(d - mu (1 + A c)) - c^T Lambda^-1 c / 2, found here
    by numpy's least-squares solver on the stacked system [C^-1/2 D; Lambda^-1/2]
    c = [C^-1/2 r; 0] -- with very wide priors, the plain weighted fit of
    Johnson et al. that the paper follows."""
    orc_o = cases.oracle_for(W_SMALL, calib_sigma=s, calib_mode=1)
    orc_0 = cases.oracle_for(W_SMALL)
    th = cases.theta_rows(W_SMALL, 3, seed=74)
    a = orc_o.eval(th)
    lam = np.asarray(orc_0.spec_lam)
    x = (2.0 * lam - (lam[0] + lam[-1])) / (lam[-1] - lam[0])
    A = cheb(x, len(s))
    for r in range(th.shape[0]):
        mu, d, sig, lnl_rest = _lnl_parts(orc_0, th, r)
        Dw = mu[:, None] * A / sig[:, None]
        rw = (d - mu) / sig
        G = np.vstack([Dw, np.diag(1.0 / np.asarray(s))])
        c = np.linalg.lstsq(G, np.concatenate([rw, np.zeros(len(s))]), rcond=None)[0]
        resid = (d - mu * (1.0 + A @ c)) / sig
        want = (np.sum(-0.5 * resid ** 2 - 0.5 * np.log(2 * np.pi * sig ** 2)) - 0.5 * np.sum((c / np.asarray(s)) ** 2)
                + lnl_rest)
        assert abs(a["lnl"][r] - want) < 1e-7 * max(1.0, abs(want)), (r, a["lnl"][r], want)


def test_optimised_and_marginalised_differ_by_the_occam_terms():
    """lnL(optimised) - lnL(marginalised) = ln|M| / 2 + ln|Lambda| / 2 (Eq.
    app_polymarg's last two terms), with M = D^T C^-1 D + Lambda^-1 from numpy."""
    s = [0.2, 0.1, 0.1, 0.05]
    orc_o = cases.oracle_for(W_SMALL, calib_sigma=s, calib_mode=1)
    orc_m = cases.oracle_for(W_SMALL, calib_sigma=s)
    orc_0 = cases.oracle_for(W_SMALL)
    th = cases.theta_rows(W_SMALL, 3, seed=75)
    lo, lm = orc_o.eval(th)["lnl"], orc_m.eval(th)["lnl"]
    lam = np.asarray(orc_0.spec_lam)
    x = (2.0 * lam - (lam[0] + lam[-1])) / (lam[-1] - lam[0])
    A = cheb(x, len(s))
    for r in range(th.shape[0]):
        mu, d, sig, _ = _lnl_parts(orc_0, th, r)
        Dw = mu[:, None] * A / sig[:, None]
        M = Dw.T @ Dw + np.diag(1.0 / np.asarray(s) ** 2)
        want = 0.5 * np.linalg.slogdet(M)[1] + 0.5 * np.sum(np.log(np.asarray(s) ** 2))
        # both lnL are large for random rows (far from the data): the difference
        # carries their FP64 rounding
        assert lo[r] - lm[r] == pytest.approx(want, rel=1e-8, abs=1e-8 + 4e-16 * abs(lm[r]))
