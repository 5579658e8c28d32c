"""Pins of the oracle's analytic gradient (FP64 reverse pass) against facts
that do not reuse its derivation:

- central finite differences of the oracle's own forward model (which the
  pins of test_oracle_pins.py tie to the paper), on every parameter column,
  for five workload shapes (photometry with a power-law diffuse law;
  nebular + Kriek & Conroy dust; [a/Fe] + an LSF-convolved spectrum; the same
  with a sampled sigma_gal; the same with a marginalised calibration
  polynomial);
- the closed form of d lnL / d logmass (every model datum scales with
  10^logmass, Sec. 2.6);
- homogeneity of the weights in the SFH masses (App. B: W is linear in m_i),
  so that sum_i m_i dlnL/dm_i = dlnL/dlogmass / ln 10 exactly.
"""
import math

import numpy as np
import pytest

import oracle
import synth
from tests import cases

SHAPES = {
    "tiny": ("tiny_phot_16x4x512", None),
    "neb_kc13": ("phot_107x12x6000_b1024", dict(n_lam=1200, n_sfh=16)),
    "afe_spec": ("specphot_afe_107x12x5x6000_b2048", dict(n_lam=1200, n_sfh=16, n_pix=240)),
    "sgal_spec": ("specphot_afe_sgal_107x12x5x6000_b2048", dict(n_lam=1200, n_sfh=16, n_pix=240)),
    "calib_spec": ("specphot_afe_107x12x5x6000_b2048", dict(n_lam=1200, n_sfh=16, n_pix=240)),
    "calib_opt_spec": ("specphot_afe_107x12x5x6000_b2048", dict(n_lam=1200, n_sfh=16, n_pix=240)),
}
# prior widths of a 5-term calibration polynomial, marginalised or optimised
CALIB = {"calib_spec": [0.2, 0.1, 0.1, 0.05, 0.05], "calib_opt_spec": [0.2, 0.1, 0.1, 0.05, 0.05]}
CALIB_MODE = {"calib_opt_spec": 1}


@pytest.fixture(scope="module", params=list(SHAPES))
def shape(request):
    wname, sh = SHAPES[request.param]
    w = synth.WORKLOADS[wname]
    if sh:
        w = synth.shrink(w, **sh)
    return w, cases.oracle_for(w, calib_sigma=CALIB.get(request.param), calib_mode=CALIB_MODE.get(request.param, 0))


def test_analytic_gradient_matches_central_differences(shape):
    w, orc = shape
    th = cases.theta_rows(w, 3, seed=31)
    g = orc.grad(th)
    fd = orc.grad_fd(th, h_rel=1e-7)
    ref = orc.eval(th)
    assert np.array_equal(g["status"], ref["status"])
    assert np.array_equal(g["lnl"], ref["lnl"])
    for r in range(th.shape[0]):
        sc = np.abs(fd[r]).max()
        err = np.abs(g["grad"][r] - fd[r]) / sc
        assert err.max() < 2e-6, (r, int(err.argmax()), err.max())


def test_dlogmass_closed_form_and_mass_homogeneity(shape):
    w, orc = shape
    th = cases.theta_rows(w, 3, seed=32)
    g = orc.grad(th)["grad"]
    res = orc.eval(th)
    nz = w.n_sfh if w.zmode == 0 else 1
    j_mass = w.n_sfh + nz + 1
    for r in range(th.shape[0]):
        want = 0.0
        if orc.n_filt:
            m = res["phot"][r]
            want += math.log(10) * np.sum((orc.phot_d - m) / orc.phot_sigma ** 2 * m)
        if orc.n_pix:
            m = res["spec"][r]
            # pixels without model nodes in reach are out of the likelihood (and have m = 0)
            u = (orc.spec_d - m) / orc.spec_sigma ** 2
            if orc.calib_sigma is not None:
                # marginalised calibration (App. E): with p = A c*, c* = M^-1 b and
                # q_i = A_i M^-1 A_i^T, d lnL / d mu_i = [(d - mu (1+p))(1+p) - mu q] / sigma^2
                lam = np.asarray(orc.spec_lam)
                x = (2.0 * lam - (lam[0] + lam[-1])) / (lam[-1] - lam[0])
                n = len(orc.calib_sigma)
                A = np.polynomial.chebyshev.chebvander(x, n - 1)
                inc = m != 0
                Dw = (m[:, None] * A / orc.spec_sigma[:, None])[inc]
                M = Dw.T @ Dw + np.diag(1.0 / np.asarray(orc.calib_sigma) ** 2)
                bvec = Dw.T @ ((orc.spec_d - m) / orc.spec_sigma)[inc]
                Minv = np.linalg.inv(M)
                pp = A @ (Minv @ bvec)
                # the optimised polynomial has no ln|M| term (c* is stationary)
                qq = np.einsum("im,mn,in->i", A, Minv, A) if orc.calib_mode == 0 else 0.0
                u = ((orc.spec_d - m * (1 + pp)) * (1 + pp) - m * qq) / orc.spec_sigma ** 2
                u[~inc] = 0.0
            want += math.log(10) * np.sum(u * m)
        assert g[r, j_mass] == pytest.approx(want, rel=1e-9, abs=1e-9 * abs(want))
        euler = np.dot(th[r, :w.n_sfh], g[r, :w.n_sfh])
        assert euler == pytest.approx(g[r, j_mass] / math.log(10), rel=1e-9, abs=1e-9 * abs(g[r, j_mass]))


def test_bad_rows_have_zero_gradient():
    w = synth.WORKLOADS["tiny_phot_16x4x512"]
    orc = cases.oracle_for(w)
    th = cases.theta_rows(w, 3, seed=33)
    jz = w.n_sfh * 2 + 2
    th[0, jz] = w.zf + 1
    th[1, 0] = np.nan
    g = orc.grad(th)
    assert list(g["status"][:2]) == [oracle.BAD_Z, oracle.BAD_THETA]
    assert np.all(g["grad"][:2] == 0) and np.isneginf(g["lnl"][:2]).all()
    assert g["status"][2] == 0 and np.isfinite(g["lnl"][2])
