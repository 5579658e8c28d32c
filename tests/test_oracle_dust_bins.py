"""Pins of the oracle's age-binned attenuation (App. "dust_attn", Eq.
"app_tau_bin", Eq. "app_attn"): tau_a(lam) = sum_b M_ab kappa_b(lam; theta_b)
applied per SSP age node inside the contraction, then the diffuse screen.
Each case has an exact equivalent in the default two-component model, whose
code path is pinned elsewhere:

- a one-hot bin over the birth-cloud ages with the power law at (tau_pow,
  alpha_pow) is the default model (zero rows elsewhere: no birth-cloud law);
- one power-law bin over every age with the diffuse screen off is a power-law
  diffuse screen; the same with a KC13 bin is the KC13 diffuse screen;
- rows (1/2, 1/2) over two power-law bins of one slope act as one screen of the
  mean depth (a convex row averages optical depths, not transmissions);
- zero depths everywhere give the dust-free model.
"""
import dataclasses

import numpy as np
import pytest

import oracle
import synth
from tests import cases

W = synth.shrink(synth.WORKLOADS["phot_107x12x6000_b1024"], n_age=20, n_feh=4, n_lam=1500, n_sfh=10, batch=8)
RTOL = 1e-11


@pytest.fixture(scope="module")
def base():
    return cases.oracle_for(W)


def _cols(w):
    jz = cases.z_column(w.n_sfh, w.zmode)
    return dict(tau_pow=jz + 1, alpha_pow=jz + 2, tau_d=jz + 3, delta=jz + 4)


def _binned(orc, M, laws, dust_law=None):
    kw = dict(dust_bins=(np.asarray(M, dtype=np.float64), list(laws)))
    if dust_law is not None:
        kw["dust_law"] = dust_law
    return dataclasses.replace(orc, **kw)


def _same(a, b):
    assert np.array_equal(a["status"], b["status"])
    ok = a["status"] == 0
    np.testing.assert_allclose(a["phot"][ok], b["phot"][ok], rtol=RTOL, atol=0)
    np.testing.assert_allclose(a["lnl"][ok], b["lnl"][ok], rtol=RTOL, atol=1e-9)


def test_one_hot_birth_cloud_bin_is_the_default_model(base):
    th = cases.theta_rows(W, 6, seed=101)
    c = _cols(W)
    young = (base.grid.log_age_yr <= base.bc_edge_log_age_yr).astype(np.float64)[:, None]
    orc_b = _binned(base, young, [0])
    th_b = np.concatenate([th, th[:, [c["tau_pow"], c["alpha_pow"]]]], axis=1)
    assert th_b.shape[1] == orc_b.n_param
    _same(orc_b.eval(th_b), base.eval(th))


@pytest.mark.parametrize("law", [0, 1])
def test_one_bin_over_every_age_is_a_diffuse_screen(base, law):
    """kappa_1 with the diffuse screen off = the default model's diffuse screen
    of the same law (birth-cloud depth 0)."""
    th = cases.theta_rows(W, 6, seed=102)
    c = _cols(W)
    th[:, c["tau_pow"]] = 0.0
    ref = dataclasses.replace(base, dust_law=law).eval(th)
    orc_b = _binned(base, np.ones((len(base.grid.log_age_yr), 1)), [law], dust_law=law)
    th_b = np.concatenate([th, th[:, [c["tau_d"], c["delta"]]]], axis=1)
    th_b[:, c["tau_d"]] = 0.0
    _same(orc_b.eval(th_b), ref)


def test_convex_rows_average_the_optical_depths(base):
    th = cases.theta_rows(W, 6, seed=103)
    c = _cols(W)
    th[:, c["tau_pow"]] = 0.0
    t1 = np.linspace(0.1, 0.9, 6)
    t2 = np.linspace(1.2, 0.3, 6)
    ref_th = th.copy()
    ref_th[:, c["tau_d"]] = 0.5 * (t1 + t2)
    ref = dataclasses.replace(base, dust_law=0).eval(ref_th)
    n_age = len(base.grid.log_age_yr)
    orc_b = _binned(base, np.full((n_age, 2), 0.5), [0, 0], dust_law=0)
    slope = th[:, [c["delta"]]]
    th_b = np.concatenate([th, t1[:, None], slope, t2[:, None], slope], axis=1)
    th_b[:, c["tau_d"]] = 0.0
    _same(orc_b.eval(th_b), ref)
    # the transmission average (e^-t1 + e^-t2)/2 would differ
    assert np.all(np.exp(-0.5 * (t1 + t2)) < 0.5 * (np.exp(-t1) + np.exp(-t2)))


def test_zero_depths_give_the_dust_free_model(base):
    th = cases.theta_rows(W, 6, seed=104)
    c = _cols(W)
    th[:, c["tau_pow"]] = 0.0
    th[:, c["tau_d"]] = 0.0
    ref = base.eval(th)
    M = np.zeros((len(base.grid.log_age_yr), 3))
    M[:7, 0] = 1.0
    M[7:12, 1] = 0.3
    M[7:12, 2] = 0.7
    M[12:, 2] = 1.0
    orc_b = _binned(base, M, [0, 1, 0])
    th_b = np.concatenate([th, np.zeros((6, 6))], axis=1)
    th_b[:, -1] = th_b[:, -3] = -0.7     # slopes do not matter at zero depth
    _same(orc_b.eval(th_b), ref)


def test_matrix_checks(base):
    n_age = len(base.grid.log_age_yr)
    bad = np.ones((n_age, 2)) * 0.6          # rows summing to 1.2
    with pytest.raises(ValueError):
        _binned(base, bad, [0, 0])
    with pytest.raises(ValueError):
        _binned(base, np.ones((n_age - 1, 1)), [0])
    with pytest.raises(ValueError):
        dataclasses.replace(_binned(base, np.ones((n_age, 1)), [0]), use_lines=1)
    assert oracle.pack_theta({"sfh": np.ones((1, W.n_sfh)), "logzsol": np.zeros((1, W.n_sfh)), "afe": [0.0],
                              "logmass": [9.0], "zred": [1.0], "tau_pow": [0.0], "alpha_pow": [0.0],
                              "diffuse_tau_kc": [0.0], "diffuse_dust_index": [0.0], "gas_logz": [0.0],
                              "gas_logu": [-2.0], "dust_bins": [[0.1, -0.7, 0.2, -0.5]]},
                             W.n_sfh, W.zmode, dust_n_bin=2).shape[1] == _binned(base, np.ones((n_age, 2)) * 0.5,
                                                                                 [0, 0]).n_param
