"""Pins of the oracle's systematic noise floor (App. "sys_floor", Eq. app_noise_floor):
    sigma_eff^2 = s^2 sigma^2 + (f_calib |m|)^2 + (f_data |d|)^2 + j^2,
each term's column holding log10 of its value, the log-normalisation kept.

Pinned against what the definition fixes independently of the oracle's floor
code: the unfloored oracle with sigma inflated by hand (data-anchored term,
jitter, and the model-anchored term with the row's own model flux), the closed
form in the error scale s (lnL = C - N ln s - chi^2 / (2 s^2), maximal at
s^2 = chi^2 / N, as the paper states), s = 1 reproducing the plain Gaussian,
and central differences of the forward model for every column."""
import dataclasses

import numpy as np
import pytest

import oracle
import synth
from tests import cases

W_PHOT = "tiny_phot_16x4x512"
W_SPEC = "specphot_afe_107x12x5x6000_b2048"


def spec_workload():
    return synth.shrink(synth.WORKLOADS[W_SPEC], n_age=12, n_feh=3, n_lam=800, n_sfh=6, n_pix=120, batch=8)


def with_floor(orc, floor_phot=0, floor_spec=0):
    o = dataclasses.replace(orc, floor_phot=floor_phot, floor_spec=floor_spec)
    return o


def rows(w, n, seed, floor_phot=0, floor_spec=0, values=None):
    """Parameter rows with the floor columns appended (values: {key: array or scalar})."""
    d = cases.theta_dict(w, n, seed=seed)
    for k in oracle.floor_keys(floor_phot, floor_spec):
        d[k] = np.broadcast_to(np.asarray(values[k], dtype=np.float64), (n,)).copy()
    return oracle.pack_theta(d, w.n_sfh, w.zmode, w.sample_sigma_gal, floor_phot, floor_spec)


def const_term(sigma, mask=None):
    m = np.ones(sigma.size, bool) if mask is None else mask.astype(bool)
    return -0.5 * np.sum(np.log(2 * np.pi * sigma[m] ** 2)), int(m.sum())


def test_layout_and_unit_scale_is_the_plain_gaussian():
    w = synth.WORKLOADS[W_PHOT]
    orc = cases.oracle_for(w)
    o2 = with_floor(orc, floor_phot=oracle.FLOOR_ERR_SCALE)
    assert o2.n_param == orc.n_param + 1
    th0 = rows(w, 6, 1)
    th1 = rows(w, 6, 1, floor_phot=oracle.FLOOR_ERR_SCALE, values={"log_err_scale_phot": 0.0})
    assert np.array_equal(th1[:, :-1], th0)
    a, b = orc.eval(th0), o2.eval(th1)
    assert np.array_equal(a["status"], b["status"])
    assert np.allclose(b["lnl"], a["lnl"], rtol=1e-14, atol=0)


def test_error_scale_closed_form_and_its_maximum():
    """lnL(s) = C - N ln s - chi^2/(2 s^2) with chi^2 and C from the unfloored
    oracle; the analytic d lnL / d log10 s vanishes at s^2 = chi^2 / N and lnL
    is larger there than at nearby s."""
    w = synth.WORKLOADS[W_PHOT]
    orc = cases.oracle_for(w)
    th0 = rows(w, 5, 2)
    a = orc.eval(th0)
    ok = a["status"] == 0
    assert ok.all()
    C, N = const_term(np.asarray(orc.phot_sigma))
    chi2 = 2.0 * (C - a["lnl"])
    o2 = with_floor(orc, floor_phot=oracle.FLOOR_ERR_SCALE)
    for ls in (-0.4, 0.0, 0.3, 1.1):
        th = rows(w, 5, 2, oracle.FLOOR_ERR_SCALE, values={"log_err_scale_phot": ls})
        s = 10.0 ** ls
        ref = C - N * np.log(s) - chi2 / (2 * s * s)
        assert np.allclose(o2.eval(th)["lnl"], ref, rtol=1e-12, atol=0)
    ls_best = 0.5 * np.log10(chi2 / N)
    th = rows(w, 5, 2, oracle.FLOOR_ERR_SCALE, values={"log_err_scale_phot": ls_best})
    g = o2.grad(th)["grad"][:, -1]
    assert np.abs(g).max() < 1e-8 * N
    l_best = o2.eval(th)["lnl"]
    for dl in (-0.01, 0.01):
        th_d = rows(w, 5, 2, oracle.FLOOR_ERR_SCALE, values={"log_err_scale_phot": ls_best + dl})
        assert np.all(o2.eval(th_d)["lnl"] < l_best)


@pytest.mark.parametrize("arm", ["phot", "spec"])
def test_data_anchored_floor_and_jitter_inflate_sigma(arm):
    """f_data |d| and j add in quadrature to sigma: equal to the unfloored
    oracle with sigma^2 + (f_data d)^2 + j^2 supplied as the errors."""
    w = synth.WORKLOADS[W_PHOT] if arm == "phot" else spec_workload()
    orc = cases.oracle_for(w)
    bits = oracle.FLOOR_F_DATA | oracle.FLOOR_JITTER
    d = np.asarray(orc.phot_d if arm == "phot" else orc.spec_d)
    sg = np.asarray(orc.phot_sigma if arm == "phot" else orc.spec_sigma)
    lfd, lj = -1.3, np.log10(0.5 * np.median(sg))
    vals = {f"log_f_data_{arm}": lfd, f"log_jitter_{arm}": lj}
    fp, fs = (bits, 0) if arm == "phot" else (0, bits)
    th = rows(w, 6, 3, fp, fs, vals)
    got = with_floor(orc, fp, fs).eval(th)
    sig2 = np.sqrt(sg ** 2 + (10 ** lfd * d) ** 2 + (10 ** lj) ** 2)
    ref_orc = dataclasses.replace(orc)
    if arm == "phot":
        ref_orc.set_data(phot_d=d, phot_sigma=sig2)
    else:
        ref_orc.set_data(spec_d=d, spec_sigma=sig2)
    ref = ref_orc.eval(rows(w, 6, 3))
    assert np.array_equal(got["status"], ref["status"])
    ok = ref["status"] == 0
    assert ok.any()
    assert np.allclose(got["lnl"][ok], ref["lnl"][ok], rtol=1e-12, atol=0)


@pytest.mark.parametrize("arm", ["phot", "spec"])
def test_model_anchored_floor_is_sigma_inflated_by_the_row_model(arm):
    """f_calib |m| with m the row's own model prediction: per row, equal to the
    unfloored oracle given sigma^2 + (f_calib m)^2 as the errors (the model does
    not depend on the errors)."""
    w = synth.WORKLOADS[W_PHOT] if arm == "phot" else spec_workload()
    orc = cases.oracle_for(w)
    fp, fs = (oracle.FLOOR_F_CALIB, 0) if arm == "phot" else (0, oracle.FLOOR_F_CALIB)
    lfc = -1.0
    th = rows(w, 4, 4, fp, fs, {f"log_f_calib_{arm}": lfc})
    got = with_floor(orc, fp, fs).eval(th)
    th0 = rows(w, 4, 4)
    base = orc.eval(th0)
    sg = np.asarray(orc.phot_sigma if arm == "phot" else orc.spec_sigma)
    d = np.asarray(orc.phot_d if arm == "phot" else orc.spec_d)
    for r in range(4):
        if base["status"][r]:
            continue
        m = base["phot"][r] if arm == "phot" else base["spec"][r]
        o = dataclasses.replace(orc)
        s2 = np.sqrt(sg ** 2 + (10 ** lfc * m) ** 2)
        if arm == "phot":
            o.set_data(phot_d=d, phot_sigma=s2)
        else:
            o.set_data(spec_d=d, spec_sigma=s2)
        ref = o.eval(th0[r:r + 1])
        assert np.allclose(got["lnl"][r], ref["lnl"][0], rtol=1e-12, atol=0)


@pytest.mark.parametrize("arm", ["phot", "spec"])
def test_floor_gradient_against_central_differences(arm):
    """All four terms on: the analytic gradient (every column, including the
    floor's and logmass, whose derivative gains the model-anchored term) against
    central differences of the oracle's forward model."""
    w = synth.WORKLOADS[W_PHOT] if arm == "phot" else spec_workload()
    orc = cases.oracle_for(w)
    bits = 15
    fp, fs = (bits, 0) if arm == "phot" else (0, bits)
    sg = np.asarray(orc.phot_sigma if arm == "phot" else orc.spec_sigma)
    vals = {f"log_err_scale_{arm}": 0.15, f"log_f_calib_{arm}": -1.2, f"log_f_data_{arm}": -1.6,
            f"log_jitter_{arm}": np.log10(0.3 * np.median(sg))}
    o2 = with_floor(orc, fp, fs)
    th = rows(w, 4, 5, fp, fs, vals)
    ga = o2.grad(th)
    fd = o2.grad_fd(th, h_rel=1e-6)
    ok = ga["status"] == 0
    assert ok.any()
    for r in np.nonzero(ok)[0]:
        ref = fd[r, :o2.n_param]
        scale = np.abs(ref).max()
        err = np.abs(ga["grad"][r] - ref) / np.maximum(np.abs(ref), 1e-6 * scale)
        assert err.max() < 1e-4, (r, int(err.argmax()), ga["grad"][r][err.argmax()], ref[err.argmax()])
    # the floor columns are the last four and carry a real gradient
    assert np.all(np.abs(ga["grad"][ok][:, -4:]) > 0)
