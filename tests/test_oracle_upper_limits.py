"""Pins of the oracle's photometric upper limits (Sec. 4.1 likelihood, App.
line_lik, Eq. app_line_chi2_UL): a band flagged as an upper limit adds
((d - m)/sigma_eff)^2 to chi^2 only when the model m exceeds the limit d, and
nothing while m <= d; its -1/2 ln(2 pi sigma_eff^2) stays in lnL.

Pinned against what the definition fixes independently of the oracle's
upper-limit branch: every limit respected gives the closed form sum of the
normalisations; every limit exceeded gives the plain Gaussian of the unflagged
oracle; a mix equals the unflagged oracle on data min(d, m) in the flagged
bands (the model does not depend on the data); a respected limit's value does
not enter lnL (except through a data-anchored noise floor, whose closed form is
checked too); a flag on a masked band changes nothing; and the analytic
gradient against central differences of the forward model."""
import dataclasses

import numpy as np

import oracle
import synth
from tests import cases

W_PHOT = "tiny_phot_16x4x512"


def setup(n=6, seed=11):
    w = synth.WORKLOADS[W_PHOT]
    orc = cases.oracle_for(w)
    th = cases.theta_rows(w, n, seed=seed)
    base = orc.eval(th)
    ok = base["status"] == 0
    assert ok.all()
    return w, orc, th, base


def flagged(orc, upper, d=None, sigma=None):
    o = dataclasses.replace(orc, phot_upper=np.asarray(upper, np.uint8))
    if d is not None:
        o.set_data(phot_d=d, phot_sigma=orc.phot_sigma if sigma is None else sigma)
    return o


def norm_const(sigma):
    return -0.5 * np.sum(np.log(2.0 * np.pi * np.asarray(sigma) ** 2))


def test_respected_limits_cost_only_the_normalisation():
    w, orc, th, base = setup()
    nb = len(orc.phot_sigma)
    for r in range(th.shape[0]):
        m = base["phot"][r]
        o = flagged(orc, np.ones(nb), d=m * 1.3 + 1e-3 * np.abs(m).max())
        got = o.eval(th[r:r + 1])["lnl"][0]
        assert np.isclose(got, norm_const(orc.phot_sigma), rtol=1e-14, atol=0)


def test_exceeded_limits_are_the_plain_gaussian():
    w, orc, th, base = setup()
    nb = len(orc.phot_sigma)
    for r in range(th.shape[0]):
        m = base["phot"][r]
        d = m * 0.7
        sg = 0.05 * np.maximum(np.abs(m), 1e-3 * np.abs(m).max())   # limits 6 sigma below the model
        plain = dataclasses.replace(orc)
        plain.set_data(phot_d=d, phot_sigma=sg)
        ref = plain.eval(th[r:r + 1])["lnl"][0]
        got = flagged(orc, np.ones(nb), d=d, sigma=sg).eval(th[r:r + 1])["lnl"][0]
        assert ref < norm_const(sg) - 1.0     # a real penalty
        assert np.isclose(got, ref, rtol=1e-14, atol=0)


def test_mixed_flags_equal_the_gaussian_on_clipped_data():
    """Half the bands flagged, the workload's mock data (some limits respected,
    some exceeded per row): equal to the unflagged oracle on data min(d, m)."""
    w, orc, th, base = setup(8, 12)
    nb = len(orc.phot_sigma)
    up = (np.arange(nb) % 2).astype(np.uint8)
    o = flagged(orc, up)
    got = o.eval(th)["lnl"]
    d = np.asarray(orc.phot_d)
    n_resp = n_exc = 0
    for r in range(th.shape[0]):
        m = base["phot"][r]
        dc = np.where(up == 1, np.minimum(d, m), d)
        n_resp += int(np.sum((up == 1) & (m <= d)))
        n_exc += int(np.sum((up == 1) & (m > d)))
        plain = dataclasses.replace(orc)
        plain.set_data(phot_d=dc, phot_sigma=orc.phot_sigma)
        ref = plain.eval(th[r:r + 1])["lnl"][0]
        assert np.isclose(got[r], ref, rtol=1e-13, atol=0), r
    assert n_resp > 0 and n_exc > 0


def test_respected_limit_value_does_not_enter_lnl():
    w, orc, th, base = setup(4, 13)
    nb = len(orc.phot_sigma)
    m = base["phot"][0]
    up = np.zeros(nb, np.uint8)
    up[3] = 1
    vals = []
    for f in (1.01, 3.0, 100.0):
        d = np.array(orc.phot_d, dtype=np.float64)
        d[3] = m[3] * f
        vals.append(flagged(orc, up, d=d).eval(th[:1])["lnl"][0])
    assert vals[0] == vals[1] == vals[2]


def test_respected_limits_with_a_data_anchored_floor():
    """With f_data on, a respected limit still sets sigma_eff: lnL =
    sum_b -1/2 ln(2 pi (sigma_b^2 + (f_data d_b)^2)) (Eq. app_noise_floor)."""
    w, orc, th, base = setup(3, 14)
    nb = len(orc.phot_sigma)
    lfd = -0.8
    sg = np.asarray(orc.phot_sigma)
    for r in range(th.shape[0]):
        m = base["phot"][r]
        d = m * 2.0 + 1e-3 * np.abs(m).max()
        o = flagged(orc, np.ones(nb), d=d)
        o = dataclasses.replace(o, floor_phot=oracle.FLOOR_F_DATA)
        row = np.concatenate([th[r], [lfd]])[None, :]
        got = o.eval(row)["lnl"][0]
        ref = -0.5 * np.sum(np.log(2.0 * np.pi * (sg ** 2 + (10 ** lfd * d) ** 2)))
        assert np.isclose(got, ref, rtol=1e-13, atol=0)


def test_flag_on_a_masked_band_changes_nothing():
    w, orc, th, base = setup(4, 15)
    nb = len(orc.phot_sigma)
    mask = np.ones(nb, np.uint8)
    mask[::3] = 0
    up = np.zeros(nb, np.uint8)
    up[::3] = 1
    a = dataclasses.replace(orc, phot_mask=mask).eval(th)["lnl"]
    b = dataclasses.replace(orc, phot_mask=mask, phot_upper=up).eval(th)["lnl"]
    assert np.array_equal(a, b)


def test_gradient_against_central_differences():
    """Every other band flagged on the mock data, with and without the full
    noise floor: the analytic gradient against central differences, at rows
    whose flagged bands all sit at least 1 % from their limit (the kink)."""
    w, orc, th, base = setup(10, 16)
    nb = len(orc.phot_sigma)
    up = (np.arange(nb) % 2).astype(np.uint8)
    d = np.asarray(orc.phot_d)
    far = np.array([np.all(np.abs(base["phot"][r][up == 1] / d[up == 1] - 1) > 0.01) for r in range(th.shape[0])])
    assert far.sum() >= 3
    th = th[far]
    sg = np.asarray(orc.phot_sigma)
    vals = [0.1, -1.3, -1.7, np.log10(0.3 * np.median(sg))]
    for bits in (0, 15):
        o = dataclasses.replace(orc, phot_upper=up, floor_phot=bits)
        t = th if bits == 0 else np.concatenate([th, np.tile(vals, (th.shape[0], 1))], axis=1)
        ga = o.grad(t)
        fd = o.grad_fd(t, h_rel=1e-6)
        assert np.all(ga["status"] == 0)
        assert np.allclose(ga["lnl"], o.eval(t)["lnl"], rtol=1e-14, atol=0)
        for r in range(t.shape[0]):
            ref = fd[r, :o.n_param]
            scale = np.abs(ref).max()
            # (columns below 1e-4 of the largest carry ~1e-8 of difference round-off)
            err = np.abs(ga["grad"][r] - ref) / np.maximum(np.abs(ref), 1e-4 * scale)
            assert err.max() < 1e-4, (bits, r, int(err.argmax()))
