"""Pins of the oracle's nebular age axis (App. C: the nebular cube interpolated
trilinearly in gas metallicity, ionising-source age and ionisation parameter,
queried at each SSP age, scaled by that age's ionising output Q; only SSP ages
inside the cube's tabulated ages contribute).

The nebular part of the young array (the oracle's Y output with the nebular
emission, minus the same row's stellar young flux) is recomputed here with
numpy from the oracle's weights W and ionising outputs Q: per nebular SSP age
a, q_a = sum_{n,m} W Q, times 10 to the power of the cube interpolated
bilinearly in (log U, log Z_gas) on the two planes bracketing log t_a and
linearly in log age between them.  Cases: cube ages on the SSP ages (no age
interpolation), between them (interpolation), covering part of the young ages
(the others contribute nothing and keep their ionising flux), and planes all
equal to the age-free template (the model without an age axis).
"""
import dataclasses

import numpy as np
import pytest

import synth
from tests import cases

W = synth.shrink(synth.WORKLOADS["phot_107x12x6000_b1024"], n_age=20, n_feh=4, n_lam=1500, n_sfh=10, batch=8)


@pytest.fixture(scope="module")
def base():
    return cases.oracle_for(W)


def bracket(x, v):
    x = np.asarray(x)
    if v <= x[0]:
        return 0, 1.0, min(1, len(x) - 1), 0.0
    if v >= x[-1]:
        return len(x) - 2, 0.0, len(x) - 1, 1.0
    j = np.searchsorted(x, v, side="right") - 1
    t = (v - x[j]) / (x[j + 1] - x[j])
    return j, 1.0 - t, j + 1, t


def with_axis(base, ages, planes):
    g = dataclasses.replace(base.grid, neb_log_age=np.asarray(ages, dtype=np.float64),
                            neb_tab=np.asarray(planes, dtype=np.float64))
    return dataclasses.replace(base, grid=g)


def nebular_part(orc, base, th):
    """numpy: sum over nebular SSP ages of q_a 10^(trilinear cube)."""
    g = orc.grid
    jz = cases.z_column(W.n_sfh, W.zmode)
    gas_z, gas_u = th[jz + 5], th[jz + 6]
    Wt = base.row(th)["W"]
    Q = base.q()
    la = np.asarray(g.log_age_yr)
    u0, wu0, u1, wu1 = bracket(g.neb_logu, gas_u)
    z0, wz0, z1, wz1 = bracket(g.neb_logz, gas_z)
    N = np.zeros(len(g.lam_aa))
    for a in range(len(la)):
        if la[a] > base.bc_edge_log_age_yr or la[a] < g.neb_log_age[0] or la[a] > g.neb_log_age[-1]:
            continue
        qa = np.sum(Wt[:, :, a] * Q[:, :, a])
        i0, w0, i1, w1 = bracket(g.neb_log_age, la[a])
        lg = 0.0
        for i, wi in ((i0, w0), (i1, w1)):
            P = g.neb_tab[i]
            lg = lg + wi * (wu0 * wz0 * P[u0, z0] + wu0 * wz1 * P[u0, z1] + wu1 * wz0 * P[u1, z0] + wu1 * wz1 * P[u1, z1])
        N += qa * 10.0 ** lg
    return N


def stellar_young(base, th, ages_cut):
    """The young stellar array with the ionising flux of the ages in ages_cut removed."""
    g = base.grid
    Wt = base.row(th)["W"]
    la = np.asarray(g.log_age_yr)
    lam = np.asarray(g.lam_aa)
    Y = np.zeros(len(lam))
    for a in range(len(la)):
        if la[a] > base.bc_edge_log_age_yr:
            continue
        f = np.einsum("nm,nml->l", Wt[:, :, a], g.flux[:, :, a, :])
        if a in ages_cut:
            f = np.where(lam < 912.0, 0.0, f)
        Y += f
    return Y


def _check(base, orc, ages_cut, seed):
    th = cases.theta_rows(W, 3, seed=seed)
    for r in range(3):
        got = orc.row(th[r])
        assert got["status"] == 0
        want = stellar_young(base, th[r], ages_cut) + nebular_part(orc, base, th[r])
        np.testing.assert_allclose(got["Y"], want, rtol=1e-11, atol=1e-14 * np.abs(want).max())


def _young(base):
    la = np.asarray(base.grid.log_age_yr)
    return la[la <= base.bc_edge_log_age_yr]


def test_cube_ages_on_the_ssp_ages(base):
    ya = _young(base)
    rng = np.random.default_rng(150)
    planes = np.stack([base.grid.neb_tab + rng.normal(0.0, 0.3, base.grid.neb_tab.shape[:2])[:, :, None] - 0.5 * i
                       for i in range(len(ya))])
    orc = with_axis(base, ya, planes)
    _check(base, orc, set(range(len(ya))), 151)


def test_cube_ages_between_the_ssp_ages(base):
    ya = _young(base)
    ages = np.array([ya[0] - 0.1, 0.5 * (ya[0] + ya[-1]), ya[-1] + 0.05])
    planes = np.stack([base.grid.neb_tab - 0.7 * i + 0.1 * i * np.sin(np.arange(base.grid.neb_tab.shape[2]) / 50.0)
                       for i in range(3)])
    orc = with_axis(base, ages, planes)
    _check(base, orc, set(range(len(ya))), 152)


def test_young_ages_outside_the_cube_contribute_nothing(base):
    ya = _young(base)
    assert len(ya) >= 4
    ages = np.array([ya[1] - 0.01, ya[-2] + 0.01])
    planes = np.stack([base.grid.neb_tab, base.grid.neb_tab - 0.4])
    orc = with_axis(base, ages, planes)
    inside = {a for a in range(len(ya)) if ages[0] <= ya[a] <= ages[1]}
    assert 0 < len(inside) < len(ya)
    _check(base, orc, inside, 153)


def test_equal_planes_are_the_age_free_template(base):
    ya = _young(base)
    planes = np.stack([base.grid.neb_tab] * 3)
    orc = with_axis(base, [ya[0] - 0.2, ya[0] + 0.3, ya[-1] + 0.2], planes)
    th = cases.theta_rows(W, 6, seed=154)
    a, b = orc.eval(th), base.eval(th)
    np.testing.assert_allclose(a["phot"], b["phot"], rtol=1e-12)
    np.testing.assert_allclose(a["lnl"], b["lnl"], rtol=1e-12)


def test_a_cube_past_the_birth_cloud_edge_is_refused(base):
    ya = _young(base)
    with pytest.raises(ValueError):
        with_axis(base, [ya[0], base.bc_edge_log_age_yr + 1.0], np.stack([base.grid.neb_tab] * 2))
