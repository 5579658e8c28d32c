"""Pins of the oracle's ionising-photon escape geometries (Sec. frac_obrun,
Eq. runaway_mix, the picket-fence geometry, App. dust_attn): with the runaway
fraction f_ob, the covered fraction 1 - f_ob powers the nebular continuum, the
escaping fraction of the nebular ages' ionising continuum bypasses the birth
cloud (runaway_bc) or every screen (picket), and the young array crosses
(1 - f_ob) e^{-tau_BC} + f_ob (runaway_bc) or splits into an escaping f_ob and a
covered 1 - f_ob behind both screens (picket).

Pinned against the model without a geometry (itself pinned elsewhere) and the
dust definitions: f_ob = 0 reproduces it exactly (the paper states this); at
f_ob = 1 runaway_bc equals the model with no nebular emission and no birth
cloud, and picket equals the unscreened young light plus the screened old
light of the geometry-free model; picket is affine in f_ob and runaway_bc quadratic
with the second difference -e^{-tau_d}(1 - e^{-tau_BC}) N / 2 set by the
nebular continuum N alone; values of f_ob outside [0, 1] are refused."""
import dataclasses

import numpy as np
import pytest

import oracle
import synth
from tests import cases

W_NAME = "phot_107x12x6000_b1024"


@pytest.fixture(scope="module")
def base():
    w = synth.shrink(synth.WORKLOADS[W_NAME], n_age=20, n_feh=3, n_lam=900, n_sfh=8, batch=4)
    orc = cases.oracle_for(w)
    assert w.use_nebular and orc.grid.neb_tab is not None
    d = cases.theta_dict(w, 4, seed=21)
    return w, orc, d


def geom(orc, g, **kw):
    return dataclasses.replace(orc, fesc_geometry=g, **kw)


def rows(w, d, g, fob):
    d = dict(d)
    if g:
        d["frac_obrun"] = np.full(d["sfh"].shape[0], float(fob))
    return oracle.pack_theta(d, w.n_sfh, w.zmode, fesc_geometry=g)


def test_layout_and_zero_escape_is_the_plain_model(base):
    w, orc, d = base
    ref = orc.eval(rows(w, d, 0, 0))
    assert (ref["status"] == 0).all()
    for g in (oracle.FESC_RUNAWAY_BC, oracle.FESC_PICKET):
        o = geom(orc, g)
        assert o.n_param == orc.n_param + 1
        got = o.eval(rows(w, d, g, 0.0))
        assert np.array_equal(got["status"], ref["status"])
        assert np.allclose(got["phot"], ref["phot"], rtol=1e-14, atol=0)
        assert np.allclose(got["lnl"], ref["lnl"], rtol=1e-14, atol=0)


def test_runaway_full_escape_is_no_nebular_and_no_birth_cloud(base):
    """f_ob = 1 under runaway_bc: T_BC = 1, nebular emission 0, the ionising
    continuum fully escaping: the geometry-free model without nebular emission
    and with tau_BC = 0."""
    w, orc, d = base
    o = geom(orc, oracle.FESC_RUNAWAY_BC)
    d0 = dict(d, tau_pow=np.zeros(4))
    ref = dataclasses.replace(orc, use_nebular=0)
    for r in range(4):
        got = o.row(rows(w, d, oracle.FESC_RUNAWAY_BC, 1.0)[r])
        exp = ref.row(rows(w, d0, 0, 0)[r])
        assert got["status"] == 0 and exp["status"] == 0
        assert np.allclose(got["F"], exp["F"], rtol=1e-13, atol=1e-300)


def test_picket_full_escape_is_unscreened_young_plus_screened_old(base):
    """f_ob = 1 under picket: the young light (ionising continuum included)
    escapes both screens and the old light crosses the diffuse one: F = Y +
    e^{-tau_d} O with Y and O the young and old sums of the geometry-free model
    without nebular emission (nothing removed below 912 A) and tau_d from the
    diffuse law's definition."""
    w, orc, d = base
    o = geom(orc, oracle.FESC_PICKET)
    no_neb = dataclasses.replace(orc, use_nebular=0)
    lam = np.asarray(orc.grid.lam_aa)
    for r in range(4):
        got = o.row(rows(w, d, oracle.FESC_PICKET, 1.0)[r])
        p = no_neb.row(rows(w, d, 0, 0)[r])
        td = oracle.dust_tau(w.dust_law, lam, d["diffuse_tau_kc"][r], d["diffuse_dust_index"][r])
        assert np.allclose(got["F"], p["Y"] + np.exp(-td) * p["O"], rtol=1e-12, atol=1e-300)


def test_picket_is_affine_in_the_escape_fraction(base):
    w, orc, d = base
    o = geom(orc, oracle.FESC_PICKET)
    for r in range(2):
        F = [o.row(rows(w, d, oracle.FESC_PICKET, f)[r])["F"] for f in (0.0, 0.5, 1.0)]
        assert np.allclose(F[1], 0.5 * (F[0] + F[2]), rtol=1e-12, atol=1e-300)


def test_runaway_is_quadratic_through_the_nebular_continuum(base):
    """F(f) = e^{-tau_d} [((1-f) e^{-tau_BC} + f)(Y + (1-f) N) + f Y_ion + O]:
    its second difference over f = 0, 1/2, 1 is -e^{-tau_d}(1 - e^{-tau_BC}) N / 2
    with N the nebular continuum (geometry-free Y with and without nebular
    emission) and the screens from the dust definitions; without nebular
    emission F is affine in f."""
    w, orc, d = base
    o = geom(orc, oracle.FESC_RUNAWAY_BC)
    g = orc.grid
    lam = np.asarray(g.lam_aa)
    for r in range(2):
        th = rows(w, d, oracle.FESC_RUNAWAY_BC, 0.0)[r:r + 1]
        F = [o.row(rows(w, d, oracle.FESC_RUNAWAY_BC, f)[r])["F"] for f in (0.0, 0.5, 1.0)]
        plain = orc.row(rows(w, d, 0, 0)[r])
        stellar = dataclasses.replace(orc, use_nebular=0).row(rows(w, d, 0, 0)[r])
        N = plain["Y"] - np.where(lam < 912.0, 0.0, stellar["Y"])
        assert N.max() > 0
        tbc = d["tau_pow"][r] * (lam / 5500.0) ** d["alpha_pow"][r]
        td = oracle.dust_tau(w.dust_law, lam, d["diffuse_tau_kc"][r], d["diffuse_dust_index"][r])
        want = -np.exp(-td) * (1.0 - np.exp(-tbc)) * N / 2.0
        got = F[0] - 2.0 * F[1] + F[2]
        assert np.allclose(got, want, rtol=1e-9, atol=1e-12 * np.abs(F[0]).max())
        assert th.shape[1] == o.n_param
    on = geom(dataclasses.replace(orc, use_nebular=0), oracle.FESC_RUNAWAY_BC)
    F = [on.row(rows(w, d, oracle.FESC_RUNAWAY_BC, f)[0])["F"] for f in (0.0, 0.5, 1.0)]
    assert np.allclose(F[1], 0.5 * (F[0] + F[2]), rtol=1e-12, atol=1e-300)


@pytest.mark.parametrize("g", [1, 2])
def test_escape_fraction_outside_the_unit_interval_is_refused(base, g):
    w, orc, d = base
    o = geom(orc, g)
    th = rows(w, d, g, 0.3)
    th[1, -1] = -0.01
    th[2, -1] = 1.01
    st = o.eval(th)["status"]
    assert st[0] == 0 and st[3] == 0
    assert st[1] == st[2] == 1   # ORC_BAD_THETA


@pytest.mark.parametrize("g", [1, 2])
def test_analytic_gradient_against_central_differences(base, g):
    """The oracle's hand-derived reverse pass under each geometry (d lnL / d f_ob
    included) against central differences of its forward model."""
    w, orc, d = base
    o = geom(orc, g)
    d = dict(d, frac_obrun=np.array([0.1, 0.35, 0.6, 0.9]))
    th = oracle.pack_theta(d, w.n_sfh, w.zmode, fesc_geometry=g)
    ga = o.grad(th)
    assert np.all(ga["status"] == 0)
    assert np.allclose(ga["lnl"], o.eval(th)["lnl"], rtol=1e-14, atol=0)
    fd = o.grad_fd(th, h_rel=1e-6)
    for r in range(th.shape[0]):
        ref = fd[r, :o.n_param]
        # every column within 1e-5 of the row's largest derivative (the central
        # differences' round-off, ~1e-16 |lnL| / h, is ~1e-7 here), and the f_ob
        # column within 1e-4 of itself
        err = np.abs(ga["grad"][r] - ref) / np.abs(ref).max()
        # (the redshift column's difference quotient spans kinks of the filter
        # samples' interpolation between model nodes: 1e-4 there)
        jz = cases.z_column(w.n_sfh, w.zmode)
        assert err[jz] < 1e-4
        err[jz] = 0.0
        assert err.max() < 1e-5, (r, int(err.argmax()))
        assert abs(ga["grad"][r, -1] - ref[-1]) < 1e-4 * abs(ref[-1])
    assert np.abs(ga["grad"][:, -1]).min() > 0
