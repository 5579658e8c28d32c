"""Pins of the oracle's linear SFH scheme (App. B, Eq. tent_integral): the SFR
is linear in lookback time across each bin, through per-edge rates psi_0..psi_NT,
and an SSP age node receives the integral of the SFR against its log-age tent.

The oracle integrates each piece in closed form (antiderivatives of psi and
psi ln t); the pins integrate the same definition numerically with scipy's
adaptive quadrature, node by node, and check mass conservation, the clamps at
the ends of the age axis, the clip of negative pieces and the parameter layout."""
import dataclasses

import numpy as np
import pytest

import oracle
import synth
from tests import cases

integrate = pytest.importorskip("scipy.integrate")

W_NAME = "tiny_phot_16x4x512"


def linear_case(zmode=1):
    w = synth.WORKLOADS[W_NAME]
    w = dataclasses.replace(w, zmode=zmode)
    orc = cases.oracle_for(w)
    return w, dataclasses.replace(orc, sfh_scheme=1)


def psi_rows(n_sfh, n, seed, scale=1e-9):
    """Per-edge SFRs (Msun/yr), positive and varied."""
    rng = np.random.default_rng(seed)
    return scale * rng.gamma(1.5, 1.0, (n, n_sfh + 1))


def row(w, orc, psi, zeta=0.0, z=1.0):
    d = cases.theta_dict(w, 1, seed=7)
    d["sfh"] = psi.reshape(1, -1)
    d["logzsol"] = np.full_like(d["logzsol"], zeta)
    d["zred"][:] = z
    return oracle.pack_theta(d, w.n_sfh, w.zmode, 0, 0, 0, sfh_scheme=1)[0]


def edges(orc, n_sfh, z):
    t = oracle.cosmology(orc.H0, orc.Om0, z)["t_univ"] - oracle.cosmology(orc.H0, orc.Om0, orc.zf)["t_univ"]
    return oracle.sfh_edges(n_sfh, t)


def tent_masses_by_quadrature(orc, T, psi):
    """Mass per age node: sum over bins of the integral of psi(t) tau_a(t), tau_a
    the tent of node a in log(age) (1 below the youngest / above the oldest node
    for the end nodes), by adaptive quadrature with the nodes as breakpoints."""
    la = np.asarray(orc.grid.log_age_yr, dtype=np.float64)
    ta = 10.0 ** la
    NA = la.size

    def tent(a, t):
        if t <= ta[0]:
            return 1.0 if a == 0 else 0.0
        if t >= ta[-1]:
            return 1.0 if a == NA - 1 else 0.0
        j = np.searchsorted(ta, t) - 1
        u = (np.log(t) - np.log(ta[j])) / (np.log(ta[j + 1]) - np.log(ta[j]))
        return (1.0 - u) if a == j else (u if a == j + 1 else 0.0)

    out = np.zeros(NA)
    for i in range(len(T) - 1):
        t0, t1 = T[i], T[i + 1]

        def sfr(t):
            return psi[i] + (psi[i + 1] - psi[i]) * (t - t0) / (t1 - t0)
        pts = [p for p in ta if t0 < p < t1]
        for a in range(NA):
            lo = t0 if a == 0 else max(t0, ta[a - 1])
            hi = t1 if a == NA - 1 else min(t1, ta[a + 1])
            if hi <= lo:
                continue
            v, _ = integrate.quad(lambda t: sfr(t) * tent(a, t), lo, hi,
                                  points=[p for p in pts if lo < p < hi] or None, epsabs=0, epsrel=1e-12,
                                  limit=200)
            out[a] += v
    return out


@pytest.mark.parametrize("z", [0.3, 2.0, 6.0])
def test_linear_weights_match_quadrature_of_the_tent_integral(z):
    w, orc = linear_case()
    psi = psi_rows(w.n_sfh, 1, seed=int(10 * z))[0]
    th = row(w, orc, psi, zeta=float(orc.grid.feh[1]), z=z)   # [Fe/H] at a grid node: one metallicity
    st, W = orc.weights(th)
    assert st == 0
    got = W.sum(axis=(0, 1))
    T = edges(orc, w.n_sfh, z)
    ref = tent_masses_by_quadrature(orc, T, psi)
    assert np.allclose(got, ref, rtol=1e-9, atol=1e-12 * ref.max())
    # all of it at the [Fe/H] node
    assert np.allclose(W[0, 1], got, rtol=0, atol=0)


def test_linear_weights_conserve_each_bins_trapezoidal_mass():
    w, orc = linear_case(zmode=0)
    for seed in range(4):
        psi = psi_rows(w.n_sfh, 1, seed=seed)[0]
        th = row(w, orc, psi, z=1.5)
        st, W = orc.weights(th)
        T = edges(orc, w.n_sfh, 1.5)
        m = 0.5 * (psi[:-1] + psi[1:]) * np.diff(T)
        assert st == 0
        assert np.isclose(W.sum(), m.sum(), rtol=1e-13)
        assert np.all(W >= 0)


def test_constant_sfr_same_total_as_the_step_scheme():
    """A constant SFR forms psi dT_i in every bin under both schemes (the paper's
    figure: same mass per bin and in total, distributed differently)."""
    w, orc = linear_case()
    psi = np.full(w.n_sfh + 1, 2e-9)
    th = row(w, orc, psi, z=1.0)
    st, W = orc.weights(th)
    T = edges(orc, w.n_sfh, 1.0)
    step = dataclasses.replace(orc, sfh_scheme=0)
    d = cases.theta_dict(w, 1, seed=7)
    d["sfh"] = (2e-9 * np.diff(T)).reshape(1, -1)
    d["logzsol"] = np.zeros_like(d["logzsol"])
    d["zred"][:] = 1.0
    th_s = oracle.pack_theta(d, w.n_sfh, w.zmode)[0]
    st2, W2 = step.weights(th_s)
    assert st == 0 and st2 == 0
    assert np.isclose(W.sum(), W2.sum(), rtol=1e-13)
    assert not np.allclose(W, W2)   # the two schemes place it differently


def test_negative_rates_are_clipped_and_renormalised():
    w, orc = linear_case()
    psi = psi_rows(w.n_sfh, 1, seed=3)[0]
    psi[4] = -0.5 * psi[4]
    th = row(w, orc, psi, z=1.0)
    st, W = orc.weights(th)
    assert st == 0
    assert np.all(W >= 0)


def test_layout_has_one_more_sfh_column_and_forward_runs():
    w, orc = linear_case()
    step = dataclasses.replace(orc, sfh_scheme=0)
    assert orc.n_param == step.n_param + 1
    psi = psi_rows(w.n_sfh, 4, seed=5)
    th = np.stack([row(w, orc, p, z=1.0 + 0.5 * k) for k, p in enumerate(psi)])
    r = orc.eval(th)
    assert np.all(r["status"] == 0) and np.all(np.isfinite(r["lnl"]))


@pytest.mark.parametrize("clip", [False, True])
@pytest.mark.parametrize("zmode", [0, 1])
def test_analytic_gradient_against_central_differences(zmode, clip):
    """The oracle's hand-derived reverse pass of the linear scheme (each edge
    rate through two bins' tent shares and their scale to the trapezoidal
    mass, each edge's lookback time through T_max) against central differences
    of its forward model, every column.  With clip, every third edge rate is
    negative, so pieces are clipped and the scale to the trapezoidal mass
    differs from 1 (without clipping the shares sum to the trapezoid exactly
    and the scale's derivative vanishes)."""
    import dataclasses
    w = dataclasses.replace(synth.WORKLOADS["tiny_phot_16x4x512"], sfh_scheme=1, zmode=zmode)
    orc = cases.oracle_for(w)
    th = cases.theta_rows(w, 6, seed=31)
    if clip:
        th[:, 1:w.n_sfh + 1:3] *= -0.4
    ga = orc.grad(th)
    ok = ga["status"] == 0
    assert ok.sum() >= 4
    assert np.allclose(ga["lnl"][ok], orc.eval(th)["lnl"][ok], rtol=1e-14, atol=0)
    # central differences with steps relative to each value (edge SFRs are
    # ~1e-10 Msun/yr, far below the unit floor of the oracle's own grad_fd)
    fd = np.zeros_like(th)
    for j in range(th.shape[1]):
        h = np.where(th[:, j] == 0, 1e-6, 1e-6 * np.abs(th[:, j]))
        a, b = th.copy(), th.copy()
        a[:, j] += h
        b[:, j] -= h
        fd[:, j] = (orc.eval(a)["lnl"] - orc.eval(b)["lnl"]) / (2 * h)
    jz = cases.z_column(w.n_sfh, w.zmode, 1)
    for r in np.nonzero(ok)[0]:
        ref = fd[r, :orc.n_param]
        err = np.abs(ga["grad"][r] - ref) / np.abs(ref).max()
        # (the redshift column's difference quotient spans kinks of the filter
        # samples' interpolation between model nodes: 1e-4 there)
        assert err[jz] < 1e-4
        err[jz] = 0.0
        assert err.max() < 1e-5, (r, int(err.argmax()))
        # the edge rates: each within 1e-4 of itself where it is not tiny
        js = np.arange(w.n_sfh + 1)
        big = np.abs(ref[js]) > 1e-3 * np.abs(ref[js]).max()
        assert np.all(np.abs(ga["grad"][r, js][big] - ref[js][big]) < 1e-4 * np.abs(ref[js][big]))
