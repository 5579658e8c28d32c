"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against a value that does not come from the oracle
itself: a closed form, an invariant, an independent library routine, brute
force on a tiny input, or a constant printed in the paper (tests/golden).
"""
import math
import os

import numpy as np
import pytest
from scipy import integrate

import oracle
import synth
from tests import cases

C_KMS = 299792.458
C_AA = 2.99792458e18
MPC_CM = 3.0856775814913673e24
GOLD = os.path.join(os.path.dirname(__file__), "golden", "paper_constants.txt")


def golden():
    out = {}
    for line in open(GOLD):
        if line.startswith("#") or not line.strip():
            continue
        name, val = line.split()[:2]
        out[name] = val
    return out


TINY = synth.WORKLOADS["tiny_phot_16x4x512"]


@pytest.fixture(scope="module")
def tiny():
    return cases.oracle_for(TINY)


# ---------------------------------------------------------------- cosmology
@pytest.mark.parametrize("z", [0.01, 0.5, 1.0, 3.0, 8.0, 12.0])
def test_cosmology_einstein_de_sitter(z):
    """Omega_m = 1: D_L = (2c/H0)(1+z)(1-(1+z)^-1/2), t = (2/3H0)(1+z)^-3/2."""
    H0 = 70.0
    c = oracle.cosmology(H0, 1.0, z)
    dl = 2 * C_KMS / H0 * (1 + z) * (1 - (1 + z) ** -0.5) * MPC_CM
    th = 3.0856775814913673e19 / H0 / 3.15576e7
    t = 2.0 / 3.0 * th * (1 + z) ** -1.5
    assert c["D_L"] == pytest.approx(dl, rel=1e-11)
    assert c["t_univ"] == pytest.approx(t, rel=1e-11)


@pytest.mark.parametrize("z", [0.0, 0.3, 2.0, 10.0, 30.0])
def test_age_lcdm_asinh_closed_form(z):
    H0, Om = 67.66, 0.3097
    OL = 1 - Om
    th = 3.0856775814913673e19 / H0 / 3.15576e7
    t = th * 2.0 / (3.0 * math.sqrt(OL)) * math.asinh(math.sqrt(OL / Om) * (1 + z) ** -1.5)
    assert oracle.cosmology(H0, Om, z)["t_univ"] == pytest.approx(t, rel=1e-11)


@pytest.mark.parametrize("z", [0.1, 1.0, 6.0, 12.0])
def test_comoving_distance_vs_scipy_quad(z):
    H0, Om = 67.66, 0.3097
    val, _ = integrate.quad(lambda x: 1 / math.sqrt(Om * (1 + x) ** 3 + 1 - Om), 0, z,
                            epsabs=0, epsrel=1e-13)
    dc = C_KMS / H0 * MPC_CM * val
    c = oracle.cosmology(H0, Om, z)
    assert c["D_C"] == pytest.approx(dc, rel=1e-11)
    assert c["D_L"] == pytest.approx((1 + z) * dc, rel=1e-12)


# ---------------------------------------------------------------- SFH edges / weights
def test_sfh_edges_layout():
    T = oracle.sfh_edges(8, 1.197e10)
    assert T[0] == 0 and T[1] == 5e6 and T[2] == 1e7
    assert T[-1] == pytest.approx(1.197e10, rel=1e-14)
    r = np.diff(np.log(T[2:]))
    assert np.allclose(r, r[0], rtol=1e-10)


def test_weights_conserve_mass(tiny):
    th = cases.theta_rows(TINY, 16, seed=11)
    th[:, :TINY.n_sfh] *= np.linspace(0.3, 3.0, 16)[:, None]
    for r in range(16):
        st, W = tiny.weights(th[r])
        assert st == 0
        assert W.sum() == pytest.approx(th[r, :TINY.n_sfh].sum(), rel=1e-13)
        assert (W >= 0).all()


def _grid_with_ages(log_ages, n_feh=3, n_lam=64, afe=None):
    g = synth.make_grid(n_age=len(log_ages), log_age=(log_ages[0], log_ages[-1]), n_feh=n_feh,
                        afe_nodes=afe, n_lam=n_lam, lam_um=(0.05, 3.0), seed=7)
    g.log_age_yr = np.asarray(log_ages, dtype=np.float64)
    return g


def test_single_bin_at_grid_metallicity_reproduces_ssp():
    """All mass in one SFH bin lying inside one Voronoi cell, [Fe/H] at a grid
    node, no dust, no nebular: F = mass * f_SSP exactly."""
    g = _grid_with_ages([6.9, 7.6, 8.3, 9.0, 9.7, 10.1])
    orc = oracle.Oracle(grid=g, n_sfh=8, zf=10.0, zmode=1, filters=synth.pack_filters(
        synth.make_filters_gauss(3, 0.6, 2.0)), phot_d=np.ones(3), phot_sigma=np.ones(3))
    th = np.zeros(orc.n_param)
    mass = 0.734
    th[0] = mass                      # bin 0 = [0, 5 Myr] inside cell of 10^6.9 yr
    th[8] = g.feh[1]                  # constant [Fe/H] at a node
    th[8 + 1 + 2] = 1.0               # zred
    res = orc.row(th)
    assert res["status"] == 0
    W = res["W"]
    assert W[0, 1, 0] == mass and np.count_nonzero(W) == 1
    np.testing.assert_array_equal(res["F"], mass * g.flux[0, 1, 0])


def test_weights_brute_force_quadrature():
    """W_a = int psi(t) 1[t nearer to t_a than to any other node] dt, by point
    classification on 2e5 sub-steps per bin (midpoint rule)."""
    g = _grid_with_ages(np.linspace(6.0, 10.1, 9))
    orc = oracle.Oracle(grid=g, n_sfh=6, zf=10.0, zmode=1)
    rng = np.random.default_rng(3)
    m = rng.random(6)
    th = np.zeros(orc.n_param)
    th[:6] = m
    th[6] = g.feh[0]
    th[6 + 1 + 2] = 0.7
    st, W = orc.weights(th)
    assert st == 0
    tmax = orc.row(th)["T_max"]
    T = oracle.sfh_edges(6, tmax)
    ta = 10 ** g.log_age_yr
    brute = np.zeros(len(ta))
    ns = 200000
    for i in range(6):
        t = T[i] + (np.arange(ns) + 0.5) * (T[i + 1] - T[i]) / ns
        a = np.abs(t[:, None] - ta[None, :]).argmin(axis=1)
        brute += np.bincount(a, minlength=len(ta)) * m[i] / ns
    np.testing.assert_allclose(W[0, 0], brute, atol=2e-5 * m.sum())


def test_metallicity_split_linear_and_clamped():
    g = _grid_with_ages([6.9, 7.6, 8.3, 9.0, 9.7, 10.1], n_feh=4)
    orc = oracle.Oracle(grid=g, n_sfh=8, zf=10.0, zmode=1)
    th = np.zeros(orc.n_param)
    th[0] = 1.0
    th[8 + 1 + 2] = 1.0
    for zeta, expect in [(g.feh[2], {2: 1.0}), (0.5 * (g.feh[1] + g.feh[2]), {1: 0.5, 2: 0.5}),
                         (g.feh[0] + 0.25 * (g.feh[1] - g.feh[0]), {0: 0.75, 1: 0.25}),
                         (g.feh[0] - 5, {0: 1.0}), (g.feh[-1] + 5, {3: 1.0})]:
        th[8] = zeta
        st, W = orc.weights(th)
        col = W[0, :, 0]
        want = np.zeros(4)
        for k, v in expect.items():
            want[k] = v
        np.testing.assert_allclose(col, want, rtol=1e-13, atol=1e-15)


def test_afe_bilinear_is_product_of_linears():
    g = _grid_with_ages([6.9, 7.6, 8.3, 9.0, 9.7, 10.1], n_feh=4, afe=(-0.2, 0.0, 0.2, 0.4, 0.6))
    orc = oracle.Oracle(grid=g, n_sfh=8, zf=10.0, zmode=1, use_afe=1)
    th = np.zeros(orc.n_param)
    th[:8] = 1.0 / 8
    th[8] = -0.3
    th[9] = 0.27      # afe
    th[9 + 2] = 1.0   # zred
    st, W = orc.weights(th)
    assert st == 0
    wa = np.zeros(5)
    wa[2], wa[3] = 1 - 0.35, 0.35
    orc0 = oracle.Oracle(grid=g, n_sfh=8, zf=10.0, zmode=1, use_afe=0)
    th0 = th.copy()
    _, W0 = orc0.weights(th0)      # afe ignored: all weight on the 0.0 node
    assert np.allclose(W0[1], W0.sum(axis=0)) and W0[1].sum() == pytest.approx(1.0)
    np.testing.assert_allclose(W, wa[:, None, None] * W0[1][None], rtol=1e-12, atol=1e-16)


# ---------------------------------------------------------------- Q (Eq. app_q)
def test_q_closed_form_linear_flux():
    """f = A*lam (f/lam constant): Q = (Lsun/h) A (912 - lam_0) exactly."""
    gold = golden()
    g = _grid_with_ages([6.9, 7.6, 8.3])
    A = 3e-18
    g.flux[:] = A * g.lam_aa
    orc = oracle.Oracle(grid=g, n_sfh=8, zf=10.0, zmode=1)
    Q = orc.q()
    want = float(gold["L_sun_erg_s"]) / 6.62607015e-27 * A * (float(gold["lyman_limit_aa"]) - g.lam_aa[0])
    np.testing.assert_allclose(Q, want, rtol=1e-12)


# ---------------------------------------------------------------- dust
def test_zero_dust_gives_unit_attenuation(tiny):
    th = cases.theta_rows(TINY, 4, seed=12)
    nz = TINY.n_sfh
    th[:, 2 * nz + 3] = 0.0   # tau_pow
    th[:, 2 * nz + 5] = 0.0   # diffuse_tau_kc
    for r in range(4):
        res = tiny.row(th[r])
        np.testing.assert_array_equal(res["F"], res["Y"] + res["O"])


def test_power_law_at_5500():
    assert oracle.dust_tau(0, [5500.0], 0.77, -0.7)[0] == 0.77
    lam = np.array([2750.0, 11000.0])
    np.testing.assert_allclose(oracle.dust_tau(0, lam, 1.0, -1.0), [2.0, 0.5], rtol=1e-15)


def test_kc13_calzetti_normalisation_and_drude_bump():
    """delta = 0: tau/tau_V*4.05 = k'(lam) + D(lam) with E_b = 0.85.  Calzetti's
    k' is normalised to R_V = k'(V) = 4.05 and k'(B) - k'(V) = 1 (E(B-V));
    the Drude bump peaks at 2175 A with height E_b and half maximum where
    lam^2 - lam0^2 = +-lam*350 A (FWHM 350 A)."""
    lam = np.array([4400.0, 5500.0])
    d_b = 0.85 / 1.9                     # delta that switches the bump off
    k_nob = oracle.dust_tau(1, lam, 1.0, d_b) * 4.05 / (lam / 5500.0) ** d_b
    assert k_nob[1] == pytest.approx(4.05, abs=0.01)
    assert k_nob[0] - k_nob[1] == pytest.approx(1.0, abs=0.02)
    lb = np.array([2175.0, 2007.03, 2357.03, 1500.0, 3500.0])
    with_b = oracle.dust_tau(1, lb, 1.0, 0.0) * 4.05
    no_b = oracle.dust_tau(1, lb, 1.0, d_b) * 4.05 / (lb / 5500.0) ** d_b
    bump = with_b - no_b
    assert bump[0] == pytest.approx(0.85, rel=1e-12)
    assert bump[1] == pytest.approx(0.425, rel=2e-4)
    assert bump[2] == pytest.approx(0.425, rel=2e-4)
    assert bump[3] < 0.2 and bump[4] < 0.2


# ---------------------------------------------------------------- photometry
def _phot_oracle(filters, n=1):
    lens, lam, tr = synth.pack_filters(filters)
    g = _grid_with_ages([6.9, 7.6, 8.3])
    return oracle.Oracle(grid=g, n_sfh=8, zf=10.0, zmode=1, filters=(lens, lam, tr),
                         phot_d=np.ones(len(lens)), phot_sigma=np.ones(len(lens)))


def test_flat_fnu_gives_constant_ab_magnitude_exact():
    """Filter samples on model nodes at z = 0: a flat f_nu of K*3631 Jy is K maggies."""
    gold = golden()
    lam = np.geomspace(3000.0, 60000.0, 4000)
    filt = []
    for c0, c1 in [(400, 700), (1000, 1600), (2500, 3100)]:
        tr = np.sin(np.linspace(0, np.pi, c1 - c0)) ** 2
        filt.append((lam[c0:c1].copy(), tr))
    orc = _phot_oracle(filt)
    K = 2.7e-9
    fnu = np.full(lam.size, K * float(gold["AB_fnu_cgs"]))
    np.testing.assert_allclose(orc.photometry(lam, fnu, 0.0), K, rtol=1e-13)


@pytest.mark.parametrize("z", [0.0, 0.37, 2.9, 7.2])
def test_flat_fnu_bounded_by_interpolation_error(z):
    """Generic z and filter grid: error bounded by linear interpolation of
    c/lam^2 on 512 log-spaced nodes, ~(dlnlam)^2, far below 1e-4 mag."""
    lam = np.geomspace(1000.0, 50000.0, 512)
    filt = synth.make_filters_gauss(8, 0.6, 4.5, 0.2, 200)
    orc = _phot_oracle(filt)
    K = 1.3e-8
    fnu = np.full(lam.size, K * 3.631e-20)
    out = orc.photometry(lam, fnu, z)
    # bands whose samples all lie on the redshifted model grid
    ok = np.array([f[0][0] >= lam[0] * (1 + z) and f[0][-1] <= lam[-1] * (1 + z) for f in filt])
    assert ok.sum() >= 3
    mag = -2.5 * np.log10(out[ok] / K)
    assert np.abs(mag).max() < 1e-4


def test_redshift_is_exact_shift_on_log_grid():
    """1+z = e^(n dlnlam): observing at z equals observing the index-shifted
    array at z = 0."""
    lam = np.geomspace(1000.0, 60000.0, 3000)
    dln = math.log(lam[1] / lam[0])
    n = 137
    z = math.exp(n * dln) - 1
    orc = _phot_oracle(synth.make_filters_gauss(5, 0.6, 2.5, 0.2, 150))
    rng = np.random.default_rng(5)
    fnu = rng.random(lam.size) * 1e-28
    shifted = np.zeros(lam.size)
    shifted[n:] = fnu[:-n]
    np.testing.assert_allclose(orc.photometry(lam, fnu, z), orc.photometry(lam, shifted, 0.0),
                               rtol=1e-9)


# ---------------------------------------------------------------- spectrum
def _spec_oracle(lam_grid, pix, mode, value, sigma_gal=0.0, z_ref=0.0, siglib=None):
    g = _grid_with_ages([6.9, 7.6, 8.3])
    g.lam_aa = lam_grid
    g.flux = np.ones(g.flux.shape[:3] + (lam_grid.size,))
    if siglib is not None:
        g.sigma_lib_kms = siglib
    return oracle.Oracle(grid=g, n_sfh=8, zf=10.0, zmode=1, spec_lam=pix, spec_d=np.ones(pix.size),
                         spec_sigma=np.ones(pix.size), lsf_mode=mode,
                         lsf_value=np.full(pix.size, float(value)), sigma_gal_kms=sigma_gal,
                         z_ref=z_ref)


def test_spectrum_rows_sum_to_one():
    lam = np.geomspace(3000, 9000, 3000)
    pix = np.geomspace(4000, 7000, 200)
    orc = _spec_oracle(lam, pix, 0, 800.0, sigma_gal=150.0)
    out, valid = orc.spectrum(lam, np.full(lam.size, 4.2e-29), 0.1)
    assert valid.all()
    np.testing.assert_allclose(out, 4.2e-29, rtol=1e-13)


def test_spectrum_narrow_kernel_is_linear_interpolation():
    lam = np.geomspace(3000, 9000, 300)          # coarse: 0.37% log pixels
    pix = np.geomspace(4000, 7000, 77)
    siglib = np.zeros(lam.size)
    orc = _spec_oracle(lam, pix, 4, 1e-3)        # sigma_inst = 1e-3 km/s
    g_lam = orc.grid.lam_aa
    # two-pixel floor exceeds the instrument: fixed width 0, no sigma_gal -> linear
    f = 3.0 + 2.0 * np.log(lam)
    z = 0.05
    out, valid = orc.spectrum(lam, f, z)
    x = np.log(pix) - math.log1p(z)
    np.testing.assert_allclose(out, 3.0 + 2.0 * x, rtol=1e-12)


def test_spectrum_gaussian_width_composes_in_quadrature():
    """Gaussian line of width s0 (in ln lam) on a fine log grid, LSF sigma_inst
    (km/s), library floor 2*c*sinh(dln)/2.3548 of that grid, sigma_gal: the
    pixel at the line centre sees amplitude s0/sqrt(s0^2 + s^2) with
    s^2 = (sigma_inst^2 - sigma_lib^2 + sigma_gal^2)/c^2."""
    gold = golden()
    fw = float(gold["fwhm_over_sigma"])
    lam = np.geomspace(5000, 5400, 8001)
    dln = math.log(lam[1] / lam[0])
    sig_inst, sig_gal = 60.0, 45.0
    pix = np.array([5200.0 * 1.3])
    orc = _spec_oracle(lam, pix, 4, sig_inst, sigma_gal=sig_gal, z_ref=0.3)
    s0 = 40.0 / C_KMS
    f = np.exp(-0.5 * ((np.log(lam) - math.log(5200.0)) / s0) ** 2)
    out, valid = orc.spectrum(lam, f, 0.3)
    siglib = C_KMS / 2.3548200450309493 * 2 * math.sinh(dln)
    assert abs(fw - 2.3548200450309493) < 1e-4
    s2 = (sig_inst ** 2 - siglib ** 2 + sig_gal ** 2) / C_KMS ** 2
    np.testing.assert_allclose(out[0], s0 / math.sqrt(s0 ** 2 + s2), rtol=1e-6)


@pytest.mark.parametrize("mode,val,sig", [(0, 1000.0, C_KMS / (2.3548200450309493 * 1000)),
                                          (1, 1000.0, C_KMS / 1000),
                                          (4, 120.0, 120.0), (5, 120.0, 120.0 / 2.3548200450309493)])
def test_lsf_modes(mode, val, sig):
    lam = np.geomspace(5000, 5400, 8001)
    pix = np.array([5200.0])
    orc = _spec_oracle(lam, pix, mode, val, siglib=np.zeros(lam.size))
    # siglib array of zeros does not lower the two-pixel floor; floor ~ 0.5 km/s here
    dln = math.log(lam[1] / lam[0])
    floor = C_KMS / 2.3548200450309493 * 2 * math.sinh(dln)
    s0 = 30.0 / C_KMS
    f = np.exp(-0.5 * ((np.log(lam) - math.log(5200.0)) / s0) ** 2)
    out, _ = orc.spectrum(lam, f, 0.0)
    s2 = (sig ** 2 - floor ** 2) / C_KMS ** 2
    np.testing.assert_allclose(out[0], s0 / math.sqrt(s0 ** 2 + s2), rtol=1e-6)


# ---------------------------------------------------------------- likelihood / constants
def test_likelihood_normalisation_at_d_equals_m(tiny):
    th = cases.theta_rows(TINY, 1, seed=21)
    res = tiny.eval(th)
    m = res["phot"][0]
    sig = np.abs(m) / 7.0
    tiny2 = cases.oracle_for(TINY, with_data=False)
    tiny2.set_data(phot_d=m.copy(), phot_sigma=sig)
    lnl = tiny2.eval(th)["lnl"][0]
    assert lnl == pytest.approx(-0.5 * np.sum(np.log(2 * np.pi * sig ** 2)), rel=1e-13)


def test_dlnl_dlogmass_closed_form(tiny):
    """d lnL/d logmass = ln10 * sum_b r_b m_b / sigma_b (all bands scale with 10^logmass)."""
    th = cases.theta_rows(TINY, 3, seed=22)
    g = tiny.grad_fd(th, h_rel=1e-6)
    res = tiny.eval(th)
    j = 2 * TINY.n_sfh + 1
    for r in range(3):
        m = res["phot"][r]
        rr = (tiny.phot_d - m) / tiny.phot_sigma
        want = math.log(10) * np.sum(rr * m / tiny.phot_sigma)
        assert g[r, j] == pytest.approx(want, rel=1e-6, abs=1e-6 * abs(want) + 1e-6)


def test_fd_gradient_second_order(tiny):
    th = cases.theta_rows(TINY, 2, seed=23)
    g1 = tiny.grad_fd(th, h_rel=2e-5)
    g2 = tiny.grad_fd(th, h_rel=1e-5)
    scale = np.abs(g2).max()
    assert np.nanmax(np.abs(g1 - g2)) < 1e-5 * scale


def test_paper_constants_in_observer_frame(tiny):
    """fnu = 10^logmass Lsun f (1+z) / (4 pi D_L^2): a one-hot W pins Lsun."""
    gold = golden()
    g = _grid_with_ages([6.9, 7.6, 8.3, 9.0, 9.7, 10.1])
    orc = oracle.Oracle(grid=g, n_sfh=8, zf=10.0, zmode=1, bc_edge_log_age_yr=7.0 + float(gold["bc_edge_log_age_gyr"]) + 2.0)
    th = np.zeros(orc.n_param)
    th[0] = 1.0
    th[8] = g.feh[0]
    th[8 + 2] = 9.3     # logmass
    th[8 + 3] = 1.5     # zred
    res = orc.row(th)
    dl = oracle.cosmology(orc.H0, orc.Om0, 1.5)["D_L"]
    lsun = res["fnu"] / (10 ** 9.3 * g.flux[0, 0, 0] * 2.5 / (4 * np.pi * dl ** 2))
    np.testing.assert_allclose(lsun, float(gold["L_sun_erg_s"]), rtol=1e-12)
    assert orc.bc_edge_log_age_yr == pytest.approx(7.03)


def test_status_codes(tiny):
    th = cases.theta_rows(TINY, 3, seed=24)
    jz = 2 * TINY.n_sfh + 2
    th[0, jz] = TINY.zf + 1
    th[1, jz] = -0.1
    th[2, 3] = np.nan
    st = tiny.eval(th)["status"]
    assert list(st) == [oracle.BAD_Z, oracle.BAD_Z, oracle.BAD_THETA]
    # oldest edge not older than 10 Myr: zf barely above z
    th2 = cases.theta_rows(TINY, 1, seed=25)
    th2[0, jz] = TINY.zf - 1e-4
    assert tiny.eval(th2)["status"][0] == oracle.BAD_TMAX


# ---------------------------------------------------------------- nebular
def test_nebular_zero_without_young_mass_and_node_exact():
    w = synth.shrink(synth.WORKLOADS["phot_107x12x6000_b1024"], n_age=30, n_feh=3, n_lam=800, n_sfh=12)
    g = synth.make_grid(**w.grid_kw, seed=1)
    orc = oracle.Oracle(grid=g, n_sfh=12, zf=30.0, zmode=0, use_nebular=1, dust_law=1)
    th = np.zeros(orc.n_param)
    th[12:24] = g.feh[1]
    th[24 + 2] = 1.0
    th[24 + 7] = g.neb_logz[4]
    th[24 + 8] = g.neb_logu[2]
    th[11] = 1.0                # all mass in the oldest bin: no young mass
    r0 = orc.row(th)
    assert r0["Q_young"] == 0.0
    assert not r0["Y"].any()
    th[11] = 0.0
    th[0] = 1.0                 # all mass in 0-5 Myr: young only
    r1 = orc.row(th)
    W = r1["W"]
    qy = r1["Q_young"]
    assert qy > 0
    stellar = np.einsum("nma,nmak->k", W, g.flux)
    stellar[g.lam_aa < 912.0] = 0.0
    neb = qy * 10 ** g.neb_tab[2, 4]
    np.testing.assert_allclose(r1["Y"], stellar + neb, rtol=1e-12, atol=1e-300)
    assert r1["Q_young"] == pytest.approx(np.sum(W * orc.q()), rel=1e-12)
