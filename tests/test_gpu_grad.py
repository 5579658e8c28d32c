"""GPU adjoint (sed_loglike_grad) against the FP64 oracle's analytic gradient
and against central finite differences of the oracle's forward model, through
the C ABI, element by element.

Tolerance: the FP32 paths evaluate the model, and its derivatives, in FP32
(3xTF32 or FFMA contractions, FP32 epilogue sums, FP64 final sums).  Every
gradient column is a sum over data of u_b dm_b/dtheta with u_b = (d_b - m_b) /
sigma_b^2, so its error is bounded by a few FP32 roundings of the largest
terms of the row rather than of the column itself; a column that cancels to
near zero keeps that absolute error.  The bar is therefore
    |g_gpu - g_ref| <= tol * max(|g_ref|, 1e-3 * max_j |g_ref_j|)
with tol per workload (GRAD_TOL) about three times the worst error measured
on a GB300 over both FP32 paths (setting SED_TEST_ERR_LOG to a file path
makes the tests log each row's error there).
"""
import json
import os

import numpy as np
import pytest

import synth
from tests import cases

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

# worst measured error (both FP32 paths) -> tolerance
GRAD_TOL = {
    "tiny": 8e-4,          # 2.4e-4
    "phot": 4e-4,          # 1.2e-4
    "specphot": 6e-4,      # 2.1e-4
    "mixed_lsf": 6e-4,     # 1.8e-4
    "sigma_gal": 1.5e-3,   # 4.4e-4
    "calib": 1e-3,         # 3.2e-4
    "floor": 4e-4,         # 1.1e-4
    "upper": 1.5e-3,       # 4.4e-4
    "escape": 6e-4,        # 1.9e-4 (picket), 2.5e-5 (runaway_bc)
    "linear_sfh": 2e-5,    # 4.9e-6
    "specphot_fd": 1e-3,   # 3.0e-4
}
PRECS = ["fp32", "fp32_simt"]


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2609_30145_gb300 import build
    build.build()
    from paper_2609_30145_gb300 import Context
    c = Context(0)
    yield c
    c.close()


_CACHE = {}


def case(ctx, key):
    if key not in _CACHE:
        name = {"tiny": "tiny_phot_16x4x512", "phot": "phot_107x12x6000_b1024",
                "spec": "specphot_afe_107x12x5x6000_b2048"}[key]
        w = synth.WORKLOADS[name]
        orc = cases.oracle_for(w)
        _CACHE[key] = (w, orc, cases.gpu_model_for(ctx, orc, w))
    return _CACHE[key]


def gpu_grad(model, th32, prec, ld=None):
    n = th32.shape[0]
    ld = ld or th32.shape[1]
    t = torch.zeros((n, ld), dtype=torch.float32, device="cuda")
    # first a call on other rows of the same size (stale values in the workspace
    # must not stand in for outputs the tested call fails to write)
    t[:, :th32.shape[1]] = torch.from_numpy(cases.poison_rows(model, th32)).cuda()
    model.loglike_grad(t, prec)
    t[:, :th32.shape[1]] = torch.from_numpy(th32).cuda()
    lnl, g, st = model.loglike_grad(t, prec)
    torch.cuda.synchronize()
    return lnl.cpu().numpy(), g.cpu().numpy(), st.cpu().numpy()


def check_grad(g_gpu, g_ref, status, tol, skip=None):
    """skip: optional {row: column} entries left out (a one-sided derivative at a kink)."""
    ok = status == 0
    assert ok.any()
    worst = 0.0
    for r in np.nonzero(ok)[0]:
        ref = g_ref[r]
        floor = 1e-3 * np.abs(ref).max()
        e = np.abs(g_gpu[r, :ref.size] - ref) / np.maximum(np.abs(ref), floor)
        if skip and r in skip:
            e[skip[r]] = 0.0
        worst = max(worst, e.max())
        if os.environ.get("SED_TEST_ERR_LOG"):   # measured worst errors, for setting the tolerances
            with open(os.environ["SED_TEST_ERR_LOG"], "a") as f:
                f.write(json.dumps({"test": os.environ.get("PYTEST_CURRENT_TEST", "?"), "row": int(r),
                                    "err": float(e.max()), "col": int(e.argmax())}) + "\n")
        assert e.max() < tol, f"row {r} column {int(e.argmax())}: {g_gpu[r, e.argmax()]} vs {ref[e.argmax()]}"
    return worst


@pytest.mark.parametrize("prec", PRECS)
def test_tiny_grad_vs_oracle(ctx, prec):
    """C1 shape at 200 rows (two 128-row tiles, ragged): every row, every column."""
    w, orc, model = case(ctx, "tiny")
    th32, th64 = cases.theta_pair(w, 200, seed=51)
    lnl, g, st = gpu_grad(model, th32, prec)
    ref = orc.grad(th64)
    assert np.array_equal(st, ref["status"])
    check_grad(g, ref["grad"], st, GRAD_TOL["tiny"])
    ok = st == 0
    fwd = orc.eval(th64)
    assert np.allclose(lnl[ok], fwd["lnl"][ok], rtol=1e-5, atol=0)


@pytest.mark.parametrize("prec", PRECS)
def test_paper_scale_phot_grad_sampled_rows(ctx, prec):
    """107 x 12 x 6000 grid, 120 bins with per-bin [Fe/H], nebular, KC13 dust,
    20 filters: the full 1024-row batch on the GPU, 12 sampled rows against the
    oracle's analytic gradient (all 249 columns)."""
    w, orc, model = case(ctx, "phot")
    th32, th64 = cases.theta_pair(w, 1024, seed=52)
    lnl, g, st = gpu_grad(model, th32, prec)
    rows = np.unique(np.concatenate([[0, 1023], np.random.default_rng(9).choice(1024, 10, replace=False)]))
    ref = orc.grad(th64[rows])
    assert np.array_equal(st[rows], ref["status"])
    check_grad(g[rows], ref["grad"], ref["status"], GRAD_TOL["phot"])


@pytest.mark.parametrize("prec", PRECS)
def test_specphot_afe_grad_sampled_rows(ctx, prec):
    """107 x 12 x 5 x 6000 grid with [a/Fe], 1500-pixel spectrum + 20 filters:
    300 rows on the GPU, 8 sampled rows against the oracle's analytic gradient."""
    w, orc, model = case(ctx, "spec")
    th32, th64 = cases.theta_pair(w, 300, seed=53)
    lnl, g, st = gpu_grad(model, th32, prec)
    rows = np.array([0, 77, 150, 299, 11, 222, 45, 180])
    ref = orc.grad(th64[rows])
    assert np.array_equal(st[rows], ref["status"])
    check_grad(g[rows], ref["grad"], ref["status"], GRAD_TOL["specphot"])


@pytest.mark.parametrize("prec", PRECS)
def test_mixed_lsf_grad_vs_oracle(ctx, prec):
    """A spectrum whose resolution alternates pixel by pixel between R = 40
    (Gaussian rows several nodes wide) and R = 30000 with no stellar dispersion
    (rows narrower than half a model log-pixel: linear interpolation), with
    every seventh pixel masked.  The pixels' node ranges are then out of order,
    which sends the adjoint's spectral gather down its tested-run path; every
    row and column against the oracle's analytic gradient."""
    w = synth.shrink(synth.WORKLOADS["specphot_afe_107x12x5x6000_b2048"], n_age=20, n_feh=4, n_lam=1500,
                     n_sfh=10, n_pix=240, batch=150)
    n_pix = w.spectrum["n_pix"]
    r = np.where(np.arange(n_pix) % 2 == 0, 40.0, 30000.0)
    mask = (np.arange(n_pix) % 7 != 3).astype(np.uint8)
    orc = cases.oracle_for(w, lsf_r=r, spec_mask=mask, sigma_gal_kms=0.0)
    model = cases.gpu_model_for(ctx, orc, w)
    th32, th64 = cases.theta_pair(w, w.batch, seed=57)
    lnl, g, st = gpu_grad(model, th32, prec)
    ref = orc.grad(th64)
    assert np.array_equal(st, ref["status"])
    check_grad(g, ref["grad"], st, GRAD_TOL["mixed_lsf"])
    ok = st == 0
    assert np.allclose(lnl[ok], orc.eval(th64)["lnl"][ok], rtol=1e-5, atol=0)


@pytest.mark.parametrize("prec", PRECS)
def test_sampled_sigma_gal_grad_vs_oracle(ctx, prec):
    """The adjoint with a sampled stellar dispersion (its column is
    d lnL / d sigma_gal through the kernel width): 150 rows, every row and
    column against the oracle's analytic gradient."""
    w = synth.shrink(synth.WORKLOADS["specphot_afe_sgal_107x12x5x6000_b2048"], n_age=20, n_feh=4,
                     n_lam=1500, n_sfh=10, n_pix=240, batch=150)
    if "sgal" not in _CACHE:
        orc = cases.oracle_for(w)
        _CACHE["sgal"] = (w, orc, cases.gpu_model_for(ctx, orc, w))
    w, orc, model = _CACHE["sgal"]
    th32, th64 = cases.theta_pair(w, w.batch, seed=58)
    lnl, g, st = gpu_grad(model, th32, prec)
    ref = orc.grad(th64)
    assert np.array_equal(st, ref["status"])
    # redshift column of rows with a spectral pixel on a model node: a kink
    kinks = {int(r): model.offsets["zred"] for r in np.nonzero(cases.kink_rows(orc, th64))[0]}
    assert len(kinks) < 20
    check_grad(g, ref["grad"], st, GRAD_TOL["sigma_gal"], skip=kinks)
    j = model.offsets["sigma_gal"]
    ok = st == 0
    assert np.abs(ref["grad"][ok, j]).max() > 0      # the column carries a real derivative


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("prec", PRECS)
def test_calibration_polynomial_grad_vs_oracle(ctx, prec, mode):
    """The adjoint with a 6-term calibration polynomial, marginalised (each
    pixel's d lnL / d mu carries the posterior-mean polynomial and the
    T^T M^-1 T term) or optimised at each call (no ln|M| term): 150 rows,
    every row and column against the oracle."""
    w = synth.shrink(synth.WORKLOADS["specphot_afe_107x12x5x6000_b2048"], n_age=20, n_feh=4,
                     n_lam=1500, n_sfh=10, n_pix=240, batch=150)
    key = f"calib{mode}"
    if key not in _CACHE:
        orc = cases.calib_case(w, [0.2, 0.1, 0.1, 0.05, 0.05, 0.05], calib_mode=mode)
        _CACHE[key] = (w, orc, cases.gpu_model_for(ctx, orc, w))
    w, orc, model = _CACHE[key]
    th32, th64 = cases.theta_pair(w, w.batch, seed=59)
    lnl, g, st = gpu_grad(model, th32, prec)
    ref = orc.grad(th64)
    assert np.array_equal(st, ref["status"])
    kinks = {int(r): model.offsets["zred"] for r in np.nonzero(cases.kink_rows(orc, th64))[0]}
    check_grad(g, ref["grad"], st, GRAD_TOL["calib"], skip=kinks)
    ok = st == 0
    fwd = orc.eval(th64)
    # lnL within 1e-5 of the magnitude of its terms (it can cancel to ~0)
    scale = cases.lnl_scale(orc, fwd)[ok]
    assert (np.abs(lnl[ok] - fwd["lnl"][ok]) / scale).max() < 1e-5


@pytest.mark.parametrize("prec", PRECS)
def test_noise_floor_grad_vs_oracle(ctx, prec):
    """The adjoint with every noise-floor term on for both arms: 150 rows, every
    column (the eight floor columns and logmass, whose derivative gains the
    model-anchored term) against the oracle's analytic gradient."""
    w = synth.shrink(synth.WORKLOADS["specphot_afe_floor_107x12x5x6000_b2048"], n_age=20, n_feh=4,
                     n_lam=1500, n_sfh=10, n_pix=240, batch=150)
    if "floor" not in _CACHE:
        orc = cases.oracle_for(w)
        _CACHE["floor"] = (w, orc, cases.gpu_model_for(ctx, orc, w))
    w, orc, model = _CACHE["floor"]
    th32, th64 = cases.theta_pair(w, w.batch, seed=62, orc=orc)
    lnl, g, st = gpu_grad(model, th32, prec)
    ref = orc.grad(th64)
    assert np.array_equal(st, ref["status"])
    kinks = {int(r): model.offsets["zred"] for r in np.nonzero(cases.kink_rows(orc, th64))[0]}
    check_grad(g, ref["grad"], st, GRAD_TOL["floor"], skip=kinks)
    ok = st == 0
    fwd = orc.eval(th64)
    scale = cases.lnl_scale(orc, fwd)[ok]
    assert (np.abs(lnl[ok] - fwd["lnl"][ok]) / scale).max() < 1e-5
    # the floor columns carry a gradient
    assert np.abs(g[ok][:, orc.n_param - 8:orc.n_param]).max() > 0


@pytest.mark.parametrize("prec", PRECS)
def test_upper_limits_grad_vs_oracle(ctx, prec):
    """The adjoint with every other band an upper limit (Eq. app_line_chi2_UL)
    and the full noise floor: 150 rows, every column against the oracle's
    analytic gradient (the one-sided term is continuous in value and slope)."""
    w = synth.shrink(synth.WORKLOADS["specphot_afe_floor_107x12x5x6000_b2048"], n_age=20, n_feh=4,
                     n_lam=1500, n_sfh=10, n_pix=240, batch=150)
    if "floor_ul" not in _CACHE:
        orc = cases.with_upper_limits(cases.oracle_for(w))
        _CACHE["floor_ul"] = (w, orc, cases.gpu_model_for(ctx, orc, w))
    w, orc, model = _CACHE["floor_ul"]
    th32, th64 = cases.theta_pair(w, w.batch, seed=65, orc=orc)
    lnl, g, st = gpu_grad(model, th32, prec)
    ref = orc.grad(th64)
    assert np.array_equal(st, ref["status"])
    kinks = {int(r): model.offsets["zred"] for r in np.nonzero(cases.kink_rows(orc, th64))[0]}
    check_grad(g, ref["grad"], st, GRAD_TOL["upper"], skip=kinks)
    ok = st == 0
    fwd = orc.eval(th64)
    exceeded, respected = cases.limit_regimes(orc, fwd["phot"][ok])
    assert exceeded > 20 and respected > 20
    scale = cases.lnl_scale(orc, fwd)[ok]
    assert (np.abs(lnl[ok] - fwd["lnl"][ok]) / scale).max() < 1e-5


@pytest.mark.parametrize("geometry", [1, 2])
def test_escape_geometry_grad_vs_central_differences(ctx, geometry):
    """The adjoint with an escape geometry (Sec. frac_obrun; runaway_bc and
    picket): every column, d lnL / d f_ob included, against central differences
    of the oracle's forward model on 16 rows of the photometric fit with
    nebular emission."""
    import dataclasses
    w = synth.shrink(synth.WORKLOADS["phot_107x12x6000_b1024"], n_age=20, n_feh=4, n_lam=1500, n_sfh=10,
                     batch=150)
    key = f"fesc{geometry}"
    if key not in _CACHE:
        orc = dataclasses.replace(cases.oracle_for(w), fesc_geometry=geometry)
        _CACHE[key] = (w, orc, cases.gpu_model_for(ctx, orc, w))
    w, orc, model = _CACHE[key]
    th32, th64 = cases.escape_pair(w, 16, seed=67, geometry=geometry)
    lnl, g, st = gpu_grad(model, th32, "fp32")
    ok = st == 0
    assert ok.sum() >= 12
    fd = orc.grad_fd(th64, h_rel=1e-7)
    check_grad(g, fd[:, :orc.n_param], st, GRAD_TOL["escape"])
    assert np.abs(g[ok, model.offsets["frac_obrun"]]).max() > 0
    ref = orc.eval(th64)
    assert (np.abs(lnl[ok] - ref["lnl"][ok]) / cases.lnl_scale(orc, ref)[ok]).max() < 1e-5


def central_differences(orc, th64, rel=1e-5):
    """d lnL / d theta by central differences of the oracle's forward model, each
    column stepped by rel x |value| (rel where the value is 0)."""
    g = np.zeros_like(th64)
    for j in range(th64.shape[1]):
        h = rel * np.maximum(np.abs(th64[:, j]), 1e-300)
        h = np.where(th64[:, j] == 0, rel, h)
        a, b = th64.copy(), th64.copy()
        a[:, j] += h
        b[:, j] -= h
        g[:, j] = (orc.eval(a)["lnl"] - orc.eval(b)["lnl"]) / (2 * h)
    return g


@pytest.mark.parametrize("zmode", [0, 1])
def test_linear_sfh_grad_vs_central_differences(ctx, zmode):
    """The adjoint of the linear SFH scheme (App. B, Eq. tent_integral): d lnL /
    d psi at every edge (each rate feeds two bins' tent shares and their
    scale to the trapezoidal mass), d/dzeta, and d/dz through the edges'
    dependence on T_max, against central differences of the oracle's forward
    model on 12 rows of the tiny workload."""
    import dataclasses
    w = dataclasses.replace(synth.WORKLOADS["tiny_phot_16x4x512"], sfh_scheme=1, zmode=zmode)
    key = f"linsfh_tiny_{zmode}"
    if key not in _CACHE:
        orc = cases.oracle_for(w)
        _CACHE[key] = (w, orc, cases.gpu_model_for(ctx, orc, w))
    w, orc, model = _CACHE[key]
    th32, th64 = cases.theta_pair(w, 12, seed=64)
    lnl, g, st = gpu_grad(model, th32, "fp32")
    ok = st == 0
    assert ok.sum() >= 8
    fd = central_differences(orc, th64[ok])
    check_grad(g[ok], fd[:, :orc.n_param], st[ok], GRAD_TOL["linear_sfh"])
    ref = orc.eval(th64)
    assert (np.abs(lnl[ok] - ref["lnl"][ok]) / cases.lnl_scale(orc, ref)[ok]).max() < 1e-5


def test_specphot_grad_vs_central_differences(ctx):
    """The adjoint against central finite differences of the FP64 oracle's
    forward model (h = 1e-7 relative) on 16 rows x all parameters."""
    w, orc, model = case(ctx, "spec")
    th32, th64 = cases.theta_pair(w, 16, seed=54)
    lnl, g, st = gpu_grad(model, th32, "fp32")
    fd = orc.grad_fd(th64, h_rel=1e-7)
    check_grad(g, fd[:, :orc.n_param], st, GRAD_TOL["specphot_fd"])


def test_grad_bad_rows_padding_and_determinism(ctx):
    w, orc, model = case(ctx, "tiny")
    th32, _ = cases.theta_pair(w, 40, seed=55)
    th32[0, model.offsets["zred"]] = w.zf + 1
    th32[1, 2] = np.nan
    ld = model.n_param + 5
    a = gpu_grad(model, th32, "fp32", ld=ld)
    b = gpu_grad(model, th32, "fp32", ld=ld)
    assert np.array_equal(a[1], b[1]) and np.array_equal(a[0], b[0])
    lnl, g, st = a
    assert st[0] != 0 and st[1] != 0 and np.isneginf(lnl[:2]).all()
    assert np.all(g[:2] == 0)
    assert np.all(g[:, model.n_param:] == 0)
    assert np.isfinite(g[2:]).all()


def test_autograd_function_backward(ctx):
    from paper_2609_30145_gb300 import SedLogLike
    w, orc, model = case(ctx, "tiny")
    th32, _ = cases.theta_pair(w, 30, seed=56)
    t = torch.from_numpy(th32).cuda().requires_grad_(True)
    lnl = SedLogLike.apply(t, model, "fp32")
    wts = torch.linspace(0.5, 1.5, 30, device="cuda", dtype=torch.float64)
    (lnl * wts).sum().backward()
    _, g, _ = gpu_grad(model, th32, "fp32")
    want = wts.cpu().numpy()[:, None] * g
    assert np.allclose(t.grad.cpu().numpy(), want, rtol=1e-6, atol=0)
