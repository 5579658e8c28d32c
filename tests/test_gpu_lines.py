"""GPU parity of the emission lines (App. C line cube, App. line_proj, Eq.
app_line_profile) and the line-catalogue arm (Sec. 3.3, Eq.
app_line_chi2_det / app_line_chi2_UL) against the FP64 oracle, through the C
ABI, element by element: photometry, spectrum (lines on the pixels) and lnL
(with blends, upper limits and a masked entry), in every precision, for a
sampled, a fixed and a tied gas dispersion, on a small grid at 150 rows and
on the paper-scale JADES-like fit at 1024 rows (sampled rows)."""
import numpy as np
import pytest

import synth
from tests import cases
from tests.test_gpu_parity import FLUX_TOL, FLUX_FLOOR, LNL_TOL, PRECS, run_gpu, check

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

W_SMALL = synth.shrink(synth.WORKLOADS["specphot_lines_107x12x6000_b1024"], n_age=20, n_feh=4, n_lam=2000,
                       n_sfh=10, n_pix=400, batch=150)


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


def lines_model(ctx, w, mode):
    key = (w.name, mode)
    if key not in _CACHE:
        orc = cases.lines_case(w, gas_sigma_mode=mode, sigma_gas_kms=120.0)
        _CACHE[key] = (orc, cases.gpu_model_for(ctx, orc, w))
    return _CACHE[key]


@pytest.mark.parametrize("mode", [2, 1, 0])
@pytest.mark.parametrize("prec", PRECS)
def test_lines_parity_small(ctx, prec, mode):
    """150 rows (two tiles, ragged): every row's photometry, spectrum and lnL."""
    orc, model = lines_model(ctx, W_SMALL, mode)
    assert model.n_param == orc.n_param
    th32, th64 = cases.lines_theta_pair(W_SMALL, orc, W_SMALL.batch, seed=91)
    ref = orc.eval(th64)
    got = run_gpu(model, th32, prec)
    check(ref, got, prec, orc=orc)


@pytest.mark.parametrize("prec", PRECS)
def test_lines_parity_paper_scale(ctx, prec):
    """107 x 12 x 6000 grid with a 30-line cube, 1500-pixel spectrum, 20
    filters, 12-entry line catalogue, sigma_gas sampled: 1024 rows on the GPU,
    24 sampled rows against the oracle."""
    w = synth.WORKLOADS["specphot_lines_107x12x6000_b1024"]
    orc, model = lines_model(ctx, w, 2)
    th32, th64 = cases.lines_theta_pair(w, orc, 1024, seed=92)
    got = run_gpu(model, th32, prec)
    rows = np.unique(np.concatenate([[0, 1023], np.random.default_rng(12).choice(1024, 22, replace=False)]))
    ref = orc.eval(th64[rows])
    check(ref, got, prec, rows, orc=orc)


@pytest.mark.parametrize("prec", PRECS)
def test_line_fluxes_match_the_oracle(ctx, prec):
    """sed_line_fluxes: every grid line's observer-frame flux of 150 rows
    (sampled sigma_gas) against the oracle's, 2e-5 relative per line (the fluxes
    do not pass through the contraction, so every precision gives FP32-grade
    values); rows with a bad status give zeros."""
    orc, model = lines_model(ctx, W_SMALL, 2)
    th32, th64 = cases.lines_theta_pair(W_SMALL, orc, W_SMALL.batch, seed=95)
    th32[3, model.offsets["sigma_gas"]] = -5.0          # refused row
    th64 = th32.astype(np.float64)
    got = model.line_fluxes(torch.from_numpy(th32).cuda(), prec).cpu().numpy().astype(np.float64)
    ref = orc.line_fluxes(th64)
    st = orc.eval(th64)["status"]
    ok = st == 0
    assert not ok[3] and np.all(got[3] == 0.0)
    e = np.abs(got[ok] - ref[ok]) / np.maximum(np.abs(ref[ok]), 1e-6 * np.abs(ref[ok]).max(axis=1, keepdims=True))
    assert e.max() < 2e-5, e.max()
    base = cases.gpu_model_for(ctx, cases.oracle_for(W_SMALL), W_SMALL)
    from paper_2609_30145_gb300 import _ffi
    from paper_2609_30145_gb300.api import SedError
    with pytest.raises(SedError) as e:
        base.line_fluxes(torch.from_numpy(np.ascontiguousarray(th32[:, :base.n_param])).cuda(), prec)
    assert e.value.status == _ffi.SED_EUNSUPPORTED


def test_lines_change_the_model_where_the_paper_puts_them(ctx):
    """The line part of the GPU model (lines on minus lines off) sits on the
    pixels within 5 s_l of each line's observed wavelength and is positive
    there; a sampled sigma_gas outside [0, max] marks the row invalid."""
    orc, model = lines_model(ctx, W_SMALL, 2)
    orc0 = cases.oracle_for(W_SMALL)
    base = cases.gpu_model_for(ctx, orc0, W_SMALL)
    th32, th64 = cases.lines_theta_pair(W_SMALL, orc, 8, seed=93)
    a = run_gpu(model, th32, "fp32")
    b = run_gpu(base, np.ascontiguousarray(th32[:, :base.n_param]), "fp32")
    dsp = a["spec"] - b["spec"]
    lam = np.asarray(orc.spec_lam)
    jz = model.offsets["zred"]
    for r in range(th32.shape[0]):
        lo = orc.grid.line_lam * (1 + th32[r, jz])
        near = np.zeros(lam.size, bool)
        for x in lo:
            near |= np.abs(np.log(lam / x)) < 0.05
        assert np.all(np.abs(dsp[r, ~near]) <= 1e-6 * np.abs(b["spec"][r]).max())
        assert dsp[r, near].max() > 0
    th_bad = th32.copy()
    th_bad[0, model.offsets["sigma_gas"]] = 700.0   # above the declared 600 km/s
    th_bad[1, model.offsets["sigma_gas"]] = -1.0
    got = run_gpu(model, th_bad, "fp32")
    assert got["status"][0] == 1 and got["status"][1] == 1 and np.all(got["status"][2:] == 0)


@pytest.mark.parametrize("mode", [2, 0])
def test_lines_gradient_vs_central_differences(ctx, mode):
    """The adjoint with emission lines and the line catalogue (sigma_gas
    sampled, or tied to a fixed sigma_gal): every column of 12 rows against
    central differences of the oracle's forward model, and lnL against the
    oracle."""
    from tests.test_gpu_grad import check_grad, gpu_grad
    orc, model = lines_model(ctx, W_SMALL, mode)
    th32, th64 = cases.lines_theta_pair(W_SMALL, orc, 12, seed=94)
    lnl, g, st = gpu_grad(model, th32, "fp32")
    ok = st == 0
    assert ok.sum() >= 10
    fd = orc.grad_fd(th64, h_rel=1e-7)
    check_grad(g, fd[:, :orc.n_param], st, LINES_GRAD_TOL)
    if mode == 2:
        assert np.abs(g[ok, model.offsets["sigma_gas"]]).max() > 0
    ref = orc.eval(th64)
    assert (np.abs(lnl[ok] - ref["lnl"][ok]) / cases.lnl_scale(orc, ref)[ok]).max() < 1e-5


LINES_GRAD_TOL = 2e-4   # about three times the worst error measured on a GB300 (5.7e-5)
