"""GPU parity of the nebular age axis (App. C: the nebular cube interpolated
trilinearly and queried at each SSP age inside its tabulated ages, each age
weighted by its own ionising output) against the FP64 oracle, through the C
ABI: photometry and lnL of every row in every precision, the gradient of every
column against central differences of the oracle's forward model, planes all
equal to the age-free template against the model without an axis, and the
combinations the library refuses."""
import dataclasses

import numpy as np
import pytest

import synth
from tests import cases
from tests.test_gpu_parity import PRECS, check, run_gpu

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

BASE = synth.shrink(synth.WORKLOADS["phot_107x12x6000_b1024"], n_age=30, n_feh=6, n_lam=2000, n_sfh=12, batch=200)
W = dataclasses.replace(BASE, grid_kw=dict(BASE.grid_kw, nebular=dict(seed=2, n_logu=7, n_logz=12,
                                                                      age_axis=(5, 5.6, 7.0))))
NEB_AGE_GRAD_TOL = 2e-4


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


def axis_case(ctx):
    if "m" not in _CACHE:
        orc = cases.oracle_for(W)
        la = np.asarray(orc.grid.log_age_yr)
        inside = (la >= 5.6) & (la <= 7.0)
        assert 2 <= inside.sum() <= 32 and np.all(la[inside] <= orc.bc_edge_log_age_yr)
        _CACHE["m"] = (orc, cases.gpu_model_for(ctx, orc, W))
    return _CACHE["m"]


@pytest.mark.parametrize("prec", PRECS)
def test_nebular_age_axis_parity(ctx, prec):
    orc, model = axis_case(ctx)
    th32, th64 = cases.theta_pair(W, W.batch, seed=161)
    ref = orc.eval(th64)
    got = run_gpu(model, th32, prec)
    check(ref, got, prec, orc=orc)


def test_equal_planes_are_the_model_without_an_axis(ctx):
    orc0 = cases.oracle_for(BASE)
    g = orc0.grid
    ga = dataclasses.replace(g, neb_log_age=np.array([5.0, 6.0, 7.0]), neb_tab=np.stack([g.neb_tab] * 3))
    m_axis = cases.gpu_model_for(ctx, dataclasses.replace(orc0, grid=ga), BASE)
    m0 = cases.gpu_model_for(ctx, orc0, BASE)
    th32, _ = cases.theta_pair(BASE, 150, seed=162)
    scale = cases.lnl_scale(orc0, orc0.eval(th32.astype(np.float64)))
    for prec in ("fp32", "fp32_simt"):
        a, b = run_gpu(m_axis, th32, prec), run_gpu(m0, th32, prec)
        assert np.array_equal(a["status"], b["status"])
        ok = a["status"] == 0
        np.testing.assert_allclose(a["phot"][ok], b["phot"][ok], rtol=5e-6, atol=1e-7 * np.abs(b["phot"][ok]).max())
        assert (np.abs(a["lnl"][ok] - b["lnl"][ok]) / scale[ok]).max() < 5e-6


@pytest.mark.parametrize("prec", ["fp32", "fp32_simt"])
def test_nebular_age_axis_gradient_vs_central_differences(ctx, prec):
    from tests.test_gpu_grad import check_grad, gpu_grad
    orc, model = axis_case(ctx)
    th32, th64 = cases.theta_pair(W, 12, seed=163)
    lnl, g, st = gpu_grad(model, th32, prec)
    ok = st == 0
    assert ok.sum() >= 10
    fd = orc.grad_fd(th64, h_rel=1e-7)
    check_grad(g, fd[:, :orc.n_param], st, NEB_AGE_GRAD_TOL)
    ref = orc.eval(th64)
    assert (np.abs(lnl[ok] - ref["lnl"][ok]) / cases.lnl_scale(orc, ref)[ok]).max() < 1e-5


def test_nebular_age_axis_refusals(ctx):
    import copy
    from paper_2609_30145_gb300 import _ffi
    from paper_2609_30145_gb300.api import SedError
    orc, model = axis_case(ctx)
    g = orc.grid
    # a line cube with an age axis
    gl = dataclasses.replace(g, line_lam=np.array([4000.0, 6563.0]), line_tab=np.zeros(g.neb_tab.shape[1:3] + (2,)))
    with pytest.raises(SedError) as e:
        ctx.load_grid(gl)
    assert e.value.status == _ffi.SED_EUNSUPPORTED
    # an escape geometry, and a cube past the birth-cloud edge (the library's own checks)
    o = copy.copy(orc)
    object.__setattr__(o, "fesc_geometry", 1)
    with pytest.raises(SedError) as e:
        cases.gpu_model_for(ctx, o, W)
    assert e.value.status == _ffi.SED_EUNSUPPORTED
    gp = dataclasses.replace(g, neb_log_age=np.array([5.6, 7.6]), neb_tab=g.neb_tab[:2])
    o = copy.copy(orc)
    object.__setattr__(o, "grid", gp)
    with pytest.raises(SedError) as e:
        cases.gpu_model_for(ctx, o, W)
    assert e.value.status == _ffi.SED_EUNSUPPORTED
    th32, _ = cases.theta_pair(W, 8, seed=164)
    with pytest.raises(SedError) as e:
        model.loglike_noalloc(torch.from_numpy(th32).cuda(), "fp32")
    assert e.value.status == _ffi.SED_EUNSUPPORTED
