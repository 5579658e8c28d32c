"""GPU parity of the IGM transmission (Sec. 2.6, the Madau 1995 prescription
with its scaling igm_factor) against the FP64 oracle, through the C ABI:
photometry and lnL of the photometric fit at z in [3, 8] (the Lyman-alpha
forest and the Lyman limit cross the bluest bands) in every precision; the
emission lines through the same transmission (sed_line_fluxes, the catalogue's
lnL); igm_factor = 0 gives the model without the IGM bit for bit; the gradient
of every column, the factor and the redshift included, against central
differences of the oracle's forward model."""
import dataclasses

import numpy as np
import pytest

import synth
from tests import cases
from tests.test_gpu_parity import PRECS, check, run_gpu

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

W = synth.shrink(synth.WORKLOADS["phot_107x12x6000_b1024"], n_age=30, n_feh=6, n_lam=2000, n_sfh=12, batch=200)
IGM_GRAD_TOL = 2e-4


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


def igm_case(ctx):
    if "m" not in _CACHE:
        base = cases.oracle_for(W)
        orc = dataclasses.replace(base, use_igm=1)
        _CACHE["m"] = (base, orc, cases.gpu_model_for(ctx, orc, W))
    return _CACHE["m"]


def rows(w, n, seed, f=None):
    th32, _ = cases.theta_pair(w, n, seed=seed)
    rng = np.random.default_rng(seed + 1)
    jz = cases.z_column(w.n_sfh, w.zmode)
    th32[:, jz] = rng.uniform(3.0, 8.0, n).astype(np.float32)
    fac = rng.uniform(0.5, 2.0, n) if f is None else np.full(n, f)
    th = np.ascontiguousarray(np.concatenate([th32, fac[:, None].astype(np.float32)], axis=1))
    return th, th.astype(np.float64)


@pytest.mark.parametrize("prec", PRECS)
def test_igm_parity(ctx, prec):
    base, orc, model = igm_case(ctx)
    assert model.n_param == orc.n_param == base.n_param + 1
    th32, th64 = rows(W, W.batch, seed=141)
    ref = orc.eval(th64)
    got = run_gpu(model, th32, prec)
    check(ref, got, prec, orc=orc)
    # the transmission moves lnL (the factor-free model differs)
    m0 = cases.gpu_model_for(ctx, base, W)
    assert np.abs(got["lnl"] - run_gpu(m0, np.ascontiguousarray(th32[:, :-1]), prec)["lnl"]).max() > 1.0


def test_zero_factor_is_the_model_without_igm(ctx):
    base, orc, model = igm_case(ctx)
    m0 = cases.gpu_model_for(ctx, base, W)
    th32, _ = rows(W, 150, seed=142, f=0.0)
    for prec in ("fp32", "bf16"):
        a = run_gpu(model, th32, prec)
        b = run_gpu(m0, np.ascontiguousarray(th32[:, :-1]), prec)
        for key in ("lnl", "status", "phot"):
            assert np.array_equal(a[key], b[key]), (prec, key)


@pytest.mark.parametrize("prec", ["fp32", "fp32_simt"])
def test_igm_gradient_vs_central_differences(ctx, prec):
    from tests.test_gpu_grad import check_grad, gpu_grad
    _, orc, model = igm_case(ctx)
    th32, th64 = rows(W, 12, seed=143)
    lnl, g, st = gpu_grad(model, th32, prec)
    ok = st == 0
    assert ok.sum() >= 10
    fd = orc.grad_fd(th64, h_rel=1e-7)
    check_grad(g, fd[:, :orc.n_param], st, IGM_GRAD_TOL)
    assert np.abs(g[ok, -1]).max() > 0      # the factor moves lnL
    ref = orc.eval(th64)
    assert (np.abs(lnl[ok] - ref["lnl"][ok]) / cases.lnl_scale(orc, ref)[ok]).max() < 1e-5


def test_lines_through_the_igm(ctx):
    """Emission lines and a line catalogue with the IGM: every line's flux
    (sed_line_fluxes) and lnL of 150 rows against the oracle."""
    w = synth.shrink(synth.WORKLOADS["specphot_lines_107x12x6000_b1024"], n_age=20, n_feh=4, n_lam=2000,
                     n_sfh=10, n_pix=400, batch=150)
    orc0 = cases.lines_case(w, gas_sigma_mode=1, sigma_gas_kms=120.0)
    orc = dataclasses.replace(orc0, use_igm=1)
    model = cases.gpu_model_for(ctx, orc, w)
    th32, th64 = rows(w, w.batch, seed=144)
    ref = orc.eval(th64)
    got = run_gpu(model, th32, "fp32")
    check(ref, got, "fp32", orc=orc)
    fl = model.line_fluxes(torch.from_numpy(th32).cuda(), "fp32").cpu().numpy().astype(np.float64)
    rf = orc.line_fluxes(th64)
    ok = ref["status"] == 0
    e = np.abs(fl[ok] - rf[ok]) / np.maximum(np.abs(rf[ok]), 1e-6 * np.abs(rf[ok]).max(axis=1, keepdims=True))
    assert e.max() < 2e-5, e.max()
