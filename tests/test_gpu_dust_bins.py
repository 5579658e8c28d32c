"""GPU parity of the age-binned attenuation (App. "dust_attn", Eq.
"app_tau_bin", Eq. "app_attn") against the FP64 oracle, through the C ABI:
three laws over the SSP age axis (a power law over the birth-cloud ages, the
Kriek & Conroy law over the next decade, a power law to 1 Gyr, the two later
bins overlapping with rows (1/2, 1/2), older ages in no bin) -- four attenuated
blocks in the contraction -- with the nebular emission and the KC13 diffuse
screen.  Photometry and lnL of every row in every precision; the gradient of
every column against central differences of the oracle's forward model; a
one-hot birth-cloud bin against the default two-component model; the
combinations the library refuses."""
import copy
import dataclasses

import numpy as np
import pytest

import synth
from tests import cases
from tests.test_gpu_parity import PRECS, check, run_gpu

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

W = synth.shrink(synth.WORKLOADS["phot_107x12x6000_b1024"], n_age=30, n_feh=6, n_lam=2000, n_sfh=12, batch=200)
LAWS = [0, 1, 0]
BINS_GRAD_TOL = 2e-4


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


def age_matrix(log_age):
    M = np.zeros((len(log_age), 3))
    for a, t in enumerate(log_age):
        if t <= 7.0:
            M[a, 0] = 1.0
        elif t <= 7.7:
            M[a, 1] = 1.0
        elif t <= 8.0:
            M[a, 1] = M[a, 2] = 0.5
        elif t <= 9.0:
            M[a, 2] = 1.0
    return M


_CACHE = {}


def binned(ctx):
    if "m" not in _CACHE:
        base = cases.oracle_for(W)
        M = age_matrix(base.grid.log_age_yr)
        assert len({tuple(r) for r in M if r.sum() > 0}) == 4
        orc = dataclasses.replace(base, dust_bins=(M, LAWS))
        _CACHE["m"] = (base, orc, cases.gpu_model_for(ctx, orc, W))
    return _CACHE["m"]


def rows(n, seed):
    """The workload's draws with z in [0, 5] (the Lyman limit then lies blueward
    of every band: a band straddling it has |d ln m / dz| ~ 50, where the FP32
    resolution of 1 + z alone moves it by ~3e-5 whatever the attenuation; the
    default model's tests cover that regime) and the bins' parameters."""
    th32, _ = cases.theta_pair(W, n, seed=seed)
    rng = np.random.default_rng(seed + 1)
    jz = cases.z_column(W.n_sfh, W.zmode)
    th32[:, jz] = rng.uniform(0.0, 5.0, n).astype(np.float32)
    extra = np.zeros((n, 6))
    extra[:, 0::2] = rng.uniform(0.0, 1.5, (n, 3))          # optical depths at 5500 A
    extra[:, 1] = rng.uniform(-1.3, -0.3, n)                 # power-law slopes
    extra[:, 3] = rng.uniform(-1.0, 0.3, n)                  # KC13 delta
    extra[:, 5] = rng.uniform(-1.3, -0.3, n)
    th = np.concatenate([th32, extra.astype(np.float32)], axis=1)
    return th, th.astype(np.float64)


@pytest.mark.parametrize("prec", PRECS)
def test_binned_dust_parity(ctx, prec):
    """200 rows (two tiles, ragged): every row's photometry and lnL."""
    base, orc, model = binned(ctx)
    assert model.n_param == orc.n_param == base.n_param + 6
    th32, th64 = rows(W.batch, seed=121)
    ref = orc.eval(th64)
    got = run_gpu(model, th32, prec)
    check(ref, got, prec, orc=orc)
    # the bins change the model: the default model's lnL differs
    assert np.abs(got["lnl"] - run_gpu(cases.gpu_model_for(ctx, base, W),
                                       np.ascontiguousarray(th32[:, :base.n_param]), prec)["lnl"]).max() > 1.0


def test_one_hot_birth_cloud_bin_is_the_default_model(ctx):
    base, _, _ = binned(ctx)
    young = (base.grid.log_age_yr <= base.bc_edge_log_age_yr).astype(np.float64)[:, None]
    m1 = cases.gpu_model_for(ctx, dataclasses.replace(base, dust_bins=(young, [0])), W)
    m0 = cases.gpu_model_for(ctx, base, W)
    th32, _ = cases.theta_pair(W, 150, seed=122)
    jz = cases.z_column(W.n_sfh, W.zmode)
    th_b = np.ascontiguousarray(np.concatenate([th32, th32[:, [jz + 1, jz + 2]]], axis=1))
    for prec in ("fp32", "fp32_simt"):
        a, b = run_gpu(m1, th_b, prec), run_gpu(m0, th32, prec)
        assert np.array_equal(a["status"], b["status"])
        ok = a["status"] == 0
        np.testing.assert_allclose(a["phot"][ok], b["phot"][ok], rtol=2e-6,
                                   atol=1e-7 * np.abs(b["phot"][ok]).max())
        scale = cases.lnl_scale(base, base.eval(th32.astype(np.float64)))
        assert (np.abs(a["lnl"][ok] - b["lnl"][ok]) / scale[ok]).max() < 2e-6


@pytest.mark.parametrize("prec", ["fp32", "fp32_simt"])
def test_binned_dust_gradient_vs_central_differences(ctx, prec):
    from tests.test_gpu_grad import check_grad, gpu_grad
    _, orc, model = binned(ctx)
    th32, th64 = rows(12, seed=123)
    lnl, g, st = gpu_grad(model, th32, prec)
    ok = st == 0
    assert ok.sum() >= 10
    fd = orc.grad_fd(th64, h_rel=1e-7)
    check_grad(g, fd[:, :orc.n_param], st, BINS_GRAD_TOL)
    assert np.all(np.abs(g[ok][:, -6:]).max(axis=0) > 0)     # every bin parameter moves lnL
    ref = orc.eval(th64)
    assert (np.abs(lnl[ok] - ref["lnl"][ok]) / cases.lnl_scale(orc, ref)[ok]).max() < 1e-5


def test_binned_dust_refusals(ctx):
    from paper_2609_30145_gb300 import Server, _ffi
    from paper_2609_30145_gb300.api import SedError
    base, orc, model = binned(ctx)
    M = age_matrix(base.grid.log_age_yr)

    def refused(status, **kw):
        # the library's own checks (a shallow copy: the oracle would refuse first)
        o = copy.copy(base)
        for k, v in kw.items():
            object.__setattr__(o, k, v)
        with pytest.raises(SedError) as e:
            cases.gpu_model_for(ctx, o, W)
        assert e.value.status == status, kw

    bad = M.copy()
    bad[0] = [0.6, 0.6, 0.0]
    refused(_ffi.SED_EINVAL, dust_bins=(bad, LAWS))
    refused(_ffi.SED_EINVAL, dust_bins=(M, [0, 2, 0]))
    five = np.zeros((len(M), 3))
    for a in range(len(M)):
        five[a] = [[1, 0, 0], [0, 1, 0], [0, 0, 1], [0.5, 0.5, 0], [0, 0.5, 0.5]][a % 5]
    refused(_ffi.SED_EUNSUPPORTED, dust_bins=(five, LAWS))
    refused(_ffi.SED_EUNSUPPORTED, dust_bins=(M, LAWS), fesc_geometry=1)
    th32, _ = rows(8, seed=124)
    t = torch.from_numpy(th32).cuda()
    with pytest.raises(SedError) as e:
        model.loglike_noalloc(t, "fp32")
    assert e.value.status == _ffi.SED_EUNSUPPORTED
    with pytest.raises(SedError) as e:
        Server(ctx, ctx._grid_ids[id(orc.grid)][0], model, precision="fp32")
    assert e.value.status == _ffi.SED_EUNSUPPORTED
