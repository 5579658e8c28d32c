"""Nested slice sampling on the GPU (Sec. 4.3, sed_nss_run) against quantities
fixed without the sampler:

- the evidence of a three-parameter fit (three SFH bins' masses sampled, every
  other key fixed: the likelihood is then Gaussian in the masses) against its
  closed form built from the FP64 oracle's photometry of each bin, and the
  posterior mean and width of each mass against that Gaussian truncated to the
  box prior;
- the evidence bookkeeping: ln Z recomputed here from the returned dead points'
  lnL in removal order (prior volume shrinking by exp(-1 / (n - j)) for the j-th
  of n, the final live points at X / n each), and posterior weights summing to 1;
- the constrained sampling: insertion ranks of the replacements among the
  survivors uniform (chi-square over ten bins), in 3 and in 8 dimensions;
- descriptor checks (SED_EINVAL) and a too-small output (SED_ERANGE).
"""
import dataclasses
import math

import numpy as np
import pytest

import oracle
import synth
from tests import cases

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

FIX = dict(logzsol=-0.5, afe=0.0, logmass=9.5, zred=1.5, tau_pow=0.3, alpha_pow=-1.0, diffuse_dust_index=-0.7,
           gas_logz=0.0, gas_logu=-2.0)


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


def _case(ctx, n_sfh, fixed, truth, seed=5):
    """Tiny grid, one constant [Fe/H], n_sfh bins; data = the oracle's model of
    the true row with 5% noise; the GPU model fixes the keys in `fixed`."""
    w = dataclasses.replace(synth.shrink(synth.WORKLOADS["tiny_phot_16x4x512"], n_sfh=n_sfh, batch=8), zmode=1)
    orc = cases.oracle_for(w, with_data=False)
    th = _full_rows(w, np.array([truth["sfh"]]), {**FIX, **{k: v for k, v in truth.items() if k != "sfh"}})
    res = orc.eval(th)
    assert res["status"][0] == 0
    ph = res["phot"][0]
    nz = synth.noise(ph.size, seed=seed)
    orc.set_data(phot_d=ph * (1 + nz / 20.0), phot_sigma=np.abs(ph) / 20.0)
    model = cases.gpu_model_for(ctx, orc, w, fixed=fixed)
    return w, orc, model


def _full_rows(w, sfh, vals):
    n = sfh.shape[0]
    d = {"sfh": sfh, "logzsol": np.full((n, 1), vals["logzsol"])}
    for k in ("afe", "logmass", "zred", "tau_pow", "alpha_pow", "diffuse_tau_kc", "diffuse_dust_index", "gas_logz",
              "gas_logu"):
        d[k] = np.broadcast_to(np.asarray(vals[k], dtype=np.float64), (n,)).reshape(n, 1)
    return oracle.pack_theta(d, w.n_sfh, w.zmode)


def _lnz_from_dead(lnl, n, k, n_iter):
    """ln Z from the dead points in removal order: k per iteration, then the n
    final live points."""
    lnX, terms = 0.0, []
    for it in range(n_iter):
        for j in range(k):
            step = 1.0 / (n - j)
            terms.append(lnl[it * k + j] + lnX + math.log(-math.expm1(-step)))
            lnX -= step
    for j in range(n):
        terms.append(lnl[n_iter * k + j] + lnX - math.log(n))
    t = np.array(terms)
    t = t[np.isfinite(t)]
    m = t.max()
    return m + math.log(np.exp(t - m).sum())


def _ranks_uniform(ranks, n_surv):
    """Chi-square statistic of the insertion ranks (0..n_surv) over ten equal bins."""
    f = (np.asarray(ranks) + 0.5) / (n_surv + 1)
    h = np.histogram(f, bins=10, range=(0.0, 1.0))[0]
    e = len(f) / 10.0
    return float(((h - e) ** 2 / e).sum())


def test_three_mass_evidence_and_posterior_match_the_gaussian_closed_form(ctx):
    """Three SFH bins' masses sampled, every other key fixed.  The model
    photometry is then linear in the masses (the step scheme's weights are), so
    with the oracle's photometry of each bin at unit mass, P, the likelihood is
    exactly Gaussian in the masses: lnL = lnL_max - (m - mu)^T F (m - mu) / 2 with
    F = P^T S^-1 P, S = diag(sigma^2).  Over the box prior of volume V,
    ln Z = lnL_max + (3/2) ln 2 pi - ln|F| / 2 + ln P_box - ln V, P_box the
    Gaussian's probability inside the box (scipy); the posterior is that
    Gaussian truncated to the box (moments from numpy draws)."""
    stats = pytest.importorskip("scipy.stats")
    # the young bins outshine the old one by decades: masses of 1e-3, 1e-3 and 1
    # give a correlated posterior (|rho| ~ 0.9) well inside the box
    truth = {"sfh": [1e-3, 1e-3, 1.0], "diffuse_tau_kc": 0.5}
    fixed = dict(FIX, diffuse_tau_kc=0.5)
    w, orc, model = _case(ctx, 3, fixed, truth)
    assert model.n_param == 3
    lo, hi = np.zeros(3), np.array([0.004, 0.008, 2.0])
    n, k = 400, 100
    res = model.nss(lo, hi, n_live=n, n_replace=k, n_slice_steps=20, seed=7)
    assert res["converged"]
    vals = dict(FIX, diffuse_tau_kc=0.5)
    P = orc.eval(_full_rows(w, np.eye(3), vals))["phot"].T            # [band][bin]
    m_test = np.array([[0.31, 0.07, 0.66]])
    np.testing.assert_allclose(orc.eval(_full_rows(w, m_test, vals))["phot"][0], P @ m_test[0], rtol=1e-12)
    d, sig = np.asarray(orc.phot_d), np.asarray(orc.phot_sigma)
    Fm = P.T @ (P / sig[:, None] ** 2)
    mu = np.linalg.solve(Fm, P.T @ (d / sig ** 2))
    r = (d - P @ mu) / sig
    lnl_max = -0.5 * r @ r - 0.5 * np.sum(np.log(2 * np.pi * sig ** 2))
    cov = np.linalg.inv(Fm)
    p_box = stats.multivariate_normal(mean=mu, cov=cov).cdf(hi, lower_limit=lo)
    lnz_ref = (lnl_max + 1.5 * math.log(2 * math.pi) - 0.5 * np.linalg.slogdet(Fm)[1] + math.log(p_box)
               - math.log(np.prod(hi - lo)))
    err = math.sqrt(max(res["info_h"], 0.0) / n)
    assert abs(res["lnz"] - lnz_ref) < 4.0 * err + 0.02, (res["lnz"], lnz_ref, err)
    # posterior moments against the truncated Gaussian
    x = np.random.default_rng(3).multivariate_normal(mu, cov, size=2_000_000)
    x = x[np.all((x >= lo) & (x <= hi), axis=1)]
    wts = np.exp(res["logw"])
    assert abs(wts.sum() - 1.0) < 1e-9
    for j in range(3):
        mean_g, sd_g = x[:, j].mean(), x[:, j].std()
        xs = res["theta"][:, j].astype(np.float64)
        mean_s = (wts * xs).sum()
        sd_s = math.sqrt((wts * (xs - mean_s) ** 2).sum())
        assert abs(mean_s - mean_g) < 0.2 * sd_g, (j, mean_s, mean_g, sd_g)
        assert abs(sd_s / sd_g - 1.0) < 0.15, (j, sd_s, sd_g)
    # bookkeeping and sampling quality
    assert abs(_lnz_from_dead(res["lnl"], n, k, res["n_iter"]) - res["lnz"]) < 1e-9 * max(1.0, abs(res["lnz"]))
    assert res["n_like"] > 0 and res["n_rows"] >= res["n_like"]
    assert _ranks_uniform(res["ins_rank"], n - k) < 27.9   # chi-square, 9 dof, p = 0.001


def test_eight_parameters_bookkeeping_ranks_and_determinism(ctx):
    """Six SFH bins, logmass and the diffuse depth sampled (8 columns, full
    covariance): converges, ln Z equals its recomputation from the dead points,
    the insertion ranks are uniform, the best point reaches the true row's
    likelihood, and a second run with the same seed gives the same result bit
    for bit."""
    truth = {"sfh": [0.3, 0.2, 0.2, 0.1, 0.1, 0.1], "diffuse_tau_kc": 0.5}
    fixed = {k: v for k, v in FIX.items() if k != "logmass"}
    w, orc, model = _case(ctx, 6, fixed, truth)
    assert model.n_param == 8
    lo = np.array([0.0] * 6 + [9.0, 0.1])
    hi = np.array([1.0] * 6 + [10.0, 1.0])
    n, k = 300, 64
    res = model.nss(lo, hi, n_live=n, n_replace=k, n_slice_steps=24, seed=11)
    assert res["converged"]
    assert abs(_lnz_from_dead(res["lnl"], n, k, res["n_iter"]) - res["lnz"]) < 1e-9 * max(1.0, abs(res["lnz"]))
    assert _ranks_uniform(res["ins_rank"], n - k) < 27.9
    # the run reaches the likelihood peak: its best point is at least as good
    # as the true row (oracle lnL) less one unit
    th_true = _full_rows(w, np.array([truth["sfh"]]), dict(FIX, diffuse_tau_kc=truth["diffuse_tau_kc"]))
    assert res["lnl"].max() > orc.eval(th_true)["lnl"][0] - 1.0
    again = model.nss(lo, hi, n_live=n, n_replace=k, n_slice_steps=24, seed=11)
    assert again["lnz"] == res["lnz"] and np.array_equal(again["lnl"], res["lnl"])


def test_descriptor_checks(ctx):
    from paper_2609_30145_gb300 import _ffi
    from paper_2609_30145_gb300.api import SedError
    w, orc, model = _case(ctx, 3, dict(FIX, diffuse_tau_kc=0.5), {"sfh": [0.2, 0.3, 0.5], "diffuse_tau_kc": 0.5})
    lo, hi = np.zeros(3), np.ones(3)
    for kw in (dict(n_live=1), dict(n_replace=0), dict(n_live=10, n_replace=6), dict(n_slice_steps=0),
               dict(max_iter=0)):
        with pytest.raises(SedError) as e:
            model.nss(lo, hi, **{**dict(n_live=50, n_replace=10), **kw})
        assert e.value.status == _ffi.SED_EINVAL, kw
    with pytest.raises(SedError) as e:
        model.nss(np.array([0.0, 1.0, 0.0]), np.ones(3), n_live=50, n_replace=10)   # lo == hi
    assert e.value.status == _ffi.SED_EINVAL
    with pytest.raises(SedError) as e:
        model.nss(lo, hi, n_live=50, n_replace=10, max_dead=20)
    assert e.value.status == _ffi.SED_ERANGE
