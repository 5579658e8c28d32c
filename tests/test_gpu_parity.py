"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on the
same seeded inputs, element by element.

Tolerances (FP32-grade paths, SED_PREC_FP32 = tcgen05 3xTF32 and
SED_PREC_FP32_SIMT = FFMA): model photometry and spectra within 2e-5
relative per datum (floored at 1e-6 of the row's brightest datum), log-
likelihood within 1e-5 relative to the magnitude of its terms.  The BF16 and
FP8 paths are held to the bounds measured for them (BF16: flux 1e-2, lnL 1e-2;
FP8 E4M3 with its 3-bit mantissa: flux 0.2 per datum floored at 1% of the row's
brightest datum -- faint pixels, two to six decades below it, reach relative
errors of 0.3 and more, while lnL stays within its bound -- and lnL 0.1) and their error
distributions are reported by the benchmark.
"""
import numpy as np
import pytest

import synth
from tests import cases

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

FLUX_TOL = {"fp32": 2e-5, "fp32_simt": 2e-5, "bf16": 1e-2, "fp8": 0.2}
# floor of the per-datum relative error, as a fraction of the row's brightest datum
FLUX_FLOOR = {"fp32": 1e-6, "fp32_simt": 1e-6, "bf16": 1e-6, "fp8": 1e-2}
LNL_TOL = {"fp32": 1e-5, "fp32_simt": 1e-5, "bf16": 1e-2, "fp8": 0.1}
PRECS = ["fp32_simt", "fp32", "bf16", "fp8"]


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


def _case(ctx, wname, shrink=None, seed_data=None):
    w = synth.WORKLOADS[wname]
    if shrink:
        w = synth.shrink(w, **shrink)
    orc = cases.oracle_for(w)
    return w, orc, cases.gpu_model_for(ctx, orc, w)


_CACHE = {}


def case(ctx, key):
    if key not in _CACHE:
        if key == "tiny":
            _CACHE[key] = _case(ctx, "tiny_phot_16x4x512")
        elif key == "phot":
            _CACHE[key] = _case(ctx, "phot_107x12x6000_b1024")
        elif key == "spec":
            _CACHE[key] = _case(ctx, "specphot_afe_107x12x5x6000_b2048")
    return _CACHE[key]


def run_gpu(model, th32, prec):
    # first a call on other rows of the same size, so that an output element the
    # tested call does not write holds another row's value, not this row's
    model.forward(torch.from_numpy(cases.poison_rows(model, th32)).cuda(), prec)
    t = torch.from_numpy(th32).cuda()
    lnl, st = model.loglike(t, prec)
    phot, spec = model.forward(t, prec)
    torch.cuda.synchronize()
    return dict(lnl=lnl.cpu().numpy(), status=st.cpu().numpy(),
                phot=None if phot is None else phot.cpu().numpy(),
                spec=None if spec is None else spec.cpu().numpy())


lnl_scale = cases.lnl_scale


def check(ref, got, prec, rows=None, orc=None, ltol=None):
    rows = np.arange(len(ref["lnl"])) if rows is None else rows
    assert np.array_equal(ref["status"], got["status"][rows])
    ok = ref["status"] == 0
    assert ok.any()
    ftol, ltol = FLUX_TOL[prec], LNL_TOL[prec] if ltol is None else ltol
    if got["phot"] is not None:
        # per-band relative error, floored at 1e-6 of the row's brightest band
        # (bands 15 magnitudes fainter than the brightest carry no information
        # at the workloads' S/N, and sit at or below FP32's normal range)
        ph_ref = ref["phot"][ok]
        floor = FLUX_FLOOR[prec] * np.abs(ph_ref).max(axis=1, keepdims=True)
        e = np.abs(got["phot"][rows][ok] - ph_ref) / np.maximum(np.abs(ph_ref), floor)
        assert e.max() < ftol, f"photometry rel err {e.max():.3e}"
    if got["spec"] is not None:
        sp_ref = ref["spec"][ok]
        scale = np.abs(sp_ref).max(axis=1, keepdims=True)
        e = np.abs(got["spec"][rows][ok] - sp_ref) / np.maximum(np.abs(sp_ref), FLUX_FLOOR[prec] * scale)
        assert e.max() < ftol, f"spectrum rel err {e.max():.3e}"
    scale = lnl_scale(orc, ref)[ok] if orc is not None else np.abs(ref["lnl"][ok])
    e = np.abs(got["lnl"][rows][ok] - ref["lnl"][ok]) / scale
    assert e.max() < ltol, f"lnL rel err {e.max():.3e}"
    assert np.all(np.isneginf(got["lnl"][rows][~ok]))


@pytest.mark.parametrize("prec", PRECS)
def test_tiny_phot_parity(ctx, prec):
    """C1 shape (16 ages x 4 [Fe/H] x 512 lam, 8 bins, 8 filters) at 200 rows:
    two 128-row tiles with a ragged tail."""
    w, orc, model = case(ctx, "tiny")
    th32, th64 = cases.theta_pair(w, 200, seed=41)
    ref = orc.eval(th64)
    got = run_gpu(model, th32, prec)
    check(ref, got, prec, orc=orc)


@pytest.mark.parametrize("prec", PRECS)
def test_paper_scale_phot_sampled_rows(ctx, prec):
    """107 x 12 x 6000 grid, 120 bins, nebular, KC13, 20 filters: the full
    1024-row batch on the GPU, 40 sampled rows against the oracle."""
    w, orc, model = case(ctx, "phot")
    th32, th64 = cases.theta_pair(w, 1024, seed=42)
    got = run_gpu(model, th32, prec)
    rows = np.unique(np.concatenate([np.arange(4), np.random.default_rng(7).choice(1024, 36, replace=False)]))
    ref = orc.eval(th64[rows])
    check(ref, got, prec, rows, orc=orc)


@pytest.mark.parametrize("prec", ["bf16", "fp8", "fp32"])
def test_mixed_precision_batch_4096(ctx, prec):
    """The mixed-precision batch of the paper-scale photometric fit: 4096 rows
    (32 M tiles, four of the persistent schedule's waves per kind) on the GPU,
    48 sampled rows -- the first, the last and rows of every 1024-row quarter
    -- against the oracle."""
    w, orc, model = case(ctx, "phot")
    th32, th64 = cases.theta_pair(w, 4096, seed=43)
    got = run_gpu(model, th32, prec)
    rows = np.unique(np.concatenate([[0, 4095], np.random.default_rng(13).choice(4096, 46, replace=False)]))
    ref = orc.eval(th64[rows])
    check(ref, got, prec, rows, orc=orc)


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_batch_past_the_persistent_schedule(ctx, prec):
    """8300 rows = 65 M tiles, one more than the persistent contraction
    schedules: the launch takes the grid schedule (one CTA per tile), and
    sampled rows -- including the last tile's ragged tail -- still match the
    oracle."""
    w, orc, model = case(ctx, "phot")
    n = 8300
    th32, th64 = cases.theta_pair(w, n, seed=44)
    got = run_gpu(model, th32, prec)
    rows = np.unique(np.concatenate([[0, 8191, 8192, n - 1], np.random.default_rng(14).choice(n, 28, replace=False)]))
    ref = orc.eval(th64[rows])
    check(ref, got, prec, rows, orc=orc)


def test_k_tile_masks_past_the_persistent_schedule(ctx):
    """The [a/Fe] spectro-photometric fit (one [Fe/H] and [a/Fe] per row, so
    the 3xTF32 contraction skips K tiles) at 8300 rows: the grid schedule with
    each M tile's K-tile mask; sampled rows against the oracle."""
    w, orc, model = case(ctx, "spec")
    n = 8300
    th32, th64 = cases.theta_pair(w, n, seed=45)
    got = run_gpu(model, th32, "fp32")
    rows = np.unique(np.concatenate([[0, 8192, n - 1], np.random.default_rng(15).choice(n, 13, replace=False)]))
    ref = orc.eval(th64[rows])
    check(ref, got, "fp32", rows, orc=orc)


@pytest.mark.parametrize("prec", PRECS)
def test_specphot_afe_sampled_rows(ctx, prec):
    """107 x 12 x 5 x 6000 grid with [a/Fe], 1500-pixel R=100-1000 spectrum +
    20 filters: 300 rows on the GPU (3 tiles, ragged), 24 sampled against the oracle."""
    w, orc, model = case(ctx, "spec")
    th32, th64 = cases.theta_pair(w, 300, seed=43)
    got = run_gpu(model, th32, prec)
    rows = np.unique(np.concatenate([[0, 1, 299], np.random.default_rng(8).choice(300, 21, replace=False)]))
    ref = orc.eval(th64[rows])
    check(ref, got, prec, rows, orc=orc)


@pytest.mark.parametrize("prec", PRECS)
def test_sampled_sigma_gal_parity(ctx, prec):
    """Spectro-photometric [a/Fe] model with a sampled stellar dispersion
    (sigma_gal in U[50, 500] km/s, a parameter column; App. E kernel of width
    sqrt(sigma_fix^2 + sigma_gal^2)): 150 rows, every row against the oracle,
    with two rows outside the declared range [0, 600] km/s."""
    w = synth.shrink(synth.WORKLOADS["specphot_afe_sgal_107x12x5x6000_b2048"], n_age=20, n_feh=4,
                     n_lam=1500, n_sfh=10, n_pix=240, batch=150)
    if "sgal" not in _CACHE:
        orc = cases.oracle_for(w)
        _CACHE["sgal"] = (w, orc, cases.gpu_model_for(ctx, orc, w))
    w, orc, model = _CACHE["sgal"]
    th32, _ = cases.theta_pair(w, w.batch, seed=46)
    j = model.offsets["sigma_gal"]
    assert j == orc.n_param - 1 == model.n_param - 1
    th32[3, j] = -5.0
    th32[7, j] = 700.0
    th64 = th32.astype(np.float64)
    ref = orc.eval(th64)
    assert ref["status"][3] != 0 and ref["status"][7] != 0
    got = run_gpu(model, th32, prec)
    check(ref, got, prec, orc=orc)


CALIB_SIGMA = [0.2, 0.1, 0.1, 0.05, 0.05, 0.05]


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("prec", PRECS)
def test_calibration_polynomial_parity(ctx, prec, mode):
    """Spectro-photometric [a/Fe] model with a 6-term Chebyshev calibration
    polynomial (App. E), marginalised or optimised at each call, and distorted
    spectral data: 150 rows, every row's lnL (which now carries the
    polynomial's gain, and for the marginal form its Occam terms) and the
    uncalibrated model spectrum against the oracle."""
    w = synth.shrink(synth.WORKLOADS["specphot_afe_107x12x5x6000_b2048"], n_age=20, n_feh=4,
                     n_lam=1500, n_sfh=10, n_pix=240, batch=150)
    key = f"calib{mode}"
    if key not in _CACHE:
        orc = cases.calib_case(w, CALIB_SIGMA, calib_mode=mode)
        _CACHE[key] = (w, orc, cases.gpu_model_for(ctx, orc, w))
    w, orc, model = _CACHE[key]
    th32, th64 = cases.theta_pair(w, w.batch, seed=47)
    ref = orc.eval(th64)
    got = run_gpu(model, th32, prec)
    check(ref, got, prec, orc=orc)


def test_edge_cases_status_and_single_row(ctx):
    w, orc, model = case(ctx, "tiny")
    th32, th64 = cases.theta_pair(w, 6, seed=44)
    jz = model.offsets["zred"]
    th32[0, jz] = w.zf + 1          # z beyond formation redshift
    th32[1, jz] = -0.5              # negative z
    th32[2, 3] = np.nan             # non-finite parameter
    th32[3, jz] = np.float32(w.zf - 1e-4)   # oldest edge younger than 10 Myr
    th64 = th32.astype(np.float64)
    ref = orc.eval(th64)
    for prec in ("fp32_simt", "fp32"):
        got = run_gpu(model, th32, prec)
        assert list(got["status"]) == list(ref["status"])
        assert np.isneginf(got["lnl"][:4]).all()
        one = run_gpu(model, th32[5:6], prec)
        sc = lnl_scale(orc, ref)[5]
        assert abs(one["lnl"][0] - ref["lnl"][5]) < 1e-5 * sc


def test_empty_batch_is_a_noop(ctx):
    w, orc, model = case(ctx, "tiny")
    t = torch.zeros((0, model.n_param), dtype=torch.float32, device="cuda")
    lnl, st = model.loglike(t, "fp32_simt")
    assert lnl.numel() == 0


def test_deterministic_bitwise(ctx):
    w, orc, model = case(ctx, "phot")
    th32, _ = cases.theta_pair(w, 257, seed=45)
    a = run_gpu(model, th32, "fp32")
    b = run_gpu(model, th32, "fp32")
    assert np.array_equal(a["lnl"], b["lnl"])
    assert np.array_equal(a["phot"], b["phot"])


def test_masked_band_excluded(ctx):
    w = synth.WORKLOADS["tiny_phot_16x4x512"]
    orc = cases.oracle_for(w)
    mask = np.ones(8, np.uint8)
    mask[[1, 5]] = 0
    orc.phot_mask = mask
    orc._rebuild_model()
    model = cases.gpu_model_for(ctx, orc, w)
    th32, th64 = cases.theta_pair(w, 50, seed=46)
    ref = orc.eval(th64)
    got = run_gpu(model, th32, "fp32_simt")
    check(ref, got, "fp32_simt", orc=orc)


def test_host_buffer_entry_point(ctx):
    w, orc, model = case(ctx, "tiny")
    th32, th64 = cases.theta_pair(w, 100, seed=47)
    ref = orc.eval(th64)
    lnl, st = model.loglike_host(th32, "fp32_simt")
    ok = ref["status"] == 0
    assert np.array_equal(st.astype(np.int64), ref["status"].astype(np.int64))
    assert (np.abs(lnl[ok] - ref["lnl"][ok]) / lnl_scale(orc, ref)[ok]).max() < 1e-5


def test_set_data_keeps_null_pairs_and_rejects_atomically(ctx):
    """sed_set_data: a pair passed as NULL keeps its last value; a call with a
    bad datum (here a spectral 1/sigma beyond FP32's range) fails with
    SED_EINVAL and changes nothing; after a good call lnL follows the oracle."""
    w = synth.shrink(synth.WORKLOADS["specphot_afe_107x12x5x6000_b2048"], n_age=20, n_feh=4,
                     n_lam=1500, n_sfh=10, n_pix=240, batch=40)
    orc = cases.oracle_for(w)
    model = cases.gpu_model_for(ctx, orc, w)
    th32, th64 = cases.theta_pair(w, w.batch, seed=48)
    t = torch.from_numpy(th32).cuda()
    ref = orc.eval(th64)
    ok = ref["status"] == 0
    base = model.loglike(t, "fp32")[0].cpu().numpy()
    assert (np.abs(base[ok] - ref["lnl"][ok]) / lnl_scale(orc, ref)[ok]).max() < 1e-5
    # spectrum only: the photometric pair is kept
    model.set_data(spec_d=orc.spec_d, spec_sigma=orc.spec_sigma)
    assert np.array_equal(model.loglike(t, "fp32")[0].cpu().numpy(), base)
    # a spectral sigma of 1e-40 (1/sigma overflows FP32): rejected, nothing changes
    bad = np.array(orc.spec_sigma, dtype=np.float64)
    bad[7] = 1e-40
    with pytest.raises(Exception):
        model.set_data(phot_d=orc.phot_d * 2, phot_sigma=orc.phot_sigma, spec_d=orc.spec_d, spec_sigma=bad)
    assert np.array_equal(model.loglike(t, "fp32")[0].cpu().numpy(), base)
    # new photometry alone: lnL follows the oracle with that photometry
    pd2 = np.asarray(orc.phot_d) * 1.1
    model.set_data(phot_d=pd2, phot_sigma=orc.phot_sigma)
    orc.set_data(phot_d=pd2, phot_sigma=orc.phot_sigma, spec_d=orc.spec_d, spec_sigma=orc.spec_sigma)
    ref2 = orc.eval(th64)
    got = model.loglike(t, "fp32")[0].cpu().numpy()
    assert (np.abs(got[ok] - ref2["lnl"][ok]) / lnl_scale(orc, ref2)[ok]).max() < 1e-5


def test_spectrum_never_set_stays_out_of_lnl(ctx):
    """A model created with a spectrum's wavelengths but without its data: lnL
    is the photometric part alone (the oracle with every pixel masked)."""
    w = synth.shrink(synth.WORKLOADS["specphot_afe_107x12x5x6000_b2048"], n_age=20, n_feh=4,
                     n_lam=1500, n_sfh=10, n_pix=240, batch=40)
    orc = cases.oracle_for(w, spec_mask=np.zeros(240, np.uint8))
    full = cases.oracle_for(w)
    model = cases.gpu_model_for(ctx, full, w, with_spec_data=False)
    th32, th64 = cases.theta_pair(w, w.batch, seed=49)
    ref = orc.eval(th64)
    ok = ref["status"] == 0
    got = model.loglike(torch.from_numpy(th32).cuda(), "fp32")[0].cpu().numpy()
    assert (np.abs(got[ok] - ref["lnl"][ok]) / lnl_scale(orc, ref)[ok]).max() < 1e-5


def test_host_entry_point_pinned_in_place_and_pageable_staged(ctx):
    """sed_loglike_host: page-locked buffers are read and written in place by
    the kernels, pageable ones staged through device memory; both give the
    same result, bit for bit, equal to the device entry point's, and both
    match the oracle."""
    w, orc, model = case(ctx, "spec")
    th32, th64 = cases.theta_pair(w, 300, seed=50)
    ref = orc.eval(th64[:24])
    lnl_p, st_p = model.loglike_host(th32, "fp32")
    assert ctx.last_host_path() == 0
    th_pin = torch.from_numpy(th32).pin_memory()
    out = torch.empty(300, dtype=torch.float64).pin_memory()
    sto = torch.empty(300, dtype=torch.int32).pin_memory()
    model.loglike_host(th_pin, "fp32", out=out, status=sto)
    assert ctx.last_host_path() == 3
    assert np.array_equal(out.numpy(), lnl_p)
    assert np.array_equal(sto.numpy().astype(np.uint32), st_p)
    lnl_d, st_d = model.loglike(torch.from_numpy(th32).cuda(), "fp32")
    assert np.array_equal(lnl_d.cpu().numpy(), lnl_p)
    ok = ref["status"] == 0
    assert np.array_equal(st_p[:24].astype(np.int64), ref["status"].astype(np.int64))
    assert (np.abs(lnl_p[:24][ok] - ref["lnl"][ok]) / lnl_scale(orc, ref)[ok]).max() < 1e-5


def test_host_entry_point_graph_replay_follows_live_data(ctx):
    """sed_loglike_host on page-locked buffers and a caller's stream: the first
    call runs the launches directly, the second captures them into a CUDA
    graph, later ones replay it.  Every call equals the device entry point bit
    for bit, including after the theta buffer's contents and the model's data
    change between replays, and a new row count falls back to direct launches."""
    w, orc, model = case(ctx, "tiny")
    th32, _ = cases.theta_pair(w, 200, seed=52)
    th_pin = torch.from_numpy(th32).pin_memory()
    out = torch.empty(200, dtype=torch.float64).pin_memory()
    sto = torch.empty(200, dtype=torch.int32).pin_memory()
    stream = torch.cuda.Stream()

    def device_ref(th):
        lnl, st = model.loglike(torch.from_numpy(th).cuda(), "fp32")
        torch.cuda.synchronize()
        return lnl.cpu().numpy(), st.cpu().numpy()

    paths = []
    for _ in range(3):
        model.loglike_host(th_pin, "fp32", stream=stream, out=out, status=sto)
        paths.append(ctx.last_host_path())
        ref, st_ref = device_ref(th32)
        assert np.array_equal(out.numpy(), ref)
        assert np.array_equal(sto.numpy(), st_ref)
    assert paths == [3, 7, 7]
    # new contents in the same page-locked buffer: the replay reads them
    th2, _ = cases.theta_pair(w, 200, seed=53)
    th_pin.copy_(torch.from_numpy(th2))
    model.loglike_host(th_pin, "fp32", stream=stream, out=out, status=sto)
    assert ctx.last_host_path() == 7
    assert np.array_equal(out.numpy(), device_ref(th2)[0])
    # new data for the model: updated in place, so the replay sees it too
    model.set_data(phot_d=np.asarray(orc.phot_d) * 1.2, phot_sigma=orc.phot_sigma)
    try:
        model.loglike_host(th_pin, "fp32", stream=stream, out=out, status=sto)
        assert ctx.last_host_path() == 7
        assert np.array_equal(out.numpy(), device_ref(th2)[0])
    finally:
        model.set_data(phot_d=orc.phot_d, phot_sigma=orc.phot_sigma)
    # another row count: a new call, launched directly
    model.loglike_host(th_pin[:150], "fp32", stream=stream, out=out[:150], status=sto[:150])
    assert ctx.last_host_path() == 3
    assert np.array_equal(out.numpy()[:150], device_ref(th2[:150])[0])


@pytest.mark.parametrize("prec", PRECS)
def test_noise_floor_parity(ctx, prec):
    """Spectro-photometric [a/Fe] model with every term of the systematic noise
    floor on for both arms (App. sys_floor, Eq. app_noise_floor: error scale,
    model- and data-anchored fractions, jitter; eight log10 columns): 150 rows,
    every row's lnL and model against the oracle."""
    w = synth.shrink(synth.WORKLOADS["specphot_afe_floor_107x12x5x6000_b2048"], n_age=20, n_feh=4,
                     n_lam=1500, n_sfh=10, n_pix=240, batch=150)
    if "floor" not in _CACHE:
        orc = cases.oracle_for(w)
        _CACHE["floor"] = (w, orc, cases.gpu_model_for(ctx, orc, w))
    w, orc, model = _CACHE["floor"]
    assert model.n_param == orc.n_param
    th32, th64 = cases.theta_pair(w, w.batch, seed=61, orc=orc)
    ref = orc.eval(th64)
    got = run_gpu(model, th32, prec)
    check(ref, got, prec, orc=orc)


@pytest.mark.parametrize("prec", PRECS)
def test_linear_sfh_parity(ctx, prec):
    """The paper-scale photometric fit with the linear SFH scheme (App. B, Eq.
    tent_integral: per-edge SFRs, N_T + 1 columns, tent integrals per age
    node): 300 rows on the GPU, 30 sampled rows' photometry and lnL against the
    oracle."""
    w = synth.WORKLOADS["phot_linsfh_107x12x6000_b1024"]
    if "linsfh" not in _CACHE:
        orc = cases.oracle_for(w)
        _CACHE["linsfh"] = (w, orc, cases.gpu_model_for(ctx, orc, w))
    w, orc, model = _CACHE["linsfh"]
    assert model.n_param == orc.n_param == 2 * w.n_sfh + 1 + 9
    th32, th64 = cases.theta_pair(w, 300, seed=63)
    got = run_gpu(model, th32, prec)
    rows = np.unique(np.concatenate([[0, 299], np.random.default_rng(10).choice(300, 28, replace=False)]))
    ref = orc.eval(th64[rows])
    check(ref, got, prec, rows, orc=orc)


@pytest.mark.parametrize("prec", PRECS)
def test_upper_limits_parity(ctx, prec):
    """Every other band an upper limit (Sec. 4.1 likelihood, Eq.
    app_line_chi2_UL) in the spectro-photometric fit with the full noise floor
    on both arms: 150 rows' lnL and models against the oracle, the rows
    exceeding some limits and respecting others."""
    w = synth.shrink(synth.WORKLOADS["specphot_afe_floor_107x12x5x6000_b2048"], n_age=20, n_feh=4,
                     n_lam=1500, n_sfh=10, n_pix=240, batch=150)
    if "floor_ul" not in _CACHE:
        orc = cases.with_upper_limits(cases.oracle_for(w))
        _CACHE["floor_ul"] = (w, orc, cases.gpu_model_for(ctx, orc, w))
    w, orc, model = _CACHE["floor_ul"]
    th32, th64 = cases.theta_pair(w, w.batch, seed=64, orc=orc)
    ref = orc.eval(th64)
    exceeded, respected = cases.limit_regimes(orc, ref["phot"][ref["status"] == 0])
    assert exceeded > 20 and respected > 20
    got = run_gpu(model, th32, prec)
    check(ref, got, prec, orc=orc)


def escape_case(ctx, geometry):
    """The paper-scale photometric fit (nebular emission, KC13 dust) on a
    smaller grid, with an escape geometry (Sec. frac_obrun)."""
    import dataclasses
    w = synth.shrink(synth.WORKLOADS["phot_107x12x6000_b1024"], n_age=20, n_feh=4, n_lam=1500, n_sfh=10,
                     batch=150)
    key = f"fesc{geometry}"
    if key not in _CACHE:
        orc = dataclasses.replace(cases.oracle_for(w), fesc_geometry=geometry)
        _CACHE[key] = (w, orc, cases.gpu_model_for(ctx, orc, w))
    return _CACHE[key]


@pytest.mark.parametrize("geometry", [1, 2])
@pytest.mark.parametrize("prec", PRECS)
def test_escape_geometry_parity(ctx, prec, geometry):
    """runaway_bc (Eq. runaway_mix) and picket escape of the young light with
    f_ob ~ U[0.05, 0.95] (Sec. frac_obrun): 150 rows' photometry and lnL
    against the oracle, two rows with f_ob outside [0, 1] refused."""
    w, orc, model = escape_case(ctx, geometry)
    assert model.n_param == orc.n_param and model.offsets["frac_obrun"] == orc.n_param - 1
    th32, _ = cases.escape_pair(w, w.batch, seed=66, geometry=geometry)
    th32[5, -1] = -0.1
    th32[9, -1] = 1.2
    th64 = th32.astype(np.float64)
    ref = orc.eval(th64)
    assert ref["status"][5] != 0 and ref["status"][9] != 0
    got = run_gpu(model, th32, prec)
    # FP8 under picket: the young light reaches the bands unscreened, ionising
    # continuum included, so the E4M3 rounding of the young columns weighs more
    # (lnL error 0.100 of the term scale measured at this workload)
    check(ref, got, prec, orc=orc, ltol=0.15 if (prec == "fp8" and geometry == 2) else None)


def test_model_descriptor_validation(ctx):
    """sed_create_model refuses what it cannot evaluate, before anything runs:
    an unknown SFH scheme, noise-floor bits or escape geometry (SED_EINVAL), a
    floor on an arm without data (SED_EINVAL), and a spectral floor together
    with the calibration polynomial (SED_EUNSUPPORTED)."""
    from paper_2609_30145_gb300.api import SedError
    w = synth.shrink(synth.WORKLOADS["specphot_afe_107x12x5x6000_b2048"], n_age=20, n_feh=4,
                     n_lam=1500, n_sfh=10, n_pix=240, batch=8)
    orc = cases.oracle_for(w)
    gid = ctx.load_grid(orc.grid)
    base = dict(use_afe=w.use_afe, dust_law=w.dust_law, filters=orc.filters, phot_d=orc.phot_d,
                phot_sigma=orc.phot_sigma)
    spec = dict(spec_lam=orc.spec_lam, spec_d=orc.spec_d, spec_sigma=orc.spec_sigma, lsf_mode=orc.lsf_mode,
                lsf_value=orc.lsf_value, sigma_gal_kms=orc.sigma_gal_kms, z_ref=orc.z_ref)

    def refused(code, **kw):
        with pytest.raises(SedError) as e:
            ctx.create_model(gid, w.n_sfh, w.zf, w.zmode, **kw)
        assert e.value.status == code, str(e.value)

    refused(1, **base, sfh_scheme=2)
    refused(1, **base, noise_floor_phot=16)
    refused(1, **base, noise_floor_spec=1)                      # no spectrum
    refused(8, **base, **spec, calib_sigma=[0.1, 0.1], noise_floor_spec=2)
    refused(1, **base, fesc_geometry=3)
    refused(1, **base, fesc_geometry=-1)
    ok = ctx.create_model(gid, w.n_sfh, w.zf, w.zmode, **base, **spec, noise_floor_phot=9, sfh_scheme=1)
    assert ok.n_param == orc.n_param + 1 + 2
    esc = ctx.create_model(gid, w.n_sfh, w.zf, w.zmode, **base, fesc_geometry=2)
    assert esc.n_param == orc.n_param + 1 and esc.offsets["frac_obrun"] == orc.n_param


def test_fixed_keys_match_the_sampled_model(ctx):
    """Keys fixed in the model descriptor (the paper's fixed vs sampled keys,
    Sec. 4) leave the parameter rows and the gradient, and give the same
    lnL, model and remaining gradient columns as the sampled model whose rows
    carry the same values, bit for bit; the redshift fixed too (the calls then
    keep the caller's row order).  lnL against the oracle on the full rows."""
    w = synth.shrink(synth.WORKLOADS["specphot_afe_107x12x5x6000_b2048"], n_age=20, n_feh=4,
                     n_lam=1500, n_sfh=10, n_pix=240, batch=150)
    orc = cases.oracle_for(w)
    full = cases.gpu_model_for(ctx, orc, w)
    fixed = {"logzsol": np.float32(-0.3), "afe": np.float32(0.15), "zred": np.float32(1.75),
             "diffuse_dust_index": np.float32(-0.4), "alpha_pow": np.float32(-1.0)}
    fix = cases.gpu_model_for(ctx, orc, w, fixed={k: float(v) for k, v in fixed.items()})
    assert fix.n_param == full.n_param - len(fixed)
    for k in fixed:   # zero width in the fixed model's layout
        i = list(fix.offsets).index(k)
        nxt = list(fix.offsets.values())[i + 1] if i + 1 < len(fix.offsets) else fix.n_param
        assert fix.offsets[k] == nxt
    th32, th64 = cases.theta_pair(w, w.batch, seed=71)
    for k, v in fixed.items():
        th32[:, full.offsets[k]] = v
    th64 = th32.astype(np.float64)
    keep = np.ones(full.n_param, bool)
    keep[[full.offsets[k] for k in fixed]] = False
    t_full = torch.from_numpy(th32).cuda()
    t_fix = torch.from_numpy(np.ascontiguousarray(th32[:, keep])).cuda()
    for prec in ("fp32", "bf16"):
        a = run_gpu(full, th32, prec)
        b = run_gpu(fix, np.ascontiguousarray(th32[:, keep]), prec)
        for key in ("lnl", "status", "phot", "spec"):
            assert np.array_equal(a[key], b[key]), (prec, key)
    la, ga, sa = full.loglike_grad(t_full, "fp32")
    lb, gb, sb = fix.loglike_grad(t_fix, "fp32")
    torch.cuda.synchronize()
    assert np.array_equal(la.cpu().numpy(), lb.cpu().numpy())
    assert np.array_equal(ga.cpu().numpy()[:, keep], gb.cpu().numpy())
    ref = orc.eval(th64)
    check(ref, run_gpu(fix, np.ascontiguousarray(th32[:, keep]), "fp32"), "fp32", orc=orc)
    # what cannot be fixed
    from paper_2609_30145_gb300.api import SedError
    for bad in ({"sfh": 0.1}, {"sigma_gal": 100.0}, {"log_jitter_phot": -3.0}, {"logmass": float("nan")}):
        with pytest.raises(SedError) as e:
            cases.gpu_model_for(ctx, orc, w, fixed=bad)
        assert e.value.status == 1, bad
    w0 = synth.shrink(synth.WORKLOADS["tiny_phot_16x4x512"], batch=8)   # per-bin [Fe/H]: logzsol has N_T columns
    orc0 = cases.oracle_for(w0)
    with pytest.raises(SedError):
        cases.gpu_model_for(ctx, orc0, w0, fixed={"logzsol": 0.0})


def test_grid_precision_mask_keeps_only_the_named_copies(ctx):
    """A grid loaded with precision_mask keeps only those operand copies: a
    BF16-only grid takes less device memory, refuses the other precisions
    (SED_EUNSUPPORTED) and gives the default grid's BF16 results bit for bit; an
    FP8 copy asked for at load gives the FP8 results of the copy that the
    default grid builds on first use."""
    from paper_2609_30145_gb300 import _ffi
    from paper_2609_30145_gb300.api import SedError
    w = synth.shrink(synth.WORKLOADS["phot_107x12x6000_b1024"], n_age=30, n_feh=6, n_lam=2000, n_sfh=20,
                     batch=200)
    orc = cases.oracle_for(w)
    ref_model = cases.gpu_model_for(ctx, orc, w)
    th32, _ = cases.theta_pair(w, w.batch, seed=73)
    want = {p: run_gpu(ref_model, th32, p) for p in ("bf16", "fp8")}
    kw = dict(use_nebular=w.use_nebular, dust_law=w.dust_law, filters=orc.filters, phot_d=orc.phot_d,
              phot_sigma=orc.phot_sigma, phot_mask=orc.phot_mask, H0=orc.H0, Om0=orc.Om0)
    before = ctx.memory_used()
    ctx.create_model(ctx.load_grid(orc.grid), w.n_sfh, w.zf, w.zmode, **kw)
    grown_default = ctx.memory_used() - before
    for mask, precs in ((_ffi.GRID_COPY_BF16, ("bf16",)), (_ffi.GRID_COPY_FP8, ("fp8",))):
        before = ctx.memory_used()
        gid = ctx.load_grid(orc.grid, precision_mask=mask)
        m = ctx.create_model(gid, w.n_sfh, w.zf, w.zmode, **kw)
        grown = ctx.memory_used() - before
        for p in ("fp32", "fp32_simt", "bf16", "fp8"):
            if p in precs:
                got = run_gpu(m, th32, p)
                for key in ("lnl", "status", "phot"):
                    assert np.array_equal(got[key], want[p][key]), (mask, p, key)
            else:
                with pytest.raises(SedError) as e:
                    m.loglike(torch.from_numpy(th32).cuda(), p)
                assert e.value.status == _ffi.SED_EUNSUPPORTED, (mask, p)
        # one copy of 2 (BF16) or 1 (FP8) bytes per element instead of 8 + 4 + 2
        assert grown < 0.3 * grown_default, (mask, grown, grown_default)


@pytest.mark.parametrize("prec", ["fp32", "bf16", "fp8"])
def test_k_tile_skipping_leaves_every_row_unchanged(ctx, prec):
    """With one [Fe/H] and [a/Fe] per row the rows are grouped by their bracket
    pair and the contraction skips the K tiles that no row of a 128-row tile
    touches.  Skipped tiles hold exact zeros and the accumulation groups keep
    their places, so a row's result must not depend on which rows share its
    tile: the same rows in another order give the same lnL, model and gradient
    bit for bit (the paper-scale [a/Fe] spectro-photometric fit, 1100 rows)."""
    w, orc, model = case(ctx, "spec")
    th32, _ = cases.theta_pair(w, 1100, seed=75)
    perm = np.random.default_rng(5).permutation(th32.shape[0])
    a = run_gpu(model, th32, prec)
    b = run_gpu(model, np.ascontiguousarray(th32[perm]), prec)
    for key in ("lnl", "status", "phot", "spec"):
        assert np.array_equal(a[key][perm], b[key]), key
    if prec == "fp32":
        la, ga, _ = model.loglike_grad(torch.from_numpy(th32).cuda(), prec)
        lb, gb, _ = model.loglike_grad(torch.from_numpy(np.ascontiguousarray(th32[perm])).cuda(), prec)
        torch.cuda.synchronize()
        assert np.array_equal(la.cpu().numpy()[perm], lb.cpu().numpy())
        assert np.array_equal(ga.cpu().numpy()[perm], gb.cpu().numpy())
