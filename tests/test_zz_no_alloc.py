"""sed_loglike_noalloc: the entry point for callers that cannot let the library
allocate device memory during a call (for example a host framework whose own
allocator already owns the GPU's memory, or a sampler step that cannot absorb
the device synchronisation of a cudaMalloc).  It runs sed_loglike's kernels
and schedule on buffers carved from one fixed scratch array, so on two calls
in a row that share that array it must give sed_loglike's results and agree
with the FP64 oracle like sed_loglike does; it must refuse batches beyond the
scratch limit, and FP8, without launching anything.

Cases: the tiny photometric fit (two 128-row tiles and a ragged tail), the
paper-scale photometric fit (107 x 12 x 6000 grid, nebular, KC13, 20 filters),
and the paper-scale [a/Fe] spectro-photometric fit (107 x 12 x 5 x 6000 grid,
1500-pixel spectrum + 20 filters) once with a marginalised 13-term calibration
polynomial and once with every noise-floor term on for both arms.

Collected last on purpose (file name), so that a run stopping at the first
failure has already run every other test.
"""
import numpy as np
import pytest

import synth
from tests import cases

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

# lnL tolerances relative to the magnitude of its terms (as in the parity tests)
LNL_TOL = {"fp32": 1e-5, "fp32_simt": 1e-5, "bf16": 1e-2}
PRECS = ["fp32", "fp32_simt", "bf16"]
SCRATCH = 32 * 1024 * 1024


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


_CASES = {}


def _case(ctx, key):
    if key not in _CASES:
        if key == "tiny":
            w = synth.WORKLOADS["tiny_phot_16x4x512"]
            orc = cases.oracle_for(w)
            rows = (200, 77)
        elif key == "phot":
            w = synth.WORKLOADS["phot_107x12x6000_b1024"]
            orc = cases.oracle_for(w)
            rows = (300, 129)          # three tiles (ragged), then two
        elif key == "calib":
            w = synth.WORKLOADS["specphot_afe_calib13_107x12x5x6000_b2048"]
            orc = cases.calib_case(w, w.extra["calib_sigma"])
            rows = (200, 65)
        else:
            w = synth.WORKLOADS["specphot_afe_floor_107x12x5x6000_b2048"]
            orc = cases.oracle_for(w)
            rows = (200, 65)
        _CASES[key] = (w, orc, cases.gpu_model_for(ctx, orc, w), rows)
    return _CASES[key]


@pytest.mark.parametrize("key", ["tiny", "phot", "calib", "floor"])
@pytest.mark.parametrize("prec", PRECS)
def test_noalloc_matches_loglike_and_oracle_on_two_calls(ctx, key, prec):
    w, orc, model, sizes = _case(ctx, key)
    for call, n in enumerate(sizes):            # two calls in a row, different batches
        th32, th64 = cases.theta_pair(w, n, seed=61 + call, orc=orc)
        th32[3, model.offsets["zred"]] = w.zf + 1   # one bad row: its status must come through too
        th64[3] = th32[3]
        t = torch.from_numpy(th32).cuda()
        ref_l, ref_s = model.loglike(t, prec)
        got_l, got_s = model.loglike_noalloc(t, prec)
        torch.cuda.synchronize()
        ref_l, ref_s = ref_l.cpu().numpy(), ref_s.cpu().numpy()
        got_l, got_s = got_l.cpu().numpy(), got_s.cpu().numpy()
        assert np.array_equal(ref_s, got_s)
        ok = ref_s == 0
        assert ok.sum() == n - 1
        assert np.isneginf(got_l[~ok]).all()
        # against sed_loglike: the same kernels and schedule
        rows = np.nonzero(ok)[0]
        sample = np.unique(np.concatenate([rows[:2], rows[-1:],
                                           np.random.default_rng(call).choice(rows, 13, replace=False)]))
        ref = orc.eval(th64[sample])
        scale = cases.lnl_scale(orc, ref)
        e_loglike = np.max(np.abs(got_l[sample] - ref_l[sample]) / scale)
        assert e_loglike < LNL_TOL[prec], f"vs sed_loglike: {e_loglike:.3e}"
        # against the FP64 oracle on sampled rows
        assert np.array_equal(ref["status"], got_s[sample])
        e_oracle = np.max(np.abs(got_l[sample] - ref["lnl"]) / scale)
        assert e_oracle < LNL_TOL[prec], f"vs the oracle: {e_oracle:.3e}"


def test_noalloc_refuses_fp8_and_batches_beyond_scratch(ctx):
    from paper_2609_30145_gb300 import SedError, _ffi
    w, orc, model, _ = _case(ctx, "phot")
    th32, _ = cases.theta_pair(w, 8, seed=3)
    t = torch.from_numpy(th32).cuda()
    with pytest.raises(SedError) as ei:
        model.loglike_noalloc(t, "fp8")
    assert ei.value.status == _ffi.SED_EUNSUPPORTED
    # rows x (2 x 4 x 6144 bytes of contraction output, Y and O) alone exceed the scratch
    n = SCRATCH // (2 * 4 * 6144) + 1
    big = torch.zeros((n, model.n_param), dtype=torch.float32, device="cuda")
    with pytest.raises(SedError) as ei:
        model.loglike_noalloc(big, "fp32")
    assert ei.value.status == _ffi.SED_ERANGE
    assert "maximum" in str(ei.value)
    # the refused calls launched nothing: a valid call still matches sed_loglike
    ref_l, _ = model.loglike(t, "fp32")
    got_l, _ = model.loglike_noalloc(t, "fp32")
    torch.cuda.synchronize()
    assert np.array_equal(np.isfinite(ref_l.cpu().numpy()), np.isfinite(got_l.cpu().numpy()))
