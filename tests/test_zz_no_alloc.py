"""sed_loglike_noalloc: the entry point for callers that cannot let the library
allocate device memory during a call (for example a host framework whose own
allocator already owns the GPU's memory).  It must give the same result as
sed_loglike, whose workspace comes from cudaMalloc, on two calls in a row
that share its fixed scratch array, and refuse batches beyond the scratch
limit without launching anything.

Collected last on purpose (file name), so that a run stopping at the first
failure has already run every other test.
"""
import ctypes as C

import numpy as np
import pytest

import synth
from tests import cases

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def setup():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2609_30145_gb300 import build
    build.build()
    from paper_2609_30145_gb300 import Context, _ffi
    ctx = Context(0)
    w = synth.WORKLOADS["tiny_phot_16x4x512"]
    orc = cases.oracle_for(w)
    model = cases.gpu_model_for(ctx, orc, w)
    yield ctx, model, orc, w, _ffi
    ctx.close()


def _noalloc(ctx, model, t, prec, _ffi):
    n, ld = t.shape[0], t.stride(0)
    lnl = torch.empty(n, dtype=torch.float64, device=t.device)
    st = torch.empty(n, dtype=torch.int32, device=t.device)
    rc = ctx._lib.sed_loglike_noalloc(ctx._h, model.id, C.c_void_p(t.data_ptr()), n, ld,
                                      C.c_void_p(lnl.data_ptr()), C.c_void_p(st.data_ptr()),
                                      _ffi.PREC_FP32 if prec == "fp32" else
                                      (_ffi.PREC_BF16 if prec == "bf16" else _ffi.PREC_FP32_SIMT),
                                      C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0, ctx._lib.sed_last_error(ctx._h).decode()
    return lnl, st


@pytest.mark.parametrize("prec", ["fp32", "fp32_simt", "bf16"])
def test_noalloc_matches_loglike_on_two_calls(setup, prec):
    ctx, model, orc, w, _ffi = setup
    tol = 1e-5 if prec != "bf16" else 1e-2
    for seed, n in ((61, 200), (62, 77)):          # two calls in a row, different batches
        th32, _ = cases.theta_pair(w, n, seed=seed)
        th32[3, model.offsets["zred"]] = w.zf + 1  # one bad row: status must come through too
        t = torch.from_numpy(th32).cuda()
        ref_l, ref_s = model.loglike(t, prec)
        got_l, got_s = _noalloc(ctx, model, t, prec, _ffi)
        torch.cuda.synchronize()
        ref_l, ref_s = ref_l.cpu().numpy(), ref_s.cpu().numpy()
        got_l, got_s = got_l.cpu().numpy(), got_s.cpu().numpy()
        assert np.array_equal(ref_s, got_s)
        ok = ref_s == 0
        assert np.isneginf(got_l[~ok]).all()
        assert np.max(np.abs(got_l[ok] - ref_l[ok]) / np.abs(ref_l[ok])) < tol


def test_noalloc_rejects_batches_beyond_scratch(setup):
    ctx, model, orc, w, _ffi = setup
    n = 200000        # far beyond the 32 MiB scratch for this grid
    t = torch.zeros((1, model.n_param), dtype=torch.float32, device="cuda")
    lnl = torch.empty(1, dtype=torch.float64, device="cuda")
    rc = ctx._lib.sed_loglike_noalloc(ctx._h, model.id, C.c_void_p(t.data_ptr()), n, model.n_param,
                                      C.c_void_p(lnl.data_ptr()), None, _ffi.PREC_FP32,
                                      C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == _ffi.SED_ERANGE
    assert b"maximum" in ctx._lib.sed_last_error(ctx._h)
