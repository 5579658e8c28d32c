"""Rows placed in the redshift order by the preparation kernel itself.

A single-fit launch of at most 1024 rows, with theta in device memory and no
K-tile masks, runs without the ordering kernel: each prep CTA counts the rows
whose (redshift bin, index) key is below its own row's and writes the row's
weights and scalars at that place.  theta in mapped host memory still goes
through the ordering kernel (its CTAs would otherwise each read every row over
the host link).  No row's result depends on the order or on which rows share
its 128-row tile, so both launches must give the same lnL and status bit for
bit, and agree with the FP64 oracle on sampled rows.  Cases: rows spread in
redshift, every row at one redshift (all keys equal: the caller's order), rows
with invalid redshifts (the last bin), every row invalid, one row, a ragged batch, and the
limit.

Each call's epilogue empties the per-tile windows that the contraction read,
so that the next self-ordered call starts from empty windows; a sequence of
calls of different sizes and redshift ranges, with an FFMA call and a gradient
call in between, must give every call the ordering kernel's results.
"""
import numpy as np
import pytest

import synth
from tests import cases

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

LNL_TOL = {"fp32": 1e-5, "fp32_simt": 1e-5, "bf16": 1e-2}


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


_CASE = {}


def phot_case(ctx):
    if "phot" not in _CASE:
        w = synth.WORKLOADS["phot_107x12x6000_b1024"]
        orc = cases.oracle_for(w)
        _CASE["phot"] = (w, orc, cases.gpu_model_for(ctx, orc, w))
    return _CASE["phot"]


def rows(w, model, n, seed, kind, z_range=None):
    th32, _ = cases.theta_pair(w, n, seed=seed)
    zc = model.offsets["zred"]
    rng = np.random.default_rng(seed)
    if z_range is not None:
        th32[:, zc] = rng.uniform(*z_range, n).astype(np.float32)
    if kind == "one_z":
        th32[:, zc] = np.float32(3.0)
    elif kind == "all_bad":
        th32[:, zc] = np.float32(w.zf + 1.0)
    elif kind == "bad_z":
        k = max(n // 7, 1)
        bad = rng.choice(n, k, replace=False)
        th32[bad[::2], zc] = np.float32(w.zf + 1.0)
        th32[bad[1::2], zc] = np.float32(-0.5)
    return th32


def via_device(model, th32, prec):
    lnl, st = model.loglike(torch.from_numpy(th32).cuda(), prec)
    torch.cuda.synchronize()
    return lnl.cpu().numpy(), st.cpu().numpy().astype(np.uint32)


def via_ordering_kernel(ctx, model, th32, prec):
    """theta read in place from page-locked host memory: the ordering kernel runs."""
    th_pin = torch.from_numpy(th32).pin_memory()
    lnl, st = model.loglike_host(th_pin, prec)
    assert ctx.last_host_path() & 1, "theta was not read in place"
    return np.asarray(lnl), np.asarray(st).astype(np.uint32)


@pytest.mark.parametrize("prec", ["fp32", "bf16", "fp32_simt"])
@pytest.mark.parametrize("n,kind", [(1, "spread"), (77, "spread"), (300, "one_z"), (300, "bad_z"),
                                    (1000, "spread"), (1024, "bad_z"), (1024, "all_bad")])
def test_self_ordered_launch_matches_ordering_kernel(ctx, prec, n, kind):
    w, orc, model = phot_case(ctx)
    th32 = rows(w, model, n, 100 + n, kind)
    l_self, s_self = via_device(model, th32, prec)
    l_ord, s_ord = via_ordering_kernel(ctx, model, th32, prec)
    assert np.array_equal(s_self, s_ord)
    assert np.array_equal(l_self, l_ord)
    ok = s_self == 0
    if kind == "bad_z":
        assert (~ok).sum() == max(n // 7, 1) and np.isneginf(l_self[~ok]).all()
    if kind == "all_bad":   # every row in the invalid bin: no tile is computed, every lnL is -inf
        assert not ok.any() and np.isneginf(l_self).all()
        return
    # the FP64 oracle on sampled rows
    idx = np.nonzero(ok)[0]
    sample = np.unique(np.concatenate([idx[:2], idx[-2:], np.random.default_rng(n).choice(idx, min(8, len(idx)),
                                                                                          replace=False)]))
    ref = orc.eval(th32[sample].astype(np.float64))
    assert np.array_equal(ref["status"], s_self[sample])
    err = np.max(np.abs(l_self[sample] - ref["lnl"]) / cases.lnl_scale(orc, ref))
    assert err < LNL_TOL[prec], f"{err:.3e}"


def test_windows_left_empty_between_calls(ctx):
    w, orc, model = phot_case(ctx)
    seq = [("fp32", 1024, (0.0, 0.3)), ("fp32", 300, (8.0, 11.0)), ("fp32_simt", 500, (2.0, 5.0)),
           ("grad", 200, (0.5, 1.0)), ("fp32", 1024, None), ("bf16", 129, (6.0, 6.5)), ("fp32", 1024, (0.0, 0.3))]
    for i, (prec, n, zr) in enumerate(seq):
        th32 = rows(w, model, n, 300 + i, "spread", z_range=zr)
        if prec == "grad":
            lg, g, sg = model.loglike_grad(torch.from_numpy(th32).cuda(), "fp32")
            torch.cuda.synchronize()
            l_self, s_self = lg.cpu().numpy(), sg.cpu().numpy().astype(np.uint32)
            assert np.isfinite(g.cpu().numpy()[s_self == 0]).all()
            l_ref, s_ref = via_ordering_kernel(ctx, model, th32, "fp32")
            # the adjoint epilogue evaluates lnL in its own FP32 order (as in the gradient tests)
            assert np.array_equal(s_self, s_ref)
            ok = s_self == 0
            assert np.allclose(l_self[ok], l_ref[ok], rtol=1e-5, atol=0)
            continue
        else:
            l_self, s_self = via_device(model, th32, prec)
            l_ref, s_ref = via_ordering_kernel(ctx, model, th32, prec)
        assert np.array_equal(s_self, s_ref), (i, prec)
        assert np.array_equal(l_self, l_ref), (i, prec)
