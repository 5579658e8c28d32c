"""Continuous-batching server (sed_server_*): fits of different shapes (filter
count, spectrum length, SFH bins, constant or per-bin [Fe/H], [a/Fe] on or
off) share one grid; calls submitted from many threads at once are packed
into shared launches, and each call's lnL and row status must equal those of
sed_loglike on the same rows alone (bitwise: no row's arithmetic depends on
the other rows of a launch).  Also: admission by the fit budget.
"""
import threading

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
    from paper_2609_30145_gb300 import Context
    ctx = Context(0)
    base = synth.WORKLOADS["specphot_afe_107x12x5x6000_b2048"]
    grid = synth.make_grid(**dict(base.grid_kw, n_lam=1500), seed=1)
    gid = ctx.load_grid(grid)
    specs = [  # (n_filt, n_pix, n_sfh, zmode, use_afe)
        (8, 0, 10, 0, 0), (20, 300, 30, 1, 1), (30, 0, 120, 0, 1), (12, 200, 60, 1, 0)]
    fits = []
    for i, (nf, npix, nsfh, zmode, afe) in enumerate(specs):
        filt = synth.pack_filters(synth.make_filters_nircam_like(nf // 2, nf - nf // 2, seed=10 + i))
        kw = dict(use_afe=afe, dust_law=1, filters=filt, phot_d=np.full(nf, 1e-9),
                  phot_sigma=np.full(nf, 1e-10))
        if npix:
            lam, r = synth.make_spectrum_pixels(npix, 0.7, 5.0, 100.0, 800.0)
            kw.update(spec_lam=lam, spec_d=np.full(npix, 1e-30), spec_sigma=np.full(npix, 1e-31),
                      lsf_mode=0, lsf_value=r, sigma_gal_kms=300.0, z_ref=5.0)
        m = ctx.create_model(gid, nsfh, 30.0, zmode, **kw)
        w = synth.shrink(base, n_sfh=nsfh)
        w.zmode = zmode
        w.use_afe = afe
        fits.append((m, w))
    yield ctx, gid, fits
    ctx.close()


def _rows(w, n, seed):
    return cases.theta_rows(w, n, seed=seed).astype(np.float32)


@pytest.mark.parametrize("prec", ["bf16", "fp32"])
def test_results_alone_equal_results_in_the_mix(setup, prec):
    from paper_2609_30145_gb300 import Server
    ctx, gid, fits = setup
    sizes = [64, 300, 1000, 130]
    thetas = [_rows(w, n, seed=70 + i) for i, ((m, w), n) in enumerate(zip(fits, sizes))]
    thetas[1][5, fits[1][0].offsets["zred"]] = 99.0   # one bad row: its status must come through
    alone = []
    for (m, w), th in zip(fits, thetas):
        lnl, st = m.loglike(torch.from_numpy(th).cuda(), prec)
        torch.cuda.synchronize()
        alone.append((lnl.cpu().numpy(), st.cpu().numpy().astype(np.uint32)))
    srv = Server(ctx, gid, fits[0][0], precision=prec, max_launch_rows=2048, n_slots=3)
    fit_ids = [srv.open_fit(m, 1024) for m, _ in fits]
    results = [None] * len(fits)
    barrier = threading.Barrier(len(fits))

    def client(i):
        barrier.wait()
        out = []
        for rep in range(3):   # three calls in a row per fit, all fits at once
            t = srv.submit(fit_ids[i], thetas[i])
            out.append(srv.wait(t, thetas[i].shape[0], timeout_ms=60000))
        results[i] = out

    th = [threading.Thread(target=client, args=(i,)) for i in range(len(fits))]
    for t in th:
        t.start()
    for t in th:
        t.join()
    stats = srv.stats()
    for i in range(len(fits)):
        for lnl, st, lat in results[i]:
            assert np.array_equal(st, alone[i][1])
            assert np.array_equal(lnl, alone[i][0]), (i, np.max(np.abs(lnl - alone[i][0])))
            assert lat > 0
    assert stats["calls"] == 3 * len(fits)
    assert stats["launches"] <= stats["calls"]
    for f in fit_ids:
        srv.close_fit(f)
    srv.close()

    # one launch slot and back-to-back submissions from one thread: the calls
    # that arrive while the first one runs are packed into one launch
    srv = Server(ctx, gid, fits[0][0], precision=prec, max_launch_rows=2048, n_slots=1)
    fit_ids = [srv.open_fit(m, 1024) for m, _ in fits]
    tickets = [srv.submit(f, th) for f, th in zip(fit_ids, thetas)]
    for i, t in enumerate(tickets):
        lnl, st, _ = srv.wait(t, thetas[i].shape[0], timeout_ms=60000)
        assert np.array_equal(lnl, alone[i][0]) and np.array_equal(st, alone[i][1])
    stats = srv.stats()
    assert stats["calls"] == len(fits) and stats["launches"] < len(fits), stats
    for f in fit_ids:
        srv.close_fit(f)
    srv.close()


def test_admission_by_fit_budget_and_device_submit(setup):
    from paper_2609_30145_gb300 import Server
    ctx, gid, fits = setup
    m, w = fits[0]
    per_fit = ((512 * m.n_param * 4 + 255) // 256) * 256
    srv = Server(ctx, gid, m, precision="fp32", max_launch_rows=1024, n_slots=2, fit_budget_bytes=2 * per_fit)
    a = srv.open_fit(m, 512)
    b = srv.open_fit(m, 512)
    assert a is not None and b is not None
    assert srv.open_fit(m, 512) is None              # over budget: SED_EBUSY
    srv.close_fit(a)
    c = srv.open_fit(m, 512)
    assert c is not None
    # live points written on the device, then a device-side submit
    th = _rows(w, 100, seed=80)
    ptr = srv.fit_theta_ptr(c)
    assert ptr

    class _DeviceRows:   # the fit's live-point buffer seen as a torch tensor
        def __init__(self, p, shape):
            self.__cuda_array_interface__ = {"shape": shape, "typestr": "<f4", "data": (p, False),
                                             "version": 3, "strides": None}
    live = torch.as_tensor(_DeviceRows(ptr, (512, m.n_param)), device="cuda")
    dev = torch.from_numpy(th).cuda()
    live[:100].copy_(dev)
    torch.cuda.synchronize()
    t = srv.submit_device(c, 100)
    lnl, st, _ = srv.wait(t, 100, timeout_ms=60000)
    ref_l, ref_s = m.loglike(dev, "fp32")
    torch.cuda.synchronize()
    assert np.array_equal(lnl, ref_l.cpu().numpy())
    srv.close_fit(b)
    srv.close_fit(c)
    srv.close()
