"""Small cases for ncu captures of the hot-path kernels (not a pytest module).

Default: the paper-scale photometric batch (107 x 12 x 6000 grid, 120 bins,
20 filters, 1024 parameter rows): three FP32 (3xTF32) sed_loglike calls, then
one BF16, one FP8 and one FP32-SIMT call, then one FP32 sed_loglike_grad.
About 1 GB of device memory.  Launch order of k_contract_tc: 3xTF32 x3, BF16,
FP8, adjoint.

``specphot``: the [a/Fe] spectro-photometric workload (107 x 12 x 5 x 6000
grid, 1500-pixel spectrum + 20 filters) at 512 rows: one FP32 sed_loglike and
two FP32 sed_loglike_grad calls.

``calib``: the same with a marginalised 13-term Chebyshev calibration
polynomial on the spectrum (prior widths 0.2, then 0.1).
"""
import os
import sys

import numpy as np
import torch

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import synth  # noqa: E402
from paper_2609_30145_gb300 import Context  # noqa: E402


def specphot(calib=False):
    w = synth.WORKLOADS["specphot_afe_107x12x5x6000_b2048"]
    grid = synth.make_grid(**w.grid_kw, seed=1)
    filt = synth.pack_filters(synth.workload_filters(w))
    sp = w.spectrum
    lam, r = synth.make_spectrum_pixels(sp["n_pix"], sp["lo_um"], sp["hi_um"], sp["r_lo"], sp["r_hi"])
    nb = len(filt[0])
    ctx = Context(0)
    gid = ctx.load_grid(grid)
    m = ctx.create_model(gid, w.n_sfh, w.zf, w.zmode, use_afe=w.use_afe, use_nebular=w.use_nebular,
                         dust_law=w.dust_law, filters=filt, phot_d=np.ones(nb), phot_sigma=np.ones(nb),
                         spec_lam=lam, spec_d=np.ones(lam.size), spec_sigma=np.ones(lam.size), lsf_mode=0,
                         lsf_value=r, sigma_gal_kms=w.sigma_gal_kms, z_ref=w.z_ref,
                         calib_sigma=np.array([0.2] + [0.1] * 12) if calib else None)
    # mock data: the model at a true row (z = 2) with 5% offsets
    d_true = synth.make_theta(1, w.n_sfh, w.zmode, w.ranges, seed=99)
    d_true["zred"][:] = 2.0
    ph, s0 = m.forward(torch.from_numpy(m.pack(d_true)).cuda(), "fp32")
    ph = ph.cpu().numpy()[0].astype(np.float64)
    s0 = s0.cpu().numpy()[0].astype(np.float64)
    m.set_data(phot_d=ph * 1.05, phot_sigma=np.abs(ph) / 20.0, spec_d=s0 * 0.95, spec_sigma=np.abs(s0) / 20.0)
    t = torch.from_numpy(m.pack(synth.make_theta(512, w.n_sfh, w.zmode, w.ranges, seed=5))).cuda()
    m.loglike(t, "fp32")
    m.loglike_grad(t, "fp32")
    m.loglike_grad(t, "fp32")
    torch.cuda.synchronize()
    ctx.close()
    print("ok")


def main():
    if len(sys.argv) > 1 and sys.argv[1] in ("specphot", "calib"):
        return specphot(calib=sys.argv[1] == "calib")
    w = synth.WORKLOADS["phot_107x12x6000_b1024"]
    grid = synth.make_grid(**w.grid_kw, seed=1)
    filt = synth.pack_filters(synth.workload_filters(w))
    nb = len(filt[0])
    ctx = Context(0)
    gid = ctx.load_grid(grid)
    m = ctx.create_model(gid, w.n_sfh, w.zf, w.zmode, use_nebular=w.use_nebular, dust_law=w.dust_law,
                         filters=filt, phot_d=np.full(nb, 1e-9), phot_sigma=np.full(nb, 1e-10))
    t = torch.from_numpy(m.pack(synth.make_theta(w.batch, w.n_sfh, w.zmode, w.ranges, seed=5))).cuda()
    for prec in ["fp32", "fp32", "fp32", "bf16", "fp8", "fp32_simt"]:
        m.loglike(t, prec)
    m.loglike_grad(t, "fp32")
    torch.cuda.synchronize()
    ctx.close()
    print("ok")


if __name__ == "__main__":
    main()
