"""Small case for ncu captures of the hot-path kernels (not a pytest module).

The paper-scale photometric batch (107 x 12 x 6000 grid, 120 bins, 20 filters,
1024 parameter rows): three FP32 (3xTF32) sed_loglike calls, then one BF16,
one FP8 and one FP32-SIMT call, then one FP32 sed_loglike_grad.  About 1 GB of
device memory.  Launch order of k_contract_tc: 3xTF32 x3, BF16, FP8, adjoint.
"""
import os
import sys

import numpy as np
import torch

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import synth  # noqa: E402
from paper_2609_30145_gb300 import Context  # noqa: E402


def main():
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
