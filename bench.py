#!/usr/bin/env python
"""Throughput benchmark of the batched SED log-likelihood on GB300.

Workload (default): the paper-scale photometric batch -- SSP grid 107 ages x
12 [Fe/H] x 6000 wavelengths, 120 SFH bins with one [Fe/H] per bin,
birth-cloud + Kriek & Conroy diffuse dust, nebular template 7 logU x 12 Z,
20 filters, z in [0, 12], 1024 parameter rows per step.

A step is one call of sed_loglike over the 1024-row batch (parameter
preparation -> contraction -> fused epilogue -> lnL).  Inputs are resident
in HBM when the timed region starts; L2 is flushed (256 MiB memset) before
every timed step and the flush is outside the per-step CUDA-event timing.
Under torchrun each rank evaluates its own batch (weak scaling, no
collective on the data path); rank 0 prints one JSON line.

--impl reference times the FP64 CPU oracle (the reference of this build) on
the host cores, on bounded samples of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "phot_107x12x6000_b1024"
GRAD_WORKLOAD = "specphot_afe_107x12x5x6000_b2048"
SGAL_WORKLOAD = "specphot_afe_sgal_107x12x5x6000_b2048"   # the same with a sampled sigma_gal
CALIB_WORKLOAD = "specphot_afe_calib13_107x12x5x6000_b2048"  # the same with a 13-term calibration polynomial
FLOOR_WORKLOAD = "specphot_afe_floor_107x12x5x6000_b2048"    # the same with every noise-floor term on
LINSFH_WORKLOAD = "phot_linsfh_107x12x6000_b1024"   # the headline fit with the linear SFH scheme
LINES_WORKLOAD = "specphot_lines_107x12x6000_b1024"  # JADES-like: emission lines, spectrum, line catalogue
PRECS = ("fp32", "fp32_simt", "bf16", "fp8")
SELF_ORDER_MAX = 1024   # a device-theta batch of at most this many rows (one fit, no K-tile masks) runs no ordering kernel
PREC_NOTE = {"fp32": "3xTF32 split on tcgen05, FP32 accumulate, FP64 likelihood sums",
             "bf16": "BF16 tcgen05, FP32 accumulate, FP64 likelihood sums",
             "fp8": "FP8 E4M3 tcgen05 (power-of-two scales per SSP column and per row), FP32 accumulate, FP64 likelihood sums",
             "fp32_simt": "FP32 FFMA contraction, FP64 likelihood sums"}
PEAKS_FALLBACK = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}
TF32_PER_BF16 = 1.1 / 2.25          # nominal dense tensor ratio (recipe table)
METRIC = "SED loglike evals/sec vs plain FP32 path at stated FP64-error; p50/p99 latency"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp32_simt", "bf16", "fp8"])
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-grad", action="store_true")
    ap.add_argument("--serve-requests", type=int, default=200)
    ap.add_argument("--serve-threads", type=int, default=48)
    ap.add_argument("--serve-mean-calls", type=float, default=5.0,
                    help="mean calls per request of the serving mix (the full serving config: 20, with "
                         "--serve-requests 10000)")
    ap.add_argument("--serve-budget-mb", type=int, default=4096)
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--no-sampler", action="store_true",
                    help="skip the nested-slice-sampling leg (time per fit of a JADES-like model)")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the per-config accuracy and throughput leg (tiny, paper-scale photometric at 1024 "
                         "and 4096 rows, spectro-photometric [a/Fe], serving mix)")
    ap.add_argument("--profile-case", default=None, choices=["phot", "specphot", "calib", "nss"],
                    help="run one small case of the hot path for an ncu capture and exit (no timing, no JSON)")
    return ap.parse_args()


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d, "measured"
    return PEAKS_FALLBACK, "fallback"


# --------------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-lms", "100", "-i", str(self.index)],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (FileNotFoundError, OSError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# --------------------------------------------------------------------------- workload
def build_workload(wname, ctx, seed_rows, device):
    import torch
    import synth

    optimised = wname.endswith(":optimised")   # the same workload, calibration optimised at each call
    w = synth.WORKLOADS[wname.split(":")[0]]
    if optimised:
        w = synth.Workload(**{**w.__dict__, "name": w.name + "_optimised", "extra": {**w.extra, "calib_mode": 1}})
    grid = synth.make_grid(**w.grid_kw, seed=1)
    filt = synth.pack_filters(synth.workload_filters(w))
    nb = len(filt[0])
    kw = dict(use_afe=w.use_afe, use_nebular=w.use_nebular, dust_law=w.dust_law, filters=filt,
              phot_d=np.ones(nb), phot_sigma=np.ones(nb), sample_sigma_gal=w.sample_sigma_gal,
              sigma_gal_max_kms=w.sigma_gal_max_kms, noise_floor_phot=w.floor_phot,
              noise_floor_spec=w.floor_spec, sfh_scheme=w.sfh_scheme)
    if w.spectrum is not None and w.extra.get("calib_sigma"):
        kw.update(calib_sigma=np.asarray(w.extra["calib_sigma"]), calib_mode=w.extra.get("calib_mode", 0))
    ln = w.extra.get("lines")
    if ln:
        # emission lines and a line catalogue of single lines and blends; its data
        # are seeded values at the level of a strong line (the timing does not
        # depend on them)
        rng = np.random.default_rng(17)
        blends, k = [], 0
        while len(blends) < ln["n_lcat"]:
            size = 1 + (len(blends) % 3 == 1) * int(rng.integers(0, 3))
            blends.append(list(range(k, k + size)))
            k += size
        kw.update(use_lines=1, gas_sigma_mode=ln["gas_sigma_mode"], sigma_gas_max_kms=ln["sigma_gas_max_kms"],
                  lcat=(blends, 1e-18 * (1 + 0.05 * rng.standard_normal(len(blends))),
                        np.full(len(blends), 5e-20), None, None))
    spec = None
    if w.spectrum is not None:
        sp = w.spectrum
        lam, r = synth.make_spectrum_pixels(sp["n_pix"], sp["lo_um"], sp["hi_um"], sp["r_lo"], sp["r_hi"])
        kw.update(spec_lam=lam, spec_d=np.ones(lam.size), spec_sigma=np.ones(lam.size), lsf_mode=0,
                  lsf_value=r, sigma_gal_kms=w.sigma_gal_kms, z_ref=w.z_ref)
        spec = lam
    gid = ctx.load_grid(grid)
    model = ctx.create_model(gid, w.n_sfh, w.zf, w.zmode, **kw)
    # mock data: the model at a true parameter row (z = 2), 5% Gaussian noise
    d_true = synth.make_theta(1, w.n_sfh, w.zmode, w.ranges, seed=99)
    if w.sfh_scheme == 1:   # linear SFH scheme: per-edge SFRs
        d_true["sfh"] = synth.edge_sfr(1, w.n_sfh, seed=99)
    d_true["zred"][:] = 2.0
    # noise-floor columns, if any: the model fluxes do not depend on them
    d_true.update(synth.floor_theta(1, w.floor_phot, w.floor_spec, np.ones(nb), np.ones(1)))
    if "sigma_gas" in w.ranges:
        d_true["sigma_gas"] = np.array([150.0])
    th_true = torch.from_numpy(model.pack(d_true)).to(device)
    ph, sp_ = model.forward(th_true, "fp32")
    torch.cuda.synchronize()
    ph = ph.cpu().numpy()[0].astype(np.float64)
    nz = synth.noise(nb + (0 if spec is None else spec.size), seed=5)
    pd = ph * (1 + nz[:nb] / 20.0)
    if spec is None:
        model.set_data(phot_d=pd, phot_sigma=np.abs(ph) / 20.0)
    else:
        s0 = sp_.cpu().numpy()[0].astype(np.float64)
        model.set_data(phot_d=pd, phot_sigma=np.abs(ph) / 20.0, spec_d=s0 * (1 + nz[nb:] / 20.0),
                       spec_sigma=np.abs(s0) / 20.0)
    d = synth.make_theta(w.batch, w.n_sfh, w.zmode, w.ranges, seed=seed_rows)
    if w.sfh_scheme == 1:
        d["sfh"] = synth.edge_sfr(w.batch, w.n_sfh, seed=seed_rows)
    d.update(synth.floor_theta(w.batch, w.floor_phot, w.floor_spec, np.abs(ph) / 20.0,
                               None if spec is None else np.abs(s0) / 20.0, seed=seed_rows + 1000))
    if "sigma_gas" in w.ranges:
        lo, hi = w.ranges["sigma_gas"]
        d["sigma_gas"] = np.random.default_rng(seed_rows + 3000).uniform(lo, hi, w.batch)
    theta = model.pack(d)
    return w, grid, filt, model, theta, (pd, np.abs(ph) / 20.0)


# --------------------------------------------------------------------------- roofline
def contraction_peak(prec, pk, pk_kind):
    """Dense peak of the contraction's instruction kind.  The contraction is
    timed per launch inside a ~0.1 ms step, so the burst figure applies; TF32
    and FP8 take the measured BF16 burst peak times the nominal dense ratio."""
    bf = pk["bf16_tflops"]
    if prec == "fp32":
        return bf * TF32_PER_BF16, f"TF32 dense = burst BF16 {bf} x {TF32_PER_BF16:.3f} (nominal ratio), of {pk_kind}"
    if prec == "bf16":
        return bf, f"burst BF16 dense, of {pk_kind}"
    if prec == "fp8":
        return bf * 2.0, f"FP8 dense = burst BF16 {bf} x 2 (nominal ratio), of {pk_kind}"
    return 152 * 128 * 2 * 2.07e9 / 1e12, "FP32 FFMA: 152 SMs x 128 lanes x 2 FLOP x 2070 MHz (recipe unit counts)"


def stage_roofline(ctx, fn, stream, flush, prec, B, pk, pk_kind, reps):
    """Per-kernel times of `reps` direct calls (the library's events), and the
    contraction's algorithmic and issued rates against its dense peak; the
    epilogue's algorithmic bytes (Y and O per row) against measured HBM."""
    import torch

    ctx.set_profiling(True)
    stats = []
    with torch.cuda.stream(stream):
        for _ in range(reps):
            flush.zero_()
            torch.cuda._sleep(200000)
            fn(stream)
            stats.append(ctx.last_stats(stream))
    ctx.set_profiling(False)
    c_ms = statistics.mean(st["ms_contract"] for st in stats)
    e_ms = statistics.mean(st["ms_epilogue"] for st in stats)
    p_ms = statistics.mean(st["ms_prep"] for st in stats)
    nnz, n_lam = stats[-1]["nnz_w"], stats[-1]["n_lam"]
    issued = statistics.mean(st["issued_flop"] for st in stats)
    alg_flop = 2.0 * nnz * n_lam
    peak_tf, note = contraction_peak(prec, pk, pk_kind)
    achieved = alg_flop / (c_ms * 1e-3) / 1e12
    epi_bytes = B * n_lam * 8.0 + B * 8
    return {"kernel": "k_contract_tc" if prec != "fp32_simt" else "k_contract_simt",
            "bound": "tensor" if prec != "fp32_simt" else "alu", "achieved": round(achieved, 3),
            "peak": round(peak_tf, 1), "unit": "TFLOP/s", "frac": round(achieved / peak_tf, 4),
            "peak_note": note, "algorithmic_flop_per_launch": alg_flop, "nnz_w_per_launch": nnz,
            "issued_tflops": round(issued / (c_ms * 1e-3) / 1e12, 2),
            "issued_frac": round(issued / (c_ms * 1e-3) / 1e12 / peak_tf, 4),
            "contract_ms": round(c_ms, 4), "prep_ms": round(p_ms, 4), "epilogue_ms": round(e_ms, 4),
            "epilogue_hbm": {"bound": "hbm", "achieved_gbs": round(epi_bytes / (e_ms * 1e-3) / 1e9, 1),
                             "peak": pk["hbm_gbs"], "frac": round(epi_bytes / (e_ms * 1e-3) / 1e9 / pk["hbm_gbs"], 4),
                             "bytes_per_launch": epi_bytes}}


# --------------------------------------------------------------------------- GPU leg
def capture_step(fn, stream, warm=3):
    """One step (a library call on `stream`) as a CUDA graph, after warm-up calls
    on the same stream (the library keeps one workspace per stream)."""
    import torch

    with torch.cuda.stream(stream):
        for _ in range(warm):
            fn(stream)
    stream.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        fn(stream)
    stream.synchronize()
    return g


def time_replays(g, stream, steps, flush, after=None):
    """Device time of each replay (CUDA events on the launching stream), L2
    flushed by a 256 MiB memset before every replay, outside the events."""
    import torch

    per = []
    with torch.cuda.stream(stream):
        for _ in range(steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            g.replay()
            e1.record(stream)
            per.append((e0, e1))
            if after is not None:
                after()
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in per]


def time_direct(fn, stream, steps, flush):
    """Same, with the library called directly each step (no graph)."""
    import torch

    per = []
    with torch.cuda.stream(stream):
        for _ in range(steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn(stream)
            e1.record(stream)
            per.append((e0, e1))
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in per]


def run_ours(args):
    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)

    import __graft_entry__
    if rank == 0:
        __graft_entry__.build()
    if dist:
        dist.barrier()
    from paper_2609_30145_gb300 import Context

    ctx = Context(local)
    w, grid, filt, model, theta, data = build_workload(args.workload, ctx, 4 + rank, device)
    B = w.batch
    t = torch.from_numpy(theta).to(device)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=device)
    prec = args.precision
    lnl = torch.empty(B, dtype=torch.float64, device=device)
    stt = torch.empty(B, dtype=torch.int32, device=device)

    def step_fn(p):
        return lambda s: model.loglike(t, p, stream=s, out=lnl, status=stt)

    # one step = one sed_loglike over the batch, replayed as a CUDA graph
    main_stream = torch.cuda.Stream(device=device)
    graphs = {p: capture_step(step_fn(p), main_stream, warm=max(args.warmup, 3)) for p in PRECS}
    for _ in range(max(args.warmup, 3)):
        graphs[prec].replay()
    torch.cuda.synchronize()

    clocks = ClockSampler(local)
    clocks.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ms = time_replays(graphs[prec], main_stream, args.steps, flush)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ck = clocks.stop()
    total_ms = sum(ms)
    if dist:
        from paper_2609_30145_gb300.shard import max_over_ranks
        total_ms = max_over_ranks(total_ms, device=device)
    ms_step = total_ms / args.steps
    value = world * B * args.steps / (total_ms * 1e-3)
    comm = None
    if dist:
        # the one exchange of the row-sharded path: every rank's lnL rows to all
        # ranks (outside the timed region), and a check that they all arrived
        from paper_2609_30145_gb300.shard import gather_rows
        full = gather_rows(lnl, world * B, world)
        torch.cuda.synchronize()
        comm = {"backend": dist.get_backend(), "world_size": dist.get_world_size(),
                "gathered_rows": int(full.shape[0]),
                "gathered_ok": bool(full.shape[0] == world * B and torch.equal(full[rank * B:(rank + 1) * B], lnl))}

    # per-kernel times: direct calls with the library's per-stage events on the
    # stream; a ~0.1 ms spin kernel ahead of each call lets the host enqueue all
    # of the call's kernels before the GPU reaches them (no host gaps between them)
    pk, pk_kind = peaks()
    by_prec = {p: stage_roofline(ctx, step_fn(p), main_stream, flush, p, B, pk, pk_kind,
                                 max(5, args.steps // 2)) for p in PRECS}
    roof = dict(by_prec[prec])
    roof["traffic"] = read_traffic() if prec == "fp32" else None
    roof["traffic_note"] = ("dram__bytes_read.sum + dram__bytes_write.sum of one k_contract_tc launch "
                            "(3xTF32) from the ncu capture in profiles/k_contract_tc_phot_b1024.md, taken on "
                            "the current kernel source (null when the source changed since)")
    roof["stage_times_note"] = ("contract/prep/epilogue times come from direct calls with the library's "
                                "CUDA events around each kernel, so they include the launch gaps that the "
                                "graph-replayed step (ms_per_step) does not have")
    roof["other_precisions"] = {p: v for p, v in by_prec.items() if p != prec}

    p50 = float(np.percentile(ms, 50))
    p99 = float(np.percentile(ms, 99))

    # the other precisions (graph replays), and direct calls without a graph
    variants = {}
    for vp in PRECS:
        vms = ms if vp == prec else time_replays(graphs[vp], main_stream, max(10, args.steps // 2), flush)
        variants[vp] = {"evals_per_s": round(B * len(vms) / (sum(vms) * 1e-3), 1),
                        "ms_per_step": round(sum(vms) / len(vms), 4)}
    dms = time_direct(step_fn(prec), main_stream, max(10, args.steps // 2), flush)
    variants[prec + "_direct_calls"] = {"evals_per_s": round(B * len(dms) / (sum(dms) * 1e-3), 1),
                                        "ms_per_step": round(sum(dms) / len(dms), 4)}
    # the same fit with the linear SFH scheme (per-edge SFRs, tent integrals)
    if args.workload == "phot_107x12x6000_b1024":
        wl, _, _, model_l, theta_l, _ = build_workload(LINSFH_WORKLOAD, ctx, 4 + rank, device)
        tl = torch.from_numpy(theta_l).to(device)
        gl = capture_step(lambda s: model_l.loglike(tl, prec, stream=s, out=lnl, status=stt), main_stream)
        lms = time_replays(gl, main_stream, max(10, args.steps // 2), flush)
        variants[prec + "_linear_sfh"] = {"evals_per_s": round(B * len(lms) / (sum(lms) * 1e-3), 1),
                                          "ms_per_step": round(sum(lms) / len(lms), 4),
                                          "workload": wl.name}

    # end to end through the host-buffer entry point (pinned host theta, lnL back to host)
    th_host = torch.from_numpy(theta).pin_memory()
    lnl_host = torch.empty(B, dtype=torch.float64).pin_memory()
    st_host = torch.empty(B, dtype=torch.int32).pin_memory()
    stream = torch.cuda.Stream()   # the caller's stream (a replayable graph needs one that is not the legacy default)
    for _ in range(3):
        model.loglike_host(th_host, prec, stream=stream, out=lnl_host, status=st_host)
    e2e_t = []
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        model.loglike_host(th_host, prec, stream=stream, out=lnl_host, status=st_host)
        e2e_t.append(time.perf_counter() - t0)
    e2e_total = sum(e2e_t)
    if dist:
        from paper_2609_30145_gb300.shard import max_over_ranks
        e2e_total = max_over_ranks(e2e_total, device=device)
    ld = theta.shape[1]
    e2e = {"value": round(world * B * args.steps / e2e_total, 1), "unit": "evals/s",
           "h2d_bytes_per_step": B * ld * 4, "d2h_bytes_per_step": B * 8 + B * 4,
           "p50_ms": round(1e3 * float(np.percentile(e2e_t, 50)), 4),
           "p99_ms": round(1e3 * float(np.percentile(e2e_t, 99)), 4),
           "what": "sed_loglike_host with pinned host buffers: theta host -> device, order/prep/contraction/"
                   "epilogue, lnL + status device -> host, stream synchronised; wall clock around each call",
           "host_path": {3: "in place: the kernels read theta and write lnL/status over the host link",
                         7: "in place over the host link, the call's launches replayed as a CUDA graph"}.get(
                             ctx.last_host_path(), "staged through device memory by async copies")}

    # GPU results for the accuracy comparison of the CPU-baseline leg
    gpu_res = {}
    for vp in PRECS:
        l, s = model.loglike(t, vp, stream=stream)
        ph, _ = model.forward(t, vp, stream=stream)
        torch.cuda.synchronize()
        gpu_res[vp] = (l.cpu().numpy(), s.cpu().numpy(), ph.cpu().numpy())

    out = {"metric": METRIC, "value": round(value, 1), "unit": "evals/s", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_step, 4),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
           "data": "synthetic: seeded SSP grid, nebular template, NIRCam-like filters and parameter rows "
                   "shaped like the paper's workloads; mock data = model at a true row + 5% noise",
           "config": {"workload": w.name, "batch_per_gpu": B, "n_age": int(grid.flux.shape[2]),
                      "n_feh": int(grid.flux.shape[1]), "n_lam": int(grid.flux.shape[3]),
                      "n_sfh": w.n_sfh, "n_filt": int(len(filt[0])), "nebular": bool(w.use_nebular),
                      "dust": "birth-cloud power law + Kriek & Conroy 2013 diffuse",
                      "precision": PREC_NOTE[prec],
                      "step": "one sed_loglike call over the batch (%s), replayed as a CUDA graph" % (
                          "3 kernels: prep (rows placed in redshift order by the prep kernel itself), contraction, epilogue"
                          if B <= SELF_ORDER_MAX else "4 kernels: row order, prep, contraction, epilogue"),
                      "l2": "flushed before every timed step (256 MiB memset, outside the timing)",
                      "parallelism": f"replicas x{world} (independent batches per GPU)",
                      "comm": comm},
           "latency_ms": {"p50": round(p50, 4), "p99": round(p99, 4), "what": "device time of one batch step"},
           "variants": variants, "roofline": roof, "clocks": ck, "e2e": e2e,
           "gpu_launches": (3 if B <= SELF_ORDER_MAX else 4) * args.steps}
    if rank == 0 and world == 1 and not args.no_grad:
        out["gradient"] = bench_gradient(ctx, device, flush, args)
    if rank == 0 and world == 1 and args.serve_requests > 0:
        out["serving"] = bench_serving(ctx, device, args)
    if rank == 0 and world == 1 and not args.no_sampler:
        out["sampler"] = bench_sampler(ctx, device)
    if rank == 0 and world == 1 and not args.no_configs:
        out["configs"] = bench_configs(ctx, device, flush, args)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"], out["accuracy_vs_fp64_oracle"] = cpu_baseline(w, grid, filt, data, theta, gpu_res,
                                                                            args.cpu_seconds)
    if rank == 0:
        print(json.dumps(out), flush=True)
    ctx.close()
    if dist:
        dist.barrier()
        dist.destroy_process_group()


def bench_gradient(ctx, device, flush, args):
    """Forward + adjoint (sed_loglike_grad) on the spectro-photometric [a/Fe]
    workload (107 x 12 x 5 x 6000 grid, 1500-pixel spectrum + 20 filters,
    2048 rows), one graph replay per step."""
    import torch

    w, grid, filt, model, theta, data = build_workload(GRAD_WORKLOAD, ctx, 4, device)
    B = w.batch
    t = torch.from_numpy(theta).to(device)
    lnl = torch.empty(B, dtype=torch.float64, device=device)
    grad = torch.empty_like(t)
    stt = torch.empty(B, dtype=torch.int32, device=device)
    s = torch.cuda.Stream(device=device)
    res = {"workload": w.name, "batch": B, "n_param": int(theta.shape[1])}
    # the same workload with a sampled sigma_gal (one more parameter column; the
    # spectral kernels' widths are per row): forward and gradient, 3xTF32
    ws, _, _, model_s, theta_s, _ = build_workload(SGAL_WORKLOAD, ctx, 4, device)
    ts = torch.from_numpy(theta_s).to(device)
    grad_s = torch.empty_like(ts)
    gs = capture_step(lambda st: model_s.loglike_grad(ts, "fp32", stream=st, out=(lnl, grad_s, stt)), s)
    gsm = time_replays(gs, s, max(5, args.steps // 4), flush)
    fs = capture_step(lambda st: model_s.loglike(ts, "fp32", stream=st, out=lnl, status=stt), s)
    fsm = time_replays(fs, s, max(5, args.steps // 4), flush)
    # and with a marginalised 13-term calibration polynomial on the spectrum
    wc, _, _, model_c, theta_c, _ = build_workload(CALIB_WORKLOAD, ctx, 4, device)
    tc = torch.from_numpy(theta_c).to(device)
    grad_c = torch.empty_like(tc)
    gc = capture_step(lambda st: model_c.loglike_grad(tc, "fp32", stream=st, out=(lnl, grad_c, stt)), s)
    gcm = time_replays(gc, s, max(5, args.steps // 4), flush)
    fc = capture_step(lambda st: model_c.loglike(tc, "fp32", stream=st, out=lnl, status=stt), s)
    fcm = time_replays(fc, s, max(5, args.steps // 4), flush)
    # and with the systematic noise floor (all four terms, both arms)
    wf, _, _, model_f, theta_f, _ = build_workload(FLOOR_WORKLOAD, ctx, 4, device)
    tf = torch.from_numpy(theta_f).to(device)
    grad_f = torch.empty_like(tf)
    gf = capture_step(lambda st: model_f.loglike_grad(tf, "fp32", stream=st, out=(lnl, grad_f, stt)), s)
    gfm = time_replays(gf, s, max(5, args.steps // 4), flush)
    ff = capture_step(lambda st: model_f.loglike(tf, "fp32", stream=st, out=lnl, status=stt), s)
    ffm = time_replays(ff, s, max(5, args.steps // 4), flush)
    # emission lines on the spectrum and photometry plus a line catalogue
    wl, _, _, model_l, theta_l, _ = build_workload(LINES_WORKLOAD, ctx, 4, device)
    tl = torch.from_numpy(theta_l).to(device)
    Bl = wl.batch
    lnl_l = torch.empty(Bl, dtype=torch.float64, device=device)
    stt_l = torch.empty(Bl, dtype=torch.int32, device=device)
    grad_l = torch.empty_like(tl)
    gl = capture_step(lambda st: model_l.loglike_grad(tl, "fp32", stream=st, out=(lnl_l, grad_l, stt_l)), s)
    glm = time_replays(gl, s, max(5, args.steps // 4), flush)
    fl = capture_step(lambda st: model_l.loglike(tl, "fp32", stream=st, out=lnl_l, status=stt_l), s)
    flm = time_replays(fl, s, max(5, args.steps // 4), flush)
    res["emission_lines"] = {"workload": wl.name, "batch": Bl, "n_param": int(theta_l.shape[1]),
                             "lines": 30, "catalogue_entries": wl.extra["lines"]["n_lcat"],
                             "grad_evals_per_s": round(Bl * len(glm) / (sum(glm) * 1e-3), 1),
                             "grad_ms_per_step": round(sum(glm) / len(glm), 4),
                             "loglike_evals_per_s": round(Bl * len(flm) / (sum(flm) * 1e-3), 1),
                             "loglike_ms_per_step": round(sum(flm) / len(flm), 4)}
    # the calibration polynomial optimised at each call instead of marginalised
    wo, _, _, model_o, theta_o, _ = build_workload(CALIB_WORKLOAD + ":optimised", ctx, 4, device)
    to = torch.from_numpy(theta_o).to(device)
    grad_o = torch.empty_like(to)
    go = capture_step(lambda st: model_o.loglike_grad(to, "fp32", stream=st, out=(lnl, grad_o, stt)), s)
    gom = time_replays(go, s, max(5, args.steps // 4), flush)
    fo = capture_step(lambda st: model_o.loglike(to, "fp32", stream=st, out=lnl, status=stt), s)
    fom = time_replays(fo, s, max(5, args.steps // 4), flush)
    res["calibration_polynomial_optimised"] = {
        "workload": wo.name, "grad_evals_per_s": round(B * len(gom) / (sum(gom) * 1e-3), 1),
        "grad_ms_per_step": round(sum(gom) / len(gom), 4),
        "loglike_evals_per_s": round(B * len(fom) / (sum(fom) * 1e-3), 1),
        "loglike_ms_per_step": round(sum(fom) / len(fom), 4)}
    res["noise_floor"] = {"workload": wf.name, "n_param": int(theta_f.shape[1]),
                          "terms": "error scale, f_calib, f_data, jitter on photometry and spectrum",
                          "grad_evals_per_s": round(B * len(gfm) / (sum(gfm) * 1e-3), 1),
                          "grad_ms_per_step": round(sum(gfm) / len(gfm), 4),
                          "loglike_evals_per_s": round(B * len(ffm) / (sum(ffm) * 1e-3), 1),
                          "loglike_ms_per_step": round(sum(ffm) / len(ffm), 4)}
    res["calibration_polynomial"] = {"workload": wc.name, "n_coef": len(wc.extra["calib_sigma"]),
                                     "grad_evals_per_s": round(B * len(gcm) / (sum(gcm) * 1e-3), 1),
                                     "grad_ms_per_step": round(sum(gcm) / len(gcm), 4),
                                     "loglike_evals_per_s": round(B * len(fcm) / (sum(fcm) * 1e-3), 1),
                                     "loglike_ms_per_step": round(sum(fcm) / len(fcm), 4)}
    res["sampled_sigma_gal"] = {"workload": ws.name, "n_param": int(theta_s.shape[1]),
                                "sigma_gal_kms": list(ws.ranges["sigma_gal"]),
                                "grad_evals_per_s": round(B * len(gsm) / (sum(gsm) * 1e-3), 1),
                                "grad_ms_per_step": round(sum(gsm) / len(gsm), 4),
                                "loglike_evals_per_s": round(B * len(fsm) / (sum(fsm) * 1e-3), 1),
                                "loglike_ms_per_step": round(sum(fsm) / len(fsm), 4)}
    for p in ("fp32", "fp32_simt"):
        g = capture_step(lambda st, p=p: model.loglike_grad(t, p, stream=st, out=(lnl, grad, stt)), s)
        gms = time_replays(g, s, max(5, args.steps // 4), flush)
        fwd = capture_step(lambda st, p=p: model.loglike(t, p, stream=st, out=lnl, status=stt), s)
        fms = time_replays(fwd, s, max(5, args.steps // 4), flush)
        res[p] = {"grad_evals_per_s": round(B * len(gms) / (sum(gms) * 1e-3), 1),
                  "grad_ms_per_step": round(sum(gms) / len(gms), 4),
                  "loglike_evals_per_s": round(B * len(fms) / (sum(fms) * 1e-3), 1),
                  "loglike_ms_per_step": round(sum(fms) / len(fms), 4)}
        # per-kernel times of the gradient call (library events, spin kernel ahead)
        ctx.set_profiling(True)
        stats = []
        with torch.cuda.stream(s):
            for _ in range(5):
                flush.zero_()
                torch.cuda._sleep(200000)
                model.loglike_grad(t, p, stream=s, out=(lnl, grad, stt))
                stats.append(ctx.last_stats(s))
        ctx.set_profiling(False)
        res[p]["stages_ms"] = {k: round(statistics.mean(st[f] for st in stats), 4) for k, f in
                               (("prep", "ms_prep"), ("contract", "ms_contract"), ("adjoint_epilogue", "ms_epilogue"),
                                ("dw", "ms_dw"), ("prep_bwd", "ms_prep_bwd"))}
    return res


# --------------------------------------------------------------------------- per-config accuracy and speed
CONFIGS = [  # (label, workload, rows on the GPU, rows sampled for the oracle)
    ("C1", "tiny_phot_16x4x512", 64, 64),
    ("C2", "phot_107x12x6000_b1024", 1024, 256),
    ("C3", "specphot_afe_107x12x5x6000_b2048", 2048, 128),
    ("C4", "phot_107x12x6000_b4096", 4096, 256),
]


def _q(x):
    x = np.asarray(x, dtype=np.float64)
    return {"median": float(np.median(x)), "p99": float(np.percentile(x, 99)), "max": float(x.max())}


def norm_const(orc):
    """C = -1/2 sum ln(2 pi sigma^2) over the data in the likelihood (lnL = -chi2/2 + C)."""
    c = 0.0
    for sig, mask in ((orc.phot_sigma, orc.phot_mask), (orc.spec_sigma, orc.spec_mask)):
        if sig is None or len(sig) == 0:
            continue
        m = np.ones(len(sig), bool) if mask is None else np.asarray(mask).astype(bool)
        c += -0.5 * np.sum(np.log(2 * np.pi * np.asarray(sig)[m] ** 2))
    return c


def err_stats(orc, ref, lnl, status, phot=None, spec=None):
    """Errors of GPU results against the FP64 oracle on the same rows: per datum
    relative flux error (floored at 1e-6 of the row's brightest datum), lnL
    error over the magnitude of its terms, absolute lnL error (what a sampler
    feels), relative error of chi2 alone (the normalisation C is the same on
    both sides and can hide chi2 errors), and the plain relative lnL error."""
    ok = ref["status"] == 0
    out = {"rows": int(ok.sum()), "status_match": bool(np.array_equal(status, ref["status"]))}
    fe = []
    for got, key in ((phot, "phot"), (spec, "spec")):
        if got is None or ref[key].size == 0:
            continue
        r, g = ref[key][ok], got[ok]
        floor = 1e-6 * np.abs(r).max(axis=1, keepdims=True)
        fe.append((np.abs(g - r) / np.maximum(np.abs(r), floor)).ravel())
    if fe:
        out["flux_rel_err"] = _q(np.concatenate(fe))
    c = norm_const(orc)
    lr = ref["lnl"][ok]
    d = np.abs(lnl[ok] - lr)
    chi2 = 2.0 * (c - lr)
    out["lnl_err_over_term_scale"] = _q(d / np.maximum(np.abs(lr), chi2 / 2 + abs(c)))
    out["lnl_abs_err"] = _q(d)
    out["chi2_rel_err"] = _q(2.0 * d / np.maximum(chi2, 1e-300))
    out["lnl_rel_err"] = _q(d / np.abs(lr))
    return out


def near_truth_rows(w, n, seed):
    """Rows around the row the mock data were made from (what a sampler's live
    points look like late in a run): its SFH masses times 1 + 5% noise and
    small Gaussian steps in the scalar keys (0.02 dex in metallicity, 0.01 dex
    in mass, 0.002 in redshift, 0.02 in the dust and gas keys), in the
    oracle's layout."""
    import oracle
    import synth
    from tests import cases

    d = synth.make_theta(1, w.n_sfh, w.zmode, w.ranges, seed=99)
    d["zred"][:] = min(2.0, w.zf * 0.5)
    rng = np.random.default_rng(seed)
    out = {}
    for k, v in d.items():
        v = np.repeat(np.asarray(v, dtype=np.float64), n, axis=0)
        step = {"sfh": None, "logzsol": 0.02, "afe": 0.02, "logmass": 0.01, "zred": 0.002, "tau_pow": 0.02,
                "diffuse_tau_kc": 0.02, "diffuse_dust_index": 0.02, "gas_logz": 0.02, "gas_logu": 0.02}.get(k, 0.0)
        if k == "sfh":
            v = v * (1.0 + 0.05 * rng.standard_normal(v.shape))
        elif step and np.ptp(np.atleast_1d(w.ranges.get(k, 0.0))) > 0:
            v = v + step * rng.standard_normal(v.shape)
        out[k] = v
    out["tau_pow"] = np.clip(out["tau_pow"], 0.0, None)
    out["diffuse_tau_kc"] = np.clip(out["diffuse_tau_kc"], 0.0, None)
    th = oracle.pack_theta(out, w.n_sfh, w.zmode).astype(np.float32)
    assert th.shape[1] == cases.z_column(w.n_sfh, w.zmode) + 7
    return th


def bench_configs(ctx, device, flush, args):
    """Every stated config on the GPU at its batch, in every precision: graph-
    replayed sed_loglike throughput, and errors against the FP64 oracle on
    sampled rows (C3 also the gradient against the oracle's analytic one)."""
    import torch
    import synth
    from tests import cases

    res = {}
    s = torch.cuda.Stream(device=device)
    for label, wname, n, n_orc in CONFIGS:
        w = synth.WORKLOADS[wname]
        orc = cases.oracle_for(w)
        model = cases.gpu_model_for(ctx, orc, w)
        th32, th64 = cases.theta_pair(w, n, seed=4)
        t = torch.from_numpy(th32).to(device)
        rows = np.arange(n) if n_orc >= n else np.sort(np.random.default_rng(11).choice(n, n_orc, replace=False))
        t0 = time.perf_counter()
        ref = orc.eval(th64[rows], nthreads=os.cpu_count() or 1)
        t_orc = time.perf_counter() - t0
        th_near = near_truth_rows(w, min(n, 128), seed=13)
        ref_near = orc.eval(th_near.astype(np.float64), nthreads=os.cpu_count() or 1)
        chi2_near = 2.0 * (norm_const(orc) - ref_near["lnl"])
        n_data = len(orc.phot_sigma) + (0 if orc.spec_sigma is None else len(orc.spec_sigma))
        lnl = torch.empty(n, dtype=torch.float64, device=device)
        stt = torch.empty(n, dtype=torch.int32, device=device)
        block = {"workload": w.name, "rows": n, "oracle_rows": int(rows.size),
                 "oracle_s": round(t_orc, 2), "precisions": {}}
        for p in PRECS:
            g = capture_step(lambda st, p=p: model.loglike(t, p, stream=st, out=lnl, status=stt), s)
            ms = time_replays(g, s, max(10, args.steps // 2), flush)
            l, st = model.loglike(t, p, stream=s)
            ph, sp = model.forward(t, p, stream=s)
            torch.cuda.synchronize()
            l, st = l.cpu().numpy()[rows], st.cpu().numpy()[rows]
            ph = None if ph is None else ph.cpu().numpy()[rows]
            sp = None if sp is None else sp.cpu().numpy()[rows]
            e = err_stats(orc, ref, l, st, ph, sp)
            # absolute lnL error where a sampler spends its late iterations
            tn = torch.from_numpy(th_near).to(device)
            ln, stn = model.loglike(tn, p, stream=s)
            torch.cuda.synchronize()
            ln, stn = ln.cpu().numpy(), stn.cpu().numpy()
            okn = (stn == 0) & (ref_near["status"] == 0)
            dn = np.abs(ln[okn] - ref_near["lnl"][okn])
            e["near_truth"] = {"rows": int(okn.sum()), "lnl_abs_err": _q(dn),
                               "chi2_per_datum_median": float(np.median(chi2_near[okn]) / n_data)}
            e["evals_per_s"] = round(n * len(ms) / (sum(ms) * 1e-3), 1)
            e["ms_per_step"] = round(sum(ms) / len(ms), 4)
            block["precisions"][p] = e
            del g
        if label == "C3":
            gr = [0, 1, n - 1] + list(np.random.default_rng(12).choice(n, 9, replace=False))
            gr = np.array(sorted(set(int(x) for x in gr)))
            _, gg, gst = model.loglike_grad(t, "fp32", stream=s)
            torch.cuda.synchronize()
            gg, gst = gg.cpu().numpy()[gr], gst.cpu().numpy()[gr]
            gref = orc.grad(th64[gr])["grad"]
            ok = gst == 0
            e = [np.max(np.abs(gg[i, :gref.shape[1]] - gref[i]) /
                        np.maximum(np.abs(gref[i]), 1e-3 * np.abs(gref[i]).max())) for i in np.nonzero(ok)[0]]
            block["gradient_fp32"] = {"rows": int(ok.sum()), "rel_err_max": float(max(e)),
                                      "what": "|g - g_oracle| / max(|g_oracle|, 1e-3 max_j |g_oracle_j|) over "
                                              "every column of each sampled row, worst row"}
        res[label] = block
        model.close()
    return res


def make_serving_requests(n_req, seed=6, mean_calls=5.0):
    """Seeded request mix shaped like the serving workload: photometry only
    (8-30 filters) or spectrum + photometry (200-3000 pixels), z in [0, 12],
    live-point batches log-uniform in 64..4096, 10-120 SFH bins, [a/Fe] on or
    off, each a dependent chain of a geometric number of calls."""
    rng = np.random.Generator(np.random.PCG64(seed))
    reqs = []
    for i in range(n_req):
        spec = bool(rng.random() < 0.5)
        reqs.append(dict(
            n_filt=int(rng.integers(8, 31)), n_pix=int(rng.integers(200, 3001)) if spec else 0,
            batch=int(np.exp(np.log(64) + rng.random() * (np.log(4096) - np.log(64)))),
            n_sfh=int(rng.integers(10, 121)), zmode=int(rng.integers(0, 2)), use_afe=int(rng.random() < 0.5),
            calls=int(min(4 * mean_calls, rng.geometric(1.0 / mean_calls))), seed=1000 + i))
    return reqs


def bench_serving(ctx, device, args):
    """Serving mix on the shared 107 x 12 x 5 x 6000 [a/Fe] grid: a bounded
    sample of seeded requests, first all arriving at once (saturated), then as
    a Poisson stream at 70% of the saturated throughput; BF16 server with the
    3xTF32 (FP32-grade) server timed beside it."""
    import threading
    import synth
    from paper_2609_30145_gb300 import Server

    base = synth.WORKLOADS[GRAD_WORKLOAD]
    grid = synth.make_grid(**base.grid_kw, seed=1)
    gid = ctx.load_grid(grid)
    reqs = make_serving_requests(args.serve_requests, mean_calls=args.serve_mean_calls)
    models, thetas, okws = [], [], []
    t_setup = time.perf_counter()
    for q in reqs:
        rng = np.random.Generator(np.random.PCG64(q["seed"]))
        nw = q["n_filt"] // 3
        filt = synth.pack_filters(synth.make_filters_nircam_like(nw, q["n_filt"] - nw, seed=q["seed"]))
        kw = dict(use_afe=q["use_afe"], dust_law=1, filters=filt, phot_d=np.ones(q["n_filt"]),
                  phot_sigma=np.ones(q["n_filt"]))
        if q["n_pix"]:
            lam, r = synth.make_spectrum_pixels(q["n_pix"], 0.6, 5.3, 100.0, 1000.0)
            kw.update(spec_lam=lam, spec_d=np.ones(q["n_pix"]), spec_sigma=np.ones(q["n_pix"]), lsf_mode=0,
                      lsf_value=r, sigma_gal_kms=300.0, z_ref=6.0)
        m = ctx.create_model(gid, q["n_sfh"], 30.0, q["zmode"], **kw)
        ranges = dict(base.ranges, afe=(-0.2, 0.6) if q["use_afe"] else 0.0)
        d_true = synth.make_theta(1, q["n_sfh"], q["zmode"], ranges, seed=q["seed"])
        d_true["zred"][:] = float(rng.random() * 11.0 + 0.5)
        ph, sp = m.forward(torch_from(m.pack(d_true), device), "fp32")
        ph = ph.cpu().numpy()[0].astype(np.float64)
        nz = synth.noise(q["n_filt"] + q["n_pix"], seed=q["seed"])
        # S/N 20 with a noise floor of 1e-3 of the brightest datum's sigma (bands
        # and pixels the model leaves dark keep a finite weight)
        def sig(x):
            a = np.abs(x)
            return a / 20 + max(1e-3 * a.max() / 20, 1e-30)
        if q["n_pix"]:
            s0 = sp.cpu().numpy()[0].astype(np.float64)
            data = dict(phot_d=ph * (1 + nz[:q["n_filt"]] / 20), phot_sigma=sig(ph),
                        spec_d=s0 * (1 + nz[q["n_filt"]:] / 20), spec_sigma=sig(s0))
        else:
            data = dict(phot_d=ph * (1 + nz / 20), phot_sigma=sig(ph))
        m.set_data(**data)
        kw.update(data)
        okws.append(dict(kw, n_sfh=q["n_sfh"], zf=30.0, zmode=q["zmode"]))
        models.append(m)
        thetas.append(m.pack(synth.make_theta(q["batch"], q["n_sfh"], q["zmode"], ranges, seed=q["seed"] + 1)))
    t_setup = time.perf_counter() - t_setup
    total_evals = sum(q["batch"] * q["calls"] for q in reqs)

    def run_direct(prec, rate):
        """The same mix through plain batched sed_loglike calls: each client
        calls the library on its own CUDA stream and waits for its result (the
        plain FP32 batched path, no server)."""
        import torch
        call_lat, req_lat = [], []
        lock = threading.Lock()
        rng = np.random.Generator(np.random.PCG64(7))
        arrivals = np.cumsum(rng.exponential(1.0 / rate, len(reqs))) if rate else np.zeros(len(reqs))
        t0 = time.perf_counter()
        nxt = [0]

        def worker():
            st_ = torch.cuda.Stream(device=device)
            while True:
                with lock:
                    i = nxt[0]
                    nxt[0] += 1
                if i >= len(reqs):
                    return
                q, m, th = reqs[i], models[i], thetas[i].copy()
                delay = t0 + arrivals[i] - time.perf_counter()
                if delay > 0:
                    time.sleep(delay)
                t_arr = time.perf_counter()
                jm = m.offsets["logmass"]
                lat = []
                for c in range(q["calls"]):
                    tc0 = time.perf_counter()
                    td = torch.from_numpy(th).to(device, non_blocking=False)
                    with torch.cuda.stream(st_):
                        l_, s_ = m.loglike(td, prec, stream=st_)
                        lnl = l_.cpu().numpy()
                    lat.append(1e3 * (time.perf_counter() - tc0))
                    good = np.isfinite(lnl)
                    if good.any():
                        med = np.median(lnl[good])
                        th[good, jm] += np.where(lnl[good] > med, 0.02, -0.02).astype(np.float32)
                with lock:
                    call_lat.extend(lat)
                    req_lat.append(1e3 * (time.perf_counter() - t_arr))

        threads = [threading.Thread(target=worker) for _ in range(args.serve_threads)]
        for t in threads:
            t.start()
        for t in threads:
            t.join()
        wall = time.perf_counter() - t0
        return {"evals_per_s": round(total_evals / wall, 1), "wall_s": round(wall, 3),
                "call_latency_ms": {"p50": round(float(np.percentile(call_lat, 50)), 3),
                                    "p99": round(float(np.percentile(call_lat, 99)), 3)},
                "request_latency_ms": {"p50": round(float(np.percentile(req_lat, 50)), 3),
                                       "p99": round(float(np.percentile(req_lat, 99)), 3)}}

    def run(prec, rate):
        srv = Server(ctx, gid, models[0], precision=prec, max_launch_rows=8192, n_slots=3,
                     fit_budget_bytes=args.serve_budget_mb << 20)
        call_lat, req_lat, admitted_wait = [], [], []
        lock = threading.Lock()
        rng = np.random.Generator(np.random.PCG64(7))
        arrivals = np.cumsum(rng.exponential(1.0 / rate, len(reqs))) if rate else np.zeros(len(reqs))
        t0 = time.perf_counter()
        nxt = [0]

        def worker():
            while True:
                with lock:
                    i = nxt[0]
                    nxt[0] += 1
                if i >= len(reqs):
                    return
                q, m, th = reqs[i], models[i], thetas[i].copy()
                delay = t0 + arrivals[i] - time.perf_counter()
                if delay > 0:
                    time.sleep(delay)
                t_arr = time.perf_counter()
                fit = srv.open_fit(m, q["batch"])
                while fit is None:          # admission: wait for device memory
                    time.sleep(0.0005)
                    fit = srv.open_fit(m, q["batch"])
                t_adm = time.perf_counter()
                lat = []
                jm = m.offsets["logmass"]
                for c in range(q["calls"]):
                    t = srv.submit(fit, th)
                    lnl, st, ms = srv.wait(t, th.shape[0])
                    lat.append(ms)
                    # toy slice step: the next call's rows depend on this call's lnL
                    good = np.isfinite(lnl)
                    if good.any():
                        med = np.median(lnl[good])
                        th[good, jm] += np.where(lnl[good] > med, 0.02, -0.02).astype(np.float32)
                srv.close_fit(fit)
                with lock:
                    call_lat.extend(lat)
                    req_lat.append(1e3 * (time.perf_counter() - t_arr))
                    admitted_wait.append(1e3 * (t_adm - t_arr))

        threads = [threading.Thread(target=worker) for _ in range(args.serve_threads)]
        for t in threads:
            t.start()
        for t in threads:
            t.join()
        wall = time.perf_counter() - t0
        st = srv.stats()
        srv.close()
        return {"evals_per_s": round(total_evals / wall, 1), "wall_s": round(wall, 3),
                "call_latency_ms": {"p50": round(float(np.percentile(call_lat, 50)), 3),
                                    "p99": round(float(np.percentile(call_lat, 99)), 3)},
                "request_latency_ms": {"p50": round(float(np.percentile(req_lat, 50)), 3),
                                       "p99": round(float(np.percentile(req_lat, 99)), 3)},
                "admission_wait_ms_p99": round(float(np.percentile(admitted_wait, 99)), 3),
                "launches": int(st["launches"]), "calls": int(st["calls"]),
                "rows_per_launch": round(st["rows"] / max(st["launches"], 1), 1)}

    out = {"requests": len(reqs), "calls": int(sum(q["calls"] for q in reqs)), "evals": int(total_evals),
           "grid": "107 x 12 x 5 x 6000 (FP32 + BF16 copies resident)", "setup_s": round(t_setup, 1),
           "clients": args.serve_threads, "fit_budget_mb": args.serve_budget_mb,
           "what": "latency = submit -> lnL on the host per call; request = arrival -> last call's result; "
                   "requests are dependent chains (each call's rows move with the previous call's lnL)"}
    for prec in ("bf16", "fp32"):
        sat = run(prec, 0.0)
        rate = 0.7 * sat["evals_per_s"] / (total_evals / len(reqs))
        out[prec] = {"saturated": sat, "poisson_0.7": run(prec, rate)}
        out[prec]["poisson_0.7"]["arrival_rate_per_s"] = round(rate, 2)
    out["accuracy_vs_fp64_oracle"] = serving_accuracy(ctx, gid, grid, reqs, models, thetas, okws)
    # like for like: the same mix through plain FP32 batched sed_loglike calls
    sat = run_direct("fp32", 0.0)
    rate = 0.7 * sat["evals_per_s"] / (total_evals / len(reqs))
    out["fp32_plain_batched"] = {"saturated": sat, "poisson_0.7": run_direct("fp32", rate),
                                 "what": "each client calls sed_loglike on its own stream and waits (no server)"}
    out["fp32_plain_batched"]["poisson_0.7"]["arrival_rate_per_s"] = round(rate, 2)
    return out


def bench_sampler(ctx, device, n_fits=2, max_iter=5000):
    """Nested slice sampling of a fit shaped like the paper's JADES benchmark:
    15 NIRCam-like bands and a 22-entry emission-line catalogue, 8 SFH bins, one
    constant [Fe/H], nebular continuum and lines (30-line cube), birth-cloud +
    Kriek & Conroy dust, redshift fixed; 15 sampled columns over a box prior;
    300 live points, 64 replaced per iteration, 40 slice steps per replacement,
    stop at ln(Z_live / Z) < -5.  Data: the model of a true row with 5% noise
    on the bands and 10% on the lines.  Wall time per fit includes every host
    sync of the run."""
    import torch
    import synth

    wl = synth.WORKLOADS["specphot_lines_107x12x6000_b1024"]
    grid = synth.make_grid(**wl.grid_kw, seed=1)
    gid = ctx.load_grid(grid)
    filt = synth.pack_filters(synth.make_filters_nircam_like(6, 9, seed=17))
    n_sfh, nl = 8, len(grid.line_lam)
    blends = [[i] for i in range(0, min(nl, 19))] + [[19, 20], [21, 22, 23], [24, 25]]
    fixed = {"afe": 0.0, "zred": 5.0, "alpha_pow": -1.0}
    kw = dict(use_nebular=1, dust_law=1, use_lines=1, filters=filt, phot_d=np.ones(15), phot_sigma=np.ones(15),
              fixed=fixed)
    truth = synth.make_theta(1, n_sfh, 1, dict(wl.ranges, feh=(-0.7, -0.7)), seed=99)
    truth.update(logmass=np.array([9.3]), tau_pow=np.array([0.4]), diffuse_tau_kc=np.array([0.3]),
                 diffuse_dust_index=np.array([-0.3]), gas_logz=np.array([-0.5]), gas_logu=np.array([-2.5]))
    m0 = ctx.create_model(gid, n_sfh, 30.0, 1, **kw)
    th0 = torch_from(m0.pack(truth), device)
    ph = m0.forward(th0, "fp32")[0].cpu().numpy()[0].astype(np.float64)
    fl = m0.line_fluxes(th0, "fp32").cpu().numpy()[0].astype(np.float64)
    m0.close()
    nz = synth.noise(15 + len(blends), seed=21)
    lf = np.array([fl[b].sum() for b in blends])
    lcat = (blends, lf * (1 + nz[15:] / 10.0), np.abs(lf) / 10.0, None, None)
    kw.update(phot_d=ph * (1 + nz[:15] / 20.0), phot_sigma=np.abs(ph) / 20.0)
    model = ctx.create_model(gid, n_sfh, 30.0, 1, lcat=lcat, **kw)
    lo = np.concatenate([np.zeros(n_sfh), [-2.0, 7.0, 0.0, 0.0, -1.0, -1.3, -4.0]])
    hi = np.concatenate([np.ones(n_sfh), [0.3, 12.0, 2.0, 2.0, 0.4, 0.3, -1.0]])
    assert model.n_param == lo.size
    model.nss(lo, hi, n_live=300, n_replace=64, n_slice_steps=40, max_iter=min(4, max_iter) if n_fits else max_iter,
              seed=1)   # warm-up (the whole run for a profile case)
    fits = []
    for f in range(n_fits):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = model.nss(lo, hi, n_live=300, n_replace=64, n_slice_steps=40, max_iter=max_iter, seed=100 + f)
        dt = time.perf_counter() - t0
        fits.append({"seconds": round(dt, 3), "lnz": round(r["lnz"], 3), "info_h": round(r["info_h"], 3),
                     "n_iter": r["n_iter"], "n_like": int(r["n_like"]), "n_rows": int(r["n_rows"]),
                     "converged": r["converged"], "like_evals_per_s": round(r["n_like"] / dt, 1)})
    model.close()
    return {"model": "15 bands + 22 line-catalogue entries, 8 SFH bins, constant [Fe/H], nebular + lines, "
                     "birth-cloud + KC13 dust, z fixed; 15 sampled columns, box prior",
            "settings": {"n_live": 300, "n_replace": 64, "n_slice_steps": 40, "stop_dlnz": -5.0,
                         "precision": "fp32"},
            "fits": fits,
            "seconds_per_fit_median": round(float(np.median([f["seconds"] for f in fits])), 3) if fits else None,
            "paper_context": "4.0 min per fit and ~1.4e6 likelihood evaluations on one A100 (JADES 170891, "
                             "15 bands + 22 lines; other model and hardware)"}


def serving_accuracy(ctx, gid, grid, reqs, models, thetas, okws, n_req=8, n_rows=16):
    """Errors of the served lnL against the FP64 oracle on the mix: the first
    n_rows live points of the first n_req requests (photometric and
    spectro-photometric fits, with and without [a/Fe]), each request's rows
    submitted through a server of each precision."""
    import oracle
    from paper_2609_30145_gb300 import Server

    sel = list(range(min(n_req, len(reqs))))
    refs, orcs = [], []
    for i in sel:
        okw = okws[i]
        orc = oracle.Oracle(grid=grid, n_sfh=okw["n_sfh"], zf=okw["zf"], zmode=okw["zmode"], use_afe=okw["use_afe"],
                            dust_law=okw["dust_law"], filters=okw["filters"], phot_d=okw["phot_d"],
                            phot_sigma=okw["phot_sigma"], spec_lam=okw.get("spec_lam"), spec_d=okw.get("spec_d"),
                            spec_sigma=okw.get("spec_sigma"), lsf_mode=okw.get("lsf_mode", 0),
                            lsf_value=okw.get("lsf_value"), sigma_gal_kms=okw.get("sigma_gal_kms", 0.0),
                            z_ref=okw.get("z_ref", 0.0))
        th = thetas[i][:n_rows]
        refs.append(orc.eval(th.astype(np.float64)))
        orcs.append(orc)
    out = {"requests": len(sel), "rows_per_request": n_rows,
           "what": "first live points of the first requests of the mix, served, against the FP64 oracle"}
    for prec in ("fp32", "bf16"):
        srv = Server(ctx, gid, models[0], precision=prec, max_launch_rows=8192, n_slots=1)
        rel, ab, match = [], [], True
        for j, i in enumerate(sel):
            th = np.ascontiguousarray(thetas[i][:n_rows])
            fit = srv.open_fit(models[i], th.shape[0])
            lnl, st, _ = srv.wait(srv.submit(fit, th), th.shape[0])
            srv.close_fit(fit)
            ref = refs[j]
            match &= bool(np.array_equal(st, ref["status"]))
            ok = ref["status"] == 0
            c = norm_const(orcs[j])
            lr = ref["lnl"][ok]
            d = np.abs(lnl[ok] - lr)
            rel.append(d / np.maximum(np.abs(lr), (c - lr) + abs(c)))
            ab.append(d)
        srv.close()
        out[prec] = {"status_match": match, "rows": int(sum(a.size for a in ab)),
                     "lnl_err_over_term_scale": _q(np.concatenate(rel)), "lnl_abs_err": _q(np.concatenate(ab))}
    return out


def torch_from(a, device):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(device)


def kernel_source_sha16(path="paper_2609_30145_gb300/csrc/k_contract_tc.cu"):
    import hashlib
    with open(os.path.join(ROOT, path), "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()[:16]


def read_traffic():
    """DRAM bytes per launch of the 3xTF32 contraction from the committed ncu
    summary, if it was taken on the current kernel source (its
    kernel_source_sha16 line), else None."""
    p = os.path.join(ROOT, "profiles", "k_contract_tc_phot_b1024.md")
    if not os.path.exists(p):
        return None
    vals = {}
    for line in open(p):
        if ":" in line:
            k, v = line.split(":", 1)
            vals[k.strip()] = v.strip()
    if vals.get("kernel_source_sha16") != kernel_source_sha16():
        return None
    try:
        return float(vals["traffic_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


# --------------------------------------------------------------------------- ncu cases
def profile_case(which):
    """Small cases of the hot path for ncu captures (the commands in profiles/).

    phot: the paper-scale photometric batch (107 x 12 x 6000 grid, 120 bins,
    20 filters, 1024 rows): three FP32 (3xTF32) sed_loglike calls, then one
    BF16, one FP8 and one FP32-SIMT call, then one FP32 sed_loglike_grad;
    about 1 GB of device memory.  Launch order of k_contract_tc: 3xTF32 x3,
    BF16, FP8, adjoint.
    specphot: the [a/Fe] spectro-photometric workload (107 x 12 x 5 x 6000
    grid, 1500-pixel spectrum + 20 filters) at 512 rows: one FP32 sed_loglike,
    then two FP32 sed_loglike_grad calls.
    calib: the same with the marginalised 13-term calibration polynomial.
    nss: 30 iterations of nested slice sampling of the JADES-like fit of the
    sampler leg (300 live points, 64 replaced, 40 slice steps)."""
    import torch
    import synth

    torch.cuda.set_device(0)
    device = torch.device("cuda", 0)
    import __graft_entry__
    __graft_entry__.build()
    from paper_2609_30145_gb300 import Context

    ctx = Context(0)
    if which == "nss":
        bench_sampler(ctx, device, n_fits=0, max_iter=30)
        torch.cuda.synchronize()
        ctx.close()
        print("ok")
        return
    if which == "phot":
        w, _, _, m, theta, _ = build_workload(WORKLOAD, ctx, 5, device)
        t = torch.from_numpy(theta).to(device)
        for prec in ["fp32", "fp32", "fp32", "bf16", "fp8", "fp32_simt"]:
            m.loglike(t, prec)
        m.loglike_grad(t, "fp32")
    else:
        wname = CALIB_WORKLOAD if which == "calib" else GRAD_WORKLOAD
        w, _, _, m, theta, _ = build_workload(wname, ctx, 5, device)
        t = torch.from_numpy(theta[:512]).to(device)
        m.loglike(t, "fp32")
        m.loglike_grad(t, "fp32")
        m.loglike_grad(t, "fp32")
    torch.cuda.synchronize()
    ctx.close()
    print("ok")


# --------------------------------------------------------------------------- CPU baseline / reference
def _oracle_for(w, grid, filt, data):
    import oracle

    oracle.build()
    return oracle.Oracle(grid=grid, n_sfh=w.n_sfh, zf=w.zf, zmode=w.zmode, use_afe=w.use_afe,
                         use_nebular=w.use_nebular, dust_law=w.dust_law, filters=filt,
                         phot_d=data[0], phot_sigma=data[1])


def cpu_baseline(w, grid, filt, data, theta32, gpu_res, seconds):
    orc = _oracle_for(w, grid, filt, data)
    cores = os.cpu_count() or 1
    th64 = theta32.astype(np.float64)
    rows, evals, t_used, chunk = 0, 0, 0.0, 64
    ref_lnl, ref_ph, ref_st = [], [], []
    # one pass over the batch for the accuracy comparison, then repeated passes
    # until about `seconds` of CPU work have been timed
    while t_used < seconds:
        lo = evals % th64.shape[0]
        sl = slice(lo, min(lo + chunk, th64.shape[0]))
        t0 = time.perf_counter()
        r = orc.eval(th64[sl], nthreads=cores)
        t_used += time.perf_counter() - t0
        evals += sl.stop - sl.start
        if rows < th64.shape[0] and sl.start == rows:
            ref_lnl.append(r["lnl"]); ref_ph.append(r["phot"]); ref_st.append(r["status"])
            rows = sl.stop
    cb = {"value": round(evals / t_used, 2), "unit": "evals/s", "cores": cores, "kind": "oracle",
          "sample": f"{evals} evaluations cycling over the {th64.shape[0]} parameter rows of the workload, "
                    f"FP64 C oracle, OpenMP over rows ({t_used:.1f} s)"}
    ref_lnl, ref_ph, ref_st = np.concatenate(ref_lnl), np.concatenate(ref_ph), np.concatenate(ref_st)
    ok = ref_st == 0
    c = -0.5 * np.sum(np.log(2 * np.pi * data[1] ** 2))
    scale = np.maximum(np.abs(ref_lnl[ok]), (c - ref_lnl[ok]) + abs(c))
    acc = {}
    for vp, (l, s, ph) in gpu_res.items():
        l, ph = l[:rows][ok], ph[:rows][ok]
        rp = ref_ph[ok]
        good = rp > 1e-6 * np.abs(rp).max(axis=1, keepdims=True)
        e_f = np.abs(ph[good] - rp[good]) / rp[good]
        e_l = np.abs(l - ref_lnl[ok]) / scale
        e_l_raw = np.abs(l - ref_lnl[ok]) / np.abs(ref_lnl[ok])
        acc[vp] = {"flux_rel_err": {"median": float(np.median(e_f)), "p99": float(np.percentile(e_f, 99)),
                                    "max": float(e_f.max())},
                   "lnl_err_over_term_scale": {"median": float(np.median(e_l)), "p99": float(np.percentile(e_l, 99)),
                                               "max": float(e_l.max())},
                   "lnl_rel_err": {"median": float(np.median(e_l_raw)), "max": float(e_l_raw.max())},
                   "status_match": bool(np.array_equal(s[:rows], ref_st)), "rows": int(ok.sum())}
    return cb, acc


def run_reference(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import synth
    import oracle

    w = synth.WORKLOADS[args.workload]
    grid = synth.make_grid(**w.grid_kw, seed=1)
    filt = synth.pack_filters(synth.workload_filters(w))
    nb = len(filt[0])
    orc = oracle.Oracle(grid=grid, n_sfh=w.n_sfh, zf=w.zf, zmode=w.zmode, use_afe=w.use_afe,
                        use_nebular=w.use_nebular, dust_law=w.dust_law, filters=filt,
                        phot_d=np.ones(nb), phot_sigma=np.ones(nb))
    th_true = oracle.pack_theta(synth.make_theta(1, w.n_sfh, w.zmode, w.ranges, seed=99), w.n_sfh, w.zmode)
    th_true[0, w.n_sfh + (w.n_sfh if w.zmode == 0 else 1) + 2] = 2.0
    ph = orc.eval(th_true)["phot"][0]
    nz = synth.noise(nb, seed=5)
    orc.set_data(phot_d=ph * (1 + nz / 20.0), phot_sigma=np.abs(ph) / 20.0)
    theta = oracle.pack_theta(synth.make_theta(w.batch, w.n_sfh, w.zmode, w.ranges, seed=4), w.n_sfh,
                              w.zmode).astype(np.float32).astype(np.float64)
    cores = os.cpu_count() or 1
    sample = 64
    for i in range(args.warmup):
        orc.eval(theta[:sample], nthreads=cores)
    ts = []
    for i in range(args.steps):
        sl = slice((i * sample) % w.batch, (i * sample) % w.batch + sample)
        t0 = time.perf_counter()
        orc.eval(theta[sl], nthreads=cores)
        ts.append(time.perf_counter() - t0)
    value = sample * args.steps / sum(ts)
    out = {"impl": "reference", "metric": METRIC, "value": round(value, 2), "unit": "evals/s",
           "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": round(1e3 * sum(ts) / args.steps, 3), "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic (same seeded workload as the GPU arm)",
           "config": {"workload": w.name, "batch_per_step": sample,
                      "what": "FP64 C oracle (plain loops, OpenMP over rows) on the host cores; each step a "
                              f"{sample}-row sample of the {w.batch}-row workload"},
           "cpu_baseline": {"kind": "oracle", "cores": cores, "value": round(value, 2), "unit": "evals/s",
                            "sample": f"{args.steps} steps x {sample} rows"},
           "e2e": {"value": round(value, 2), "unit": "evals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def relaunch_under_torchrun(n):
    """`bench.py --gpus N` started as a single process: start it again under
    torchrun with one rank per GPU (the driver's own N > 1 launch sets
    WORLD_SIZE and never comes here)."""
    import socket

    sk = socket.socket()
    sk.bind(("127.0.0.1", 0))
    port = sk.getsockname()[1]
    sk.close()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", f"--nproc-per-node={n}",
           "--master-addr=127.0.0.1", f"--master-port={port}", os.path.abspath(__file__)] + sys.argv[1:]
    return subprocess.call(cmd)


def main():
    args = parse()
    if args.profile_case:
        profile_case(args.profile_case)
        return
    if args.gpus > 1 and "WORLD_SIZE" not in os.environ:
        sys.exit(relaunch_under_torchrun(args.gpus))
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
