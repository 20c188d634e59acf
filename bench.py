#!/usr/bin/env python
"""Benchmark of the shifted-system TEM hot path on one GB300.

Workload: 46^3-cube Kuhn box (700,534 edges, 662,446 unknowns), two seeded
conductive blocks (0.1, 0.3 S/m) in 0.01 S/m under 1e-8 S/m air, 32 square
loops, 128 surface receivers, 40 times, 10 conjugate pole pairs.  Synthetic
data: the forward of the true model plus 3% Gaussian noise; the Gauss-Newton
step starts from the 0.01 S/m half-space (also the reference model).

Metric: J.v + J^T.w pairs per second (one LSQR iteration = one pair, all
10 poles x 32 transmitters, refinement included), with the factor time of
all shifts reported beside it.  A step is one LSQR iteration of the
Gauss-Newton system at the factored start model; the factor (median of 5)
and the forward are timed before the steps.  Refined FP32 (headline: floored
complex-float factors, 3 corrections per forward and J.v solve and 1 per
adjoint solve, each with the gradient-space correction) and FP64 are
measured on the same GPU, and the refined outputs are checked against the
FP64 path's.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
Under torchrun (N > 1) every rank runs an independent replica (the path is
not sharded across GPUs); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

CONFIG = 4
LAMBDA = 10.0
N_LSQR_GN = 30          # LSQR iterations of one Gauss-Newton iteration (configuration)
def _hbm_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"])
    except Exception:
        return 6800.0   # fallback figure for this GPU type


HBM_PEAK_GBS = _hbm_peak()
METRIC = "J.v+J^T.w pairs/s and factor time at 700k DoF, refined FP32 vs FP64, same GPU"
BWD21_TRAFFIC_RATIO = 1.07   # DRAM bytes / factor bytes of the BWD21 product (ncu, 24^3 box)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64 comparison leg")
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle CPU baseline")
    ap.add_argument("--no-kscale", action="store_true", help="skip the time-channel scaling study")
    ap.add_argument("--levels", action="store_true",
                    help="instead of the bench line: per-level times and rates of the four front-product "
                         "classes in one J.v (CUDA events per class and tree level)")
    ap.add_argument("--c5", action="store_true",
                    help="instead of the bench line: configuration C5, 48 uneven surveys, forward + J^T.w each, "
                         "one CUDA graph per wave of models")
    ap.add_argument("--c5-budget-gb", type=float, default=110.0,
                    help="device memory per C5 wave (estimated from the factor entries)")
    ap.add_argument("--configs", action="store_true",
                    help="instead of the bench line: factor / forward / pair times of C1-C3 on the GPU in both "
                         "precisions and of the oracle on this host for C1-C2")
    ap.add_argument("--peaks", action="store_true",
                    help="instead of the bench line: cuBLAS FP64, FP32 and TF32 GEMM rates (torch.matmul)")
    ap.add_argument("--gn", type=int, default=0, metavar="ITERS",
                    help="instead of the bench line: a Gauss-Newton inversion of the workload's synthetic data "
                         "from the half-space start model, ITERS iterations (Section 3.3 loop)")
    ap.add_argument("--n", type=int, default=46,
                    help="cubes per side (46 = the 700k-DoF workload; smaller only for profiling captures)")
    return ap.parse_args()


# ---------------------------------------------------------------------------
class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons.  The sampler is
    started before the warm-up (its start-up is slow) and only the samples
    stamped inside [mark_begin, mark_end] are kept."""

    Q = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, local_rank):
        vis = os.environ.get("CUDA_VISIBLE_DEVICES")
        ids = [x for x in vis.split(",") if x.strip()] if vis else []
        self.index = ids[local_rank].strip() if local_rank < len(ids) else str(local_rank)
        self.proc = None
        self.path = None
        self.t0 = self.t1 = None

    def mark_begin(self):
        self.t0 = time.time()

    def mark_end(self):
        self.t1 = time.time()

    def wait_first_sample(self, timeout=30.0):
        end = time.time() + timeout
        while self.proc is not None and time.time() < end:
            try:
                if os.path.getsize(self.path) > 0:
                    return
            except OSError:
                return
            time.sleep(0.05)

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        self.proc.wait()
        import datetime
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 10:
                continue
            try:
                ts = datetime.datetime.strptime(f[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
            except ValueError:
                ts = None
            if ts is not None and self.t0 is not None and self.t1 is not None and not (
                    self.t0 - 0.25 <= ts <= self.t1 + 0.25):
                continue
            try:
                sm.append(float(f[2]))
                smax.append(float(f[3]))
            except ValueError:
                continue
            for nm, val in zip(names, f[6:10]):
                if val.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def synthetic(tem, s, xi, al, torch):
    """Observed data: forward of the true model (refined FP32 library call) + 3% noise."""
    import numpy as np
    mdl = tem.Model(s.xyz, s.tets, s.sigma, s.is_param, s.loops, s.rx, xi, al,
                    precision=tem.TEM_FP32_REFINED)
    m_true = torch.as_tensor(s.log_sigma(), device="cuda")
    mdl.factor(m_true)
    d_true = mdl.forward().cpu().numpy()
    rng = np.random.default_rng(19951 + CONFIG)
    eps_a = 1e-4 * np.abs(d_true).reshape(d_true.shape[0], -1).max(axis=1)[:, None, None]
    sd = 0.03 * np.abs(d_true) + eps_a
    d_obs = d_true + sd * rng.standard_normal(d_true.shape)
    wd = 1.0 / (0.03 * np.abs(d_obs) + eps_a)
    return mdl, d_obs, wd


def k_scaling(torch, mdl, n_param, counts=(10, 40, 160, 640)):
    """Forward and J.v + J^T.w pair time against the number of time channels K
    (Section 2.3: the solves do not depend on the times, only the residue
    sums do).  For each K the residues of the fixed poles are fitted on the
    device (tem_times, log-spaced times in [1e-5, 1e-2] s); the factors stay."""
    import numpy as np
    gen = torch.Generator(device="cuda").manual_seed(4321)
    v = torch.randn(n_param, dtype=torch.float64, device="cuda", generator=gen)
    res = {"K": [], "fit_ms": [], "forward_ms": [], "pair_ms": []}
    for K in counts:
        t0 = time.perf_counter()
        mdl.set_times(np.logspace(-5, -2, K))
        fit_ms = 1e3 * (time.perf_counter() - t0)
        fw = statistics.median([timed(torch, lambda: mdl.forward())[0] for _ in range(3)])
        w = torch.randn(*mdl.shape, dtype=torch.float64, device="cuda", generator=gen)
        pr = statistics.median([timed(torch, lambda: (mdl.jvp(v), mdl.jtvp(w)))[0] for _ in range(3)])
        for k, x in (("K", K), ("fit_ms", fit_ms), ("forward_ms", fw), ("pair_ms", pr)):
            res[k].append(round(x, 2) if k != "K" else x)
    res["note"] = ("factors of the 40-time model kept; per K: residues fitted on the device (host clock, "
                   "includes the call's synchronisations), forward and pair medians of 3 (CUDA events)")
    return res


def max_over_ranks(torch, dist, values, device):
    """Each timing's largest value over all ranks (unchanged on one rank)."""
    if dist is None:
        return [float(v) for v in values]
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.tolist()]


def whole_job_rate(units_per_rank, world, ms):
    """Units processed by all ranks per second, over the slowest rank's time."""
    return units_per_rank * world / (ms * 1e-3)


def timed(torch, fn):
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    out = fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1), out


def run_ours(args):
    import numpy as np
    import torch
    from paper_2605_19951_gb300 import inputs, tem

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()

    s = inputs.make_config(CONFIG, n=args.n)
    xi, al = inputs.load_rational(s.m, s.times)
    mdl, d_obs_h, wd_h = synthetic(tem, s, xi, al, torch)
    info = mdl.info()
    m0 = torch.as_tensor(np.log(s.sigma_start[s.is_param.astype(bool)]), device="cuda")
    d_obs = torch.as_tensor(d_obs_h, device="cuda")
    wd = torch.as_tensor(wd_h, device="cuda")

    # factor time of all shifts (median of 5) and the forward at the start model
    factor_ms = statistics.median([timed(torch, lambda: mdl.factor(m0))[0] for _ in range(5)])
    forward_ms, _ = timed(torch, lambda: mdl.forward())

    # which kernel class dominates a pair (one untimed profiling pass per class)
    per_class = {}
    for cls in ("fwd", "fwd21", "bwd", "bwd_upd", "residual", "refine_vec", "jacobian", "nodal"):
        tem.tem_set_profiling(mdl.ctx, cls)
        mdl.lsqr(d_obs, wd, m0, LAMBDA, 1)
        per_class[cls] = tem.tem_kernel_time(mdl.ctx)
    tem.tem_set_profiling(mdl.ctx, None)
    dom = max(("fwd", "fwd21", "bwd", "bwd_upd"), key=lambda c: per_class[c][0])

    # warm-up, then K timed LSQR iterations in one device-resident LSQR call
    clocks = Clocks(local)
    clocks.start()
    clocks.wait_first_sample()
    for _ in range(args.warmup):
        mdl.lsqr(d_obs, wd, m0, LAMBDA, 1)
    tem.tem_set_profiling(mdl.ctx, dom)
    barrier()
    torch.cuda.synchronize()
    l0 = tem.tem_launch_count()
    torch.cuda.nvtx.range_push("tem_timed")
    clocks.mark_begin()
    t_ms, _ = timed(torch, lambda: mdl.lsqr(d_obs, wd, m0, LAMBDA, args.steps))
    clocks.mark_end()
    torch.cuda.nvtx.range_pop()
    launches = tem.tem_launch_count() - l0
    ck = clocks.stop()
    barrier()
    dom_ms, dom_launches = tem.tem_kernel_time(mdl.ctx)
    tem.tem_set_profiling(mdl.ctx, None)
    t_ms, = max_over_ranks(torch, dist, [t_ms], "cuda")

    # end to end through the public API: pinned host inputs, result read back
    d_obs_p = torch.as_tensor(d_obs_h).pin_memory()
    wd_p = torch.as_tensor(wd_h).pin_memory()
    m0_p = m0.cpu().pin_memory()
    dm_p = torch.empty(info["n_param"], dtype=torch.float64).pin_memory()

    def e2e():
        a = d_obs_p.to("cuda", non_blocking=True)
        b = wd_p.to("cuda", non_blocking=True)
        c = m0_p.to("cuda", non_blocking=True)
        dm = mdl.lsqr(a, b, c, LAMBDA, args.steps)
        dm_p.copy_(dm, non_blocking=True)
        return dm_p

    e2e_ms, _ = timed(torch, e2e)
    e2e_ms, = max_over_ranks(torch, dist, [e2e_ms], "cuda")
    # one Gauss-Newton iteration measured as a whole: factor + forward + a 30-iteration LSQR call
    gn_ms, _ = timed(torch, lambda: (mdl.factor(m0), mdl.forward(), mdl.lsqr(d_obs, wd, m0, LAMBDA, N_LSQR_GN)))
    h2d = (d_obs_p.numel() + wd_p.numel() + m0_p.numel()) * 8
    d2h = dm_p.numel() * 8

    # roofline of the dominant kernel class: the front products stream the
    # factor once per sweep, so they are bound by HBM; algorithmic bytes = the
    # factor entries the class applies (8 bytes each) x poles x sweeps
    N, m, nrhs = info["n_dof"], info["m"], info["n_tx"]
    refine, refine_adj = info["refine_steps"], info["refine_steps_adjoint"]
    # one LSQR call of K iterations: its start-up J^T.w, then K x (J.v + J^T.w)
    sweeps = args.steps * (1 + refine) + (args.steps + 1) * (1 + refine_adj)
    l11 = info["nnz_l11"]                         # pivot blocks: T11 = L11^-1, lower triangle
    l21 = info["nnz_l"] - info["nnz_l11"]
    entries = {"fwd": l11, "fwd21": l21, "bwd": l11, "bwd_upd": l21}[dom]
    alg_bytes = 8.0 * entries * m * sweeps
    achieved = alg_bytes / (dom_ms * 1e-3) / 1e9
    # DRAM traffic per launch: ncu (dram__bytes_read.sum + dram__bytes_write.sum) on the 24^3 box's
    # BWD21 launches of this kernel read 1.07x their factor bytes (the gathered B rows and tile padding
    # are the excess); the full-size launch is scaled by its factor bytes (entries x 8 B x poles)
    traffic = round(BWD21_TRAFFIC_RATIO * alg_bytes / max(dom_launches, 1)) if dom == "bwd_upd" else None
    roof = {"kernel": "k_tc_kint<%s>" % {"fwd": "TRI_F", "fwd21": "FWD21", "bwd": "TRI_B", "bwd_upd": "BWD21"}[dom],
            "bound": "hbm", "achieved": round(achieved, 1), "peak": HBM_PEAK_GBS, "unit": "GB/s",
            "frac": round(achieved / HBM_PEAK_GBS, 4), "traffic": traffic,
            "launches": dom_launches, "avg_launch_us": round(1e3 * dom_ms / max(dom_launches, 1), 2),
            "alg_bytes_per_launch": round(alg_bytes / max(dom_launches, 1)),
            "share_of_step": round(dom_ms / t_ms, 3),
            "peak_note": "measured HBM copy bandwidth (MEASURED_PEAKS.json hbm_gbs), of measured",
            "bytes_note": "factor entries of the class (c64) x poles x sweeps; B rows and outputs (<3%) not counted",
            "traffic_note": "DRAM bytes per launch: ncu on the 24^3 box (BWD21 read 1.07x its factor bytes), "
                            "scaled to this launch's factor bytes"}

    pairs_per_s = whole_job_rate(args.steps, world, t_ms)
    out = {
        "metric": METRIC, "value": round(pairs_per_s, 4), "unit": "pairs/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(t_ms / args.steps, 2),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "c64 factor/solves, double-float (FP32 pair) refinement residual, f64 residue sums and LSQR",
        "data": "synthetic (seeded model, forward of the true model + 3% noise)",
        "config": {"workload": f"{s.n}^3 Kuhn box, {N} DoF, 10 pole pairs, 32 loops, 128 rx, 40 times",
                   "precision": "fp32-refined", "refine_steps": refine, "refine_steps_adjoint": refine_adj,
                   "gradient_space_correction": bool(info["nodal"]), "nodal_dof": info["n_nodes"],
                   "l2": "inputs larger than L2 (factors %.1f GB per sweep)" % (info["nnz_l"] * m * 8 / 1e9),
                   "step": "one LSQR iteration = one J.v + one J^T.w over all poles x transmitters"},
        "factor_s": round(factor_ms / 1e3, 3), "factor_note": "median of 5 tem_factor calls (all 10 shifts)",
        "forward_s": round(forward_ms / 1e3, 3),
        "gn_iteration_s": round((factor_ms + forward_ms + N_LSQR_GN * t_ms / args.steps) / 1e3, 2),
        "gn_iteration_note": "factor + forward + 30 LSQR pairs at the measured rates (linear model, Fig. 10)",
        "gn_iteration_measured_s": round(gn_ms / 1e3, 2),
        "gn_iteration_measured_note": "one tem_factor + tem_forward + tem_lsqr(30 iterations) timed as a whole "
                                      "(CUDA events; includes LSQR's start-up J^T.w)",
        "roofline": roof,
        "e2e": {"value": round(whole_job_rate(args.steps, world, e2e_ms), 4), "unit": "pairs/s",
                "h2d_bytes_per_step": h2d // args.steps, "d2h_bytes_per_step": d2h // args.steps},
        "gpu_launches": int(launches), "clocks": ck,
        "per_class_ms_lsqr_call": {k: round(v[0], 2) for k, v in per_class.items()},
    }
    # accuracy check against the FP64 path on the same workload (seeded J.v and J^T.w vectors)
    gen = torch.Generator(device="cuda").manual_seed(1234)
    vv = torch.randn(info["n_param"], dtype=torch.float64, device="cuda", generator=gen)
    ww = torch.randn(*mdl.shape, dtype=torch.float64, device="cuda", generator=gen)
    acc32 = (mdl.forward().cpu().numpy(), mdl.jvp(vv).cpu().numpy(), mdl.jtvp(ww).cpu().numpy())
    if not args.no_kscale:
        out["k_scaling"] = k_scaling(torch, mdl, info["n_param"])
    mdl.close()
    del mdl
    torch.cuda.empty_cache()

    if not args.no_fp64:
        md = tem.Model(s.xyz, s.tets, s.sigma, s.is_param, s.loops, s.rx, xi, al, precision=tem.TEM_FP64)
        f64_factor, _ = timed(torch, lambda: md.factor(m0))
        fw = [timed(torch, lambda: md.forward()) for _ in range(5)]
        pr = [timed(torch, lambda: (md.jvp(vv), md.jtvp(ww))) for _ in range(5)]
        f64_fwd = statistics.median([t for t, _ in fw])
        f64_pair = statistics.median([t for t, _ in pr])
        d64 = fw[-1][1].cpu().numpy()
        jv64, jtw64 = pr[-1][1][0].cpu().numpy(), pr[-1][1][1].cpu().numpy()

        def floored(a, ref, floor=1e-4):   # per channel, floored at 1e-4 of its peak over time
            peak = np.abs(ref).max(axis=2, keepdims=True)
            return float((np.abs(a - ref) / np.maximum(np.abs(ref), floor * peak)).max())
        out["fp64"] = {"factor_s": round(f64_factor / 1e3, 2), "forward_s": round(f64_fwd / 1e3, 3),
                       "pair_s": round(f64_pair / 1e3, 3), "pairs_per_s": round(1e3 / f64_pair, 4),
                       "gn_iteration_s": round((f64_factor + f64_fwd + N_LSQR_GN * f64_pair) / 1e3, 1),
                       "note": "one factor (59 s of FP64 fronts; not repeated), forward and J.v + J^T.w pair "
                               "medians of 5, CUDA events"}
        out["fp32r_vs_fp64"] = {"data": floored(acc32[0], d64), "jv": floored(acc32[1], jv64),
                                "jtw": float(np.linalg.norm(acc32[2] - jtw64) / np.linalg.norm(jtw64)),
                                "note": "refined FP32 against the FP64 path at the start model: data and J.v "
                                        "max per-channel error floored at 1e-4 of the channel's peak over time, "
                                        "J^T.w relative 2-norm"}
        md.close()
        del md
        torch.cuda.empty_cache()

    if rank == 0 and world == 1 and not args.no_cpu:
        out["cpu_baseline"] = cpu_baseline(steps=1, n=args.n)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def cpu_baseline(steps=1, warmup=0, n=46):
    """The oracle as it stands, on this host, on a bounded sample: `steps`
    J.v + J^T.w pairs of the 20^3 box (8 poles x 4 loops, poles on parallel
    host threads) after its factorisation, scaled to the 46^3 workload by the
    oracle's own factor entries x right-hand sides x poles (its symbolic
    analysis of both meshes; the solves dominate an oracle pair)."""
    import numpy as np
    from oracle.fem import FEModel
    from oracle.sparse_ldlt import nested_dissection, symbolic_nnz
    from oracle.tem import Oracle
    from paper_2605_19951_gb300 import inputs

    s2 = inputs.make_config(2)
    xi2, al2 = inputs.load_rational(s2.m, s2.times)
    o = Oracle(s2.xyz, s2.tets, s2.sigma, s2.is_param, s2.loops, s2.rx, xi2, al2)
    o.set_model(s2.log_sigma())
    rng = np.random.default_rng(7)
    v = rng.standard_normal(s2.n_param)
    w = rng.standard_normal(o.forward_shape)
    for _ in range(warmup):
        o.jvp(v)
        o.jtvp(w)
    t0 = time.perf_counter()
    for _ in range(steps):
        o.jvp(v)
        o.jtvp(w)
    t_pair = (time.perf_counter() - t0) / steps
    s4 = inputs.make_config(CONFIG, n=n)
    fe4 = FEModel(s4.xyz, s4.tets)
    perm4 = nested_dissection(fe4.tdof, fe4.N, fe4.xyz[fe4.tv].mean(axis=1))
    nnz2, nnz4 = o.lu[0].nnz_L, symbolic_nnz(fe4.K, perm4)
    scale = (nnz4 * s4.m * len(s4.loops)) / (nnz2 * s2.m * len(s2.loops))
    return {"value": round(1.0 / (t_pair * scale), 6), "unit": "pairs/s", "cores": int(o.threads),
            "nproc": os.cpu_count(), "kind": "oracle",
            "sample": f"{steps} oracle pair(s) of the 20^3 box measured ({t_pair:.2f} s each, {o.threads} threads, "
                      f"one per pole), scaled to the {n}^3 workload by the oracle's nnz(L) x RHS x poles "
                      f"({nnz4:.3g} / {nnz2:.3g} entries, x{scale:.0f})",
            "pair_s_sample": round(t_pair, 3), "scale": round(scale, 1), "scale_source": "oracle symbolic nnz(L)",
            "sample_config": "20^3 Kuhn box (52,460 DoF), 8 poles, 4 loops, 32 rx, 24 times",
            "workload_dof": int(fe4.N)}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    t0 = time.perf_counter()
    cb = cpu_baseline(steps=args.steps, warmup=args.warmup, n=args.n)
    n, N = args.n, cb["workload_dof"]
    per_pair_s = 1.0 / cb["value"]
    out = {"metric": METRIC, "value": cb["value"], "unit": "pairs/s", "n_gpus": 1, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": round(per_pair_s * 1e3, 1), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": f"{n}^3 Kuhn box, {N} DoF, 10 pole pairs, 32 loops, 128 rx, 40 times",
                      "sample": cb["sample"], "measured_on": cb["sample_config"], "extrapolated": True},
           "impl": "reference", "cpu_baseline": cb,
           "e2e": {"value": cb["value"], "unit": "pairs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
           "wall_s": round(time.perf_counter() - t0, 1)}
    print(json.dumps(out), flush=True)


def run_levels(args):
    """One J.v on the workload, each front-product class timed level by level
    (tem_set_profiling with a tree level); rate = the level's factor entries
    of that class x 8 B x poles x launches / time."""
    import numpy as np
    import torch
    from paper_2605_19951_gb300 import inputs, tem
    torch.cuda.set_device(0)
    s = inputs.make_config(CONFIG, n=args.n)
    xi, al = inputs.load_rational(s.m, s.times)
    mdl = tem.Model(s.xyz, s.tets, s.sigma, s.is_param, s.loops, s.rx, xi, al, precision=tem.TEM_FP32_REFINED)
    m0 = torch.as_tensor(s.log_sigma(), device="cuda")
    mdl.factor(m0)
    mdl.forward()
    lv = tem.tem_level_info(mdl.ctx)
    m = mdl.info()["m"]
    gen = torch.Generator(device="cuda").manual_seed(99)
    v = torch.randn(s.n_param, dtype=torch.float64, device="cuda", generator=gen)
    for _ in range(2):
        mdl.jvp(v)
    names = {"fwd": "TRI_F", "fwd21": "FWD21", "bwd_upd": "BWD21", "bwd": "TRI_B"}
    out = {"workload": f"{s.n}^3 Kuhn box, {mdl.info()['n_dof']} DoF, 10 pole pairs, 32 loops",
           "call": "one tem_jvp (forward + 3 corrections = 4 sweep pairs)", "levels": []}
    for h in range(lv.shape[0]):
        row = {"level": h, "fronts": int(lv[h, 0]), "l11_entries": int(lv[h, 1]), "l21_entries": int(lv[h, 2]),
               "max_k": int(lv[h, 3])}
        for cls, name in names.items():
            tem.tem_set_profiling(mdl.ctx, tem.KERNEL_CLASSES[cls] + 64 * (h + 1))
            mdl.jvp(v)
            ms, nl = tem.tem_kernel_time(mdl.ctx)
            ent = lv[h, 1] if cls in ("fwd", "bwd") else lv[h, 2]
            row[name + "_ms"] = round(ms, 3)
            row[name + "_GBps"] = round(8.0 * ent * m * nl / (ms * 1e-3) / 1e9, 1) if ms > 0 and ent > 0 else None
        out["levels"].append(row)
    tem.tem_set_profiling(mdl.ctx, None)
    mdl.close()
    print(json.dumps(out), flush=True)


def run_c5(args):
    """Configuration C5: 48 independent surveys on meshes of 12..28 cubes per
    side (seeded), each with its own log-normal conductivity and 2..8 loops;
    per survey one forward and one J^T.w with seeded w, refined FP32.  The
    surveys are issued together by tem_batch on their own streams and the
    whole call is captured into one CUDA graph per wave; waves are filled in
    order of size up to a device-memory budget estimated from each survey's
    factor entries.  Reported: the graph replays (median of 3 per wave, CUDA
    events) against issuing the same calls without a graph."""
    import numpy as np
    import torch
    from paper_2605_19951_gb300 import batch, inputs, tem
    torch.cuda.set_device(0)
    n_models = 48
    surveys = [inputs.make_c5_model(i) for i in range(n_models)]
    xi, al = inputs.load_rational(8, inputs.times_log(24))
    est = []
    for s in surveys:   # factor entries from the host analysis alone (no numeric storage)
        ctx = tem.tem_create(tem.TEM_FP32_REFINED)
        try:
            tem.tem_mesh(ctx, s.xyz, s.tets, s.sigma, s.is_param)
            # device bytes of a refined-FP32 context at C4 were 4.3x its c64 factor (row copies,
            # update arena, vectors): 4.5 x leaves a margin
            est.append(4.5 * 8.0 * 8 * tem.tem_info(ctx)["nnz_l"])
        finally:
            tem.tem_destroy(ctx)
    order = sorted(range(n_models), key=lambda i: surveys[i].n)
    waves, cur, used = [], [], 0.0
    for i in order:
        if cur and used + est[i] > args.c5_budget_gb * 1e9:
            waves.append(cur)
            cur, used = [], 0.0
        cur.append(i)
        used += est[i]
    waves.append(cur)
    rng = np.random.default_rng(19951 + 5)
    graph_ms, eager_ms, dof = [], [], 0

    def ev(fn):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record()
        fn()
        b.record()
        torch.cuda.synchronize()
        return a.elapsed_time(b)
    for wv in waves:
        sv = [surveys[i] for i in wv]
        b = batch.Batch(sv, xi, al)
        try:
            logs = [torch.as_tensor(s.log_sigma(), device="cuda") for s in sv]
            ws = [torch.as_tensor(rng.standard_normal((len(s.loops), len(s.rx), len(s.times))), device="cuda")
                  for s in sv]
            b.run(logs, ws)                                   # allocations
            eager_ms.append(statistics.median([ev(lambda: b.run(logs, ws)) for _ in range(3)]))
            b.capture(logs, ws)
            b.replay()
            graph_ms.append(statistics.median([ev(b.replay) for _ in range(3)]))
            dof += sum(m.info()["n_dof"] for m in b.models)
        finally:
            b.close()
            del b
            torch.cuda.empty_cache()
    out = {"config": "C5: 48 surveys, meshes of 12..28 cubes per side (seeded), 2..8 loops, 16 rx, 24 times, "
                     "8 pole pairs; forward + one J^T.w each, refined FP32",
           "waves": [len(w) for w in waves], "total_dof": dof,
           "graph_ms": round(sum(graph_ms), 1), "eager_ms": round(sum(eager_ms), 1),
           "models_per_s": round(n_models / (sum(graph_ms) / 1e3), 2),
           "per_wave_graph_ms": [round(x, 1) for x in graph_ms], "per_wave_eager_ms": [round(x, 1) for x in eager_ms],
           "note": "factor + forward + J^T.w of every survey; one graph launch per wave (CUDA events, median of 3)"}
    print(json.dumps(out), flush=True)


def run_peaks(args):
    """Dense-GEMM rates of the pipes the method uses, measured with cuBLAS
    through torch.matmul (square n^3 products, 2 n^3 flops, best of 10 after
    warm-up, CUDA events): FP64, FP32 with TF32 off (the SIMT FP32 pipe) and
    TF32 (the tensor pipe the solve products and front updates run on)."""
    import torch
    torch.cuda.set_device(0)
    out = {"how": "torch.matmul n^3, 2 n^3 flops, best of 10 (CUDA events)"}
    for name, dt, tf32, n in (("fp64", torch.float64, False, 4096), ("fp32_simt", torch.float32, False, 8192),
                              ("tf32", torch.float32, True, 8192)):
        torch.backends.cuda.matmul.allow_tf32 = tf32
        a = torch.randn(n, n, dtype=dt, device="cuda")
        b = torch.randn(n, n, dtype=dt, device="cuda")
        for _ in range(3):
            torch.matmul(a, b)
        best = min(timed(torch, lambda: torch.matmul(a, b))[0] for _ in range(10))
        out[name + "_tflops"] = round(2.0 * n ** 3 / (best * 1e-3) / 1e12, 2)
        del a, b
    torch.backends.cuda.matmul.allow_tf32 = False
    print(json.dumps(out), flush=True)


def oracle_config_baseline(s, xi, al, v, w):
    """CPU baseline leg of --configs: the oracle as it stands on this host
    (poles on parallel threads), factor + forward, then one J.v + J^T.w pair."""
    from oracle.tem import Oracle
    t0 = time.perf_counter()
    o = Oracle(s.xyz, s.tets, s.sigma, s.is_param, s.loops, s.rx, xi, al)
    o.set_model(s.log_sigma())
    o.forward()
    t1 = time.perf_counter()
    o.jvp(v)
    o.jtvp(w)
    t2 = time.perf_counter()
    return {"oracle_factor_forward_s": round(t1 - t0, 2), "oracle_pair_s": round(t2 - t1, 2),
            "oracle_threads": int(o.threads), "nproc": os.cpu_count()}


def run_configs(args):
    """Configurations C1-C3: GPU factor, forward and J.v + J^T.w pair times
    (CUDA events, median of 3) in both precisions, and the oracle on this host
    (factor + forward + one pair, poles on parallel threads) for C1 and C2."""
    import numpy as np
    import torch
    from paper_2605_19951_gb300 import inputs, tem
    torch.cuda.set_device(0)
    rows = []
    for cfg in (1, 2, 3):
        s = inputs.make_config(cfg)
        xi, al = inputs.load_rational(s.m, s.times)
        rng = np.random.default_rng(cfg)
        v = rng.standard_normal(s.n_param)
        w = rng.standard_normal((len(s.loops), len(s.rx), len(s.times)))
        row = {"config": f"C{cfg}", "n": s.n, "poles": s.m, "loops": len(s.loops)}
        for prec, name in ((tem.TEM_FP64, "fp64"), (tem.TEM_FP32_REFINED, "fp32r")):
            mdl = tem.Model(s.xyz, s.tets, s.sigma, s.is_param, s.loops, s.rx, xi, al, precision=prec)
            try:
                m0 = torch.as_tensor(s.log_sigma(), device="cuda")
                vv, ww = torch.as_tensor(v, device="cuda"), torch.as_tensor(w, device="cuda")
                mdl.factor(m0)
                mdl.forward()
                mdl.jvp(vv), mdl.jtvp(ww)
                row[name + "_factor_ms"] = round(statistics.median([timed(torch, lambda: mdl.factor(m0))[0]
                                                                    for _ in range(3)]), 2)
                row[name + "_forward_ms"] = round(statistics.median([timed(torch, lambda: mdl.forward())[0]
                                                                     for _ in range(3)]), 2)
                row[name + "_pair_ms"] = round(statistics.median([timed(torch, lambda: (mdl.jvp(vv), mdl.jtvp(ww)))[0]
                                                                  for _ in range(3)]), 2)
                row["dof"] = mdl.info()["n_dof"]
            finally:
                mdl.close()
            torch.cuda.empty_cache()
        if cfg <= 2:
            row.update(oracle_config_baseline(s, xi, al, v, w))
        rows.append(row)
        print(json.dumps(row), flush=True)


def run_gn(args):
    """The inversion itself at the workload's size: the observed data are the
    forward of the true model (two conductive blocks) plus 3% noise with the
    error model of Section 4.2; from the 0.01 S/m half-space, Gauss-Newton
    iterations of Section 3.3 (30 LSQR iterations per direction, Armijo
    backtracking, lambda cooling from 10).  Per iteration: chi^2, lambda, step
    length, line-search trials and its time (CUDA events); at the end the
    model's misfit to the true log-conductivity inside and outside the blocks."""
    import numpy as np
    import torch
    from paper_2605_19951_gb300 import gn as gnmod
    from paper_2605_19951_gb300 import inputs, tem
    torch.cuda.set_device(0)
    s = inputs.make_config(CONFIG, n=args.n)
    xi, al = inputs.load_rational(s.m, s.times)
    mdl, d_obs_h, wd_h = synthetic(tem, s, xi, al, torch)
    d_obs = torch.as_tensor(d_obs_h, device="cuda")
    wd = torch.as_tensor(wd_h, device="cuda")
    m0 = torch.as_tensor(np.log(s.sigma_start[s.is_param.astype(bool)]), device="cuda")
    m_true = s.log_sigma()
    g = gnmod.GaussNewton(mdl, d_obs, wd, m0.clone(), m0, lam=LAMBDA, n_lsqr=N_LSQR_GN)
    rows = []
    t_all = 0.0
    for _ in range(args.gn):
        if g.converged():
            break
        ms, rec = timed(torch, g.step)
        t_all += ms
        rows.append({"it": rec["it"], "chi2_before": round(rec["chi2_0"], 4), "chi2": round(rec["chi2"], 4),
                     "lam": rec["lam"], "eta": round(rec["eta"], 4),
                     "trials": rec["trials"], "ms": round(ms, 1)})
        print(json.dumps(rows[-1]), flush=True)
    m = g.m.cpu().numpy()
    anomal = np.abs(m_true - np.log(0.01)) > 1e-9
    out = {"config": f"{s.n}^3 Kuhn box, {mdl.info()['n_dof']} DoF, 10 pole pairs, 32 loops, 128 rx, 40 times",
           "iterations": len(rows), "total_s": round(t_all / 1e3, 1),
           "chi2_start": rows[0]["chi2_before"] if rows else None, "chi2_end": rows[-1]["chi2"] if rows else None,
           "rms_log_sigma_error_blocks": float(np.sqrt(np.mean((m - m_true)[anomal] ** 2))),
           "rms_log_sigma_error_start_blocks": float(np.sqrt(np.mean((m0.cpu().numpy() - m_true)[anomal] ** 2))),
           "history": rows}
    mdl.close()
    print(json.dumps(out), flush=True)


if __name__ == "__main__":
    a = parse()
    if a.gn:
        run_gn(a)
    elif a.peaks:
        run_peaks(a)
    elif a.configs:
        run_configs(a)
    elif a.c5:
        run_c5(a)
    elif a.levels:
        run_levels(a)
    elif a.impl == "reference":
        run_reference(a)
    else:
        run_ours(a)
