#!/usr/bin/env python
"""Throughput benchmark of the CSE hot path on GB300.

Workload (default): the two-arm pooled z-test design, n = 100 patients per arm,
256 x 256 grid over [-2, 2]^2 keeping the 32,896 tiles that meet
theta_1 <= theta_0, K = 16,384 sims per tile, lambda = -1.96 (z > 1.96),
delta = 0.01, alpha = 0.025.

One step = one pass of the whole hot path over a fresh batch of simulations:
new CRN uniforms (reseed), success thresholds, axis count tables, alpha' per
tile, the fused simulation / rejection / selection pass, Clopper-Pearson +
optimised Tilt-Bound per tile, the minimum over tiles, and the score-function
backward.  Metric: sim x gridpoints per second (each (sim, tile) pair fully
processed).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl chosen|reference]

Under torchrun each rank processes its own independent calibration problem of
the same size (independent problems: weak scaling, no data-path collective).
--impl reference times the CPU FP64 oracle (the only reference this method
has) on a bounded sample of the same workload on the host cores.
"""
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

METRIC = "sim·gridpoints/s (TIE+score+tilt bound) on 1 GB300, chosen vs plain; % ALU roofline"
UNIT = "sim·gridpoints/s"
DELTA, ALPHA = 0.01, 0.025
CPU_SAMPLE_S = 10.0   # seconds of oracle work timed for cpu_baseline
# workload -> (config key of workloads.CONFIGS or a builder, lambda, description)
WORKLOADS = {
    "c2": ("c2", -1.96, "two-arm pooled z-test, n=100/arm, 256x256 grid over [-2,2]^2, "
                        "32,896 null tiles (theta1<=theta0), K=16,384 sims/tile"),
    "c1": ("c1", -1.96, "one-arm z-test, n=50, 64 tiles over [-2,0], K=8192"),
    "c3": ("c3", -1.96, "two-arm pooled z-test, 2^18 mixed-level tiles (h=2^-4..2^-7), K in 2^12..2^16"),
    "c4": ("c4", 0.06, "four-arm Bayesian selection design, looks 10/20/40, 16^4 grid over "
                       "logit[0.27,0.76]^4, 51,136 null tiles, K=2^14"),
    "c5": ("c5", 0.06, "four-arm Bayesian selection design, 2^20 adaptively refined tiles, K=2^16"),
    "c2_small": (None, -1.96, "two-arm pooled z-test, 64x64 grid over [-2,2]^2, 2,080 null tiles, "
                              "K=16,384 (profiling case)"),
    "c4_small": (None, 0.06, "four-arm Bayesian selection design, 8^4 grid over logit[0.27,0.76]^4, "
                             "K=2^14 (profiling case)"),
    "berry": ("berry", 0.15, "basket trial of Sec. 10.1 (4 arms, n=35, hierarchical posterior, reject arm i when "
                             "P(p_i > p_0i | data) > 85%), 16^4 grid over theta in [-3.5,1]^4, 59,992 tiles meeting "
                             "a null set, K=2^14; null rates 0.10/0.15/0.20/0.25 (synthetic stand-in)"),
    "berry_small": (None, 0.15, "basket trial of Sec. 10.1, 8^4 grid over [-3.5,1]^4, K=2^14 (profiling case)"),
    "c2_adaptive": (None, None, "adaptive calibration of the two-arm pooled z-test from a 64x64 grid over "
                                "[-2,2]^2 at K=4096: critical tiles split (half-width down to 1/512) or "
                                "double K (up to 2^16) for up to 6 rounds"),
}
SM_COUNT, LANES_PER_SM, SM_MAX_MHZ = 152, 128, 2070.0
# algorithmic lane operations per (sim, tile) of the fused two-arm pass: two
# count reads, cell index, rank read, compare, three predicated accumulates,
# one histogram increment (calibration)
OPS_PER_SIM_TILE = 9
# DRAM bytes (read + write) per launch of the dominant kernel from one ncu
# capture of the same workload and build (profiles/k_sim_cells_two_arm_256x256_K16384.md);
# reported as the roofline's traffic until that kernel changes
MEASURED_TRAFFIC = {("c2", "sim_ztest"): 9051136}   # ncu: 9.05 MB read, 0 written
# designs whose statistic is an FP32 posterior (decisions may flip against the FP64 oracle)
POSTERIOR = ("bayes4", "berry4")
# the simulation kernel of each design: the one timed with events inside the timed region
DOMINANT = {"one_arm_z": "sim_ztest", "two_arm_pooled_z": "sim_ztest", "bayes4": "sim_bayes4",
            "berry4": "sim_basket"}
# the paper's basket validation: 7.34e12 trial simulations in 4 h on one V100
PAPER_BASKET_SIMS_PER_S = 7.34e12 / (4 * 3600.0)


def load_workload(name):
    from paper_2212_10042_gb300 import workloads as W
    key = WORKLOADS[name][0]
    if name == "c2_small":
        return W.TWO_ARM, W.two_arm_grid(64, 16384)
    if name == "c4_small":
        return W.BAYES4, W.four_arm_grid(8, 1 << 14)
    if name == "berry_small":
        return W.BERRY4, W.berry_grid(8, 1 << 14)
    return W.CONFIGS[key]()


def workload_config(name, tiles=None):
    cfg = {"workload": WORKLOADS[name][2], "name": name, "lambda": WORKLOADS[name][1],
           "delta": DELTA, "alpha": ALPHA,
            "step": "reseed CRN + thresholds + axis counts + alpha' + fused sim/reject/select + "
                    "Clopper-Pearson + q-optimised Tilt-Bound + min over tiles + score backward",
            "l2": "flushed between timed steps (512 MiB write)",
            "parallelism": "independent problem per rank"}
    if tiles is not None:
        cfg.update({"tiles": tiles.n_tiles, "K_max": tiles.K_max, "sim_tiles_per_step": int(tiles.K.sum())})
    return cfg


def env_rank():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.f = None

    def start(self):
        try:
            self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.gpu)], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.flush()
        self.f.seek(0)
        rows = [r.split(",") for r in self.f.read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except ValueError:
                continue
            for n, v in zip(names, r[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(sm)}


def oracle_sample(name, design, tiles, n_tiles, seed, keep=None):
    """Run the CPU oracle on `n_tiles` tiles drawn from the workload; returns
    (sim x tiles processed, seconds, threads).  With `keep` (a dict), the sampled
    rows and the oracle's outputs are stored there."""
    from oracle import oracle as O
    import numpy as np
    rng = np.random.default_rng(seed)
    rows = np.sort(rng.choice(tiles.n_tiles, n_tiles, replace=False))
    sub = tiles.subset(rows)
    lam = WORKLOADS[name][1]
    t0 = time.perf_counter()
    sim = O.simulate(design, sub, lam)
    vb = O.validate_bounds(design, sub, sim["R"], DELTA)
    cal = O.calibrate(design, sub, ALPHA)
    O.score_backward(np.ones(sub.n_tiles), sim["score"], sub.K)
    dt = time.perf_counter() - t0
    if keep is not None:
        keep.update(rows=rows, sim=sim, vb=vb, cal=cal)
    return int(sub.K.sum()), dt, O.num_threads()


def accuracy_report(out, ref, bayes):
    """GPU outputs of the sampled tiles against the FP64 oracle's."""
    import numpy as np
    rows = ref["rows"]
    R = out["R"].cpu().numpy()[rows]
    X = out["Xrej"].cpu().numpy()[rows]
    b = out["bound"].cpu().numpy()[rows]
    ap = out["alpha_prime"].cpu().numpy()[rows]
    lt = out["lambda_tile"].cpu().numpy()[rows]
    rel = lambda a, r: float(np.max(np.abs(a - r) / np.maximum(np.abs(r), 1e-300)))
    rep = {"tiles_checked": int(len(rows)), "sims_checked": int(ref["sims"]),
           "R_tiles_differing": int(np.sum(R != ref["sim"]["R"])),
           "R_abs_diff_total": int(np.abs(R - ref["sim"]["R"]).sum()),
           "Xrej_tiles_differing": int(np.sum(np.any(X != ref["sim"]["Xrej"], axis=1))),
           "alpha_prime_max_rel_err": rel(ap, ref["cal"]["alpha_prime"])}
    if not bayes:
        rep["bound_max_rel_err"] = rel(b, ref["vb"]["bound"])
        rep["lambda_tile_exact"] = int(np.sum(lt == ref["cal"]["lambda_tile"]))
    else:
        fin = np.isfinite(ref["cal"]["lambda_tile"]) & np.isfinite(lt)
        rep["lambda_tile_max_abs_err"] = float(np.max(np.abs(lt[fin] - ref["cal"]["lambda_tile"][fin]))) \
            if fin.any() else 0.0
        rep["note"] = "FP32 posterior vs FP64 oracle: R differences are decision flips"
    return rep


def run_reference(args):
    rank, world, _ = env_rank()
    if rank != 0:
        return 0
    from oracle import build as ob
    ob.build()
    design, tiles = load_workload(args.workload)
    n_sample = 24 if design.stat not in POSTERIOR else 4
    for i in range(args.warmup):
        oracle_sample(args.workload, design, tiles, n_sample, 1000 + i)
    units, secs = 0, 0.0
    threads = 1
    for i in range(args.steps):
        u, dt, threads = oracle_sample(args.workload, design, tiles, n_sample, 2000 + i)
        units += u
        secs += dt
    v = units / secs
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded Philox CRN)", "config": workload_config(args.workload, tiles),
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": "%d random tiles of the workload per step at their full K" % n_sample},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_adaptive(args):
    """The adaptive calibration loop (paper_2212_10042_gb300.adaptive) on the GPU:
    every round calibrates the whole current platten; the units are the
    sim-tiles of all rounds, the time the whole loop (device work, the host's
    refinement decisions and the tile-set copies between rounds)."""
    import torch
    rank, world, local = env_rank()
    torch.cuda.set_device(local)
    import __graft_entry__
    __graft_entry__.build()
    from paper_2212_10042_gb300 import adaptive as A
    from paper_2212_10042_gb300 import workloads as W
    cfg = A.RefineConfig(alpha=ALPHA, max_iter=6, crit_frac=0.05, slack_tol=0.05, min_halfwidth=1.0 / 512,
                         K_cap=1 << 16)
    t0 = W.two_arm_grid(64, 4096)
    cal = A.GpuCalibrator(W.TWO_ARM, ALPHA, cfg.K_cap, seed=1_000_003)
    A.run(t0, cal, A.RefineConfig(alpha=ALPHA, max_iter=1), one_arm=False)   # warm-up round
    torch.cuda.synchronize()
    best = None
    for rep in range(max(1, args.steps)):
        t = time.perf_counter()
        res = A.run(t0, cal, cfg, one_arm=False)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t
        if best is None or dt < best[0]:
            best = (dt, res)
    dt, res = best
    units = sum(r["sum_K"] for r in res["trace"])
    line = {"metric": METRIC, "value": units / dt, "unit": UNIT, "n_gpus": 1, "steps": max(1, args.steps),
            "warmup": 1, "ms_per_step": dt * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u8/i32 counts + f32 statistic + f64 bounds",
            "data": "synthetic (seeded Philox CRN; no dataset)",
            "config": {"workload": WORKLOADS["c2_adaptive"][2], "name": "c2_adaptive", "alpha": ALPHA,
                       "step": "one whole adaptive loop (best of the timed repetitions, wall clock)"},
            "adaptive": {"rounds": len(res["trace"]), "converged": res["converged"], "trace": res["trace"],
                         "final_tiles": res["tiles"].n_tiles, "lambda_star": res["lam"]}}
    print(json.dumps(line))


def run_chosen(args):
    import torch
    import torch.distributed as dist

    rank, world, local = env_rank()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    import __graft_entry__
    if rank == 0 or world == 1:
        __graft_entry__.build()
    if world > 1:
        dist.barrier()
    from paper_2212_10042_gb300 import binding as B
    from paper_2212_10042_gb300 import workloads as W

    design, tiles = load_workload(args.workload)
    LAMBDA = WORKLOADS[args.workload][1]
    seed0 = 1_000_003 * (rank + 1)
    ctx = B.Context(design, seed=seed0, K_max=tiles.K_max)
    dt = B.DeviceTiles(tiles)
    out = ctx.step_buffers(dt)
    ones = torch.ones(tiles.n_tiles, dtype=torch.float64, device="cuda")
    units = int(tiles.K.astype("int64").sum())
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()

    def step(i):
        ctx.reseed(seed0 + i)
        ctx.step(dt, LAMBDA, DELTA, ALPHA, out)
        return B.score_backward(ones, out["score"], dt.K)

    for i in range(args.warmup):
        step(i)
    torch.cuda.synchronize()
    ctx.sync()
    if args.sim_threads:   # fixed block size (e.g. to match a live run's choice under a profiler)
        ctx.set_option(B.OPT_SIM_THREADS, args.sim_threads)
        tuned_threads = args.sim_threads
    else:
        tuned_threads = ctx.autotune(dt, LAMBDA, ALPHA)   # block size of the simulation kernel

    clocks = ClockSampler(local)
    clocks.start()
    # events around the simulation kernel only: a pair around every kernel costs
    # ~2 us of step time each and delays the table kernels beside alpha'
    ctx.profile(True, only=DOMINANT[design.stat])
    ctx.profile_read()
    launches0 = ctx.launch_count()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    for i in range(args.steps):
        flush.fill_(i & 0xFF)
        evs[i][0].record(stream)
        step(args.warmup + i)
        evs[i][1].record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    ms = sum(a.elapsed_time(b) for a, b in evs)
    launches = ctx.launch_count() - launches0 + args.steps   # + one backward kernel per step
    prof_dom = ctx.profile_read()
    ctx.profile(False)
    clk = clocks.stop()
    ctx.sync()

    # per-kernel breakdown (diagnostic): a separate pass with every kernel timed
    n_diag = max(1, min(args.steps, 20))
    ctx.profile(True)
    ctx.profile_read()
    for i in range(n_diag):
        flush.fill_(i & 0xFF)
        step(args.warmup + args.steps + i)
    prof = ctx.profile_read()
    ctx.profile(False)
    ctx.sync()

    t = torch.tensor([ms], dtype=torch.float64, device="cuda")
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms_max = float(t.item())
    value = units * world * args.steps / (ms_max * 1e-3)

    # ---- the same step replayed from a captured CUDA graph (one launch per step) ----
    graph_ms = None
    if not args.no_graph:
        sg = B.StepGraph(ctx, dt, LAMBDA, DELTA, ALPHA, seed0 + 123, out, ones)
        for _ in range(3):
            sg.replay()
        torch.cuda.synchronize()
        gev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(args.steps)]
        for i in range(args.steps):
            flush.fill_(i & 0xFF)
            gev[i][0].record(stream)
            sg.replay()
            gev[i][1].record(stream)
        torch.cuda.synchronize()
        graph_ms = sum(a.elapsed_time(b) for a, b in gev) / args.steps
        del sg

    # ---- the plain comparison path on the same GPU (same results, see cse.h) ----
    plain = None
    if not args.no_plain:
        n_plain = max(3, min(args.steps, 20))
        ctx.set_option(B.OPT_PLAIN, 1)
        for i in range(2):
            step(50_000 + i)
        torch.cuda.synchronize()
        ctx.profile(True)
        ctx.profile_read()
        pev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(n_plain)]
        for i in range(n_plain):
            flush.fill_(i & 0xFF)
            pev[i][0].record(stream)
            step(60_000 + i)
            pev[i][1].record(stream)
        torch.cuda.synchronize()
        pms = sum(a.elapsed_time(b) for a, b in pev) / n_plain
        pprof = ctx.profile_read()
        ctx.profile(False)
        ctx.set_option(B.OPT_PLAIN, 0)
        plain = {"value": units / (pms * 1e-3), "ms_per_step": pms, "steps": n_plain,
                 "kernels_ms_per_launch": {k: tms / max(n, 1) for k, (n, tms) in pprof.items()},
                 "what": "per-(tile,sim) binary search counts, FP64-only bound pass"
                         + (", direct per-trial posterior" if design.stat in POSTERIOR else "")}

    # ---- two-sided validation band (lower and upper tile bounds at delta / 2) ----
    band = None
    if not args.no_band:
        n_band = max(3, min(args.steps, 20))
        for i in range(2):
            ctx.reseed(seed0 + 70_000 + i)
            ctx.validate_band(dt, LAMBDA, DELTA)
        torch.cuda.synchronize()
        bev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(n_band)]
        for i in range(n_band):
            flush.fill_(i & 0xFF)
            bev[i][0].record(stream)
            ctx.reseed(seed0 + 80_000 + i)
            ctx.validate_band(dt, LAMBDA, DELTA)
            bev[i][1].record(stream)
        torch.cuda.synchronize()
        ctx.sync()
        bms = sum(a.elapsed_time(b) for a, b in bev) / n_band
        band = {"value": units / (bms * 1e-3), "unit": UNIT, "ms_per_step": bms, "steps": n_band,
                "what": "reseed + simulation + lower and upper tile bounds at delta/2 (cse_validate_band)"}

    # ---- randomised calibration (pairs (S, w), lexicographic; z-tests) ----
    rand = None
    if not args.no_band and design.stat not in POSTERIOR:
        n_rand = max(3, min(args.steps, 10))
        ctx.reseed(seed0 + 90_000)
        ctx.calibrate_rand(dt, ALPHA)
        torch.cuda.synchronize()
        t_r = []
        for i in range(n_rand):
            flush.fill_(i & 0xFF)
            ctx.reseed(seed0 + 91_000 + i)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            cr = ctx.calibrate_rand(dt, ALPHA)
            e1.record(stream)
            torch.cuda.synchronize()
            t_r.append(e0.elapsed_time(e1))
        rms = sum(t_r) / n_rand
        rand = {"value": units / (rms * 1e-3), "unit": UNIT, "ms_per_step": rms, "steps": n_rand,
                "lambda_star": cr["lam"], "c_star": cr["c"],
                "what": "alpha' + randomised simulation/selection + lexicographic min (cse_calibrate_rand)"}

    # ---- end to end through the public API with host buffers ----
    host_in = {"axis": [a.cpu().pin_memory() for a in dt.axis], "idx": dt.idx.cpu().pin_memory(),
               "hw": dt.halfwidth.cpu().pin_memory(), "nm": dt.null_mask.cpu().pin_memory(),
               "K": dt.K.cpu().pin_memory()}
    h2d = sum(a.numel() * a.element_size() for a in host_in["axis"]) + sum(
        host_in[k].numel() * host_in[k].element_size() for k in ("idx", "hw", "nm", "K"))
    host_out = {k: torch.empty(v.shape, dtype=v.dtype, pin_memory=True) for k, v in out.items()}
    grad_host = torch.empty((tiles.n_tiles, tiles.d), dtype=torch.float64, pin_memory=True)
    d2h = sum(v.numel() * v.element_size() for v in host_out.values()) + grad_host.numel() * 8
    e2e_steps = max(1, args.steps)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    t0 = time.perf_counter()
    for i in range(e2e_steps):
        for a, h in zip(dt.axis, host_in["axis"]):
            a.copy_(h, non_blocking=True)
        dt.idx.copy_(host_in["idx"], non_blocking=True)
        dt.halfwidth.copy_(host_in["hw"], non_blocking=True)
        dt.null_mask.copy_(host_in["nm"], non_blocking=True)
        dt.K.copy_(host_in["K"], non_blocking=True)
        g = step(10_000 + i)
        for k, v in out.items():
            host_out[k].copy_(v, non_blocking=True)
        grad_host.copy_(g, non_blocking=True)
        torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    t = torch.tensor([e2e_s], dtype=torch.float64, device="cuda")
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    e2e_value = units * world * e2e_steps / float(t.item())

    # ---- roofline of the dominant kernel ----
    kern = {k: {"launches": n, "ms_per_launch": tms / max(n, 1), "share": 0.0} for k, (n, tms) in prof.items()}
    tot = sum(tms for _, tms in prof.values()) or 1.0
    for k, (n, tms) in prof.items():
        kern[k]["share"] = tms / tot
    roof = None
    if "sim_ztest" in prof_dom and design.stat == "two_arm_pooled_z":
        n_dom, ms_dom = prof_dom["sim_ztest"]
        achieved = OPS_PER_SIM_TILE * units / (ms_dom / max(n_dom, 1) * 1e-3) / 1e12
        peak = SM_COUNT * LANES_PER_SM * SM_MAX_MHZ * 1e6 / 1e12
        roof = {"kernel": "sim_ztest", "bound": "alu", "achieved": achieved, "peak": peak,
                "unit": "Tlane-op/s", "frac": achieved / peak,
                "traffic": MEASURED_TRAFFIC.get((args.workload, "sim_ztest")),
                "peak_source": "152 SMs x 128 lanes x 2070 MHz issue rate (derived, see DESIGN.md)",
                "ops_per_unit": OPS_PER_SIM_TILE, "ms_per_launch": ms_dom / max(n_dom, 1)}

    cpu = None
    accuracy = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        try:
            from oracle import build as ob
            ob.build()
            import dataclasses
            n_s = 64 if design.stat not in POSTERIOR else 6
            acc_seed = 777
            keep = {}
            u, secs, thr = oracle_sample(args.workload, dataclasses.replace(design, seed=acc_seed), tiles,
                                         n_s, 7, keep)
            keep["sims"] = u
            # more random samples of the workload until ~CPU_SAMPLE_S seconds of oracle work are timed
            tot_u, tot_s, draws, n2 = u, secs, 1, n_s
            if secs < CPU_SAMPLE_S:
                n2 = min(tiles.n_tiles, max(n_s, int(n_s * 1.1 * (CPU_SAMPLE_S - secs) / max(secs, 1e-3))))
                while tot_s < CPU_SAMPLE_S and draws < 1000:
                    u2, s2, _ = oracle_sample(args.workload, design, tiles, n2, 100 + draws)
                    tot_u += u2
                    tot_s += s2
                    draws += 1
            cpu = {"value": tot_u / tot_s, "unit": UNIT, "cores": thr, "kind": "oracle",
                   "sample": "%d draws of random tiles of the workload at their full K (the first %d tiles, "
                             "then %d tiles each): simulate + validate bounds + calibrate + backward, %.3g "
                             "sim-tiles in %.1f s" % (draws, n_s, n2, tot_u, tot_s)}
            # the same seed on the GPU: accuracy of this run's outputs against the oracle
            ctx.reseed(acc_seed)
            ctx.step(dt, LAMBDA, DELTA, ALPHA, out)
            torch.cuda.synchronize()
            accuracy = accuracy_report(out, keep, design.stat in POSTERIOR)
        except Exception as e:  # noqa: BLE001
            cpu = {"value": None, "unit": UNIT, "cores": None, "kind": "oracle", "sample": "failed: %s" % e}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None,
                "dtype": "u8/i32 counts + f32 statistic + f64 bounds",
                "data": "synthetic (seeded Philox CRN; no dataset)",
                "config": workload_config(args.workload, tiles),
                "roofline": roof, "cpu_baseline": cpu,
                "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d,
                        "d2h_bytes_per_step": d2h},
                "clocks": clk, "gpu_launches": launches, "kernels": kern,
                "kernels_note": "events around every kernel in a separate pass of %d steps after the timed "
                                "region (the timed region has events around the simulation kernel only)" % n_diag,
                "plain": plain, "validate_band": band, "calibrate_rand": rand, "chosen_over_plain": (value / world / plain["value"]) if plain else None,
                "accuracy_vs_oracle": accuracy,
                "cuda_graph": None if graph_ms is None else {
                    "ms_per_step": graph_ms, "value": units * world / (graph_ms * 1e-3),
                    "note": "same step replayed from one captured CUDA graph (CRN key fixed in the graph)"},
                "autotune": {"sim_threads_per_block": tuned_threads},
                "lambda_star": float(out["lam"].item())}
        if design.stat == "berry4":
            line["paper_context"] = {
                "value": PAPER_BASKET_SIMS_PER_S, "unit": "trial sims/s",
                "what": "the paper's basket validation on one V100 (7.34e12 sims in 4 h; its null rates are not "
                        "given, so the workloads differ): context, not a baseline"}
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["chosen", "reference"], default="chosen")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-plain", action="store_true", help="skip the plain-path comparison")
    ap.add_argument("--no-band", action="store_true", help="skip the validation-band timing")
    ap.add_argument("--sim-threads", type=int, default=0, choices=[0, 128, 256, 512],
                    help="fix the simulation kernel's block size instead of autotuning (z-tests)")
    ap.add_argument("--no-graph", action="store_true", help="skip the CUDA-graph replay timing")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="c2",
                    help="c2 (default) is the benchmark workload; the others serve profiling "
                         "and per-design throughput figures")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "c2_adaptive":
        return run_adaptive(args)
    return run_chosen(args)


if __name__ == "__main__":
    sys.exit(main())
