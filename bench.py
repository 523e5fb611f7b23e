#!/usr/bin/env python
"""Throughput benchmark of the CSE hot path on GB300.

Workload (default): the largest single-GPU configuration, calibration of the
four-arm Bayesian selection design (control + 3 treatments, looks after 10, 20
and 40 patients per arm, hierarchical posterior in FP32) on 1,048,582
adaptively refined tiles over logit[0.27, 0.76]^4 with K = 65,536 sims per
tile, lambda = 0.06, delta = 0.01, alpha = 0.025 (the stand-in for the paper's
Phase II/III calibration, Sec. 10.2).  --workload c2 selects the two-arm pooled
z-test on the 256 x 256 grid (32,896 tiles, K = 16,384).

One step = one pass of the whole hot path over a fresh batch of simulations:
new CRN uniforms (reseed), success thresholds, axis count tables, alpha' per
tile, the fused simulation / rejection / selection pass, Clopper-Pearson +
optimised Tilt-Bound per tile, the minimum over tiles, and the score-function
backward.  Metric: sim x gridpoints per second (each (sim, tile) pair fully
processed).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl chosen|reference] [--workload NAME]

The roofline of the dominant (simulation) kernel is taken against peaks this
run measures itself with the library's pipe probes (cse_probe_peak), with the
SM clock sampled while they run.

Under torchrun each rank processes its own independent calibration problem of
the same size (independent problems: weak scaling, no data-path collective).
--impl reference times the CPU FP64 oracle (the only reference this method
has) on a bounded sample of the same workload on the host cores.
"""
import argparse
import json
import math
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
    "c5": ("c5", 0.06, "four-arm Bayesian selection design, looks 10/20/40, 1,048,582 adaptively refined "
                       "tiles over logit[0.27,0.76]^4, K=2^16"),
    "c5_sample": (None, 0.06, "four-arm Bayesian selection design, 65,536 consecutive tiles from the middle of the "
                              "refined 2^20-tile platten, K=2^16 (profiling case)"),
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
# Algorithmic lane operations per (sim, tile) of each design's simulation pass,
# the method's own work in the form this library computes it:
#   one arm: 1 count read, 1 compare, 2 predicated accumulates (R, X), 1
#     selection insert;
#   two arms (axis count tables, rejection monotone in both counts): 2 count
#     reads, 1 cell index, 1 compare-or-insert, 2 predicated accumulates;
#   four-arm selection design, tabulated posterior: 12 count reads (4 arms x 3
#     looks), 3 table gathers (drop bits at looks 1 and 2, final-look
#     probabilities), 1 compare, 5 predicated accumulates (R, 4 X), 1 selection
#     insert (the one-off table build is reported apart);
#   basket design, tabulated posterior: 4 count reads, 1 table gather, 1
#     compare, 5 predicated accumulates, 1 selection insert.
OPS_PER_SIM_TILE = {"one_arm_z": 5, "two_arm_pooled_z": 6, "bayes4": 22, "berry4": 12}
# What bounds each simulation kernel, from its ncu profile (profiles/)
LIMITER = {
    "sim_ztest": "issue and latency: the histogram loop (byte extracts, index, one shared-memory increment per "
                 "sim) and each tile's loads, barriers and read-off",
    "sim_bayes4": "L1 throughput (83 %: the final-table gathers, count reads, key stores and the radix passes' "
                  "key reads) and the integer ALU pipe (71 %: byte transposes, table indexing, code sorts)",
    "sim_basket": "L1 tag throughput of the scattered 16-byte table gathers",
}
# DRAM bytes (read + write) per launch of the dominant kernel from one ncu
# capture of the same kernel build, scaled to the workload where the capture
# ran on a smaller case; None until captured for the current kernel
MEASURED_TRAFFIC = {
    # profiles/k_sim_bayes4_four_arm_refined_sample_65536x65536.md: 26.73 GB on the
    # 65,536-tile sample, scaled by the sim-tiles to the full platten (x 16.0)
    ("c5", "sim_bayes4"): 427.70e9,
    ("c5_sample", "sim_bayes4"): 26.73e9,
    # profiles/k_sim_cells_two_arm_256x256_K16384.md: one capture at the full size
    ("c2", "sim_ztest"): 9.09e6,
}
# designs whose statistic is an FP32 posterior (decisions may flip against the FP64 oracle)
POSTERIOR = ("bayes4", "berry4")
# the simulation kernel of each design: the one timed with events inside the timed region
DOMINANT = {"one_arm_z": "sim_ztest", "two_arm_pooled_z": "sim_ztest", "bayes4": "sim_bayes4",
            "berry4": "sim_basket"}
# the paper's basket validation: 7.34e12 trial simulations in 4 h on one V100
PAPER_BASKET_SIMS_PER_S = 7.34e12 / (4 * 3600.0)


def load_workload(name):
    import numpy as np
    from paper_2212_10042_gb300 import workloads as W
    key = WORKLOADS[name][0]
    if name == "c2_small":
        return W.TWO_ARM, W.two_arm_grid(64, 16384)
    if name == "c4_small":
        return W.BAYES4, W.four_arm_grid(8, 1 << 14)
    if name == "berry_small":
        return W.BERRY4, W.berry_grid(8, 1 << 14)
    if name == "c5_sample":
        design, tiles = W.CONFIGS["c5"]()
        mid = tiles.n_tiles // 2
        return design, tiles.subset(np.arange(mid, mid + (1 << 16)))
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


def measure_peaks(B, gpu_index):
    """Pipe probes of the library (cse_probe_peak), with the SM clock sampled while
    they run: lane-operations per second of the integer ALU pipe (lop3), the FP32
    FMA and FP64 pipes, and conflict-free shared-memory atomics."""
    clk = ClockSampler(gpu_index)
    clk.start()
    res = {}
    for kind, iters, reps in (("alu", 4096, 60), ("fma", 4096, 100), ("dfma", 256, 30), ("smem_atomic", 1024, 60)):
        ops, ms = B.probe_peak(kind, blocks_per_sm=4, iters=iters, reps=reps)
        res[kind] = {"lane_ops_per_s": ops, "ms_per_launch": ms}
    c = clk.stop()
    res["clocks"] = c
    mhz = c.get("sm_mhz")
    import torch
    sms = torch.cuda.get_device_properties(gpu_index).multi_processor_count
    res["sm_count"] = sms
    if mhz:
        for kind in ("alu", "fma", "dfma", "smem_atomic"):
            res[kind]["lane_ops_per_sm_clock"] = res[kind]["lane_ops_per_s"] / (sms * mhz * 1e6)
    res["how"] = ("cse_probe_peak: 4 CTAs of 256 threads per SM, 128 independent instructions of one kind per "
                  "thread and iteration, CUDA events around repeated launches after one warm-up")
    return res


def run_reference(args):
    rank, world, _ = env_rank()
    if rank != 0:
        return 0
    from oracle import build as ob
    ob.build()
    design, tiles = load_workload(args.workload)
    n_sample = 24 if design.stat not in POSTERIOR else 16
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

    peaks = measure_peaks(B, local)
    design, tiles = load_workload(args.workload)
    LAMBDA = WORKLOADS[args.workload][1]
    seed0 = 1_000_003 * (rank + 1)
    torch.cuda.synchronize()
    t_setup = time.perf_counter()
    ctx = B.Context(design, seed=seed0, K_max=tiles.K_max)   # synchronises: uniforms + statistic tables
    setup_ms = (time.perf_counter() - t_setup) * 1e3
    dt = B.DeviceTiles(tiles)
    out = ctx.step_buffers(dt)
    ones = torch.ones(tiles.n_tiles, dtype=torch.float64, device="cuda")
    units = int(tiles.K.astype("int64").sum())
    # workloads of more than 2e10 sim-tiles per step (hundreds of ms): the
    # diagnostic, graph and band sections run fewer steps, the plain path a sample
    heavy = units > 2e10
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
    if args.sim_threads:   # fixed configuration (e.g. to match a live run's choice under a profiler)
        ctx.set_option(B.OPT_SIM_THREADS, args.sim_threads)
        ctx.set_option(B.OPT_SIM_TILES, args.sim_tiles)
        tuned = (args.sim_threads, args.sim_tiles)
    else:
        tuned = ctx.autotune(dt, LAMBDA, ALPHA)   # (threads, tiles) per block of the simulation kernel

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
    n_diag = max(1, min(args.steps, 5 if heavy else 20))
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
        for _ in range(1 if heavy else 3):
            sg.replay()
        torch.cuda.synchronize()
        n_graph = max(1, min(args.steps, 5 if heavy else args.steps))
        gev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(n_graph)]
        for i in range(n_graph):
            flush.fill_(i & 0xFF)
            gev[i][0].record(stream)
            sg.replay()
            gev[i][1].record(stream)
        torch.cuda.synchronize()
        graph_ms = sum(a.elapsed_time(b) for a, b in gev) / n_graph
        del sg

    # ---- the plain comparison path on the same GPU (same results, see cse.h) ----
    plain = None
    if not args.no_plain:
        # heavy workloads: both paths on the same seeded sample of 4,096 tiles (the
        # plain path's direct posterior would take minutes per full step)
        import numpy as np
        if heavy:
            rows = np.sort(np.random.default_rng(5).choice(tiles.n_tiles, 4096, replace=False))
            p_tiles = tiles.subset(rows)
        else:
            p_tiles = tiles
        p_dt = B.DeviceTiles(p_tiles) if heavy else dt
        p_out = ctx.step_buffers(p_dt) if heavy else out
        p_ones = torch.ones(p_tiles.n_tiles, dtype=torch.float64, device="cuda")
        p_units = int(p_tiles.K.astype("int64").sum())

        def p_step(i):
            ctx.reseed(seed0 + i)
            ctx.step(p_dt, LAMBDA, DELTA, ALPHA, p_out)
            return B.score_backward(p_ones, p_out["score"], p_dt.K)

        def timed(n, base):
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n)]
            for i in range(n):
                flush.fill_(i & 0xFF)
                ev[i][0].record(stream)
                p_step(base + i)
                ev[i][1].record(stream)
            torch.cuda.synchronize()
            return sum(a.elapsed_time(b) for a, b in ev) / n

        n_plain = max(3, min(args.steps, 20))
        sample_chosen_ms = timed(n_plain, 40_000) if heavy else None
        ctx.set_option(B.OPT_PLAIN, 1)
        for i in range(2):
            p_step(50_000 + i)
        torch.cuda.synchronize()
        ctx.profile(True)
        ctx.profile_read()
        pms = timed(n_plain, 60_000)
        pprof = ctx.profile_read()
        ctx.profile(False)
        ctx.set_option(B.OPT_PLAIN, 0)
        plain = {"value": p_units / (pms * 1e-3), "ms_per_step": pms, "steps": n_plain,
                 "kernels_ms_per_launch": {k: tms / max(n, 1) for k, (n, tms) in pprof.items()},
                 "what": "per-(tile,sim) binary search counts, FP64-only bound pass"
                         + (", direct per-trial posterior" if design.stat in POSTERIOR else "")}
        if heavy:
            plain["sample"] = "4,096 seeded random tiles of the workload at their full K (%.3g sim-tiles)" % p_units
            plain["chosen_on_sample"] = {"value": p_units / (sample_chosen_ms * 1e-3),
                                         "ms_per_step": sample_chosen_ms}

    # ---- two-sided validation band (lower and upper tile bounds at delta / 2) ----
    band = None
    if not args.no_band:
        n_band = 3 if heavy else max(3, min(args.steps, 20))
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
    kname = DOMINANT[design.stat]
    if kname in prof_dom:
        n_dom, ms_dom = prof_dom[kname]
        ms_l = ms_dom / max(n_dom, 1)
        ops = OPS_PER_SIM_TILE[design.stat]
        achieved = ops * units / (ms_l * 1e-3) / 1e12
        peak = peaks["alu"]["lane_ops_per_s"] / 1e12
        roof = {"kernel": kname, "bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tlane-op/s",
                "frac": achieved / peak, "traffic": MEASURED_TRAFFIC.get((args.workload, kname)),
                "peak_source": "measured in this run: integer ALU pipe (lop3) probe of cse_probe_peak at a median "
                               "SM clock of %s MHz" % peaks["clocks"].get("sm_mhz"),
                "ops_per_unit": ops, "units_per_launch": units, "ms_per_launch": ms_l,
                "limiter": LIMITER.get(kname)}
        if design.stat in ("one_arm_z", "two_arm_pooled_z"):
            # the cell histogram: one shared-memory atomic increment per (sim, tile)
            a_peak = peaks["smem_atomic"]["lane_ops_per_s"] / 1e12
            roof["smem_atomic"] = {"achieved": units / (ms_l * 1e-3) / 1e12, "peak": a_peak, "unit": "Tatomic/s",
                                   "frac": units / (ms_l * 1e-3) / 1e12 / a_peak,
                                   "what": "one shared-memory atomic increment per (sim, tile) against the "
                                           "conflict-free shared-atomic probe"}

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
                "plain": plain, "validate_band": band, "calibrate_rand": rand, "chosen_over_plain": (None if not plain else (
                    plain["chosen_on_sample"]["value"] if heavy else value / world) / plain["value"]),
                "accuracy_vs_oracle": accuracy,
                "cuda_graph": None if graph_ms is None else {
                    "ms_per_step": graph_ms, "value": units * world / (graph_ms * 1e-3),
                    "note": "same step replayed from one captured CUDA graph (CRN key fixed in the graph)"},
                "autotune": {"sim_threads_per_block": tuned[0], "tiles_per_block": tuned[1],
                             "sims_per_block_step": 16 * tuned[0] if design.stat not in POSTERIOR else 4 * tuned[0]},
                "peaks_measured": peaks,
                "context_setup": {"ms": setup_ms, "what": "cse_create, once per context (host clock): the first CRN "
                                  "uniforms and the design's statistic tables (the four-arm and basket designs' "
                                  "posterior tables); not part of a step"},
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
    ap.add_argument("--steps", type=int, default=None, help="timed steps (default 20, or 200 below 2e10 "
                                                             "sim-tiles per step)")
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["chosen", "reference"], default="chosen")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-plain", action="store_true", help="skip the plain-path comparison")
    ap.add_argument("--no-band", action="store_true", help="skip the validation-band timing")
    ap.add_argument("--sim-threads", type=int, default=0, choices=[0, 64, 128, 256, 512],
                    help="fix the simulation kernel's block size instead of autotuning (z-tests)")
    ap.add_argument("--sim-tiles", type=int, default=1, choices=[1, 2, 4],
                    help="with --sim-threads: tiles per block of the z-test cell kernel")
    ap.add_argument("--no-graph", action="store_true", help="skip the CUDA-graph replay timing")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="c5",
                    help="c5 (default) is the benchmark workload, the largest single-GPU configuration; the "
                         "others serve per-design throughput figures and profiling")
    args = ap.parse_args()
    if args.steps is None:
        args.steps = 20 if args.workload in ("c5",) else 200
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "c2_adaptive":
        return run_adaptive(args)
    return run_chosen(args)


if __name__ == "__main__":
    sys.exit(main())
