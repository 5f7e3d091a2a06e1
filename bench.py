"""Benchmark: snake env-steps/s at residual <= 1e-4 on one GB300 (per rank).

A step is one env-step (dt = 1/60 s, 20 substeps, Jacobi to residual 1e-4) of the whole
batch: 16384 snakes with 2..8 links of 10 segments (0.02 m, 0.01 kg per node), drawn
like the paper's snake (four links, Sec. V) but uneven, with the gait of Eq. 9.  The
batch state stays resident in HBM; L2 is flushed between timed steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Under torchrun (N ranks) one seeded batch of N x 16384 snakes is split into N contiguous
ranges balanced by node count (sim_partition), one per rank and GPU (independent snakes,
no data-path collective, weak scaling); rank 0 prints one JSON line.  `--impl reference`
times the FP64 CPU oracle instead on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

METRIC = "snake env-steps/s at residual<=1e-4, learned warm-start vs plain, 1 GB300"
N_SNAKES = 16384
# plain env-steps that take the batch from its straight resting pose into steady
# locomotion (1 s of simulated time) before anything is timed: the first ~20 env-steps
# are the touchdown of the gait, which every mode runs 30-50 % faster than the steps after
SETTLE = 60
TOL = 1e-4
CAP = 5000
SKIP = 0.5  # learned warm start: lambda0 = SKIP lambda_prev + m g h^2 network(features)
# the learned warm start the metric is quoted on: the network on the stretch rows at
# every third substep, its prediction on SKIP x the previous multipliers, LEARNED_BETA x
# the previous multipliers at the other substeps and rows, trained on targets solved from
# SKIP x the previous multipliers along trajectories that use the network in this same
# configuration; PREV_BETA for the previous-multiplier start.  Each is the fastest value
# measured on the settled 16384-snake batch (network every 2nd / 3rd / 4th substep on the
# bilateral rows: 505 k / 530 k / 498 k env-steps/s; stretch rows against bilateral rows at
# every 3rd, each trained for its rows: 546 k / 536 k; LEARNED_BETA 0.5 ... 0.9: 458 k ...
# 530 k (0.8) ... 517 k; PREV_BETA 0.65 ... 0.8: 409 k ... 432 k (0.75) ... 401 k); the
# other learned variants, with the same network and weights, are reported under `modes`
LEARNED = dict(net_rows=2, net_every=3)
LEARNED_BETA = 0.8   # weight of lambda_prev at the learned mode's substeps without the network
PREV_BETA = 0.75     # the previous-multiplier warm start's weight of lambda_prev
TARGET_WARM = 1  # training targets: solves started from SKIP x the previous multipliers
LEARNED_VARIANTS = {"all_every1": dict(net_rows=0, net_every=1), "bilateral_every1": dict(net_rows=1, net_every=1),
                    "bilateral_every2": dict(net_rows=1, net_every=2), "bilateral_every3": dict(net_rows=1, net_every=3),
                    "bilateral_every4": dict(net_rows=1, net_every=4),
                    "all_every4": dict(net_rows=0, net_every=4), "stretch_every1": dict(net_rows=2, net_every=1),
                    "stretch_every2": dict(net_rows=2, net_every=2), "stretch_every3": dict(net_rows=2, net_every=3)}
# Algorithmic FP32 operations of one Jacobi pass per node (segment geometry 29, stretch
# 23, yaw 46, pitch 52, contact + friction 54, update 12; a division, square root or
# transcendental counts as one operation).
FLOP_PER_NODE_PASS = 216
# DRAM bytes per row of the network kernel: ncu (80.80 MB read + 1.98 MB written) over a
# 1,261,356-row launch of the current mlp_infer_kernel
MLP_DRAM_BYTES_PER_ROW = (80.797440e6 + 1.975808e6) / 1261356
# DRAM bytes per node of a split-mode launch of the 32-lane x 3-node solver kernel: ncu
# (8.275712 MB read + 768 B written, a launch of three substeps in steady locomotion,
# features of the stretch rows) over the 93,177 nodes that layout owns in the 4096-snake
# batch (the features it writes are consumed from L2 by the network)
SPLIT_DRAM_BYTES_PER_NODE = (8.275712e6 + 768.0) / 93177
# Minimal HBM bytes of one launch per node (float4 position and velocity read + written,
# six float multipliers read + written), per link (float2 pressures read + written) and
# per snake (96-byte parameters, offsets, residual, update count, status).
BYTES_PER_NODE = 112
BYTES_PER_LINK = 16
BYTES_PER_SNAKE = 116


EVAL_SEED = 4  # the evaluation batch's seed, disjoint from the training seeds (1000+)


def eval_batch(world: int) -> dict:
    """The whole job's batch: N_SNAKES snakes per GPU drawn from one seed."""
    return W.learned(n=N_SNAKES * world, seed=EVAL_SEED)


def shard(w_all: dict, rank: int, world: int) -> dict:
    """This rank's contiguous range of the batch (sim_partition: balanced by node count)."""
    from paper_1904_02833_gb300.sim import partition
    first = partition(w_all, world)
    return W.subset(w_all, np.arange(first[rank], first[rank + 1]))


def device_alu_peak(local: int):
    """FP32 roof of the device: SMs x 128 FP32 lanes x 2 FLOP x the maximum SM clock, with
    the SM count read from the device and the clock from nvidia-smi (else the measured
    peaks file).  Returns (TFLOP/s, description)."""
    import torch
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    mhz = None
    try:
        out = subprocess.run(["nvidia-smi", "-i", str(local), "--query-gpu=clocks.max.sm",
                              "--format=csv,noheader,nounits"], capture_output=True, text=True, timeout=20)
        mhz = float(out.stdout.strip().splitlines()[0])
    except Exception:
        mhz = peaks().get("sm_max_mhz")
    mhz = float(mhz or 2070.0)
    return sms * 128 * 2 * mhz * 1e6 / 1e12, "%d SMs x 128 FP32 lanes x 2 FLOP x %.0f MHz" % (sms, mhz)


def aggregate(t_local: float, units_local: int, dist=None, device="cpu"):
    """Whole-job throughput: the slowest rank's time and the units all ranks processed."""
    import torch
    t = torch.tensor([t_local], dtype=torch.float64, device=device)
    u = torch.tensor([float(units_local)], dtype=torch.float64, device=device)
    if dist is not None and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(u.item()) / float(t.item()), float(t.item()), float(u.item())


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


class Clocks:
    """Samples SM clocks and throttle reasons with nvidia-smi while running."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.p = None
        return self

    def __exit__(self, *a):
        self.lines = []
        if self.p is not None:
            self.p.terminate()
            try:
                out, _ = self.p.communicate(timeout=5)
            except Exception:
                self.p.kill()
                out = ""
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in getattr(self, "lines", []):
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)),
                "reasons": sorted(reasons), "samples": len(sm)}


def run_gpu(args):
    import torch
    import torch.distributed as dist

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if args.net_every < 1:
        raise SystemExit("--net-every must be >= 1")
    skip = float(args.skip)
    lbeta = float(args.learned_beta)
    if not (0.0 <= skip <= 1.0 and 0.0 <= lbeta <= 1.0):
        raise SystemExit("--skip and --learned-beta must lie in [0, 1]")
    # the timed learned warm start: the network's prediction on skip x lambda_prev at its
    # substeps, lbeta x lambda_prev elsewhere
    learned = dict(net_rows=args.net_rows, net_every=args.net_every, beta=lbeta, beta_net=skip)
    if world > 1:
        dist.init_process_group("nccl")
    from paper_1904_02833_gb300.mlp import train_warm_start
    from paper_1904_02833_gb300.sim import SnakeSim

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    # untimed set-up: the warm-start network is trained on solver data (training seeds)
    t_train = time.perf_counter()
    if args.load_net:
        from paper_1904_02833_gb300.mlp import WarmStartMLP
        net, record = WarmStartMLP(np.load(args.load_net)), [{"loaded": args.load_net}]
    else:
        net, record = train_warm_start(n_snakes=args.train_snakes, rounds=args.train_rounds, skip=skip,
                                       target_warm=args.target_warm, settle=max(6, args.settle),
                                       deploy=(dict(net_rows=learned["net_rows"], net_every=learned["net_every"],
                                                    beta=learned["beta"])
                                               if args.train_schedule == "deploy" else None))
    if args.save_net:
        np.save(args.save_net, net.params())
    t_train = time.perf_counter() - t_train

    w_all = eval_batch(world)  # disjoint from the training seeds
    w = shard(w_all, rank, world)
    n_local = len(w["n_links"])
    n_nodes_snake = w["n_links"] * w["seg_per_link"] + 1
    total_nodes = int(n_nodes_snake.sum())
    total_links = int(w["n_links"].sum())
    alu_peak, alu_peak_source = device_alu_peak(local)
    sim = SnakeSim(w, W.solver_settings(iters=CAP, tol=TOL, warm=W_COLD))
    sim.set_mlp(net)
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    # the batch into steady locomotion (plain solver), then the warm-up env-steps
    for _ in range(args.settle + args.warmup):
        sim.step(1, graph=True)
    barrier()
    sim.snapshot_save()

    modes = [("plain", dict(warm=0, beta=1.0)), ("previous", dict(warm=1, beta=args.prev_beta)),
             ("learned", dict(warm=2, **learned))]
    if not args.no_learned_variants:
        # the network on other row kinds and at other periods
        modes += [("learned_" + k, dict(warm=2, beta=lbeta, beta_net=skip, **v))
                  for k, v in LEARNED_VARIANTS.items() if dict(v, beta=lbeta, beta_net=skip) != learned]
    results = {}
    clk_all = None
    layouts = {}
    for name, cfg in modes:
        sim.set_config(**cfg)
        sim.snapshot_restore()
        if not args.no_autotune:
            sim.autotune(1)  # lane layouts per node count for this mode (untimed set-up)
        layouts[name] = {int(N): "%dx%d" % sim.layout(int(N)) for N in np.unique(n_nodes_snake)}
        sim.snapshot_restore()
        sim.step(1, graph=True)  # capture / first replay, untimed
        sim.snapshot_restore()
        barrier()
        l0 = sim.launches()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(args.steps)]
        passes, resid_max, unconv, upd = 0, 0.0, 0, []
        clk = Clocks(local)
        with clk:
            barrier()
            torch.cuda.nvtx.range_push("timed_" + name)  # lets a profiler take the timed steps alone
            for k in range(args.steps):
                flush.zero_()  # L2 (129 MB) flush between timed steps, outside the events
                ev[k][0].record(stream)
                sim.step(1, graph=True)
                ev[k][1].record(stream)
                st = sim.state()
                its = st["iters"].double().cpu().numpy()
                # Jacobi passes: applied updates + the final evaluation of each substep
                passes += int(((its + 20) * n_nodes_snake).sum())
                upd.append(float(its.mean()) / 20)
                resid_max = max(resid_max, float(st["resid"].max()))
                unconv += int((st["resid"] > TOL).sum())
            torch.cuda.nvtx.range_pop()
            barrier()
        ms = [a.elapsed_time(b) for a, b in ev]
        t_local = sum(ms) / 1e3
        value_all, t_max, _ = aggregate(t_local, n_local * args.steps, dist, "cuda")
        results[name] = dict(t=t_max, value=value_all, t_local=t_local, passes=passes, resid_max=resid_max,
                             unconverged=unconv, updates=upd, launches=sim.launches() - l0,
                             clocks=clk.summary(), ms=ms)
        if name == "learned":
            clk_all = clk

    # the network alone, timed on the feature buffer of the batch (CUDA events)
    feat = sim.features()
    rows = feat.shape[0]
    for _ in range(3):
        net.forward(feat)
    import ctypes
    out = torch.empty(rows, device="cuda")
    reps = 10
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_push("network_alone")
    for a, b in evs:
        a.record(stream)
        net.lib.mlp_forward(net.h, ctypes.c_void_p(feat.data_ptr()), rows, ctypes.c_void_p(out.data_ptr()))
        b.record(stream)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    mlp_ms = float(np.median([a.elapsed_time(b) for a, b in evs]))

    # end to end, learned mode, through the public C-ABI with the state in pinned host
    # memory (is_device = 0: the library copies in and out): the same K env-steps from the
    # same start, state copied in and out every step
    sim.set_config(warm=2, **learned)
    sim.snapshot_restore()
    start = sim.state()
    pin = lambda t: t.cpu().pin_memory()
    host = {"pos": pin(start["pos"]), "vel": pin(start["vel"]), "press": pin(start["press"]),
            "lam": pin(sim.lam()), "resid": pin(start["resid"]), "iters": pin(start["iters"])}
    inputs = ("pos", "vel", "press", "lam")
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        sim.set_state_host(*(host[k] for k in inputs))
        sim.step(1, graph=True)
        sim.get_state_host(host["pos"], host["vel"], host["press"], host["lam"], host["resid"], host["iters"])
    torch.cuda.synchronize()
    t_e2e = time.perf_counter() - t0
    e2e_value, _, _ = aggregate(t_e2e, n_local * args.steps, dist, "cuda")
    h2d = int(sum(host[k].numel() * host[k].element_size() for k in inputs))
    d2h = int(sum(v.numel() * v.element_size() for v in host.values()))

    # per-layout kernel times of the learned step (direct launches with an event pair
    # around every solver kernel, on the stream it is launched on), for the roofline of
    # the dominant kernel
    sim.set_config(warm=2, **learned)
    sim.snapshot_restore()
    sim.step(1)
    sim.kernel_times()
    sim.kernel_timing(True)
    kflop = {}
    for _ in range(2):
        sim.step(1)
        its = sim.state()["iters"].double().cpu().numpy()
        for N in np.unique(n_nodes_snake):
            lay = sim.layout(int(N))
            sel = n_nodes_snake == N
            kflop[lay] = kflop.get(lay, 0.0) + FLOP_PER_NODE_PASS * float(((its[sel] + 20) * N).sum())
    ktimes = sim.kernel_times()
    sim.kernel_timing(False)

    solvers = None if args.no_solver_comparison else solver_comparison(args, flush, stream, local)
    calib = None if args.no_calibration else calibration_leg(stream)
    fem = None if args.no_fem else fem_link_leg(flush, stream, alu_peak)
    single = None if args.no_configs else single_snake_leg(stream)
    fixed = None if args.no_configs else fixed_iterations_leg(flush, stream, alu_peak)

    if rank == 0:
        pk = peaks()
        L = results["learned"]
        value = L["value"]
        alu_measured = fp32_peak_measured(stream, local)
        # solver family in the learned mode: Jacobi passes per step x 216 FLOP / time
        # (the network's share of the step is taken out with its own measured time)
        solver_time = L["t_local"] / args.steps - 20 * mlp_ms / 1e3
        family = FLOP_PER_NODE_PASS * L["passes"] / args.steps / solver_time / 1e12
        # the dominant kernel: the lane layout with the most kernel time in the learned step
        dom = max(ktimes, key=lambda k: ktimes[k][0])
        dom_ms, dom_n = ktimes[dom]
        achieved = kflop.get(dom, 0.0) / (dom_ms / 1e3) / 1e12
        dom_nodes = int(sum(int(N) * int((n_nodes_snake == N).sum()) for N in np.unique(n_nodes_snake)
                            if sim.layout(int(N)) == dom))
        traffic = SPLIT_DRAM_BYTES_PER_NODE * dom_nodes if dom == (32, 3) else None
        per_layout = {"%dx%d" % k: {"ms_per_launch": v[0] / v[1], "launches": v[1],
                                    "tflops": kflop.get(k, 0.0) / (v[0] / 1e3) / 1e12}
                      for k, v in sorted(ktimes.items())}
        bytes_step = (BYTES_PER_NODE * total_nodes + BYTES_PER_LINK * total_links
                      + BYTES_PER_SNAKE * n_local)
        mlp_flop_row = 2 * (24 * 128 + 128 * 128 + 128)
        mlp_tflops = mlp_flop_row * rows / (mlp_ms / 1e3) / 1e12
        bf16_peak = pk.get("bf16_tflops", 1900.0)
        modes_out = {}
        for name, _ in modes:
            R = results[name]
            modes_out[name] = {
                "value": R["value"], "ms_per_step": R["t"] * 1e3 / args.steps,
                "updates_per_substep_by_step": [round(u, 2) for u in R["updates"]],
                "ms_by_step": [round(x, 3) for x in R["ms"]],
                "residual_max": R["resid_max"], "unconverged_snake_steps": R["unconverged"],
                "gpu_launches": R["launches"], "clocks": R["clocks"], "layouts": layouts[name]}
        res = {
            "metric": METRIC,
            "value": value,
            "unit": "env-steps/s",
            "n_gpus": world,
            "steps": args.steps,
            "warmup": args.warmup,
            "ms_per_step": L["t"] * 1e3 / args.steps,
            "higher_is_better": True,
            "scaling": "weak",
            "vs_baseline": None,
            "dtype": "f32",
            "data": "synthetic",
            "mode": "learned warm start (network trained on the plain solver's data, disjoint seeds; "
                    "%s rows, network every %d substep(s))" % (("all", "bilateral", "stretch")[learned["net_rows"]],
                                                                learned["net_every"]),
            "learned_config": dict(learned, target_warm=args.target_warm,
                                   train_schedule=args.train_schedule),
            "previous_value": modes_out["previous"]["value"],
            "learned_vs_previous": value / modes_out["previous"]["value"],
            "plain_value": modes_out["plain"]["value"],
            "learned_vs_plain": value / modes_out["plain"]["value"],
            "modes": modes_out,
            "config": workload_config(int(W.n_nodes(w_all).sum()), world, args.settle),
            "l2": "flushed between timed steps (256 MB write)",
            "training": {"seconds": round(t_train, 1), "rounds": record},
            "shard": {"rank": rank, "snakes": n_local, "nodes": total_nodes,
                      "rule": "contiguous snake ranges of one seeded batch, balanced by node count"},
            "roofline": {"bound": "alu", "achieved": achieved, "peak": alu_peak, "unit": "TFLOP/s",
                         "frac": achieved / alu_peak, "traffic": traffic,
                         "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum of one "
                                           "launch on the 4096-snake batch, scaled by the layout's nodes",
                         "kernel": "snake_solver_kernel<%d, %d, 1, 0> (learned mode, %d lanes x %d nodes "
                                   "per lane)" % (dom[1], dom[0], dom[0], dom[1]),
                         "ms_per_launch": dom_ms / dom_n,
                         "timing": "the layouts' launches one after another, an event pair around each; "
                                   "with the batch in steady locomotion a launch lasts as long as its "
                                   "slowest snake (6-13x its class's mean updates per env-step), so this "
                                   "fraction counts the SMs waiting for it; `solver_family` is the same "
                                   "kernels overlapped in the timed step, `fixed_iterations` the pass "
                                   "without slow snakes",
                         "flop_per_node_pass": FLOP_PER_NODE_PASS,
                         "solver_family": {"achieved": family, "frac": family / alu_peak,
                                           "note": "all layout kernels of the learned step, step time "
                                                   "minus the network's"},
                         "per_layout": per_layout,
                         "peak_source": alu_peak_source,
                         "peak_measured": alu_measured,
                         "frac_of_measured": achieved / alu_measured,
                         "peak_measured_source": "sim_fp32_fma_probe: 1216 x 256 threads, 8 independent "
                                                 "FMA chains each, best of 3 launches",
                         "hbm": {"algorithmic_bytes_per_launch": bytes_step,
                                 "peak_gbs": pk.get("hbm_gbs")},
                         "mlp": {"bound": "tensor", "achieved": mlp_tflops, "peak": bf16_peak,
                                 "unit": "TFLOP/s", "frac": mlp_tflops / bf16_peak,
                                 "ms_per_launch": mlp_ms, "rows": rows,
                                 "traffic": MLP_DRAM_BYTES_PER_ROW * rows,
                                 "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum of "
                                                   "one 1,261,356-row launch, scaled by rows",
                                 "peak_source": "MEASURED_PEAKS bf16_tflops (burst, of measured)"}},
            "e2e": {"value": e2e_value, "unit": "env-steps/s",
                    "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "gpu_launches": int(L["launches"]),
            "clocks": clk_all.summary() if clk_all else None,
        }
        if solvers is not None:
            res["solver_comparison"] = solvers
        if calib is not None:
            res["calibration"] = calib
        if single is not None:
            res["single_snake"] = single
        if fixed is not None:
            fixed["roofline"]["peak_measured"] = alu_measured
            fixed["roofline"]["frac_of_measured"] = fixed["roofline"]["achieved"] / alu_measured
            res["fixed_iterations"] = fixed
        if fem is not None:
            fem["roofline"]["peak_measured"] = alu_measured
            fem["roofline"]["frac_of_measured"] = fem["roofline"]["achieved"] / alu_measured
            res["fem_link"] = fem
        if world == 1 and not args.no_cpu_baseline:
            res["cpu_baseline"] = cpu_baseline(w, W.solver_settings(iters=CAP, tol=TOL, warm=W_COLD),
                                               settle=args.settle)
            res["cpu_baseline"]["sample"] += " (the workload's snakes, FP64 oracle)"
        print(json.dumps(res), flush=True)
    sim.close()
    net.close()
    if world > 1:
        dist.destroy_process_group()


W_COLD = 0


def solver_comparison(args, flush, stream, local, n=4096, steps=3):
    """The Jacobi relaxation against the paper's Newton + PCR solve (Sec. IV-D; 20 PCR
    iterations per Newton step), cold and from 0.5 x the previous multipliers, to the same
    residual on a contact-free batch (the gait running, the snakes in free fall): time per
    env-step and updates (Jacobi passes / matrix-vector products) per substep."""
    import torch
    from paper_1904_02833_gb300.sim import SnakeSim
    w = W.batched(n=n, seed=7)
    base = dict(iters=CAP, tol=TOL, contact=False)
    sim = SnakeSim(w, W.solver_settings(**base))
    for _ in range(args.warmup):
        sim.step(1, graph=True)
    sim.snapshot_save()
    out = {"workload": "%d uneven snakes (2-8 links x 10 segments), contact off, residual %g, cap %d"
                       % (n, TOL, CAP), "steps": steps}
    for name, cfg in (("jacobi_cold", dict(solver=0, warm=0, beta=1.0)),
                      ("jacobi_previous", dict(solver=0, warm=1, beta=0.5)),
                      ("newton_pcr_cold", dict(solver=1, warm=0, beta=1.0)),
                      ("newton_pcr_previous", dict(solver=1, warm=1, beta=0.5))):
        sim.set_config(**cfg)
        sim.snapshot_restore()
        sim.step(1, graph=True)
        sim.snapshot_restore()
        ms, upd, rmax = [], [], 0.0
        for _ in range(steps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            sim.step(1, graph=True)
            b.record(stream)
            st = sim.state()
            upd.append(float(st["iters"].double().mean()) / 20)
            rmax = max(rmax, float(st["resid"].max()))
            ms.append(a.elapsed_time(b))
        out[name] = {"ms_per_step": float(np.mean(ms)), "env_steps_per_s": n * steps / (sum(ms) / 1e3),
                     "updates_per_substep": round(float(np.mean(upd)), 2), "residual_max": rmax}
    sim.close()
    return out


# Arithmetic of the soft-link kernel per element, counted from its code (rounded): one
# product with its PCR vector updates (scatter 120, particle sums 14, element rows 145,
# vector updates and dot products 84) and one linearisation (deformation gradient, polar
# iteration, strains, diagonal and right-hand side 500) plus the final M^-1 J^T dlambda
# (130); per substep at one Newton step: 363 x products + 2 x 500 + 130.
FEM_FLOP_PER_ELEMENT_PRODUCT = 363
FEM_FLOP_PER_ELEMENT_SUBSTEP = 2 * 500 + 130
# DRAM bytes of one soft-link launch (ncu: 6.70 MB read, 0 written for 1216 links).
FEM_DRAM_BYTES_PER_LINK = 6.701568e6 / 1216


def fp32_peak_measured(stream, local=0, iters=20000):
    """The library's FMA probe (8 independent chains per thread, 8 blocks of 256 threads per
    SM), best of three timed launches: the measured FP32 roof beside the derived one."""
    import ctypes
    import torch
    from paper_1904_02833_gb300 import _native as N
    L = N.load()
    n_blocks = 8 * torch.cuda.get_device_properties(local).multi_processor_count
    out = torch.empty(n_blocks * 256, dtype=torch.float32, device="cuda")
    args = (ctypes.c_void_p(out.data_ptr()), n_blocks, iters, ctypes.c_void_p(stream.cuda_stream))
    N.check(L.sim_fp32_fma_probe(*args))
    best = None
    for _ in range(3):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        N.check(L.sim_fp32_fma_probe(*args))
        b.record(stream)
        b.synchronize()
        ms = a.elapsed_time(b)
        best = ms if best is None else min(best, ms)
    assert bool(torch.isfinite(out).all().item())
    return n_blocks * 256 * iters * 256 / (best / 1e3) / 1e12


def fem_link_leg(flush, stream, alu_peak, n=1216, frames=10, warmup=3):
    """The tetrahedral soft link (Sec. III-B; the paper's frame: 2 substeps, 20 PCR
    iterations each): a batch of 1216 links (8 per SM) on the 13-cross-section mesh, one
    thread block per link, timed per frame with CUDA events, L2 flushed between frames;
    the FP64 oracle on the host cores on a sample of the batch for comparison."""
    import torch
    from paper_1904_02833_gb300.fem import FemSim
    import oracle.fem as OF
    M = W.fem_link_mesh()
    w = W.fem_links(n, seed=6)
    s = W.fem_settings()
    sim = FemSim(M, w, s)
    sim.step(warmup)
    ms = []
    for _ in range(frames):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        sim.step(1)
        b.record(stream)
        b.synchronize()
        ms.append(a.elapsed_time(b))
    x, v, r, mv = sim.state()
    t = float(np.mean(ms))
    NT = len(M["tets"])
    flop = NT * (FEM_FLOP_PER_ELEMENT_PRODUCT * float(mv.astype(np.float64).sum())
                 + FEM_FLOP_PER_ELEMENT_SUBSTEP * s["n_sub"] * n)
    achieved = flop / (t / 1e3) / 1e12
    cores = os.cpu_count() or 1
    sample = W.fem_links(n, seed=6)
    sel = np.arange(cores)
    o = OF.OracleFem(M, {k: a[sel] for k, a in sample.items()}, s, n_threads=cores)
    t0 = time.perf_counter()
    o.step(2)
    dt_o = time.perf_counter() - t0
    out = {"workload": "%d soft links x %d elements, %d particles, %d distance rows; frame 1/60 s = %d substeps"
                       " x (1 Newton step, %d PCR iterations)" % (n, NT, len(M["X"]), len(M["rows"]),
                                                                  s["n_sub"], s["pcr_iters"]),
           "ms_per_frame": t, "link_frames_per_s": n / (t / 1e3),
           "products_per_substep": float(mv.mean()) / s["n_sub"],
           "residual_mean": float(r.mean()), "residual_max": float(r.max()),
           "roofline": {"bound": "alu", "achieved": achieved, "peak": alu_peak, "unit": "TFLOP/s",
                        "frac": achieved / alu_peak, "traffic": FEM_DRAM_BYTES_PER_LINK * n,
                        "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum of one "
                                          "1216-link launch, scaled by links",
                        "flop_model": "elements x (363 per product + 1130 per substep)"},
           "cpu_oracle": {"link_frames_per_s": len(sel) * 2 / dt_o, "cores": cores,
                          "sample": "%d links x 2 frames (FP64, OpenMP over links)" % len(sel)},
           "paper_context": "Table II: one FEM link 5.70 ms per frame on a GTX 1080 Ti"}
    del sim
    return out


# Jacobi passes per substep at a fixed budget of K updates: K applied passes and the final
# evaluation pass (the residual at the last iterate is measured, its update not applied).
def passes_fixed(K):
    return K + 1


def single_snake_leg(stream, steps=600, calls=120):
    """The paper's real-time setting (the one-snake configuration): one 4-link snake of 41
    nodes, env-steps of 1/60 s with 20 substeps of exactly 10 Jacobi updates.  Timed with
    CUDA events two ways: 600 env-steps in one call (the persistent kernel runs them all),
    and one call per env-step (a captured one-step graph, the way a 60 Hz control loop
    would step it), against the real-time budget of 1/60 s per env-step (Sec. VI); the
    lane layout is autotuned first."""
    import torch
    from paper_1904_02833_gb300.sim import SnakeSim
    w = W.single_snake()
    sim = SnakeSim(w, W.solver_settings(iters=10))
    sim.step(3)
    sim.autotune(1)  # the lane layout with the shortest env-step for this one snake
    sim.step(1, graph=True)  # capture, untimed
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    sim.step(steps)
    b.record(stream)
    b.synchronize()
    batched = a.elapsed_time(b) / steps
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(calls)]
    for e0, e1 in ev:
        e0.record(stream)
        sim.step(1, graph=True)
        e1.record(stream)
    torch.cuda.synchronize()
    per = np.array([e0.elapsed_time(e1) for e0, e1 in ev])
    st = sim.state_host()
    sim_layout = sim.layout(41)
    sim.close()
    budget = 1000.0 / 60.0
    return {"workload": "1 snake x 41 nodes (4 links x 10 segments), 20 substeps x 10 Jacobi updates, "
                        "%d env-steps in one call; %d calls of one env-step" % (steps, calls),
            "ms_per_env_step_batched": batched,
            "ms_per_env_step_per_call": {"median": float(np.median(per)), "p99": float(np.percentile(per, 99)),
                                         "max": float(per.max())},
            "layout": "%dx%d" % sim_layout, "realtime_budget_ms": budget,
            "realtime_factor_per_call": budget / float(np.median(per)),
            "updates_per_substep": float(st["iters"][0]) / 20, "finite": bool(np.isfinite(st["pos"]).all()),
            "paper_context": "Table II: one snake, 1/60 s frames, real time on a GTX 1080 Ti"}


def fixed_iterations_leg(flush, stream, alu_peak, n=4096, steps=600, K=10):
    """Batched locomotion at a fixed budget (the 4096-snake configuration): uneven snakes of
    2-8 links, 20 substeps of exactly 10 Jacobi updates, 600 env-steps, lane layouts chosen
    by sim_autotune, the 600 env-steps replayed as one captured CUDA graph (one persistent
    kernel per layout).  env-steps/s, and the ALU roofline of the whole replay (every
    snake runs the same passes, so no tail of slow snakes)."""
    import torch
    from paper_1904_02833_gb300.sim import SnakeSim
    w = W.batched(n=n, seed=3)
    sim = SnakeSim(w, W.solver_settings(iters=K))
    sim.step(3)
    sim.autotune(1)
    sim.snapshot_save()
    sim.step(steps, graph=True)  # capture and first replay, untimed
    sim.snapshot_restore()
    flush.zero_()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    sim.step(steps, graph=True)
    b.record(stream)
    b.synchronize()
    t = a.elapsed_time(b) / 1e3
    st = sim.state_host()
    layouts = {int(N): "%dx%d" % sim.layout(int(N)) for N in np.unique(W.n_nodes(w))}
    sim.close()
    nodes = int(W.n_nodes(w).sum())
    flop = FLOP_PER_NODE_PASS * passes_fixed(K) * 20 * nodes * steps
    achieved = flop / t / 1e12
    return {"workload": "%d uneven snakes (2-8 links x 10 segments, %d nodes), 20 substeps x %d Jacobi updates, "
                        "%d env-steps in one graph replay, autotuned layouts" % (n, nodes, K, steps),
            "env_steps_per_s": n * steps / t, "ms_per_env_step": t * 1e3 / steps,
            "layouts": layouts, "updates_per_substep": float(st["iters"].mean()) / 20,
            "finite": bool(np.isfinite(st["pos"]).all()),
            "roofline": {"bound": "alu", "achieved": achieved, "peak": alu_peak, "unit": "TFLOP/s",
                         "frac": achieved / alu_peak,
                         "flop_model": "216 FLOP per node and pass x 11 passes per substep (10 updates + the "
                                       "final evaluation) x 20 substeps x nodes x env-steps"}}


def calibration_leg(stream, n=1024, steps=200, ckpt=20):
    """The differentiable calibration rollout: 1024 four-link snakes, 200 env-steps of 20
    substeps with 10 Jacobi updates each, checkpoints every 20 env-steps; the forward
    rollout and the adjoint (backward) pass of a mean squared tip-trajectory loss against
    a ground-truth rollout, timed with CUDA events."""
    import torch
    from paper_1904_02833_gb300.calib import rollout, theta_of
    from paper_1904_02833_gb300.sim import SnakeSim
    truth, guess = W.calibration(n=n, seed=5)
    s = W.solver_settings(iters=10)
    gt = SnakeSim(truth, s)
    gt.step(1)
    with torch.no_grad():
        target = rollout(gt, theta_of(truth).cuda(), steps, ckpt)
    sim = SnakeSim(guess, s)
    sim.step(1)
    sim.snapshot_save()
    th = theta_of(guess).cuda().requires_grad_(True)
    # full-length warm-up of exactly the timed computation (buffers sized, every kernel,
    # the loss's included, loaded and launched once)
    ((rollout(sim, th, steps, ckpt) - target) ** 2).sum(-1).mean(0).sum().backward()
    sim.snapshot_restore()
    th.grad = None
    e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    e[0].record(stream)
    tips = rollout(sim, th, steps, ckpt)
    loss = ((tips - target) ** 2).sum(-1).mean(0).sum()
    e[1].record(stream)
    loss.backward()
    e[2].record(stream)
    torch.cuda.synchronize()
    fwd, bwd = e[0].elapsed_time(e[1]), e[1].elapsed_time(e[2])
    g = th.grad
    out = {"workload": "%d snakes x 41 nodes, %d env-steps x 20 substeps x 10 updates, checkpoints every %d"
                       % (n, steps, ckpt),
           "forward_ms": fwd, "backward_ms": bwd,
           "env_steps_per_s_forward": n * steps / (fwd / 1e3),
           "env_steps_per_s_forward_backward": n * steps / ((fwd + bwd) / 1e3),
           "gradient_finite": bool(torch.isfinite(g).all().item()), "loss": float(loss.item())}
    sim.close()
    gt.close()
    return out


def oracle_settled(oracle, w, s, n_threads, settle):
    """The oracle on batch w after `settle` untimed plain env-steps (the benchmark's
    steady-locomotion start)."""
    o = oracle.OracleSim(w, s, n_threads=n_threads)
    if settle > 0:
        o.step(settle)
    return o


def cpu_baseline(w, s, n_sample=None, budget_s=20.0, settle=SETTLE):
    """The FP64 oracle on the host cores, on a bounded sample of the same batch, from the
    same settled state."""
    import oracle
    cores = os.cpu_count() or 1
    rng = np.random.default_rng(123)
    n_sample = n_sample or 2 * cores
    sel = np.sort(rng.choice(len(w["n_links"]), n_sample, replace=False))
    o = oracle_settled(oracle, W.subset(w, sel), s, cores, settle)
    # the same oracle on one host core, on the first few of those snakes in the same state
    n1 = max(1, min(4, n_sample))
    o1 = oracle.OracleSim(W.subset(w, sel[:n1]), s, n_threads=1)
    nodes, links = slice(0, int(o.node_off[n1])), slice(0, int(o.link_off[n1]))
    o1.x[:], o1.v[:], o1.lam[:] = o.x[nodes], o.v[nodes], o.lam[nodes]
    o1.press[:] = o.press[links]
    o1.step_index = o.step_index
    t0 = time.perf_counter()
    steps = 0
    while True:
        o.step(1)
        steps += 1
        if time.perf_counter() - t0 > budget_s / 2 or steps >= 8:
            break
    dt = time.perf_counter() - t0
    t1 = time.perf_counter()
    o1.step(1)
    dt1 = time.perf_counter() - t1
    return {"value": n_sample * steps / dt, "unit": "env-steps/s", "cores": cores, "kind": "oracle",
            "sample": "%d snakes drawn from the batch x %d env-steps after %d untimed settling env-steps "
                      "(FP64, OpenMP over snakes), %.1f s" % (n_sample, steps, settle, dt),
            "single_thread": {"value": n1 / dt1, "unit": "env-steps/s", "cores": 1,
                              "sample": "%d of those snakes x 1 env-step, %.1f s" % (n1, dt1)}}


def workload_config(total_nodes, world, settle):
    """The benchmark's workload, the same dict in both arms (total_nodes: the whole job's
    batch of N_SNAKES x world snakes)."""
    return {"workload": "%d uneven snakes per GPU (2-8 links x 10 segments), dt 1/60 s, 20 substeps, Jacobi"
                        " to residual %g (cap %d updates/substep), in steady locomotion (%d plain env-steps"
                        " from the straight resting pose before timing); %d GPU(s), one seeded batch split"
                        " into contiguous node-balanced ranges" % (N_SNAKES, TOL, CAP, settle, world),
            "snakes_per_gpu": N_SNAKES, "nodes_per_gpu": round(total_nodes / world, 1),
            "settle_steps": settle,
            "parallelism": "independent snakes per GPU (dp%d)" % world}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle
    w_all = eval_batch(world)
    s = W.solver_settings(iters=CAP, tol=TOL, warm=W_COLD)
    cores = os.cpu_count() or 1
    rng = np.random.default_rng(7)
    n_sample = cores
    sel = np.sort(rng.choice(len(w_all["n_links"]), n_sample, replace=False))
    o = oracle_settled(oracle, W.subset(w_all, sel), s, cores, args.settle)
    for _ in range(args.warmup):
        o.step(1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        o.step(1)
    dt = time.perf_counter() - t0
    value = n_sample * args.steps / dt
    sample = ("%d snakes drawn from the %d-snake batch, 1 env-step per timed step after %d untimed "
              "settling env-steps (FP64 oracle, OpenMP)" % (n_sample, len(w_all["n_links"]), args.settle))
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": "env-steps/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": dt * 1e3 / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(int(W.n_nodes(w_all).sum()), world, args.settle),
        "reference_sample": sample,
        "cpu_baseline": {"value": value, "unit": "env-steps/s", "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "env-steps/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }), flush=True)


def main():
    global N_SNAKES
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--settle", type=int, default=SETTLE,
                    help="untimed plain env-steps from the resting pose before the warm-up steps")
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-solver-comparison", action="store_true",
                    help="skip the Jacobi vs Newton + PCR leg (contact-free batch)")
    ap.add_argument("--no-calibration", action="store_true",
                    help="skip the differentiable calibration leg (forward + adjoint)")
    ap.add_argument("--no-fem", action="store_true",
                    help="skip the tetrahedral soft-link leg")
    ap.add_argument("--target-warm", type=int, default=TARGET_WARM, choices=[0, 1],
                    help="start of the solves that make the network's training targets: 0 cold, "
                         "1 beta x the previous multipliers")
    ap.add_argument("--no-learned-variants", action="store_true",
                    help="time only the headline learned configuration (not its variants)")
    ap.add_argument("--net-rows", type=int, default=LEARNED["net_rows"], choices=[0, 1, 2],
                    help="row kinds of the timed learned warm start: 0 all, 1 bilateral, 2 stretch")
    ap.add_argument("--net-every", type=int, default=LEARNED["net_every"],
                    help="the timed learned warm start runs the network every this many substeps")
    ap.add_argument("--skip", type=float, default=SKIP,
                    help="weight of lambda_prev under the network's prediction "
                         "(lambda0 = skip lambda_prev + m g h^2 y)")
    ap.add_argument("--learned-beta", type=float, default=LEARNED_BETA,
                    help="weight of lambda_prev at the learned mode's substeps without the network")
    ap.add_argument("--prev-beta", type=float, default=PREV_BETA,
                    help="beta of the previous-multiplier warm start (lambda0 = beta lambda_prev)")
    ap.add_argument("--train-rounds", type=int, default=2,
                    help="on-policy training rounds after the cold-start round")
    ap.add_argument("--train-snakes", type=int, default=2048, help="snakes per training batch")
    ap.add_argument("--train-schedule", default="deploy", choices=["all", "deploy"],
                    help="row kinds and period of the network on the learned training trajectories: "
                         "every row and substep, or the timed configuration (--net-rows, --net-every)")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the default lane layouts instead of timing them per mode (sim_autotune)")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the single-snake and fixed-iteration (4096 snakes) legs")
    ap.add_argument("--save-net", default=None, help="write the trained network parameters (.npy)")
    ap.add_argument("--load-net", default=None, help="use saved network parameters instead of training")
    ap.add_argument("--snakes", type=int, default=N_SNAKES,
                    help="batch size per GPU (smaller batches for profiler captures)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    N_SNAKES = args.snakes
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
