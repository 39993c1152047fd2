"""Benchmark of the coupled LB-FEM step on GB300.

Workload: two R=12 level-4 capsules (2562 nodes each) at centre distance 3R in
a 128x64x64 lattice with a substrate, film height 0.6R, FP32 populations.  One
bench step = one coupled time step (streaming with bounce-back and Ladd
exchange, Shan-Chen forces with decoupling, BGK, membrane forces, node
update, cut-link rebuild).  Metric: coupled MLUPS = nodes x steps / s / 1e6.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
  python bench.py --sweep [--steps K]      # batched distance x softness sweep
  python bench.py --warm                   # learned warm start vs flat film
  python bench.py --drying --precision fp16  # drying film, 16 capsules, 256x256x96

--drying measures the mixed-precision drying film instead: a 256x256x96
lattice with 16 R=10 capsules on a seeded random layout, the film lowered by a
steady conversion of A into B (0.6R to 0.2R over 50k steps).

--sweep measures the batched step instead: 64 independent lattices of uneven
size (147k-819k nodes, two capsules each, 16 distances x 4 moduli) stepped
together after the autotuner has picked the launch shape, against the same
lattices stepped one by one.

Under torchrun (N > 1) every rank runs an independent replica of the workload
(weak scaling: no data-path collective); time = max over ranks.
"""
import argparse
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

ALG_BYTES_PER_LU = 2 * 19 * 2 * 4  # two components x 19 populations x (read + write) x float32
# 16-bit storage: 18 moving populations x 2 B + the float rest population, per component
ALG_BYTES_PER_LU_16 = 2 * (18 * 2 + 4) * 2
PRECISIONS = {"fp32": 0, "fp16": 1, "bf16": 2}
METRIC = "coupled LB+IBM MLUPS (% HBM roofline)"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=200)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-sample-steps", type=int, default=None)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--precision", default="fp32", choices=sorted(PRECISIONS),
                    help="population storage (arithmetic is float32 in every mode)")
    ap.add_argument("--sweep", action="store_true",
                    help="batched 64-lattice sweep instead of the capsule pair")
    ap.add_argument("--tune-steps", type=int, default=8)
    ap.add_argument("--warm", action="store_true",
                    help="train the warm-start network and measure its gain on held-out set-ups")
    ap.add_argument("--sweep-n", type=int, default=16,
                    help="distances of the sweep (x 4 moduli lattices)")
    ap.add_argument("--drying", action="store_true",
                    help="drying film with 16 capsules (256x256x96) instead of the capsule pair")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except FileNotFoundError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([v.strip() for v in line.split(",")])

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[0]))
                mx = float(r[1])
                for k, nm in enumerate(names):
                    if r[3 + k].lower() == "active":
                        reasons.add(nm)
            except (ValueError, IndexError):
                continue
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def profiled_traffic():
    """DRAM bytes per step of the two lattice passes from the committed ncu
    summary, if it was taken on the current kernel source (else None)."""
    import hashlib
    try:
        txt = open(os.path.join(ROOT, "profiles", "lattice_passes_capsule_pair.md")).read()
        src = open(os.path.join(ROOT, "paper_2007_15405_gb300", "csrc", "lb_kernel.cu"), "rb").read()
    except OSError:
        return None
    sha = hashlib.sha256(src).hexdigest()[:16]
    t = h = None
    for line in txt.splitlines():
        if line.startswith("traffic_bytes_per_step:"):
            t = int(line.split(":")[1])
        if line.startswith("lb_kernel.cu sha256[:16]:"):
            h = line.rsplit(":", 1)[1].strip()
    return t if (t is not None and h == sha) else None


def measured_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def cpu_baseline(wl, steps):
    """The FP64 oracle as it stands, on the host cores, on a bounded sample:
    `steps` time steps of the full workload."""
    import oracle as O
    o = O.Oracle.from_workload(wl)
    o.step(1)  # warm-up (first-touch of the arrays)
    t = time.perf_counter()
    o.step(steps)
    dt = time.perf_counter() - t
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return {"value": wl.nodes * steps / dt / 1e6, "unit": "MLUPS", "cores": cores, "kind": "oracle",
            "sample": f"{steps} coupled steps of the full {wl.nx}x{wl.ny}x{wl.nz} workload "
                      f"({dt:.1f} s, FP64, OpenMP over lattice planes)"}


def workload(args=None):
    from paper_2007_15405_gb300 import inputs as I
    if args is not None and args.drying:
        return I.drying_film()
    return I.capsule_pair(steps=20000)


def config_of(wl, world, l2note):
    if wl.dry_dm > 0.0:
        desc = (f"drying film: {wl.nx}x{wl.ny}x{wl.nz} lattice, substrate, {len(wl.capsules)} R=10 "
                f"level-4 capsules (2562 nodes / 5120 elements each) on a seeded random layout, "
                f"film lowered from 0.6R to 0.2R over 50k steps by converting {wl.dry_dm:.4f} of A "
                f"into B per step, free capsules")
    else:
        desc = ("capsule pair: 128x64x64 lattice, substrate, two R=12 level-4 capsules "
                "(2562 nodes / 5120 elements each) at d=3R, film 0.6R, free capsules")
    return {"workload": desc,
            "lattice": [wl.nx, wl.ny, wl.nz], "capsules": len(wl.capsules), "nodes": wl.nodes,
            "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
            "l2": l2note}


def l2_note(ws):
    rel = "exceeds" if ws > 129e6 else "does not exceed"
    return f"no flush: per-step working set {ws / 1e6:.0f} MB of populations (src + dst) {rel} the 129 MB L2"


def max_over_ranks(x, device="cpu"):
    """The largest x over the ranks of the process group (x itself alone)."""
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist = torch.distributed
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_mlups(nodes, steps, world, seconds):
    """Whole-job throughput: the node updates of all ranks (each rank runs its
    own replica) over the slowest rank's time."""
    return nodes * steps * world / seconds / 1e6


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    wl = workload(args)
    steps_per = args.cpu_sample_steps or 2
    import oracle as O
    o = O.Oracle.from_workload(wl)
    for _ in range(args.warmup):
        o.step(steps_per)
    t = time.perf_counter()
    for _ in range(args.steps):
        o.step(steps_per)
    dt = time.perf_counter() - t
    val = wl.nodes * steps_per * args.steps / dt / 1e6
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "MLUPS", "n_gpus": 0,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": dt / (args.steps * steps_per) * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_of(wl, 1, "host CPU"),
            "cpu_baseline": {"value": val, "unit": "MLUPS", "cores": cores, "kind": "oracle",
                             "sample": f"each bench step = {steps_per} oracle time steps of the "
                                       f"full workload"},
            "e2e": {"value": val, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args):
    import torch
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    from paper_2007_15405_gb300 import build as B
    if rank == 0:
        B.build()
    if world > 1:
        torch.distributed.barrier()
    from paper_2007_15405_gb300 import capfilm as cfm

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    wl = workload(args)
    prec = PRECISIONS[args.precision]
    alg_bytes = ALG_BYTES_PER_LU if prec == 0 else ALG_BYTES_PER_LU_16
    sim = cfm.Simulation.from_workload(wl, precision=prec)
    stream = sim.stream  # the events must be recorded on the stream the steps run on
    # warm-up
    sim.step(args.warmup)
    sim.sync()
    # ---- device-resident throughput: K steps through cf_step (graph replay)
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    sim.step(args.steps)
    e1.record(stream)
    e1.synchronize()
    launches = sim.launches()
    barrier()
    ms = e0.elapsed_time(e1)
    clk = clocks.stop()
    sim.sync()
    ms_max = max_over_ranks(ms, "cuda")
    value = job_mlups(wl.nodes, args.steps, world, ms_max / 1e3)
    # ---- per-phase device time (lattice kernel, membrane phase, cut links)
    nprof = min(200, max(20, args.steps // 10))
    ph = sim.time_phases(nprof)
    lb_ms = ph[0]
    peak, peak_kind = measured_peak()
    achieved = alg_bytes * wl.nodes / (lb_ms / 1e3) / 1e9
    # ---- end to end through the public API with host buffers
    from paper_2007_15405_gb300.inputs import RHO_MAJ, RHO_MIN, RHO_MIX
    jit = wl.jitter()
    jit_pinned = torch.from_numpy(jit.reshape(-1)).pin_memory().numpy()
    sample_every = 100
    nsamp = max(1, args.steps // sample_every)
    barrier()
    t0 = time.perf_counter()
    sim.set_film(wl.h_top, RHO_MAJ, RHO_MIN, RHO_MIX, jit_pinned)
    forces = []
    for _ in range(nsamp):
        sim.step(sample_every)
        forces.append(sim.lateral_force(0, 1))
    barrier()
    t_e2e = max_over_ranks(time.perf_counter() - t0, "cuda")
    e2e_steps = nsamp * sample_every
    e2e_val = job_mlups(wl.nodes, e2e_steps, world, t_e2e)
    h2d = jit.nbytes / e2e_steps
    d2h = 16 * 8 * len(wl.capsules) * nsamp / e2e_steps
    sim.close()
    if world > 1:
        torch.distributed.destroy_process_group()
    if rank != 0:
        return
    cpu = None
    if not args.no_cpu_baseline and world == 1:
        # about 10-20 s of oracle work on 16 host cores
        cpu = cpu_baseline(wl, args.cpu_sample_steps or max(2, int(5.2e7 // wl.nodes)))
    line = {
        "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": config_of(wl, world, l2_note(alg_bytes * wl.nodes)),
        "roofline": {"bound": "hbm", "kernel": "lattice update: k_density + k_collide_eq (tau = 1)",
                     "achieved": achieved, "peak": peak,
                     "peak_kind": f"{peak_kind} copy bandwidth (burst)", "unit": "GB/s",
                     "frac": achieved / peak,
                     "traffic": profiled_traffic() if prec == 0 else None,
                     "algorithmic_bytes_per_launch": alg_bytes * wl.nodes,
                     "kernel_ms": lb_ms},
        "phases_ms": {"lattice": ph[0], "membrane": ph[1], "cut_links": ph[2], "bounce_prep": ph[3]},
        "clocks": clk,
        "e2e": {"value": e2e_val, "unit": "MLUPS", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h,
                "note": f"film set-up from pinned host jitter, {e2e_steps} steps, lateral force "
                        f"read back every {sample_every} steps"},
        "gpu_launches": launches,
        "cpu_baseline": cpu,
    }
    line["config"]["population_storage"] = args.precision
    print(json.dumps(line), flush=True)


def run_sweep(args):
    import torch
    from paper_2007_15405_gb300 import build as B
    B.build()
    from paper_2007_15405_gb300 import capfilm as cfm
    from paper_2007_15405_gb300 import inputs as I
    torch.cuda.set_device(0)
    prec = PRECISIONS[args.precision]
    wls = I.batched_sweep(n_dist=args.sweep_n)
    nodes = sum(w.nodes for w in wls)
    sims = [cfm.Simulation.from_workload(w, precision=prec) for w in wls]
    batch = cfm.Batch(sims)
    t0 = time.perf_counter()
    cfg = batch.autotune(steps=args.tune_steps)
    t_tune = time.perf_counter() - t0
    batch.step(max(3, args.warmup))
    clocks = ClockSampler(0)
    clocks.start()
    time.sleep(0.3)
    ms = batch.time(args.steps)
    launches = batch.launches()
    clk = clocks.stop()
    value = nodes * args.steps / (ms / 1e3) / 1e6
    # the same lattices stepped one after the other (each replaying its own graph)
    k = max(4, min(args.steps, 40))
    seq_ms = 0.0
    for s in sims:
        s.step(3)
        s.sync()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(s.stream)
        s.step(k)
        e1.record(s.stream)
        e1.synchronize()
        seq_ms += e0.elapsed_time(e1)
    seq_value = nodes * k / (seq_ms / 1e3) / 1e6
    batch.close()
    line = {
        "metric": "batched sweep coupled MLUPS", "value": value, "unit": "MLUPS", "n_gpus": 1,
        "steps": args.steps, "warmup": max(3, args.warmup), "ms_per_step": ms / args.steps,
        "higher_is_better": True, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"{len(wls)} lattices 64x48x48..160x80x64 ({nodes} nodes), two R=8 "
                               "level-3 capsules each, d in [2.2R, 6R] x kS in {1e-3, 1e-2, 1e-1, rigid}",
                   "population_storage": args.precision,
                   "l2": f"no flush: per-step working set {nodes * 304 / 1e9:.1f} GB of populations "
                         "exceeds the 129 MB L2"},
        "autotune": dict(cfg, seconds=t_tune),
        "one_by_one": {"value": seq_value, "unit": "MLUPS", "steps": k},
        "speedup_vs_one_by_one": value / seq_value,
        "clocks": clk, "gpu_launches": launches,
    }
    print(json.dumps(line), flush=True)


def run_warm(args):
    import torch
    from paper_2007_15405_gb300 import build as B
    B.build()
    from paper_2007_15405_gb300 import inputs as I
    from paper_2007_15405_gb300 import warm
    torch.cuda.set_device(0)
    # fixed capsules: their capillary force settles when the film does, so
    # the time to 1% of the equilibrium force is well defined
    n_train, n_test, eq_steps, total, every = 48, 32, 3000, 8000, 50
    t0 = time.perf_counter()
    X, T, M = warm.dataset(I.warm_dataset(n_train, seed=11, mode=I.MODE_FIXED), eq_steps)
    t_data = time.perf_counter() - t0
    net = warm.WarmNet(seed=0)
    t0 = time.perf_counter()
    losses = warm.train(net, X, T, M, steps=400, batch=8, lr=2e-3)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    test = I.warm_dataset(n_test, seed=99, mode=I.MODE_FIXED)
    err_p, err_w = [], []
    Xh, Th, Mh = warm.dataset(test, eq_steps)
    for k in range(n_test):
        pred = net.predict(Xh[k])
        err_p.append(float(np.sqrt((Th[k] ** 2 * Mh[k]).sum() / Mh[k].sum())))
        err_w.append(float(np.sqrt(((pred - Th[k]) ** 2 * Mh[k]).sum() / Mh[k].sum())))
    res, timing = warm.convergence(net, test, total=total, every=every)
    sp = [r[0] for r in res]
    sw = [r[1] for r in res]
    both = [(a, b) for a, b in zip(sp, sw) if a is not None and b is not None]
    line = {
        "metric": "steps to capsule force within 1% of equilibrium, learned warm start vs flat film",
        "unit": "steps", "higher_is_better": False, "data": "synthetic", "dtype": "bf16 network / f32 lattice",
        "config": {"workload": f"{n_test} held-out lattices 48x32x32, one fixed capsule R in [5, 7] "
                               "(level 3), film 0.3R..0.9R above the repulsive plane; network trained on "
                               f"{n_train} equilibria of {eq_steps} steps; settling judged over {total} "
                               f"steps sampled every {every}"},
        "network": {"params": net.n_params, "train_steps": len(losses), "loss_first": losses[0],
                    "loss_last": losses[-1], "train_seconds": t_train, "data_seconds": t_data},
        "density_rms_error": {"flat_film": float(np.mean(err_p)), "warm": float(np.mean(err_w)),
                              "unit": "(rho_maj - rho_min), against the equilibria"},
        "settle_steps": {"flat_film_mean": float(np.mean([a for a, _ in both])) if both else None,
                         "warm_mean": float(np.mean([b for _, b in both])) if both else None,
                         "pairs": len(both), "flat_film_unsettled": sum(a is None for a in sp),
                         "warm_unsettled": sum(b is None for b in sw)},
        "fallbacks": sum(not r[2] for r in res),
        "time_to_force_seconds": ({
            "flat_film": float(np.mean([a for a, _ in both])) * timing["step_seconds"],
            "warm": float(np.mean([b for _, b in both])) * timing["step_seconds"] + timing["warm_start_seconds"],
            "step_seconds_per_lattice": timing["step_seconds"],
            "warm_start_seconds": timing["warm_start_seconds"],
            "note": f"per lattice within a batch of {n_test}; the warm start (inference, predicted state, "
                    "51 judging steps run alone) is counted, the offline training is not"} if both else None),
        "value": float(np.mean([b for _, b in both])) if both else None,
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.warm:
        run_warm(args)
        return
    if args.sweep:
        run_sweep(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
