#!/usr/bin/env python
"""Throughput of the three-phase colour-gradient LBM step (arXiv:2102.04709) on one GB300.

One "step" is one timestep of the whole hot path: the wetting pass over the solid boundary
nodes (Eq.21-22) and the fused step kernel (Eq.1-16).  The workload is the compound droplet
through 60 seeded pillars on a 4096 x 2048 D2Q9 grid (Section III.D), FP32 populations;
inputs (2 x 0.9 GB of populations) are larger than L2, so no flush is needed.

Prints ONE JSON line (rank 0):  value = whole-job MLUPS (grid nodes x steps / s / 1e6).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the FP64 CPU oracle (the only reference this paper has) on the box's
host cores (OpenMP), one 512 x 512 window of the same workload per step.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

FALLBACK_HBM_GBS = 6800.0
E2E_LONG = 2000   # steps of the second end-to-end timing when the run itself is shorter
PRECISIONS = {"fp32": 0, "fp16": 1, "bf16": 2}
WORKLOAD = "pillars_4096x2048_theta90"
REF_WINDOW = 512


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--theta", type=float, default=90.0)
    ap.add_argument("--workload", choices=["pillars_4096x2048", "pillars_2048x1024", "five_pillars_800x375"],
                    default="pillars_4096x2048",
                    help="the half-size case exists for detailed kernel profiles; five_pillars_800x375 "
                         "is the paper's own Section III.D set-up (wall triple (90, 180 - theta, theta))")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--precision", choices=["fp32", "fp16", "bf16"], default="fp32",
                    help="population storage of the headline run")
    ap.add_argument("--no-alt-storage", action="store_true",
                    help="skip the extra FP16 / BF16 storage timings")
    ap.add_argument("--no-adjoint", action="store_true",
                    help="skip the adjoint timing (512 x 256, 6 pillars, 2000 steps)")
    return ap.parse_args()


def max_over_ranks(x, ws, device):
    """Largest x over the ranks of the default process group (x itself with one rank): the
    whole job takes as long as its slowest replica."""
    if ws <= 1:
        return float(x)
    import torch
    t = torch.tensor([float(x)], device=device, dtype=torch.float64)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def job_mlups(nodes, steps, ws, ms):
    """Whole-job throughput: the grid nodes that all ws replicas advanced, per second of the
    slowest replica, in millions."""
    return nodes * steps * ws / (ms * 1e-3) / 1e6


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# ------------------------------------------------------------------------------------------
# clocks during the timed region
# ------------------------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("timestamp", "clocks.sm", "clocks.max.sm", "power.draw",
              "clocks_event_reasons.active", "clocks_event_reasons.hw_slowdown",
              "clocks_event_reasons.hw_thermal_slowdown", "clocks_event_reasons.sw_thermal_slowdown",
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.samples = []
        self.proc = None
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(device_index), "--query-gpu=" + ",".join(self.FIELDS),
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) == len(self.FIELDS):
                self.samples.append((time.time(), parts))

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self, t0, t1):
        sel = [s for (t, s) in self.samples if t0 <= t <= t1]
        window = "timed region"
        if not sel:
            sel = [s for (_, s) in self.samples[-5:]]
            window = "nearest samples (timed region shorter than the sampling period)"
        if not sel:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}

        def num(v):
            try:
                return float(v)
            except ValueError:
                return None
        sm = [num(s[1]) for s in sel if num(s[1]) is not None]
        smax = [num(s[2]) for s in sel if num(s[2]) is not None]
        pw = [num(s[3]) for s in sel if num(s[3]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[j] for s in sel for j in range(4) if s[5 + j].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "power_w": statistics.median(pw) if pw else None,
                "reasons": reasons, "samples": len(sel), "window": window}


def measured_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        for key in ("hbm_gbs", "hbm_GBs", "hbm"):
            if key in d and isinstance(d[key], (int, float)):
                return float(d[key]), "measured (MEASURED_PEAKS.json hbm_gbs)"
    except (OSError, ValueError):
        pass
    return FALLBACK_HBM_GBS, "fallback 6.8 TB/s (no MEASURED_PEAKS.json)"


KERNEL_SOURCES = ("lbm3_step.cu", "lbm3_common.cuh", "lbm3_device.cuh")


def kernel_source_hash():
    """First 16 hex digits of the SHA-256 of the step kernels' sources."""
    h = hashlib.sha256()
    for name in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_2102_04709_gb300", "csrc", name), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_traffic(pure_nodes):
    """DRAM bytes of one pure-tile launch from the committed ncu summary, if it was taken on the
    current kernel sources (hash match), scaled to this workload's pure-tile nodes."""
    path = os.path.join(ROOT, "profiles", "k_step_f32_traffic.txt")
    try:
        d = {}
        with open(path) as fh:
            for line in fh:
                if ":" in line and not line.startswith("#"):
                    k, v = line.split(":", 1)
                    d[k.strip()] = v.strip()
        if d.get("source_sha256_16") != kernel_source_hash():
            return None
        return float(d["dram_bytes_per_pure_node"]) * pure_nodes
    except (OSError, ValueError, KeyError):
        return None


# ------------------------------------------------------------------------------------------
# CPU oracle timing
# ------------------------------------------------------------------------------------------
def oracle_window(w, x0, y0, size):
    """A size x size window of workload w, periodic on both sides (same per-node work)."""
    from paper_2102_04709_gb300 import workloads as W
    sl = (slice(y0, y0 + size), slice(x0, x0 + size))
    return W.Workload(f"{w.name}_window{size}", size, size, 1, W.BC_PERIODIC,
                      w.solid[sl].copy(), w.rho[:, sl[0], sl[1]].copy(), w.angles[sl].copy(),
                      w.sigma, w.nu, w.beta0)


def cpu_baseline(w, steps_all=8, steps_one=2):
    """The FP64 oracle on full timesteps of the whole workload: on every host core (OpenMP over
    the per-node loops; the headline figure) and on one core."""
    from oracle import oracle as ora
    cores = ora.host_threads()
    o = ora.Oracle.from_workload(w, threads=cores)
    o.step(1)                                   # first touch of the arrays on every thread
    t = time.perf_counter()
    o.step(steps_all)
    dt_all = time.perf_counter() - t
    o.set_threads(1)
    t = time.perf_counter()
    o.step(steps_one)
    dt_one = time.perf_counter() - t
    return {"value": w.n * steps_all / dt_all / 1e6, "unit": "MLUPS", "cores": cores, "kind": "oracle",
            "sample": f"{steps_all} full timesteps of {w.name} ({w.nx}x{w.ny}) by the FP64 oracle on "
                      f"{cores} OpenMP threads, {dt_all:.1f} s; then {steps_one} on one core, {dt_one:.1f} s",
            "single_core_value": w.n * steps_one / dt_one / 1e6}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    from oracle import oracle as ora
    from paper_2102_04709_gb300 import workloads as W
    ora.build()
    w = W.config4(args.theta)
    # a 512 x 512 window holding the droplet's front and pillars, periodic on both sides (the
    # same work per node as the full grid), on every host core
    win = oracle_window(w, 400, 768, REF_WINDOW)
    cores = ora.host_threads()
    o = ora.Oracle.from_workload(win, threads=cores)
    o.step(args.warmup)
    t = time.perf_counter()
    o.step(args.steps)
    dt = time.perf_counter() - t
    v = win.n * args.steps / dt / 1e6
    line = {"impl": "reference", "metric": "MLUPS", "value": v, "unit": "MLUPS", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample": f"{REF_WINDOW}x{REF_WINDOW} window of the "
                                                          "workload per step",
                       "storage": "fp64 (oracle)"},
            "cpu_baseline": {"value": v, "unit": "MLUPS", "cores": cores, "kind": "oracle",
                             "sample": f"one timestep of a {REF_WINDOW}x{REF_WINDOW} window of the "
                                       f"pillar workload per step, FP64 oracle on {cores} OpenMP "
                                       "threads"},
            "e2e": {"value": v, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "gpu_launches": 0}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------------------------------
# GPU arm
# ------------------------------------------------------------------------------------------
def run_ours(args):
    import numpy as np
    import torch

    ws, rank, local = dist_env()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a GPU")
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_2102_04709_gb300 import build, lbm3
    from paper_2102_04709_gb300 import workloads as W
    build.build()
    lbm3.load()

    if args.workload == "pillars_4096x2048":
        w = W.config4(args.theta)
    elif args.workload == "pillars_2048x1024":
        w = W.pillars_half(args.theta)
    else:
        w = W.five_pillars((90.0, 180.0 - args.theta, args.theta))
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    prec = PRECISIONS[args.precision]
    sim = lbm3.Lbm3.from_workload(w, precision=prec, stream=stream.cuda_stream)
    info = sim.info()

    def barrier():
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    sim.step(args.warmup)
    barrier()
    sampler = ClockSampler(local)
    time.sleep(0.5)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    barrier()
    t0 = time.time()
    e0.record(stream)
    ms_wet, ms_pure, ms_wall, ms_edge, ms_run = sim.step_timed_detail(args.steps)
    ms_gen = ms_wall + ms_edge
    e1.record(stream)
    barrier()
    t1 = time.time()
    sampler.stop()
    # the device time of exactly the K steps, from the event before the first launch to the one
    # after the last step (e0 -> e1 also holds the host's read-back of the 7 K per-launch events,
    # during which the device is idle)
    ms = max_over_ranks(ms_run, ws, "cuda")
    ms_call = max_over_ranks(e0.elapsed_time(e1), ws, "cuda")
    d = sim.diag(check=False)

    # end to end through the C ABI with host buffers: H2D of the initial densities, the steps,
    # D2H of the densities and velocity
    e2e = None
    if not args.no_e2e:
        rho_host = torch.from_numpy(np.ascontiguousarray(w.rho)).pin_memory().numpy()
        barrier()
        ta = time.perf_counter()
        sim.set_fields(rho_host)
        sim.step(args.steps)
        rho_out, u_out = sim.fields()
        barrier()
        tb = time.perf_counter()
        e2e_ms = max_over_ranks((tb - ta) * 1e3, ws, "cuda")
        e2e = {"value": job_mlups(w.n, args.steps, ws, e2e_ms), "unit": "MLUPS",
               "h2d_bytes_per_step": int(math.ceil(rho_host.nbytes / args.steps)),
               "d2h_bytes_per_step": int(math.ceil((rho_out.nbytes + u_out.nbytes) / args.steps)),
               "steps": args.steps,
               "note": "one call sequence per run: lbm3_set_fields (H2D of the FP64 initial "
                       "densities), lbm3_step(steps), lbm3_fields (D2H of FP64 densities and "
                       "velocity); the copies are amortised over `steps`"}
        if args.steps < E2E_LONG:
            # the same sequence over a run length where the copies no longer dominate
            barrier()
            ta = time.perf_counter()
            sim.set_fields(rho_host)
            sim.step(E2E_LONG)
            rho_out, u_out = sim.fields()
            barrier()
            tb = time.perf_counter()
            e2e["long_run"] = {"steps": E2E_LONG, "value": job_mlups(
                w.n, E2E_LONG, ws, max_over_ranks((tb - ta) * 1e3, ws, "cuda")), "unit": "MLUPS"}

    # the same steps through lbm3_step itself, which replays captured CUDA graphs of 8 steps and
    # records no per-launch events (the timed region above records five events per step so that
    # the roofline can use each kernel's own duration)
    g0 = torch.cuda.Event(enable_timing=True)
    g1 = torch.cuda.Event(enable_timing=True)
    barrier()
    g0.record(stream)
    sim.step(args.steps)
    g1.record(stream)
    barrier()
    gms = max_over_ranks(g0.elapsed_time(g1), ws, "cuda")
    graphs = {"value": job_mlups(w.n, args.steps, ws, gms), "unit": "MLUPS",
              "ms_per_step": gms / args.steps, "steps": args.steps}

    # the same workload with the other population storages (shorter timed region each)
    alt = {}
    if not args.no_alt_storage:
        for name, p in PRECISIONS.items():
            if name == args.precision:
                continue
            del sim
            sim = lbm3.Lbm3.from_workload(w, precision=p, stream=stream.cuda_stream)
            sim.step(args.warmup)
            barrier()
            n_alt = max(args.steps // 2, 1)
            _, msp, _, _, arun = sim.step_timed_detail(n_alt)
            barrier()
            ams = max_over_ranks(arun, ws, "cuda")
            ainfo = sim.info()
            alt[name] = {"value": job_mlups(w.n, n_alt, ws, ams), "unit": "MLUPS",
                         "ms_per_step": ams / n_alt, "steps": n_alt,
                         "bytes_per_fluid_node": 216 if p == 0 else 120,
                         "pure_kernel_gbs": ainfo["pure_bytes"] / (msp / n_alt * 1e-3) / 1e9}

    # adjoint: J = x-centroid of fluid 0 after 2000 steps of the 512 x 256 six-pillar case,
    # gradients for every wall-node angle and the inflow velocity; every state kept on the device
    # (2000 x 17.3 MB), and, beside it, checkpoints every 100 steps with the segments recomputed
    adj = None
    if not args.no_adjoint:
        w5 = W.config5()
        s5 = lbm3.Lbm3.from_workload(w5, stream=stream.cuda_stream)

        def timed_adjoint(K):
            # the first call of a size allocates the store the handle keeps for the next ones
            # (an optimisation loop's steady state); both are timed, the second is the figure
            times = []
            for _ in range(2):
                s5.set_fields(w5.rho)
                barrier()
                ta = time.perf_counter()
                out = s5.adjoint_centroid(w5.steps, K)
                barrier()
                times.append(time.perf_counter() - ta)
            s5.adjoint_release()
            return out, times[1], times[0]

        (J, dang, du), t_all, t_all_first = timed_adjoint(w5.steps)
        _, t_k100, t_k100_first = timed_adjoint(100)
        s5.set_fields(w5.rho)
        barrier()
        tc = time.perf_counter()
        s5.step(w5.steps)
        barrier()
        td = time.perf_counter()
        fwd_ms = (td - tc) / w5.steps * 1e3
        adj = {"workload": w5.name, "steps": w5.steps, "checkpoint_every": w5.steps,
               "wall_nodes": int(dang.shape[0]),
               "steps_per_s": w5.steps / t_all, "unit": "adjoint steps/s (forward + reverse, every state kept)",
               "ms_per_step": t_all / w5.steps * 1e3,
               "first_call_ms_per_step": t_all_first / w5.steps * 1e3,
               "forward_only_ms_per_step": fwd_ms,
               "ratio_to_forward": t_all / w5.steps * 1e3 / fwd_ms,
               "recompute": {"checkpoint_every": 100, "ms_per_step": t_k100 / w5.steps * 1e3,
                             "first_call_ms_per_step": t_k100_first / w5.steps * 1e3,
                             "unit": "forward + recompute + reverse"},
               "J": J, "dJ_du": du, "grad_angles_norm": float(np.linalg.norm(dang))}
        del s5

    if rank != 0:
        return
    value = job_mlups(w.n, args.steps, ws, ms)
    # dominant kernel: the fused step on the pure tiles (216 B per node, no class bytes)
    bytes_launch = info["pure_bytes"]
    achieved = bytes_launch / (ms_pure / args.steps * 1e-3) / 1e9
    peak, peak_src = measured_peak()
    traffic = profiled_traffic(info["pure_nodes"])
    clocks = sampler.summary(t0, t1)
    line = {
        "metric": "MLUPS", "value": value, "unit": "MLUPS", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": w.name, "nx": w.nx, "ny": w.ny, "fluid_nodes": info["n_fluid"],
                   "wall_nodes": info["n_wall"], "storage": args.precision,
                   "alt_storage": alt, "adjoint": adj, "lbm3_step_graphs": graphs,
                   "mflups": info["n_fluid"] * args.steps * ws / (ms * 1e-3) / 1e6,
                   "l2": "populations 2 x 0.91 GB > 129 MB L2: no flush between steps",
                   "replicas": ws, "ms_wet_per_step": ms_wet / args.steps,
                   "ms_step_pure_tiles_per_step": ms_pure / args.steps,
                   "ms_step_other_tiles_per_step": ms_gen / args.steps,
                   "ms_step_wall_tiles_per_step": ms_wall / args.steps,
                   "ms_step_edge_tiles_per_step": ms_edge / args.steps,
                   "ms_call_per_step": ms_call / args.steps,
                   "timing": "ms_per_step: CUDA events on the main stream around exactly the "
                             "timed steps (before the first launch, after the last step's "
                             "joins); ms_call_per_step: the same call bracketed from Python, "
                             "with the host's read-back of the per-launch events inside",
                   "pure_tile_nodes": info["pure_nodes"],
                   "step_algorithmic_bytes": info["step_bytes"],
                   "step_effective_gbs": info["step_bytes"] / (ms / args.steps * 1e-3) / 1e9,
                   "max_u": float(d[5])},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic, "peak_source": peak_src,
                     "kernel": {"ring": "k_step_ring (pure tiles, warp-specialised ring of bulk "
                                        "tensor copies)",
                                "bulk copies": "k_step_tma (pure tiles, bulk tensor copies)",
                                "plain": "k_step<pure tiles>"}[info["pure_kernel"]],
                     "algorithmic_bytes_per_launch": bytes_launch},
        "gpu_launches": (info["step_kernels"] + info["wet_kernels"]) * args.steps,
        "clocks": clocks,
        "e2e": e2e,
    }
    if ws == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(w)
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
