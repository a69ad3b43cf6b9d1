"""Benchmark: HF-QMC spin-flip proposals/s of one RDMFT iteration on the 20x20 trap.

Workload (one "step" = one full RDMFT iteration, every row of the hot path): 20x20 open square
trap, t = 1, U = 8, V0 = 0.05, mu tuned to ~100 atoms, beta = 8, dtau = 0.25 (L = 32); C4v
reduces it to 55 inequivalent sites x 32 Markov chains = 1760 chains; 500 warm-up + 2000
measured sweeps per iteration, FP64 Dyson refresh every 10 sweeps; lattice step over 500
Matsubara frequencies x 2 spins; transforms and self-energy update.  Inputs are synthetic
(seeded fields, the model's own seeded self-energy); there is no dataset.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 runs N independent replicas (one per GPU, launched by torch.distributed.run), timed with
a barrier and the max over ranks; rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1006_2716_gb300 import workloads as wl  # noqa: E402

CFG = dict(wl.CONFIGS["square20"])
METRIC = "HF-QMC spin-flip proposals/s"
WORKLOAD = ("square20: 20x20 open trap, U=8, V0=0.05, mu=%.4f, beta=8, dtau=0.25 (L=32), "
            "55 inequivalent sites x 32 chains, 500+2000 sweeps, refresh every 10, "
            "500 Matsubara frequencies; one step = one RDMFT iteration" % CFG["mu"])
FP64_PEAK_TFLOPS = 2.0 * 2 * 152 * 2.07e9 / 1e12   # 2 DFMA/clk/SM x 152 SMs x 2.07 GHz
CLOCK_QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
               "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
               "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def qmc_flops(L, nchain, sweeps, accepts, n_measure, n_refresh):
    """Algorithmic FP64 flops of the fused QMC kernel: 10 per proposal (ratio and test),
    4 L^2 per accepted flip (two rank-1 updates), 2 L^2 per measurement, 2 (8/3) L^3 per
    refresh (both spins)."""
    return (10.0 * L * nchain * sweeps + 4.0 * L * L * accepts + 2.0 * L * L * nchain * n_measure
            + 2.0 * (8.0 / 3.0) * L ** 3 * nchain * n_refresh)


# ---------------------------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------------------------
class ClockSampler:
    def __init__(self, index):
        self.path = tempfile.mktemp(prefix="clocks_", suffix=".csv")
        self.proc = None
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(index), "--query-gpu=" + CLOCK_QUERY, "--format=csv",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (FileNotFoundError, OSError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path).read().splitlines()[1:]:
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                rows.append((float(f[1].split()[0]), float(f[2].split()[0]), f[5:9]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[2][k] == "Active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------------------------------------
# CPU oracle leg (spawned process, one thread)
# ---------------------------------------------------------------------------------------------
def _oracle_sample(q, n_chains, n_freq):
    import numpy as np

    import oracle as o
    from oracle.lattice import Lattice, lattice_step
    from oracle.rdmft import RDMFT

    cfg = CFG
    L = 32
    r = RDMFT(cfg["Lx"], cfg["Ly"], U=cfg["U"], V0=cfg["V0"], mu=cfg["mu"], beta=cfg["beta"], L=L,
              nw=cfg["n_matsubara"], chains=1, seed=cfg["seed"], h_seed=cfg["h_seed"])
    full = r.expand_sigma()
    t0 = time.perf_counter()
    idx = np.arange(n_freq) * (cfg["n_matsubara"] // n_freq)
    for sp in range(2):
        lattice_step(r.lat.H0, cfg["mu"], cfg["beta"], full[sp][idx], n_index=idx)
    t_lat = (time.perf_counter() - t0) * (cfg["n_matsubara"] / n_freq)
    baths = wl.random_baths(2, n_chains, cfg["beta"], L)
    _, lam = o.constants(cfg["beta"], cfg["U"], L)
    t0 = time.perf_counter()
    for c in range(n_chains):
        g0u, g0d = o.build_g0(baths[c, 0]), o.build_g0(baths[c, 1])
        s = o.init_fields(cfg["seed"], c, 0, L)
        Gu, _ = o.dyson(g0u, s, 1, lam)
        Gd, _ = o.dyson(g0d, s, -1, lam)
        bins = np.zeros((cfg["n_measure"] // cfg["bin_size"], 2 * L + 3))
        o.run_chain(lam, g0u, g0d, cfg["seed"], c, 0, 0, cfg["n_warmup"], cfg["n_measure"],
                    cfg["refresh_every"], cfg["bin_size"], s, Gu, Gd, bins)
    t_qmc = (time.perf_counter() - t0) * (1760.0 / n_chains)
    q.put((t_lat, t_qmc))


def cpu_oracle(n_chains=160, n_freq=20):
    """Oracle time of one full iteration, extrapolated from a bounded sample (seconds).

    Runs in a spawned process with one BLAS / OpenMP thread (the variables are set before the
    child starts, so numpy in the child sees them at import)."""
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
    for k in saved:
        os.environ[k] = "1"
    try:
        p = ctx.Process(target=_oracle_sample, args=(q, n_chains, n_freq))
        p.start()
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    t_lat, t_qmc = q.get()
    p.join()
    sample = ("%d of 1760 chains x 2500 sweeps (L=32) + lattice step at %d of 500 frequencies x "
              "2 spins (dense inverse, N=400), each scaled to the full iteration" % (n_chains, n_freq))
    return t_lat + t_qmc, sample


# ---------------------------------------------------------------------------------------------
def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    proposals = 1760 * 2500 * 32
    times = []
    sample = ""
    for _ in range(args.warmup):
        cpu_oracle(2, 4)
    for _ in range(args.steps):
        t, sample = cpu_oracle(64, 10)
        times.append(t)
    sec = sum(times) / len(times)
    v = proposals / sec
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "proposals/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": sec * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD},
            "cpu_baseline": {"value": v, "unit": "proposals/s", "cores": 1, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": v, "unit": "proposals/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def run_ours(args):
    import numpy as np
    import torch

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", init_method="env://")
    # the CPU oracle leg is spawned before any CUDA work (rank 0, N = 1 only)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        t_cpu, sample = cpu_oracle()
        cpu = {"value": 1760 * 2500 * 32 / t_cpu, "unit": "proposals/s", "cores": 1,
               "kind": "oracle", "sample": sample}
    torch.cuda.set_device(local)
    from paper_1006_2716_gb300 import hf

    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(dev)
    cfg = dict(CFG, precision=args.precision, team_warps=args.team_warps)
    if args.sweeps:
        # short QMC launch for profiling captures only (not a benchmark value)
        cfg.update(n_warmup=args.sweeps // 5, n_measure=args.sweeps - args.sweeps // 5,
                   bin_size=max(1, (args.sweeps - args.sweeps // 5) // 4))
        cfg["max_bins"] = -(-cfg["n_measure"] // cfg["bin_size"])
    ctx = hf.Context(hf.make_params(cfg), device=dev, stream=stream)
    L, ns, nc, nw = ctx.L, ctx.n_sites, ctx.n_chains, ctx.nw
    sweeps = cfg["n_warmup"] + cfg["n_measure"]
    proposals = nc * sweeps * L
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)   # > 129 MB L2

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    for _ in range(args.warmup):
        hf.hf_rdmft_step(ctx.handle)
    torch.cuda.synchronize(dev)
    barrier()
    clocks = ClockSampler(local)
    ms_steps, qmc_ms, phase = [], [], np.zeros(5)
    acc0 = hf.hf_get_accepts(ctx.handle, nc).sum()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    for _ in range(args.steps):
        with torch.cuda.stream(stream):
            flush.zero_()                       # evict L2 between timed steps
        torch.cuda.synchronize(dev)
        ev0.record(stream)
        hf.hf_rdmft_step(ctx.handle)
        ev1.record(stream)
        ev1.synchronize()
        ms_steps.append(ev0.elapsed_time(ev1))
        t = hf.hf_get_timings(ctx.handle)
        phase += t[:5]
        qmc_ms.append(t[2])
    torch.cuda.synchronize(dev)
    barrier()
    clk = clocks.stop()
    accepts = int(hf.hf_get_accepts(ctx.handle, nc).sum() - acc0)
    ms_total = sum(ms_steps)
    if world > 1:
        tt = torch.tensor([ms_total], device=dev, dtype=torch.float64)
        torch.distributed.all_reduce(tt, op=torch.distributed.ReduceOp.MAX)
        ms_total = float(tt.item())
    ms_per_step = ms_total / args.steps
    value = proposals * world / (ms_per_step / 1e3)

    # end to end through the public API with host buffers: H2D self-energy, iteration,
    # D2H observables and self-energy, every step
    pin_sig = torch.empty(ns * 2 * nw * 2, dtype=torch.float64, pin_memory=True)
    pin_obs = torch.empty(2 * ns * (2 * L + 4), dtype=torch.float64, pin_memory=True)
    sig_np = pin_sig.numpy().view(np.complex128).reshape(ns, 2, nw)
    sig_np[:] = hf.hf_get_sigma(ctx.handle, ns, nw)
    h2d = sig_np.nbytes
    d2h = pin_obs.numpy().nbytes + sig_np.nbytes
    torch.cuda.synchronize(dev)
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        hf.lib().hf_set_sigma(ctx.handle, sig_np.ctypes.data_as(hf._DP))
        hf.hf_rdmft_step(ctx.handle)
        obs = pin_obs.numpy()
        hf.lib().hf_get_observables(ctx.handle, obs.ctypes.data_as(hf._DP),
                                    obs[ns * (2 * L + 4):].ctypes.data_as(hf._DP))
        hf.lib().hf_get_sigma(ctx.handle, sig_np.ctypes.data_as(hf._DP))
    torch.cuda.synchronize(dev)
    e2e_s = (time.perf_counter() - t0) / args.steps
    if world > 1:
        tt = torch.tensor([e2e_s], device=dev, dtype=torch.float64)
        torch.distributed.all_reduce(tt, op=torch.distributed.ReduceOp.MAX)
        e2e_s = float(tt.item())
    e2e = {"value": proposals * world / e2e_s, "unit": "proposals/s", "h2d_bytes_per_step": h2d,
           "d2h_bytes_per_step": d2h}

    # roofline of the dominant kernel (the fused QMC sweep kernel), FP64 ALU bound
    n_refresh = 1 + sweeps // cfg["refresh_every"]
    flops = qmc_flops(L, nc, sweeps, accepts / args.steps, cfg["n_measure"], n_refresh)
    qmc_s = statistics.mean(qmc_ms) / 1e3
    achieved = flops / qmc_s / 1e12
    roofline = {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": achieved / FP64_PEAK_TFLOPS, "traffic": None,
                "kernel": "qmc_f64_kernel", "acceptance": accepts / (args.steps * proposals),
                "peak_source": "FP64 nominal: 2 DFMA/clk/SM x 152 SMs x 2.07 GHz"}
    # our kernels per iteration: lattice step (chunks of <= 1 GiB of band buffers), Weiss/tau,
    # QMC, reduction, self-energy update
    per_matrix = ctx.N * (20 + 1) * 16
    launches_per_step = -(-2 * nw // max(1, min(2 * nw, (1 << 30) // per_matrix))) + 4
    line = {"metric": METRIC, "value": value, "unit": "proposals/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "global_batch": nc * world, "seq_len": L,
                       "parallelism": "replicas%d" % world,
                       "l2": "flushed (256 MB write) between timed steps"},
            "rdmft_iteration_ms": ms_per_step,
            "phase_ms": dict(zip(["lattice", "weiss_tau", "qmc", "reduce", "sigma"],
                                 [float(x) for x in phase / args.steps])),
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": launches_per_step * args.steps, "clocks": clk}
    if args.sweeps:
        line["profile_case"] = "sweeps overridden to %d: not a benchmark value" % args.sweeps
    if rank == 0:
        print(json.dumps(line))
    ctx.close()
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle leg")
    ap.add_argument("--team-warps", type=int, default=0, choices=[0, 1, 2, 4],
                    help="warps per Markov chain (0: library default)")
    ap.add_argument("--precision", type=int, default=0, choices=[0, 2],
                    help="sweep arithmetic: 0 FP64, 2 FP32 pairs (both with FP64 refresh)")
    ap.add_argument("--sweeps", type=int, default=0,
                    help="profiling only: override sweeps per iteration (result is not a bench value)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
