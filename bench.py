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
DFMA_PROBE_TFLOPS = 1.008   # independent DFMA chains, 152 SMs x 8 blocks x 256 threads, this GPU


def _measured_peak(key, fallback):
    """A measured peak of this GPU pool (MEASURED_PEAKS.json), else the fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)[key])
    except (OSError, ValueError, KeyError):
        return fallback


MEASURED_BF16_SUSTAINED = _measured_peak("bf16_tflops_sustained", 1700.0)
CLOCK_QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
               "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
               "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(x, device):
    """Largest x over the ranks of the default process group (x itself on one rank): the slowest
    replica sets a job's time."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank, seconds, world):
    """Whole-job rate of `world` replicas that each process units_per_rank units, timed by the
    slowest rank's seconds."""
    return units_per_rank * world / seconds


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
# CPU oracle legs (spawned processes: one thread, and one worker per host core)
# ---------------------------------------------------------------------------------------------
# all host cores: a pool of spawned workers (one BLAS thread each) that hold the workload's
# lattice and seeded self-energy; the parent computes the baths between the two parallel phases
_W = {}


def _square20_rdmft():
    from oracle.rdmft import RDMFT

    cfg = CFG
    return RDMFT(cfg["Lx"], cfg["Ly"], U=cfg["U"], V0=cfg["V0"], mu=cfg["mu"], beta=cfg["beta"],
                 L=32, nw=cfg["n_matsubara"], chains=1, seed=cfg["seed"], h_seed=cfg["h_seed"],
                 n_warmup=cfg["n_warmup"], n_measure=cfg["n_measure"],
                 refresh_every=cfg["refresh_every"], bin_size=cfg["bin_size"])


def _pool_init():
    r = _square20_rdmft()
    _W["r"], _W["full"] = r, r.expand_sigma()


def _pool_lattice(idx):
    """eq. 2 at the frequencies idx for both spins; G_ii of the inequivalent sites [2, k, ns]."""
    import numpy as np

    from oracle.lattice import lattice_step

    r = _W["r"]
    idx = np.asarray(idx)
    return idx, [lattice_step(r.lat.H0, CFG["mu"], CFG["beta"], _W["full"][sp][idx],
                              n_index=idx)[:, r.reps] for sp in range(2)]


def _pool_chains(job):
    """Whole 2500-sweep chains c (site c // 32, chain c % 32) on the given baths; returns their
    bins [len(chains), nbins, 2L+3] and the worker's seconds."""
    import numpy as np

    import oracle as o

    chains, g0_tau = job
    t0 = time.perf_counter()
    cfg, L, cps = CFG, 32, CFG["chains_per_site"]
    _, lam = o.constants(cfg["beta"], cfg["U"], L)
    out = np.zeros((len(chains), cfg["n_measure"] // cfg["bin_size"], 2 * L + 3))
    for k, c in enumerate(chains):
        site, ch = divmod(c, cps)
        g0u, g0d = o.build_g0(g0_tau[site, 0, :L]), o.build_g0(g0_tau[site, 1, :L])
        s = o.init_fields(cfg["seed"], site, ch, L)
        Gu, _ = o.dyson(g0u, s, 1, lam)
        Gd, _ = o.dyson(g0d, s, -1, lam)
        o.run_chain(lam, g0u, g0d, cfg["seed"], site, ch, 0, cfg["n_warmup"], cfg["n_measure"],
                    cfg["refresh_every"], cfg["bin_size"], s, Gu, Gd, out[k])
    return out, time.perf_counter() - t0


def _spawn_pool(n, initializer=None):
    """A spawned pool of n worker processes with one BLAS / OpenMP thread each (the variables
    are set before the children start, so numpy in them sees them at import)."""
    ctx = mp.get_context("spawn")
    saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
    for k in saved:
        os.environ[k] = "1"
    try:
        return ctx.Pool(n, initializer=initializer)
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v


def oracle_iteration(pool, workers, n_chains=1760, n_freq=500):
    """Seconds of one RDMFT iteration of the oracle on the square20 workload from its seeded
    self-energy: the lattice step (eq. 2, dense inverse) at n_freq of the 500 frequencies, the
    baths, n_chains of the 1760 chains (evenly spaced, so every site is sampled) on those baths,
    then reduction, tau -> i w and the self-energy update; the lattice step and the chains are
    each scaled to the full iteration when sampled (n_freq < 500 or n_chains < 1760).  With
    everything in, it is the oracle's own iteration, whose chains make the GPU's decisions on
    the same baths and seeds."""
    import numpy as np

    from oracle.fourier import tau_to_iw

    r = _square20_rdmft()
    nw, ns, L = CFG["n_matsubara"], r.nsite, 32
    t0 = time.perf_counter()
    if n_freq >= nw:
        idx = list(range(nw))
    else:
        idx = [k * (nw // n_freq) for k in range(n_freq)]
    chunks = [idx[w::workers] for w in range(workers) if idx[w::workers]]
    Gloc = np.zeros((ns, 2, nw), dtype=np.complex128)
    for ids, g in pool.map(_pool_lattice, chunks, chunksize=1):
        for sp in range(2):
            Gloc[:, sp, ids] = g[sp].T
    t_lat = (time.perf_counter() - t0) * (nw / len(idx))
    t0 = time.perf_counter()
    if len(idx) < nw:   # sampled: the baths of the seeded self-energy from the full step anyway
        for ids, g in pool.map(_pool_lattice, [list(range(w, nw, workers)) for w in range(workers)],
                               chunksize=1):
            for sp in range(2):
                Gloc[:, sp, ids] = g[sp].T
        t0 = time.perf_counter()
    weiss_inv, gw_t = r.weiss(Gloc)
    g0_tau = r.bath_tau(gw_t)
    t_bath = time.perf_counter() - t0
    # a sample takes chains evenly spaced over all 1760 (every site's chains are represented)
    chains = sorted({int(k * 1760 // n_chains) for k in range(n_chains)})
    n_chains = len(chains)
    t0 = time.perf_counter()
    parts = pool.map(_pool_chains, [(chains[w::workers], g0_tau) for w in range(workers)
                                    if chains[w::workers]], chunksize=1)
    if n_chains >= 1760:
        t_qmc = time.perf_counter() - t0
    else:
        # sampled: the workers' summed chain time, spread over all workers and scaled to the
        # 1760 chains (the whole set balances over the workers; a small sample would not)
        t_qmc = sum(t for _, t in parts) / workers * (1760.0 / n_chains)
    parts = [b for b, _ in parts]
    t0 = time.perf_counter()
    bins = np.zeros((1760, CFG["n_measure"] // CFG["bin_size"], 2 * L + 3))
    for w, part in enumerate(parts):
        bins[chains[w::workers]] = part
    if n_chains < 1760:   # a sample: every chain of the reduction gets a sampled chain's bins
        have = np.array(chains)
        for c in range(1760):
            bins[c] = bins[have[np.abs(have - c).argmin()]]
    mean, _ = r.reduce(bins.reshape(ns, CFG["chains_per_site"], *bins.shape[1:]))
    for i in range(ns):
        for sp in range(2):
            gimp = tau_to_iw(CFG["beta"], mean[i, sp * L:(sp + 1) * L], g0_tau[i, sp, :L], gw_t[i, sp])
            r.sigma[i, sp] = r.mix * (weiss_inv[i, sp] - 1.0 / gimp) + (1.0 - r.mix) * r.sigma[i, sp]
    t_rest = time.perf_counter() - t0
    return t_lat + t_bath + t_qmc + t_rest


def cpu_oracle_all_cores():
    """One whole oracle iteration of the square20 workload on every host core (nothing sampled);
    returns (seconds, cores, description)."""
    cores = host_cores()
    pool = _spawn_pool(cores, _pool_init)
    try:
        oracle_iteration(pool, cores, n_chains=cores, n_freq=cores)   # warm: imports, builds
        sec = oracle_iteration(pool, cores)
    finally:
        pool.close()
        pool.join()
    sample = ("one whole RDMFT iteration (lattice step at all 500 frequencies x 2 spins, dense "
              "inverse N=400; baths; all 1760 chains x 2500 sweeps, L=32, FP64, on the workload's "
              "own baths and seeds; reduction and self-energy update) over %d worker processes"
              % cores)
    return sec, cores, sample


def cpu_oracle(n_chains=64, n_freq=10):
    """Oracle seconds of one iteration on one core (one process, one BLAS thread), from a
    bounded sample: n_chains chains and n_freq frequencies, each part scaled to the full
    iteration."""
    pool = _spawn_pool(1, _pool_init)
    try:
        oracle_iteration(pool, 1, n_chains=1, n_freq=1)
        sec = oracle_iteration(pool, 1, n_chains=n_chains, n_freq=n_freq)
    finally:
        pool.close()
        pool.join()
    sample = ("%d of 1760 chains x 2500 sweeps (L=32, on the workload's own baths) + the lattice "
              "step at %d of 500 frequencies x 2 spins (dense inverse, N=400), one process, each "
              "part scaled to the full iteration" % (n_chains, n_freq))
    return sec, sample


def _pool_chains_sq30(job):
    """Oracle (FP64 throughout) chains of the 30x30 workload: L = 128, refresh every sweep."""
    import numpy as np

    import oracle as o

    chains, sweeps = job
    cfg, L = wl.CONFIGS["square30"], 128
    baths = wl.random_baths(3, max(chains) + 1, cfg["beta"], L)
    _, lam = o.constants(cfg["beta"], cfg["U"], L)
    for c in chains:
        g0u, g0d = o.build_g0(baths[c, 0]), o.build_g0(baths[c, 1])
        s = o.init_fields(cfg["seed"], c, 0, L)
        Gu, _ = o.dyson(g0u, s, 1, lam)
        Gd, _ = o.dyson(g0d, s, -1, lam)
        bins = np.zeros((1, 2 * L + 3))
        o.run_chain(lam, g0u, g0d, cfg["seed"], c, 0, 0, 0, sweeps, 1, sweeps, s, Gu, Gd, bins)
    return len(chains)


def cpu_oracle_square30(chains_per_core=2, sweeps=10):
    """Proposals/s of the oracle on the 30x30 workload (L = 128, FP64 sweeps, refresh every
    sweep) on every host core, from a bounded sample; returns (value, cores, sample)."""
    cores = host_cores()
    ctx = mp.get_context("spawn")
    saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
    for k in saved:
        os.environ[k] = "1"
    try:
        pool = ctx.Pool(cores)
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    try:
        pool.map(_pool_chains_sq30, [([w], 1) for w in range(cores)], chunksize=1)   # warm
        n = cores * chains_per_core
        t0 = time.perf_counter()
        pool.map(_pool_chains_sq30, [(list(range(w, n, cores)), sweeps) for w in range(cores)],
                 chunksize=1)
        wall = time.perf_counter() - t0
    finally:
        pool.close()
        pool.join()
    sample = ("%d chains x %d sweeps (L=128, FP64, Dyson refresh every sweep) over %d worker "
              "processes" % (n, sweeps, cores))
    return n * sweeps * 128 / wall, cores, sample


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


# ---------------------------------------------------------------------------------------------
def run_reference(args):
    """The oracle as it stands on every host core: each timed step is one RDMFT iteration of the
    square20 workload with its chains sampled (20 per core, scaled; everything else whole, see
    oracle_iteration), so that --steps 20 ends within a few minutes; warm-up steps run a small
    sample."""
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    proposals = 1760 * 2500 * 32
    cores = host_cores()
    pool = _spawn_pool(cores, _pool_init)
    try:
        oracle_iteration(pool, cores, n_chains=cores, n_freq=cores)     # imports, builds
        for _ in range(args.warmup):
            oracle_iteration(pool, cores, n_chains=cores, n_freq=cores)
        n_ch = min(1760, 20 * cores)
        times = [oracle_iteration(pool, cores, n_chains=n_ch) for _ in range(args.steps)]
    finally:
        pool.close()
        pool.join()
    sample = ("per step one RDMFT iteration: lattice step at all 500 frequencies x 2 spins (dense "
              "inverse N=400), the baths, %d of the 1760 chains x 2500 sweeps (L=32, FP64, evenly "
              "spaced over the sites, on the workload's own baths and seeds; the workers' summed chain "
              "time scaled by 1760/%d and spread over the workers), "
              "reduction and self-energy update, over %d worker processes"
              % (n_ch, n_ch, cores))
    sec = sum(times) / len(times)
    v = proposals / sec
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "proposals/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": sec * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD},
            "cpu_baseline": {"value": v, "unit": "proposals/s", "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": v, "unit": "proposals/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


FP32_PEAK_TFLOPS = 2.0 * 128 * 152 * 2.07e9 / 1e12   # 128 FFMA/clk/SM
DF_OPS_PER_FMA = 12          # FP32-pipe ops of one double-float multiply-add (lazy renormalisation)
# DRAM bytes (read + write) of one full-size launch, from one ncu capture of the kernel built from
# sources whose sha256 starts with the given prefix (the capture's command and counters are kept
# in the profile summaries); a kernel whose sources changed since reports null.
MEASURED_TRAFFIC = {"qmc_f64_kernel": (2295808 + 3584, "04c6f020ee92be69"),
                    "qmc_df64_kernel": (2386432 + 3584, "5e3b37f3293b93e3"),
                    # the blocked lattice step, one launch of all 500 matrices: slab16 (N = 1024,
                    # b = 128) and box16p (N = 4096, b = 512)
                    "lattice_wide_kernel:slab16": (2160.4e6 + 2092.8e6, "9b62c014a9ceece6"),
                    "lattice_wide_kernel:box16p": (310.53e9 + 279.17e9, "9b62c014a9ceece6"),
                    # square30: one refresh launch and one sweep launch of all 1920 chains
                    "refresh_tc_kernel": (351.7e6 + 1055.7e6, "6ebecb2c46502445"),
                    "qmc_f32_kernel": (256.3e6 + 193.2e6, "a376070c58476eac")}
KERNEL_SOURCES = {"qmc_df64_kernel": ("k_qmc_df64.cu", "qmc_common.cuh", "hf_internal.cuh"),
                  "qmc_f64_kernel": ("k_qmc_f64.cu", "qmc_common.cuh", "hf_internal.cuh"),
                  "lattice_wide_kernel:slab16": ("k_lattice_wide.cu", "k_lattice.cuh",
                                                 "k_lattice_dev.cuh", "tc_ozaki.cuh", "hf_internal.cuh"),
                  "lattice_wide_kernel:box16p": ("k_lattice_wide.cu", "k_lattice.cuh",
                                            "k_lattice_dev.cuh", "tc_ozaki.cuh", "hf_internal.cuh"),
                  "refresh_tc_kernel": ("k_refresh_tc.cu", "k_refresh_tc.cuh", "tc_ozaki.cuh",
                                        "refresh_measure.cuh", "hf_internal.cuh"),
                  "qmc_f32_kernel": ("k_qmc_f32.cu", "tc_ozaki.cuh", "refresh_measure.cuh",
                                     "hf_internal.cuh")}


def measured_traffic(kernel):
    """Bytes per launch from the last ncu capture of this kernel, or None if it has changed."""
    import hashlib

    if kernel not in MEASURED_TRAFFIC:
        return None
    h = hashlib.sha256()
    for f in KERNEL_SOURCES[kernel]:
        with open(os.path.join(ROOT, "paper_1006_2716_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    nbytes, digest = MEASURED_TRAFFIC[kernel]
    return nbytes if h.hexdigest().startswith(digest) else None


def qmc_alg_bytes(L, nchain, nsite, n_measure, bin_size):
    """DRAM bytes one sweep launch must move: per chain its G (written back), its fields (read and
    written) and its bins (written); per inequivalent site its two inverse bath matrices (read)."""
    bins = -(-n_measure // bin_size) * (2 * L + 3) * 8
    return nchain * (2 * L * L * 8 + 2 * L + bins) + nsite * 2 * L * L * 8


def qmc_roofline(form, L, nchain, sweeps, accepts, n_measure, n_refresh, qmc_s, kernel,
                 alg_bytes=None):
    """Roofline of the fused QMC kernel for one launch (algorithmic flops of the method).

    form 0 (FP64): every flop runs on the FP64 pipe; peak = nominal FP64 (2 DFMA/clk/SM x 152 SMs
    x 2.07 GHz).  The rate a plain DFMA probe reached on this GPU is reported beside it.
    form 2 (FP32 pairs): the refresh runs on the FP64 pipe, the sweep arithmetic on the FP32 pipe
    at DF_OPS_PER_FMA ops per FP64-equivalent multiply-add.  The two do not overlap on this GPU
    (measured), so the roof is total flops / (FP64 time + FP32 time); the roof of both pipes
    overlapped is reported beside it."""
    f_ratio = 10.0 * L * nchain * sweeps
    f_upd = 4.0 * L * L * accepts
    f_meas = 2.0 * L * L * nchain * n_measure
    f_ref = 2.0 * (8.0 / 3.0) * L ** 3 * nchain * n_refresh
    total = f_ratio + f_upd + f_meas + f_ref
    achieved = total / qmc_s / 1e12
    extra = {}
    if form == 0:
        peak, src = FP64_PEAK_TFLOPS, "FP64 nominal: 2 DFMA/clk/SM x 152 SMs x 2.07 GHz"
        extra = {"dfma_probe_tflops": DFMA_PROBE_TFLOPS,
                 "frac_of_dfma_probe": achieved / DFMA_PROBE_TFLOPS}
    else:
        t64 = f_ref / (FP64_PEAK_TFLOPS * 1e12)
        t32 = (f_ratio + f_upd + f_meas) / 2.0 * DF_OPS_PER_FMA / (FP32_PEAK_TFLOPS * 1e12 / 2.0)
        peak = total / (t64 + t32) / 1e12
        over = total / max(t64, t32) / 1e12
        extra = {"peak_overlapped": over, "frac_overlapped": achieved / over}
        src = ("serial two-pipe roof: refresh on FP64 (2 DFMA/clk/SM), then the pair arithmetic "
               "on FP32 (128 FFMA/clk/SM, %d ops per FP64-equivalent FMA), both at 2.07 GHz"
               % DF_OPS_PER_FMA)
    # the refreshes invert G^{-1} by Gauss-Jordan: 2 L^3 executed flops per spin against the
    # 2 (8/3) L^3 of the algorithmic Dyson solve counted in f_ref
    executed = (total - 0.25 * f_ref) / qmc_s / 1e12
    return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak, "traffic": measured_traffic(kernel),
            "algorithmic_bytes": alg_bytes,
            "kernel": kernel, "executed_tflops": executed, "peak_source": src, **extra}


def e2e_iterations(hf, ctx, dev, steps, proposals):
    """The same RDMFT iterations end to end through the public API with host buffers: per step the
    self-energy from pinned host memory (H2D), the iteration, and the observables and the new
    self-energy back to pinned host memory (D2H); wall clock over the steps."""
    import numpy as np
    import torch

    L, ns, nw = ctx.L, ctx.n_sites, ctx.nw
    pin_sig = torch.empty(ns * 2 * nw * 2, dtype=torch.float64, pin_memory=True)
    pin_obs = torch.empty(2 * ns * (2 * L + 4), dtype=torch.float64, pin_memory=True)
    sig_np = pin_sig.numpy().view(np.complex128).reshape(ns, 2, nw)
    sig_np[:] = hf.hf_get_sigma(ctx.handle, ns, nw)
    obs = pin_obs.numpy()
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for _ in range(steps):
        hf.lib().hf_set_sigma(ctx.handle, sig_np.ctypes.data_as(hf._DP))
        hf.hf_rdmft_step(ctx.handle)
        hf.lib().hf_get_observables(ctx.handle, obs.ctypes.data_as(hf._DP),
                                    obs[ns * (2 * L + 4):].ctypes.data_as(hf._DP))
        hf.lib().hf_get_sigma(ctx.handle, sig_np.ctypes.data_as(hf._DP))
    torch.cuda.synchronize(dev)
    secs = (time.perf_counter() - t0) / steps
    return {"value": proposals / secs, "unit": "proposals/s", "h2d_bytes_per_step": sig_np.nbytes,
            "d2h_bytes_per_step": obs.nbytes + sig_np.nbytes}


def _time_iterations(hf, ctx, stream, flush, steps):
    import numpy as np
    import torch

    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ms_steps, qmc_ms, phase = [], [], np.zeros(5)
    for _ in range(steps):
        with torch.cuda.stream(stream):
            flush.zero_()                       # evict L2 between timed steps
        torch.cuda.synchronize()
        ev0.record(stream)
        hf.hf_rdmft_step(ctx.handle)
        ev1.record(stream)
        ev1.synchronize()
        ms_steps.append(ev0.elapsed_time(ev1))
        t = hf.hf_get_timings(ctx.handle)
        phase += t[:5]
        qmc_ms.append(t[2])
    return ms_steps, qmc_ms, phase


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
        t_all, cores, sample_all = cpu_oracle_all_cores()
        single = {"value": 1760 * 2500 * 32 / t_cpu, "unit": "proposals/s", "cores": 1,
                  "sample": sample}
        cpu = {"value": 1760 * 2500 * 32 / t_all, "unit": "proposals/s", "cores": cores,
               "kind": "oracle", "sample": sample_all, "single_core": single}
    torch.cuda.set_device(local)
    from paper_1006_2716_gb300 import autotune, hf

    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(dev)
    L = 32
    if args.precision < 0:
        # the headline is the FP64 solver the workload names: FP64 sweeps and refreshes, team
        # width autotuned on the workload itself
        tune = autotune.tune_workload("square20" if args.refresh_stagger == 0 else "square20_stagger",
                                      dict(CFG, refresh_stagger=args.refresh_stagger),
                                      forms=(0,), device=dev, stream=stream)
        form, tw, dk = 0, tune["team_warps"], 1
    else:
        form, tw, dk, tune = args.precision, args.team_warps, args.delay_k, None
    cfg = dict(CFG, precision=form, team_warps=tw, delay_k=dk, refresh_stagger=args.refresh_stagger)
    if args.sweeps:
        # short QMC launch for profiling captures only (not a benchmark value)
        cfg.update(n_warmup=args.sweeps // 5, n_measure=args.sweeps - args.sweeps // 5,
                   bin_size=max(1, (args.sweeps - args.sweeps // 5) // 4))
        cfg["max_bins"] = -(-cfg["n_measure"] // cfg["bin_size"])
    ctx = hf.Context(hf.make_params(cfg), device=dev, stream=stream)
    L, ns, nc, nw = ctx.L, ctx.n_sites, ctx.n_chains, ctx.nw
    sweeps = cfg["n_warmup"] + cfg["n_measure"]
    proposals = nc * sweeps * L
    n_refresh = 1 + sweeps // cfg["refresh_every"]
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)   # > 129 MB L2

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    for _ in range(args.warmup):
        hf.hf_rdmft_step(ctx.handle)
    torch.cuda.synchronize(dev)
    barrier()
    clocks = ClockSampler(local)
    acc0 = hf.hf_get_accepts(ctx.handle, nc).sum()
    ms_steps, qmc_ms, phase = _time_iterations(hf, ctx, stream, flush, args.steps)
    torch.cuda.synchronize(dev)
    barrier()
    clk = clocks.stop()
    accepts = int(hf.hf_get_accepts(ctx.handle, nc).sum() - acc0)
    ms_total = max_over_ranks(sum(ms_steps), dev)
    ms_per_step = ms_total / args.steps
    value = job_throughput(proposals, ms_per_step / 1e3, world)

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
    e2e_s = max_over_ranks((time.perf_counter() - t0) / args.steps, dev)
    e2e = {"value": job_throughput(proposals, e2e_s, world), "unit": "proposals/s",
           "h2d_bytes_per_step": h2d,
           "d2h_bytes_per_step": d2h}
    kernel = "qmc_df64_kernel" if form == 2 else "qmc_f64_kernel"
    alg_bytes = qmc_alg_bytes(L, nc, ns, cfg["n_measure"], cfg["bin_size"])
    roofline = qmc_roofline(form, L, nc, sweeps, accepts / args.steps, cfg["n_measure"],
                            n_refresh, statistics.mean(qmc_ms) / 1e3, kernel, alg_bytes)
    roofline["acceptance"] = accepts / (args.steps * proposals)
    ctx.close()

    # the other sweep form beside the headline one, same workload and the same number of timed
    # iterations: the FP32-pair form (48-bit significand sweeps, FP64 refresh) beside the FP64
    # headline, or the FP64 form beside a pair-form run asked for with --precision 2
    other = None
    if not args.sweeps and not args.no_other_form:
        of = 2 if form == 0 else 0
        c0 = hf.Context(hf.make_params(dict(CFG, precision=of, team_warps=1 if of == 2 else 0,
                                            refresh_stagger=args.refresh_stagger)), device=dev,
                        stream=stream)
        for _ in range(2):
            hf.hf_rdmft_step(c0.handle)
        a0 = hf.hf_get_accepts(c0.handle, nc).sum()
        ms0, q0, _ = _time_iterations(hf, c0, stream, flush, args.steps)
        acc_0 = int(hf.hf_get_accepts(c0.handle, nc).sum() - a0)
        other = {"value": proposals / (statistics.mean(ms0) / 1e3), "unit": "proposals/s",
                 "ms_per_step": statistics.mean(ms0), "steps": args.steps,
                 "dtype": "f64" if of == 0 else "f32x2+f64",
                 "roofline": qmc_roofline(of, L, nc, sweeps, acc_0 / args.steps, cfg["n_measure"],
                                          n_refresh, statistics.mean(q0) / 1e3,
                                          "qmc_f64_kernel" if of == 0 else "qmc_df64_kernel",
                                          alg_bytes)}
        if of == 2:
            other["note"] = ("FP32-pair sweeps: 48-bit significand between FP64 refreshes, so G "
                             "drifts further from the FP64 chain than FP64 arithmetic does; not "
                             "an FP64 result")
        c0.close()

    launches_per_step = lattice_launches(hf, cfg) + 5
    dtype = "f64" if form == 0 else "f32x2+f64"
    line = {"metric": METRIC, "value": value, "unit": "proposals/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": dtype,
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "chains": nc * world, "time_slices": L,
                       "parallelism": "replicas%d" % world, "sweep_form": form,
                       "team_warps": tw if tw else "default", "delay_k": dk,
                       "refresh_stagger": args.refresh_stagger,
                       "l2": "flushed (256 MB write) between timed steps"},
            "rdmft_iteration_ms": ms_per_step,
            "phase_ms": dict(zip(["lattice", "weiss_tau", "qmc", "reduce", "sigma"],
                                 [float(x) for x in phase / args.steps])),
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": launches_per_step * args.steps, "clocks": clk,
            ("pair_form" if form == 0 else "fp64_form"): other, "autotune": tune}
    if args.sweeps:
        line["profile_case"] = "sweeps overridden to %d: not a benchmark value" % args.sweeps
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def lattice_launches(hf, cfg):
    """Lattice-step launches of one iteration, as the library plans them: the nspin x nw
    matrices in chunks of as many band buffers as fit in 1 GiB (at most 2 nw), one launch each;
    in the blocked band form (band half-width 128 and above unless lattice_form 2 asks for the
    window, or lattice_form 1) as many as fit in 24 GiB, split evenly, one launch each
    (factorisations and forward solves as the tasks of one persistent kernel)."""
    N, _, b, nspin, _, _, _ = hf.hf_lattice_info(hf.make_params(cfg))
    nw = cfg["n_matsubara"]
    per = N * (b + 1) * 16
    form = cfg.get("lattice_form", 0)
    if b > 165 or form == 1 or (form == 0 and b >= 128):
        return -(-nspin * nw // max(1, (24 << 30) // per))
    batch = max(1, min(2 * nw, (1 << 30) // per))
    return -(-nspin * nw // batch)


def lattice_flops(N, b, nspin, nw):
    """Algorithmic FP64 flops of one lattice step: per matrix, the band LDL^T trailing updates
    (dmax (dmax + 1) / 2 complex multiply-adds at step k, dmax = min(b, N - 1 - k)) and the
    selected-inversion products (dmax^2 + dmax), 8 real flops per complex multiply-add."""
    cfma = 0
    for k in range(N):
        d = min(b, N - 1 - k)
        cfma += d * (d + 1) // 2 + d * d + d
    return 8.0 * cfma * nspin * nw


_W3 = {}


def _pool3_lattice(job):
    import numpy as np

    from oracle.lattice import lattice_step
    from oracle.rdmft import RDMFT

    name, idx = job
    cfg = wl.CONFIGS[name]
    if _W3.get("name") != name:
        r = RDMFT(cfg["Lx"], cfg["Ly"], geometry=cfg["geometry"], periodic=bool(cfg["periodic"]),
                  U=cfg["U"], V0=cfg["V0"], mu=cfg["mu"], beta=cfg["beta"], L=8,
                  nw=cfg["n_matsubara"], chains=1, seed=cfg["seed"], h_seed=cfg["h_seed"],
                  Lz=cfg["Lz"])
        _W3.update(name=name, H0=r.lat.H0, full=r.expand_sigma())
    idx = np.asarray(idx)
    for sp in range(2):
        lattice_step(_W3["H0"], cfg["mu"], cfg["beta"], _W3["full"][sp][idx], n_index=idx)
    return len(idx)


def _pool3_chains(job):
    import numpy as np

    import oracle as o

    name, chains = job
    cfg = wl.CONFIGS[name]
    L = int(round(cfg["beta"] / cfg["dtau"]))
    baths = wl.random_baths(cfg["seed"], max(chains) + 1, cfg["beta"], L)
    _, lam = o.constants(cfg["beta"], cfg["U"], L)
    for c in chains:
        g0u, g0d = o.build_g0(baths[c, 0]), o.build_g0(baths[c, 1])
        s = o.init_fields(cfg["seed"], c, 0, L)
        Gu, _ = o.dyson(g0u, s, 1, lam)
        Gd, _ = o.dyson(g0d, s, -1, lam)
        bins = np.zeros((cfg["n_measure"] // cfg["bin_size"], 2 * L + 3))
        o.run_chain(lam, g0u, g0d, cfg["seed"], c, 0, 0, cfg["n_warmup"], cfg["n_measure"],
                    cfg["refresh_every"], cfg["bin_size"], s, Gu, Gd, bins)
    return len(chains)


def cpu_oracle_3d(name, n_chains_total, chains_per_core=8, freqs_per_core=1):
    """Oracle seconds of one iteration of a three-dimensional workload on every host core, from a
    bounded sample (chains and lattice frequencies over a spawned pool, one BLAS thread each);
    returns (seconds, cores, sample)."""
    cfg = wl.CONFIGS[name]
    cores = host_cores()
    ctx = mp.get_context("spawn")
    saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
    for k in saved:
        os.environ[k] = "1"
    try:
        pool = ctx.Pool(cores)
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    try:
        nw = cfg["n_matsubara"]
        pool.map(_pool3_lattice, [(name, [0])] * cores, chunksize=1)      # warm: lattice, imports
        n_freq = min(nw, cores * freqs_per_core)
        idx = [int(k * (nw // n_freq)) for k in range(n_freq)]
        t0 = time.perf_counter()
        pool.map(_pool3_lattice, [(name, idx[w::cores]) for w in range(cores) if idx[w::cores]],
                 chunksize=1)
        t_lat = (time.perf_counter() - t0) * (nw / n_freq)
        n = cores * chains_per_core
        t0 = time.perf_counter()
        pool.map(_pool3_chains, [(name, list(range(w, n, cores))) for w in range(cores)], chunksize=1)
        t_qmc = (time.perf_counter() - t0) * (n_chains_total / n)
    finally:
        pool.close()
        pool.join()
    L = int(round(cfg["beta"] / cfg["dtau"]))
    sample = ("%d of %d chains x 2500 sweeps (L=%d) + lattice step at %d of %d frequencies x 2 "
              "spins (dense inverse) over %d worker processes, each scaled to the full iteration"
              % (n, n_chains_total, L, n_freq, nw, cores))
    return t_lat + t_qmc, cores, sample


def run_lattice3d(args):
    """Three-dimensional workloads (slab16, box12, box14p, box16p): whole RDMFT iterations with the FP32-pair
    sweeps, reported with the rooflines of both the impurity sweeps and the lattice step, which
    in three dimensions is no longer small."""
    import torch

    from paper_1006_2716_gb300 import hf

    rank, world, local = dist_env()
    if rank != 0:
        return 0
    name = args.workload
    cfg = dict(wl.CONFIGS[name])
    if args.sweeps:
        # short QMC launch for profiling captures only (not a benchmark value)
        nm = args.sweeps - args.sweeps // 5
        cfg.update(n_warmup=args.sweeps // 5, n_measure=nm, bin_size=max(1, nm // 4))
    if args.matsubara:
        cfg.update(n_matsubara=args.matsubara)   # profiling captures only (not a benchmark value)
    if args.lattice_form:
        cfg.update(lattice_form=args.lattice_form)
    N, ns, b, nspin, _, _, _ = hf.hf_lattice_info(hf.make_params(cfg))
    nc = ns * cfg["chains_per_site"]
    cpu = None
    if not args.no_cpu:   # spawned before any CUDA work
        secs, cores, sample = cpu_oracle_3d(name, nc)
        L0 = int(round(cfg["beta"] / cfg["dtau"]))
        cpu = {"value": nc * (cfg["n_warmup"] + cfg["n_measure"]) * L0 / secs,
               "unit": "proposals/s", "cores": cores, "kind": "oracle", "sample": sample}
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    stream = torch.cuda.Stream(dev)
    ctx = hf.Context(hf.make_params(cfg), device=dev, stream=stream)
    L, nw = ctx.L, ctx.nw
    sweeps = cfg["n_warmup"] + cfg["n_measure"]
    proposals = nc * sweeps * L
    n_refresh = sweeps // cfg["refresh_every"] + 1
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    for _ in range(args.warmup):
        hf.hf_rdmft_step(ctx.handle)
    torch.cuda.synchronize(dev)
    clocks = ClockSampler(local)
    acc0 = hf.hf_get_accepts(ctx.handle, nc).sum()
    ms_steps, qmc_ms, phase = _time_iterations(hf, ctx, stream, flush, args.steps)
    clk = clocks.stop()
    accepts = int(hf.hf_get_accepts(ctx.handle, nc).sum() - acc0) / args.steps
    ms_per = statistics.mean(ms_steps)
    phase = phase / args.steps
    e2e = e2e_iterations(hf, ctx, dev, args.steps, proposals)
    qroof = qmc_roofline(2, L, nc, sweeps, accepts, cfg["n_measure"], n_refresh,
                         statistics.mean(qmc_ms) / 1e3, "qmc_df64_kernel")
    qroof["acceptance"] = accepts / proposals
    lform, lat_launches, cfma, tc_flops = hf.hf_get_lattice_plan(ctx.handle)
    fl = 8.0 * cfma * nspin * nw
    lat_s = phase[0] / 1e3
    lkern = "lattice_wide_kernel" if lform == 1 else "lattice_kernel"
    form = ("blocked band L D L^T + forward solves" if lform == 1
            else "band L D L^T + selected inversion in a shared-memory window")
    if tc_flops > 0:
        # panels, trailing updates and solves as exact digit products on the tensor cores: the
        # roof is the bf16 pipe; the FP64-equivalent rate of the algorithm is reported beside it
        tfl = tc_flops * nspin * nw
        lroof = {"bound": "tensor", "achieved": tfl / lat_s / 1e12, "peak": MEASURED_BF16_SUSTAINED,
                 "unit": "TFLOP/s", "frac": tfl / lat_s / 1e12 / MEASURED_BF16_SUSTAINED,
                 "traffic": measured_traffic(lkern + ":" + name),
                 "kernel": lkern, "matrices": nspin * nw, "N": N, "band": b,
                 "form": form + ", products on the tensor cores", "seconds": lat_s,
                 "work": "bf16 flops of the exact digit products (panels below their diagonal "
                         "blocks, trailing updates, forward solves); the diagonal blocks and the "
                         "solves' own triangles run on the FP64 pipe",
                 "algorithmic_fp64_tflops": fl / lat_s / 1e12,
                 "algorithmic_fp64_vs_fp64_nominal": fl / lat_s / 1e12 / FP64_PEAK_TFLOPS,
                 "peak_source": "measured dense bf16 (cuBLAS, sustained) of this GPU"}
    else:
        lroof = {"bound": "alu", "achieved": fl / lat_s / 1e12, "peak": FP64_PEAK_TFLOPS,
                 "unit": "TFLOP/s", "frac": fl / lat_s / 1e12 / FP64_PEAK_TFLOPS,
                 "traffic": measured_traffic(lkern + ":" + name),
                 "kernel": lkern, "matrices": nspin * nw, "N": N, "band": b,
                 "form": form, "seconds": lat_s,
                 "peak_source": "FP64 nominal: 2 DFMA/clk/SM x 152 SMs x 2.07 GHz"}
    dominant = lroof if phase[0] > phase[2] else qroof
    geo = ("%dx%d slab of %d layers, periodic in all directions, cylindrical trap" % (cfg["Lx"], cfg["Ly"], cfg["Lz"])
           if cfg["geometry"] == 3 else
           "%dx%dx%d %s box, spherical trap" % (cfg["Lx"], cfg["Ly"], cfg["Lz"],
                                                 "periodic" if cfg["periodic"] else "open"))
    line = {"metric": METRIC, "value": proposals / (ms_per / 1e3), "unit": "proposals/s",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32x2+f64", "data": "synthetic",
            "config": {"workload": "%s: %s (%d sites, %d inequivalent, band half-width %d), U=%g, "
                                   "V0=%g, mu=%g, beta=%g, dtau=%g (L=%d), %d chains per site, "
                                   "500+2000 sweeps, 500 Matsubara frequencies; one step = one "
                                   "RDMFT iteration" % (name, geo, N, ns, b, cfg["U"], cfg["V0"],
                                                        cfg["mu"], cfg["beta"], cfg["dtau"], L,
                                                        cfg["chains_per_site"]),
                       "chains": nc, "time_slices": L,
                       "l2": "flushed (256 MB write) between timed steps"},
            "rdmft_iteration_ms": ms_per,
            "phase_ms": dict(zip(["lattice", "weiss_tau", "qmc", "reduce", "sigma"],
                                 [float(x) for x in phase])),
            "roofline": dominant, "qmc_roofline": qroof, "lattice_roofline": lroof,
            "gpu_launches": (lattice_launches(hf, cfg) + 5) * args.steps,
            "cpu_baseline": cpu, "e2e": e2e, "clocks": clk}
    if args.sweeps or args.matsubara:
        over = []
        if args.sweeps:
            over.append("sweeps to %d" % args.sweeps)
        if args.matsubara:
            over.append("Matsubara frequencies to %d" % args.matsubara)
        line["profile_case"] = "overridden: %s; not a benchmark value" % ", ".join(over)
    print(json.dumps(line))
    ctx.close()
    return 0


def run_entropy6(args):
    """Entropy from dS/dmu = dN/dT on the 6x6 trap at U = 4, T = 0.5 (beta = 2, L = 8): RDMFT runs
    at T -+ 0.05 on 41 chemical potentials from -10 (empty trap) to 2 (half filling at the centre),
    6 iterations each, in fused batches of 8 runs; one step = the whole scan.  Timed on the host
    clock (context set-up included, as a user of the scan sees it)."""
    import numpy as np
    import torch

    from paper_1006_2716_gb300 import hf, thermo

    rank, world, local = dist_env()
    if rank != 0:
        return 0
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    cfg = dict(wl.CONFIGS["square6"], U=4.0, precision=2, chains_per_site=8, n_warmup=200,
               n_measure=800, bin_size=100)
    T, dT, L, iters = 0.5, 0.05, 8, 6
    mus = np.linspace(-10.0, 2.0, 41)
    _, ns, _, _, rep, _, _ = hf.hf_lattice_info(hf.make_params(cfg))
    sweeps = cfg["n_warmup"] + cfg["n_measure"]
    proposals = 2 * len(mus) * iters * ns * cfg["chains_per_site"] * sweeps * L
    # launches of one scan: per batch of nb runs and iteration, nb x (lattice, Weiss/tau, g0^-1,
    # reduction, self-energy) and one fused sweep launch; one field initialisation per run
    runs = 2 * len(mus)
    sizes = [min(8, runs - b) for b in range(0, runs, 8)]
    launches = sum(iters * ((lattice_launches(hf, cfg) + 4) * nb + 1) + nb for nb in sizes)
    # centre of the bond-centred square: the orbit closest to the trap centre
    c = (cfg["Lx"] - 1) / 2.0
    centre = int(np.argmin([(r % cfg["Lx"] - c) ** 2 + (r // cfg["Lx"] - c) ** 2 for r in rep]))
    for _ in range(max(0, args.warmup)):
        thermo.entropy_scan(cfg, T, dT, mus[:3], L, 1, device=dev)
    torch.cuda.synchronize(dev)
    clocks = ClockSampler(local)
    times, res = [], None
    for _ in range(args.steps):
        t0 = time.perf_counter()
        res = thermo.entropy_scan(cfg, T, dT, mus, L, iters, device=dev)
        torch.cuda.synchronize(dev)
        times.append(time.perf_counter() - t0)
    clk = clocks.stop()
    wall = statistics.mean(times)
    line = {"metric": METRIC, "value": proposals / wall, "unit": "proposals/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": wall * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32x2+f64", "data": "synthetic",
            "config": {"workload": "entropy6: 6x6 trap, U=4, V0=0.1, T=0.5 -+ 0.05 (beta ~2, L=8), "
                                   "41 mu in [-10, 2], 6 RDMFT iterations per point, 8 chains per "
                                   "site, 200+800 sweeps; one step = the whole scan (82 runs)",
                       "timing": "host clock around the scan, context set-up included"},
            "scan_points_per_s": 2 * len(mus) / wall,
            "entropy": {"mu": float(res["mu"][-1]), "S": float(res["S"][-1]),
                        "N": float(res["N"][-1]), "S_per_particle": float(res["S"][-1] / res["N"][-1]),
                        "centre_site_entropy": float(res["s_site"][centre, -1]),
                        "centre_site_density": float(res["n_site"][-1, centre])},
            "gpu_launches": launches * args.steps, "cpu_baseline": None, "clocks": clk}
    print(json.dumps(line))
    return 0


def run_fig1(args):
    """Physics cross-check with the parameters of the paper's Fig. 1 (square lattice, V0 = 0.25,
    U = 10, dtau = 0.1): a site-centred 17x17 trap half filled at its centre (mu = U/2), converged
    RDMFT (mixing 0.5 from the staggered seed field) at T = 0.156, 0.25 and 0.5 (L = 64, 40, 20).
    Reports the radial profiles of density, double occupancy and staggered moment, and the
    paper's statements: a core polarised up to 90% at low T, no order above T_N ~ 0.32, a double
    occupancy near 0.02 at the centre at high T that the AF core enhances by up to 50%, and a
    density that hardly changes with T.  One step = all three runs."""
    import numpy as np
    import torch

    from paper_1006_2716_gb300 import hf

    rank, world, local = dist_env()
    if rank != 0:
        return 0
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    stream = torch.cuda.Stream(dev)
    base = dict(wl.CONFIGS["square20"], Lx=17, Ly=17, U=10.0, V0=0.25, mu=5.0, dtau=0.1,
                chains_per_site=16, precision=2, h_seed=0.1, mix=0.5)
    runs = ((0.15625, 64), (0.25, 40), (0.5, 20))
    iters = args.iterations
    _, ns, _, _, rep, _, _ = hf.hf_lattice_info(hf.make_params(dict(base, beta=6.4)))
    c = 8.0
    r = np.sqrt([(q % 17 - c) ** 2 + (q // 17 - c) ** 2 for q in rep])
    parity = np.array([1 if ((q % 17) + (q // 17)) % 2 == 0 else -1 for q in rep])
    order = np.argsort(r, kind="stable")
    clocks = ClockSampler(local)
    t0 = time.perf_counter()
    prof, proposals, launches = {}, 0, 0
    for T, L in runs:
        cfg = dict(base, beta=1.0 / T)
        ctx = hf.Context(hf.make_params(cfg), device=dev, stream=stream)
        for _ in range(iters):
            hf.hf_rdmft_step(ctx.handle)
        mean, err = hf.hf_get_observables(ctx.handle, ns, L)
        n = mean[:, 2 * L] + mean[:, 2 * L + 1]
        d, m = mean[:, 2 * L + 2], mean[:, 2 * L + 3]
        prof[T] = {"n": n, "d": d, "d_err": err[:, 2 * L + 2], "m_stag": m * parity}
        proposals += ctx.n_chains * (cfg["n_warmup"] + cfg["n_measure"]) * L * iters
        # per iteration: lattice step, Weiss/tau, g0^-1, sweeps, reduction, self-energy; one
        # field initialisation per run
        launches += iters * (lattice_launches(hf, cfg) + 5) + 1
        ctx.close()
    torch.cuda.synchronize(dev)
    wall = time.perf_counter() - t0
    clk = clocks.stop()
    lo, mid, hi = (prof[T] for T, _ in runs)
    ctr = int(order[0])
    core = r <= 3.0
    checks = {
        "centre_polarisation_T0.156": float(abs(lo["m_stag"][ctr]) / lo["n"][ctr]),
        "centre_polarisation_T0.5": float(abs(hi["m_stag"][ctr]) / hi["n"][ctr]),
        "max_abs_m_stag_T0.5": float(np.abs(hi["m_stag"]).max()),
        "centre_double_occupancy_T0.5": float(hi["d"][ctr]),
        "max_double_occupancy_T0.5": float(hi["d"].max()),
        "core_double_occupancy_enhancement_T0.156_vs_T0.5": float(lo["d"][core].mean() / hi["d"][core].mean()),
        "max_density_change_T0.156_vs_T0.5": float(np.abs(lo["n"] - hi["n"]).max()),
    }
    line = {"metric": METRIC, "value": proposals / wall, "unit": "proposals/s", "n_gpus": 1,
            "steps": 1, "warmup": 0, "ms_per_step": wall * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32x2+f64", "data": "synthetic",
            "config": {"workload": "fig1: site-centred 17x17 square trap, U=10, V0=0.25, mu=5, "
                                   "dtau=0.1, T = 0.156/0.25/0.5 (L = 64/40/20), 45 inequivalent "
                                   "sites x 16 chains, %d RDMFT iterations per temperature, "
                                   "500+2000 sweeps" % iters,
                       "timing": "host clock around the three runs"},
            "checks": checks,
            "profiles": {str(T): {"r": [float(x) for x in r[order]],
                                  "n": [float(x) for x in prof[T]["n"][order]],
                                  "d": [float(x) for x in prof[T]["d"][order]],
                                  "m_stag": [float(x) for x in prof[T]["m_stag"][order]]}
                         for T, _ in runs},
            "gpu_launches": launches, "cpu_baseline": None, "clocks": clk}
    print(json.dumps(line))
    return 0


def run_square30(args):
    """Mixed precision on the 30x30 trap (120 inequivalent sites x 16 chains, L = 128): FP32
    sweeps with FP32 accumulation, an FP64 Dyson refresh (and the measurement) after every
    sweep; one step = one RDMFT iteration (500 + 2000 sweeps)."""
    import torch

    from paper_1006_2716_gb300 import hf

    rank, world, local = dist_env()
    if rank != 0:
        return 0
    cpu = None
    if not args.no_cpu:   # spawned before any CUDA work
        v, cores, sample = cpu_oracle_square30()
        cpu = {"value": v, "unit": "proposals/s", "cores": cores, "kind": "oracle", "sample": sample}
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    stream = torch.cuda.Stream(dev)
    cfg = dict(wl.CONFIGS["square30"], refresh_gj=args.refresh_gj)
    if args.sweeps:
        # short QMC launch for profiling captures only (not a benchmark value)
        nm = args.sweeps - args.sweeps // 5
        cfg.update(n_warmup=args.sweeps // 5, n_measure=nm, bin_size=max(1, nm // 4))
    ctx = hf.Context(hf.make_params(cfg), device=dev, stream=stream)
    L, nc, ns, nw = ctx.L, ctx.n_chains, ctx.n_sites, ctx.nw
    sweeps = cfg["n_warmup"] + cfg["n_measure"]
    proposals = nc * sweeps * L
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    for _ in range(args.warmup):
        hf.hf_rdmft_step(ctx.handle)
    torch.cuda.synchronize(dev)
    clocks = ClockSampler(local)
    acc0 = hf.hf_get_accepts(ctx.handle, nc).sum()
    ms_steps, qmc_ms, phase = _time_iterations(hf, ctx, stream, flush, args.steps)
    clk = clocks.stop()
    accepts = int(hf.hf_get_accepts(ctx.handle, nc).sum() - acc0) / args.steps
    ms_per = statistics.mean(ms_steps)
    qmc_s = statistics.mean(qmc_ms) / 1e3
    n_tc, n_fb, n_prod = hf.hf_get_refresh_stats(ctx.handle)   # of the last timed iteration
    e2e = e2e_iterations(hf, ctx, dev, args.steps, proposals)
    # the sweeps alone, timed live on a twin context that never refreshes within the launch: the
    # refresh kernels' share of the QMC phase is the difference
    twin = hf.Context(hf.make_params(dict(cfg, refresh_every=100000)), device=dev, stream=stream)
    hf.hf_compute_baths(twin.handle)
    hf.hf_sweep(twin.handle, 2, 0, 1)
    n_tw = min(sweeps, 200)
    hf.hf_sweep(twin.handle, n_tw, 0, 0)
    sweep_s = hf.hf_get_timings(twin.handle)[5] / 1e3 * sweeps / n_tw
    twin.close()
    refresh_s = max(qmc_s - sweep_s, 1e-9)
    f_ref = 2.0 * (8.0 / 3.0) * L ** 3 * nc * sweeps
    f_sweep = 10.0 * L * nc * sweeps + 4.0 * L * L * accepts + 2.0 * L * L * nc * cfg["n_measure"]
    tc = not cfg.get("refresh_gj", 0)
    # FP32 sweeps with delayed rank-8 updates: each G element is read and written once per 8
    # multiply-adds, so the FP32 pipe (128 FFMA/clk/SM), not shared memory, is the roof
    sweep_roof = {"bound": "alu", "kernel": "qmc_f32_kernel", "achieved": f_sweep / sweep_s / 1e12,
                  "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                  "frac": f_sweep / sweep_s / 1e12 / FP32_PEAK_TFLOPS,
                  "traffic": measured_traffic("qmc_f32_kernel"), "seconds": sweep_s,
                  "peak_source": "FP32 nominal: 128 FFMA/clk/SM x 152 SMs x 2.07 GHz"}
    if tc:
        # executed tensor-core work: the digit products the Newton steps ran in the last timed
        # iteration (the library counts them), 2 x 128^3 bf16 flops each
        tflop = n_prod * 2.0 * L ** 3
        ref_roof = {"bound": "tensor", "kernel": "refresh_tc_kernel", "achieved": tflop / refresh_s / 1e12,
                    "peak": MEASURED_BF16_SUSTAINED, "unit": "TFLOP/s",
                    "frac": tflop / refresh_s / 1e12 / MEASURED_BF16_SUSTAINED,
                    "traffic": measured_traffic("refresh_tc_kernel"),
                    "seconds": refresh_s, "algorithmic_fp64_tflops": f_ref / refresh_s / 1e12,
                    "peak_source": "measured dense bf16 (cuBLAS, sustained) of this GPU",
                    "work": "bf16 flops of the exact digit products the refreshes ran",
                    "tensor_refreshes": n_tc, "gauss_jordan_fallbacks": n_fb,
                    "digit_products_per_refresh": n_prod / max(n_tc + n_fb, 1)}
    else:
        ref_roof = {"bound": "alu", "kernel": "refresh_f64_kernel", "achieved": f_ref / refresh_s / 1e12,
                    "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                    "frac": f_ref / refresh_s / 1e12 / FP64_PEAK_TFLOPS, "traffic": None,
                    "seconds": refresh_s, "peak_source": "FP64 nominal: 2 DFMA/clk/SM x 152 SMs x 2.07 GHz"}
    dominant = ref_roof if refresh_s > sweep_s else sweep_roof
    line = {"metric": METRIC, "value": proposals / (ms_per / 1e3), "unit": "proposals/s",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": "square30: 30x30 open trap, U=8, V0=0.03, mu=%.4f, beta=16, "
                                   "dtau=0.125 (L=128), 120 inequivalent sites x 16 chains, "
                                   "500+2000 FP32 sweeps, FP64 refresh every sweep, 500 Matsubara "
                                   "frequencies; one step = one RDMFT iteration" % cfg["mu"],
                       "l2": "flushed (256 MB write) between timed steps"},
            "rdmft_iteration_ms": ms_per,
            "phase_ms": dict(zip(["lattice", "weiss_tau", "qmc", "reduce", "sigma"],
                                 [float(x) for x in phase / args.steps])),
            "roofline": dominant, "sweep_roofline": sweep_roof, "refresh_roofline": ref_roof,
            "refresh": "tensor-core Newton steps" if tc else "FP64 Gauss-Jordan",
            "acceptance": accepts / proposals,
            # per iteration: an FP32 sweep launch and the refresh launches per sweep (tensor-core
            # Newton steps and the Gauss-Jordan pass over the chains they flag, or Gauss-Jordan
            # alone), the first refresh, g0^-1 (and its digits), lattice step, Weiss/tau,
            # reduction, self-energy update
            "gpu_launches": (((3 if tc else 2) * sweeps) + (7 if tc else 6)) * args.steps,
            "cpu_baseline": cpu, "e2e": e2e, "clocks": clk}
    if args.sweeps:
        line["profile_case"] = "sweeps overridden to %d: not a benchmark value" % args.sweeps
    print(json.dumps(line))
    ctx.close()
    return 0


def run_dtau_scan(args):
    """Trotter scan of one impurity (beta = 2, U = 2, 4-pole bath): dtau = beta / L for L = 16,
    24, 32, 48, 64, 2048 chains each, 200 + 2000 sweeps, all five in one fused launch; one step
    = one launch.  Reports proposals/s and the double occupancy extrapolated to dtau -> 0 (fit
    a + b dtau^2 with the measured errors); tests/test_gpu_trotter.py compares that value with
    the exact diagonalisation of the same impurity."""
    import numpy as np
    import torch

    from paper_1006_2716_gb300 import hf

    rank, world, local = dist_env()
    if rank != 0:
        return 0
    beta, U, seed = 2.0, 2.0, 3
    e, w = wl.bath_poles(seed)
    Ls = [16, 24, 32, 48, 64]
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    stream = torch.cuda.Stream(dev)
    ctxs = []
    for k, L in enumerate(Ls):
        cfg = dict(wl.CONFIGS["square6"], Lx=1, Ly=1, beta=beta, dtau=beta / L, U=U, mu=0.0,
                   V0=0.0, precision=2, chains_per_site=2048, n_matsubara=4, refresh_every=10,
                   bin_size=100, max_bins=20, seed=900 + k)
        ctx = hf.Context(hf.make_params(cfg), device=dev, stream=stream)
        bath = wl.pole_bath_tau(beta, L, e, w)
        hf.hf_set_g0(ctx.handle, 0, 0, bath)
        hf.hf_set_g0(ctx.handle, 0, 1, bath)
        ctxs.append(ctx)
    b = hf.hf_batch_create([c.handle for c in ctxs], 0)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def one_step():
        for c in ctxs:
            hf.hf_clear_measurements(c.handle)
        with torch.cuda.stream(stream):
            flush.zero_()
        torch.cuda.synchronize(dev)
        hf.hf_batch_sweep(b, 200, 2000, 1)
        return hf.hf_batch_elapsed(b)

    for _ in range(args.warmup):
        one_step()
    clocks = ClockSampler(local)
    ms = [one_step() for _ in range(args.steps)]
    clk = clocks.stop()
    d, sd = [], []
    for c, L in zip(ctxs, Ls):
        _, _, dd, _, errs = hf.hf_measure(c.handle, 0, L)
        d.append(dd)
        sd.append(errs[2 * L + 2])
    hf.hf_batch_free(b)
    for c in ctxs:
        c.close()
    d, sd = np.array(d), np.array(sd)
    dt = beta / np.array(Ls, dtype=float)
    A = np.stack([np.ones_like(dt), dt ** 2], axis=1) / sd[:, None]
    coef, *_ = np.linalg.lstsq(A, d / sd, rcond=None)
    sa = float(np.sqrt(np.linalg.inv(A.T @ A)[0, 0]))
    proposals = sum(2048 * 2200 * L for L in Ls)
    ms_per = statistics.mean(ms)
    line = {"metric": METRIC, "value": proposals / (ms_per / 1e3), "unit": "proposals/s",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32x2+f64", "data": "synthetic",
            "config": {"workload": "dtau_scan: one impurity, beta=2, U=2, 4-pole bath (seed 3), "
                                   "L 16/24/32/48/64 x 2048 chains in one fused launch, 200+2000 "
                                   "sweeps; one step = one launch",
                       "l2": "flushed (256 MB write) between timed steps"},
            "double_occupancy": {"per_L": dict(zip(map(str, Ls), d.tolist())),
                                 "err_per_L": dict(zip(map(str, Ls), sd.tolist())),
                                 "extrapolated": float(coef[0]), "extrapolated_err": sa},
            "clocks": clk}
    print(json.dumps(line))
    return 0


def _pool_scan_job(job):
    """Oracle work of the scan's cpu baseline: ('chains', beta, [c...]) runs whole 2500-sweep
    chains at that temperature; ('lattice', beta, [n...]) the dense lattice step at those
    frequencies.  Returns seconds."""
    import numpy as np

    import oracle as o
    from oracle.lattice import lattice_step
    from oracle.rdmft import RDMFT

    kind, beta, items = job
    cfg = dict(CFG, beta=beta)
    L = int(round(beta / cfg["dtau"]))
    t0 = time.perf_counter()
    if kind == "lattice":
        r = RDMFT(cfg["Lx"], cfg["Ly"], U=cfg["U"], V0=cfg["V0"], mu=cfg["mu"], beta=beta, L=L,
                  nw=cfg["n_matsubara"], chains=1, seed=cfg["seed"], h_seed=cfg["h_seed"])
        full = r.expand_sigma()
        t0 = time.perf_counter()
        idx = np.asarray(items)
        for sp in range(2):
            lattice_step(r.lat.H0, cfg["mu"], beta, full[sp][idx], n_index=idx)
        return time.perf_counter() - t0
    baths = wl.random_baths(L, max(items) + 1, beta, L)
    _, lam = o.constants(beta, cfg["U"], L)
    for c in items:
        g0u, g0d = o.build_g0(baths[c, 0]), o.build_g0(baths[c, 1])
        s = o.init_fields(cfg["seed"], c, 0, L)
        Gu, _ = o.dyson(g0u, s, 1, lam)
        Gd, _ = o.dyson(g0d, s, -1, lam)
        bins = np.zeros((cfg["n_measure"] // cfg["bin_size"], 2 * L + 3))
        o.run_chain(lam, g0u, g0d, cfg["seed"], c, 0, 0, cfg["n_warmup"], cfg["n_measure"],
                    cfg["refresh_every"], cfg["bin_size"], s, Gu, Gd, bins)
    return time.perf_counter() - t0


def cpu_oracle_scan20(chains_per_core=1):
    """Oracle seconds of one batched scan iteration (4 temperatures x 1760 chains x 2500 sweeps,
    and 4 lattice steps of 500 frequencies x 2 spins) on every host core, from a bounded sample:
    per temperature, chains_per_core chains and one frequency per core, over a spawned pool (one
    process and one BLAS thread per core); each part scaled to the full iteration."""
    cores = host_cores()
    ctx = mp.get_context("spawn")
    saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
    for k in saved:
        os.environ[k] = "1"
    try:
        pool = ctx.Pool(cores)
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    total = 0.0
    try:
        pool.map(_pool_scan_job, [("chains", 5.0, [w]) for w in range(cores)], chunksize=1)
        nw = CFG["n_matsubara"]
        for beta in wl.SCAN20_BETAS:
            n = cores * chains_per_core
            t0 = time.perf_counter()
            pool.map(_pool_scan_job, [("chains", beta, list(range(w, n, cores))) for w in range(cores)],
                     chunksize=1)
            total += (time.perf_counter() - t0) * 1760.0 / n
            idx = [k * (nw // cores) for k in range(cores)]
            t0 = time.perf_counter()
            pool.map(_pool_scan_job, [("lattice", beta, [i]) for i in idx], chunksize=1)
            total += (time.perf_counter() - t0) * nw / len(idx)
    finally:
        pool.close()
        pool.join()
    sample = ("per beta in {5,8,10,16}: %d of 1760 chains x 2500 sweeps (L=20/32/40/64, FP64, "
              "refresh every 10) + the dense lattice step (N=400) at %d of 500 frequencies x 2 "
              "spins, over %d worker processes, each part scaled to the full iteration"
              % (cores * chains_per_core, cores, cores))
    return total, cores, sample


def qmc_flops(L, nchain, sweeps, accepts, n_measure, n_refresh):
    """Algorithmic flops of one sweep launch (proposals, accepted updates, measurements, Dyson
    refreshes as 2 (8/3) L^3 per chain and refresh)."""
    return (10.0 * L * nchain * sweeps + 4.0 * L * L * accepts + 2.0 * L * L * nchain * n_measure
            + 2.0 * (8.0 / 3.0) * L ** 3 * nchain * n_refresh)


def run_scan20(args):
    """Batched uneven-L temperature scan: the 20x20 trap at beta = 5, 8, 10, 16 (L = 20, 32, 40,
    64), 1760 chains each, one fused graph-captured launch per iteration, FP64 sweeps and
    refreshes, team width and delay depth autotuned per L."""
    import numpy as np
    import torch

    from paper_1006_2716_gb300 import autotune, hf

    rank, world, local = dist_env()
    if rank != 0:
        return 0
    cpu = None
    if not args.no_cpu:   # spawned before any CUDA work
        secs, cores, sample = cpu_oracle_scan20()
        props = sum(1760 * 2500 * int(round(b / 0.25)) for b in wl.SCAN20_BETAS)
        cpu = {"value": props / secs, "unit": "proposals/s", "cores": cores, "kind": "oracle",
               "sample": sample}
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    stream = torch.cuda.Stream(dev)
    betas = wl.SCAN20_BETAS
    Ls = [int(round(b / 0.25)) for b in betas]
    form = 0 if args.precision < 0 else args.precision
    tune = {L: autotune.tune_workload("scan20_beta%g" % b, dict(CFG, beta=b), forms=(form,),
                                      device=dev, stream=stream) for b, L in zip(betas, Ls)}
    ctxs = [hf.Context(hf.make_params(dict(CFG, beta=b, precision=form,
                                           team_warps=tune[L]["team_warps"],
                                           delay_k=tune[L]["delay_k"])),
                       device=dev, stream=stream) for b, L in zip(betas, Ls)]
    batch = hf.hf_batch_create([c.handle for c in ctxs], 1)
    for _ in range(max(args.warmup, 2)):      # first call plain, second captures the graph
        hf.hf_batch_rdmft_step(batch)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    ms = []
    acc0 = [hf.hf_get_accepts(c.handle, c.n_chains).sum() for c in ctxs]
    clocks = ClockSampler(local)
    for _ in range(args.steps):
        with torch.cuda.stream(stream):
            flush.zero_()
        torch.cuda.synchronize(dev)
        ms.append(hf.hf_batch_rdmft_step(batch))
    clk = clocks.stop()
    accepts = [(hf.hf_get_accepts(c.handle, c.n_chains).sum() - a) / args.steps
               for c, a in zip(ctxs, acc0)]
    proposals = sum(c.n_chains * 2500 * c.L for c in ctxs)
    ms_per = statistics.mean(ms)
    # the fused sweep launch alone (its g0^-1 launch included), for the kernel's roofline
    with torch.cuda.stream(stream):
        flush.zero_()
    torch.cuda.synchronize(dev)
    for c in ctxs:
        hf.hf_clear_measurements(c.handle)
    hf.hf_batch_sweep(batch, CFG["n_warmup"], CFG["n_measure"], 1)
    qmc_ms = hf.hf_batch_elapsed(batch)
    flops = sum(qmc_flops(c.L, c.n_chains, 2500, a, CFG["n_measure"], 1 + 2500 // CFG["refresh_every"])
                for c, a in zip(ctxs, accepts))
    achieved = flops / (qmc_ms / 1e3) / 1e12
    if form == 0:
        peak, src = FP64_PEAK_TFLOPS, "FP64 nominal: 2 DFMA/clk/SM x 152 SMs x 2.07 GHz"
    else:
        f_ref = sum(2.0 * (8.0 / 3.0) * c.L ** 3 * c.n_chains * (1 + 2500 // CFG["refresh_every"])
                    for c in ctxs)
        t_roof = (f_ref / (FP64_PEAK_TFLOPS * 1e12) +
                  (flops - f_ref) / 2.0 * DF_OPS_PER_FMA / (FP32_PEAK_TFLOPS * 1e12 / 2.0))
        peak, src = flops / t_roof / 1e12, "serial two-pipe roof (refresh FP64, pairs FP32)"
    roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak, "traffic": None, "kernel": "qmc_%s_kernel (fused, 4 problems)"
            % ("f64" if form == 0 else "df64"), "qmc_ms": qmc_ms, "peak_source": src,
            "algorithmic_bytes": sum(qmc_alg_bytes(c.L, c.n_chains, c.n_sites, CFG["n_measure"],
                                                   CFG["bin_size"]) for c in ctxs)}
    # end to end through the public API with host buffers: every step sends each run's
    # self-energy to the device, runs the batched iteration and reads back each run's observables
    # and self-energy
    nw = ctxs[0].nw
    pins = [(torch.empty(c.n_sites * 2 * nw * 2, dtype=torch.float64, pin_memory=True),
             torch.empty(2 * c.n_sites * (2 * c.L + 4), dtype=torch.float64, pin_memory=True))
            for c in ctxs]
    sig = []
    for c, (ps, _) in zip(ctxs, pins):
        v = ps.numpy().view(np.complex128).reshape(c.n_sites, 2, nw)
        v[:] = hf.hf_get_sigma(c.handle, c.n_sites, nw)
        sig.append(v)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        for c, v in zip(ctxs, sig):
            hf.lib().hf_set_sigma(c.handle, v.ctypes.data_as(hf._DP))
        hf.hf_batch_rdmft_step(batch)
        for c, v, (_, po) in zip(ctxs, sig, pins):
            obs = po.numpy()
            hf.lib().hf_get_observables(c.handle, obs.ctypes.data_as(hf._DP),
                                        obs[c.n_sites * (2 * c.L + 4):].ctypes.data_as(hf._DP))
            hf.lib().hf_get_sigma(c.handle, v.ctypes.data_as(hf._DP))
    torch.cuda.synchronize(dev)
    e2e_s = (time.perf_counter() - t0) / args.steps
    h2d = sum(v.nbytes for v in sig)
    d2h = h2d + sum(po.numpy().nbytes for _, po in pins)
    line = {"metric": METRIC, "value": proposals / (ms_per / 1e3), "unit": "proposals/s",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if form == 0 else "f32x2+f64", "data": "synthetic",
            "config": {"workload": "scan20: 20x20 trap at beta 5/8/10/16 (L 20/32/40/64), "
                                   "4 x 1760 chains in one fused graph-captured launch, "
                                   "500+2000 sweeps; one step = one batched RDMFT iteration",
                       "l2": "flushed (256 MB write) between timed steps"},
            "rdmft_iteration_ms": ms_per, "roofline": roof, "cpu_baseline": cpu,
            "e2e": {"value": proposals / e2e_s, "unit": "proposals/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h},
            # per step: one graph replay holding, per run, the lattice-step launches, Weiss/tau,
            # g0^-1 and two memsets, reduction and self-energy update, plus the fused sweep launch
            "gpu_launches": args.steps * (sum(lattice_launches(hf, dict(CFG, beta=b)) + 4
                                              for b in betas) + 1),
            "clocks": clk, "autotune": {str(L): tune[L] for L in Ls}}
    print(json.dumps(line))
    hf.hf_batch_free(batch)
    for c in ctxs:
        c.close()
    return 0


def run_disc40(args):
    """Serving (FP64 sweeps unless --precision 2): impurity solves for the radius-40 disc (5025 sites, 663 inequivalent, U = 8)
    from 4 concurrent RDMFT runs at (beta, V0) = (8, .010), (10, .010), (16, .010), (8, .015),
    i.e. L = 32, 40, 64, 32; 16 chains x (200 + 1000) sweeps per solve.  Baths come from each
    run's own lattice step.  Capacity = all 2652 solves submitted at once; then Poisson streams at
    0.5 / 0.7 / 0.9 of capacity over warm keys give p50 / p99 latency."""
    import numpy as np
    import torch

    from paper_1006_2716_gb300 import hf

    rank, world, local = dist_env()
    if rank != 0:
        return 0
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    runs = [(8.0, 0.010), (10.0, 0.010), (16.0, 0.010), (8.0, 0.015)]
    form = 0 if args.precision < 0 else args.precision
    baths, Ls = [], []
    for beta, V0 in runs:
        cfg = dict(Lx=40, geometry=1, U=8.0, V0=V0, mu=4.0, beta=beta, dtau=0.25,
                   chains_per_site=1, n_warmup=1, n_measure=1, bin_size=1, max_bins=1,
                   precision=2, seed=7)
        ctx = hf.Context(hf.make_params(cfg), device=dev)
        hf.hf_compute_baths(ctx.handle)
        baths.append(hf.hf_get_g0(ctx.handle, ctx.n_sites, ctx.L))
        Ls.append(ctx.L)
        nsite = ctx.n_sites
        ctx.close()
    sp = hf.hf_srv_params()
    for k, v in dict(chains_per_request=16, n_warmup=200, n_measure=1000, refresh_every=10,
                     bin_size=100, precision=form, team_warps=0, max_L=64, max_inflight=160,
                     max_keys=len(runs) * nsite, n_streams=12, requests_per_launch=16).items():
        setattr(sp, k, v)
    srv = hf.Server(sp, device=dev)

    def req(run, site):
        beta = runs[run][0]
        return hf.make_request(run, site, Ls[run], beta, 8.0, 1000 + run, baths[run][site])

    # one solve on an idle service: the per-impurity latency floor
    t = hf.hf_srv_submit(srv.handle, req(0, 0))
    alone = hf.hf_srv_wait(srv.handle, t, 600)["latency_s"]
    # capacity: every (run, site) solve at once (cold keys)
    keys = [(r, s) for s in range(nsite) for r in range(len(runs))]
    clocks = ClockSampler(local)
    t0 = time.perf_counter()
    tickets = [hf.hf_srv_submit(srv.handle, req(r, s)) for r, s in keys]
    lat_cap = [hf.hf_srv_wait(srv.handle, tk, 600)["latency_s"] for tk in tickets]
    cap_s = time.perf_counter() - t0
    capacity = len(keys) / cap_s
    rng = np.random.default_rng(5)
    loads = []
    n_req = args.serve_requests
    for frac in (0.5, 0.7, 0.9):
        rate = frac * capacity
        pick = rng.integers(0, len(keys), n_req)
        gaps = rng.exponential(1.0 / rate, n_req)
        tks = []
        t_start = time.perf_counter()
        t_next = t_start
        for i in range(n_req):
            t_next += gaps[i]
            while time.perf_counter() < t_next:
                time.sleep(min(2e-4, max(0.0, t_next - time.perf_counter())))
            r, s = keys[pick[i]]
            tks.append(hf.hf_srv_submit(srv.handle, req(r, s)))
        res = [hf.hf_srv_wait(srv.handle, tk, 600) for tk in tks]
        wall = time.perf_counter() - t_start
        lat = np.array([x["latency_s"] for x in res])
        loads.append({"offered_fraction": frac, "offered_solves_per_s": rate,
                      "achieved_solves_per_s": n_req / wall, "p50_s": float(np.percentile(lat, 50)),
                      "p99_s": float(np.percentile(lat, 99)),
                      "warm_fraction": float(np.mean([x["warm"] for x in res]))})
    clk = clocks.stop()
    st = hf.hf_srv_stats(srv.handle)
    srv.close()
    line = {"metric": "p50/p99 solve latency and solves/s (served)", "value": capacity,
            "unit": "solves/s", "n_gpus": 1, "steps": 1, "warmup": 0, "ms_per_step": cap_s * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if form == 0 else "f32x2+f64", "data": "synthetic",
            "config": {"workload": "disc40: site-centred disc r=40 (5025 sites, 663 inequivalent), "
                                   "U=8, mu=4, 4 runs (beta,V0)=(8,.010),(10,.010),(16,.010),(8,.015) "
                                   "-> L 32/40/64/32; 16 chains x (200+1000) sweeps per solve",
                       "inflight_cap": sp.max_inflight, "streams": sp.n_streams},
            "alone_latency_s": alone, "per_impurity_solves_per_s": 1.0 / alone,
            "capacity_solves_per_s": capacity,
            "capacity_latency_p50_s": float(np.percentile(lat_cap, 50)),
            "capacity_latency_p99_s": float(np.percentile(lat_cap, 99)),
            "poisson": loads, "clocks": clk, "peak_inflight": st["peak_inflight"],
            "peak_device_bytes": st["peak_bytes"]}
    print(json.dumps(line))
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
    ap.add_argument("--delay-k", type=int, default=1, choices=[1, 4, 8, 16, 32],
                    help="delayed-update depth (FP32-pair form)")
    ap.add_argument("--precision", type=int, default=-1, choices=[-1, 0, 2],
                    help="sweep arithmetic: 0 FP64, 2 FP32 pairs (48-bit; both with FP64 "
                         "refresh); -1 (default): FP64 with the autotuned team width")
    ap.add_argument("--workload", default="square20",
                    choices=["square20", "scan20", "square30", "disc40", "dtau_scan", "slab16",
                             "box12", "box14p", "box16p", "entropy6", "fig1"])
    ap.add_argument("--refresh-stagger", type=int, default=0, choices=[0, 1],
                    help="1: per-chain refresh phases; 0 (default): every chain refreshes on the "
                         "same sweeps")
    ap.add_argument("--refresh-gj", type=int, default=0, choices=[0, 1],
                    help="square30: 1 refreshes by FP64 Gauss-Jordan instead of the tensor-core "
                         "Newton steps")
    ap.add_argument("--serve-requests", type=int, default=600,
                    help="disc40: requests per Poisson load level")
    ap.add_argument("--no-other-form", action="store_true",
                    help="skip the second sweep form measured beside the headline one")
    ap.add_argument("--iterations", type=int, default=20,
                    help="fig1: RDMFT iterations per temperature")
    ap.add_argument("--sweeps", type=int, default=0,
                    help="profiling only: override sweeps per iteration (result is not a bench value)")
    ap.add_argument("--matsubara", type=int, default=0,
                    help="profiling only, 3D workloads: override the Matsubara frequencies, i.e. "
                         "the lattice step's matrices (result is not a bench value)")
    ap.add_argument("--lattice-form", type=int, default=0, choices=(0, 1, 2),
                    help="3D workloads: the lattice step's form (0 automatic, 1 blocked band "
                         "form, 2 shared-memory window form)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "scan20":
        return run_scan20(args)
    if args.workload == "disc40":
        return run_disc40(args)
    if args.workload == "square30":
        return run_square30(args)
    if args.workload == "fig1":
        return run_fig1(args)
    if args.workload == "entropy6":
        return run_entropy6(args)
    if args.workload in ("slab16", "box12", "box14p", "box16p"):
        return run_lattice3d(args)
    if args.workload == "dtau_scan":
        return run_dtau_scan(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
