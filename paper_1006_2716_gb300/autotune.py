"""Autotuner of the sweep kernels: for each slice count L, the arithmetic form of the FP64-class
sweeps (0 = FP64, 2 = FP32 pairs with FP64 refresh; both meet the FP64 parity bar), the number of
warps per Markov chain and the delayed-update depth k in {1, 4, 8, 16, 32} (FP32-pair form) that
give the most proposals per second on this GPU.

Each candidate runs the real fused sweep kernel and is timed with CUDA events on the context
stream (hf_get_timings): ``tune_workload`` runs whole RDMFT iterations of a workload configuration
(its own baths, measurement cadence and acceptance rates); ``tune`` probes a synthetic
single-impurity problem per L.  Results are cached per GPU name in ``_build/autotune.json``.
"""
from __future__ import annotations

import json
import os

import numpy as np

from . import hf
from . import workloads as wl

_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "autotune.json")


DELAYS = (1, 4, 8, 16, 32)


def _fits(L, tw, k):
    # per-block shared memory of the FP32-pair kernel: (4 / tw) chains x (G pair buffers and
    # scratch + delayed-update buffers), limit 227 KB
    team = ((2 * L * L + 7 * L + 11) * 8 + 16 + ((L + 15) // 16) * 16 + 15) // 16 * 16
    delayed = (4 * k * L + 2 * L) * 8 if k > 1 else 0
    return (4 // tw) * (team + delayed) <= 227 * 1024


def candidates(L, forms=(0, 2)):
    """(form, warps per chain, delay depth) triples.  Delayed updates exist in the FP32-pair form
    and run with one warp per chain (L <= 32)."""
    tws = (1, 2, 4) if L <= 32 else (2, 4)
    out = []
    for f in forms:
        for tw in tws:
            for k in (DELAYS if (f == 2 and tw == 1) else (1,)):
                if f == 0 or _fits(L, tw, k):
                    out.append((f, tw, k))
    return out


def _probe(L, chains, form, tw, k, sweeps, device, stream):
    beta = 0.25 * L
    cfg = dict(Lx=1, Ly=1, geometry=0, U=8.0, V0=0.0, mu=4.0, beta=beta, dtau=0.25,
               n_matsubara=4, chains_per_site=chains, precision=form, team_warps=tw, delay_k=k,
               refresh_every=10, bin_size=max(1, sweeps), max_bins=1, n_warmup=0,
               n_measure=sweeps, seed=12345)
    ctx = hf.Context(hf.make_params(cfg), device=device, stream=stream)
    bath = wl.random_baths(L, 1, beta, L)[0]
    hf.hf_set_g0(ctx.handle, 0, 0, bath[0])
    hf.hf_set_g0(ctx.handle, 0, 1, bath[1])
    hf.hf_sweep(ctx.handle, 2, 0, 1)                     # warm-up (module load, attributes)
    best = np.inf
    for _ in range(2):
        hf.hf_sweep(ctx.handle, sweeps, 0, 0)
        best = min(best, hf.hf_get_timings(ctx.handle)[5])
    ctx.close()
    return best / sweeps                                  # ms per sweep of all chains


def _probe_workload(cfg, form, tw, k, iterations, device, stream):
    """ms per sweep of the QMC phase of a full RDMFT iteration of the workload itself (its own
    warm-up/measurement mix, refresh cadence and equilibrium acceptance); best of the iterations
    after the first."""
    c = dict(cfg, precision=form, team_warps=tw, delay_k=k)
    ctx = hf.Context(hf.make_params(c), device=device, stream=stream)
    best = np.inf
    for it in range(iterations):
        hf.hf_rdmft_step(ctx.handle)
        if it > 0:
            best = min(best, hf.hf_get_timings(ctx.handle)[2])
    ctx.close()
    return best / (c["n_warmup"] + c["n_measure"])


def tune_workload(name, cfg, forms=(0, 2), iterations=2, device="cuda:0", stream=None,
                  use_cache=True):
    """Best (form, team width, delay depth) for one workload configuration, probed on that
    workload: each candidate runs whole RDMFT iterations of it (lattice step, sweeps with the
    workload's measurement cadence, reduction, self-energy update)."""
    import torch

    L = int(round(cfg["beta"] / cfg["dtau"]))
    gpu = torch.cuda.get_device_name(torch.device(device))
    cache = {}
    if use_cache and os.path.exists(_CACHE):
        try:
            cache = json.load(open(_CACHE))
        except (OSError, ValueError):
            cache = {}
    key = "%s|%s|L=%d|forms=%s|v4" % (gpu, name, L, ",".join(map(str, forms)))
    if key not in cache:
        table = {}
        for form, tw, k in candidates(L, forms):
            table["%d/%d/%d" % (form, tw, k)] = _probe_workload(cfg, form, tw, k, iterations,
                                                                device, stream)
        pick = min(table, key=table.get)
        f, tw, k = map(int, pick.split("/"))
        cache[key] = {"precision": f, "team_warps": tw, "delay_k": k, "ms_per_sweep": table[pick],
                      "table": table}
    if use_cache:
        os.makedirs(os.path.dirname(_CACHE), exist_ok=True)
        json.dump(cache, open(_CACHE, "w"), indent=1, sort_keys=True)
    return cache[key]


def tune(Ls, chains, forms=(0, 2), sweeps=30, device="cuda:0", stream=None, use_cache=True):
    """{L: {"precision": f, "team_warps": tw, "ms_per_sweep": t, "table": {...}}} for every L."""
    import torch

    name = torch.cuda.get_device_name(torch.device(device))
    cache = {}
    if use_cache and os.path.exists(_CACHE):
        try:
            cache = json.load(open(_CACHE))
        except (OSError, ValueError):
            cache = {}
    out = {}
    for L in Ls:
        key = "%s|L=%d|chains=%d|forms=%s|v3" % (name, L, chains, ",".join(map(str, forms)))
        if key not in cache:
            table = {}
            for form, tw, k in candidates(L, forms):
                table["%d/%d/%d" % (form, tw, k)] = _probe(L, chains, form, tw, k, sweeps, device,
                                                           stream)
            pick = min(table, key=table.get)
            f, tw, k = map(int, pick.split("/"))
            cache[key] = {"precision": f, "team_warps": tw, "delay_k": k,
                          "ms_per_sweep": table[pick], "table": table}
        out[L] = cache[key]
    if use_cache:
        os.makedirs(os.path.dirname(_CACHE), exist_ok=True)
        json.dump(cache, open(_CACHE, "w"), indent=1, sort_keys=True)
    return out
