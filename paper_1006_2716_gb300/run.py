"""Command-line RDMFT run on one GPU: iterate the self-consistency of eq. 2 with the Hirsch-Fye
impurity solver, log every iteration as one JSON line, and checkpoint and resume.

    python -m paper_1006_2716_gb300.run --workload square20 --iterations 20 --log run.jsonl
    python -m paper_1006_2716_gb300.run --config my.json --set U=10 --set V0=0.25 \\
        --iterations 30 --checkpoint ck.npz
    python -m paper_1006_2716_gb300.run --resume ck.npz --iterations 10 --log more.jsonl

A configuration is a workload of `workloads.CONFIGS` or a JSON object with the same keys (the
fields of hf_params: lattice, model, QMC settings), overridden by --set key=value.  Between
iterations the whole state of a run is its self-energy, its Ising fields and their sweep
counters.  The checkpoint holds exactly these (with the configuration and the iteration count),
so a resumed run continues the same Markov chains.
"""
from __future__ import annotations

import argparse
import json
import sys

import numpy as np

from . import hf
from . import workloads as wl

# the configuration keys make_params reads, with their types
_KEYS = {"Lx": int, "Ly": int, "Lz": int, "geometry": int, "periodic": int, "t": float,
         "U": float, "V0": float, "mu": float, "beta": float, "dtau": float,
         "n_matsubara": int, "chains_per_site": int, "precision": int, "refresh_every": int,
         "refresh_stagger": int, "check_drift": int, "refresh_gj": int, "lattice_form": int, "delay_k": int, "team_warps": int,
         "bin_size": int, "max_bins": int, "n_warmup": int, "n_measure": int, "seed": int,
         "h_seed": float, "mix": float}


def parse_overrides(items):
    """['U=10', 'Lx=16'] -> {'U': 10.0, 'Lx': 16}; unknown keys are an error."""
    out = {}
    for it in items or ():
        if "=" not in it:
            raise ValueError("--set expects key=value, got %r" % it)
        k, v = it.split("=", 1)
        k = k.strip()
        if k not in _KEYS:
            raise ValueError("unknown configuration key %r (known: %s)" % (k, ", ".join(sorted(_KEYS))))
        out[k] = _KEYS[k](v)
    return out


def load_config(workload=None, path=None, overrides=None):
    """A workload's configuration or a JSON file's, with overrides applied."""
    if (workload is None) == (path is None):
        raise ValueError("give exactly one of a workload name and a configuration file")
    if workload is not None:
        if workload not in wl.CONFIGS:
            raise ValueError("unknown workload %r (known: %s)" % (workload, ", ".join(sorted(wl.CONFIGS))))
        cfg = dict(wl.CONFIGS[workload])
    else:
        with open(path) as fh:
            cfg = json.load(fh)
        bad = sorted(set(cfg) - set(_KEYS))
        if bad:
            raise ValueError("unknown configuration keys in %s: %s" % (path, ", ".join(bad)))
    cfg.update(overrides or {})
    return cfg


def iteration_record(iteration, phase_ms, mean, err, L, sigma_before, sigma_after, multiplicity,
                     drift=None):
    """One JSON-serialisable line per iteration: device times of the phases, the per-site
    (inequivalent site) density n = n_up + n_dn, double occupancy d and moment m = n_up - n_dn
    with their errors, the particle number N = sum of multiplicity x n, and the largest change of
    the self-energy over the iteration."""
    n = mean[:, 2 * L] + mean[:, 2 * L + 1]
    n_err = np.hypot(err[:, 2 * L], err[:, 2 * L + 1])
    rec = {
        "iteration": int(iteration),
        "ms": {k: float(v) for k, v in zip(("lattice", "weiss_tau", "qmc", "reduce", "sigma"),
                                           phase_ms[:5])},
        "n": [float(x) for x in n], "n_err": [float(x) for x in n_err],
        "d": [float(x) for x in mean[:, 2 * L + 2]], "d_err": [float(x) for x in err[:, 2 * L + 2]],
        "m": [float(x) for x in mean[:, 2 * L + 3]], "m_err": [float(x) for x in err[:, 2 * L + 3]],
        "N": float(np.dot(np.asarray(multiplicity, dtype=np.float64), n)),
        "sigma_change": float(np.abs(np.asarray(sigma_after) - np.asarray(sigma_before)).max()),
    }
    if drift is not None:
        rec["drift"] = {"max": float(drift[0]), "refreshes": int(drift[1])}
    return rec


def save_checkpoint(path, cfg, iteration, sigma, fields, counters):
    np.savez(path, config=np.array(json.dumps(cfg)), iteration=np.array(int(iteration)),
             sigma=np.asarray(sigma, dtype=np.complex128), fields=np.asarray(fields, dtype=np.int8),
             counters=np.asarray(counters, dtype=np.uint32))


def load_checkpoint(path):
    """(cfg, iteration, sigma, fields, counters)."""
    z = np.load(path, allow_pickle=False)
    return (json.loads(str(z["config"])), int(z["iteration"]), z["sigma"], z["fields"],
            z["counters"])


def run(cfg, iterations, log=None, checkpoint=None, resume=None, device="cuda:0"):
    """Iterate on the device; returns the list of iteration records."""
    import torch

    start = 0
    state = None
    if resume is not None:
        cfg, start, *state = load_checkpoint(resume)
    p = hf.make_params(cfg)
    _, _, _, _, _, rep_of, _ = hf.hf_lattice_info(p)
    ctx = hf.Context(p, device=device, stream=torch.cuda.Stream(device))
    L, ns, nw, nc = ctx.L, ctx.n_sites, ctx.nw, ctx.n_chains
    mult = np.bincount(rep_of, minlength=ns)
    if state is not None:
        sigma, fields, counters = state
        hf.hf_set_sigma(ctx.handle, sigma)
        hf.hf_set_fields(ctx.handle, fields, counters)
    records = []
    out = open(log, "a") if log else None
    try:
        for it in range(start, start + iterations):
            before = hf.hf_get_sigma(ctx.handle, ns, nw)
            hf.hf_rdmft_step(ctx.handle)
            mean, err = hf.hf_get_observables(ctx.handle, ns, L)
            drift = hf.hf_get_drift(ctx.handle) if cfg.get("check_drift", 0) else None
            rec = iteration_record(it, hf.hf_get_timings(ctx.handle), mean, err, L, before,
                                   hf.hf_get_sigma(ctx.handle, ns, nw), mult, drift)
            records.append(rec)
            if out:
                out.write(json.dumps(rec) + "\n")
                out.flush()
            if checkpoint:
                f, cnt = hf.hf_get_fields(ctx.handle, nc, L)
                save_checkpoint(checkpoint, cfg, it + 1, hf.hf_get_sigma(ctx.handle, ns, nw), f, cnt)
    finally:
        if out:
            out.close()
        ctx.close()
    return records


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    src = ap.add_mutually_exclusive_group(required=True)
    src.add_argument("--workload", help="a named configuration (%s)" % ", ".join(sorted(wl.CONFIGS)))
    src.add_argument("--config", help="a JSON file of configuration keys")
    src.add_argument("--resume", help="a checkpoint written by --checkpoint")
    ap.add_argument("--set", action="append", default=[], metavar="KEY=VALUE",
                    help="override a configuration key (not with --resume)")
    ap.add_argument("--iterations", type=int, default=10)
    ap.add_argument("--log", help="append one JSON line per iteration to this file")
    ap.add_argument("--checkpoint", help="write the run's state here after every iteration")
    ap.add_argument("--device", default="cuda:0")
    a = ap.parse_args(argv)
    if a.resume and a.set:
        ap.error("--set cannot change a resumed run's configuration")
    cfg = None if a.resume else load_config(a.workload, a.config, parse_overrides(a.set))
    recs = run(cfg, a.iterations, log=a.log, checkpoint=a.checkpoint, resume=a.resume,
               device=a.device)
    last = recs[-1] if recs else None
    if last:
        print(json.dumps({"iterations": len(recs), "last_iteration": last["iteration"],
                          "N": last["N"], "sigma_change": last["sigma_change"],
                          "ms": last["ms"]}))
    return 0


if __name__ == "__main__":
    sys.exit(main())
