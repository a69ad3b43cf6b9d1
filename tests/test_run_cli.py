"""The command-line RDMFT driver's host side (no GPU): configuration loading and overrides,
the per-iteration record, and the checkpoint file round trip."""
import json

import numpy as np
import pytest

from paper_1006_2716_gb300 import run
from paper_1006_2716_gb300 import workloads as wl


def test_overrides_and_config(tmp_path):
    assert run.parse_overrides(["U=10", "Lx=16", "periodic=1"]) == {"U": 10.0, "Lx": 16, "periodic": 1}
    with pytest.raises(ValueError):
        run.parse_overrides(["Ux=1"])
    with pytest.raises(ValueError):
        run.parse_overrides(["U"])
    cfg = run.load_config("square20", overrides={"U": 10.0})
    assert cfg["U"] == 10.0 and cfg["Lx"] == 20 and wl.CONFIGS["square20"]["U"] == 8.0
    p = tmp_path / "c.json"
    p.write_text(json.dumps(dict(wl.CONFIGS["slab16"])))
    assert run.load_config(path=str(p)) == wl.CONFIGS["slab16"]
    p.write_text(json.dumps({"Lx": 4, "bogus": 1}))
    with pytest.raises(ValueError):
        run.load_config(path=str(p))
    with pytest.raises(ValueError):
        run.load_config("nope")
    with pytest.raises(ValueError):
        run.load_config()


def test_iteration_record():
    L, ns = 4, 3
    mean = np.zeros((ns, 2 * L + 4))
    err = np.zeros((ns, 2 * L + 4))
    mean[:, 2 * L] = [0.5, 0.4, 0.1]
    mean[:, 2 * L + 1] = [0.5, 0.2, 0.1]
    mean[:, 2 * L + 2] = [0.05, 0.02, 0.0]
    mean[:, 2 * L + 3] = [0.0, 0.2, 0.0]
    err[:, 2 * L] = 0.03
    err[:, 2 * L + 1] = 0.04
    s0 = np.zeros((ns, 2, 5), dtype=complex)
    s1 = s0.copy()
    s1[1, 0, 2] = 0.25 - 0.1j
    rec = run.iteration_record(7, [1.0, 2.0, 3.0, 4.0, 5.0, -1.0], mean, err, L, s0, s1,
                               [4, 8, 4], drift=(1.5e-9, 30))
    assert rec["iteration"] == 7 and rec["ms"]["qmc"] == 3.0 and rec["ms"]["sigma"] == 5.0
    assert np.allclose(rec["n"], [1.0, 0.6, 0.2]) and np.allclose(rec["n_err"], 0.05)
    assert np.isclose(rec["N"], 4 * 1.0 + 8 * 0.6 + 4 * 0.2)
    assert np.isclose(rec["sigma_change"], abs(0.25 - 0.1j))
    assert rec["m"] == [0.0, pytest.approx(0.2), 0.0] and rec["drift"] == {"max": 1.5e-9, "refreshes": 30}
    json.dumps(rec)


def test_checkpoint_round_trip(tmp_path):
    cfg = dict(wl.CONFIGS["square6"], U=5.0)
    rng = np.random.default_rng(0)
    sigma = rng.normal(size=(6, 2, 10)) + 1j * rng.normal(size=(6, 2, 10))
    fields = rng.choice(np.array([-1, 1], dtype=np.int8), size=(6, 16))
    counters = np.arange(6, dtype=np.uint32) * 2500
    path = str(tmp_path / "ck.npz")
    run.save_checkpoint(path, cfg, 12, sigma, fields, counters)
    c2, it, s2, f2, n2 = run.load_checkpoint(path)
    assert c2 == cfg and it == 12
    assert np.array_equal(s2, sigma) and np.array_equal(f2, fields) and np.array_equal(n2, counters)
    assert f2.dtype == np.int8 and n2.dtype == np.uint32


def test_cli_rejects_overrides_on_resume(tmp_path):
    with pytest.raises(SystemExit):
        run.main(["--resume", str(tmp_path / "x.npz"), "--set", "U=1"])
