"""The command-line RDMFT driver on the GPU: a run checkpointed after two iterations and resumed
for a third ends in exactly the state (self-energy, Ising fields, sweep counters) and reports
exactly the observables of the same run done in one go."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_1006_2716_gb300 import run

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def built():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_1006_2716_gb300 import build as B

    B.build()


def _run(args, cwd):
    r = subprocess.run([sys.executable, "-m", "paper_1006_2716_gb300.run", *args], cwd=ROOT,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    return r.stdout


def test_checkpoint_resume_continues_bitwise(built, tmp_path):
    common = ["--set", "n_warmup=20", "--set", "n_measure=40", "--set", "bin_size=10",
              "--set", "chains_per_site=4"]
    a_log, a_ck = str(tmp_path / "a.jsonl"), str(tmp_path / "a.npz")
    _run(["--workload", "square6", *common, "--iterations", "3", "--log", a_log,
          "--checkpoint", a_ck], tmp_path)
    b_ck = str(tmp_path / "b.npz")
    _run(["--workload", "square6", *common, "--iterations", "2", "--checkpoint", b_ck], tmp_path)
    c_log, c_ck = str(tmp_path / "c.jsonl"), str(tmp_path / "c.npz")
    out = _run(["--resume", b_ck, "--iterations", "1", "--log", c_log, "--checkpoint", c_ck],
               tmp_path)
    assert json.loads(out.strip().splitlines()[-1])["last_iteration"] == 2
    ca, ia, sa, fa, na = run.load_checkpoint(a_ck)
    cc, ic, sc, fc, nc = run.load_checkpoint(c_ck)
    assert ca == cc and ia == ic == 3
    assert np.array_equal(sa, sc) and np.array_equal(fa, fc) and np.array_equal(na, nc)
    ra = [json.loads(x) for x in open(a_log)]
    rc = [json.loads(x) for x in open(c_log)]
    assert [r["iteration"] for r in ra] == [0, 1, 2] and [r["iteration"] for r in rc] == [2]
    for k in ("n", "n_err", "d", "d_err", "m", "m_err", "N", "sigma_change"):
        assert ra[2][k] == rc[0][k], k
