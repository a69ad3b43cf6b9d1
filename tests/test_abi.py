"""The C-ABI library loads, exports every symbol declared in include/*.h, and its host-side
validation and sizing work without a GPU (no compute call is made here)."""
import ctypes as C
import glob
import os
import re

import pytest

from paper_1006_2716_gb300 import build as B
from paper_1006_2716_gb300 import hf
from paper_1006_2716_gb300 import workloads as wl

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return hf.lib()


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        txt = open(h).read()
        txt = re.sub(r"/\*.*?\*/", " ", txt, flags=re.S)
        for m in re.finditer(r"\b(hf_[a-z0-9_]+)\s*\(", txt):
            names.add(m.group(1))
    return sorted(names)


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert "hf_init" in names and "hf_rdmft_step" in names and "hf_sweep" in names
    raw = C.CDLL(hf.LIB_PATH)
    for n in names:
        assert hasattr(raw, n), n


def test_binding_covers_every_symbol():
    bound = {n for n, _, _ in hf.SIGNATURES}
    assert set(_declared()) <= bound


def test_workspace_size_and_orbit_counts(lib):
    p = hf.make_params(wl.CONFIGS["square20"])
    n = hf.hf_workspace_size(p)
    # G (1760 chains x 2 x 32 x 32 doubles) dominates the QMC state
    assert n > 1760 * 2 * 32 * 32 * 8
    p6 = hf.make_params(wl.CONFIGS["square6"])
    assert hf.hf_workspace_size(p6) < n


@pytest.mark.parametrize("over,frag", [
    (dict(beta=4.0, dtau=0.3), "integer"),
    (dict(beta=4.0, dtau=4.0 / 17), "L in"),
    (dict(chains_per_site=0), "chains_per_site"),
    (dict(mix=0.0), "mix"),
    (dict(U=-1.0), "U must"),
    (dict(geometry=5), "geometry"),
    (dict(precision=1, beta=4.0, dtau=0.25, refresh_every=0), "refresh"),
    (dict(precision=1, beta=4.0, dtau=0.25, refresh_every=5, refresh_stagger=1), "stagger"),
    (dict(refresh_stagger=2), "stagger"),
    (dict(check_drift=2), "check_drift"),
    (dict(team_warps=3), "team_warps"),
    (dict(beta=16.0, dtau=0.25, team_warps=1), "team_warps"),
    (dict(precision=3), "precision"),
    (dict(delay_k=4), "delay_k"),
    (dict(precision=2, delay_k=5), "delay_k"),
    (dict(precision=2, beta=8.0, dtau=0.25, team_warps=2, delay_k=4), "one warp per chain"),
    (dict(precision=2, beta=16.0, dtau=0.25, delay_k=8), "one warp per chain"),
])
def test_invalid_params_rejected(lib, over, frag):
    p = hf.make_params(wl.CONFIGS["square6"], **over)
    with pytest.raises(hf.HFError) as e:
        hf.hf_workspace_size(p)
    assert e.value.status == hf.HF_EINVAL
    assert frag in str(e.value)


def test_init_rejects_small_workspace_without_touching_gpu(lib):
    p = hf.make_params(wl.CONFIGS["square6"])
    with pytest.raises(hf.HFError) as e:
        hf.hf_init(p, 256, 1024)
    assert e.value.status == hf.HF_ENOMEM


def _c_struct_fields(name):
    """Field names, in order, of `typedef struct name {...} name;` in include/hf.h."""
    txt = open(os.path.join(ROOT, "include", "hf.h")).read()
    body = txt[txt.index("typedef struct %s {" % name):txt.index("} %s;" % name)]
    body = re.sub(r"/\*.*?\*/", " ", body, flags=re.S)
    names = []
    for line in body.splitlines()[1:]:
        line = line.strip().rstrip(";")
        parts = line.split(None, 1)
        if len(parts) < 2:
            continue
        for n in parts[1].split(","):
            names.append(re.sub(r"\[.*", "", n.strip().lstrip("*")))
    return names


@pytest.mark.parametrize("cname,pyname", [("hf_params", "hf_params"), ("hf_srv_params", "hf_srv_params"),
                                          ("hf_request", "hf_request"), ("hf_result", "hf_result"),
                                          ("hf_srv_stats_t", "hf_srv_stats_t")])
def test_binding_structs_mirror_the_header(cname, pyname):
    """The ctypes mirrors list the C structs' fields in the same order (a mismatch would shift
    every later field silently)."""
    py = [f[0] for f in getattr(hf, pyname)._fields_]
    assert _c_struct_fields(cname) == py


def _srv_params(**over):
    p = hf.hf_srv_params()
    d = dict(chains_per_request=8, n_warmup=10, n_measure=40, refresh_every=10, bin_size=10,
             precision=2, team_warps=0, max_L=64, max_inflight=64, max_keys=256, n_streams=4,
             requests_per_launch=16)
    d.update(over)
    for k, v in d.items():
        setattr(p, k, v)
    return p


def test_server_pool_size_grows_with_its_limits(lib):
    n = hf.hf_srv_workspace_size(_srv_params())
    assert n > 0
    assert hf.hf_srv_workspace_size(_srv_params(max_inflight=128)) > n
    assert hf.hf_srv_workspace_size(_srv_params(max_keys=512)) > n
    assert hf.hf_srv_workspace_size(_srv_params(max_L=32)) < n


@pytest.mark.parametrize("over,frag", [
    (dict(chains_per_request=0), "chains_per_request"),
    (dict(n_measure=0), "n_measure"),
    (dict(n_measure=45), "multiple of bin_size"),
    (dict(refresh_every=-1), "refresh_every"),
    (dict(refresh_stagger=3), "refresh_stagger"),
    (dict(precision=1), "precision"),
    (dict(max_L=128), "max_L"),
    (dict(n_streams=0), "n_streams"),
    (dict(max_inflight=0), "max_inflight"),
    (dict(team_warps=3), "team_warps"),
])
def test_server_rejects_invalid_params(lib, over, frag):
    with pytest.raises(hf.HFError) as e:
        hf.hf_srv_workspace_size(_srv_params(**over))
    assert e.value.status == hf.HF_EINVAL and frag in str(e.value)
