"""The autotuner's candidate set against the library's own validation (host only, no GPU): a
(form, warps per chain, delay depth) triple is offered for L exactly when hf_workspace_size
accepts it, so the Python shared-memory estimate and the C++ limits agree."""
import pytest

from paper_1006_2716_gb300 import autotune
from paper_1006_2716_gb300 import build as B
from paper_1006_2716_gb300 import hf
from paper_1006_2716_gb300 import workloads as wl


@pytest.fixture(scope="module")
def lib():
    B.build()
    return hf.lib()


@pytest.mark.parametrize("L", [8, 12, 16, 20, 24, 32, 40, 48, 64])
def test_candidates_are_exactly_the_accepted_configurations(lib, L):
    offered = set(autotune.candidates(L))
    for form in (0, 2):
        for tw in (1, 2, 4):
            for k in autotune.DELAYS:
                p = hf.make_params(wl.CONFIGS["square6"], beta=0.25 * L, dtau=0.25,
                                   precision=form, team_warps=tw, delay_k=k)
                try:
                    hf.hf_workspace_size(p)
                    accepted = True
                except hf.HFError as e:
                    assert e.status == hf.HF_EINVAL
                    accepted = False
                assert accepted == ((form, tw, k) in offered), (L, form, tw, k)
    assert (2, 1 if L <= 32 else 2, 1) in offered      # the rank-1 pair form always exists
