"""Direct pin of the device random-number generator: the raw Philox4x32-10 blocks that the
sweep kernels draw from equal the published known-answer vectors (Salmon et al., SC'11) and,
block for block, the oracle's independent implementation over many counters and keys."""
import os

import numpy as np
import pytest

import oracle as o

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def hf():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_1006_2716_gb300 import build as B

    B.build()
    from paper_1006_2716_gb300 import hf as H

    return H


def _device_blocks(hf, key, ctr):
    import torch

    ctr = np.ascontiguousarray(ctr, dtype=np.uint32).reshape(-1, 4)
    n = ctr.shape[0]
    d_ctr = torch.from_numpy(ctr.view(np.int32).copy()).cuda()
    d_out = torch.zeros((n, 4), dtype=torch.int32, device="cuda")
    hf.hf_philox_blocks(int(key[0]), int(key[1]), d_ctr.data_ptr(), n, d_out.data_ptr())
    torch.cuda.synchronize()
    return d_out.cpu().numpy().view(np.uint32)


def test_known_answer_vectors(hf):
    for line in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")):
        if line.startswith("#") or not line.strip():
            continue
        w = [int(x, 16) for x in line.split()]
        got = _device_blocks(hf, w[4:6], [w[0:4]])
        assert list(got[0]) == w[6:10]


def test_blocks_equal_the_oracle(hf):
    rng = np.random.default_rng(2024)
    for key in ([0, 0], [1, 0], [0xDEADBEEF, 0x01234567], list(rng.integers(0, 2 ** 32, 2))):
        ctr = rng.integers(0, 2 ** 32, size=(4096, 4), dtype=np.uint64).astype(np.uint32)
        # the counters the sweeps use: (sweep, slice, chain, site), and the field-draw sweep tag
        ctr[:64] = [[w, l, 3, 7] for w in (0, 1, 2, 0xFFFFFFFF) for l in range(16)]
        got = _device_blocks(hf, key, ctr)
        want = np.array([o.philox4x32_10(c, key) for c in ctr], dtype=np.uint32)
        assert np.array_equal(got, want)


def test_rejects_bad_arguments(hf):
    import torch

    buf = torch.zeros(8, dtype=torch.int32, device="cuda")
    with pytest.raises(hf.HFError):
        hf.hf_philox_blocks(0, 0, buf.data_ptr(), -1, buf.data_ptr())
    with pytest.raises(hf.HFError):
        hf.hf_philox_blocks(0, 0, buf.data_ptr() + 4, 1, buf.data_ptr())   # not 16-byte aligned
    hf.hf_philox_blocks(0, 0, 0, 0, 0)                                    # nothing to do
