"""Host side of the library's lattices (no GPU): the orbit tables that hf_lattice_info reports
equal the oracle's, bit for bit, for every geometry, and the band half-width of the folded band
order is the one its construction gives."""
import numpy as np
import pytest

from oracle.lattice import Lattice
from paper_1006_2716_gb300 import build as B
from paper_1006_2716_gb300 import hf
from paper_1006_2716_gb300 import workloads as wl


@pytest.fixture(scope="module")
def lib():
    B.build()
    return hf.lib()


CASES = [
    # geometry, Lx, Ly, Lz, periodic, band half-width of the folded order
    (0, 1, 1, 1, 0, 0),             # a single site: N = 1, no band
    (1, 0, 0, 1, 0, 0),             # the disc of radius 0
    (3, 1, 1, 4, 0, 2),             # a column of 4 layers: one orbit, folded ring
    (0, 6, 6, 1, 0, 6),
    (0, 7, 5, 1, 1, 14),
    (0, 20, 20, 1, 1, 40),
    (1, 7, 7, 1, 0, None),
    (1, 40, 40, 1, 0, 80),          # serving disc, 663 orbits: (40 - x) + (x + 39) + 1
    (2, 4, 4, 4, 1, 32),
    (2, 5, 5, 5, 0, 25),
    (2, 4, 4, 6, 0, 16),
    (2, 6, 6, 6, 1, 72),
    (3, 6, 6, 4, 0, 24),
    (3, 8, 6, 4, 1, 64),
    (3, 24, 24, 4, 0, 96),
    (2, 12, 12, 12, 0, 144),
    (3, 20, 20, 4, 1, 160),
]


@pytest.mark.parametrize("geom,Lx,Ly,Lz,per,band", CASES)
def test_orbit_tables_match_the_oracle(lib, geom, Lx, Ly, Lz, per, band):
    p = hf.make_params(wl.CONFIGS["square6"], geometry=geom, Lx=Lx, Ly=Ly, Lz=Lz, periodic=per,
                       n_matsubara=4, chains_per_site=1)
    N, ns, b, nsp, rep, rep_of, flip = hf.hf_lattice_info(p)
    lat = Lattice(Lx, Ly, geometry=geom, periodic=bool(per), V0=0.1, Lz=Lz)
    r2, ro2, f2 = lat.orbits()
    assert N == lat.N and ns == len(r2)
    assert np.array_equal(rep, r2) and np.array_equal(rep_of, ro2) and np.array_equal(flip, f2)
    if band is not None:
        assert b == band
    # one matrix per frequency exactly when some operation exchanges the sublattices
    has_flip = any(np.all(lat.parity[im] != lat.parity) for im in lat._images)
    assert nsp == (1 if has_flip else 2)


@pytest.mark.parametrize("over,frag", [
    (dict(geometry=2, Lx=5, Ly=5, Lz=5, periodic=1), "even length"),
    (dict(geometry=3, Lx=6, Ly=6, Lz=3), "even length"),
    (dict(geometry=3, Lx=6, Ly=6, Lz=2), "even length"),
    (dict(geometry=2, Lx=4, Ly=4, Lz=0), ">= 1"),
    (dict(geometry=3, Lx=212, Ly=2, Lz=4), "band half-width"),     # b = 848 > 840
])
def test_invalid_three_dimensional_lattices(lib, over, frag):
    p = hf.make_params(wl.CONFIGS["square6"], **over)
    with pytest.raises(hf.HFError) as e:
        hf.hf_lattice_info(p)
    assert e.value.status == hf.HF_EINVAL
    assert frag in str(e.value)


def test_bench_lattice_bookkeeping(lib):
    """bench.py's launch count and algorithmic flop count of the lattice step: one launch per
    iteration while the band buffers of all matrices fit in 1 GiB; for a dense band (b >= N - 1)
    the count is the textbook one, N^3/6 multiply-adds for LDL^T plus N^3/3 for the selected
    inversion to leading order (exactly sum_d [d(d+1)/2 + d^2 + d], d = 0..N-1)."""
    import bench

    assert bench.lattice_launches(hf, wl.CONFIGS["square20"]) == 1
    assert bench.lattice_launches(hf, wl.CONFIGS["slab16"]) == 1
    # 12^3 box (b = 144): the blocked form by default, 500 matrices of 1728 x 145 x 16 bytes =
    # 2.0 GB in one launch; in the window form (lattice_form 2) two launches under 1 GiB
    assert bench.lattice_launches(hf, wl.CONFIGS["box12"]) == 1
    assert bench.lattice_launches(hf, dict(wl.CONFIGS["box12"], lattice_form=2)) == 2
    # periodic 16^3 box (blocked band form): 500 matrices of 4096 x 513 x 16 bytes = 16.8 GB,
    # under the 24 GiB cap: one launch of the persistent kernel
    assert bench.lattice_launches(hf, wl.CONFIGS["box16p"]) == 1
    assert bench.lattice_launches(hf, dict(wl.CONFIGS["slab16"], lattice_form=1)) == 1
    # above the cap, split evenly: 1000 matrices of the 16^3 box (33.6 GB) -> two launches of 500
    assert bench.lattice_launches(hf, dict(wl.CONFIGS["box16p"], n_matsubara=1000)) == 2
    N = 40
    exact = 8.0 * sum(d * (d + 1) // 2 + d * d + d for d in range(N))
    assert bench.lattice_flops(N, N - 1, 1, 1) == exact
    assert bench.lattice_flops(N, 100, 2, 3) == 6 * exact
    assert abs(bench.lattice_flops(400, 399, 1, 1) / (8 * 400 ** 3 / 2) - 1) < 0.01


def test_band_limits(lib):
    """The shared-memory window form takes b <= 165 (an 11x15x3 open box has b = Lx Ly = 165);
    wider bands go to the blocked band form, up to b = 840 (a 28x30x2 box; 29x29x2 has 841 and
    is rejected).  The periodic boxes of Fig. 4 have b = 2 n^2 in the folded band order."""
    sq = wl.CONFIGS["square6"]
    assert hf.hf_lattice_info(hf.make_params(sq, geometry=2, Lx=11, Ly=15, Lz=3, periodic=0))[2] == 165
    assert hf.hf_lattice_info(hf.make_params(sq, geometry=2, Lx=2, Ly=83, Lz=2, periodic=0))[2] == 166
    assert hf.hf_lattice_info(hf.make_params(sq, geometry=2, Lx=28, Ly=30, Lz=2, periodic=0))[2] == 840
    for name, n, b, ns in (("box14p", 14, 392, 84), ("box16p", 16, 512, 120)):
        N, nsite, band, nspin, _, _, _ = hf.hf_lattice_info(hf.make_params(wl.CONFIGS[name]))
        assert (N, band, nsite, nspin) == (n ** 3, b, ns, 1)
    p = hf.make_params(sq, geometry=2, Lx=29, Ly=29, Lz=2, periodic=0)
    with pytest.raises(hf.HFError) as e:
        hf.hf_lattice_info(p)
    assert e.value.status == hf.HF_EINVAL and "largest: 840" in str(e.value)
    with pytest.raises(hf.HFError) as e:
        hf.hf_lattice_info(hf.make_params(sq, lattice_form=3))
    assert e.value.status == hf.HF_EINVAL
    # the window form asked for where it does not fit
    with pytest.raises(hf.HFError) as e:
        hf.hf_lattice_info(hf.make_params(sq, geometry=2, Lx=2, Ly=83, Lz=2, periodic=0, lattice_form=2))
    assert e.value.status == hf.HF_EINVAL and "window form" in str(e.value)
    hf.hf_lattice_info(hf.make_params(sq, geometry=2, Lx=11, Ly=15, Lz=3, periodic=0, lattice_form=2))
