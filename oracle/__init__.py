"""Plain, slow CPU oracle for the Hirsch-Fye QMC based real-space DMFT of
arXiv:1006.2716 (Bluemer & Gorelik).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The product path (``paper_1006_2716_gb300``) never imports it, and the
two share no code.

Layout
------
* ``hf_oracle.c``  -- FP64 C core: Philox4x32-10, Trotter/HS constants, bath
  matrix, Dyson refresh, single-flip sweeps with Sherman-Morrison updates,
  measurements, chain runner, brute-force enumeration over 2^L fields.
* ``lattice.py``   -- eq. 1 geometry (square / disc, trap V_i = V0 r_i^2),
  C4v orbits, and the eq. 2 lattice step as a dense matrix inverse.
* ``fourier.py``   -- Matsubara grid, tau <-> i omega_n transforms with the
  high-frequency tail, natural cubic spline.
* ``rdmft.py``     -- one self-consistency iteration in the paper's order.
* ``ed.py``        -- exact diagonalisation of a small Anderson impurity with a
  pole bath: the continuous-time (dtau -> 0) answer the Hirsch-Fye
  discretisation approaches.
"""
from .core import (  # noqa: F401
    lib, build, philox4x32_10, uniform, init_fields, constants, build_g0, dyson,
    ratio, sweep, measure, run_chain, brute_force, tie_watch, tie_count,
)
