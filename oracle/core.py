"""ctypes wrapper of the oracle's C core (``hf_oracle.c``).

TEST INFRASTRUCTURE ONLY (see the package docstring).  Builds ``hf_oracle.c``
with gcc on first use into ``oracle/_build/``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libhforacle.so")
_SRC = os.path.join(_HERE, "hf_oracle.c")
_HDR = os.path.join(_HERE, "hf_oracle.h")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the C core (plain -O2, no fused multiply-add contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < newest:
        tmp = _SO + ".tmp.%d" % os.getpid()
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
               "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            u32p = C.POINTER(C.c_uint32)
            dp = C.POINTER(C.c_double)
            i8p = C.POINTER(C.c_int8)
            L.hfo_philox4x32_10.argtypes = [u32p, u32p, u32p]
            L.hfo_philox4x32_10.restype = None
            L.hfo_uniform.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint32, C.c_uint32]
            L.hfo_uniform.restype = C.c_double
            L.hfo_init_fields.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32, C.c_int, i8p]
            L.hfo_init_fields.restype = None
            L.hfo_constants.argtypes = [C.c_double, C.c_double, C.c_int, dp, dp]
            L.hfo_constants.restype = None
            L.hfo_build_g0.argtypes = [C.c_int, dp, dp]
            L.hfo_build_g0.restype = None
            L.hfo_dyson.argtypes = [C.c_int, dp, i8p, C.c_int, C.c_double, dp, dp]
            L.hfo_dyson.restype = C.c_int
            L.hfo_ratio.argtypes = [C.c_int, C.c_double, i8p, C.c_int, dp, dp, dp, dp]
            L.hfo_ratio.restype = C.c_double
            L.hfo_sweep.argtypes = [C.c_int, C.c_double, C.c_uint64, C.c_uint32, C.c_uint32,
                                    C.c_uint32, i8p, dp, dp]
            L.hfo_sweep.restype = C.c_int
            L.hfo_measure.argtypes = [C.c_int, dp, dp, dp]
            L.hfo_measure.restype = None
            L.hfo_run_chain.argtypes = [C.c_int, C.c_double, dp, dp, C.c_uint64, C.c_uint32,
                                        C.c_uint32, u32p, C.c_int, C.c_int, C.c_int, C.c_int,
                                        C.c_int, i8p, dp, dp, dp]
            L.hfo_run_chain.restype = C.c_long
            L.hfo_tie_watch.argtypes = [C.c_double]
            L.hfo_tie_watch.restype = None
            L.hfo_tie_count.argtypes = []
            L.hfo_tie_count.restype = C.c_long
            L.hfo_brute_force.argtypes = [C.c_int, C.c_double, dp, dp, dp]
            L.hfo_brute_force.restype = C.c_int
            _lib = L
    return _lib


def _p(a, ct):
    return a.ctypes.data_as(C.POINTER(ct))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def philox4x32_10(ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().hfo_philox4x32_10(_p(c, C.c_uint32), _p(k, C.c_uint32), _p(out, C.c_uint32))
    return out


def uniform(seed, site, chain, sweep, l):
    return lib().hfo_uniform(seed, site, chain, sweep, l)


def init_fields(seed, site, chain, L):
    s = np.zeros(L, dtype=np.int8)
    lib().hfo_init_fields(seed, site, chain, L, _p(s, C.c_int8))
    return s


def constants(beta, U, L):
    dt = C.c_double()
    lam = C.c_double()
    lib().hfo_constants(beta, U, L, C.byref(dt), C.byref(lam))
    return dt.value, lam.value


def build_g0(gt):
    gt = _f64(gt)
    L = gt.shape[0]
    g0 = np.zeros((L, L))
    lib().hfo_build_g0(L, _p(gt, C.c_double), _p(g0, C.c_double))
    return g0


def dyson(g0, s, sigma, lam):
    g0 = _f64(g0)
    s = np.ascontiguousarray(s, dtype=np.int8)
    L = g0.shape[0]
    G = np.zeros((L, L))
    det = C.c_double()
    rc = lib().hfo_dyson(L, _p(g0, C.c_double), _p(s, C.c_int8), int(sigma), lam,
                         _p(G, C.c_double), C.byref(det))
    if rc != 0:
        raise FloatingPointError("singular Dyson matrix")
    return G, det.value


def ratio(lam, s, l, Gup, Gdn):
    """(p, a[2], R[2]) of the proposal s_l -> -s_l."""
    s = np.ascontiguousarray(s, dtype=np.int8)
    L = s.shape[0]
    a = np.zeros(2)
    R = np.zeros(2)
    p = lib().hfo_ratio(L, lam, _p(s, C.c_int8), int(l), _p(_f64(Gup), C.c_double),
                        _p(_f64(Gdn), C.c_double), _p(a, C.c_double), _p(R, C.c_double))
    return p, a, R


def sweep(lam, seed, site, chain, sweep_id, s, Gup, Gdn):
    """In place on s (int8), Gup, Gdn (C-contiguous float64).  Returns accepts."""
    L = s.shape[0]
    return lib().hfo_sweep(L, lam, seed, site, chain, sweep_id, _p(s, C.c_int8),
                           _p(Gup, C.c_double), _p(Gdn, C.c_double))


def measure(Gup, Gdn):
    L = Gup.shape[0]
    acc = np.zeros(2 * L + 3)
    lib().hfo_measure(L, _p(_f64(Gup), C.c_double), _p(_f64(Gdn), C.c_double),
                      _p(acc, C.c_double))
    return acc


def run_chain(lam, g0up, g0dn, seed, site, chain, nsw, n_warmup, n_measure,
              refresh_every, bin_size, s, Gup, Gdn, bins, refresh_stagger=0):
    """In place on s, Gup, Gdn, bins ([nbins, 2L+3]).  Returns (accepts, new nsw).
    refresh_stagger=1 offsets the chain's refresh sweeps by (site + chain) % refresh_every."""
    L = s.shape[0]
    g0up = _f64(g0up)
    g0dn = _f64(g0dn)
    n = C.c_uint32(nsw)
    acc = lib().hfo_run_chain(L, lam, _p(g0up, C.c_double), _p(g0dn, C.c_double), seed,
                              site, chain, C.byref(n), n_warmup, n_measure, refresh_every,
                              int(refresh_stagger), bin_size, _p(s, C.c_int8), _p(Gup, C.c_double),
                              _p(Gdn, C.c_double), _p(bins, C.c_double))
    if acc < 0:
        raise FloatingPointError("singular Dyson refresh")
    return int(acc), int(n.value)


def tie_watch(rel):
    """Count, from now on, the sweep proposals with |u - R_up R_dn| < rel |R_up R_dn| (0: off)."""
    lib().hfo_tie_watch(float(rel))


def tie_count():
    return int(lib().hfo_tie_count())


def brute_force(lam, g0up, g0dn):
    g0up = _f64(g0up)
    g0dn = _f64(g0dn)
    L = g0up.shape[0]
    out = np.zeros(2 * L + 3)
    rc = lib().hfo_brute_force(L, lam, _p(g0up, C.c_double), _p(g0dn, C.c_double),
                               _p(out, C.c_double))
    if rc != 0:
        raise FloatingPointError("brute force failed")
    return out
