"""Thin Python binding of the C ABI in ``include/hf.h`` (argument marshalling only).

Every step of the method runs in the CUDA library ``_build/libhfqmc.so``; this module only
converts arguments.  PyTorch supplies the device workspace and the CUDA stream.  If the library
is missing the import of a function fails loudly: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, os.environ.get("HF_BUILD_DIR", "_build"), "libhfqmc.so")

HF_OK, HF_EINVAL, HF_ENOMEM, HF_ECUDA, HF_ETIMEOUT, HF_ENUMERIC, HF_EBUSY, HF_ENOTREADY = (
    0, -1, -2, -3, -4, -5, -6, -7)


class HFError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("hf status %d: %s" % (status, msg))
        self.status = status


class hf_params(C.Structure):
    _fields_ = [
        ("Lx", C.c_int), ("Ly", C.c_int), ("Lz", C.c_int), ("geometry", C.c_int), ("periodic", C.c_int),
        ("t", C.c_double), ("U", C.c_double), ("V0", C.c_double), ("mu", C.c_double),
        ("beta", C.c_double), ("dtau", C.c_double),
        ("n_matsubara", C.c_int), ("chains_per_site", C.c_int), ("precision", C.c_int),
        ("refresh_every", C.c_int), ("refresh_stagger", C.c_int), ("check_drift", C.c_int),
        ("refresh_gj", C.c_int), ("lattice_form", C.c_int),
        ("delay_k", C.c_int),
        ("team_warps", C.c_int),
        ("bin_size", C.c_int),
        ("max_bins", C.c_int), ("n_warmup", C.c_int), ("n_measure", C.c_int),
        ("seed", C.c_uint64), ("h_seed", C.c_double), ("mix", C.c_double),
        ("cuda_stream", C.c_void_p),
    ]


class hf_srv_params(C.Structure):
    _fields_ = [
        ("chains_per_request", C.c_int), ("n_warmup", C.c_int), ("n_measure", C.c_int),
        ("refresh_every", C.c_int), ("refresh_stagger", C.c_int), ("bin_size", C.c_int),
        ("precision", C.c_int),
        ("team_warps", C.c_int), ("max_L", C.c_int), ("max_inflight", C.c_int),
        ("max_keys", C.c_int), ("n_streams", C.c_int), ("requests_per_launch", C.c_int),
    ]


class hf_request(C.Structure):
    _fields_ = [
        ("run", C.c_int), ("site", C.c_int), ("L", C.c_int), ("beta", C.c_double),
        ("U", C.c_double), ("seed", C.c_uint64), ("g0_tau", (C.c_double * 64) * 2),
    ]


class hf_result(C.Structure):
    _fields_ = [
        ("ticket", C.c_uint64), ("status", C.c_int), ("L", C.c_int), ("warm", C.c_int),
        ("sweeps_done", C.c_uint32), ("gtau", (C.c_double * 64) * 2), ("n", C.c_double * 2),
        ("d", C.c_double), ("m", C.c_double), ("err", C.c_double * 132),
        ("latency_s", C.c_double),
    ]


class hf_srv_stats_t(C.Structure):
    _fields_ = [
        ("queued", C.c_int), ("inflight", C.c_int), ("peak_inflight", C.c_int),
        ("warm_keys", C.c_int), ("completed", C.c_uint64), ("bytes_in_use", C.c_size_t),
        ("peak_bytes", C.c_size_t), ("arena_bytes", C.c_size_t),
    ]


_lib = None

# (name, restype, argtypes) of every entry point declared in include/hf.h
_VP, _DP, _IP = C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_int)
SIGNATURES = [
    ("hf_workspace_size", C.c_int, [C.POINTER(hf_params), C.POINTER(C.c_size_t)]),
    ("hf_lattice_info", C.c_int, [C.POINTER(hf_params), _IP, _IP, _IP, _IP, _IP, _IP, _IP]),
    ("hf_init", C.c_int, [C.POINTER(hf_params), _VP, C.c_size_t, C.POINTER(_VP)]),
    ("hf_get_sizes", C.c_int, [_VP, _IP, _IP, _IP, _IP]),
    ("hf_get_orbits", C.c_int, [_VP, _IP, _IP, _IP]),
    ("hf_set_g0", C.c_int, [_VP, C.c_int, C.c_int, _DP]),
    ("hf_sweep", C.c_int, [_VP, C.c_int, C.c_int, C.c_int]),
    ("hf_clear_measurements", C.c_int, [_VP]),
    ("hf_measure", C.c_int, [_VP, C.c_int, _DP, _DP, _DP, _DP, _DP]),
    ("hf_rdmft_step", C.c_int, [_VP, _DP]),
    ("hf_compute_baths", C.c_int, [_VP]),
    ("hf_get_sigma", C.c_int, [_VP, _DP]),
    ("hf_set_sigma", C.c_int, [_VP, _DP]),
    ("hf_get_observables", C.c_int, [_VP, _DP, _DP]),
    ("hf_get_gloc", C.c_int, [_VP, _DP]),
    ("hf_get_g0", C.c_int, [_VP, _DP]),
    ("hf_get_fields", C.c_int, [_VP, C.POINTER(C.c_int8), C.POINTER(C.c_uint32)]),
    ("hf_set_fields", C.c_int, [_VP, C.POINTER(C.c_int8), C.POINTER(C.c_uint32)]),
    ("hf_get_green", C.c_int, [_VP, C.c_int, _DP]),
    ("hf_get_accepts", C.c_int, [_VP, C.POINTER(C.c_ulonglong)]),
    ("hf_get_timings", C.c_int, [_VP, _DP]),
    ("hf_sync", C.c_int, [_VP]),
    ("hf_get_drift", C.c_int, [_VP, _DP, C.POINTER(C.c_ulonglong)]),
    ("hf_get_refresh_stats", C.c_int, [_VP, C.POINTER(C.c_ulonglong), C.POINTER(C.c_ulonglong),
                                        C.POINTER(C.c_ulonglong)]),
    ("hf_lattice_step_noalloc", C.c_int, [_VP, _VP, _VP]),
    ("hf_get_lattice_plan", C.c_int, [_VP, C.POINTER(C.c_int), C.POINTER(C.c_int), _DP, _DP]),
    ("hf_get_impurity_iw", C.c_int, [_VP, _DP, _DP, _DP, _DP]),
    ("hf_philox_blocks", C.c_int, [C.c_uint32, C.c_uint32, _VP, C.c_int, _VP, _VP]),
    ("hf_tc_dgemm128", C.c_int, [_VP, _VP, _VP, C.c_int, C.c_int, _VP, _VP]),
    ("hf_batch_create", C.c_int, [C.POINTER(_VP), C.c_int, C.c_int, C.POINTER(_VP)]),
    ("hf_batch_sweep", C.c_int, [_VP, C.c_int, C.c_int, C.c_int]),
    ("hf_batch_rdmft_step", C.c_int, [_VP, _DP]),
    ("hf_batch_elapsed", C.c_int, [_VP, _DP]),
    ("hf_batch_free", None, [_VP]),
    ("hf_batch_last_error", C.c_char_p, [_VP]),
    ("hf_srv_workspace_size", C.c_int, [C.POINTER(hf_srv_params), C.POINTER(C.c_size_t)]),
    ("hf_srv_create", C.c_int, [C.POINTER(hf_srv_params), _VP, C.c_size_t, C.POINTER(_VP)]),
    ("hf_srv_submit", C.c_int, [_VP, C.POINTER(hf_request), C.POINTER(C.c_uint64)]),
    ("hf_srv_poll", C.c_int, [_VP, C.c_uint64, C.POINTER(hf_result)]),
    ("hf_srv_wait", C.c_int, [_VP, C.c_uint64, C.c_double, C.POINTER(hf_result)]),
    ("hf_srv_stats", C.c_int, [_VP, C.POINTER(hf_srv_stats_t)]),
    ("hf_srv_free", None, [_VP]),
    ("hf_srv_last_error", C.c_char_p, [_VP]),
    ("hf_free", None, [_VP]),
    ("hf_last_error", C.c_char_p, [_VP]),
]


def lib():
    """The loaded CUDA library; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("CUDA library %s is missing: run __graft_entry__.build()" % LIB_PATH)
        L = C.CDLL(LIB_PATH)
        for name, res, args in SIGNATURES:
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(_DP)


def _check(st, ctx=None):
    if st != HF_OK:
        msg = lib().hf_last_error(ctx)
        raise HFError(st, msg.decode() if msg else "")


# --- one wrapper per entry point, same names as the C ABI -----------------------------------

def hf_lattice_info(p: hf_params):
    """Host-only lattice description: (N, n_sites, band, spins, rep, rep_of, flip)."""
    N, ns, b, nsp = C.c_int(), C.c_int(), C.c_int(), C.c_int()
    _check(lib().hf_lattice_info(C.byref(p), C.byref(N), C.byref(ns), C.byref(b), C.byref(nsp),
                                 None, None, None))
    rep = np.zeros(ns.value, dtype=np.int32)
    rep_of = np.zeros(N.value, dtype=np.int32)
    flip = np.zeros(N.value, dtype=np.int32)
    _check(lib().hf_lattice_info(C.byref(p), None, None, None, None, rep.ctypes.data_as(_IP),
                                 rep_of.ctypes.data_as(_IP), flip.ctypes.data_as(_IP)))
    return N.value, ns.value, b.value, nsp.value, rep, rep_of, flip


def hf_workspace_size(p: hf_params) -> int:
    n = C.c_size_t()
    _check(lib().hf_workspace_size(C.byref(p), C.byref(n)))
    return n.value


def hf_init(p: hf_params, d_ws: int, ws_bytes: int):
    h = C.c_void_p()
    _check(lib().hf_init(C.byref(p), C.c_void_p(d_ws), ws_bytes, C.byref(h)))
    return h


def hf_get_sizes(ctx):
    a, b, c, d = C.c_int(), C.c_int(), C.c_int(), C.c_int()
    _check(lib().hf_get_sizes(ctx, C.byref(a), C.byref(b), C.byref(c), C.byref(d)), ctx)
    return a.value, b.value, c.value, d.value


def hf_get_orbits(ctx, n_sites, N):
    rep = np.zeros(n_sites, dtype=np.int32)
    rep_of = np.zeros(N, dtype=np.int32)
    flip = np.zeros(N, dtype=np.int32)
    _check(lib().hf_get_orbits(ctx, rep.ctypes.data_as(_IP), rep_of.ctypes.data_as(_IP),
                               flip.ctypes.data_as(_IP)), ctx)
    return rep, rep_of, flip


def hf_set_g0(ctx, site, spin, g0_tau):
    g = np.ascontiguousarray(g0_tau, dtype=np.float64)
    _check(lib().hf_set_g0(ctx, int(site), int(spin), _dp(g)), ctx)


def hf_sweep(ctx, n_warmup, n_measure, refresh_first):
    _check(lib().hf_sweep(ctx, int(n_warmup), int(n_measure), int(refresh_first)), ctx)


def hf_clear_measurements(ctx):
    _check(lib().hf_clear_measurements(ctx), ctx)


def hf_measure(ctx, site, L):
    gtau = np.zeros(2 * L)
    n = np.zeros(2)
    d = C.c_double()
    m = C.c_double()
    errs = np.zeros(2 * L + 4)
    _check(lib().hf_measure(ctx, int(site), _dp(gtau), _dp(n), C.byref(d), C.byref(m),
                            _dp(errs)), ctx)
    return gtau, n, d.value, m.value, errs


def hf_rdmft_step(ctx):
    t = C.c_double()
    _check(lib().hf_rdmft_step(ctx, C.byref(t)), ctx)
    return t.value


def hf_compute_baths(ctx):
    _check(lib().hf_compute_baths(ctx), ctx)


def hf_get_sigma(ctx, n_sites, nw):
    out = np.zeros((n_sites, 2, nw), dtype=np.complex128)
    _check(lib().hf_get_sigma(ctx, out.ctypes.data_as(_DP)), ctx)
    return out


def hf_set_sigma(ctx, sigma):
    s = np.ascontiguousarray(sigma, dtype=np.complex128)
    _check(lib().hf_set_sigma(ctx, s.ctypes.data_as(_DP)), ctx)


def hf_get_observables(ctx, n_sites, L):
    mean = np.zeros((n_sites, 2 * L + 4))
    err = np.zeros((n_sites, 2 * L + 4))
    _check(lib().hf_get_observables(ctx, _dp(mean), _dp(err)), ctx)
    return mean, err


def hf_get_gloc(ctx, n_sites, nw):
    out = np.zeros((n_sites, 2, nw), dtype=np.complex128)
    _check(lib().hf_get_gloc(ctx, out.ctypes.data_as(_DP)), ctx)
    return out


def hf_get_impurity_iw(ctx, n_sites, nw):
    """(G~0(i w_n), 1/G0, G_imp(i w_n), unmixed Sigma) of the last RDMFT iteration, each
    [n_sites][2][nw] complex."""
    out = [np.zeros((n_sites, 2, nw), dtype=np.complex128) for _ in range(4)]
    _check(lib().hf_get_impurity_iw(ctx, *[o.ctypes.data_as(_DP) for o in out]), ctx)
    return tuple(out)


def hf_get_g0(ctx, n_sites, L):
    out = np.zeros((n_sites, 2, L))
    _check(lib().hf_get_g0(ctx, _dp(out)), ctx)
    return out


def hf_get_fields(ctx, n_chains, L):
    f = np.zeros((n_chains, L), dtype=np.int8)
    cnt = np.zeros(n_chains, dtype=np.uint32)
    _check(lib().hf_get_fields(ctx, f.ctypes.data_as(C.POINTER(C.c_int8)),
                               cnt.ctypes.data_as(C.POINTER(C.c_uint32))), ctx)
    return f, cnt


def hf_set_fields(ctx, fields, counters=None):
    f = np.ascontiguousarray(fields, dtype=np.int8)
    cp = None
    if counters is not None:
        c = np.ascontiguousarray(counters, dtype=np.uint32)
        cp = c.ctypes.data_as(C.POINTER(C.c_uint32))
    _check(lib().hf_set_fields(ctx, f.ctypes.data_as(C.POINTER(C.c_int8)), cp), ctx)


def hf_get_green(ctx, chain, L):
    G = np.zeros((2, L, L))
    _check(lib().hf_get_green(ctx, int(chain), _dp(G)), ctx)
    return G


def hf_get_accepts(ctx, n_chains):
    a = np.zeros(n_chains, dtype=np.uint64)
    _check(lib().hf_get_accepts(ctx, a.ctypes.data_as(C.POINTER(C.c_ulonglong))), ctx)
    return a


def hf_sync(ctx):
    _check(lib().hf_sync(ctx), ctx)


def hf_get_drift(ctx):
    """(largest |G_SM - G_Dyson| at the checked refreshes, number of chain refreshes checked)."""
    m = C.c_double()
    n = C.c_ulonglong()
    _check(lib().hf_get_drift(ctx, C.byref(m), C.byref(n)), ctx)
    return m.value, n.value


def hf_get_lattice_plan(ctx):
    """(form, kernel launches per lattice step, complex multiply-adds per (w_n, sigma) matrix,
    bf16 flops per matrix of the tensor-core trailing updates)."""
    f, n, w, t = C.c_int(), C.c_int(), C.c_double(), C.c_double()
    _check(lib().hf_get_lattice_plan(ctx, C.byref(f), C.byref(n), C.byref(w), C.byref(t)), ctx)
    return f.value, n.value, w.value, t.value


def hf_get_refresh_stats(ctx):
    """(tensor-core refreshes, fallbacks to Gauss-Jordan, digit products) since the last clear."""
    a, b, n = C.c_ulonglong(), C.c_ulonglong(), C.c_ulonglong()
    _check(lib().hf_get_refresh_stats(ctx, C.byref(a), C.byref(b), C.byref(n)), ctx)
    return a.value, b.value, n.value


def hf_get_timings(ctx):
    ms = np.zeros(6)
    _check(lib().hf_get_timings(ctx, _dp(ms)), ctx)
    return ms


def hf_lattice_step_noalloc(ctx, d_sigma: int, d_gloc: int):
    """d_sigma, d_gloc: device addresses of [n_sites][2][nw] complex128 buffers."""
    _check(lib().hf_lattice_step_noalloc(ctx, C.c_void_p(d_sigma), C.c_void_p(d_gloc)), ctx)


def hf_philox_blocks(key_lo, key_hi, d_ctr: int, n: int, d_out: int, stream=None):
    _check(lib().hf_philox_blocks(key_lo, key_hi, d_ctr, n, d_out, stream))


def hf_tc_dgemm128(d_A: int, d_B: int, d_C: int, n: int, digits: int, d_status=None, stream=None):
    _check(lib().hf_tc_dgemm128(d_A, d_B, d_C, n, digits, d_status, stream))


def _bcheck(st, b=None):
    if st != HF_OK:
        msg = lib().hf_batch_last_error(b)
        raise HFError(st, msg.decode() if msg else "")


def hf_batch_create(handles, use_graph=1):
    arr = (C.c_void_p * len(handles))(*[h.value if isinstance(h, C.c_void_p) else h for h in handles])
    out = C.c_void_p()
    _bcheck(lib().hf_batch_create(arr, len(handles), int(use_graph), C.byref(out)))
    return out


def hf_batch_sweep(b, n_warmup, n_measure, refresh_first):
    _bcheck(lib().hf_batch_sweep(b, int(n_warmup), int(n_measure), int(refresh_first)), b)


def hf_batch_rdmft_step(b):
    t = C.c_double()
    _bcheck(lib().hf_batch_rdmft_step(b, C.byref(t)), b)
    return t.value


def hf_batch_elapsed(b):
    t = C.c_double()
    _bcheck(lib().hf_batch_elapsed(b, C.byref(t)), b)
    return t.value


def hf_batch_free(b):
    lib().hf_batch_free(b)


def hf_batch_last_error(b=None):
    m = lib().hf_batch_last_error(b)
    return m.decode() if m else ""


def _scheck(st, srv=None):
    if st != HF_OK:
        msg = lib().hf_srv_last_error(srv)
        raise HFError(st, msg.decode() if msg else "")


def hf_srv_workspace_size(p: hf_srv_params) -> int:
    n = C.c_size_t()
    _scheck(lib().hf_srv_workspace_size(C.byref(p), C.byref(n)))
    return n.value


def hf_srv_create(p: hf_srv_params, d_pool: int, nbytes: int):
    h = C.c_void_p()
    _scheck(lib().hf_srv_create(C.byref(p), C.c_void_p(d_pool), nbytes, C.byref(h)))
    return h


def make_request(run, site, L, beta, U, seed, g0_tau):
    r = hf_request()
    r.run, r.site, r.L, r.beta, r.U, r.seed = int(run), int(site), int(L), float(beta), float(U), int(seed)
    g = np.asarray(g0_tau, dtype=np.float64)
    for sp in range(2):
        for m in range(L):
            r.g0_tau[sp][m] = g[sp, m]
    return r


def hf_srv_submit(srv, req: hf_request) -> int:
    t = C.c_uint64()
    _scheck(lib().hf_srv_submit(srv, C.byref(req), C.byref(t)), srv)
    return t.value


def _result_dict(r: hf_result):
    L = r.L
    return {"ticket": r.ticket, "status": r.status, "L": L, "warm": r.warm,
            "sweeps_done": r.sweeps_done, "latency_s": r.latency_s,
            "gtau": np.array([[r.gtau[sp][m] for m in range(L)] for sp in range(2)]),
            "n": np.array([r.n[0], r.n[1]]), "d": r.d, "m": r.m,
            "err": np.array([r.err[k] for k in range(2 * L + 4)])}


def hf_srv_poll(srv, ticket):
    r = hf_result()
    st = lib().hf_srv_poll(srv, C.c_uint64(ticket), C.byref(r))
    if st == HF_ENOTREADY:
        return None
    _scheck(st, srv)
    return _result_dict(r)


def hf_srv_wait(srv, ticket, timeout_s=60.0):
    r = hf_result()
    _scheck(lib().hf_srv_wait(srv, C.c_uint64(ticket), float(timeout_s), C.byref(r)), srv)
    return _result_dict(r)


def hf_srv_stats(srv):
    s = hf_srv_stats_t()
    _scheck(lib().hf_srv_stats(srv, C.byref(s)), srv)
    return {k: getattr(s, k) for k, _ in hf_srv_stats_t._fields_}


def hf_srv_free(srv):
    lib().hf_srv_free(srv)


def hf_srv_last_error(srv=None):
    m = lib().hf_srv_last_error(srv)
    return m.decode() if m else ""


class Server:
    """Owns the device pool (a torch uint8 CUDA tensor) and the service handle."""

    def __init__(self, params: hf_srv_params, device="cuda:0", pool_bytes=None):
        import torch

        need = hf_srv_workspace_size(params)
        n = max(int(pool_bytes or 0), need)
        self.pool = torch.empty(n + 256, dtype=torch.uint8, device=torch.device(device))
        base = self.pool.data_ptr()
        aligned = (base + 255) & ~255
        self.handle = hf_srv_create(params, aligned, n + 256 - (aligned - base))

    def close(self):
        if getattr(self, "handle", None) is not None:
            hf_srv_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def hf_free(ctx):
    lib().hf_free(ctx)


def hf_last_error(ctx=None):
    m = lib().hf_last_error(ctx)
    return m.decode() if m else ""


# --- convenience: a context whose workspace is a torch CUDA tensor ---------------------------

def make_params(cfg: dict, stream=None, **over) -> hf_params:
    d = dict(cfg)
    d.update(over)
    p = hf_params()
    p.Lx = int(d.get("Lx", 6))
    p.Ly = int(d.get("Ly", p.Lx))
    p.Lz = int(d.get("Lz", 1))
    p.geometry = int(d.get("geometry", 0))
    p.periodic = int(d.get("periodic", 0))
    p.t = float(d.get("t", 1.0))
    p.U = float(d["U"])
    p.V0 = float(d.get("V0", 0.0))
    p.mu = float(d["mu"])
    p.beta = float(d["beta"])
    p.dtau = float(d["dtau"])
    p.n_matsubara = int(d.get("n_matsubara", 500))
    p.chains_per_site = int(d.get("chains_per_site", 1))
    p.precision = int(d.get("precision", 0))
    p.refresh_every = int(d.get("refresh_every", 10))
    p.refresh_stagger = int(d.get("refresh_stagger", 0))
    p.check_drift = int(d.get("check_drift", 0))
    p.refresh_gj = int(d.get("refresh_gj", 0))
    p.lattice_form = int(d.get("lattice_form", 0))
    p.delay_k = int(d.get("delay_k", 1))
    p.team_warps = int(d.get("team_warps", 0))
    p.bin_size = int(d.get("bin_size", 100))
    p.n_warmup = int(d.get("n_warmup", 500))
    p.n_measure = int(d.get("n_measure", 2000))
    p.max_bins = int(d.get("max_bins", max(1, -(-p.n_measure // p.bin_size))))
    p.seed = int(d.get("seed", 1))
    p.h_seed = float(d.get("h_seed", 0.1))
    p.mix = float(d.get("mix", 0.5))
    p.cuda_stream = stream
    return p


class Context:
    """Owns a device workspace (a torch uint8 CUDA tensor) and the library handle."""

    def __init__(self, params: hf_params, device="cuda:0", stream=None):
        import torch

        self.torch = torch
        dev = torch.device(device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(dev)
        params.cuda_stream = C.c_void_p(self.stream.cuda_stream)
        self.params = params
        nbytes = hf_workspace_size(params)
        self.workspace = torch.empty(nbytes + 256, dtype=torch.uint8, device=dev)
        base = self.workspace.data_ptr()
        aligned = (base + 255) & ~255
        self.handle = hf_init(params, aligned, nbytes + 256 - (aligned - base))
        self.n_sites, self.n_chains, self.L, self.N = hf_get_sizes(self.handle)
        self.nw = params.n_matsubara

    def close(self):
        if getattr(self, "handle", None) is not None:
            hf_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
