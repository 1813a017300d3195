"""CPU FP64 oracle for the SIDM scattering step -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the CUDA library and
its Python binding) never calls it and shares no code with it.

The arithmetic lives in ``sidm_oracle.cpp`` (plain C++17, FP64, no FMA
contraction); this module compiles it into ``liboracle.so`` on first use and
wraps it with ctypes.  Each wrapped function cites the passage of Zier et al.
(AREPO-2 SIDM) it restates; see the C++ header comment for the readings taken
where the paper is silent.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sidm_oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile liboracle.so (g++, -O2, OpenMP, no FP contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-fopenmp", "-ffp-contract=off",
                               "-fno-fast-math", "-fPIC", "-shared", _SRC, "-o", tmp])
        os.replace(tmp, _LIB)
    return _LIB


_tables = []   # keeps the arrays behind table pointers (Config, Sigma) alive


class Config(C.Structure):
    _fields_ = [("n_ngb", C.c_int), ("ngb_tol", C.c_int), ("c_sidm", C.c_double),
                ("box", C.c_double), ("kernel", C.c_int), ("fixed_h", C.c_double),
                ("use_tree", C.c_int), ("n_threads", C.c_int), ("estimator", C.c_int),
                ("ov_na", C.c_int), ("ov_ns", C.c_int), ("ov_table", C.POINTER(C.c_double))]


class Sigma(C.Structure):
    _fields_ = [("kind", C.c_int), ("sigma0", C.c_double), ("w", C.c_double),
                ("inelastic", C.c_double), ("tab_n", C.c_int32),
                ("tab_v", C.POINTER(C.c_double)), ("tab_s", C.POINTER(C.c_double))]


class Stats(C.Structure):
    _fields_ = [("n_active", C.c_int64), ("n_candidate_pairs", C.c_int64),
                ("n_accepted", C.c_int64), ("n_p_ge_1", C.c_int64),
                ("n_h_nonconv", C.c_int64), ("n_dir_fail", C.c_int64),
                ("e_before", C.c_double), ("e_after", C.c_double),
                ("p_before", C.c_double * 3), ("p_after", C.c_double * 3),
                ("sum_p", C.c_double)]

    def as_dict(self) -> dict:
        d = {k: getattr(self, k) for k, _ in self._fields_}
        d["p_before"] = list(self.p_before)
        d["p_after"] = list(self.p_after)
        return d


def _p(a, t):
    return a.ctypes.data_as(C.POINTER(t)) if a is not None else None


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            dp, u32p, i64p, u8p, i8p, u64p, ip = (C.POINTER(C.c_double), C.POINTER(C.c_uint32),
                                                    C.POINTER(C.c_int64), C.POINTER(C.c_uint8),
                                                    C.POINTER(C.c_int8), C.POINTER(C.c_uint64),
                                                    C.POINTER(C.c_int))
            L.orc_philox4x32_10.argtypes = [u32p, u32p, u32p]
            L.orc_uniform53.argtypes = [C.c_uint32, C.c_uint32]
            L.orc_uniform53.restype = C.c_double
            L.orc_kernel_w.argtypes = [C.c_int, C.c_double, C.c_double]
            L.orc_kernel_w.restype = C.c_double
            L.orc_sigma_over_m.argtypes = [C.POINTER(Sigma), C.c_double]
            L.orc_sigma_over_m.restype = C.c_double
            L.orc_overlap_quadrature.argtypes = [C.c_int, C.c_double, C.c_double, C.c_int]
            L.orc_overlap_quadrature.restype = C.c_double
            L.orc_overlap_table.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, dp]
            L.orc_overlap_table.restype = None
            L.orc_overlap_g.argtypes = [C.POINTER(Config), C.c_double, C.c_double, C.c_double]
            L.orc_overlap_g.restype = C.c_double
            L.orc_directed_probability.argtypes = [C.c_int, C.POINTER(Sigma), C.c_double, dp, dp,
                                                   C.c_double, C.c_double, C.c_double]
            L.orc_directed_probability.restype = C.c_double
            L.orc_direction.argtypes = [C.c_uint64, C.c_uint64, C.c_uint32, C.c_uint32, dp]
            L.orc_direction.restype = C.c_int
            L.orc_kick.argtypes = [C.c_double, C.c_double, dp, dp, dp, C.c_double]
            L.orc_initial_h.argtypes = [C.c_double, C.c_int64, C.c_int]
            L.orc_initial_h.restype = C.c_double
            L.orc_counts.argtypes = [C.c_int64, dp, C.c_double, C.c_int, C.c_int64, i64p, dp, i64p]
            L.orc_h_for.argtypes = [C.POINTER(Config), C.c_int64, dp, C.c_int64, i64p, dp, i64p, ip]
            L.orc_step.argtypes = [C.POINTER(Config), C.c_int64, dp, dp, dp, u32p, u8p, i8p,
                                   C.c_double, C.POINTER(Sigma), C.c_uint64, C.c_uint64, dp, dp,
                                   C.c_int64, u32p, u64p, dp, i64p, C.POINTER(Stats)]
            L.orc_step.restype = C.c_int
            L.orc_apply_pairs.argtypes = [C.c_int64, C.c_int64, u64p, u32p, u32p, i64p, i64p, dp,
                                          dp, C.c_uint64, C.c_uint64, C.c_double]
            L.orc_apply_pairs.restype = C.c_int64
            _lib = L
    return _lib


def make_config(n_ngb=32, ngb_tol=5, c_sidm=0.1, box=0.0, kernel=0, fixed_h=0.0,
                use_tree=1, n_threads=0, overlap_table=None) -> Config:
    """overlap_table: None (one-sided estimator, Eq. 14) or a (na+1, ns+1) array
    of ghat on a = k / (2 na), s = l / ns (kernel-overlap estimator, Eq. 15)."""
    cfg = Config(int(n_ngb), int(ngb_tol), float(c_sidm), float(box), int(kernel),
                 float(fixed_h), int(use_tree), int(n_threads), 0, 0, 0, None)
    if overlap_table is not None:
        t = np.ascontiguousarray(overlap_table, np.float64)
        _tables.append((t,))
        del _tables[:-8]
        cfg.estimator = 1
        cfg.ov_na, cfg.ov_ns = t.shape[0] - 1, t.shape[1] - 1
        cfg.ov_table = t.ctypes.data_as(C.POINTER(C.c_double))
    return cfg




def make_sigma(kind=0, sigma0=1.0, w=1.0, inelastic=0.0, table=None) -> Sigma:
    """Cross-section model; kind 2 takes table = (v nodes, sigma/m values)."""
    s = Sigma(int(kind), float(sigma0), float(w), float(inelastic), 0, None, None)
    if table is not None:
        tv = np.ascontiguousarray(table[0], np.float64)
        ts = np.ascontiguousarray(table[1], np.float64)
        _tables.append((tv, ts))
        del _tables[:-8]
        s.tab_n = int(tv.shape[0])
        s.tab_v = tv.ctypes.data_as(C.POINTER(C.c_double))
        s.tab_s = ts.ctypes.data_as(C.POINTER(C.c_double))
    return s


# ------------------------------------------------------------ primitives ---

def philox4x32_10(key, ctr) -> np.ndarray:
    """Philox-4x32-10 block (Salmon et al., SC'11)."""
    k = np.ascontiguousarray(key, np.uint32)
    c = np.ascontiguousarray(ctr, np.uint32)
    o = np.zeros(4, np.uint32)
    lib().orc_philox4x32_10(_p(k, C.c_uint32), _p(c, C.c_uint32), _p(o, C.c_uint32))
    return o


def uniform53(wa: int, wb: int) -> float:
    return lib().orc_uniform53(int(wa), int(wb))


def kernel_w(r: float, h: float, kernel: int = 0) -> float:
    """Cubic spline W_CS (kernel 0) or top-hat W_TH (kernel 1), Sec. 4.2."""
    return lib().orc_kernel_w(int(kernel), float(r), float(h))


def sigma_over_m(vrel: float, kind=0, sigma0=1.0, w=1.0, table=None) -> float:
    s = make_sigma(kind, sigma0, w, table=table)
    return lib().orc_sigma_over_m(C.byref(s), float(vrel))


def directed_probability(m_j, v_i, v_j, r2, h_i, dt_i, kernel=0, kind=0, sigma0=1.0, w=1.0):
    """P(i|j) of Eq. 11 with the rate of Eq. 10 and g_ij of Eq. 14."""
    s = make_sigma(kind, sigma0, w)
    vi = np.ascontiguousarray(v_i, np.float64)
    vj = np.ascontiguousarray(v_j, np.float64)
    return lib().orc_directed_probability(int(kernel), C.byref(s), float(m_j), _p(vi, C.c_double),
                                          _p(vj, C.c_double), float(r2), float(h_i), float(dt_i))


def overlap_quadrature(a: float, s: float, kernel=0, panels=24) -> float:
    """ghat(a, s) of the kernel-overlap estimator (Eq. 15) by quadrature."""
    return lib().orc_overlap_quadrature(int(kernel), float(a), float(s), int(panels))


def overlap_table(na=32, ns=128, kernel=0, panels=24) -> np.ndarray:
    """Table of ghat on a = k / (2 na), s = l / ns (Appendix A)."""
    out = np.zeros((na + 1, ns + 1))
    lib().orc_overlap_table(int(kernel), int(na), int(ns), int(panels), _p(out, C.c_double))
    return out


def overlap_g(table, h_i, h_j, r2) -> float:
    """g_ij from the table: ghat(min(h)/H, r/H) / H^3, H = h_i + h_j."""
    cfg = make_config(overlap_table=table)
    return lib().orc_overlap_g(C.byref(cfg), float(h_i), float(h_j), float(r2))


def direction(seed: int, step: int, a: int, b: int):
    e = np.zeros(3)
    ok = lib().orc_direction(seed, step, a, b, _p(e, C.c_double))
    return e, bool(ok)


def kick(mi, mj, vi, vj, e, eps=1.0):
    """Centre-of-momentum kick, Sec. 4.1: outgoing relative speed eps times
    the incoming one (eps = 1: elastic)."""
    vi = np.array(vi, np.float64)
    vj = np.array(vj, np.float64)
    e = np.ascontiguousarray(e, np.float64)
    lib().orc_kick(float(mi), float(mj), _p(vi, C.c_double), _p(vj, C.c_double), _p(e, C.c_double),
                   float(eps))
    return vi, vj


def initial_h(l_ext: float, n: int, n_ngb: int) -> float:
    return lib().orc_initial_h(float(l_ext), int(n), int(n_ngb))


def counts(pos, h, query=None, box=0.0, use_tree=True) -> np.ndarray:
    """Neighbour counts #{j != i : r_ij < h_i} for the query particles."""
    pos = np.ascontiguousarray(pos, np.float64)
    n = pos.shape[0]
    q = np.arange(n, dtype=np.int64) if query is None else np.ascontiguousarray(query, np.int64)
    hh = np.ascontiguousarray(np.broadcast_to(np.asarray(h, np.float64), q.shape), np.float64)
    out = np.zeros(q.shape[0], np.int64)
    lib().orc_counts(n, _p(pos, C.c_double), float(box), int(use_tree), q.shape[0],
                     _p(q, C.c_int64), _p(hh, C.c_double), _p(out, C.c_int64))
    return out


def h_for(pos, query, n_ngb=32, ngb_tol=5, box=0.0, use_tree=True, n_threads=0):
    """h_SI by bisection for the query particles (Sec. 4.2/4.5)."""
    pos = np.ascontiguousarray(pos, np.float64)
    q = np.ascontiguousarray(query, np.int64)
    cfg = make_config(n_ngb, ngb_tol, 0.1, box, 0, 0.0, int(use_tree), n_threads)
    h = np.zeros(q.shape[0])
    cnt = np.zeros(q.shape[0], np.int64)
    nc = np.zeros(q.shape[0], np.int32)
    lib().orc_h_for(C.byref(cfg), pos.shape[0], _p(pos, C.c_double), q.shape[0], _p(q, C.c_int64),
                    _p(h, C.c_double), _p(cnt, C.c_int64), nc.ctypes.data_as(C.POINTER(C.c_int)))
    return h, cnt, nc


def step(pos, vel, mass, ids, active, bins, dt_max, *, n_ngb=32, ngb_tol=5, c_sidm=0.1,
         box=0.0, kernel=0, fixed_h=0.0, sigma_kind=0, sigma0=1.0, w=1.0, inelastic=0.0,
         table=None, overlap_table=None, seed=0, step=0,
         use_tree=True, n_threads=0, max_pairs=None, h_init=None, dtlim_init=None):
    """One scattering step (Sec. 4); returns a dict with the new velocities,
    h and dt-limits (active particles updated, others from *_init or 0/inf),
    the accepted pairs sorted by (ord, a, b), and the step statistics."""
    pos = np.ascontiguousarray(pos, np.float64)
    n = pos.shape[0]
    vel = np.array(vel, np.float64, order="C", copy=True)
    mass = np.ascontiguousarray(mass, np.float64)
    ids = np.ascontiguousarray(ids, np.uint32)
    act = None if active is None else np.ascontiguousarray(active, np.uint8)
    bins = np.ascontiguousarray(bins, np.int8)
    h = np.zeros(n) if h_init is None else np.array(h_init, np.float64, copy=True)
    dl = np.full(n, np.inf) if dtlim_init is None else np.array(dtlim_init, np.float64, copy=True)
    cap = (4 * n + 16) if max_pairs is None else int(max_pairs)
    ab = np.zeros((cap, 2), np.uint32)
    ords = np.zeros(cap, np.uint64)
    pp = np.zeros(cap, np.float64)
    npairs = C.c_int64(0)
    st = Stats()
    cfg = make_config(n_ngb, ngb_tol, c_sidm, box, kernel, fixed_h, int(use_tree), n_threads,
                      overlap_table)
    sg = make_sigma(sigma_kind, sigma0, w, inelastic, table)
    rc = lib().orc_step(C.byref(cfg), n, _p(pos, C.c_double), _p(vel, C.c_double),
                        _p(mass, C.c_double), _p(ids, C.c_uint32), _p(act, C.c_uint8),
                        _p(bins, C.c_int8), float(dt_max), C.byref(sg), int(seed), int(step),
                        _p(h, C.c_double), _p(dl, C.c_double), cap, _p(ab, C.c_uint32),
                        _p(ords, C.c_uint64), _p(pp, C.c_double), C.byref(npairs), C.byref(st))
    if rc != 0:
        raise ValueError("oracle step: invalid arguments")
    k = min(npairs.value, cap)
    return {"vel": vel, "h": h, "dtlim": dl, "pairs_ab": ab[:k].copy(), "pairs_ord": ords[:k].copy(),
            "pairs_p": pp[:k].copy(), "n_pairs": npairs.value, "stats": st.as_dict()}


def apply_pairs(vel, mass, ords, ab, idx, seed, step, eps=1.0):
    """Canonical application of given accepted pairs (Sec. 4.1 kick, Sec. 4.4
    multiple scatters): ascending (ord, a, b), equal keys in the order given,
    each kick reading the current velocities.  ab: (k, 2) ids a < b; idx:
    (k, 2) storage indices of the a- and b-particle.  Returns the new
    velocities and the number of exhausted direction draws."""
    vel = np.array(vel, np.float64, order="C", copy=True)
    mass = np.ascontiguousarray(mass, np.float64)
    o = np.ascontiguousarray(ords, np.uint64)
    ab = np.asarray(ab)
    idx = np.asarray(idx)
    a = np.ascontiguousarray(ab[:, 0], np.uint32)
    b = np.ascontiguousarray(ab[:, 1], np.uint32)
    ia = np.ascontiguousarray(idx[:, 0], np.int64)
    ib = np.ascontiguousarray(idx[:, 1], np.int64)
    r = lib().orc_apply_pairs(vel.shape[0], o.shape[0], _p(o, C.c_uint64), _p(a, C.c_uint32),
                              _p(b, C.c_uint32), _p(ia, C.c_int64), _p(ib, C.c_int64),
                              _p(vel, C.c_double), _p(mass, C.c_double), int(seed), int(step),
                              float(eps))
    if r < 0:
        raise ValueError("oracle apply_pairs: index outside [0, n) or a pair names one particle twice")
    return vel, int(r)
