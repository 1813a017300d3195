"""Python binding of libsidm.so (include/sidm.h) -- argument marshalling only.

Every step of the scattering path runs in the CUDA library; this module only
converts numpy arrays / torch tensors to pointers and status codes to
exceptions.  It never computes any part of the step itself and has no CPU
fallback: if the library cannot be loaded, :func:`lib` raises.

The functions ``sidm_*`` mirror the C entry points one to one; :class:`Context`
is a convenience wrapper that owns one ``sidm_ctx``.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import build as _build

HOST, DEVICE = 0, 1
KERNEL_CUBIC, KERNEL_TOPHAT = 0, 1
FP64_PLAIN, FP32_SPLIT = 0, 1
ESTIMATOR_ONE_SIDED, ESTIMATOR_OVERLAP = 0, 1
SIGMA_CONST, SIGMA_YUKAWA, SIGMA_TABLE = 0, 1, 2
SIGMA_TABLE_MAX = 256

OK = 0
WARN_H_NOT_CONVERGED, WARN_P_GE_1, WARN_DIRECTION = 1, 2, 4
ERR_INVALID_ARG, ERR_OOM, ERR_CUDA, ERR_DEVICE_LIMIT, ERR_NOT_READY = -1, -2, -3, -4, -5
ERR_TOO_LARGE = -6
NOALLOC_MAX_PARTICLES, NOALLOC_MAX_PAIRS = 1 << 20, 1 << 18
# record layout of sidm_pair (include/sidm.h)
PAIR_DTYPE = np.dtype([("ord", "<u8"), ("a", "<u4"), ("b", "<u4"), ("ia", "<i4"), ("ib", "<i4")])


class SidmError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__(f"{what}: {error_string(status)} (status {status})")
        self.status = status


# allocator hooks of sidm_config: alloc(bytes, stream, user) -> ptr, free(ptr, stream, user)
ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p, C.c_void_p)


class Config(C.Structure):
    _fields_ = [("n_ngb", C.c_int), ("ngb_tol", C.c_int), ("c_sidm", C.c_double),
                ("box", C.c_double), ("kernel", C.c_int), ("precision", C.c_int),
                ("fixed_h", C.c_double), ("n_max", C.c_int64), ("pair_capacity", C.c_int64),
                ("stream", C.c_void_p), ("device", C.c_int), ("profile", C.c_int),
                ("use_graph", C.c_int), ("estimator", C.c_int), ("rebuild_every", C.c_int),
                ("max_resolver_passes", C.c_int), ("alloc", ALLOC_FN), ("free", FREE_FN),
                ("alloc_user", C.c_void_p), ("search_hint", C.c_int)]


class Tuning(C.Structure):
    _fields_ = [("search_window", C.c_int), ("search_chunk", C.c_int),
                ("search_blocks_per_sm", C.c_int), ("pairs_chunk", C.c_int),
                ("pairs_blocks_per_sm", C.c_int), ("search_run", C.c_int)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class SigmaModel(C.Structure):
    _fields_ = [("kind", C.c_int), ("sigma0", C.c_double), ("w", C.c_double),
                ("inelastic", C.c_double)]


class HaloParams(C.Structure):
    _fields_ = [("dt_max", C.c_double), ("sigma", SigmaModel), ("seed", C.c_uint64),
                ("step", C.c_uint64)]


class StepStats(C.Structure):
    _fields_ = [("n_active", C.c_int64), ("n_candidate_pairs", C.c_int64),
                ("n_accepted", C.c_int64), ("n_rounds", C.c_int64), ("n_p_ge_1", C.c_int64),
                ("n_h_nonconv", C.c_int64), ("n_dir_fail", C.c_int64),
                ("max_multiplicity", C.c_int64), ("sum_p", C.c_double),
                ("e_before", C.c_double), ("e_after", C.c_double),
                ("p_before", C.c_double * 3), ("p_after", C.c_double * 3),
                ("status", C.c_int32), ("reserved", C.c_int32)]

    def as_dict(self) -> dict:
        d = {k: getattr(self, k) for k, _ in self._fields_ if k != "reserved"}
        d["p_before"] = list(self.p_before)
        d["p_after"] = list(self.p_after)
        return d


# names of every entry point declared in include/sidm.h
ENTRY_POINTS = ("sidm_default_config", "sidm_create", "sidm_set_particles",
                "sidm_set_velocities", "sidm_set_positions", "sidm_get_changed", "sidm_update_velocities",
                "sidm_set_velocity_mirror", "sidm_step", "sidm_sync", "sidm_get_particles",
                "sidm_timestep_limits", "sidm_get_pairs", "sidm_get_step", "sidm_set_step",
                "sidm_phase_times", "sidm_kernel_launches", "sidm_error_string", "sidm_destroy",
                "sidm_apply_pairs_noalloc", "sidm_set_haloes", "sidm_step_haloes",
                "sidm_set_tuning", "sidm_get_tuning", "sidm_autotune", "sidm_graph_state",
                "sidm_set_sigma_table", "sidm_set_overlap_table", "sidm_overlap_table",
                "sidm_write_particles", "sidm_set_count", "sidm_read_particles",
                "sidm_context_bytes", "sidm_move_particles")

N_PHASES = 6
PHASES = ("keys", "sort", "structure", "search", "pairs", "resolve")

_lock = threading.Lock()
_lib = None


def lib_path() -> str:
    return _build.LIB


def lib():
    """Loads libsidm.so (building it first if sources are newer and nvcc exists)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if not _build.up_to_date():
            if os.path.exists(_build.NVCC):
                _build.build()
            elif not os.path.exists(path):
                raise ImportError(f"libsidm.so not found at {path} and nvcc unavailable")
        L = C.CDLL(path)
        vp, i64, dp = C.c_void_p, C.c_int64, C.c_double
        L.sidm_default_config.argtypes = [C.POINTER(Config)]
        L.sidm_default_config.restype = None
        L.sidm_create.argtypes = [C.POINTER(Config), C.POINTER(vp)]
        L.sidm_set_particles.argtypes = [vp, i64, vp, vp, vp, dp, vp, C.c_int]
        L.sidm_set_velocities.argtypes = [vp, vp, C.c_int]
        L.sidm_set_positions.argtypes = [vp, vp, C.c_int]
        L.sidm_get_changed.argtypes = [vp, vp, vp, i64, C.POINTER(i64), C.c_int]
        L.sidm_update_velocities.argtypes = [vp, vp]
        L.sidm_set_velocity_mirror.argtypes = [vp, vp, i64]
        L.sidm_step.argtypes = [vp, vp, vp, dp, C.POINTER(SigmaModel), C.c_uint64,
                                C.POINTER(StepStats)]
        L.sidm_sync.argtypes = [vp]
        L.sidm_get_particles.argtypes = [vp, vp, vp, C.c_int]
        L.sidm_timestep_limits.argtypes = [vp, vp, C.c_int]
        L.sidm_get_pairs.argtypes = [vp, vp, vp, i64, C.POINTER(i64)]
        L.sidm_get_step.argtypes = [vp, C.POINTER(C.c_uint64)]
        L.sidm_set_step.argtypes = [vp, C.c_uint64]
        L.sidm_phase_times.argtypes = [vp, C.POINTER(C.c_float), C.c_int]
        L.sidm_kernel_launches.argtypes = [vp]
        L.sidm_error_string.argtypes = [C.c_int]
        L.sidm_error_string.restype = C.c_char_p
        L.sidm_destroy.argtypes = [vp]
        L.sidm_destroy.restype = None
        L.sidm_apply_pairs_noalloc.argtypes = [vp, i64, vp, vp, i64, C.c_uint64, C.c_uint64, vp]
        L.sidm_set_haloes.argtypes = [vp, C.c_int32, C.POINTER(C.c_int64)]
        L.sidm_step_haloes.argtypes = [vp, vp, vp, C.POINTER(HaloParams), C.POINTER(StepStats)]
        L.sidm_set_tuning.argtypes = [vp, C.POINTER(Tuning)]
        L.sidm_get_tuning.argtypes = [vp, C.POINTER(Tuning)]
        L.sidm_autotune.argtypes = [vp, vp, vp, C.POINTER(HaloParams), C.c_int,
                                    C.POINTER(Tuning)]
        L.sidm_graph_state.argtypes = [vp]
        L.sidm_set_sigma_table.argtypes = [vp, C.c_int32, vp, vp]
        L.sidm_set_overlap_table.argtypes = [vp, C.c_int32, C.c_int32, vp]
        L.sidm_overlap_table.argtypes = [C.c_int, C.c_int32, C.c_int32, vp]
        L.sidm_write_particles.argtypes = [vp, i64, i64, vp, vp, vp, dp, vp, C.c_int]
        L.sidm_set_count.argtypes = [vp, i64]
        L.sidm_move_particles.argtypes = [vp, i64, i64, i64]
        L.sidm_read_particles.argtypes = [vp, i64, i64, vp, vp, C.c_int]
        L.sidm_context_bytes.argtypes = [C.POINTER(Config), i64, C.POINTER(i64)]
        for name in ENTRY_POINTS:
            fn = getattr(L, name)
            if name not in ("sidm_default_config", "sidm_error_string", "sidm_destroy"):
                fn.restype = C.c_int
        L.sidm_kernel_launches.restype = C.c_int64
        _lib = L
        return L


def error_string(status: int) -> str:
    return lib().sidm_error_string(int(status)).decode()


def _check(status: int, what: str) -> int:
    if status < 0:
        raise SidmError(status, what)
    return status


def _ptr(a):
    """(pointer, ptr_kind) of a numpy array or a torch tensor (None -> NULL)."""
    if a is None:
        return None, HOST
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data, HOST
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr(), (DEVICE if a.is_cuda else HOST)
    raise TypeError(type(a))


# ------------------------------------------------------- C entry points ---

def sidm_default_config() -> Config:
    c = Config()
    lib().sidm_default_config(C.byref(c))
    return c


def sidm_create(cfg: Config) -> int:
    h = C.c_void_p()
    _check(lib().sidm_create(C.byref(cfg), C.byref(h)), "sidm_create")
    return h.value


def sidm_set_particles(ctx, pos, vel, mass, mass_scalar, ids) -> int:
    n = int(pos.shape[0])
    pp, kind = _ptr(pos)
    return _check(lib().sidm_set_particles(ctx, n, pp, _ptr(vel)[0], _ptr(mass)[0],
                                           float(mass_scalar), _ptr(ids)[0], kind),
                  "sidm_set_particles")


def sidm_set_velocities(ctx, vel) -> int:
    p, kind = _ptr(vel)
    return _check(lib().sidm_set_velocities(ctx, p, kind), "sidm_set_velocities")


def sidm_set_positions(ctx, pos) -> int:
    p, kind = _ptr(pos)
    return _check(lib().sidm_set_positions(ctx, p, kind), "sidm_set_positions")


def sidm_write_particles(ctx, offset, pos, vel, mass, mass_scalar, ids) -> int:
    n = int(pos.shape[0])
    pp, kind = _ptr(pos)
    return _check(lib().sidm_write_particles(ctx, int(offset), n, pp, _ptr(vel)[0], _ptr(mass)[0],
                                             float(mass_scalar), _ptr(ids)[0], kind),
                  "sidm_write_particles")


def sidm_set_count(ctx, n) -> int:
    return _check(lib().sidm_set_count(ctx, int(n)), "sidm_set_count")


def sidm_move_particles(ctx, src, dst, count) -> int:
    return _check(lib().sidm_move_particles(ctx, int(src), int(dst), int(count)),
                  "sidm_move_particles")


def sidm_read_particles(ctx, offset, count, vel_out, h_out=None) -> int:
    p, kind = _ptr(vel_out if vel_out is not None else h_out)
    return _check(lib().sidm_read_particles(ctx, int(offset), int(count), _ptr(vel_out)[0],
                                            _ptr(h_out)[0], kind), "sidm_read_particles")


def sidm_context_bytes(cfg: Config, n) -> int:
    b = C.c_int64(0)
    _check(lib().sidm_context_bytes(C.byref(cfg), int(n), C.byref(b)), "sidm_context_bytes")
    return b.value


def torch_allocator(device: int):
    """(alloc, free) hooks that take the context's device memory from
    PyTorch's caching allocator on `device` (kept alive by the caller)."""
    import torch

    @ALLOC_FN
    def _alloc(nbytes, stream, user):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), device, int(stream or 0))
        except Exception:
            return None

    @FREE_FN
    def _free(ptr, stream, user):
        torch.cuda.caching_allocator_delete(int(ptr))

    return _alloc, _free


def sidm_step(ctx, active_mask, dt_bins, dt_max, sigma: SigmaModel, seed, stats=None) -> int:
    return _check(lib().sidm_step(ctx, _ptr(active_mask)[0], _ptr(dt_bins)[0], float(dt_max),
                                  C.byref(sigma), int(seed),
                                  C.byref(stats) if stats is not None else None), "sidm_step")


def sidm_set_haloes(ctx, offsets) -> int:
    off = np.ascontiguousarray(offsets, np.int64)
    return _check(lib().sidm_set_haloes(ctx, int(off.shape[0] - 1),
                                        off.ctypes.data_as(C.POINTER(C.c_int64))),
                  "sidm_set_haloes")


def sidm_step_haloes(ctx, active_mask, dt_bins, params, stats=None) -> int:
    arr = (HaloParams * len(params))(*params)
    return _check(lib().sidm_step_haloes(ctx, _ptr(active_mask)[0], _ptr(dt_bins)[0], arr,
                                         C.byref(stats) if stats is not None else None),
                  "sidm_step_haloes")


def sidm_set_tuning(ctx, t: Tuning) -> int:
    return _check(lib().sidm_set_tuning(ctx, C.byref(t)), "sidm_set_tuning")


def sidm_get_tuning(ctx) -> Tuning:
    t = Tuning()
    _check(lib().sidm_get_tuning(ctx, C.byref(t)), "sidm_get_tuning")
    return t


def sidm_autotune(ctx, active_mask, dt_bins, params, reps=3) -> Tuning:
    arr = (HaloParams * len(params))(*params)
    t = Tuning()
    _check(lib().sidm_autotune(ctx, _ptr(active_mask)[0], _ptr(dt_bins)[0], arr, int(reps),
                               C.byref(t)), "sidm_autotune")
    return t


def sidm_set_sigma_table(ctx, v, sigma_over_m) -> int:
    v = np.ascontiguousarray(v, np.float64)
    s = np.ascontiguousarray(sigma_over_m, np.float64)
    if v.shape != s.shape:
        raise ValueError("table arrays differ in length")
    return _check(lib().sidm_set_sigma_table(ctx, int(v.shape[0]), v.ctypes.data, s.ctypes.data),
                  "sidm_set_sigma_table")


def sidm_set_overlap_table(ctx, table) -> int:
    t = np.ascontiguousarray(table, np.float64)
    if t.ndim != 2:
        raise ValueError("overlap table must be (na + 1) x (ns + 1)")
    return _check(lib().sidm_set_overlap_table(ctx, t.shape[0] - 1, t.shape[1] - 1, t.ctypes.data),
                  "sidm_set_overlap_table")


def sidm_overlap_table(kernel=KERNEL_CUBIC, na=32, ns=128) -> np.ndarray:
    """The kernel-overlap table ghat on a = k / (2 na), s = l / ns (host)."""
    out = np.zeros((na + 1, ns + 1))
    _check(lib().sidm_overlap_table(int(kernel), int(na), int(ns), out.ctypes.data),
           "sidm_overlap_table")
    return out


def sidm_graph_state(ctx) -> int:
    return int(lib().sidm_graph_state(ctx))


def sidm_sync(ctx) -> int:
    return _check(lib().sidm_sync(ctx), "sidm_sync")


def sidm_get_particles(ctx, vel_out, h_out=None) -> int:
    p, kind = _ptr(vel_out)
    return _check(lib().sidm_get_particles(ctx, p, _ptr(h_out)[0], kind), "sidm_get_particles")


def sidm_get_changed(ctx, idx_out, vel_out) -> int:
    """Fills idx_out (int32) and vel_out (k x 3) with the particles the last
    step changed, up to their length; returns the full count."""
    p, kind = _ptr(idx_out)
    n = C.c_int64(0)
    _check(lib().sidm_get_changed(ctx, p, _ptr(vel_out)[0], int(idx_out.shape[0]),
                                  C.byref(n), kind), "sidm_get_changed")
    return int(n.value)


def sidm_update_velocities(ctx, vel_inout) -> int:
    """Writes the velocities the last step changed into the host array
    vel_inout (n x 3, float64, C-contiguous) in place."""
    if not (isinstance(vel_inout, np.ndarray) and vel_inout.dtype == np.float64 and
            vel_inout.flags.c_contiguous):
        raise SidmError(ERR_INVALID_ARG, "sidm_update_velocities: host float64 C-contiguous array")
    return _check(lib().sidm_update_velocities(ctx, vel_inout.ctypes.data_as(C.c_void_p)),
                  "sidm_update_velocities")


def sidm_set_velocity_mirror(ctx, host_vel) -> int:
    """From the next step on, the device writes every changed velocity into
    host_vel (n x 3 float64, C-contiguous, pinned memory the device can
    address, e.g. a numpy view of a pinned torch tensor); None stops it.
    The array must stay alive while it is set."""
    if host_vel is None:
        return _check(lib().sidm_set_velocity_mirror(ctx, None, 0), "sidm_set_velocity_mirror")
    if not (isinstance(host_vel, np.ndarray) and host_vel.dtype == np.float64 and
            host_vel.flags.c_contiguous and host_vel.ndim == 2 and host_vel.shape[1] == 3):
        raise SidmError(ERR_INVALID_ARG, "sidm_set_velocity_mirror: host float64 (n, 3) array")
    return _check(lib().sidm_set_velocity_mirror(ctx, host_vel.ctypes.data_as(C.c_void_p),
                                                 int(host_vel.shape[0])),
                  "sidm_set_velocity_mirror")


def sidm_timestep_limits(ctx, out) -> int:
    p, kind = _ptr(out)
    return _check(lib().sidm_timestep_limits(ctx, p, kind), "sidm_timestep_limits")


def sidm_get_pairs(ctx, ab, ord_, cap) -> int:
    n = C.c_int64(0)
    _check(lib().sidm_get_pairs(ctx, _ptr(ab)[0], _ptr(ord_)[0], int(cap), C.byref(n)),
           "sidm_get_pairs")
    return n.value


def sidm_get_step(ctx) -> int:
    s = C.c_uint64(0)
    _check(lib().sidm_get_step(ctx, C.byref(s)), "sidm_get_step")
    return s.value


def sidm_set_step(ctx, step) -> int:
    return _check(lib().sidm_set_step(ctx, int(step)), "sidm_set_step")


def sidm_phase_times(ctx) -> list:
    ms = (C.c_float * N_PHASES)()
    _check(lib().sidm_phase_times(ctx, ms, N_PHASES), "sidm_phase_times")
    return list(ms)


def sidm_kernel_launches(ctx) -> int:
    return int(lib().sidm_kernel_launches(ctx))


def sidm_destroy(ctx) -> None:
    if ctx:
        lib().sidm_destroy(ctx)


def sidm_apply_pairs_noalloc(pairs, n_pairs, vel, mass, n, seed, step, stream=None) -> int:
    """Kicks of the given accepted pairs applied to ``vel`` in place, with no
    device allocation (fixed scratch inside the library; device pointers or
    CUDA tensors).  Returns the status (negative statuses raise)."""
    return _check(lib().sidm_apply_pairs_noalloc(_ptr(pairs)[0], int(n_pairs), _ptr(vel)[0],
                                                 _ptr(mass)[0], int(n), int(seed), int(step),
                                                 stream), "sidm_apply_pairs_noalloc")


# ------------------------------------------------------------- wrapper ---

class Context:
    """One library context.  Host (numpy) and device (torch CUDA) inputs both
    work; outputs are numpy arrays unless device tensors are passed in."""

    def __init__(self, n_ngb=32, ngb_tol=5, c_sidm=0.1, box=0.0, kernel=KERNEL_CUBIC,
                 fixed_h=0.0, n_max=0, pair_capacity=0, stream=None, device=-1, profile=False,
                 precision=FP64_PLAIN, use_graph=False, rebuild_every=0,
                 estimator=ESTIMATOR_ONE_SIDED, max_resolver_passes=0, allocator=None,
                 search_hint=False):
        """allocator: None (the library's cudaMalloc) or "torch" (PyTorch's
        caching allocator on the context's device)."""
        cfg = sidm_default_config()
        cfg.n_ngb, cfg.ngb_tol, cfg.c_sidm, cfg.box = int(n_ngb), int(ngb_tol), float(c_sidm), float(box)
        cfg.kernel, cfg.fixed_h, cfg.n_max = int(kernel), float(fixed_h), int(n_max)
        cfg.pair_capacity = int(pair_capacity)
        cfg.stream = stream
        cfg.device = int(device)
        cfg.profile = int(bool(profile))
        cfg.precision = int(precision)
        cfg.use_graph = int(bool(use_graph))
        cfg.rebuild_every = int(rebuild_every)
        cfg.estimator = int(estimator)
        cfg.max_resolver_passes = int(max_resolver_passes)
        cfg.search_hint = int(bool(search_hint))
        self._hooks = None
        if allocator == "torch":
            import torch
            dev = int(device) if int(device) >= 0 else torch.cuda.current_device()
            self._hooks = torch_allocator(dev)
            cfg.alloc, cfg.free = self._hooks
        elif allocator is not None:
            raise ValueError(f"unknown allocator {allocator!r}")
        self.cfg = cfg
        self.handle = sidm_create(cfg)
        self.n = 0

    def close(self):
        if self.handle:
            sidm_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def set_particles(self, pos, vel, ids, mass=None, mass_scalar=0.0):
        if isinstance(pos, np.ndarray):
            pos = np.ascontiguousarray(pos, np.float64)
            vel = np.ascontiguousarray(vel, np.float64)
            ids = np.ascontiguousarray(ids, np.uint32)
            mass = None if mass is None else np.ascontiguousarray(mass, np.float64)
        self._keep = (pos, vel, ids, mass)
        sidm_set_particles(self.handle, pos, vel, mass, mass_scalar, ids)
        self.n = int(pos.shape[0])

    def write_particles(self, offset, pos, vel, ids, mass=None, mass_scalar=0.0):
        """Replaces particles [offset, offset + len(pos)) (growing the loaded
        count when it reaches past it); the other particles are kept."""
        if isinstance(pos, np.ndarray):
            pos = np.ascontiguousarray(pos, np.float64)
            vel = np.ascontiguousarray(vel, np.float64)
            ids = np.ascontiguousarray(ids, np.uint32)
            mass = None if mass is None else np.ascontiguousarray(mass, np.float64)
        sidm_write_particles(self.handle, offset, pos, vel, mass, mass_scalar, ids)
        self.n = max(self.n, int(offset) + int(pos.shape[0]))

    def set_count(self, n):
        sidm_set_count(self.handle, n)
        self.n = int(n)

    def move_particles(self, src, dst, count):
        """Moves particles [src, src + count) to [dst, dst + count)."""
        sidm_move_particles(self.handle, src, dst, count)

    def read_velocities(self, offset, count, out=None):
        """Velocities of particles [offset, offset + count) (numpy unless a
        device tensor `out` is given)."""
        v = np.empty((int(count), 3)) if out is None else out
        sidm_read_particles(self.handle, offset, count, v)
        return v

    def set_velocities(self, vel):
        if isinstance(vel, np.ndarray):
            vel = np.ascontiguousarray(vel, np.float64)
        sidm_set_velocities(self.handle, vel)

    def set_positions(self, pos):
        """New positions of the loaded particles (masses, ids, h and limits kept)."""
        if isinstance(pos, np.ndarray):
            pos = np.ascontiguousarray(pos, np.float64)
            self._keep = (pos,) + tuple(self._keep[1:])
        sidm_set_positions(self.handle, pos)

    def step(self, dt_max, active=None, bins=None, sigma0=1.0, sigma_kind=SIGMA_CONST, w=1.0,
             seed=0, stats=True, inelastic=0.0):
        if isinstance(active, np.ndarray):
            active = np.ascontiguousarray(active, np.uint8)
        if isinstance(bins, np.ndarray):
            bins = np.ascontiguousarray(bins, np.int8)
        sg = SigmaModel(int(sigma_kind), float(sigma0), float(w), float(inelastic))
        st = StepStats() if stats else None
        status = sidm_step(self.handle, active, bins, dt_max, sg, seed, st)
        if st is not None:
            d = st.as_dict()
            d["return"] = status
            return d
        return status

    def set_haloes(self, offsets):
        """Segments the loaded particles into independent haloes:
        halo k = particles [offsets[k], offsets[k+1])."""
        sidm_set_haloes(self.handle, offsets)

    def step_haloes(self, params, active=None, bins=None, stats=True):
        """One step of every halo; params: list of HaloParams or dicts with
        dt_max, sigma0, sigma_kind, w, seed, step."""
        if isinstance(active, np.ndarray):
            active = np.ascontiguousarray(active, np.uint8)
        if isinstance(bins, np.ndarray):
            bins = np.ascontiguousarray(bins, np.int8)
        hp = [p if isinstance(p, HaloParams) else
              HaloParams(float(p["dt_max"]), SigmaModel(int(p.get("sigma_kind", 0)),
                                                          float(p.get("sigma0", 1.0)),
                                                          float(p.get("w", 1.0)),
                                                          float(p.get("inelastic", 0.0))),
                         int(p.get("seed", 0)), int(p.get("step", 0))) for p in params]
        st = StepStats() if stats else None
        status = sidm_step_haloes(self.handle, active, bins, hp, st)
        if st is not None:
            d = st.as_dict()
            d["return"] = status
            return d
        return status

    def sync(self):
        return sidm_sync(self.handle)

    @property
    def tuning(self) -> dict:
        return sidm_get_tuning(self.handle).as_dict()

    def set_tuning(self, **kw):
        t = sidm_get_tuning(self.handle)
        for k, v in kw.items():
            setattr(t, k, int(v))
        sidm_set_tuning(self.handle, t)

    def autotune(self, params, active=None, bins=None, reps=3) -> dict:
        """Times launch shapes on the next step (params: one HaloParams per
        halo) and keeps the fastest; the simulation state is left unchanged."""
        if isinstance(active, np.ndarray):
            active = np.ascontiguousarray(active, np.uint8)
        if isinstance(bins, np.ndarray):
            bins = np.ascontiguousarray(bins, np.int8)
        return sidm_autotune(self.handle, active, bins, params, reps).as_dict()

    def set_overlap_table(self, table):
        """ghat table of the kernel-overlap estimator ((na + 1) x (ns + 1))."""
        sidm_set_overlap_table(self.handle, table)

    def set_sigma_table(self, v, sigma_over_m):
        """Tabulated sigma/m(v) for models of kind SIGMA_TABLE (linear in log v
        between nodes, held at the ends)."""
        sidm_set_sigma_table(self.handle, v, sigma_over_m)

    @property
    def graph_state(self) -> int:
        return sidm_graph_state(self.handle)

    def set_velocity_mirror(self, host_vel):
        """Pinned host (n, 3) array the device keeps current with every
        velocity a step changes (None: stop); the context holds a reference."""
        sidm_set_velocity_mirror(self.handle, host_vel)
        self._mirror = host_vel

    def changed(self):
        """(indices, velocities) of the particles the last step changed."""
        idx = np.empty(self.n, np.int32)
        vel = np.empty((self.n, 3))
        k = sidm_get_changed(self.handle, idx, vel)
        return idx[:k].copy(), vel[:k].copy()

    def velocities(self):
        v = np.empty((self.n, 3))
        h = np.empty(self.n)
        sidm_get_particles(self.handle, v, h)
        return v, h

    def timestep_limits(self):
        out = np.empty(self.n)
        sidm_timestep_limits(self.handle, out)
        return out

    def pairs(self, cap=None):
        cap = (4 * self.n + 16) if cap is None else int(cap)
        ab = np.zeros((cap, 2), np.uint32)
        ords = np.zeros(cap, np.uint64)
        n = sidm_get_pairs(self.handle, ab, ords, cap)
        k = min(n, cap)
        return ab[:k].copy(), ords[:k].copy()

    def phase_times(self) -> dict:
        return dict(zip(PHASES, sidm_phase_times(self.handle)))

    @property
    def kernel_launches(self) -> int:
        return sidm_kernel_launches(self.handle)

    @property
    def step_counter(self) -> int:
        return sidm_get_step(self.handle)

    @step_counter.setter
    def step_counter(self, v: int):
        sidm_set_step(self.handle, v)
