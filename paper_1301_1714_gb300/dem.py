"""Python binding of the C ABI in include/dem.h (libdemgb.so), same function names.

Argument marshalling only: every step of the timestep runs in the CUDA library. Host
arrays are numpy; device arrays are torch CUDA tensors (PyTorch supplies device memory
and streams). If the library has not been built or cannot be loaded, `lib()` raises:
there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import _build

DEM_OK = 0
DEM_ERR = {1: "DEM_ERR_INVALID_ARG", 2: "DEM_ERR_OOM", 3: "DEM_ERR_CUDA", 4: "DEM_ERR_CAPACITY",
           5: "DEM_ERR_TIMEOUT", 6: "DEM_ERR_NONFINITE", 7: "DEM_ERR_STATE"}
(DEM_ERR_INVALID_ARG, DEM_ERR_OOM, DEM_ERR_CUDA, DEM_ERR_CAPACITY, DEM_ERR_TIMEOUT, DEM_ERR_NONFINITE,
 DEM_ERR_STATE) = range(1, 8)
DEM_PRACTICAL, DEM_SIMPLE = 0, 1
DEM_LINEAR, DEM_HERTZ = 0, 1
DEM_FP64, DEM_FP32 = 0, 1
DEM_HOST, DEM_DEVICE = 0, 1
DEM_PLANE, DEM_CYLINDER_IN, DEM_HALF_PLATE = 0, 1, 2
DEM_TERM_NO_ATTRACTION, DEM_TERM_ROLLING, DEM_TERM_ETA_T, DEM_TERM_COHESION = 1, 2, 4, 8
WALL_BASE = 0xFFFFFF00

_D3 = ctypes.c_double * 3


class dem_config(ctypes.Structure):
    _fields_ = [("model", ctypes.c_int32), ("stiffness", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("resort_interval", ctypes.c_int32), ("dt", ctypes.c_double), ("rho", ctypes.c_double),
                ("g", _D3), ("kn", ctypes.c_double), ("kt", ctypes.c_double), ("cn", ctypes.c_double),
                ("ct", ctypes.c_double), ("alpha", ctypes.c_double), ("mu", ctypes.c_double),
                ("ksp", ctypes.c_double), ("kda", ctypes.c_double), ("ksh", ctypes.c_double),
                ("skin", ctypes.c_double), ("cell_size", ctypes.c_double), ("domain_lo", _D3), ("domain_hi", _D3),
                ("block_size", ctypes.c_int32), ("max_contacts", ctypes.c_int32), ("terms", ctypes.c_int32),
                ("pad", ctypes.c_int32), ("mu_roll", ctypes.c_double), ("alpha_t", ctypes.c_double),
                ("k_coh", ctypes.c_double)]


class dem_wall(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("pad", ctypes.c_int32), ("p", _D3), ("n", _D3), ("radius", ctypes.c_double),
                ("omega", _D3), ("vel", _D3), ("u", _D3)]


class DemError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{DEM_ERR.get(status, status)}: {message}")
        self.status = status


_lib = None
_EXPORTS = ["dem_create", "dem_set_particles", "dem_set_walls", "dem_step", "dem_run_until", "dem_get_state", "dem_get_forces",
            "dem_get_history", "dem_restore", "dem_get_diagnostics", "dem_debug_snapshot", "dem_get_grid",
            "dem_device_bytes", "dem_max_contacts_seen", "dem_launch_count", "dem_last_error", "dem_destroy",
            "dem_set_timing",
            "dem_get_phase_times", "dem_sort_cells_static", "dem_batch_create", "dem_batch_add", "dem_batch_run",
            "dem_batch_get_state", "dem_batch_remove", "dem_batch_info", "dem_batch_device_bytes",
            "dem_batch_launch_count", "dem_batch_last_error", "dem_batch_destroy", "dem_slab_bounds",
            "dem_slabs_create", "dem_slabs_set_walls", "dem_slabs_set_particles", "dem_slabs_step",
            "dem_slabs_get_state", "dem_slabs_info", "dem_slabs_launch_count", "dem_slabs_last_error",
            "dem_slabs_destroy"]
DEM_MAX_SLABS = 8


def lib_path() -> str:
    return _build.LIB


def lib():
    """Load libdemgb.so (built by `paper_1301_1714_gb300._build.build()`)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build the CUDA library first (python -c 'import __graft_entry__ as g; g.build()')")
    L = ctypes.CDLL(path)
    P, I64, I32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
    L.dem_create.argtypes = [ctypes.POINTER(dem_config), I32, P, ctypes.POINTER(P)]
    L.dem_set_particles.argtypes = [P, I64, P, P, P, P, P, I32]
    L.dem_set_walls.argtypes = [P, I32, P]
    L.dem_step.argtypes = [P, I64]
    L.dem_run_until.argtypes = [P, I64, ctypes.c_double, I64, ctypes.POINTER(I64), ctypes.POINTER(ctypes.c_double),
                                ctypes.POINTER(I32)]
    L.dem_get_state.argtypes = [P, P, P, P, I32]
    L.dem_get_forces.argtypes = [P, P, P, I32]
    L.dem_get_history.argtypes = [P, I64, P, P, P, ctypes.POINTER(I64)]
    L.dem_restore.argtypes = [P, I64, P, P, P, P, I64, P, P, P]
    L.dem_get_diagnostics.argtypes = [P, P]
    L.dem_debug_snapshot.argtypes = [P, P, P, I64, P, ctypes.POINTER(I64)]
    L.dem_get_grid.argtypes = [P, P, P, P]
    L.dem_sort_cells_static.argtypes = [I64, P, P, ctypes.c_double, P, P, P, P, P]
    L.dem_batch_create.argtypes = [I32, I32, I32, I32, I32, I32, P, ctypes.POINTER(P)]
    L.dem_batch_add.argtypes = [P, ctypes.POINTER(dem_config), I32, P, I64, P, P, P, P, I64, ctypes.POINTER(I32)]
    L.dem_batch_run.argtypes = [P, I64, P, I32, ctypes.POINTER(I32)]
    L.dem_batch_get_state.argtypes = [P, I32, P, P, P, I32]
    L.dem_batch_remove.argtypes = [P, I32]
    L.dem_batch_info.argtypes = [P, I32, ctypes.POINTER(I64), ctypes.POINTER(I64), ctypes.POINTER(I64)]
    L.dem_batch_device_bytes.argtypes = [P]
    L.dem_batch_device_bytes.restype = I64
    L.dem_batch_launch_count.argtypes = [P]
    L.dem_batch_launch_count.restype = I64
    L.dem_batch_last_error.argtypes = [P]
    L.dem_batch_last_error.restype = ctypes.c_char_p
    L.dem_batch_destroy.argtypes = [P]
    L.dem_batch_destroy.restype = None
    L.dem_slab_bounds.argtypes = [I64, P, I32, P]
    L.dem_slabs_create.argtypes = [ctypes.POINTER(dem_config), I32, I32, I32, P, ctypes.POINTER(P)]
    L.dem_slabs_set_walls.argtypes = [P, I32, P]
    L.dem_slabs_set_particles.argtypes = [P, I64, P, P, P, P, I32]
    L.dem_slabs_step.argtypes = [P, I64]
    L.dem_slabs_get_state.argtypes = [P, P, P, P, I32]
    L.dem_slabs_info.argtypes = [P, P, P, P, ctypes.POINTER(I64), ctypes.POINTER(I64)]
    L.dem_slabs_launch_count.argtypes = [P]
    L.dem_slabs_launch_count.restype = I64
    L.dem_slabs_last_error.argtypes = [P]
    L.dem_slabs_last_error.restype = ctypes.c_char_p
    L.dem_slabs_destroy.argtypes = [P]
    L.dem_slabs_destroy.restype = None
    L.dem_set_timing.argtypes = [P, I32]
    L.dem_get_phase_times.argtypes = [P, P]
    L.dem_device_bytes.argtypes = [P]
    L.dem_device_bytes.restype = I64
    L.dem_max_contacts_seen.argtypes = [P]
    L.dem_max_contacts_seen.restype = I64
    L.dem_launch_count.argtypes = [P]
    L.dem_launch_count.restype = I64
    L.dem_last_error.argtypes = [P]
    L.dem_last_error.restype = ctypes.c_char_p
    L.dem_destroy.argtypes = [P]
    L.dem_destroy.restype = None
    for name in _EXPORTS:
        f = getattr(L, name)
        if f.restype is ctypes.c_int or name in ("dem_create", "dem_set_particles", "dem_set_walls", "dem_step",
                                                  "dem_run_until",
                                                  "dem_get_state", "dem_get_forces", "dem_get_history", "dem_restore",
                                                  "dem_get_diagnostics", "dem_debug_snapshot", "dem_get_grid",
                                                  "dem_set_timing", "dem_get_phase_times",
                                                  "dem_sort_cells_static", "dem_batch_create", "dem_batch_add",
                                                  "dem_batch_run", "dem_batch_get_state", "dem_batch_remove",
                                                  "dem_batch_info", "dem_slab_bounds", "dem_slabs_create",
                                                  "dem_slabs_set_walls", "dem_slabs_set_particles", "dem_slabs_step",
                                                  "dem_slabs_get_state", "dem_slabs_info"):
            f.restype = ctypes.c_int
    _lib = L
    return L


def _check(h, status):
    if status != DEM_OK:
        msg = lib().dem_last_error(h).decode() if h else ""
        raise DemError(status, msg)


# ------------------------------------------------------------------ marshalling
def _host(a, dtype, shape):
    a = np.ascontiguousarray(a, dtype=dtype)
    if a.size != int(np.prod(shape)):
        raise ValueError(f"expected {shape} elements of {dtype}, got {a.shape}")
    return a


def _ptr(a):
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return a.ctypes.data_as(ctypes.c_void_p)
    return ctypes.c_void_p(a.data_ptr())


def _is_device(a):
    return a is not None and not isinstance(a, np.ndarray) and hasattr(a, "is_cuda") and a.is_cuda


def config_from_params(p, block_size=0, max_contacts=0) -> dem_config:
    """dem_config from a `scenes.Params`-like object."""
    c = dem_config()
    c.model = {"practical": DEM_PRACTICAL, "simple": DEM_SIMPLE}[p.model]
    c.stiffness = {"linear": DEM_LINEAR, "hertz": DEM_HERTZ}[p.stiffness]
    c.precision = {"fp64": DEM_FP64, "fp32": DEM_FP32}[p.precision]
    c.resort_interval = int(getattr(p, "resort_interval", 1))
    c.dt, c.rho = p.dt, p.rho
    for a in range(3):
        c.g[a] = p.g[a]
        c.domain_lo[a] = p.domain_lo[a]
        c.domain_hi[a] = p.domain_hi[a]
    c.kn, c.kt, c.cn, c.ct, c.alpha, c.mu = p.kn, p.kt, p.cn, p.ct, p.alpha, p.mu
    c.ksp, c.kda, c.ksh = p.ksp, p.kda, p.ksh
    c.skin = getattr(p, "skin", 0.0)
    c.cell_size = p.cell_size
    c.block_size = block_size
    c.max_contacts = max_contacts
    c.terms = int(getattr(p, "terms", 0))
    c.mu_roll = float(getattr(p, "mu_roll", 0.0))
    c.alpha_t = float(getattr(p, "alpha_t", 0.0))
    c.k_coh = float(getattr(p, "k_coh", 0.0))
    return c


def walls_array(walls):
    arr = (dem_wall * max(1, len(walls)))()
    for k, w in enumerate(walls):
        arr[k].kind = {"plane": DEM_PLANE, "cylinder": DEM_CYLINDER_IN, "half_plate": DEM_HALF_PLATE}[w["kind"]]
        for a in range(3):
            arr[k].p[a] = w["p"][a]
            arr[k].n[a] = w["n"][a]
            arr[k].omega[a] = w.get("omega", (0, 0, 0))[a]
            arr[k].vel[a] = w.get("vel", (0, 0, 0))[a]
            arr[k].u[a] = w.get("u", (0, 0, 0))[a]
        arr[k].radius = w.get("radius", 0.0)
    return arr


# ------------------------------------------------------------------ the C ABI, 1:1
def dem_create(config, device=0, cuda_stream=None):
    c = config if isinstance(config, dem_config) else config_from_params(config)
    h = ctypes.c_void_p()
    st = lib().dem_create(ctypes.byref(c), device, ctypes.c_void_p(cuda_stream) if cuda_stream else None,
                          ctypes.byref(h))
    if st != DEM_OK:
        raise DemError(st, "dem_create rejected the configuration or device")
    return h


def dem_set_particles(h, x, v, w, r):
    n = len(r)
    if _is_device(r):
        for t, dt in ((x, "torch.float64"), (v, "torch.float64"), (w, "torch.float64"), (r, "torch.float32")):
            if not (_is_device(t) and str(t.dtype) == dt and t.is_contiguous()):
                raise ValueError("device inputs must be contiguous CUDA tensors (x, v, w float64; r float32)")
        _check(h, lib().dem_set_particles(h, n, None, _ptr(x), _ptr(v), _ptr(w), _ptr(r), DEM_DEVICE))
        return
    x = _host(x, np.float64, (n, 3)); v = _host(v, np.float64, (n, 3)); w = _host(w, np.float64, (n, 3))
    r = _host(r, np.float32, (n,))
    _check(h, lib().dem_set_particles(h, n, None, _ptr(x), _ptr(v), _ptr(w), _ptr(r), DEM_HOST))


def dem_set_walls(h, walls):
    arr = walls_array(walls)
    _check(h, lib().dem_set_walls(h, len(walls), arr))


def dem_step(h, nsteps=1):
    _check(h, lib().dem_step(h, int(nsteps)))


def dem_run_until(h, max_steps, disp_threshold, check_every=100):
    """Steps until max |v'| dt of the last step of a chunk is below disp_threshold.
    Returns (steps_done, last_max_disp, settled)."""
    done = ctypes.c_int64(0)
    disp = ctypes.c_double(0.0)
    ok = ctypes.c_int(0)
    _check(h, lib().dem_run_until(h, int(max_steps), float(disp_threshold), int(check_every), ctypes.byref(done),
                                  ctypes.byref(disp), ctypes.byref(ok)))
    return int(done.value), float(disp.value), bool(ok.value)


def dem_get_state(h, n, x=None, v=None, w=None):
    """Host: returns (x, v, w) numpy (n, 3) arrays. Device: pass CUDA tensors to fill."""
    if _is_device(x) or _is_device(v) or _is_device(w):
        _check(h, lib().dem_get_state(h, _ptr(x), _ptr(v), _ptr(w), DEM_DEVICE))
        return x, v, w
    x = np.zeros((n, 3)); v = np.zeros((n, 3)); w = np.zeros((n, 3))
    _check(h, lib().dem_get_state(h, _ptr(x), _ptr(v), _ptr(w), DEM_HOST))
    return x, v, w


def dem_get_forces(h, n, F=None, T=None):
    if _is_device(F) or _is_device(T):
        _check(h, lib().dem_get_forces(h, _ptr(F), _ptr(T), DEM_DEVICE))
        return F, T
    F = np.zeros((n, 3)); T = np.zeros((n, 3))
    _check(h, lib().dem_get_forces(h, _ptr(F), _ptr(T), DEM_HOST))
    return F, T


HIST_DTYPE = np.dtype([("i", np.uint32), ("j", np.uint32), ("d", np.float64, (3,))])


def dem_get_history(h):
    """Stored tangential springs as a structured array (i, j, d[3]), sorted by (i, j)."""
    cnt = ctypes.c_int64(0)
    _check(h, lib().dem_get_history(h, 0, None, None, None, ctypes.byref(cnt)))
    m = cnt.value
    i = np.zeros(m, np.uint32); j = np.zeros(m, np.uint32); d = np.zeros((m, 3))
    _check(h, lib().dem_get_history(h, m, _ptr(i), _ptr(j), _ptr(d), ctypes.byref(cnt)))
    out = np.zeros(m, dtype=HIST_DTYPE)
    out["i"], out["j"], out["d"] = i, j, d
    return out


def dem_restore(h, x, v, w, r, hist=None):
    n = len(r)
    x = _host(x, np.float64, (n, 3)); v = _host(v, np.float64, (n, 3)); w = _host(w, np.float64, (n, 3))
    r = _host(r, np.float32, (n,))
    if hist is None or len(hist) == 0:
        _check(h, lib().dem_restore(h, n, _ptr(x), _ptr(v), _ptr(w), _ptr(r), 0, None, None, None))
        return
    i = np.ascontiguousarray(hist["i"], np.uint32); j = np.ascontiguousarray(hist["j"], np.uint32)
    d = np.ascontiguousarray(hist["d"], np.float64)
    _check(h, lib().dem_restore(h, n, _ptr(x), _ptr(v), _ptr(w), _ptr(r), len(i), _ptr(i), _ptr(j), _ptr(d)))


DIAG_NAMES = ["ke_trans", "ke_rot", "px", "py", "pz", "lx", "ly", "lz", "pe_grav", "mass", "pair_contacts",
              "wall_contacts", "max_overlap", "steps", "sorts", "clamped"]


def dem_get_diagnostics(h):
    out = np.zeros(16)
    _check(h, lib().dem_get_diagnostics(h, _ptr(out)))
    return out


def dem_debug_snapshot(h, n, with_pairs=True):
    """(cell per id, ids in (cell, id) order, pairs (m, 2) of the last dem_get_forces)."""
    cell = np.zeros(n, np.uint32); order = np.zeros(n, np.uint32)
    if not with_pairs:
        _check(h, lib().dem_debug_snapshot(h, _ptr(cell), _ptr(order), 0, None, None))
        return cell, order, None
    cnt = ctypes.c_int64(0)
    _check(h, lib().dem_debug_snapshot(h, None, None, 0, None, ctypes.byref(cnt)))
    pairs = np.zeros((cnt.value, 2), np.uint32)
    _check(h, lib().dem_debug_snapshot(h, _ptr(cell), _ptr(order), cnt.value, _ptr(pairs), ctypes.byref(cnt)))
    return cell, order, pairs


def dem_get_grid(h):
    o = np.zeros(3); c = np.zeros(1); d = np.zeros(3, np.int64)
    _check(h, lib().dem_get_grid(h, _ptr(o), _ptr(c), _ptr(d)))
    return o, float(c[0]), tuple(int(k) for k in d)


STATIC_SORT_MAX_N = 262144
STATIC_SORT_MAX_CELLS = 1048576


def dem_sort_cells_static(x, origin, cell, dims, cell_of, order, cell_start, cuda_stream=None):
    """Cell map and (cell, id) sort without any device allocation by the library (for
    callers that cannot allocate: see include/dem.h). x: CUDA float64 tensor (n, 3);
    cell_of, order: CUDA int32 tensors (n,); cell_start: CUDA int32 tensor
    (nx*ny*nz + 1,); the int32 buffers receive unsigned 32-bit values."""
    n = int(x.shape[0]) if x is not None else 0
    o = np.ascontiguousarray(origin, dtype=np.float64)
    d = np.ascontiguousarray(dims, dtype=np.int64)
    st = lib().dem_sort_cells_static(n, _ptr(x), _ptr(o), float(cell), _ptr(d), _ptr(cell_of), _ptr(order),
                                     _ptr(cell_start), ctypes.c_void_p(cuda_stream) if cuda_stream else None)
    if st != DEM_OK:
        raise DemError(st, "dem_sort_cells_static: sizes above the static maximum, bad arguments or a CUDA error")


def dem_set_timing(h, enable=True):
    _check(h, lib().dem_set_timing(h, 1 if enable else 0))


def dem_get_phase_times(h):
    """(force-pass ms, sort ms, force passes timed, sorts timed) since timing was enabled."""
    out = np.zeros(4)
    _check(h, lib().dem_get_phase_times(h, _ptr(out)))
    return out


def dem_device_bytes(h):
    return int(lib().dem_device_bytes(h))


def dem_max_contacts_seen(h):
    return int(lib().dem_max_contacts_seen(h))


def dem_launch_count(h):
    return int(lib().dem_launch_count(h))


def dem_last_error(h):
    return lib().dem_last_error(h).decode()


def dem_destroy(h):
    if h:
        lib().dem_destroy(h)


# ------------------------------------------------------------------ convenience
class Simulation:
    """A handle plus its particle count (marshalling only)."""

    def __init__(self, params, x, v, w, r, device=0, cuda_stream=None, block_size=0, max_contacts=0):
        self.params = params
        self.n = len(r)
        self.h = dem_create(config_from_params(params, block_size, max_contacts), device, cuda_stream)
        try:
            dem_set_walls(self.h, params.walls)
            dem_set_particles(self.h, x, v, w, r)
        except Exception:
            dem_destroy(self.h)
            self.h = None
            raise

    def step(self, nsteps=1):
        dem_step(self.h, nsteps)
        return self

    def state(self):
        return dem_get_state(self.h, self.n)

    def forces(self):
        return dem_get_forces(self.h, self.n)

    def history(self):
        return dem_get_history(self.h)

    def diagnostics(self):
        return dict(zip(DIAG_NAMES, dem_get_diagnostics(self.h)))

    def snapshot(self, with_pairs=True):
        return dem_debug_snapshot(self.h, self.n, with_pairs)

    def close(self):
        if self.h:
            dem_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------------ batches
def _bcheck(b, status):
    if status != DEM_OK:
        msg = lib().dem_batch_last_error(b).decode() if b else ""
        raise DemError(status, msg)


def dem_batch_create(precision="fp32", model="practical", stiffness="linear", max_contacts=0, block_size=0, device=0,
                     cuda_stream=None):
    b = ctypes.c_void_p()
    st = lib().dem_batch_create({"fp64": DEM_FP64, "fp32": DEM_FP32}[precision],
                                {"practical": DEM_PRACTICAL, "simple": DEM_SIMPLE}[model],
                                {"linear": DEM_LINEAR, "hertz": DEM_HERTZ}[stiffness], max_contacts, block_size, device,
                                ctypes.c_void_p(cuda_stream) if cuda_stream else None, ctypes.byref(b))
    if st != DEM_OK:
        raise DemError(st, "dem_batch_create rejected its arguments")
    return b


def dem_batch_add(b, params, x, v, w, r, step_budget):
    n = len(r)
    x = _host(x, np.float64, (n, 3)); v = _host(v, np.float64, (n, 3)); w = _host(w, np.float64, (n, 3))
    r = _host(r, np.float32, (n,))
    c = config_from_params(params)
    walls = walls_array(params.walls)
    slot = ctypes.c_int32(-1)
    _bcheck(b, lib().dem_batch_add(b, ctypes.byref(c), len(params.walls), walls, n, _ptr(x), _ptr(v), _ptr(w),
                                   _ptr(r), int(step_budget), ctypes.byref(slot)))
    return slot.value


def dem_batch_run(b, max_steps, cap=4096):
    fin = np.zeros(max(cap, 1), np.int32)
    nf = ctypes.c_int32(0)
    _bcheck(b, lib().dem_batch_run(b, int(max_steps), _ptr(fin), cap, ctypes.byref(nf)))
    return [int(k) for k in fin[:min(nf.value, cap)]]


def dem_batch_get_state(b, slot, n):
    x = np.zeros((n, 3)); v = np.zeros((n, 3)); w = np.zeros((n, 3))
    _bcheck(b, lib().dem_batch_get_state(b, slot, _ptr(x), _ptr(v), _ptr(w), DEM_HOST))
    return x, v, w


def dem_batch_remove(b, slot):
    _bcheck(b, lib().dem_batch_remove(b, slot))


def dem_batch_info(b, slot):
    n, done, budget = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    _bcheck(b, lib().dem_batch_info(b, slot, ctypes.byref(n), ctypes.byref(done), ctypes.byref(budget)))
    return n.value, done.value, budget.value


def dem_batch_device_bytes(b):
    return int(lib().dem_batch_device_bytes(b))


def dem_batch_launch_count(b):
    return int(lib().dem_batch_launch_count(b))


def dem_batch_last_error(b):
    return lib().dem_batch_last_error(b).decode()


def dem_batch_destroy(b):
    if b:
        lib().dem_batch_destroy(b)


# ------------------------------------------------------------------ slabs (sub-domains with halo exchange)
def _scheck(sl, status):
    if status != DEM_OK:
        msg = lib().dem_slabs_last_error(sl).decode() if sl else ""
        raise DemError(status, msg)


def dem_slab_bounds(z, nslabs):
    """Boundaries (nslabs + 1 doubles, -inf .. +inf) splitting the coordinates z into
    nslabs slabs of nearly equal counts (host only)."""
    z = np.ascontiguousarray(z, dtype=np.float64).ravel()
    out = np.zeros(int(nslabs) + 1)
    st = lib().dem_slab_bounds(len(z), _ptr(z), int(nslabs), _ptr(out))
    if st != DEM_OK:
        raise DemError(st, "dem_slab_bounds: nslabs outside [1, 8] or a non-finite coordinate")
    return out


def dem_slabs_create(config, nslabs, axis=-1, device=0, cuda_stream=None):
    c = config if isinstance(config, dem_config) else config_from_params(config)
    sl = ctypes.c_void_p()
    st = lib().dem_slabs_create(ctypes.byref(c), int(nslabs), int(axis), device,
                                ctypes.c_void_p(cuda_stream) if cuda_stream else None, ctypes.byref(sl))
    if st != DEM_OK:
        raise DemError(st, "dem_slabs_create rejected the configuration (resort_interval must be 1), "
                           "the slab count, the axis or the device")
    return sl


def dem_slabs_set_walls(sl, walls):
    arr = walls_array(walls)
    _scheck(sl, lib().dem_slabs_set_walls(sl, len(walls), arr))


def dem_slabs_set_particles(sl, x, v, w, r):
    n = len(r)
    if _is_device(r):
        for t, dt in ((x, "torch.float64"), (v, "torch.float64"), (w, "torch.float64"), (r, "torch.float32")):
            if not (_is_device(t) and str(t.dtype) == dt and t.is_contiguous()):
                raise ValueError("device inputs must be contiguous CUDA tensors (x, v, w float64; r float32)")
        _scheck(sl, lib().dem_slabs_set_particles(sl, n, _ptr(x), _ptr(v), _ptr(w), _ptr(r), DEM_DEVICE))
        return
    x = _host(x, np.float64, (n, 3)); v = _host(v, np.float64, (n, 3)); w = _host(w, np.float64, (n, 3))
    r = _host(r, np.float32, (n,))
    _scheck(sl, lib().dem_slabs_set_particles(sl, n, _ptr(x), _ptr(v), _ptr(w), _ptr(r), DEM_HOST))


def dem_slabs_step(sl, nsteps=1):
    _scheck(sl, lib().dem_slabs_step(sl, int(nsteps)))


def dem_slabs_get_state(sl, n, x=None, v=None, w=None):
    if _is_device(x) or _is_device(v) or _is_device(w):
        _scheck(sl, lib().dem_slabs_get_state(sl, _ptr(x), _ptr(v), _ptr(w), DEM_DEVICE))
        return x, v, w
    x = np.zeros((n, 3)); v = np.zeros((n, 3)); w = np.zeros((n, 3))
    _scheck(sl, lib().dem_slabs_get_state(sl, _ptr(x), _ptr(v), _ptr(w), DEM_HOST))
    return x, v, w


def dem_slabs_info(sl, nslabs):
    """dict: owned and ghosts per slab, boundaries, migrations so far, steps done."""
    owned = np.zeros(nslabs, np.int64); ghosts = np.zeros(nslabs, np.int64); bounds = np.zeros(nslabs + 1)
    mig = ctypes.c_int64(0); steps = ctypes.c_int64(0)
    _scheck(sl, lib().dem_slabs_info(sl, _ptr(owned), _ptr(ghosts), _ptr(bounds), ctypes.byref(mig),
                                     ctypes.byref(steps)))
    return {"owned": owned, "ghosts": ghosts, "bounds": bounds, "migrated": int(mig.value), "steps": int(steps.value)}


def dem_slabs_launch_count(sl):
    return int(lib().dem_slabs_launch_count(sl))


def dem_slabs_last_error(sl):
    return lib().dem_slabs_last_error(sl).decode()


def dem_slabs_destroy(sl):
    if sl:
        lib().dem_slabs_destroy(sl)


class Slabs:
    """One scene as nslabs sub-domains with halo exchange (marshalling only)."""

    def __init__(self, params, x, v, w, r, nslabs, axis=-1, device=0, cuda_stream=None, block_size=0,
                 max_contacts=0):
        self.params = params
        self.n = len(r)
        self.nslabs = int(nslabs)
        self.h = dem_slabs_create(config_from_params(params, block_size, max_contacts), nslabs, axis, device,
                                  cuda_stream)
        try:
            dem_slabs_set_walls(self.h, params.walls)
            dem_slabs_set_particles(self.h, x, v, w, r)
        except Exception:
            dem_slabs_destroy(self.h)
            self.h = None
            raise

    def step(self, nsteps=1):
        dem_slabs_step(self.h, nsteps)
        return self

    def state(self):
        return dem_slabs_get_state(self.h, self.n)

    def info(self):
        return dem_slabs_info(self.h, self.nslabs)

    def close(self):
        if self.h:
            dem_slabs_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
