"""FP64 CPU oracle of the DEM timestep -- TEST INFRASTRUCTURE ONLY.

Only `tests/`, `__graft_entry__.smoke()` and `bench.py`'s CPU-baseline / reference arm
import this package. It shares no code with the CUDA library (`paper_1301_1714_gb300`)
and never imports it; both receive the same seeded arrays from
`paper_1301_1714_gb300.scenes`.

The arithmetic lives in `dem_oracle.c` (plain C, FP64, no FMA contraction); this module
compiles it with gcc and marshals numpy arrays. A parameter object is anything with
the attributes of `scenes.Params` (model, stiffness, precision, dt, rho, g, kn, kt, cn,
ct, alpha, mu, ksp, kda, ksh, cell_size, domain_lo, domain_hi, walls).
"""
from __future__ import annotations

import contextlib
import ctypes
import math
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dem_oracle.c")
_SO = os.path.join(_HERE, "liboracle.so")
_lib = None

WALL_BASE = 0xFFFFFF00

HIST_DTYPE = np.dtype([("i", np.uint32), ("j", np.uint32), ("d", np.float64, (3,))])


class _Params(ctypes.Structure):
    _fields_ = [("model", ctypes.c_int32), ("stiffness", ctypes.c_int32), ("hash_mode", ctypes.c_int32),
                ("pad", ctypes.c_int32), ("dt", ctypes.c_double), ("rho", ctypes.c_double),
                ("g", ctypes.c_double * 3), ("kn", ctypes.c_double), ("kt", ctypes.c_double),
                ("cn", ctypes.c_double), ("ct", ctypes.c_double), ("alpha", ctypes.c_double),
                ("mu", ctypes.c_double), ("ksp", ctypes.c_double), ("kda", ctypes.c_double),
                ("ksh", ctypes.c_double), ("origin", ctypes.c_double * 3), ("h", ctypes.c_double),
                ("dims", ctypes.c_int64 * 3), ("terms", ctypes.c_int32), ("pad2", ctypes.c_int32),
                ("mu_roll", ctypes.c_double), ("alpha_t", ctypes.c_double), ("k_coh", ctypes.c_double)]


class _Wall(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("pad", ctypes.c_int32), ("p", ctypes.c_double * 3),
                ("n", ctypes.c_double * 3), ("radius", ctypes.c_double), ("omega", ctypes.c_double * 3),
                ("vel", ctypes.c_double * 3), ("u", ctypes.c_double * 3)]


def build(force: bool = False) -> str:
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
                               "-fno-fast-math", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def _load(path):
    """The oracle's C library at `path`, with its argument types declared."""
    lib = ctypes.CDLL(path)
    P = ctypes.c_void_p
    I64 = ctypes.c_int64
    lib.orc_cell_keys.argtypes = [P, I64, P, P, P]
    lib.orc_cell_keys.restype = None
    lib.orc_sort_by_cell.argtypes = [I64, P, P, P]
    lib.orc_sort_by_cell.restype = ctypes.c_int
    lib.orc_cell_start.argtypes = [I64, P, I64, P]
    lib.orc_cell_start.restype = None
    lib.orc_pairs_brute.argtypes = [I64, P, P, I64, P]
    lib.orc_pairs_brute.restype = I64
    lib.orc_pairs_grid.argtypes = [P, I64, P, P, I64, P, P]
    lib.orc_pairs_grid.restype = I64
    lib.orc_forces.argtypes = [P, ctypes.c_int32, P, I64, P, P, P, P, P, I64, ctypes.c_int32, P, P, P, I64, P]
    lib.orc_forces.restype = I64
    lib.orc_run.argtypes = [P, ctypes.c_int32, P, I64, P, P, P, P, P, P, I64, ctypes.c_int32, I64, P, P, P]
    lib.orc_run.restype = ctypes.c_int
    lib.orc_diagnostics.argtypes = [P, I64, P, P, P, P, P]
    lib.orc_diagnostics.restype = None
    lib.orc_struct_sizes.argtypes = [P]
    lib.orc_struct_sizes.restype = None
    return lib


def _L():
    global _lib
    if _lib is None:
        build()
        _lib = _load(_SO)
    return _lib


@contextlib.contextmanager
def variant(source_text, workdir):
    """Within the block, every oracle call runs a copy of the oracle compiled from
    `source_text` (a mutated `dem_oracle.c`) in `workdir`. The mutation tests use it to
    show that a pin fails when a named mistake is planted in the oracle."""
    global _lib
    src = os.path.join(str(workdir), "dem_oracle_variant.c")
    so = os.path.join(str(workdir), "liboracle_variant.so")
    with open(src, "w") as f:
        f.write(source_text)
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
                           "-fno-fast-math", "-o", so, src, "-lm"])
    saved = _L()
    _lib = _load(so)
    try:
        yield
    finally:
        _lib = saved


def source():
    """Text of the oracle's C source."""
    with open(_SRC) as f:
        return f.read()


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def struct_sizes_match():
    """True if the C records have the sizes of their ctypes mirrors."""
    out = np.zeros(2, dtype=np.int64)
    _L().orc_struct_sizes(_ptr(out))
    return int(out[0]) == ctypes.sizeof(_Params) and int(out[1]) == ctypes.sizeof(_Wall)


def grid_dims(params):
    lo, hi, h = params.domain_lo, params.domain_hi, params.cell_size
    return tuple(max(1, int(math.ceil((hi[a] - lo[a]) / h))) for a in range(3))


def make_params(params) -> _Params:
    c = _Params()
    c.model = {"practical": 0, "simple": 1}[params.model]
    c.stiffness = {"linear": 0, "hertz": 1}[params.stiffness]
    c.hash_mode = {"fp64": 0, "fp32": 1}[params.precision]
    c.dt = params.dt
    c.rho = params.rho
    for a in range(3):
        c.g[a] = params.g[a]
        c.origin[a] = params.domain_lo[a]
    c.kn, c.kt, c.cn, c.ct, c.alpha, c.mu = params.kn, params.kt, params.cn, params.ct, params.alpha, params.mu
    c.ksp, c.kda, c.ksh = params.ksp, params.kda, params.ksh
    c.h = params.cell_size
    d = grid_dims(params)
    for a in range(3):
        c.dims[a] = d[a]
    c.terms = int(getattr(params, "terms", 0))
    c.mu_roll = float(getattr(params, "mu_roll", 0.0))
    c.alpha_t = float(getattr(params, "alpha_t", 0.0))
    c.k_coh = float(getattr(params, "k_coh", 0.0))
    return c


def make_walls(walls):
    arr = (_Wall * max(1, len(walls)))()
    for k, w in enumerate(walls):
        arr[k].kind = {"plane": 0, "cylinder": 1, "half_plate": 2}[w["kind"]]
        for a in range(3):
            arr[k].p[a] = w["p"][a]
            arr[k].n[a] = w["n"][a]
            arr[k].u[a] = w.get("u", (0, 0, 0))[a]
            arr[k].omega[a] = w.get("omega", (0, 0, 0))[a]
            arr[k].vel[a] = w.get("vel", (0, 0, 0))[a]
        arr[k].radius = w.get("radius", 0.0)
    return arr


def _x(a):
    return np.ascontiguousarray(a, dtype=np.float64).reshape(-1, 3)


def _r(a):
    return np.ascontiguousarray(a, dtype=np.float32).reshape(-1)


# ------------------------------------------------------------------ broad phase
def cell_keys(params, x):
    """Cell key CM[j] and cell triple of every particle (Sec. 4.2 step 2)."""
    x = _x(x)
    n = len(x)
    ijk = np.zeros((n, 3), dtype=np.int64)
    key = np.zeros(n, dtype=np.uint64)
    c = make_params(params)
    _L().orc_cell_keys(ctypes.byref(c), n, _ptr(x), _ptr(ijk), _ptr(key))
    return key, ijk


def sort_by_cell(key):
    """SCCM (ids in (cell, id) order) and SCM (Eq. 11)."""
    key = np.ascontiguousarray(key, dtype=np.uint64)
    n = len(key)
    order = np.zeros(n, dtype=np.uint32)
    skey = np.zeros(n, dtype=np.uint64)
    if _L().orc_sort_by_cell(n, _ptr(key), _ptr(order), _ptr(skey)) != 0:
        raise MemoryError
    return order, skey


def cell_start(sorted_key, ncells):
    sorted_key = np.ascontiguousarray(sorted_key, dtype=np.uint64)
    start = np.zeros(ncells + 1, dtype=np.int64)
    _L().orc_cell_start(len(sorted_key), _ptr(sorted_key), ncells, _ptr(start))
    return start


def pairs_brute(x, r):
    """All contact pairs (i < j), O(N^2)."""
    x, r = _x(x), _r(r)
    cap = max(16, 8 * len(r))
    while True:
        out = np.zeros((cap, 2), dtype=np.uint32)
        np_ = _L().orc_pairs_brute(len(r), _ptr(x), _ptr(r), cap, _ptr(out))
        if np_ <= cap:
            return out[:np_].copy()
        cap = int(np_)


def pairs_grid(params, x, r, with_candidates=False):
    """Contact pairs found through the cell grid (Eq. 12); optionally per-particle
    candidate counts."""
    x, r = _x(x), _r(r)
    c = make_params(params)
    cap = max(16, 8 * len(r))
    while True:
        out = np.zeros((cap, 2), dtype=np.uint32)
        ncand = np.zeros(len(r), dtype=np.int64)
        np_ = _L().orc_pairs_grid(ctypes.byref(c), len(r), _ptr(x), _ptr(r), cap, _ptr(out), _ptr(ncand))
        if np_ < 0:
            raise MemoryError
        if np_ <= cap:
            return (out[:np_].copy(), ncand) if with_candidates else out[:np_].copy()
        cap = int(np_)


# ------------------------------------------------------------------ forces / run
def empty_history(cap=0):
    return np.zeros(cap, dtype=HIST_DTYPE)


def forces(params, x, v, w, r, hist=None, pair_mode="auto"):
    """Force and torque on every particle at the given state (gravity included) and the
    tangential springs of this step's contacts. Returns (F, T, new_hist, stats)."""
    x, v, w, r = _x(x), _x(v), _x(w), _r(r)
    n = len(r)
    if hist is None:
        hist = empty_history()
    hist = np.ascontiguousarray(hist, dtype=HIST_DTYPE)
    pm = (0 if n <= 4096 else 1) if pair_mode == "auto" else {"brute": 0, "grid": 1}[pair_mode]
    c = make_params(params)
    wl = make_walls(params.walls)
    cap = 16 * n + 64
    F = np.zeros((n, 3)); T = np.zeros((n, 3))
    stats = np.zeros(4)
    while True:
        hout = np.zeros(cap, dtype=HIST_DTYPE)
        k = _L().orc_forces(ctypes.byref(c), len(params.walls), wl, n, _ptr(x), _ptr(v), _ptr(w), _ptr(r),
                            _ptr(hist), len(hist), pm, _ptr(F), _ptr(T), _ptr(hout), cap, _ptr(stats))
        if k == -2:
            cap *= 2
            continue
        if k < 0:
            raise MemoryError
        return F, T, hout[:k].copy(), stats


class State:
    """A mutable oracle run: arrays in global-id order plus the tangential history."""

    def __init__(self, params, x, v, w, r, hist=None):
        self.params = params
        self.x = _x(x).copy(); self.v = _x(v).copy(); self.w = _x(w).copy(); self.r = _r(r).copy()
        n = len(self.r)
        self.cap = 16 * n + 64
        self.hist = np.zeros(self.cap, dtype=HIST_DTYPE)
        self.nh = 0
        if hist is not None and len(hist):
            self.hist[:len(hist)] = hist
            self.nh = len(hist)
        self.F = np.zeros((n, 3)); self.T = np.zeros((n, 3))
        self.stats = np.zeros(4)

    @property
    def history(self):
        return self.hist[:self.nh].copy()

    def run(self, nsteps, pair_mode="auto"):
        n = len(self.r)
        pm = (0 if n <= 4096 else 1) if pair_mode == "auto" else {"brute": 0, "grid": 1}[pair_mode]
        c = make_params(self.params)
        wl = make_walls(self.params.walls)
        nh = ctypes.c_int64(self.nh)
        rc = _L().orc_run(ctypes.byref(c), len(self.params.walls), wl, n, _ptr(self.x), _ptr(self.v), _ptr(self.w),
                          _ptr(self.r), _ptr(self.hist), ctypes.byref(nh), self.cap, pm, nsteps, _ptr(self.F),
                          _ptr(self.T), _ptr(self.stats))
        if rc != 0:
            raise RuntimeError(f"orc_run failed ({rc})")
        self.nh = int(nh.value)
        return self


def diagnostics(params, x, v, w, r):
    """[KE_trans, KE_rot, P(3), L(3), PE_grav, total mass]."""
    x, v, w, r = _x(x), _x(v), _x(w), _r(r)
    out = np.zeros(10)
    c = make_params(params)
    _L().orc_diagnostics(ctypes.byref(c), len(r), _ptr(x), _ptr(v), _ptr(w), _ptr(r), _ptr(out))
    return out
