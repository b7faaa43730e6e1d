"""Seeded synthetic DEM scenes (inputs shared by the CUDA library and the CPU oracle).

Nothing here computes contact forces, cell hashes, sorted orders or time integration;
it produces initial particle arrays, wall lists and the physical parameters of a run.
The paper's benchmark (Sec. 5: 131,072 equal spheres draining through a slit until
they settle) gives no geometry, radius, stiffness or time step, so the workloads below
are synthetic stand-ins with the shapes the paper describes: dense, mostly-touching
packings under gravity, monodisperse or mildly polydisperse, with planar or
cylindrical walls.

Units are SI. Arrays are numpy: positions/velocities/spins float64 of shape (n, 3),
radii float32 of shape (n,). Walls are dicts with `kind` ('plane' | 'cylinder'),
`p` (a point), `n` (plane: unit normal pointing INTO the domain; cylinder: unit axis),
`radius` (cylinder), `omega` (angular velocity of the wall surface about `p`) and
`vel` (translational velocity of the wall surface).
"""
from __future__ import annotations

import ctypes
import math
import os
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "libdemscenes.so")
_lib = None

RHO_DEFAULT = 2500.0
G_DEFAULT = (0.0, 0.0, -9.81)


def build(force: bool = False) -> str:
    """Compile the generator library in place (gcc, IEEE double, no FMA contraction)."""
    src = os.path.join(_HERE, "scenes.c")
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        import subprocess

        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math",
             "-o", tmp, src, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def _L():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_SO)
        P = ctypes.c_void_p
        I64 = ctypes.c_int64
        D = ctypes.c_double
        U64 = ctypes.c_uint64
        lib.scn_xoshiro_first.argtypes = [U64, ctypes.c_int, P]
        lib.scn_xoshiro_first.restype = U64
        lib.scn_uniform.argtypes = [U64, I64, D, D, P]
        lib.scn_uniform.restype = None
        lib.scn_normal.argtypes = [U64, I64, D, P]
        lib.scn_normal.restype = None
        lib.scn_loguniform_int.argtypes = [U64, I64, D, D, P]
        lib.scn_loguniform_int.restype = None
        lib.scn_lattice_box.argtypes = [U64, ctypes.c_int, ctypes.c_int, ctypes.c_int, D, D, P, D, D, P, P, P, P]
        lib.scn_lattice_box.restype = None
        lib.scn_rsa_box.argtypes = [U64, I64, D, D, P, P, I64, P, P, P, P]
        lib.scn_rsa_box.restype = I64
        lib.scn_drum_fill.argtypes = [U64, I64, D, D, D, D, D, P, P, P, P]
        lib.scn_drum_fill.restype = I64
        lib.scn_count_overlaps.argtypes = [I64, P, P, D]
        lib.scn_count_overlaps.restype = I64
        _lib = lib
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


# --------------------------------------------------------------------------- RNG
def xoshiro_first(seed: int, k: int) -> np.ndarray:
    out = np.zeros(k, dtype=np.uint64)
    _L().scn_xoshiro_first(seed, k, _p(out))
    return out


def uniform(seed: int, n: int, a: float, b: float) -> np.ndarray:
    out = np.zeros(n, dtype=np.float64)
    _L().scn_uniform(seed, n, a, b, _p(out))
    return out


def normal(seed: int, n: int, sigma: float) -> np.ndarray:
    out = np.zeros(n, dtype=np.float64)
    _L().scn_normal(seed, n, sigma, _p(out))
    return out


def loguniform_int(seed: int, n: int, lo: float, hi: float) -> np.ndarray:
    out = np.zeros(n, dtype=np.int64)
    _L().scn_loguniform_int(seed, n, lo, hi, _p(out))
    return out


def count_overlaps(x: np.ndarray, r: np.ndarray) -> int:
    x = np.ascontiguousarray(x, dtype=np.float64)
    r = np.ascontiguousarray(r, dtype=np.float32)
    return int(_L().scn_count_overlaps(len(r), _p(x), _p(r), float(r.max()) if len(r) else 1.0))


# ------------------------------------------------------------------ parameters
def sphere_mass(r: float, rho: float = RHO_DEFAULT) -> float:
    return rho * 4.0 / 3.0 * math.pi * r ** 3


def zeta_from_e(e: float) -> float:
    """Damping ratio of a linear spring-dashpot whose restitution coefficient is e."""
    le = math.log(e)
    return -le / math.sqrt(math.pi ** 2 + le ** 2)


def alpha_from_e(e: float) -> float:
    """alpha of Eq. 10 for a LINEAR spring: eta = alpha*sqrt(k_n*m_eff) with alpha = 2*zeta."""
    return 2.0 * zeta_from_e(e)


def linear_contact_time(kn: float, e: float, m_eff: float) -> float:
    """Duration of a linear spring-dashpot contact (used only to choose the time step)."""
    z = zeta_from_e(e)
    w0 = math.sqrt(kn / m_eff)
    return math.pi / (w0 * math.sqrt(1.0 - z * z))


def auto_cell_size(rmax: float, skin: float = 0.0) -> float:
    """Grid cell edge: one diameter of the largest sphere plus a 2^-10 relative margin
    (so that FP32 cell hashing never splits a contact pair across non-neighbouring
    cells) plus the Verlet skin."""
    return 2.0 * rmax * (1.0 + 2.0 ** -10) + skin


def grid_dims(lo, hi, h):
    return tuple(max(1, int(math.ceil((hi[a] - lo[a]) / h))) for a in range(3))


def box_walls(lo, hi):
    return [
        dict(kind="plane", p=(lo[0], 0.0, 0.0), n=(1.0, 0.0, 0.0)),
        dict(kind="plane", p=(hi[0], 0.0, 0.0), n=(-1.0, 0.0, 0.0)),
        dict(kind="plane", p=(0.0, lo[1], 0.0), n=(0.0, 1.0, 0.0)),
        dict(kind="plane", p=(0.0, hi[1], 0.0), n=(0.0, -1.0, 0.0)),
        dict(kind="plane", p=(0.0, 0.0, lo[2]), n=(0.0, 0.0, 1.0)),
        dict(kind="plane", p=(0.0, 0.0, hi[2]), n=(0.0, 0.0, -1.0)),
    ]


def drum_walls(Rd, L, omega):
    w = (omega, 0.0, 0.0)
    return [
        dict(kind="cylinder", p=(0.0, 0.0, 0.0), n=(1.0, 0.0, 0.0), radius=Rd, omega=w),
        dict(kind="plane", p=(0.0, 0.0, 0.0), n=(1.0, 0.0, 0.0), omega=w),
        dict(kind="plane", p=(L, 0.0, 0.0), n=(-1.0, 0.0, 0.0), omega=w),
    ]


def slit_plates(z, xc, half_width):
    """A horizontal plate at height z with a slit of width 2 half_width across x, centred
    at xc and running the whole length in y: two half-plates, touched from both sides."""
    return [dict(kind="half_plate", p=(xc + half_width, 0.0, z), n=(0.0, 0.0, 1.0), u=(1.0, 0.0, 0.0)),
            dict(kind="half_plate", p=(xc - half_width, 0.0, z), n=(0.0, 0.0, 1.0), u=(-1.0, 0.0, 0.0))]


def _norm_wall(w):
    d = dict(kind=w["kind"], p=tuple(w["p"]), n=tuple(w["n"]), radius=float(w.get("radius", 0.0)),
             omega=tuple(w.get("omega", (0.0, 0.0, 0.0))), vel=tuple(w.get("vel", (0.0, 0.0, 0.0))),
             u=tuple(w.get("u", (0.0, 0.0, 0.0))))
    return d


@dataclass
class Params:
    """Physical and numerical parameters of one run (inputs to both implementations)."""
    model: str = "practical"        # 'practical' (Eqs. 2-10) | 'simple' (Eq. 1)
    stiffness: str = "linear"       # 'linear' (constant k) | 'hertz' (Eqs. 8-9)
    precision: str = "fp64"         # 'fp64' | 'fp32' (FP32 forces, compensated positions)
    dt: float = 1e-6
    rho: float = RHO_DEFAULT
    g: tuple = G_DEFAULT
    kn: float = 1e4
    kt: float = 1e4 * 2.0 / 7.0
    cn: float = 0.0                  # Hertz C_{k,n}
    ct: float = 0.0                  # Hertz C_{k,t}
    alpha: float = 0.0               # Eq. 10
    mu: float = 0.3
    ksp: float = 0.0                 # Eq. 1 spring
    kda: float = 0.0                 # Eq. 1 damping
    ksh: float = 0.0                 # Eq. 1 shear
    skin: float = 0.0
    cell_size: float = 0.0
    domain_lo: tuple = (0.0, 0.0, 0.0)
    domain_hi: tuple = (1.0, 1.0, 1.0)
    resort_interval: int = 1
    terms: int = 0                   # optional terms: 1 no attraction, 2 rolling, 4 eta_t, 8 cohesion
    mu_roll: float = 0.0             # rolling resistance coefficient
    alpha_t: float = 0.0             # tangential damping factor (terms & 4)
    k_coh: float = 0.0               # cohesion energy density [N/m^2] (terms & 8)
    walls: list = field(default_factory=list)

    def copy(self, **kw):
        d = dict(self.__dict__)
        d["walls"] = [dict(w) for w in self.walls]
        d.update(kw)
        return Params(**d)


@dataclass
class Scene:
    name: str
    x: np.ndarray
    v: np.ndarray
    w: np.ndarray
    r: np.ndarray
    params: Params

    @property
    def n(self) -> int:
        return int(len(self.r))


def hertz_coeffs(kn_ref: float, kt_over_kn: float, rbar: float):
    """C_{k,n}, C_{k,t} for Eqs. 8-9 chosen so that the Hertz stiffness equals kn_ref at an
    overlap of 1% of rbar between two spheres of radius rbar (R_eff = rbar/2)."""
    cn = kn_ref / math.sqrt(0.01 * rbar * 0.5 * rbar)
    return cn, kt_over_kn * cn


# ----------------------------------------------------------- concrete workloads
def box_lattice(seed: int = 1, nx: int = 16, ny: int = 16, nz: int = 8, r: float = 1e-3,
                box=(64.0, 64.0, 128.0), spacing: float = 2.1, jitter: float = 0.025,
                vsigma: float = 0.1, e: float = 0.9, kn: float = 1e4, mu: float = 0.3,
                precision: str = "fp64", model: str = "practical", stiffness: str = "linear") -> Scene:
    """Spheres of radius r on a jittered lattice in a walled box of box*r (first layer at
    z = 1.05 r, centred in x and y), velocities N(0, vsigma) per axis, zero spin.
    Defaults: 2,048 spheres in 64r x 64r x 128r, k_n = 1e4 N/m, e = 0.9,
    k_t = (2/7) k_n, mu = 0.3, dt = contact time / 50."""
    n = nx * ny * nz
    lo = (0.0, 0.0, 0.0)
    hi = (box[0] * r, box[1] * r, box[2] * r)
    first = np.array([0.5 * (hi[0] - (nx - 1) * spacing * r), 0.5 * (hi[1] - (ny - 1) * spacing * r), 1.05 * r])
    x = np.zeros((n, 3)); v = np.zeros((n, 3)); w = np.zeros((n, 3)); rad = np.zeros(n, dtype=np.float32)
    _L().scn_lattice_box(seed, nx, ny, nz, spacing * r, jitter * r, _p(first), r, vsigma, _p(x), _p(v), _p(w), _p(rad))
    m = sphere_mass(float(np.float32(r)))
    meff = 0.5 * m
    dt = linear_contact_time(kn, e, meff) / 50.0
    alpha = alpha_from_e(e)
    eta = alpha * math.sqrt(kn * meff)
    cn, ct = hertz_coeffs(kn, 2.0 / 7.0, r)
    p = Params(model=model, stiffness=stiffness, precision=precision, dt=dt, kn=kn, kt=kn * 2.0 / 7.0, cn=cn, ct=ct,
               alpha=alpha, mu=mu, ksp=kn, kda=eta, ksh=eta, cell_size=auto_cell_size(float(rad.max())),
               domain_lo=lo, domain_hi=hi, walls=[_norm_wall(q) for q in box_walls(lo, hi)])
    return Scene(f"box_lattice_{n}_s{seed}", x, v, w, rad, p)


def box_rsa(seed: int = 1, n: int = 262_144, rbar: float = 1e-3, spread: float = 0.2,
            box=(160.0, 160.0, 400.0), phi: float = 0.35, e: float = 0.9, kn: float = 1e4,
            mu: float = 0.3, precision: str = "fp32", model: str = "practical",
            stiffness: str = "linear") -> Scene:
    """Polydisperse loose fill: radii U[(1-spread) rbar, (1+spread) rbar], random
    sequential addition into the bottom of a walled box (box*rbar) up to solid fraction
    phi, at rest. Defaults: 262,144 spheres, 160 x 160 x 400 rbar, phi = 0.35. dt is
    the contact time of the smallest pair / 50. For a smaller n the box's horizontal
    section shrinks with n^(1/2) so the fill height stays the same."""
    rmin, rmax = (1 - spread) * rbar, (1 + spread) * rbar
    scale = math.sqrt(n / 262_144.0) if n < 262_144 else 1.0
    lo = (0.0, 0.0, 0.0)
    hi = (box[0] * rbar * scale, box[1] * rbar * scale, box[2] * rbar)
    mean_vol = 4.0 / 3.0 * math.pi * (rmax ** 4 - rmin ** 4) / (4.0 * (rmax - rmin))
    fill_h = n * mean_vol / (phi * (hi[0] - lo[0]) * (hi[1] - lo[1]))
    x = np.zeros((n, 3)); v = np.zeros((n, 3)); w = np.zeros((n, 3)); rad = np.zeros(n, dtype=np.float32)
    fill_hi = np.array([hi[0], hi[1], min(hi[2], fill_h)])
    grows = _L().scn_rsa_box(seed, n, rmin, rmax, _p(np.array(lo, dtype=np.float64)), _p(fill_hi), 20000,
                             _p(x), _p(v), _p(w), _p(rad))
    if grows < 0:
        raise MemoryError("scn_rsa_box failed")
    mmin = sphere_mass(float(np.float32(rmin)))
    dt = linear_contact_time(kn, e, 0.5 * mmin) / 50.0
    alpha = alpha_from_e(e)
    mbar = sphere_mass(rbar)
    eta = alpha * math.sqrt(kn * 0.5 * mbar)
    cn, ct = hertz_coeffs(kn, 2.0 / 7.0, rbar)
    p = Params(model=model, stiffness=stiffness, precision=precision, dt=dt, kn=kn, kt=kn * 2.0 / 7.0, cn=cn, ct=ct,
               alpha=alpha, mu=mu, ksp=kn, kda=eta, ksh=eta, cell_size=auto_cell_size(float(rad.max())),
               domain_lo=lo, domain_hi=hi, walls=[_norm_wall(q) for q in box_walls(lo, hi)])
    return Scene(f"box_rsa_{n}_s{seed}", x, v, w, rad, p)


def hopper(seed: int = 1, nx: int = 64, ny: int = 32, nz: int = 64, r: float = 1e-3, spacing: float = 2.1,
           jitter: float = 0.025, vsigma: float = 0.05, slit_over_d: float = 6.0, e: float = 0.5, kn: float = 1e4,
           mu: float = 0.5, precision: str = "fp32", model: str = "practical", stiffness: str = "linear",
           open_slit: bool = True) -> Scene:
    """The shape of the paper's benchmark (Sec. 5): equal spheres fall from a box through
    a slit in its bottom onto a floor (2^17 = 131,072 spheres by default; the paper gives
    no geometry). The box has the lattice's footprint (nx x ny columns at spacing r,
    sphere edges 0.05 r from the side walls); its bottom is a plate with a slit of width
    2 slit_over_d r across x, centred, running the whole depth in y (two half-plates);
    the bin below holds all spheres at solid fraction 0.43. The spheres start on the
    jittered lattice just above the plate, velocities N(0, vsigma). With open_slit=False
    the bottom is a closed plane instead, for filling the box at rest before the slit
    opens. Walls: the four sides, the floor and a lid (planes), then the plate.
    dt = contact time / 50."""
    n = nx * ny * nz
    W = (nx * spacing * r, ny * spacing * r)
    bin_h = n * (4.0 / 3.0) * math.pi * r ** 3 / (0.43 * W[0] * W[1])
    zp = math.ceil(bin_h / r) * r
    top = zp + (1.05 + (nz - 1) * spacing + 3.0) * r
    lo, hi = (0.0, 0.0, 0.0), (W[0], W[1], top)
    first = np.array([0.5 * spacing * r, 0.5 * spacing * r, zp + 1.05 * r])
    x = np.zeros((n, 3)); v = np.zeros((n, 3)); w = np.zeros((n, 3)); rad = np.zeros(n, dtype=np.float32)
    _L().scn_lattice_box(seed, nx, ny, nz, spacing * r, jitter * r, _p(first), r, vsigma, _p(x), _p(v), _p(w), _p(rad))
    m = sphere_mass(float(np.float32(r)))
    dt = linear_contact_time(kn, e, 0.5 * m) / 50.0
    alpha = alpha_from_e(e)
    eta = alpha * math.sqrt(kn * 0.5 * m)
    cn, ct = hertz_coeffs(kn, 2.0 / 7.0, r)
    if open_slit:
        plate = slit_plates(zp, 0.5 * W[0], slit_over_d * r)
    else:
        plate = [dict(kind="plane", p=(0.0, 0.0, zp), n=(0.0, 0.0, 1.0))]
    walls = box_walls(lo, hi) + plate
    p = Params(model=model, stiffness=stiffness, precision=precision, dt=dt, kn=kn, kt=kn * 2.0 / 7.0, cn=cn, ct=ct,
               alpha=alpha, mu=mu, ksp=kn, kda=eta, ksh=eta, cell_size=auto_cell_size(float(rad.max())),
               domain_lo=lo, domain_hi=hi, walls=[_norm_wall(q) for q in walls])
    return Scene(f"hopper_{n}_s{seed}", x, v, w, rad, p)


def drum(seed: int = 1, n: int = 4_194_304, rbar: float = 1e-3, spread: float = 0.1,
         Rd_over_r: float = 300.0, L_over_r: float = 208.0, omega: float = 2.0, e: float = 0.7,
         kn: float = 1e4, mu: float = 0.5, precision: str = "fp32", model: str = "practical",
         stiffness: str = "linear") -> Scene:
    """Dense packing in the lower half of a drum rotating about its horizontal axis.
    Radii U[0.9, 1.1] rbar; drum radius 300 rbar, length 208 rbar, end caps co-rotating
    at omega = 2 rad/s; mu = 0.5, e = 0.7. The bed is built by layered vertical
    deposition (solid fraction about 0.6, each sphere resting on what is below it).
    For n smaller than the default, the drum's length and radius shrink with n^(1/3)."""
    rmin, rmax = (1 - spread) * rbar, (1 + spread) * rbar
    s = (n / 4_194_304.0) ** (1.0 / 3.0) if n < 4_194_304 else 1.0
    Rd = Rd_over_r * rbar * s
    L = max(L_over_r * rbar * s, 8.0 * rmax)
    x = np.zeros((n, 3)); v = np.zeros((n, 3)); w = np.zeros((n, 3)); rad = np.zeros(n, dtype=np.float32)
    passes = _L().scn_drum_fill(seed, n, rmin, rmax, Rd, L, 1.7 * rbar, _p(x), _p(v), _p(w), _p(rad))
    if passes < 0:
        raise RuntimeError(f"scn_drum_fill failed ({passes})")
    mmin = sphere_mass(float(np.float32(rmin)))
    dt = linear_contact_time(kn, e, 0.5 * mmin) / 50.0
    alpha = alpha_from_e(e)
    mbar = sphere_mass(rbar)
    eta = alpha * math.sqrt(kn * 0.5 * mbar)
    cn, ct = hertz_coeffs(kn, 2.0 / 7.0, rbar)
    lo = (0.0, -Rd, -Rd)
    hi = (L, Rd, Rd)
    p = Params(model=model, stiffness=stiffness, precision=precision, dt=dt, kn=kn, kt=kn * 2.0 / 7.0, cn=cn, ct=ct,
               alpha=alpha, mu=mu, ksp=kn, kda=eta, ksh=eta, cell_size=auto_cell_size(float(rad.max())),
               domain_lo=lo, domain_hi=hi, walls=[_norm_wall(q) for q in drum_walls(Rd, L, omega)])
    return Scene(f"drum_{n}_s{seed}", x, v, w, rad, p)


def batch_mix(seed: int = 1, count: int = 256, nmin: int = 1024, nmax: int = 65536,
              precision: str = "fp32", model: str = "practical"):
    """Independent box-settling scenes with log-uniform sizes, per-scene mu ~ U[0.1, 0.6]
    and e ~ U[0.5, 0.95]; each box keeps the 2,048-sphere box's number density (edges
    scaled by (N/2048)^(1/3)); monodisperse r = 1 mm."""
    sizes = loguniform_int(seed, count, nmin, nmax)
    mus = uniform(seed + 1000, count, 0.1, 0.6)
    es = uniform(seed + 2000, count, 0.5, 0.95)
    scenes = []
    for k in range(count):
        nk = int(sizes[k])
        sc = box_lattice_n(seed * 7919 + k, nk, e=float(es[k]), mu=float(mus[k]), precision=precision, model=model)
        scenes.append(sc)
    return scenes


def box_lattice_n(seed: int, n: int, r: float = 1e-3, e: float = 0.9, mu: float = 0.3, kn: float = 1e4,
                  vsigma: float = 0.1, precision: str = "fp64", model: str = "practical",
                  stiffness: str = "linear") -> Scene:
    """The 2,048-sphere box scene generalised to any n: the lattice keeps the 2:1 aspect
    (nx = ny = 2 nz, rounded up) and the box edges scale by (n/2048)^(1/3); the first n
    lattice sites are used."""
    s = (n / 2048.0) ** (1.0 / 3.0)
    nz = max(1, int(math.ceil(8 * s)))
    nx = ny = max(1, int(math.ceil(16 * s)))
    while nx * ny * nz < n:
        nz += 1
    box = (64.0 * s, 64.0 * s, 128.0 * s)
    box = (max(box[0], (nx - 1) * 2.1 + 3.0), max(box[1], (ny - 1) * 2.1 + 3.0), max(box[2], (nz - 1) * 2.1 + 3.0))
    sc = box_lattice(seed, nx, ny, nz, r=r, box=box, e=e, mu=mu, kn=kn, vsigma=vsigma, precision=precision,
                     model=model, stiffness=stiffness)
    sc.x = np.ascontiguousarray(sc.x[:n]); sc.v = np.ascontiguousarray(sc.v[:n])
    sc.w = np.ascontiguousarray(sc.w[:n]); sc.r = np.ascontiguousarray(sc.r[:n])
    sc.name = f"box_lattice_{n}_s{seed}"
    return sc
