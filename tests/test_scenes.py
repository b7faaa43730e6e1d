"""The seeded input generators: determinism, no initial overlaps, geometry of each family."""
import math

import numpy as np

from paper_1301_1714_gb300 import scenes as S


def test_generators_are_deterministic():
    a = S.box_lattice(seed=4)
    b = S.box_lattice(seed=4)
    c = S.box_lattice(seed=5)
    assert np.array_equal(a.x, b.x) and np.array_equal(a.v, b.v) and np.array_equal(a.r, b.r)
    assert not np.array_equal(a.x, c.x)
    assert np.array_equal(S.xoshiro_first(9, 8), S.xoshiro_first(9, 8))


def test_uniform_and_normal_moments():
    u = S.uniform(3, 200_000, 2.0, 5.0)
    assert u.min() >= 2.0 and u.max() < 5.0
    assert abs(u.mean() - 3.5) < 0.01 and abs(u.var() - 0.75) < 0.01
    z = S.normal(3, 200_000, 0.1)
    assert abs(z.mean()) < 1e-3 and abs(z.std() - 0.1) < 1e-3
    k = S.loguniform_int(3, 10_000, 1024, 65536)
    assert k.min() >= 1024 and k.max() <= 65536
    assert abs(np.mean(np.log(k)) - 0.5 * (math.log(1024) + math.log(65536))) < 0.05


def test_box_lattice_default_scene():
    sc = S.box_lattice()
    assert sc.n == 2048
    assert S.count_overlaps(sc.x, sc.r) == 0
    hi = np.array(sc.params.domain_hi)
    r = sc.r.astype(np.float64)[:, None]
    assert np.all(sc.x - r > 0) and np.all(sc.x + r < hi)
    assert abs(sc.v.std() - 0.1) < 0.01
    assert sc.params.dt == __import__("pytest").approx(1.43854e-6, rel=1e-5)


def test_rsa_loose_fill():
    sc = S.box_rsa(seed=2, n=8192)
    assert S.count_overlaps(sc.x, sc.r) == 0
    r = sc.r.astype(np.float64)
    assert r.min() >= 0.8e-3 * (1 - 1e-6) and r.max() <= 1.2e-3 * (1 + 1e-6)
    lo, hi = np.array(sc.params.domain_lo), np.array(sc.params.domain_hi)
    assert np.all(sc.x - r[:, None] >= lo) and np.all(sc.x + r[:, None] <= hi)
    vol = np.sum(4 / 3 * math.pi * r ** 3)
    top = sc.x[:, 2].max() + r.max()
    phi = vol / ((hi[0] - lo[0]) * (hi[1] - lo[1]) * top)
    assert 0.25 < phi < 0.4


def test_drum_dense_bed():
    sc = S.drum(seed=3, n=20000)
    assert S.count_overlaps(sc.x, sc.r) == 0
    cyl = sc.params.walls[0]
    Rd = cyl["radius"]
    L = sc.params.walls[2]["p"][0]
    r = sc.r.astype(np.float64)
    rho = np.hypot(sc.x[:, 1], sc.x[:, 2])
    assert np.all(rho + r <= Rd) and np.all(sc.x[:, 0] - r >= 0) and np.all(sc.x[:, 0] + r <= L)
    # solid fraction of the bed below its mean top
    ztop = np.percentile(sc.x[:, 2], 95)
    sel = sc.x[:, 2] < ztop - 3e-3
    h = ztop - 3e-3
    seg = Rd * Rd * math.acos(-h / Rd) + h * math.sqrt(Rd * Rd - h * h) if h < 0 else None
    area = Rd * Rd * math.acos(-h / Rd) + h * math.sqrt(Rd * Rd - h * h)
    phi = np.sum(4 / 3 * math.pi * r[sel] ** 3) / (area * L)
    assert 0.5 < phi < 0.7


def test_hopper_scene():
    """The hopper: 2^17 equal spheres (the paper's count, Sec. 5) above a plate with a
    slit; no overlaps, every sphere inside the box and above the plate; the bin below
    the plate holds them all at solid fraction 0.43; the two half-plates face each other
    across a slit of 2 slit_over_d r."""
    import os
    sc = S.hopper()
    gold = {}
    for line in open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "paper_values.txt")):
        line = line.split("#", 1)[0].strip()
        if line:
            k, v = (t.strip() for t in line.split("="))
            gold[k] = float(v)
    assert sc.n == gold["benchmark_particles"]
    assert S.count_overlaps(sc.x, sc.r) == 0
    walls = sc.params.walls
    assert len(walls) == 8 and walls[6]["kind"] == walls[7]["kind"] == "half_plate"
    zp = walls[6]["p"][2]
    r = sc.r.astype(np.float64)[:, None]
    hi = np.array(sc.params.domain_hi)
    assert np.all(sc.x - r > 0) and np.all(sc.x + r < hi)
    assert np.all(sc.x[:, 2] - sc.r > zp)
    W = hi[0] * hi[1]
    assert sc.n * 4 / 3 * math.pi * 1e-9 / (W * zp) <= 0.43 + 1e-9
    assert walls[6]["p"][0] - walls[7]["p"][0] == __import__("pytest").approx(12e-3)
    assert walls[6]["u"] == (1.0, 0.0, 0.0) and walls[7]["u"] == (-1.0, 0.0, 0.0)
    closed = S.hopper(open_slit=False)
    assert len(closed.params.walls) == 7 and closed.params.walls[6]["kind"] == "plane"
    assert np.array_equal(closed.x, sc.x)
