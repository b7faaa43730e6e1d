"""CUDA path against the FP64 oracle, through the C ABI, on the same seeded inputs.

Bars:
  cell keys, (cell, id) order ............ bit-exact
  contact pair set, FP64 mode ............ bit-exact
  contact pair set, FP32 mode ............ bit-exact outside |d^2 - R^2| <= 2^-36 R^2
                                           (inside that band both answers are valid)
  per-step force/torque .................. |dF| / S_i <= 1e-12 (FP64), 1e-5 (FP32) with
                                           S_i = m_i|g| + sum over contacts (k delta + eta|v|)(1 + mu)
  trajectories, FP64 ..................... max |dx| <= 1e-12 m after 10 steps, 1e-9 m after 1,000
"""
import math

import numpy as np
import pytest

import oracle
from paper_1301_1714_gb300 import dem, scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1301_1714_gb300 import _build
    _build.build()
    dem.lib()


def sim(params, sc, **kw):
    return dem.Simulation(params, sc.x, sc.v, sc.w, sc.r, **kw)


# ------------------------------------------------------------------ helpers
def force_scale(p, x, v, r, pairs):
    """S_i = m_i|g| + sum over i's contacts of (k delta + eta |v_ij|)(1 + mu)."""
    rr = r.astype(np.float64)
    m = p.rho * 4.0 / 3.0 * math.pi * rr ** 3
    S = m * np.linalg.norm(p.g)
    if len(pairs):
        i, j = pairs[:, 0].astype(np.int64), pairs[:, 1].astype(np.int64)
        d = np.linalg.norm(x[j] - x[i], axis=1)
        delta = rr[i] + rr[j] - d
        meff = m[i] * m[j] / (m[i] + m[j])
        reff = rr[i] * rr[j] / (rr[i] + rr[j])
        if p.stiffness == "linear":
            k = np.full_like(delta, max(p.kn, p.ksp))
        else:
            k = p.cn * np.sqrt(np.abs(delta) * reff)
        eta = max(p.alpha * np.sqrt(k * meff).max(initial=0.0), p.kda, p.ksh)
        vij = np.linalg.norm(v[i] - v[j], axis=1)
        c = (k * np.abs(delta) + eta * vij) * (1 + p.mu)
        np.add.at(S, i, c)
        np.add.at(S, j, c)
    # walls: plane overlaps and axis-aligned cylinders
    for wl in p.walls:
        if wl["kind"] == "plane":
            s = (x - np.array(wl["p"])) @ np.array(wl["n"])
            delta = rr - s
        elif wl["kind"] == "half_plate":
            q = x - np.array(wl["p"])
            h = q @ np.array(wl["n"])
            su = q @ np.array(wl["u"])
            delta = rr - np.hypot(h, np.minimum(su, 0.0))
        else:
            a = np.array(wl["n"])
            q = x - np.array(wl["p"])
            rho = np.linalg.norm(q - np.outer(q @ a, a), axis=1)
            delta = rho + rr - wl["radius"]
        on = delta > 0
        k = max(p.kn, p.ksp) if p.stiffness == "linear" else p.cn * np.sqrt(np.abs(delta) * rr)
        eta = np.maximum(p.alpha * np.sqrt(k * m), max(p.kda, p.ksh))
        S = S + np.where(on, (k * np.abs(delta) + eta * np.linalg.norm(v, axis=1)) * (1 + p.mu), 0.0)
    return S


def assert_forces_close(p, x, v, r, F, T, Fo, To, tol):
    pairs = oracle.pairs_brute(x, r) if len(r) <= 4096 else oracle.pairs_grid(p, x, r)
    S = force_scale(p, x, v, r, pairs)
    eF = np.linalg.norm(F - Fo, axis=1) / S
    eT = np.linalg.norm(T - To, axis=1) / (S * r.astype(np.float64))
    assert eF.max() <= tol, f"force error {eF.max():.3e} > {tol} at particle {eF.argmax()}"
    assert eT.max() <= tol, f"torque error {eT.max():.3e} > {tol} at particle {eT.argmax()}"


def fp32_band_pairs(x, r, pairs, band=2.0 ** -36):
    """Pairs whose |d^2 - R^2| is within the band relative to R^2."""
    out = set()
    for i, j in pairs:
        d2 = float(np.sum((x[j] - x[i]) ** 2))
        R2 = (float(r[i]) + float(r[j])) ** 2
        if abs(d2 - R2) <= band * R2:
            out.add((int(i), int(j)))
    return out


def near_pairs(x, r, band=2.0 ** -36):
    """All pairs (brute force) whose |d^2 - R^2| <= band R^2."""
    out = set()
    n = len(r)
    for i in range(n):
        d2 = np.sum((x[i + 1:] - x[i]) ** 2, axis=1)
        R2 = (float(r[i]) + r[i + 1:].astype(np.float64)) ** 2
        for k in np.nonzero(np.abs(d2 - R2) <= band * R2)[0]:
            out.add((i, i + 1 + int(k)))
    return out


SCENES = {
    "box2048": lambda: scenes.box_lattice(seed=1),
    "rsa3000": lambda: scenes.box_rsa(seed=2, n=3000),
    "drum4099": lambda: scenes.drum(seed=3, n=4099),
}
# compression toward the centroid that gives each scene many contacts (the box lattice
# has 2.1 r spacing, so it needs about 5%)
SQUEEZE = {"box2048": 0.945, "rsa3000": 0.985, "drum4099": 0.985}


# ------------------------------------------------------------ hash / sort (steps 2-4)
@pytest.mark.parametrize("name", list(SCENES))
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_cell_keys_and_order_bit_exact(name, precision):
    sc = SCENES[name]()
    p = sc.params.copy(precision=precision)
    key, _ = oracle.cell_keys(p, sc.x)
    order, _ = oracle.sort_by_cell(key)
    with sim(p, sc) as s:
        o, h, dims = dem.dem_get_grid(s.h)
        assert dims == oracle.grid_dims(p) and h == p.cell_size
        cell, gorder, _ = s.snapshot(with_pairs=False)
    assert np.array_equal(cell.astype(np.uint64), key)
    assert np.array_equal(gorder, order)


def test_hash_clamps_outside_particles_and_planted_faces():
    """Particles outside the grid use the nearest face cell; positions on cell faces."""
    sc = scenes.box_lattice(seed=5, nx=6, ny=5, nz=4, box=(16.0, 16.0, 16.0))
    p = sc.params.copy(walls=[])
    x = sc.x.copy()
    h = p.cell_size
    x[0] = [-0.01, 0.5 * h, 0.5 * h]
    x[1] = [p.domain_hi[0] + 0.02, p.domain_hi[1] + 1.0, -3.0]
    x[2] = [2 * h, 3 * h, h]                    # exactly on faces
    x[3] = [np.nextafter(2 * h, 0), np.nextafter(3 * h, 0), np.nextafter(h, 0)]
    for prec in ("fp64", "fp32"):
        pp = p.copy(precision=prec)
        key, _ = oracle.cell_keys(pp, x)
        order, _ = oracle.sort_by_cell(key)
        with dem.Simulation(pp, x, sc.v, sc.w, sc.r) as s:
            cell, gorder, _ = s.snapshot(with_pairs=False)
        assert np.array_equal(cell.astype(np.uint64), key)
        assert np.array_equal(gorder, order)


# ------------------------------------------------------------ contact pairs (step 7)
@pytest.mark.parametrize("name", list(SCENES))
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_pair_set(name, precision):
    sc = SCENES[name]()
    x = compressed(sc, SQUEEZE[name])
    p = sc.params.copy(precision=precision)
    ref = oracle.pairs_brute(x, sc.r)
    with dem.Simulation(p, x, sc.v, sc.w, sc.r) as s:
        s.forces()
        _, _, gp = s.snapshot()
    assert len(ref) > 100
    if precision == "fp64":
        assert np.array_equal(gp, ref)
    else:
        A = set(map(tuple, ref.tolist()))
        B = set(map(tuple, gp.tolist()))
        diff = A ^ B
        assert diff <= near_pairs(x, sc.r), f"{len(diff)} pairs differ outside the FP32 band"


def test_pair_set_with_planted_near_touching_pairs():
    """Pairs placed at exactly touching and one FP64 ulp inside: FP64 mode decides them
    exactly as the oracle does."""
    rng = np.random.default_rng(3)
    n = 1500
    x = rng.uniform(0.002, 0.028, size=(n, 3))
    r = rng.uniform(0.8e-3, 1.2e-3, size=n).astype(np.float32)
    for k in range(0, 90, 3):
        Rk = float(r[k]) + float(r[k + 1])
        x[k + 1] = x[k] + np.array([Rk, 0.0, 0.0])
        Rk2 = float(r[k]) + float(r[k + 2])
        x[k + 2] = x[k] + np.array([0.0, np.nextafter(Rk2, 0.0), 0.0])
    p = scenes.Params(precision="fp64", dt=1e-6, cell_size=scenes.auto_cell_size(float(r.max())),
                      domain_lo=(0, 0, 0), domain_hi=(0.03, 0.03, 0.03), walls=[], g=(0.0, 0.0, 0.0))
    ref = oracle.pairs_brute(x, r)
    z = np.zeros((n, 3))
    with dem.Simulation(p, x, z, z, r) as s:
        s.forces()
        _, _, gp = s.snapshot()
    assert np.array_equal(gp, ref)


# ------------------------------------------------------------ forces (steps 5-8)
def compressed(sc, f=0.985):
    c = sc.x.mean(axis=0)
    return c + (sc.x - c) * f


FORCE_CASES = [
    ("box2048", "practical", "linear"),
    ("box2048", "practical", "hertz"),
    ("box2048", "simple", "linear"),
    ("rsa3000", "practical", "linear"),
    ("drum4099", "practical", "linear"),
    ("drum4099", "simple", "linear"),
]


@pytest.mark.parametrize("name,model,stiff", FORCE_CASES)
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_forces_first_contact(name, model, stiff, precision):
    sc = SCENES[name]()
    x = compressed(sc, SQUEEZE[name])
    rng = np.random.default_rng(1)
    w = rng.normal(0, 20.0, size=x.shape)
    p = sc.params.copy(precision=precision, model=model, stiffness=stiff)
    Fo, To, _, stats = oracle.forces(p, x, sc.v, w, sc.r)
    assert stats[0] > 100
    with dem.Simulation(p, x, sc.v, w, sc.r) as s:
        F, T = s.forces()
    assert_forces_close(p, x, sc.v, sc.r, F, T, Fo, To, 1e-12 if precision == "fp64" else 1e-5)


@pytest.mark.parametrize("name", ["box2048", "drum4099"])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_forces_with_stored_history(name, precision):
    """The oracle runs some steps; its state and springs are restored into the GPU
    library (oracle -> GPU only) and the next step's forces are compared."""
    sc = SCENES[name]()
    p = sc.params.copy(precision="fp64")
    st = oracle.State(p, compressed(sc, SQUEEZE[name] + 0.005), sc.v, sc.w, sc.r).run(60)
    hist = st.history
    assert len(hist) > 50
    Fo, To, _, _ = oracle.forces(p, st.x, st.v, st.w, st.r, hist)
    pg = p.copy(precision=precision)
    h = dem.dem_create(dem.config_from_params(pg))
    try:
        dem.dem_set_walls(h, pg.walls)
        dem.dem_restore(h, st.x, st.v, st.w, st.r, hist)
        F, T = dem.dem_get_forces(h, len(st.r))
        back = dem.dem_get_history(h)
    finally:
        dem.dem_destroy(h)
    assert np.array_equal(back["i"], hist["i"]) and np.array_equal(back["j"], hist["j"])
    tol_d = 0.0 if precision == "fp64" else 1e-6
    assert np.all(np.abs(back["d"] - hist["d"]) <= tol_d * np.abs(hist["d"]) + (0 if precision == "fp64" else 1e-30))
    assert_forces_close(p, st.x, st.v, st.r, F, T, Fo, To, 1e-12 if precision == "fp64" else 1e-5)


# ------------------------------------------------------------ trajectories
def test_trajectory_fp64_box2048():
    """The 2,048-sphere box (FP64): positions after 10 and 1,000 steps."""
    sc = scenes.box_lattice(seed=1)
    ref = oracle.State(sc.params, sc.x, sc.v, sc.w, sc.r)
    with sim(sc.params, sc) as s:
        s.step(10)
        x10, v10, _ = s.state()
        ref.run(10)
        assert np.max(np.abs(x10 - ref.x)) <= 1e-12
        assert np.max(np.abs(v10 - ref.v)) <= 1e-9
        s.step(990)
        x1k, _, _ = s.state()
        ref.run(990)
        d = s.diagnostics()
    assert np.max(np.abs(x1k - ref.x)) <= 1e-9
    assert d["pair_contacts"] + d["wall_contacts"] > 0


def test_trajectory_fp32_short_horizon():
    """FP32 forces with compensated positions against the FP64 oracle over 200 steps:
    the position difference stays below 1e-5 of the largest displacement of the run
    (FP32 force error about 1e-6 relative, amplified by the collisions of the run)."""
    sc = scenes.box_lattice(seed=2)
    p = sc.params.copy(precision="fp32")
    ref = oracle.State(sc.params, sc.x, sc.v, sc.w, sc.r).run(200)
    with sim(p, sc) as s:
        s.step(200)
        x, v, _ = s.state()
    disp = np.max(np.linalg.norm(ref.x - sc.x, axis=1))
    assert np.max(np.abs(x - ref.x)) <= 1e-5 * disp
    assert np.max(np.abs(v - ref.v)) <= 1e-5 * np.max(np.abs(ref.v))


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_drum_short_run_matches_oracle(precision):
    sc = scenes.drum(seed=4, n=3001)
    p = sc.params.copy(precision=precision)
    ref = oracle.State(sc.params.copy(precision="fp64"), sc.x, sc.v, sc.w, sc.r).run(100)
    with sim(p, sc) as s:
        s.step(100)
        x, v, w = s.state()
    tol = 1e-12 if precision == "fp64" else 1e-9
    assert np.max(np.abs(x - ref.x)) <= tol
    assert np.max(np.abs(w - ref.w)) <= (1e-6 if precision == "fp64" else 5e-2)


# ------------------------------------------------------------ diagnostics, restore
def test_diagnostics_match_oracle():
    sc = scenes.box_lattice(seed=3)
    with sim(sc.params, sc) as s:
        s.step(50)
        x, v, w = s.state()
        d = s.diagnostics()
    o = oracle.diagnostics(sc.params, x, v, w, sc.r)
    names = dem.DIAG_NAMES[:10]
    for k, nm in enumerate(names):
        assert d[nm] == pytest.approx(o[k], rel=1e-12, abs=1e-18), nm
    assert d["steps"] == 50 and d["sorts"] == 51


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_checkpoint_restore_is_bit_exact(precision):
    """N steps, save state + springs, restore into a fresh handle, N more steps: the
    result equals 2N uninterrupted steps bit for bit."""
    sc = scenes.box_lattice(seed=4)
    p = sc.params.copy(precision=precision)
    with sim(p, sc) as a:
        a.step(150)
        xs, vs, ws = a.state()
        hist = a.history()
        a.step(150)
        xa, va, wa = a.state()
    assert len(hist) > 0
    h = dem.dem_create(dem.config_from_params(p))
    try:
        dem.dem_set_walls(h, p.walls)
        dem.dem_restore(h, xs, vs, ws, sc.r, hist)
        dem.dem_step(h, 150)
        xb, vb, wb = dem.dem_get_state(h, sc.n)
    finally:
        dem.dem_destroy(h)
    assert np.array_equal(xa, xb) and np.array_equal(va, vb) and np.array_equal(wa, wb)


# ------------------------------------------------------------ edge cases and errors
def test_empty_and_single_particle():
    sc = scenes.box_lattice(seed=1)
    z = np.zeros((0, 3))
    with dem.Simulation(sc.params, z, z, z, np.zeros(0, np.float32)) as s:
        s.step(3)
        x, _, _ = s.state()
        assert x.shape == (0, 3)
    x1 = np.array([[0.03, 0.03, 0.05]])
    v1 = np.array([[0.0, 0.0, 0.0]])
    with dem.Simulation(sc.params, x1, v1, v1, np.array([1e-3], np.float32)) as s:
        s.step(100)
        x, v, _ = s.state()
    ref = oracle.State(sc.params, x1, v1, v1, np.array([1e-3], np.float32)).run(100)
    assert np.max(np.abs(x - ref.x)) <= 1e-15 and np.max(np.abs(v - ref.v)) <= 1e-15


@pytest.mark.parametrize("block", [32, 64, 256])
def test_block_size_does_not_change_results(block):
    sc = scenes.box_rsa(seed=6, n=2500)
    p = sc.params.copy(precision="fp32")
    with sim(p, sc) as a:
        a.step(30)
        xa, va, _ = a.state()
    with sim(p, sc, block_size=block) as b:
        b.step(30)
        xb, vb, _ = b.state()
    assert np.array_equal(xa, xb) and np.array_equal(va, vb)


@pytest.mark.parametrize("block", [32, 96, 256])
def test_list_mode_block_size_does_not_change_results(block):
    """In list mode a particle's sums run over its own list in list order, so any block
    size gives the same bits."""
    sc = scenes.drum(seed=8, n=6000)
    v = np.random.default_rng(8).normal(0.0, 1.0, size=sc.x.shape)     # stirred: several sorts
    p = listed(sc.params.copy(precision="fp32"), skin_r=0.1, interval=0)
    with dem.Simulation(p, sc.x, v, sc.w, sc.r, block_size=256) as a:
        a.step(200)
        xa, va, wa = a.state()
        sorts = a.diagnostics()["sorts"]
    with dem.Simulation(p, sc.x, v, sc.w, sc.r, block_size=block) as b:
        b.step(200)
        xb, vb, wb = b.state()
    assert sorts > 2
    assert np.array_equal(xa, xb) and np.array_equal(va, vb) and np.array_equal(wa, wb)


@pytest.mark.parametrize("list_mode", [False, True])
def test_max_contacts_seen_counts_pairs_and_walls(list_mode):
    """dem_max_contacts_seen after one step = the largest per-particle count of contact
    partners (particles and walls) at the state the step started from."""
    sc = scenes.box_lattice(seed=1)
    x = compressed(sc, SQUEEZE["box2048"])
    p = listed(sc.params) if list_mode else sc.params
    pairs = oracle.pairs_brute(x, sc.r)
    cnt = np.bincount(pairs.ravel(), minlength=sc.n)
    for wl in sc.params.walls:
        s_ = (x - np.array(wl["p"])) @ np.array(wl["n"])
        cnt += (s_ < sc.r.astype(np.float64)).astype(np.int64)
    with dem.Simulation(p, x, sc.v, sc.w, sc.r) as s:
        s.step(1)
        seen = dem.dem_max_contacts_seen(s.h)
    assert seen == cnt.max() and seen > 3


@pytest.mark.parametrize("resort", [1, 0])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_contact_slot_overflow_grows_the_slots_and_reruns(resort, precision):
    """A step in which a particle has more contacts than its slots is voided on the
    device; dem_step doubles the slots (1 -> 2 -> 4 -> 8 here, one void step each) and
    runs it again, so every bit of the state and of the springs equals a run that had
    enough slots from the start. Walk mode and list mode."""
    sc = scenes.box_lattice(seed=1, precision=precision)
    x = compressed(sc, 0.95)          # six face neighbours in contact, plus walls
    p = sc.params if resort == 1 else listed(sc.params)

    def run(maxc):
        h = dem.dem_create(dem.config_from_params(p, max_contacts=maxc))
        try:
            dem.dem_set_walls(h, p.walls)
            dem.dem_set_particles(h, x, sc.v, sc.w, sc.r)
            b0 = dem.dem_device_bytes(h)
            dem.dem_step(h, 30)
            st = dem.dem_get_state(h, sc.n)
            d = dem.dem_get_diagnostics(h)
            return st, dem.dem_get_history(h), dem.dem_device_bytes(h) - b0, d[13], dem.dem_max_contacts_seen(h)
        finally:
            dem.dem_destroy(h)

    small, big = run(1), run(32)
    for a, b in zip(small[0], big[0]):
        assert np.array_equal(a, b)
    assert np.array_equal(small[1], big[1])
    assert small[2] > 0 and big[2] == 0      # the slots grew; 32 was enough
    assert small[3] == big[3] == 30          # steps taken
    assert 4 < small[4] <= 8


def test_contact_overflow_past_64_keeps_the_state_before_the_step():
    """A sphere of five radii with 80 small spheres pressed onto it: more contacts than
    the largest capacity (64). dem_step grows the slots to 64, still overflows, and
    reports DEM_ERR_CAPACITY with the state that the step started from; the handle stays
    usable."""
    rs, rb, m = 1e-3, 5e-3, 80
    k = np.arange(m) + 0.5
    th = np.arccos(1.0 - 2.0 * k / m)
    ph = np.pi * (1.0 + 5.0 ** 0.5) * k
    u = np.stack([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)], axis=1)
    c = np.array([0.032, 0.032, 0.032])
    x = np.vstack([c, c + u * (rb + rs - 1e-6)])
    n = len(x)
    v = np.zeros((n, 3)); w = np.zeros((n, 3))
    r = np.full(n, rs, dtype=np.float32); r[0] = rb
    sc = scenes.box_lattice(seed=1)
    p = sc.params.copy(g=(0.0, 0.0, 0.0), cell_size=2.0 * rb * (1.0 + 2.0 ** -9), walls=[])
    h = dem.dem_create(dem.config_from_params(p, max_contacts=32))
    try:
        dem.dem_set_particles(h, x, v, w, r)
        b0 = dem.dem_device_bytes(h)
        with pytest.raises(dem.DemError) as e:
            dem.dem_step(h, 5)
        assert e.value.status == dem.DEM_ERR_CAPACITY and "64" in str(e.value)
        xs, vs, ws = dem.dem_get_state(h, n)
        assert np.array_equal(xs, x) and np.array_equal(vs, v) and np.array_equal(ws, w)
        assert dem.dem_device_bytes(h) > b0
        assert dem.dem_get_diagnostics(h)[13] == 0
        # usable afterwards: the small spheres alone, moving, run like the oracle
        v2 = np.random.default_rng(3).normal(0.0, 0.5, size=(n - 1, 3))
        dem.dem_set_particles(h, x[1:], v2, w[1:], r[1:])
        dem.dem_step(h, 10)
        x10, _, _ = dem.dem_get_state(h, n - 1)
    finally:
        dem.dem_destroy(h)
    ref = oracle.State(p, x[1:], v2, w[1:], r[1:]).run(10)
    assert np.max(np.abs(x10 - ref.x)) <= 1e-12


def test_invalid_inputs_are_rejected():
    sc = scenes.box_lattice(seed=1)
    x = sc.x.copy()
    x[5, 1] = np.nan
    h = dem.dem_create(dem.config_from_params(sc.params))
    try:
        with pytest.raises(dem.DemError) as e:
            dem.dem_set_particles(h, x, sc.v, sc.w, sc.r)
        assert e.value.status == 1
        with pytest.raises(dem.DemError) as e:
            dem.dem_step(h, 1)
        assert e.value.status == 7
        r = sc.r.copy()
        r[3] = 0
        with pytest.raises(dem.DemError):
            dem.dem_set_particles(h, sc.x, sc.v, sc.w, r)
        small = sc.params.copy(cell_size=1.5e-3)
        h2 = dem.dem_create(dem.config_from_params(small))
        try:
            with pytest.raises(dem.DemError):
                dem.dem_set_particles(h2, sc.x, sc.v, sc.w, sc.r)
        finally:
            dem.dem_destroy(h2)
    finally:
        dem.dem_destroy(h)


@pytest.mark.parametrize("where", ["host", "device"])
def test_input_check_on_the_device(where):
    """dem_set_particles checks its arrays on the device, host and device inputs alike:
    each kind of bad value (first, middle and last particle) is rejected with its reason,
    and a good call after a rejected one gives the oracle's run."""
    import torch
    sc = scenes.box_lattice(seed=2)
    n = sc.n
    bad = [("x", (0, 2), np.inf, "non-finite"), ("v", (n // 2, 0), np.nan, "non-finite"),
           ("w", (n - 1, 1), -np.inf, "non-finite"), ("r", 0, np.nan, "radii"), ("r", n // 3, -1e-3, "radii"),
           ("r", n - 1, np.inf, "radii"), ("r", 5, 0.0, "radii")]
    h = dem.dem_create(dem.config_from_params(sc.params))
    try:
        dem.dem_set_walls(h, sc.params.walls)
        for name, idx, val, why in bad:
            a = {"x": sc.x.copy(), "v": sc.v.copy(), "w": sc.w.copy(), "r": sc.r.copy()}
            a[name][idx] = val
            args = [a["x"], a["v"], a["w"], a["r"]]
            if where == "device":
                args = [torch.tensor(t, device="cuda:0") for t in args]
            with pytest.raises(dem.DemError) as e:
                dem.dem_set_particles(h, *args)
            assert e.value.status == dem.DEM_ERR_INVALID_ARG and why in str(e.value), (name, idx, str(e.value))
        args = [sc.x, sc.v, sc.w, sc.r]
        if where == "device":
            args = [torch.tensor(t, device="cuda:0") for t in args]
        dem.dem_set_particles(h, *args)
        dem.dem_step(h, 20)
        x, _, _ = dem.dem_get_state(h, n)
    finally:
        dem.dem_destroy(h)
    ref = oracle.State(sc.params, sc.x, sc.v, sc.w, sc.r).run(20)
    assert np.max(np.abs(x - ref.x)) <= 1e-12


def test_device_pointer_inputs_and_outputs():
    import torch
    sc = scenes.box_lattice(seed=7)
    dev = torch.device("cuda:0")
    X = torch.tensor(sc.x, device=dev)
    V = torch.tensor(sc.v, device=dev)
    W = torch.tensor(sc.w, device=dev)
    R = torch.tensor(sc.r, device=dev)
    h = dem.dem_create(dem.config_from_params(sc.params))
    try:
        dem.dem_set_walls(h, sc.params.walls)
        dem.dem_set_particles(h, X, V, W, R)
        dem.dem_step(h, 20)
        xo = torch.empty_like(X); vo = torch.empty_like(V); wo = torch.empty_like(W)
        dem.dem_get_state(h, sc.n, xo, vo, wo)
        torch.cuda.synchronize()
    finally:
        dem.dem_destroy(h)
    ref = oracle.State(sc.params, sc.x, sc.v, sc.w, sc.r).run(20)
    assert np.max(np.abs(xo.cpu().numpy() - ref.x)) <= 1e-12


# ------------------------------------------------------------ skin / re-sort interval
def listed(params, skin_r=0.1, interval=0):
    skin = skin_r * 1e-3
    cs = params.cell_size + skin
    return params.copy(resort_interval=interval, skin=skin, cell_size=cs)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_list_mode_trajectory_matches_oracle(precision):
    """Sorting only when a particle has moved skin/2 (with neighbour lists built at each
    sort) finds exactly the same contacts, so the run follows the oracle as closely as
    the sort-every-step run does."""
    sc = scenes.box_lattice(seed=1)
    p = listed(sc.params.copy(precision=precision))
    ref = oracle.State(sc.params, sc.x, sc.v, sc.w, sc.r)
    with sim(p, sc) as s:
        s.step(10)
        x10, _, _ = s.state()
        ref.run(10)
        if precision == "fp64":
            assert np.max(np.abs(x10 - ref.x)) <= 1e-12
        s.step(490)
        x, v, _ = s.state()
        d = s.diagnostics()
    ref.run(490)
    disp = np.max(np.linalg.norm(ref.x - sc.x, axis=1))
    tol = 1e-9 if precision == "fp64" else 1e-5 * disp
    assert np.max(np.abs(x - ref.x)) <= tol
    assert 1 < d["sorts"] < 250      # far fewer sorts than steps
    assert d["pair_contacts"] + d["wall_contacts"] > 0


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_list_mode_drum_matches_oracle(precision):
    sc = scenes.drum(seed=5, n=3001)
    p = listed(sc.params.copy(precision=precision), skin_r=0.05, interval=25)
    ref = oracle.State(sc.params.copy(precision="fp64"), sc.x, sc.v, sc.w, sc.r).run(120)
    with sim(p, sc) as s:
        s.step(120)
        x, v, w = s.state()
        d = s.diagnostics()
    tol = 1e-12 if precision == "fp64" else 1e-9
    assert np.max(np.abs(x - ref.x)) <= tol
    assert d["sorts"] >= 120 // 25


@pytest.mark.parametrize("model,stiff", [("practical", "hertz"), ("simple", "linear")])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_list_mode_other_laws_match_oracle(model, stiff, precision):
    """Neighbour lists with the Hertz law (Eqs. 8-9) and with the simple law (Eq. 1):
    FP64 follows the oracle to 1e-12 m after 10 steps and 1e-9 m after 300; FP32 stays
    as close to the oracle as the sort-every-step FP32 run (whose difference from the
    oracle is FP32 rounding amplified by the collisions)."""
    sc = scenes.box_lattice(seed=4, stiffness=stiff, model=model)
    base = sc.params
    p = listed(base.copy(precision=precision))
    ref = oracle.State(base, sc.x, sc.v, sc.w, sc.r)
    with sim(p, sc) as s:
        s.step(10)
        x10, _, _ = s.state()
        ref.run(10)
        if precision == "fp64":
            assert np.max(np.abs(x10 - ref.x)) <= 1e-12
        s.step(290)
        x, _, _ = s.state()
        d = s.diagnostics()
    ref.run(290)
    err = np.max(np.abs(x - ref.x))
    if precision == "fp64":
        assert err <= 1e-9
    else:
        with sim(base.copy(precision="fp32"), sc) as s:
            s.step(300)
            xw, _, _ = s.state()
        err_walk = np.max(np.abs(xw - ref.x))
        disp = np.max(np.linalg.norm(ref.x - sc.x, axis=1))
        assert err <= 2.0 * err_walk + 1e-6 * disp, (err, err_walk)
    assert d["pair_contacts"] + d["wall_contacts"] > 0


def test_list_mode_pairs_equal_sort_every_step_pairs():
    """After many list-mode steps, the contact pairs found through the lists equal those
    found by a fresh 27-cell walk of the same state (GPU against GPU)."""
    sc = scenes.drum(seed=6, n=6000)
    p = listed(sc.params, skin_r=0.2)
    with sim(p, sc) as s:
        s.step(300)
        x, v, w = s.state()
        hist = s.history()
        s.forces()
        _, _, pl = s.snapshot()
        d = s.diagnostics()
    assert d["sorts"] < 300
    h = dem.dem_create(dem.config_from_params(sc.params))
    try:
        dem.dem_set_walls(h, sc.params.walls)
        dem.dem_restore(h, x, v, w, sc.r, hist)
        dem.dem_get_forces(h, sc.n)
        _, _, pw, = dem.dem_debug_snapshot(h, sc.n)
    finally:
        dem.dem_destroy(h)
    assert len(pl) > 1000
    assert np.array_equal(pl, pw)


def test_list_mode_checkpoint_restore_bit_exact():
    sc = scenes.box_lattice(seed=8)
    p = listed(sc.params.copy(precision="fp32"))
    with sim(p, sc) as a:
        a.step(100)
        xs, vs, ws = a.state()
        hist = a.history()
        a.step(100)
        xa, _, _ = a.state()
    # the restored run sorts at its start, so compare against a sort-every-step
    # continuation only through the oracle tolerance, and against itself exactly
    outs = []
    for _ in range(2):
        h = dem.dem_create(dem.config_from_params(p))
        try:
            dem.dem_set_walls(h, p.walls)
            dem.dem_restore(h, xs, vs, ws, sc.r, hist)
            dem.dem_step(h, 100)
            outs.append(dem.dem_get_state(h, sc.n)[0])
        finally:
            dem.dem_destroy(h)
    assert np.array_equal(outs[0], outs[1])
    assert np.max(np.abs(outs[0] - xa)) <= 1e-9


# ------------------------------------------------------------ statistics
def test_settling_statistics_match_oracle():
    """Loose random fill settling under gravity (the 262,144-sphere box's family, 3,000
    spheres): FP32 mode against the FP64 oracle, kinetic energy at every 100th step and
    the solid fraction of the bottom region at the end within 1%."""
    sc = scenes.box_rsa(seed=12, n=3000)
    p32 = sc.params.copy(precision="fp32")
    ref = oracle.State(sc.params.copy(precision="fp64"), sc.x, sc.v, sc.w, sc.r)
    ke_g, ke_o = [], []
    with sim(p32, sc) as s:
        for _ in range(10):
            s.step(100)
            ke_g.append(s.diagnostics()["ke_trans"])
            ref.run(100, pair_mode="grid")
            ke_o.append(oracle.diagnostics(ref.params, ref.x, ref.v, ref.w, ref.r)[0])
        xg, _, _ = s.state()
    ke_g, ke_o = np.array(ke_g), np.array(ke_o)
    assert np.all(np.abs(ke_g - ke_o) <= 0.01 * ke_o)

    def bottom_phi(x):
        h = 20 * 1e-3
        sel = x[:, 2] < h
        vol = np.sum(4.0 / 3.0 * np.pi * sc.r[sel].astype(np.float64) ** 3)
        lo, hi = sc.params.domain_lo, sc.params.domain_hi
        return vol / ((hi[0] - lo[0]) * (hi[1] - lo[1]) * h)

    assert bottom_phi(xg) == pytest.approx(bottom_phi(ref.x), rel=0.01)
