"""Pins of the FP64 oracle against things the paper and mechanics fix independently of it.

Each test names the equation it pins and the closed form or invariant it checks. None
of them retypes the oracle's force law: they check contact durations, restitution,
Hertz peak overlaps, rolling/sliding kinematics, energy and momentum balances, cell
geometry and brute force against the grid.
"""
import math
import os

import numpy as np
import pytest

import oracle
from paper_1301_1714_gb300 import scenes as S

R = 1e-3
RF = float(np.float32(R))     # the radius as stored (FP32)
RHO = 2500.0
M = RHO * 4.0 / 3.0 * math.pi * RF ** 3


def test_oracle_records_match_their_mirrors():
    assert oracle.struct_sizes_match()


def params(**kw):
    base = dict(model="practical", stiffness="linear", precision="fp64", dt=1e-6, g=(0.0, 0.0, 0.0), kn=1e4,
                kt=1e4 * 2 / 7, alpha=0.0, mu=0.3, cell_size=S.auto_cell_size(R), domain_lo=(-0.05, -0.05, -0.05),
                domain_hi=(0.05, 0.05, 0.05), walls=[])
    base.update(kw)
    return S.Params(**base)


def two_spheres(gap, vrel, r=R):
    """Spheres 0 and 1 on the x axis, surface gap `gap`, approaching at relative speed vrel."""
    x = np.array([[-r - gap / 2, 0.0, 0.0], [r + gap / 2, 0.0, 0.0]])
    v = np.array([[vrel / 2, 0.0, 0.0], [-vrel / 2, 0.0, 0.0]])
    w = np.zeros((2, 3))
    rad = np.full(2, r, dtype=np.float32)
    return x, v, w, rad


def collide(p, vrel, max_steps=200000):
    """Run a head-on collision; return (contact duration, restitution, max overlap)."""
    x, v, w, r = two_spheres(1e-7, vrel)
    st = oracle.State(p, x, v, w, r)
    steps_in = 0
    maxov = 0.0
    touched = False
    for _ in range(max_steps):
        st.run(1)
        npairs = st.stats[0]
        if npairs > 0:
            touched = True
            steps_in += 1
            maxov = max(maxov, st.stats[2])
        elif touched:
            break
    vout = st.v[1, 0] - st.v[0, 0]
    return steps_in * p.dt, vout / vrel, maxov


# ------------------------------------------------------------------ Eqs. 4, 10
@pytest.mark.parametrize("e", [0.9, 0.5])
def test_linear_head_on_duration_and_restitution(e):
    """Linear spring-dashpot head-on contact: m_eff x'' = -k x - eta x' gives
    t_c = pi / sqrt(k/m_eff - (eta/2m_eff)^2) and e = exp(-zeta pi / sqrt(1 - zeta^2)),
    zeta = eta / (2 sqrt(k m_eff)). Pins Eq. 4 (normal part), Eq. 10 and the integrator."""
    meff = M / 2
    zeta = -math.log(e) / math.sqrt(math.pi ** 2 + math.log(e) ** 2)
    eta = 2 * zeta * math.sqrt(1e4 * meff)
    tc = math.pi / math.sqrt(1e4 / meff - (eta / (2 * meff)) ** 2)
    e_closed = math.exp(-zeta * math.pi / math.sqrt(1 - zeta ** 2))
    assert e_closed == pytest.approx(e, rel=1e-12)
    # Eq. 10: eta = alpha sqrt(k_n m_eff) -> alpha = 2 zeta
    assert S.alpha_from_e(e) == pytest.approx(2 * zeta, rel=1e-12)
    p = params(alpha=2 * zeta, dt=tc / 50)
    t, ecoef, _ = collide(p, 0.2)
    assert t == pytest.approx(tc, rel=0.02)
    assert ecoef == pytest.approx(e, rel=0.02)
    # first-order convergence toward the closed form as dt shrinks
    p2 = params(alpha=2 * zeta, dt=tc / 1000)
    t2, e2, _ = collide(p2, 0.2)
    assert abs(t2 - tc) / tc < 0.002
    assert abs(e2 - e) / e < 0.001


def test_simple_model_head_on_matches_same_ode():
    """Eq. 1 head-on: -k_sp delta n - k_da v with v along n is the same ODE, so the same
    closed-form t_c and e hold with eta = k_da."""
    e = 0.8
    meff = M / 2
    zeta = -math.log(e) / math.sqrt(math.pi ** 2 + math.log(e) ** 2)
    eta = 2 * zeta * math.sqrt(1e4 * meff)
    tc = math.pi / math.sqrt(1e4 / meff - (eta / (2 * meff)) ** 2)
    p = params(model="simple", ksp=1e4, kda=eta, ksh=eta, dt=tc / 1000)
    t, ecoef, _ = collide(p, 0.2)
    assert abs(t - tc) / tc < 0.002
    assert abs(ecoef - e) / e < 0.001


# ------------------------------------------------------------------- Eqs. 8-9
def test_hertz_undamped_peak_overlap_and_duration():
    """Eqs. 8-9 give F = C_n sqrt(R_eff) delta^(3/2). Undamped: delta_max =
    (5 m_eff v^2 / (4 K))^(2/5) and t_c = 2 (delta_max / v) * (2/5) B(2/5, 1/2)."""
    cn, ct = S.hertz_coeffs(1e4, 2 / 7, R)
    reff = R / 2
    K = cn * math.sqrt(reff)
    meff = M / 2
    v = 0.2
    dmax = (5 * meff * v * v / (4 * K)) ** 0.4
    beta = math.gamma(0.4) * math.gamma(0.5) / math.gamma(0.9)
    tc = 2 * dmax / v * 0.4 * beta
    p = params(stiffness="hertz", cn=cn, ct=ct, alpha=0.0, dt=tc / 2000)
    t, ecoef, maxov = collide(p, v)
    assert maxov == pytest.approx(dmax, rel=2e-3)
    assert t == pytest.approx(tc, rel=2e-3)
    assert ecoef == pytest.approx(1.0, abs=2e-3)


def test_hertz_damped_restitution_independent_of_speed():
    """With eta = alpha sqrt(k_n m_eff) and Hertz k_n (Eqs. 8-10) the equation of motion
    is self-similar in the impact speed, so e does not depend on it."""
    cn, ct = S.hertz_coeffs(1e4, 2 / 7, R)
    es = []
    for v in (0.05, 0.2, 0.8):
        meff = M / 2
        K = cn * math.sqrt(R / 2)
        dmax = (5 * meff * v * v / (4 * K)) ** 0.4
        tc = 2.943 * dmax / v
        p = params(stiffness="hertz", cn=cn, ct=ct, alpha=0.3, dt=tc / 2000)
        _, ecoef, _ = collide(p, v)
        es.append(ecoef)
    assert max(es) - min(es) < 0.005 * np.mean(es)
    assert es[0] < 0.99


# ---------------------------------------------------------- energy and momentum
def pair_potential(p, x, r):
    """Elastic energy stored in normal springs (linear: k delta^2 / 2), pairs and planes."""
    n = len(r)
    e = 0.0
    for i in range(n):
        for j in range(i + 1, n):
            d = np.linalg.norm(x[j] - x[i])
            delta = float(r[i]) + float(r[j]) - d
            if delta > 0:
                e += 0.5 * p.kn * delta * delta
    for wl in p.walls:
        nn = np.array(wl["n"]); pp = np.array(wl["p"])
        s = (x - pp) @ nn
        delta = r.astype(np.float64) - s
        e += 0.5 * p.kn * float(np.sum(np.where(delta > 0, delta * delta, 0.0)))
    return e


def total_energy(p, st):
    d = oracle.diagnostics(p, st.x, st.v, st.w, st.r)
    return d[0] + d[1] + d[8] + pair_potential(p, st.x, st.r), d[0]


def _energy_drift(dt, steps):
    lo, hi = (0.0, 0.0, 0.0), (10 * R, 10 * R, 10 * R)
    sc = S.box_lattice(3, 4, 4, 4, r=R, box=(10.0, 10.0, 10.0), spacing=2.05, jitter=0.01, vsigma=0.3)
    p = params(alpha=0.0, mu=0.0, dt=dt, g=(0.0, 0.0, -9.81), domain_lo=lo, domain_hi=hi, walls=S.box_walls(lo, hi))
    st = oracle.State(p, sc.x, sc.v, sc.w, sc.r)
    e0, ke0 = total_energy(p, st)
    worst = 0.0
    for _ in range(steps):
        st.run(1)
        e, _ = total_energy(p, st)
        worst = max(worst, abs(e - e0))
    return worst / ke0


def test_energy_conserved_without_dissipation():
    """eta = 0 and mu = 0 (no dissipation, Eqs. 4-5): the semi-implicit Euler step is
    symplectic, so the total energy (kinetic + rotational + gravity + springs) shows no
    drift and its error is first order in dt."""
    tc = math.pi / math.sqrt(1e4 / (M / 2))
    e1 = _energy_drift(tc / 50, 1500)
    e2 = _energy_drift(tc / 100, 3000)
    assert e1 < 0.05
    assert 1.5 < e1 / e2 < 2.6


def test_momentum_conserved_and_angular_momentum_drift_bounded():
    """Without walls and gravity, pair forces are equal and opposite (Eq. 2), so linear
    momentum is conserved to round-off. With the lever arm r_i of Eq. 3, each pair adds
    dt * delta * (n x F_t) to the angular momentum, bounded by dt * delta * mu |F_n|."""
    sc = S.box_lattice(5, 5, 5, 4, r=R, box=(12.0, 12.0, 10.0), spacing=2.02, jitter=0.01, vsigma=0.5)
    rng = np.random.default_rng(0)
    w0 = rng.normal(0, 50.0, size=(len(sc.r), 3))
    e = 0.7
    p = params(alpha=S.alpha_from_e(e), mu=0.4, dt=1e-6, domain_lo=(0, 0, 0), domain_hi=(0.012, 0.012, 0.010))
    st = oracle.State(p, sc.x, sc.v, w0, sc.r)
    d0 = oracle.diagnostics(p, st.x, st.v, st.w, st.r)
    scale = float(np.sum(M * np.linalg.norm(st.v, axis=1)))
    any_contacts = 0
    for _ in range(400):
        pairs = oracle.pairs_brute(st.x, st.r)
        bound = 0.0
        meff = M / 2
        for i, j in pairs:
            dvec = st.x[j] - st.x[i]
            d = np.linalg.norm(dvec)
            n = dvec / d
            delta = float(st.r[i]) + float(st.r[j]) - d
            vn = abs(np.dot(st.v[i] - st.v[j], n))
            eta = p.alpha * math.sqrt(p.kn * meff)
            bound += delta * p.mu * (p.kn * delta + eta * vn)
        any_contacts += len(pairs)
        dA = oracle.diagnostics(p, st.x, st.v, st.w, st.r)
        st.run(1)
        dB = oracle.diagnostics(p, st.x, st.v, st.w, st.r)
        dL = np.linalg.norm(dB[5:8] - dA[5:8])
        assert dL <= p.dt * bound * (1 + 1e-6) + 1e-20
    d1 = oracle.diagnostics(p, st.x, st.v, st.w, st.r)
    assert any_contacts > 100
    assert np.max(np.abs(d1[2:5] - d0[2:5])) < 1e-13 * scale


# ------------------------------------------------- tangential law (Eqs. 3, 5-7)
def floor_params(mu, e, **kw):
    lo, hi = (-0.05, -0.05, 0.0), (0.05, 0.05, 0.05)
    walls = [dict(kind="plane", p=(0.0, 0.0, 0.0), n=(0.0, 0.0, 1.0))]
    tc = math.pi / math.sqrt(1e4 / M)
    base = dict(alpha=S.alpha_from_e(e), mu=mu, dt=tc / 50, g=(0.0, 0.0, -9.81), domain_lo=lo, domain_hi=hi,
                walls=walls)
    base.update(kw)
    return params(**base)


def test_resting_sphere_overlap_equals_weight_over_stiffness():
    """A sphere resting on a plane wall (step 8) settles at delta = m g / k_n."""
    p = floor_params(0.3, 0.3)
    st = oracle.State(p, np.array([[0.0, 0.0, R * 1.001]]), np.zeros((1, 3)), np.zeros((1, 3)),
                      np.full(1, R, np.float32))
    st.run(40000)
    delta = RF - st.x[0, 2]
    assert delta == pytest.approx(M * 9.81 / 1e4, rel=1e-3)


def test_sliding_sphere_ends_rolling_at_five_sevenths():
    """Kinetic friction (Eq. 5) decelerates a sliding sphere and its torque (Eq. 3) spins it
    up; slip (Eq. 6) stops at t = 2 v0 / (7 mu g) with v = (5/7) v0 and w r = v."""
    mu, v0 = 0.3, 0.1
    p = floor_params(mu, 0.5)
    z0 = R - M * 9.81 / 1e4
    st = oracle.State(p, np.array([[0.0, 0.0, z0]]), np.array([[v0, 0.0, 0.0]]), np.zeros((1, 3)),
                      np.full(1, R, np.float32))
    t_roll = 2 * v0 / (7 * mu * 9.81)
    steps = int(1.5 * t_roll / p.dt)
    t_stop = None
    for k in range(steps):
        st.run(1)
        slip = st.v[0, 0] - st.w[0, 1] * R
        if t_stop is None and abs(slip) < 0.01 * v0:
            t_stop = (k + 1) * p.dt
    assert st.v[0, 0] == pytest.approx(5 / 7 * v0, rel=0.02)
    assert st.w[0, 1] * R == pytest.approx(st.v[0, 0], rel=0.02)
    assert t_stop == pytest.approx(t_roll, rel=0.03)


def test_moving_wall_drags_sphere_to_two_sevenths():
    """The wall's surface velocity replaces the partner's in Eq. 6: a sphere at rest on a
    belt moving at u ends up rolling at (2/7) u."""
    u = 0.1
    p = floor_params(0.4, 0.5)
    p.walls[0]["vel"] = (u, 0.0, 0.0)
    z0 = R - M * 9.81 / 1e4
    st = oracle.State(p, np.array([[0.0, 0.0, z0]]), np.zeros((1, 3)), np.zeros((1, 3)), np.full(1, R, np.float32))
    t_star = 2 * u / (7 * 0.4 * 9.81)
    st.run(int(1.5 * t_star / p.dt))
    assert st.v[0, 0] == pytest.approx(2 / 7 * u, rel=0.02)


def test_rotating_drum_drags_sphere_to_two_sevenths_of_rim_speed():
    """Cylinder wall with angular velocity Omega about its axis: for short times the rim
    acts as a belt of speed Omega R_d, so a sphere at rest at the bottom reaches
    (2/7) Omega R_d. Also checks the resting overlap delta = m g / k_n inside a static drum."""
    Rd = 0.05
    lo, hi = (-0.01, -Rd, -Rd), (0.01, Rd, Rd)
    static = [dict(kind="cylinder", p=(0.0, 0.0, 0.0), n=(1.0, 0.0, 0.0), radius=Rd)]
    p = floor_params(0.5, 0.3, domain_lo=lo, domain_hi=hi, walls=static)
    st = oracle.State(p, np.array([[0.0, 0.0, -Rd + R * 1.001]]), np.zeros((1, 3)), np.zeros((1, 3)),
                      np.full(1, R, np.float32))
    st.run(40000)
    assert (st.x[0, 2] - RF) - (-Rd) == pytest.approx(-M * 9.81 / 1e4, rel=2e-3)
    Om = 2.0
    rot = [dict(kind="cylinder", p=(0.0, 0.0, 0.0), n=(1.0, 0.0, 0.0), radius=Rd, omega=(Om, 0.0, 0.0))]
    p2 = floor_params(0.5, 0.3, domain_lo=lo, domain_hi=hi, walls=rot)
    st2 = oracle.State(p2, st.x, np.zeros((1, 3)), np.zeros((1, 3)), st.r)
    u = Om * Rd
    t_star = 2 * u / (7 * 0.5 * 9.81)
    st2.run(int(1.3 * t_star / p2.dt))
    # the rim at the bottom, c = (0, 0, -Rd), moves at Omega x c = (0, +Omega Rd, 0)
    assert st2.v[0, 1] == pytest.approx(2 / 7 * u, rel=0.03)


@pytest.mark.parametrize("theta_deg,mu,rolling", [(10.0, 0.3, True), (60.0, 0.2, False)])
def test_incline_rolls_or_slides(theta_deg, mu, rolling):
    """On an incline a sphere rolls without slipping iff tan(theta) <= (7/2) mu, with
    acceleration (5/7) g sin(theta); otherwise it slides with g (sin(theta) - mu cos(theta))."""
    th = math.radians(theta_deg)
    g = 9.81
    nrm = (-math.sin(th), 0.0, math.cos(th))
    lo, hi = (-0.05, -0.05, -0.05), (0.05, 0.05, 0.05)
    walls = [dict(kind="plane", p=(0.0, 0.0, 0.0), n=nrm)]
    p = floor_params(mu, 0.3, domain_lo=lo, domain_hi=hi, walls=walls)
    s0 = R - M * g * math.cos(th) / 1e4
    x0 = np.array([[s0 * nrm[0], 0.0, s0 * nrm[2]]])
    st = oracle.State(p, x0, np.zeros((1, 3)), np.zeros((1, 3)), np.full(1, R, np.float32))
    down = np.array([-math.cos(th), 0.0, -math.sin(th)])
    st.run(int(2e-3 / p.dt))
    v1 = float(st.v[0] @ down)
    n2 = int(4e-3 / p.dt)
    st.run(n2)
    v2 = float(st.v[0] @ down)
    a = (v2 - v1) / (n2 * p.dt)
    expect = 5 / 7 * g * math.sin(th) if rolling else g * (math.sin(th) - mu * math.cos(th))
    assert (math.tan(th) <= 3.5 * mu) == rolling
    assert a == pytest.approx(expect, rel=0.02)


def test_coulomb_cap_and_history_projection():
    """Eq. 5: |F_t| never exceeds mu |F_n|, and equals it while slipping. Eq. 7: the
    stored tangential spring is always perpendicular to the current normal."""
    p = params(alpha=S.alpha_from_e(0.7), mu=0.25, dt=1e-6)
    x, v, w, r = two_spheres(-2e-6, 0.0)
    v = np.array([[0.0, 0.05, 0.0], [0.0, -0.05, 0.01]])
    w = np.array([[0.0, 0.0, 30.0], [10.0, 0.0, 0.0]])
    st = oracle.State(p, x, v, w, r)
    for _ in range(200):
        F, T, hist, _ = oracle.forces(p, st.x, st.v, st.w, st.r, st.history)
        if len(hist) == 0:
            break
        n = st.x[1] - st.x[0]
        n /= np.linalg.norm(n)
        Fn = np.dot(F[0], n) * n
        Ft = F[0] - Fn
        assert np.linalg.norm(Ft) <= p.mu * np.linalg.norm(Fn) * (1 + 1e-12) + 1e-18
        d = hist[0]["d"]
        assert abs(np.dot(d, n)) <= 1e-12 * max(np.linalg.norm(d), 1e-30)
        # torque: T_i = r_i n x F_t and T_j = r_j n x F_t (Eq. 3) are parallel, same sign
        assert np.allclose(T[0], T[1], rtol=1e-12, atol=1e-30)
        st.run(1)


def test_newton_third_law_per_step():
    """Eq. 2 with F_j = -F_i: without walls the forces of a step sum to the total weight."""
    sc = S.box_lattice(9, 4, 4, 4, r=R, box=(9.0, 9.0, 9.0), spacing=1.98, jitter=0.005, vsigma=0.2)
    p = params(alpha=S.alpha_from_e(0.6), mu=0.5, g=(0.0, 0.0, -9.81), domain_lo=(0, 0, 0),
               domain_hi=(0.009, 0.009, 0.009))
    F, T, hist, stats = oracle.forces(p, sc.x, sc.v, sc.w, sc.r)
    assert stats[0] > 50
    total = F.sum(axis=0)
    assert total[2] == pytest.approx(-9.81 * M * len(sc.r), rel=1e-12)
    assert abs(total[0]) < 1e-14 and abs(total[1]) < 1e-14


# ----------------------------------------------------- broad phase (Sec. 4)
def test_cell_hash_hand_values():
    """CM: floor((x - o)/h), clamped to the grid (Sec. 4.1, step 2), key (k ny + j) nx + i."""
    p = params(cell_size=0.01, domain_lo=(0.0, 0.0, 0.0), domain_hi=(0.05, 0.03, 0.02))
    assert oracle.grid_dims(p) == (5, 3, 2)
    x = np.array([[0.025, 0.015, 0.005], [-0.1, 0.0, 0.0], [0.07, 0.029999, 0.0199], [0.01, 0.02, 0.01]])
    key, ijk = oracle.cell_keys(p, x)
    assert ijk.tolist() == [[2, 1, 0], [0, 0, 0], [4, 2, 1], [1, 2, 1]]
    assert key.tolist() == [7, 0, 4 + 5 * (2 + 3 * 1), 1 + 5 * (2 + 3 * 1)]


def test_fp32_hash_mode_rounds_in_fp32():
    """In hash mode 1 the cell is floor(fl32(fl32(x) - fl32(o)) / fl32(h)): a position just
    below a cell face in FP64 can land in the upper cell after rounding to FP32."""
    p64 = params(cell_size=0.25, domain_lo=(0.0, 0.0, 0.0), domain_hi=(1.0, 1.0, 1.0))
    p32 = p64.copy(precision="fp32")
    x = np.array([[0.5 - 1e-12, 0.1, 0.1]])
    assert oracle.cell_keys(p64, x)[1][0, 0] == 1
    assert oracle.cell_keys(p32, x)[1][0, 0] == 2


def test_sort_by_cell_and_cell_start():
    """Eq. 11: SCM[j] = CM[SCCM[j]], ties broken by id; cell c holds sorted positions
    start[c] .. start[c+1]-1."""
    key = np.array([3, 1, 3, 0, 1], dtype=np.uint64)
    order, skey = oracle.sort_by_cell(key)
    assert order.tolist() == [3, 1, 4, 0, 2]
    assert np.array_equal(skey, key[order])
    start = oracle.cell_start(skey, 5)
    assert start.tolist() == [0, 1, 3, 3, 5, 5]


def test_contact_predicate_is_strict_and_brute_equals_grid():
    """Contact iff d < r_i + r_j (touching is not contact); the grid search (Eq. 12) finds
    exactly the brute-force pair set, including pairs one ulp from touching."""
    rng = np.random.default_rng(7)
    n = 600
    x = rng.uniform(0.0, 0.03, size=(n, 3))
    r = rng.uniform(0.8e-3, 1.2e-3, size=n).astype(np.float32)
    # plant touching / one-ulp pairs along x
    for k in range(0, 60, 3):
        Rk = float(r[k]) + float(r[k + 1])
        base = x[k].copy()
        x[k + 1] = base + np.array([Rk, 0.0, 0.0])
        x[k + 2] = base + np.array([0.0, np.nextafter(Rk, 0.0), 0.0])
    p = params(cell_size=S.auto_cell_size(float(r.max())), domain_lo=(0.0, 0.0, 0.0), domain_hi=(0.03, 0.03, 0.03))
    pb = oracle.pairs_brute(x, r)
    pg = oracle.pairs_grid(p, x, r)
    assert np.array_equal(pb, pg)
    s = set(map(tuple, pb.tolist()))
    for k in range(0, 60, 3):
        touching = float(np.sum((x[k + 1] - x[k]) ** 2)) < (float(r[k]) + float(r[k + 1])) ** 2
        assert ((k, k + 1) in s) == touching
        assert (k, k + 2) in s or (k + 2, k) in s or float(r[k + 2]) + float(r[k]) <= float(
            np.linalg.norm(x[k + 2] - x[k]))


def fcc(nc, a):
    basis = np.array([[0, 0, 0], [0.5, 0.5, 0], [0.5, 0, 0.5], [0, 0.5, 0.5]])
    pts = [(np.array([i, j, k]) + b) * a for i in range(nc) for j in range(nc) for k in range(nc) for b in basis]
    return np.array(pts)


def paper_values():
    out = {}
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "paper_values.txt")
    for line in open(path):
        line = line.split("#", 1)[0].strip()
        if line:
            k, v = (t.strip() for t in line.split("="))
            out[k] = float(v)
    return out


def test_fcc_close_packing_counts():
    """Sec. 6, Eq. 13: an FCC packing of diameter-d spheres has sqrt(2) spheres per d^3 cell,
    a sphere touches at most 12 others, and a 27-cell neighbourhood holds on average
    27 sqrt(2) (about 38) candidates. (The paper's "about 47" is not 27 sqrt(2); for a
    lattice misaligned with the grid single neighbourhoods hold more, so only the mean
    and the 12-contact bound are pinned.)"""
    d = 2e-3
    a = d * math.sqrt(2.0)
    nc = 8
    x = fcc(nc, a) + 1e-4
    r = np.full(len(x), np.float32(d / 2 * (1 + 1e-6)))     # neighbours overlap by ~1e-9 m
    L = nc * a + 2e-4
    p = params(cell_size=d, domain_lo=(0.0, 0.0, 0.0), domain_hi=(L, L, L))
    pairs, cand = oracle.pairs_grid(p, x, r, with_candidates=True)
    deg = np.bincount(pairs.ravel(), minlength=len(x))
    gold = paper_values()
    assert deg.max() == gold["max_simultaneous_contacts"]
    interior = np.all((x > 1.5 * a) & (x < (nc - 1.5) * a), axis=1)
    assert np.all(deg[interior] == gold["max_simultaneous_contacts"])
    # density: spheres per d^3 cell in the interior block (Eq. 13 with L = d)
    assert len(x) / (nc * a) ** 3 * d ** 3 == pytest.approx(gold["spheres_per_cell_at_edge_d"], rel=1e-9)
    cin = cand[interior] + 1
    assert np.mean(cin) == pytest.approx(gold["cells_walked"] * gold["spheres_per_cell_at_edge_d"], rel=0.05)
    assert cin.min() >= 13


def test_diagnostics_closed_forms():
    """KE, momentum and angular momentum of a two-sphere state, by hand."""
    p = params(g=(0.0, 0.0, -9.81))
    x = np.array([[1.0, 0.0, 0.0], [0.0, 2.0, 0.0]])
    v = np.array([[0.0, 1.0, 0.0], [3.0, 0.0, 0.0]])
    w = np.array([[0.0, 0.0, 5.0], [0.0, 0.0, 0.0]])
    r = np.full(2, R, np.float32)
    d = oracle.diagnostics(p, x, v, w, r)
    I = 0.4 * M * float(np.float32(R)) ** 2
    assert d[0] == pytest.approx(0.5 * M * (1 + 9))
    assert d[1] == pytest.approx(0.5 * I * 25)
    assert d[2:5] == pytest.approx([3 * M, M, 0.0])
    # L_z = m (x v_y - y v_x) summed + I w_z = M(1*1) + M(0 - 2*3) + 5 I
    assert d[7] == pytest.approx(M * 1 - 6 * M + 5 * I)
    assert d[9] == pytest.approx(2 * M)


# ------------------------------------------- parts of Eqs. 1, 5, 7, 8-9 pinned alone
def test_simple_model_shear_decays_sliding_exponentially():
    """Eq. 1 on a sphere resting on a plane and sliding along it: v is tangential, so
    v_t = v and the tangential force is -(k_da + k_sh) v, with no spin (Eq. 1 has no
    torque). Each semi-implicit Euler step multiplies v by (1 - (k_da + k_sh) dt / m)
    exactly. A dropped or sign-flipped k_sh term changes the decay rate."""
    kda, ksh, dt = 0.004, 0.0065, 1e-6
    p = floor_params(0.3, 0.5, model="simple", ksp=1e4, kda=kda, ksh=ksh, dt=dt)
    z0 = RF - M * 9.81 / 1e4
    v0 = 0.05
    st = oracle.State(p, np.array([[0.0, 0.0, z0]]), np.array([[v0, 0.0, 0.0]]), np.zeros((1, 3)),
                      np.full(1, R, np.float32))
    steps = 2000
    st.run(steps)
    factor = (1.0 - (kda + ksh) * dt / M) ** steps
    assert st.v[0, 0] == pytest.approx(v0 * factor, rel=1e-7)
    assert factor < 0.2
    assert np.all(st.w == 0.0)


def test_hertz_tangential_stiffness_sets_stick_oscillation_period():
    """Eqs. 8-9: a sphere resting on a plane at its Hertz overlap delta (R_eff = r for a
    wall) and kicked tangentially, with mu large and no damping, rolls back and forth:
    the contact point's displacement s obeys s'' = -(k_t/m + k_t r^2/I) s, a period of
    2 pi sqrt((2m/7) / k_t) with k_t = C_t sqrt(delta r). k_t formed from C_n, or without
    sqrt(delta r), gives another period."""
    cn, ct = S.hertz_coeffs(1e4, 2 / 7, R)
    delta = (M * 9.81 / (cn * math.sqrt(RF))) ** (2.0 / 3.0)
    kt = ct * math.sqrt(delta * RF)
    period = 2 * math.pi * math.sqrt((2 * M / 7) / kt)
    p = floor_params(10.0, 0.5, stiffness="hertz", cn=cn, ct=ct, alpha=0.0, dt=period / 600)
    st = oracle.State(p, np.array([[0.0, 0.0, RF - delta]]), np.array([[1e-4, 0.0, 0.0]]), np.zeros((1, 3)),
                      np.full(1, R, np.float32))
    # slip velocity of the contact point, v_x - r w_y, changes sign every half period
    prev, crossings = None, []
    for k in range(int(3.2 * 600)):
        st.run(1)
        s = st.v[0, 0] - RF * st.w[0, 1]
        if prev is not None and (prev > 0) != (s > 0):
            crossings.append((k + prev / (prev - s)) * p.dt)
        prev = s
    assert len(crossings) >= 5
    measured = 2 * (crossings[4] - crossings[0]) / 4
    assert measured == pytest.approx(period, rel=5e-3)


def _drive(p, x, v, hist, steps):
    """Evaluate `steps` steps of a kinematically driven state (positions and velocities
    held, only the springs carried), returning the tangential force on sphere 0 per step."""
    out = []
    w = np.zeros_like(x)
    r = np.full(len(x), R, np.float32)
    for _ in range(steps):
        F, _, hist, _ = oracle.forces(p, x, v, w, r, hist)
        out.append(F[0].copy())
    return np.array(out), hist


def test_spring_after_slip_keeps_eq4_an_identity_on_reversal():
    """Eq. 5 with the spring reset of the reading taken (after a cap the stored spring is
    -(F_t + eta v_t)/k_t, so Eq. 4 still gives the capped force). A sphere pressed onto a
    plane at a fixed overlap is dragged at +u until it slips, then at -u. On the first
    reversed step Eq. 7 adds -u dt to the spring and the dashpot term flips, so the
    tangential force jumps from -mu F_n to -mu F_n + 2 eta u + k_t u dt. A reset to
    -F_t/k_t gives a jump of eta u + k_t u dt; keeping the unbounded spring keeps the force
    capped at -mu F_n."""
    e, mu, kn, kt, u, dt = 0.5, 0.3, 1e4, 1e4 * 2 / 7, 0.01, 1e-6
    p = floor_params(mu, e, g=(0.0, 0.0, 0.0), dt=dt)
    eta = S.alpha_from_e(e) * math.sqrt(kn * M)
    delta0 = 1e-6
    x = np.array([[0.0, 0.0, RF - delta0]])
    fn = kn * (RF - x[0, 2])
    F1, hist = _drive(p, x, np.array([[u, 0.0, 0.0]]), oracle.empty_history(), 200)
    # loading: F_t = -k_t k u dt - eta u until the cap, then -mu F_n
    assert F1[0, 0] == pytest.approx(-kt * u * dt - eta * u, rel=1e-9)
    assert F1[-1, 0] == pytest.approx(-mu * fn, rel=1e-9)
    assert F1[-1, 2] == pytest.approx(fn, rel=1e-9)
    F2, _ = _drive(p, x, np.array([[-u, 0.0, 0.0]]), hist, 3)
    jump = 2 * eta * u + kt * u * dt
    assert F2[0, 0] == pytest.approx(-mu * fn + jump, rel=1e-9)
    assert F2[1, 0] == pytest.approx(-mu * fn + jump + kt * u * dt, rel=1e-9)


def test_history_projection_shrinks_spring_by_cos_theta():
    """Eq. 7 projects the stored spring onto the new tangent plane without rescaling:
    when the contact normal turns by theta between steps (and the contact point does not
    slip), a spring s perpendicular to the old normal and in the plane of the turn keeps
    length s cos(theta), and the tangential force is -k_t times it."""
    kt, s, theta = 1e4 * 2 / 7, 2e-7, 0.5
    p = params(alpha=0.0, mu=0.3)
    d = 2 * RF - 1e-6
    x = np.array([[0.0, 0.0, 0.0], [d * math.cos(theta), d * math.sin(theta), 0.0]])
    hist = oracle.empty_history(1)
    hist[0] = (0, 1, (0.0, s, 0.0))           # perpendicular to the old normal (1, 0, 0)
    F, _, h2, _ = oracle.forces(p, x, np.zeros((2, 3)), np.zeros((2, 3)), np.full(2, R, np.float32), hist)
    assert len(h2) == 1
    dn = h2[0]["d"]
    n = x[1] / np.linalg.norm(x[1])
    assert np.linalg.norm(dn) == pytest.approx(s * math.cos(theta), rel=1e-12)
    assert abs(np.dot(dn, n)) <= 1e-12 * s
    Ft = F[0] - np.dot(F[0], n) * n
    assert np.linalg.norm(Ft) == pytest.approx(kt * s * math.cos(theta), rel=1e-12)
