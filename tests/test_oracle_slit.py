"""Pins of the oracle's slit plate (the bottom of the paper's benchmark box, Sec. 5) and
of the stop criterion (run until every particle moves less than a set amount per step).

Closed forms checked:
  resting on the plate, from above or (gravity reversed) from below: delta = m g / k_n;
  resting in a slit narrower than the sphere: 2 k_n delta h / dist = m g on the two edges;
  falling through a slit wider than the sphere: free fall of the integrator, no contact;
  hitting a slit edge head-on in the plate's plane: restitution e, no vertical motion.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1301_1714_gb300 import scenes as S

R = 1e-3
RF = float(np.float32(R))
M = 2500.0 * 4.0 / 3.0 * math.pi * RF ** 3
KN = 1e4
G = 9.81
ZP = 0.01


def params(half, g=(0.0, 0.0, -G), e=0.3, mu=0.3, **kw):
    tc = math.pi / math.sqrt(KN / M)
    base = dict(model="practical", stiffness="linear", precision="fp64", dt=tc / 50, g=g, kn=KN, kt=KN * 2 / 7,
                alpha=S.alpha_from_e(e), mu=mu, cell_size=S.auto_cell_size(RF), domain_lo=(-0.02, -0.02, 0.0),
                domain_hi=(0.02, 0.02, 0.02), walls=S.slit_plates(ZP, 0.0, half))
    base.update(kw)
    return S.Params(**base)


def one(x, v=(0, 0, 0)):
    return np.array([x], float), np.array([v], float), np.zeros((1, 3)), np.full(1, R, np.float32)


@pytest.mark.parametrize("side", [1.0, -1.0])
def test_resting_on_either_face(side):
    p = params(2 * R, g=(0.0, 0.0, -side * G))
    st = oracle.State(p, *one((5 * R, 0.0, ZP + side * RF * 1.0005)))
    st.run(40000)
    delta = RF - side * (st.x[0, 2] - ZP)
    assert delta == pytest.approx(M * G / KN, rel=1e-3)
    assert abs(st.x[0, 0] - 5 * R) < 1e-12


def test_resting_across_a_narrow_slit():
    half = 0.6 * RF
    p = params(half, e=0.2, mu=0.0)
    st = oracle.State(p, *one((0.0, 0.0, ZP + 0.85 * RF)))
    st.run(60000)
    # equilibrium height h: 2 k_n (r - dist) h / dist = m g with dist = sqrt(half^2 + h^2)
    f = lambda h: 2 * KN * (RF - math.hypot(half, h)) * h / math.hypot(half, h) - M * G
    lo, hi = 0.5 * math.sqrt(RF ** 2 - half ** 2), math.sqrt(RF ** 2 - half ** 2)
    assert f(lo) > 0 > f(hi)
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if f(mid) > 0:
            lo = mid
        else:
            hi = mid
    h = 0.5 * (lo + hi)
    assert st.x[0, 2] - ZP == pytest.approx(h, rel=1e-6)
    assert abs(st.x[0, 0]) < 1e-12
    assert st.stats[1] == 2                                # both edges touch


def test_falls_through_a_wide_slit_untouched():
    half = 1.5 * RF
    p = params(half)
    z0 = ZP + 2 * RF
    st = oracle.State(p, *one((0.0, 0.0, z0)))
    n = 0
    while st.x[0, 2] > ZP - 3 * RF:
        st.run(1)
        n += 1
        assert st.stats[1] == 0
    # semi-implicit Euler from rest: z_n = z0 - g dt^2 n (n + 1) / 2
    assert st.x[0, 2] == pytest.approx(z0 - G * p.dt ** 2 * n * (n + 1) / 2, rel=1e-12)


@pytest.mark.parametrize("e", [0.9, 0.5])
def test_head_on_edge_collision_restitution(e):
    half = 3 * RF
    p = params(half, g=(0.0, 0.0, 0.0), e=e, dt=math.pi / math.sqrt(KN / M) / 400)
    x0 = half - RF - 1e-7
    st = oracle.State(p, *one((x0, 0.0, ZP), (0.05, 0.0, 0.0)))
    touched = False
    for _ in range(20000):
        st.run(1)
        if st.stats[1] > 0:
            touched = True
        elif touched:
            break
    assert touched
    assert st.v[0, 0] / -0.05 == pytest.approx(e, rel=5e-3)
    assert st.x[0, 2] == ZP and st.v[0, 2] == 0.0


def max_step_displacement(st, k):
    """Runs k steps; returns the largest displacement of a particle in the last one."""
    st.run(k - 1)
    x0 = st.x.copy()
    st.run(1)
    return float(np.max(np.linalg.norm(st.x - x0, axis=1)))


def run_until(p, x, v, w, r, max_steps, thr, every):
    st = oracle.State(p, x, v, w, r)
    done = 0
    while done < max_steps:
        k = min(every, max_steps - done)
        d = max_step_displacement(st, k)
        done += k
        if d < thr:
            return done, d, True, st
    return done, d, False, st


def test_bouncing_sphere_comes_to_rest():
    """The stop criterion on a sphere dropped onto the plate: it stops when the last
    step of a chunk moves it less than the threshold, which happens after the bounces
    have died out (the rest overlap m g / k_n is reached)."""
    p = params(2 * R, e=0.3)
    done, d, ok, st = run_until(p, *one((5 * R, 0.0, ZP + 1.5 * RF)), 200000, 1e-12, 500)
    assert ok and d < 1e-12 and done % 500 == 0
    assert RF - (st.x[0, 2] - ZP) == pytest.approx(M * G / KN, rel=1e-3)
    # the chunk before did not yet meet the threshold
    st2 = oracle.State(p, *one((5 * R, 0.0, ZP + 1.5 * RF)))
    st2.run(done - 501)
    x0 = st2.x.copy()
    st2.run(1)
    assert np.linalg.norm(st2.x - x0) >= 1e-12
