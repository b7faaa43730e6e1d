"""Pins of the oracle's optional force terms (none is in the paper, whose force is built
from separable terms so that terms can be added or removed; these are the usual ones).

Each test checks a closed form of mechanics that the term decides:
  terms & 1  no attractive normal force -> restitution of the clamped dashpot;
  terms & 2  rolling resistance         -> deceleration (5/7) mu_r g of a rolling sphere;
  terms & 4  separate tangential eta_t  -> decay of the stick-slip oscillation of a
                                           sphere on a plane (reduced mass 2m/7);
  terms & 8  cohesion                   -> resting overlap m g / (k_n - k_coh pi r).
"""
import math

import numpy as np
import pytest

import oracle
from paper_1301_1714_gb300 import scenes as S

R = 1e-3
RF = float(np.float32(R))
RHO = 2500.0
M = RHO * 4.0 / 3.0 * math.pi * RF ** 3
KN = 1e4
G = 9.81


def params(**kw):
    base = dict(model="practical", stiffness="linear", precision="fp64", dt=1e-6, g=(0.0, 0.0, 0.0), kn=KN,
                kt=KN * 2 / 7, alpha=0.0, mu=0.3, cell_size=S.auto_cell_size(RF), domain_lo=(-0.05, -0.05, -0.05),
                domain_hi=(0.05, 0.05, 0.05), walls=[])
    base.update(kw)
    return S.Params(**base)


def floor(**kw):
    walls = [dict(kind="plane", p=(0.0, 0.0, 0.0), n=(0.0, 0.0, 1.0))]
    base = dict(g=(0.0, 0.0, -G), domain_lo=(-0.05, -0.05, 0.0), domain_hi=(0.05, 0.05, 0.05), walls=walls)
    base.update(kw)
    return params(**base)


def one(x, v=(0, 0, 0), w=(0, 0, 0)):
    return (np.array([x], float), np.array([v], float), np.array([w], float), np.full(1, R, np.float32))


# ------------------------------------------------------------------ terms & 1
def clamped_restitution(kn, eta, meff):
    """m x'' = -k x - eta x' from x = 0, x' = v0 while k x + eta x' >= 0; once the force
    would pull, it is zero and the bodies leave at the velocity of that instant."""
    g = eta / (2 * meff)
    wd = math.sqrt(kn / meff - g * g)
    ts = (math.pi - math.atan(eta * wd / (kn - eta * g))) / wd
    return -math.exp(-g * ts) * (math.cos(wd * ts) - g / wd * math.sin(wd * ts))


@pytest.mark.parametrize("e", [0.8, 0.4])
def test_no_attraction_restitution_closed_form(e):
    meff = M / 2
    alpha = S.alpha_from_e(e)
    eta = alpha * math.sqrt(KN * meff)
    e_cl = clamped_restitution(KN, eta, meff)
    assert e_cl > e                                         # the clamp removes the final pull
    tc = math.pi / math.sqrt(KN / meff)
    x = np.array([[-RF - 5e-8, 0.0, 0.0], [RF + 5e-8, 0.0, 0.0]])
    v = np.array([[0.1, 0.0, 0.0], [-0.1, 0.0, 0.0]])
    out = []
    for terms in (0, 1):
        st = oracle.State(params(alpha=alpha, dt=tc / 2000, terms=terms), x, v, np.zeros((2, 3)),
                          np.full(2, R, np.float32))
        touched = False
        for _ in range(20000):
            st.run(1)
            if st.stats[0] > 0:
                touched = True
            elif touched:
                break
        out.append((st.v[1, 0] - st.v[0, 0]) / 0.2)
    assert out[0] == pytest.approx(e, rel=2e-3)
    assert out[1] == pytest.approx(e_cl, rel=2e-3)


def test_no_attraction_force_never_pulls():
    """Spheres separating fast at a small overlap: Eq. 4's dashpot would pull (F_n . n > 0
    on i); with the clamp the normal force is zero and only friction-free zero is left."""
    x = np.array([[-RF + 1e-7, 0.0, 0.0], [RF - 1e-7, 0.0, 0.0]])
    v = np.array([[-0.5, 0.0, 0.0], [0.5, 0.0, 0.0]])
    p0 = params(alpha=S.alpha_from_e(0.5))
    F0, _, _, _ = oracle.forces(p0, x, v, np.zeros((2, 3)), np.full(2, R, np.float32))
    F1, _, _, _ = oracle.forces(p0.copy(terms=1), x, v, np.zeros((2, 3)), np.full(2, R, np.float32))
    assert F0[0, 0] > 0.0                                   # unclamped: i pulled toward j (+x)
    assert np.all(F1 == 0.0)


# ------------------------------------------------------------------ terms & 2
def test_rolling_resistance_decelerates_at_five_sevenths_mu_r_g():
    """A sphere rolling without slip on a plane under a resisting torque mu_r r m g:
    m a = f, I alpha = -f r - mu_r r m g with a = alpha r gives a = -(5/7) mu_r g."""
    mu_r, v0 = 0.05, 0.1
    tc = math.pi / math.sqrt(KN / M)
    p = floor(alpha=S.alpha_from_e(0.3), mu=0.5, dt=tc / 50, terms=2, mu_roll=mu_r)
    z0 = RF - M * G / KN
    st = oracle.State(p, *one((0.0, 0.0, z0), (v0, 0.0, 0.0), (0.0, v0 / RF, 0.0)))
    ts, vs = [], []
    steps = int(0.08 / p.dt)
    chunk = steps // 40
    for k in range(40):
        st.run(chunk)
        ts.append((k + 1) * chunk * p.dt)
        vs.append(st.v[0, 0])
    slope = np.polyfit(ts[5:], vs[5:], 1)[0]
    assert slope == pytest.approx(-5.0 / 7.0 * mu_r * G, rel=0.01)
    assert st.w[0, 1] * RF == pytest.approx(st.v[0, 0], rel=1e-3)      # still rolling
    # without the term the sphere keeps rolling at v0
    p0 = p.copy(terms=0)
    st0 = oracle.State(p0, *one((0.0, 0.0, z0), (v0, 0.0, 0.0), (0.0, v0 / RF, 0.0)))
    st0.run(chunk * 10)
    assert st0.v[0, 0] == pytest.approx(v0, rel=1e-6)


# ------------------------------------------------------------------ terms & 4
def slip_decay(p, v0=4e-4, nsteps=3000):
    """Slip u = v_x - w_y r of a sphere resting on a plane, kicked tangentially."""
    z0 = RF - M * G / KN
    st = oracle.State(p, *one((0.0, 0.0, z0), (v0, 0.0, 0.0)))
    u = np.empty(nsteps)
    for k in range(nsteps):
        st.run(1)
        u[k] = st.v[0, 0] - st.w[0, 1] * RF
    return u


def peaks(u):
    return [k for k in range(1, len(u) - 1) if u[k] > u[k - 1] and u[k] >= u[k + 1] and u[k] > 0]


@pytest.mark.parametrize("terms,alpha_t", [(0, 0.0), (4, 0.15), (4, 0.0)])
def test_tangential_damping_sets_stick_slip_decay(terms, alpha_t):
    """Sticking contact (no cap): the spring elongation xi obeys (2m/7) xi'' = -k_t xi -
    eta_t xi' (slip acceleration F_t (1/m + r^2/I)), so successive slip maxima shrink by
    exp(-gamma T) with gamma = 7 eta_t / (4 m), T = 2 pi / sqrt(7 k_t / (2 m) - gamma^2).
    eta_t is eta = alpha sqrt(k_n m) by default and alpha_t sqrt(k_t m) with terms & 4."""
    alpha = 0.05
    kt = KN * 2 / 7
    w0 = math.sqrt(7 * kt / (2 * M))
    p = floor(alpha=alpha, mu=1.0, kt=kt, dt=0.005 / w0, terms=terms, alpha_t=alpha_t)
    eta_t = alpha_t * math.sqrt(kt * M) if terms & 4 else alpha * math.sqrt(KN * M)
    gam = 7 * eta_t / (4 * M)
    T = 2 * math.pi / math.sqrt(w0 * w0 - gam * gam)
    u = slip_decay(p, nsteps=int(3.2 * T / p.dt))
    pk = peaks(u)
    assert len(pk) >= 3
    ratio = u[pk[2]] / u[pk[1]]
    assert ratio == pytest.approx(math.exp(-gam * T), rel=5e-3, abs=2e-3)
    assert (pk[2] - pk[1]) * p.dt == pytest.approx(T, rel=0.01)


# ------------------------------------------------------------------ terms & 8
@pytest.mark.parametrize("frac", [0.0, 0.5])
def test_cohesion_resting_overlap(frac):
    """Resting on a plane (R_eff = r): k_n delta = m g + k_coh pi r delta."""
    kcoh = frac * KN / (math.pi * RF)
    tc = math.pi / math.sqrt(KN / M)
    p = floor(alpha=S.alpha_from_e(0.3), dt=tc / 50, terms=8, k_coh=kcoh)
    st = oracle.State(p, *one((0.0, 0.0, RF * 1.0001)))
    st.run(40000)
    delta = RF - st.x[0, 2]
    assert delta == pytest.approx(M * G / (KN - kcoh * math.pi * RF), rel=1e-3)


# ------------------------------------------------------------------ all terms
def test_all_terms_conserve_momentum_and_balance_couples():
    """With every term on, pair forces stay equal and opposite (cohesion is central) and
    the rolling torques are couples (+M on i, -M on j): no walls and no gravity keep
    the total momentum, and the angular momentum changes only by the lever-arm term
    dt delta (n x F_t) of Eq. 3, bounded by dt delta mu |F_n|."""
    sc = S.box_lattice(5, 5, 5, 4, r=R, box=(12.0, 12.0, 10.0), spacing=2.02, jitter=0.01, vsigma=0.5)
    rng = np.random.default_rng(3)
    w0 = rng.normal(0, 50.0, size=(len(sc.r), 3))
    p = params(alpha=S.alpha_from_e(0.7), mu=0.4, dt=1e-6, domain_lo=(0, 0, 0), domain_hi=(0.012, 0.012, 0.010),
               terms=15, mu_roll=0.1, alpha_t=0.3, k_coh=1e5)
    st = oracle.State(p, sc.x, sc.v, w0, sc.r)
    d0 = oracle.diagnostics(p, st.x, st.v, st.w, st.r)
    scale = float(np.sum(M * np.linalg.norm(st.v, axis=1)))
    seen = 0
    for _ in range(300):
        pairs = oracle.pairs_brute(st.x, st.r)
        bound = 0.0
        for i, j in pairs:
            dvec = st.x[j] - st.x[i]
            d = np.linalg.norm(dvec)
            delta = float(st.r[i]) + float(st.r[j]) - d
            vn = abs(np.dot(st.v[i] - st.v[j], dvec / d))
            bound += delta * p.mu * (p.kn * delta + p.alpha * math.sqrt(p.kn * M / 2) * vn)
        seen += len(pairs)
        dA = oracle.diagnostics(p, st.x, st.v, st.w, st.r)
        st.run(1)
        dB = oracle.diagnostics(p, st.x, st.v, st.w, st.r)
        assert np.linalg.norm(dB[5:8] - dA[5:8]) <= p.dt * bound * (1 + 1e-6) + 1e-20
    d1 = oracle.diagnostics(p, st.x, st.v, st.w, st.r)
    assert seen > 100
    assert np.max(np.abs(d1[2:5] - d0[2:5])) < 1e-13 * scale
