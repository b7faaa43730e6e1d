"""The paper's benchmark shape (Sec. 5): spheres drain from a box through a slit in its
bottom (two half-plates) onto a floor, and the run stops when every particle moves less
than a set amount per step. GPU against the FP64 oracle on the same seeded inputs.

Bars: forces |dF| / S_i <= 1e-12 (FP64), 1e-5 (FP32); FP64 positions 1e-12 m after 10
steps; the stop step of dem_run_until equals the oracle's.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1301_1714_gb300 import dem, scenes

pytestmark = pytest.mark.gpu

from test_gpu_parity import assert_forces_close  # noqa: E402
from test_oracle_slit import run_until as oracle_run_until  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1301_1714_gb300 import _build
    _build.build()
    dem.lib()


def pressed(sc, drop):
    """The lattice lowered by `drop` radii: its first layer presses into the plate and,
    over the slit, against the slit edges."""
    x = sc.x.copy()
    x[:, 2] -= drop * 1e-3
    return x


def small_hopper(precision, nz=6):
    """768 spheres; the two lattice columns over the slit lie 0.3 r inside its edges."""
    return scenes.hopper(seed=3, nx=16, ny=8, nz=nz, slit_over_d=1.35, precision=precision)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_forces_on_plate_and_slit_edges(precision):
    sc = small_hopper(precision)
    x = pressed(sc, 0.15)
    rng = np.random.default_rng(2)
    w = rng.normal(0, 20.0, size=x.shape)
    v = sc.v + rng.normal(0, 0.05, size=x.shape)
    p = sc.params
    F0, _, _, st0 = oracle.forces(p.copy(walls=p.walls[:6]), x, v, w, sc.r)
    Fo, To, _, stats = oracle.forces(p, x, v, w, sc.r)
    assert stats[1] - st0[1] > 100                 # plate and edge contacts
    with dem.Simulation(p, x, v, w, sc.r) as s:
        F, T = s.forces()
    assert_forces_close(p, x, v, sc.r, F, T, Fo, To, 1e-12 if precision == "fp64" else 1e-5)


def test_trajectory_fp64_through_the_slit():
    sc = small_hopper("fp64")
    x = pressed(sc, 0.12)
    ref = oracle.State(sc.params, x, sc.v, sc.w, sc.r)
    with dem.Simulation(sc.params, x, sc.v, sc.w, sc.r) as s:
        s.step(10)
        x10, _, _ = s.state()
        ref.run(10)
        assert np.max(np.abs(x10 - ref.x)) <= 1e-12
        s.step(390)
        xs, _, _ = s.state()
        d = s.diagnostics()
    ref.run(390)
    assert np.max(np.abs(xs - ref.x)) <= 1e-10
    assert d["wall_contacts"] > 0


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_list_mode_hopper_matches_oracle(precision):
    sc = small_hopper(precision)
    x = pressed(sc, 0.12)
    skin = 0.1e-3
    p = sc.params.copy(resort_interval=0, skin=skin, cell_size=sc.params.cell_size + skin)
    ref = oracle.State(sc.params.copy(precision="fp64"), x, sc.v, sc.w, sc.r).run(150)
    with dem.Simulation(p, x, sc.v, sc.w, sc.r) as s:
        s.step(150)
        xs, _, _ = s.state()
    assert np.max(np.abs(xs - ref.x)) <= (1e-12 if precision == "fp64" else 1e-9)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_run_until_stops_at_the_oracle_step(precision):
    """A sphere dropped onto the plate beside the slit bounces and comes to rest; the
    chunk at which its step displacement first falls below the threshold is the same."""
    from test_oracle_slit import params as slit_params, one, ZP
    p = slit_params(2e-3, e=0.3, precision=precision)
    x, v, w, r = one((5e-3, 0.0, ZP + 1.5e-3))
    thr = 1e-10
    done, disp, ok, ref = oracle_run_until(p.copy(precision="fp64"), x, v, w, r, 100000, thr, 250)
    assert ok
    with dem.Simulation(p, x, v, w, r) as s:
        g_done, g_disp, g_ok = dem.dem_run_until(s.h, 100000, thr, 250)
        xs, _, _ = s.state()
    assert g_ok and g_disp < thr
    if precision == "fp64":
        assert g_done == done
        assert np.max(np.abs(xs - ref.x)) <= 1e-12
    else:
        # FP32 velocities cross the threshold within a few chunks of the FP64 run (the
        # last small bounces differ), and the sphere is then within 1e-3 r of rest
        assert abs(g_done - done) <= 4 * 250
        rest = ZP + float(r[0]) - 2500.0 * 4.0 / 3.0 * np.pi * float(r[0]) ** 3 * 9.81 / 1e4
        assert abs(xs[0, 2] - rest) <= 1e-6


def test_run_until_respects_max_steps_and_validates():
    sc = small_hopper("fp32")
    with dem.Simulation(sc.params, sc.x, sc.v, sc.w, sc.r) as s:
        done, disp, ok = dem.dem_run_until(s.h, 300, 0.0, 128)
        assert (done, ok) == (300, False) and disp > 0.0
        assert s.diagnostics()["steps"] == 300
        for bad in ((-1, 1e-9, 10), (10, -1.0, 10), (10, 1e-9, 0)):
            with pytest.raises(dem.DemError):
                dem.dem_run_until(s.h, *bad)


def test_half_plate_validation():
    sc = small_hopper("fp32")
    bad = [dict(kind="half_plate", p=(0, 0, 0.01), n=(0.0, 0.0, 1.0), u=(0.0, 0.0, 1.0)),       # u not in the plane
           dict(kind="half_plate", p=(0, 0, 0.01), n=(0.0, 0.0, 1.0), u=(0.6, 0.8, 0.0))]       # FP32: not an axis
    with dem.Simulation(sc.params, sc.x, sc.v, sc.w, sc.r) as s:
        for wl in bad:
            with pytest.raises(dem.DemError):
                dem.dem_set_walls(s.h, [wl])
    # the same oblique plate is accepted in FP64 mode
    p64 = sc.params.copy(precision="fp64")
    with dem.Simulation(p64, sc.x, sc.v, sc.w, sc.r) as s:
        dem.dem_set_walls(s.h, [bad[1]])


def test_full_hopper_drains_through_the_slit():
    """131,072 spheres (the paper's count): after 30,000 steps (44 ms) the first layers
    over the slit have fallen through it; everything stays finite and inside the box."""
    sc = scenes.hopper(seed=1)
    zp = sc.params.walls[6]["p"][2]
    p = sc.params.copy(resort_interval=0, skin=0.1e-3, cell_size=sc.params.cell_size + 0.1e-3)
    with dem.Simulation(p, sc.x, sc.v, sc.w, sc.r) as s:
        s.step(30000)
        xs, vs, _ = s.state()
        d = s.diagnostics()
    assert np.all(np.isfinite(xs)) and np.all(np.isfinite(vs))
    below = np.count_nonzero(xs[:, 2] < zp - 1e-3)
    assert below > 300
    hi = np.array(sc.params.domain_hi)
    assert np.all(xs > -1e-4) and np.all(xs < hi + 1e-4)
    assert d["max_overlap"] < 0.05e-3
