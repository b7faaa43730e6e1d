"""Optional force terms (no attraction, rolling resistance, separate eta_t, cohesion) on
the GPU against the FP64 oracle with the same terms. Any nonzero `terms` runs a separate
compiled variant of the force kernel; the bars are those of the paper's law:
|dF| / S_i <= 1e-12 (FP64), 1e-5 (FP32), positions 1e-12 m after 10 FP64 steps.
"""
import numpy as np
import pytest

import oracle
from paper_1301_1714_gb300 import dem, scenes

pytestmark = pytest.mark.gpu

from test_gpu_parity import SCENES, SQUEEZE, assert_forces_close, compressed  # noqa: E402

ALL = dict(terms=15, mu_roll=0.1, alpha_t=0.3, k_coh=3e5)
CASES = [dict(terms=1), dict(terms=2, mu_roll=0.2), dict(terms=4, alpha_t=0.1), dict(terms=8, k_coh=5e5), ALL]


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1301_1714_gb300 import _build
    _build.build()
    dem.lib()


@pytest.mark.parametrize("kw", CASES, ids=lambda k: f"terms{k['terms']}")
@pytest.mark.parametrize("name", ["box2048", "drum4099"])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_forces_with_terms(kw, name, precision):
    sc = SCENES[name]()
    x = compressed(sc, SQUEEZE[name])
    rng = np.random.default_rng(7)
    w = rng.normal(0, 20.0, size=x.shape)
    v = sc.v + rng.normal(0, 0.05, size=x.shape)
    p = sc.params.copy(precision=precision, **kw)
    Fo, To, _, stats = oracle.forces(p, x, v, w, sc.r)
    F0, T0, _, _ = oracle.forces(p.copy(terms=0), x, v, w, sc.r)
    assert stats[0] > 100
    assert np.max(np.abs(Fo - F0)) + np.max(np.abs(To - T0)) > 0.0   # the terms act here
    with dem.Simulation(p, x, v, w, sc.r) as s:
        F, T = s.forces()
    assert_forces_close(p, x, v, sc.r, F, T, Fo, To, 1e-12 if precision == "fp64" else 1e-5)


@pytest.mark.parametrize("stiffness", ["linear", "hertz"])
def test_trajectory_with_all_terms_fp64(stiffness):
    sc = scenes.box_lattice(seed=1, stiffness=stiffness)
    p = sc.params.copy(**ALL)
    ref = oracle.State(p, sc.x, sc.v, sc.w, sc.r)
    with dem.Simulation(p, sc.x, sc.v, sc.w, sc.r) as s:
        s.step(10)
        x10, _, _ = s.state()
        ref.run(10)
        assert np.max(np.abs(x10 - ref.x)) <= 1e-12
        s.step(290)
        x, _, w = s.state()
        d = s.diagnostics()
    ref.run(290)
    assert np.max(np.abs(x - ref.x)) <= 1e-9
    assert d["pair_contacts"] + d["wall_contacts"] > 0


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_list_mode_drum_with_terms(precision):
    sc = scenes.drum(seed=5, n=3001)
    base = sc.params.copy(**ALL)
    skin = 0.05e-3
    p = base.copy(precision=precision, resort_interval=0, skin=skin, cell_size=base.cell_size + skin)
    ref = oracle.State(base.copy(precision="fp64"), sc.x, sc.v, sc.w, sc.r).run(120)
    with dem.Simulation(p, sc.x, sc.v, sc.w, sc.r) as s:
        s.step(120)
        x, _, _ = s.state()
    assert np.max(np.abs(x - ref.x)) <= (1e-12 if precision == "fp64" else 1e-9)


def test_batch_mixes_scenes_with_and_without_terms():
    a = scenes.box_lattice(seed=3)
    b = scenes.drum(seed=6, n=2001)
    pa = a.params.copy(precision="fp32", **ALL)
    pb = b.params.copy(precision="fp32")
    bt = dem.dem_batch_create(precision="fp32")
    try:
        sa = dem.dem_batch_add(bt, pa, a.x, a.v, a.w, a.r, 50)
        sb = dem.dem_batch_add(bt, pb, b.x, b.v, b.w, b.r, 50)
        dem.dem_batch_run(bt, 50)
        xa = dem.dem_batch_get_state(bt, sa, a.n)[0]
        xb = dem.dem_batch_get_state(bt, sb, b.n)[0]
    finally:
        dem.dem_batch_destroy(bt)
    ra = oracle.State(pa.copy(precision="fp64"), a.x, a.v, a.w, a.r).run(50)
    rb = oracle.State(pb.copy(precision="fp64"), b.x, b.v, b.w, b.r).run(50)
    for x, r, s in ((xa, ra, a), (xb, rb, b)):
        disp = max(np.max(np.linalg.norm(r.x - s.x, axis=1)), 1e-9)
        assert np.max(np.abs(x - r.x)) <= 1e-5 * disp + 1e-12


def test_terms_are_validated():
    sc = scenes.box_lattice(seed=1)
    for bad in (dict(terms=16), dict(terms=2, mu_roll=-1.0), dict(terms=8, k_coh=float("nan")),
                dict(terms=1, model="simple")):
        with pytest.raises(dem.DemError):
            dem.Simulation(sc.params.copy(**bad), sc.x, sc.v, sc.w, sc.r)
