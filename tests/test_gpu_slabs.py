"""Slab decomposition with halo exchange (sub-domains of one scene on one GPU), through
the C ABI.

Bars:
  owned particles' state after K steps ........ bit-exact against one undivided handle
                                                 of the same configuration (FP64 and FP32):
                                                 the 27-cell walk (Eq. 12) of an owned
                                                 particle meets the same partners in the same
                                                 (cell, id) order (Eq. 11)
  against the FP64 oracle ..................... the single-domain bars (1e-12 m after 10
                                                 steps, 1e-9 m after 300)
  owned / ghost counts per slab ............... exact, against the ownership and ghost rule
                                                 applied on the host to the exported state
"""
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


def halo_counts(x, bounds, G, axis):
    """Owned and ghost counts per slab from positions (the rule of the C header)."""
    z = x[:, axis]
    S = len(bounds) - 1
    owner = np.zeros(len(z), np.int64)
    for t in range(1, S):
        owner += (z >= bounds[t])
    owned = np.bincount(owner, minlength=S)
    ghosts = np.zeros(S, np.int64)
    for t in range(S):
        inside = (z >= bounds[t] - G) & (z < bounds[t + 1] + G)
        ghosts[t] = int(np.count_nonzero(inside & (owner != t)))
    return owned, ghosts


def single_and_slabs(sc, p, nslabs, steps, axis=-1, block=0, maxc=0):
    with dem.Simulation(p, sc.x, sc.v, sc.w, sc.r, block_size=block, max_contacts=maxc) as s:
        s.step(steps)
        ref = s.state()
    with dem.Slabs(p, sc.x, sc.v, sc.w, sc.r, nslabs, axis=axis, block_size=block, max_contacts=maxc) as sl:
        sl.step(steps)
        got = sl.state()
        info = sl.info()
    return ref, got, info


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("nslabs", [2, 3, 5])
def test_slabs_are_bit_exact_against_one_domain(precision, nslabs):
    sc = scenes.drum(seed=21, n=20000)
    p = sc.params.copy(precision=precision)
    ref, got, info = single_and_slabs(sc, p, nslabs, 300, block=128, maxc=24)
    for a, b in zip(ref, got):
        assert np.array_equal(a, b)
    assert info["steps"] == 300
    assert info["owned"].sum() == sc.n
    assert (info["ghosts"] > 0).all()
    assert info["migrated"] > 0          # particles on the boundaries cross them


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_any_axis(axis):
    sc = scenes.box_lattice_n(seed=22, n=6000, vsigma=0.3)
    ref, got, info = single_and_slabs(sc, sc.params, 3, 200, axis=axis)
    for a, b in zip(ref, got):
        assert np.array_equal(a, b)
    assert info["migrated"] > 0


def test_slabs_against_the_oracle():
    sc = scenes.box_lattice(seed=23)
    ref = oracle.State(sc.params, sc.x, sc.v, sc.w, sc.r)
    with dem.Slabs(sc.params, sc.x, sc.v, sc.w, sc.r, 3, axis=2) as sl:
        sl.step(10)
        x10, v10, _ = sl.state()
        ref.run(10)
        assert np.max(np.abs(x10 - ref.x)) <= 1e-12
        assert np.max(np.abs(v10 - ref.v)) <= 1e-9
        sl.step(290)
        x, _, _ = sl.state()
        ref.run(290)
    assert np.max(np.abs(x - ref.x)) <= 1e-9


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_counts_follow_the_halo_rule(precision):
    sc = scenes.drum(seed=24, n=8000)
    p = sc.params.copy(precision=precision)
    with dem.Slabs(p, sc.x, sc.v, sc.w, sc.r, 4, axis=2) as sl:
        info0 = sl.info()
        G = sc.params.cell_size
        owned, ghosts = halo_counts(sc.x, info0["bounds"], G, 2)   # the first distribution reads the input
        assert np.array_equal(owned, info0["owned"])
        assert np.array_equal(ghosts, info0["ghosts"])
        sl.step(150)
        info = sl.info()
        x, _, _ = sl.state()
    owned, ghosts = halo_counts(x, info["bounds"], G, 2)
    assert np.array_equal(owned, info["owned"])
    assert np.array_equal(ghosts, info["ghosts"])
    assert np.array_equal(info["bounds"], info0["bounds"])      # boundaries stay where they were set
    assert np.array_equal(info["bounds"], dem.dem_slab_bounds(sc.x[:, 2], 4))


def test_one_slab_and_empty_slabs():
    sc = scenes.box_lattice_n(seed=25, n=3)
    ref, got, info = single_and_slabs(sc, sc.params, 1, 50)
    for a, b in zip(ref, got):
        assert np.array_equal(a, b)
    ref, got, info = single_and_slabs(sc, sc.params, 8, 50)    # more slabs than particles
    for a, b in zip(ref, got):
        assert np.array_equal(a, b)
    assert info["owned"].sum() == 3 and (info["owned"] == 0).sum() >= 5


def test_no_particles():
    sc = scenes.box_lattice_n(seed=26, n=64)
    with dem.Slabs(sc.params, sc.x[:0], sc.v[:0], sc.w[:0], sc.r[:0], 2) as sl:
        sl.step(3)
        x, _, _ = sl.state()
        assert x.shape == (0, 3)
        assert sl.info()["owned"].sum() == 0


def test_device_inputs_and_outputs():
    import torch
    sc = scenes.drum(seed=27, n=5000)
    dev = torch.device("cuda", 0)
    t = lambda a, dt=torch.float64: torch.from_numpy(np.ascontiguousarray(a)).to(dev, dt)
    with dem.Slabs(sc.params, t(sc.x), t(sc.v), t(sc.w), t(sc.r, torch.float32), 3) as sl:
        sl.step(20)
        xd = torch.empty((sc.n, 3), dtype=torch.float64, device=dev)
        dem.dem_slabs_get_state(sl.h, sc.n, x=xd)
        x, _, _ = sl.state()
    assert np.array_equal(xd.cpu().numpy(), x)
    with dem.Simulation(sc.params, sc.x, sc.v, sc.w, sc.r) as s:
        s.step(20)
        assert np.array_equal(s.state()[0], x)


def test_rejected_arguments():
    sc = scenes.drum(seed=28, n=2000)
    with pytest.raises(dem.DemError):
        dem.dem_slabs_create(sc.params.copy(resort_interval=0, skin=1e-4), 2)   # list mode is not divided
    with pytest.raises(dem.DemError):
        dem.dem_slabs_create(sc.params, 0)
    with pytest.raises(dem.DemError):
        dem.dem_slabs_create(sc.params, dem.DEM_MAX_SLABS + 1)
    with pytest.raises(dem.DemError):
        dem.dem_slabs_create(sc.params, 2, axis=3)
    sl = dem.dem_slabs_create(sc.params, 2)
    try:
        with pytest.raises(dem.DemError):
            dem.dem_slabs_step(sl, 1)            # before any particles
        bad = sc.x.copy()
        bad[5, 2] = np.nan
        with pytest.raises(dem.DemError):
            dem.dem_slabs_set_particles(sl, bad, sc.v, sc.w, sc.r)
    finally:
        dem.dem_slabs_destroy(sl)
