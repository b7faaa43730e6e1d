"""Batches: many scenes advanced by the same launches. Each scene's result must be the one
it gets alone (bit for bit: the per-particle arithmetic and summation order do not depend
on the other scenes), and scenes may join and leave between runs."""
import numpy as np
import pytest

import oracle
from paper_1301_1714_gb300 import dem, scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1301_1714_gb300 import _build
    _build.build()
    dem.lib()
    return torch


def alone(sc, steps, stream=None):
    with dem.Simulation(sc.params, sc.x, sc.v, sc.w, sc.r, cuda_stream=stream) as s:
        s.step(steps)
        return s.state()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_each_scene_in_the_mix_equals_the_scene_alone(torch_cuda, precision):
    torch = torch_cuda
    stream = torch.cuda.Stream()
    mix = [scenes.box_lattice_n(seed=30 + k, n=n, e=e, mu=mu, precision=precision)
           for k, (n, e, mu) in enumerate([(1024, 0.9, 0.3), (1500, 0.6, 0.5), (3000, 0.8, 0.1), (2048, 0.95, 0.6)])]
    budgets = [60, 100, 100, 40]
    b = dem.dem_batch_create(precision=precision, cuda_stream=stream.cuda_stream)
    try:
        slots = [dem.dem_batch_add(b, sc.params, sc.x, sc.v, sc.w, sc.r, bud) for sc, bud in zip(mix, budgets)]
        done = []
        for _ in range(10):
            done += dem.dem_batch_run(b, 1000)
            if len(done) == len(mix):
                break
        assert sorted(done) == sorted(slots)
        for sc, sl, bud in zip(mix, slots, budgets):
            n, steps_done, budget = dem.dem_batch_info(b, sl)
            assert (n, steps_done, budget) == (sc.n, bud, bud)
            xb, vb, wb = dem.dem_batch_get_state(b, sl, sc.n)
            xa, va, wa = alone(sc, bud)
            assert np.array_equal(xa, xb) and np.array_equal(va, vb) and np.array_equal(wa, wb)
    finally:
        dem.dem_batch_destroy(b)


def test_scenes_join_and_leave_between_runs(torch_cuda):
    """Continuous batching: a scene admitted while others are mid-run, and a finished scene
    removed, leave every other scene's trajectory unchanged."""
    torch = torch_cuda
    stream = torch.cuda.Stream()
    A = scenes.box_lattice_n(seed=41, n=2000, precision="fp32")
    B = scenes.box_lattice_n(seed=42, n=1200, precision="fp32", e=0.7)
    C = scenes.drum(seed=43, n=2500)
    b = dem.dem_batch_create(precision="fp32", cuda_stream=stream.cuda_stream)
    try:
        sa = dem.dem_batch_add(b, A.params, A.x, A.v, A.w, A.r, 150)
        sb = dem.dem_batch_add(b, B.params, B.x, B.v, B.w, B.r, 50)
        assert dem.dem_batch_run(b, 1000) == [sb]          # B finishes first, A is at 50
        xb, _, _ = dem.dem_batch_get_state(b, sb, B.n)
        dem.dem_batch_remove(b, sb)
        sc_ = dem.dem_batch_add(b, C.params, C.x, C.v, C.w, C.r, 70)
        assert dem.dem_batch_run(b, 1000) == [sc_]         # A at 120, C at 70
        xc, _, _ = dem.dem_batch_get_state(b, sc_, C.n)
        assert dem.dem_batch_run(b, 1000) == [sa]
        xa, _, _ = dem.dem_batch_get_state(b, sa, A.n)
        assert dem.dem_batch_run(b, 1000) == []
    finally:
        dem.dem_batch_destroy(b)
    assert np.array_equal(xa, alone(A, 150)[0])
    assert np.array_equal(xb, alone(B, 50)[0])
    assert np.array_equal(xc, alone(C, 70)[0])
    ref = oracle.State(A.params.copy(precision="fp64"), A.x, A.v, A.w, A.r).run(150)
    assert np.max(np.abs(xa - ref.x)) <= 1e-9


def test_graph_replay_equals_plain_launches(torch_cuda):
    """dem_step on a non-default stream replays a captured two-step CUDA graph; the
    result equals plain launches on the legacy stream bit for bit."""
    torch = torch_cuda
    stream = torch.cuda.Stream()
    sc = scenes.box_rsa(seed=44, n=3000)
    xa = alone(sc, 101)[0]
    xb = alone(sc, 101, stream=stream.cuda_stream)[0]
    assert np.array_equal(xa, xb)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_list_mode_graph_with_conditional_sort_equals_plain_launches(torch_cuda, precision):
    """In list mode the replayed step graph runs the sort as a conditional node whose
    condition the device sets; the result equals plain launches bit for bit, and the
    launch count includes exactly the sorts that ran."""
    torch = torch_cuda
    stream = torch.cuda.Stream()
    sc = scenes.drum(seed=9, n=5000, precision=precision)
    v = np.random.default_rng(9).normal(0.0, 1.0, size=sc.x.shape)
    skin = 0.1e-3
    p = sc.params.copy(resort_interval=0, skin=skin, cell_size=sc.params.cell_size + skin)
    out = []
    for st in (None, stream.cuda_stream):
        with dem.Simulation(p, sc.x, v, sc.w, sc.r, cuda_stream=st) as s:
            s0 = s.diagnostics()["sorts"]
            l0 = dem.dem_launch_count(s.h)
            s.step(241)
            launches = dem.dem_launch_count(s.h) - l0
            out.append((s.state(), launches, s.diagnostics()["sorts"] - s0))
    (a, la, sa), (b, lb, sb) = out
    for u, w in zip(a, b):
        assert np.array_equal(u, w)
    assert sa == sb and sa >= 3
    # plain: 11 kernels per step (force pass, 9 sort kernels that return early when the
    # step does not sort, bookkeeping); graph: force pass, condition and bookkeeping per
    # step plus the 9 sort kernels of each sort that ran (the last, odd step runs plain)
    force, body = 1, 9
    plain = force + body + 1
    assert la == 241 * plain
    assert lb == 240 * (force + 2) + plain + body * sa or lb == 240 * (force + 2) + plain + body * (sa - 1)
    # phase timing on a stream: force pass plain, the sort tail as a small graph per step
    with dem.Simulation(p, sc.x, v, sc.w, sc.r, cuda_stream=stream.cuda_stream) as s:
        dem.dem_set_timing(s.h, True)
        l0 = dem.dem_launch_count(s.h)
        s.step(241)
        lt = dem.dem_launch_count(s.h) - l0
        ph = dem.dem_get_phase_times(s.h)
        c = s.state()
    for u, w in zip(a, c):
        assert np.array_equal(u, w)
    assert lt == 241 * (force + 2) + body * sa
    assert ph[0] > 0 and ph[1] > 0 and ph[2] == 241 and ph[3] == 241


def test_cancelled_scene_leaves_others_unchanged(torch_cuda):
    """A request cancelled mid-run (removed before its budget) does not disturb the rest."""
    torch = torch_cuda
    stream = torch.cuda.Stream()
    A = scenes.box_lattice_n(seed=51, n=1800, precision="fp32")
    B = scenes.box_lattice_n(seed=52, n=2600, precision="fp32", mu=0.5)
    b = dem.dem_batch_create(precision="fp32", cuda_stream=stream.cuda_stream)
    try:
        sa = dem.dem_batch_add(b, A.params, A.x, A.v, A.w, A.r, 120)
        sb = dem.dem_batch_add(b, B.params, B.x, B.v, B.w, B.r, 500)
        assert dem.dem_batch_run(b, 40) == []
        dem.dem_batch_remove(b, sb)                        # cancelled at step 40 of 500
        assert dem.dem_batch_run(b, 1000) == [sa]
        xa, _, _ = dem.dem_batch_get_state(b, sa, A.n)
        with pytest.raises(dem.DemError):
            dem.dem_batch_get_state(b, sb, B.n)
    finally:
        dem.dem_batch_destroy(b)
    assert np.array_equal(xa, alone(A, 120)[0])


def test_injected_allocation_failure_is_reported_and_recoverable(torch_cuda, monkeypatch):
    """Host-side fault injection (DEM_FAULT=alloc): the allocation error comes back as
    DEM_ERR_OOM and the same handle works once the fault is gone."""
    sc = scenes.box_lattice(seed=3)
    h = dem.dem_create(dem.config_from_params(sc.params))
    try:
        dem.dem_set_walls(h, sc.params.walls)
        monkeypatch.setenv("DEM_FAULT", "alloc")
        with pytest.raises(dem.DemError) as e:
            dem.dem_set_particles(h, sc.x, sc.v, sc.w, sc.r)
        assert e.value.status == 2 and "injected" in dem.dem_last_error(h)
        monkeypatch.delenv("DEM_FAULT")
        dem.dem_set_particles(h, sc.x, sc.v, sc.w, sc.r)
        dem.dem_step(h, 5)
    finally:
        dem.dem_destroy(h)


def listed(p, skin_frac=0.1):
    skin = skin_frac * 1e-3
    return p.copy(resort_interval=0, skin=skin, cell_size=p.cell_size + skin)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_list_mode_batch_scene_equals_alone_and_oracle(torch_cuda, precision):
    """A batch of scenes in list mode (each with its own skin) sorts all together when any
    particle has moved half its scene's skin; because a particle's contacts are summed in
    ascending partner id, each scene still gets the bits of its own run, and follows the
    oracle (FP64 within 1e-9 m)."""
    torch = torch_cuda
    stream = torch.cuda.Stream()
    mix = [scenes.box_lattice_n(seed=50 + k, n=n, e=e, mu=mu, precision=precision)
           for k, (n, e, mu) in enumerate([(1024, 0.9, 0.3), (1500, 0.6, 0.5), (2048, 0.95, 0.6)])]
    mix = [type(sc)(**dict(sc.__dict__, params=listed(sc.params, f))) for sc, f in zip(mix, (0.1, 0.05, 0.2))]
    budgets = [300, 200, 250]
    b = dem.dem_batch_create(precision=precision, cuda_stream=stream.cuda_stream)
    try:
        slots = [dem.dem_batch_add(b, sc.params, sc.x, sc.v, sc.w, sc.r, bud) for sc, bud in zip(mix, budgets)]
        done = []
        for _ in range(10):
            done += dem.dem_batch_run(b, 1000)
            if len(done) == len(mix):
                break
        assert sorted(done) == sorted(slots)
        for sc, sl, bud in zip(mix, slots, budgets):
            xb, vb, wb = dem.dem_batch_get_state(b, sl, sc.n)
            xa, va, wa = alone(sc, bud)
            assert np.array_equal(xa, xb) and np.array_equal(va, vb) and np.array_equal(wa, wb)
            if precision == "fp64":
                ref = oracle.State(sc.params, sc.x, sc.v, sc.w, sc.r).run(bud)
                assert np.max(np.abs(xb - ref.x)) <= 1e-9
    finally:
        dem.dem_batch_destroy(b)


def test_list_mode_batch_scene_joining_mid_run_equals_alone(torch_cuda):
    torch = torch_cuda
    stream = torch.cuda.Stream()
    first = scenes.box_lattice_n(seed=61, n=2000, precision="fp32")
    late = scenes.box_lattice_n(seed=62, n=1200, e=0.7, mu=0.4, precision="fp32")
    first = type(first)(**dict(first.__dict__, params=listed(first.params)))
    late = type(late)(**dict(late.__dict__, params=listed(late.params, 0.15)))
    b = dem.dem_batch_create(precision="fp32", cuda_stream=stream.cuda_stream)
    try:
        s1 = dem.dem_batch_add(b, first.params, first.x, first.v, first.w, first.r, 400)
        dem.dem_batch_run(b, 150)
        s2 = dem.dem_batch_add(b, late.params, late.x, late.v, late.w, late.r, 300)
        done = []
        for _ in range(10):
            done += dem.dem_batch_run(b, 500)
            if len(done) == 2:
                break
        for sc, sl, bud in ((first, s1, 400), (late, s2, 300)):
            xb, _, _ = dem.dem_batch_get_state(b, sl, sc.n)
            xa, _, _ = alone(sc, bud)
            assert np.array_equal(xa, xb)
        # a scene with another sort policy is refused
        with pytest.raises(dem.DemError):
            dem.dem_batch_add(b, late.params.copy(resort_interval=1, skin=0.0), late.x, late.v, late.w, late.r, 10)
    finally:
        dem.dem_batch_destroy(b)
