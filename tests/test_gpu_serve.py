"""The serving loop (continuous batching over the batch C ABI): requests that arrive while
others are on the GPU are admitted as memory frees up, and each result is the same as the
request's own run, bit for bit, and the oracle's (FP64, within 1e-9 m)."""
import numpy as np
import pytest

import oracle
from paper_1301_1714_gb300 import dem, scenes, serve

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1301_1714_gb300 import _build
    _build.build()
    dem.lib()


def requests():
    """Box-settling and drum scenes, FP64, arriving at rounds 0, 0, 2, 3, 6."""
    spec = [(0, "box", 900, 160), (0, "drum", 1500, 120), (2, "box", 1300, 200), (3, "drum", 700, 90),
            (6, "box", 2000, 140)]
    out = []
    for k, (t, kind, n, steps) in enumerate(spec):
        sc = (scenes.box_lattice_n(seed=70 + k, n=n, precision="fp64") if kind == "box"
              else scenes.drum(seed=70 + k, n=n, precision="fp64"))
        out.append(serve.Request(arrival=float(t), rid=k, scene=sc, steps=steps))
    return out


@pytest.mark.parametrize("skin_frac", [None, 0.1])
def test_served_results_equal_alone_runs_and_oracle(skin_frac):
    import torch
    stream = torch.cuda.Stream()
    reqs = requests()
    # room for about two of the scenes at a time, so later ones wait for memory
    probe = serve.Server(1 << 40, precision="fp64", skin_frac=skin_frac)
    fps = [probe.footprint(type(r)(arrival=r.arrival, rid=r.rid, scene=r.scene, steps=r.steps,
                                   params=probe.run_params(r.scene))) for r in reqs]
    probe.close()
    budget = int(sorted(fps)[-1] + sorted(fps)[-2])
    rounds = {"now": 0.0}
    with serve.Server(budget, precision="fp64", chunk=40, cuda_stream=stream.cuda_stream, keep_results=True,
                      skin_frac=skin_frac) as srv:
        for r in reqs:
            srv.submit(r)
        peak_used, overlapped = 0, False
        for _ in range(200):
            if len(srv.finished) == len(reqs):
                break
            srv.step(lambda: rounds["now"])
            peak_used = max(peak_used, srv.used)
            overlapped |= len(srv.resident) > 1
            rounds["now"] += 1.0
        assert len(srv.finished) == len(reqs)
        assert peak_used <= budget and overlapped
        # a request that arrived while another was resident was admitted before that one finished
        fin = sorted(srv.finished, key=lambda r: r.rid)
        assert any(a.admitted > b.admitted and a.admitted < b.done for a in fin for b in fin)
        for r in fin:
            sc = r.scene
            with dem.Simulation(r.params, sc.x, sc.v, sc.w, sc.r, cuda_stream=stream.cuda_stream) as s:
                s.step(r.steps)
                xa, _, _ = s.state()
            assert np.array_equal(r.result, xa), f"request {r.rid} differs from its own run"
            ref = oracle.State(sc.params, sc.x, sc.v, sc.w, sc.r).run(r.steps)
            assert np.max(np.abs(r.result - ref.x)) <= 1e-9


def test_admission_footprint_bounds_the_batch_bytes():
    """The footprint the server admits by is an upper bound of what the batch allocates."""
    reqs = requests()
    for skin_frac in (None, 0.1):
        with serve.Server(1 << 40, precision="fp64", max_contacts=24, skin_frac=skin_frac) as srv:
            total = 0
            for r in reqs:
                srv.submit(r)
                total += srv.footprint(r)
            srv.step(lambda: 10.0)      # everything has arrived and fits: one batch
            assert len(srv.resident) + len(srv.finished) == len(reqs)
            assert dem.dem_batch_device_bytes(srv.b) <= total
