"""Host-side logic that needs no GPU: the autotuner's parameter mapping, the serving
loop's request stream and footprints, and the benchmark's profile bookkeeping."""
import math
import os
import sys

import numpy as np
import pytest

from paper_1301_1714_gb300 import autotune, scenes, serve

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_autotune_apply_sets_skin_and_cell_size():
    sc = scenes.drum(n=3000)
    rmax = float(sc.r.max())
    c = autotune.Choice(block=128, resort=0, skin_frac=0.1, ms_per_step=0.0, force_ms=0.0, sort_ms=0.0)
    p = autotune.apply(sc.params, rmax, c)
    assert p.resort_interval == 0 and p.skin == pytest.approx(0.1 * rmax)
    assert p.cell_size == pytest.approx(2 * rmax * (1 + 2.0 ** -10) + 0.1 * rmax)
    c1 = autotune.Choice(block=256, resort=1, skin_frac=0.0, ms_per_step=0.0, force_ms=0.0, sort_ms=0.0)
    p1 = autotune.apply(sc.params, rmax, c1)
    assert p1.resort_interval == 1 and p1.skin == 0.0
    assert p1.cell_size == pytest.approx(scenes.auto_cell_size(rmax))
    # every candidate is a valid configuration: block sizes are multiples of 32 in [32, 256]
    for block, resort, skin in autotune.DEFAULT_CANDIDATES:
        assert block % 32 == 0 and 32 <= block <= 256
        assert (resort == 1) == (skin == 0.0)


def test_poisson_requests_are_seeded_and_shaped():
    a = serve.poisson_requests(seed=5, count=40, rate=20.0, nmin=1024, nmax=8192, smin=100, smax=300)
    b = serve.poisson_requests(seed=5, count=40, rate=20.0, nmin=1024, nmax=8192, smin=100, smax=300)
    assert [r.arrival for r in a] == [r.arrival for r in b]
    assert [r.scene.n for r in a] == [r.scene.n for r in b]
    arr = np.array([r.arrival for r in a])
    assert np.all(np.diff(arr) > 0)
    assert 0.5 / 20.0 < np.mean(np.diff(arr)) < 2.0 / 20.0          # exponential gaps of mean 1/rate
    assert all(100 <= r.steps <= 300 for r in a)
    assert all(1024 * 0.5 <= r.scene.n <= 8192 * 1.5 for r in a)
    assert {r.scene.name.split("_")[0] for r in a} == {"box", "drum"}


def test_footprint_grows_with_particles_and_cells():
    small = scenes.box_lattice_n(seed=1, n=2000, precision="fp32")
    large = scenes.box_lattice_n(seed=1, n=20000, precision="fp32")
    fs, fl = serve.footprint(small), serve.footprint(large)
    assert fl > fs > serve.bytes_per_particle("fp32") * small.n
    assert serve.bytes_per_particle("fp32", 24) < serve.bytes_per_particle("fp32", 32)
    assert serve.bytes_per_particle("fp32", 24, True) > serve.bytes_per_particle("fp32", 24)
    assert serve.footprint(small, "fp64") > fs


def test_latency_stats():
    reqs = [serve.Request(arrival=float(k), rid=k, scene=None, steps=1) for k in range(10)]
    for k, r in enumerate(reqs):
        r.done = r.arrival + 0.1 * (k + 1)
    st = serve.latency_stats(reqs)
    assert st["p50_s"] == pytest.approx(0.55) and st["max_s"] == pytest.approx(1.0)


def test_bench_reads_profiled_traffic_only_for_the_profiled_kernel(tmp_path, monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    h = bench.kernel_source_hash(True)
    assert len(h) == 16 and h != bench.kernel_source_hash(False)
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "force_kernel_list_drum.md").write_text(f"kernel_source_sha256_16: {h}\ndram_bytes_per_particle: 123.5\n")
    (prof / "force_kernel_drum.md").write_text("kernel_source_sha256_16: 0000000000000000\ndram_bytes_per_particle: 9\n")
    real_join = os.path.join

    def fake_join(*parts):
        if len(parts) >= 2 and parts[1] == "profiles":
            return real_join(str(tmp_path), *parts[1:])
        return real_join(*parts)

    monkeypatch.setattr(bench.os.path, "join", fake_join)
    assert bench.profiled_traffic_per_particle(True) == 123.5
    assert bench.profiled_traffic_per_particle(False) is None          # another kernel's capture


def test_bench_workload_text_separates_the_method():
    sys.path.insert(0, ROOT)
    import bench

    class A:
        workload = "drum"
    sc = scenes.drum(n=2000)
    ours = bench.workload_desc(A, sc)
    ref = bench.workload_desc(A, sc, impl="reference")
    assert ours.split(", FP32")[0] == ref.split(", FP64")[0]
    assert "FP64 oracle" in ref and "FP32" in ours
