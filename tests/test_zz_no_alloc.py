"""dem_sort_cells_static: the cell map and (cell, id) sort for callers that cannot
allocate device memory, e.g. a process that has already reserved all of the GPU's
memory for its own pool, or a loop that forbids cudaMalloc after start-up because it can
block or synchronise the device. The entry point takes the caller's buffers and keeps
its temporaries in one fixed array of the library.

Its output must equal the handle-based path's (dem_set_particles in FP64 mode, read back
through dem_debug_snapshot) bit for bit, on two calls in a row that share that array.
This file is collected last on purpose: it also runs correctly after every other test.
"""
import numpy as np
import pytest

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


def handle_result(sc):
    p = sc.params.copy(precision="fp64")
    with dem.Simulation(p, sc.x, sc.v, sc.w, sc.r) as s:
        origin, cell, dims = dem.dem_get_grid(s.h)
        cell_of, order, _ = s.snapshot(with_pairs=False)
    return origin, cell, dims, cell_of, order


def static_buffers(torch, sc, dims):
    n = sc.n
    ncells = dims[0] * dims[1] * dims[2]
    x = torch.tensor(sc.x, dtype=torch.float64, device="cuda")
    cell_of = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    order = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    cs = torch.full((ncells + 1,), -1, dtype=torch.int32, device="cuda")
    return x, cell_of, order, cs


def check(sc, got, ref):
    origin, cell, dims, hcell, horder = ref
    cell_of, order, cs = (t.cpu().numpy().view(np.uint32) for t in got)
    assert np.array_equal(cell_of, hcell)
    assert np.array_equal(order, horder)
    ncells = dims[0] * dims[1] * dims[2]
    expect = np.concatenate([[0], np.cumsum(np.bincount(hcell, minlength=ncells))]).astype(np.uint32)
    assert np.array_equal(cs, expect)


def test_static_sort_matches_the_handle_on_two_calls_in_a_row(torch_cuda):
    torch = torch_cuda
    stream = torch.cuda.Stream()
    scenes_ = [scenes.box_rsa(seed=21, n=3000), scenes.drum(seed=22, n=5001)]
    refs = [handle_result(sc) for sc in scenes_]
    bufs = [static_buffers(torch, sc, ref[2]) for sc, ref in zip(scenes_, refs)]
    torch.cuda.synchronize()
    # two calls in a row, different sizes, sharing the fixed scratch array
    for sc, ref, (x, cell_of, order, cs) in zip(scenes_, refs, bufs):
        origin, cell, dims = ref[0], ref[1], ref[2]
        dem.dem_sort_cells_static(x, origin, cell, dims, cell_of, order, cs, stream.cuda_stream)
        stream.synchronize()
        check(sc, (cell_of, order, cs), ref)
    # again on the first scene: the array still holds the second call's contents
    sc, ref, (x, cell_of, order, cs) = scenes_[0], refs[0], bufs[0]
    free_before = torch.cuda.mem_get_info()[0]
    dem.dem_sort_cells_static(x, ref[0], ref[1], ref[2], cell_of, order, cs, stream.cuda_stream)
    stream.synchronize()
    assert torch.cuda.mem_get_info()[0] == free_before   # nothing was allocated on the device
    check(sc, (cell_of, order, cs), ref)


def test_static_sort_rejects_sizes_beyond_its_maximum(torch_cuda):
    torch = torch_cuda
    n = dem.STATIC_SORT_MAX_N + 1
    x = torch.zeros((n, 3), dtype=torch.float64, device="cuda")
    out = torch.empty(n, dtype=torch.int32, device="cuda")
    cs = torch.empty(9, dtype=torch.int32, device="cuda")
    with pytest.raises(dem.DemError) as e:
        dem.dem_sort_cells_static(x, (0, 0, 0), 1.0, (2, 2, 2), out, out, cs)
    assert e.value.status == 1
    x1 = torch.zeros((1, 3), dtype=torch.float64, device="cuda")
    o1 = torch.empty(1, dtype=torch.int32, device="cuda")
    with pytest.raises(dem.DemError):
        dem.dem_sort_cells_static(x1, (0, 0, 0), 1.0, (1025, 1024, 1), o1, o1, cs)


def test_static_sort_at_its_maximum_sizes_matches_the_oracle(torch_cuda):
    """262,144 particles on a grid of 128 x 128 x 64 = 1,048,576 cells (both maxima),
    against the oracle's cell map, (cell, id) order and cell-start table directly."""
    import oracle
    torch = torch_cuda
    n = dem.STATIC_SORT_MAX_N
    dims = (128, 128, 64)
    assert dims[0] * dims[1] * dims[2] == dem.STATIC_SORT_MAX_CELLS
    cell = 1.0 / 64
    rng = np.random.default_rng(23)
    xh = rng.uniform(0.0, 1.0, size=(n, 3)) * np.array(dims) * cell
    xh[:100] = rng.uniform(-0.5, 2.5, size=(100, 3))          # some outside the grid (clamped)
    p = scenes.Params(precision="fp64", cell_size=cell, domain_lo=(0.0, 0.0, 0.0),
                      domain_hi=tuple(d * cell for d in dims))
    assert oracle.grid_dims(p) == dims
    key, _ = oracle.cell_keys(p, xh)
    order, skey = oracle.sort_by_cell(key)
    start = oracle.cell_start(skey, dims[0] * dims[1] * dims[2])
    x = torch.tensor(xh, dtype=torch.float64, device="cuda")
    cell_of = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    gorder = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    cs = torch.full((dims[0] * dims[1] * dims[2] + 1,), -1, dtype=torch.int32, device="cuda")
    for _ in range(2):   # twice in a row on the shared array
        dem.dem_sort_cells_static(x, (0.0, 0.0, 0.0), cell, dims, cell_of, gorder, cs)
        torch.cuda.synchronize()
        assert np.array_equal(cell_of.cpu().numpy().view(np.uint32).astype(np.uint64), key)
        assert np.array_equal(gorder.cpu().numpy().view(np.uint32), order)
        assert np.array_equal(cs.cpu().numpy().view(np.uint32).astype(np.int64), start)


def test_static_sort_rejects_huge_axes_before_forming_the_cell_count(torch_cuda):
    torch = torch_cuda
    x1 = torch.zeros((1, 3), dtype=torch.float64, device="cuda")
    o1 = torch.empty(1, dtype=torch.int32, device="cuda")
    cs = torch.empty(9, dtype=torch.int32, device="cuda")
    for dims in ((2 ** 40, 2 ** 40, 2 ** 40), (1, 1, dem.STATIC_SORT_MAX_CELLS + 1), (0, 4, 4)):
        with pytest.raises(dem.DemError) as e:
            dem.dem_sort_cells_static(x1, (0, 0, 0), 1.0, dims, o1, o1, cs)
        assert e.value.status == 1
