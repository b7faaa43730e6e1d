"""List mode (sort only after a particle moved skin/2) at the edges of its capacities, and
its brick cell order seen through the parity hooks.

* A neighbour list holds at most 64 candidates whatever max_contacts is: a scene whose
  lists stay within that runs like the oracle with max_contacts = 48, and one whose lists
  overflow (a skin so large that a particle has more than 64 candidates) makes dem_step
  report DEM_ERR_CAPACITY instead of dropping contacts.
* List mode numbers the cells brick by brick internally; the parity hooks still report
  the oracle's row-major cell keys and (cell, id) order, bit for bit.
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


def listed(params, skin):
    return params.copy(resort_interval=0, skin=skin, cell_size=params.cell_size + skin)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_list_mode_with_48_contact_slots_matches_oracle(precision):
    """Skin 2.4 mm: lists of up to 55 candidates (most beyond 32, so both words of the
    64-bit candidate mask are used)."""
    sc = scenes.drum(seed=7, n=3001)
    p = listed(sc.params.copy(precision=precision), 2.4e-3)
    ref = oracle.State(sc.params.copy(precision="fp64"), sc.x, sc.v, sc.w, sc.r).run(60)
    with dem.Simulation(p, sc.x, sc.v, sc.w, sc.r, max_contacts=48) as s:
        s.step(60)
        x, _, _ = s.state()
    tol = 1e-12 if precision == "fp64" else 1e-9
    assert np.max(np.abs(x - ref.x)) <= tol


def test_list_overflow_is_reported_not_dropped():
    """Skin of three radii: up to 80 candidates within r_i + r_j + skin per particle,
    more than a list holds."""
    sc = scenes.drum(seed=7, n=3001, precision="fp32")
    p = listed(sc.params, 3.0e-3)
    with pytest.raises(dem.DemError) as err:
        with dem.Simulation(p, sc.x, sc.v, sc.w, sc.r, max_contacts=48) as s:
            s.step(2)
    assert err.value.status == dem.DEM_ERR_CAPACITY
    assert "neighbour list" in str(err.value)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_list_mode_reports_row_major_keys_and_order(precision):
    sc = scenes.drum(seed=3, n=4000)
    p = listed(sc.params.copy(precision=precision), 0.1e-3)
    key, _ = oracle.cell_keys(p, sc.x)
    order, _ = oracle.sort_by_cell(key)
    with dem.Simulation(p, sc.x, sc.v, sc.w, sc.r) as s:
        cell, gorder, _ = s.snapshot(with_pairs=False)
    assert np.array_equal(cell.astype(np.uint64), key)
    assert np.array_equal(gorder, order)
