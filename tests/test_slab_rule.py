"""Host side of the slab decomposition: the boundaries (dem_slab_bounds, no GPU needed)
and the ghost-layer rule, checked by brute force against the oracle's contact pairs."""
import numpy as np
import pytest

import oracle
from paper_1301_1714_gb300 import dem, scenes


def test_bounds_split_counts_evenly():
    rng = np.random.default_rng(5)
    z = rng.normal(size=10_007)
    for S in range(1, dem.DEM_MAX_SLABS + 1):
        b = dem.dem_slab_bounds(z, S)
        assert b[0] == -np.inf and b[-1] == np.inf
        assert np.all(np.diff(b) >= 0)
        owner = np.searchsorted(b[1:-1], z, side="right")    # boundaries at or below z
        counts = np.bincount(owner, minlength=S)
        want = np.diff([(len(z) * k) // S for k in range(S + 1)])
        assert np.array_equal(counts, want)                  # distinct values: exact quantile split
        zs = np.sort(z)
        for k in range(1, S):
            assert b[k] == zs[(len(z) * k) // S]


def test_bounds_with_ties_and_few_values():
    b = dem.dem_slab_bounds(np.array([1.0, 1.0, 1.0, 2.0]), 4)
    assert list(b[1:-1]) == [1.0, 1.0, 2.0]
    b = dem.dem_slab_bounds(np.array([3.0, -1.0]), 5)        # more slabs than values
    assert list(b[1:-1]) == [-1.0, -1.0, 3.0, 3.0]
    b = dem.dem_slab_bounds(np.zeros(0), 3)
    assert b[0] == -np.inf and np.all(b[1:] == np.inf)


def test_bounds_reject_bad_arguments():
    with pytest.raises(dem.DemError):
        dem.dem_slab_bounds(np.ones(4), 0)
    with pytest.raises(dem.DemError):
        dem.dem_slab_bounds(np.ones(4), dem.DEM_MAX_SLABS + 1)
    with pytest.raises(dem.DemError):
        dem.dem_slab_bounds(np.array([0.0, np.inf]), 2)
    with pytest.raises(dem.DemError):
        dem.dem_slab_bounds(np.array([np.nan, 1.0]), 2)


@pytest.mark.parametrize("S", [2, 3, 6])
def test_every_contact_partner_is_in_the_owners_slab(S):
    """For every contact (distance < r_i + r_j) among overlapping polydisperse spheres,
    the partner of a particle owned by slab s lies in s's range widened by one cell edge
    (the grid's, >= 2 r_max), so it is owned by s or is one of s's ghosts: no contact is
    lost by the decomposition."""
    rng = np.random.default_rng(31)
    n = 6000
    x = rng.uniform(0.0, 0.04, size=(n, 3))
    r = rng.uniform(0.9e-3, 1.1e-3, size=n).astype(np.float32)
    pairs = oracle.pairs_brute(x, r)
    assert len(pairs) > 1000
    G = scenes.auto_cell_size(float(r.max()))
    assert G >= 2 * float(r.max())
    for axis in range(3):
        b = dem.dem_slab_bounds(x[:, axis], S)
        z = x[:, axis]
        owner = np.searchsorted(b[1:-1], z, side="right")
        for i, j in ((pairs[:, 0], pairs[:, 1]), (pairs[:, 1], pairs[:, 0])):
            s = owner[i]
            assert np.all((z[j] >= b[s] - G) & (z[j] < b[s + 1] + G))
