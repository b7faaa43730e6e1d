"""The benchmark's own size and launch configuration: the 4,194,304-sphere drum in FP32
mode with skin-driven sorting and neighbour lists (the autotuner's usual choice) and
256-thread blocks. The oracle evaluates the same state in full (its grid search makes
this a few seconds of CPU), so the pair set and every particle's force are compared.
"""
import numpy as np
import pytest

import oracle
from paper_1301_1714_gb300 import dem, scenes

pytestmark = pytest.mark.gpu

N = 4_194_304


@pytest.fixture(scope="module")
def bed():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1301_1714_gb300 import _build
    _build.build()
    dem.lib()
    sc = scenes.drum(seed=1, n=N, precision="fp32")
    # squeeze the generated bed toward the drum axis so that most spheres touch
    x = sc.x.copy()
    x[:, 1:] *= 0.9985
    rng = np.random.default_rng(5)
    w = rng.normal(0.0, 10.0, size=x.shape)
    v = rng.normal(0.0, 0.05, size=x.shape)
    skin = 0.1 * float(sc.r.max())
    p = sc.params.copy(resort_interval=0, skin=skin, cell_size=sc.params.cell_size + skin)
    return sc, p, x, v, w


def test_full_size_pairs_and_forces_match_oracle(bed):
    sc, p, x, v, w = bed
    with dem.Simulation(p, x, v, w, sc.r, block_size=256) as s:
        F, T = s.forces()
        _, _, gp = s.snapshot()
    po = sc.params.copy(precision="fp64")
    Fo, To, _, stats = oracle.forces(po, x, v, w, sc.r, pair_mode="grid")
    ref = oracle.pairs_grid(po, x, sc.r)
    assert len(ref) > N                      # a contact-rich bed
    # pair set: equal except pairs inside the FP32 decision band |d^2 - R^2| <= 2^-36 R^2
    A = ref[:, 0].astype(np.int64) * N + ref[:, 1]
    B = gp[:, 0].astype(np.int64) * N + gp[:, 1]
    diff = np.setxor1d(A, B)
    if len(diff):
        i, j = diff // N, diff % N
        d2 = np.sum((x[j] - x[i]) ** 2, axis=1)
        R2 = (sc.r[i].astype(np.float64) + sc.r[j]) ** 2
        assert np.all(np.abs(d2 - R2) <= 2.0 ** -36 * R2)
    # forces and torques, normalised per particle
    rr = sc.r.astype(np.float64)
    m = p.rho * 4.0 / 3.0 * np.pi * rr ** 3
    S = m * 9.81
    i, j = ref[:, 0].astype(np.int64), ref[:, 1].astype(np.int64)
    delta = rr[i] + rr[j] - np.linalg.norm(x[j] - x[i], axis=1)
    meff = m[i] * m[j] / (m[i] + m[j])
    c = (p.kn * delta + p.alpha * np.sqrt(p.kn * meff) * np.linalg.norm(v[i] - v[j], axis=1)) * (1 + p.mu)
    np.add.at(S, i, c)
    np.add.at(S, j, c)
    # wall contacts (drum shell and caps) add their own scale
    rho = np.hypot(x[:, 1], x[:, 2])
    Rd, L = sc.params.walls[0]["radius"], sc.params.walls[2]["p"][0]
    for dw in (rho + rr - Rd, rr - x[:, 0], x[:, 0] + rr - L):
        on = dw > 0
        S[on] += (p.kn * dw[on] + p.alpha * np.sqrt(p.kn * m[on]) * (np.linalg.norm(v[on], axis=1) + 0.7)) * (1 + p.mu)
    eF = np.linalg.norm(F - Fo, axis=1) / S
    eT = np.linalg.norm(T - To, axis=1) / (S * rr)
    assert eF.max() <= 1e-5, eF.max()
    assert eT.max() <= 1e-5, eT.max()


def test_full_size_run_keeps_invariants(bed):
    """200 steps at full size: nothing becomes non-finite, no sphere leaves the drum,
    sorts happen far less often than steps, and the largest overlap stays small."""
    sc, p, x, v, w = bed
    with dem.Simulation(p, sc.x, np.zeros_like(v), np.zeros_like(w), sc.r, block_size=256) as s:
        s.step(200)
        xo, vo, wo = s.state()
        d = s.diagnostics()
    assert np.all(np.isfinite(xo)) and np.all(np.isfinite(vo)) and np.all(np.isfinite(wo))
    Rd = sc.params.walls[0]["radius"]
    assert np.max(np.hypot(xo[:, 1], xo[:, 2]) + sc.r - Rd) < 0.05e-3
    assert d["sorts"] < 100
    assert d["max_overlap"] < 0.05e-3
    assert d["pair_contacts"] > 0


def test_full_hopper_forces_match_oracle():
    """The 131,072-sphere hopper (the paper's count) with its first layer pressed into the
    plate and against the slit edges: every particle's force and torque against the
    oracle (FP32 bars), in list mode with block 128 as the bench runs it."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1301_1714_gb300 import _build
    _build.build()
    dem.lib()
    sc = scenes.hopper(seed=2)
    x = sc.x.copy()
    x[:, 2] -= 0.12e-3
    rng = np.random.default_rng(11)
    v = sc.v + rng.normal(0.0, 0.05, size=x.shape)
    w = rng.normal(0.0, 10.0, size=x.shape)
    skin = 0.1e-3
    p = sc.params.copy(resort_interval=0, skin=skin, cell_size=sc.params.cell_size + skin)
    with dem.Simulation(p, x, v, w, sc.r, block_size=128) as s:
        F, T = s.forces()
    p64 = sc.params.copy(precision="fp64")
    Fo, To, _, stats = oracle.forces(p64, x, v, w, sc.r, pair_mode="grid")
    assert stats[1] > 1000                                  # plate and slit-edge contacts
    from test_gpu_parity import assert_forces_close
    assert_forces_close(p64, x, v, sc.r, F, T, Fo, To, 1e-5)
