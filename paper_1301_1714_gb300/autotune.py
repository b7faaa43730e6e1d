"""Autotuner: picks the force kernel's block size and the sort policy (every step, or
skin-driven with neighbour lists and a given skin, which also sets the cell size) for a
scene by timing short runs of each candidate on the device.

Every candidate finds exactly the same contacts, so the choice changes speed, not the
physics (results differ only by the rounding of the per-particle sums).
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import List, Optional, Sequence, Tuple

from . import dem

# (block size, resort_interval, skin as a fraction of the largest radius)
DEFAULT_CANDIDATES: Tuple[Tuple[int, int, float], ...] = (
    (256, 1, 0.0), (128, 1, 0.0),
    (256, 0, 0.1), (128, 0, 0.05), (128, 0, 0.1), (128, 0, 0.15), (128, 0, 0.2), (96, 0, 0.1),
)


@dataclass
class Choice:
    block: int
    resort: int
    skin_frac: float
    ms_per_step: float
    force_ms: float
    sort_ms: float


def apply(params, rmax: float, choice: Choice):
    """Parameters with the tuned sort policy (cell size = 2 r_max (1 + 2^-10) + skin)."""
    from .scenes import auto_cell_size
    skin = choice.skin_frac * rmax
    return params.copy(resort_interval=choice.resort, skin=skin, cell_size=auto_cell_size(rmax, skin))


def tune(params, x, v, w, r, candidates: Sequence[Tuple[int, int, float]] = DEFAULT_CANDIDATES, steps: int = 150,
         warmup: int = 50, device: int = 0, cuda_stream=None, max_contacts: int = 0) -> Tuple[Choice, List[Choice]]:
    """Times each candidate for `steps` steps after `warmup` (long enough that a list-mode
    candidate has sorted once with known contact counts, which order its windows, and that
    the timed steps hold several sorts); returns the fastest and the table."""
    rmax = float(max(r)) if len(r) else 1.0
    table: List[Choice] = []
    for block, resort, sk in candidates:
        c = Choice(block, resort, sk, 0.0, 0.0, 0.0)
        p = apply(params, rmax, c)
        try:
            h = dem.dem_create(dem.config_from_params(p, block_size=block, max_contacts=max_contacts), device,
                               cuda_stream)
        except dem.DemError:
            continue                      # a candidate this configuration does not allow
        try:
            dem.dem_set_walls(h, p.walls)
            dem.dem_set_particles(h, x, v, w, r)
            dem.dem_step(h, warmup)
            dem.dem_set_timing(h, True)
            dem.dem_step(h, steps)
            ph = dem.dem_get_phase_times(h)
        except dem.DemError as e:
            if e.status != dem.DEM_ERR_CAPACITY:
                raise
            continue                      # too many contacts for the capacity: not a candidate
        finally:
            dem.dem_destroy(h)
        c.force_ms = ph[0] / max(ph[2], 1)
        c.sort_ms = ph[1] / max(ph[3], 1)
        c.ms_per_step = c.force_ms + c.sort_ms
        table.append(c)
    if not table:
        raise RuntimeError("no autotune candidate ran (contact capacity too small for every one)")
    best = min(table, key=lambda t: t.ms_per_step)
    return best, table


# candidates for a batch of many small scenes: the whole batch sorts when any particle of
# any scene has moved half its skin, so larger skins pay off sooner than for one scene
BATCH_CANDIDATES: Tuple[Tuple[int, int, float], ...] = (
    (256, 1, 0.0), (128, 0, 0.1), (256, 0, 0.1), (128, 0, 0.2), (128, 0, 0.3),
)


def tune_batch(mix, precision: str = "fp32", candidates: Sequence[Tuple[int, int, float]] = BATCH_CANDIDATES,
               steps: int = 60, warmup: int = 20, device: int = 0, cuda_stream=None,
               max_contacts: int = 0) -> Tuple[Choice, List[Choice]]:
    """The block size and sort policy for a batch of scenes (each scene's skin is the
    fraction of its own largest radius), by timing short runs of the whole batch."""
    import time
    table: List[Choice] = []
    for block, resort, sk in candidates:
        c = Choice(block, resort, sk, 0.0, 0.0, 0.0)
        b = dem.dem_batch_create(precision=precision, max_contacts=max_contacts, block_size=block, device=device,
                                 cuda_stream=cuda_stream)
        try:
            for sc in mix:
                p = apply(sc.params, float(max(sc.r)), c)
                dem.dem_batch_add(b, p, sc.x, sc.v, sc.w, sc.r, warmup + steps + 1)
            dem.dem_batch_run(b, warmup)
            t0 = time.perf_counter()
            dem.dem_batch_run(b, steps)
            c.ms_per_step = (time.perf_counter() - t0) * 1e3 / steps
        except dem.DemError as e:
            if e.status != dem.DEM_ERR_CAPACITY:
                raise
            continue
        finally:
            dem.dem_batch_destroy(b)
        table.append(c)
    if not table:
        raise RuntimeError("no autotune candidate ran for the batch")
    return min(table, key=lambda t: t.ms_per_step), table
