"""Continuous-batching server of DEM scenes over the batch C ABI.

Requests (a scene and a step budget) arrive over time. The server admits waiting
requests into one device-resident batch while the batch's device-memory footprint stays
within a budget, advances all admitted scenes together (one launch sequence per step
for every scene, replayed as a CUDA graph), returns each scene's final state when it
reaches its budget, removes it and admits the next ones. Scenes that arrive while others
are running join at the next step chunk, so their work overlaps on the device.

Latency of a request = completion time - arrival time (wall clock).
"""
from __future__ import annotations

import heapq
import time
from dataclasses import dataclass, field
from typing import Dict, List, Optional

import numpy as np

from . import dem

# device bytes of a batch, as dem_batch_device_bytes counts them: per particle two state
# sets, two spring buffers of max_contacts slots, the sort arrays, the staging and map
# buffers, and (list mode) the neighbour list of 64 entries with its count, reference
# position and window maps; per cell the counts and the starts
LIST_CAP = 64
BYTES_PER_CELL = 8


def bytes_per_particle(precision: str = "fp32", max_contacts: int = 32, list_mode: bool = False) -> int:
    state, t = (68, 4) if precision == "fp32" else (80, 8)
    m = max_contacts or 32
    b = 2 * state + 2 * (4 + 4 * m + t * 3 * m) + 20 + 76 + 4
    if list_mode:
        b += 4 + 4 * LIST_CAP + 4 + 16 + 8
    return b


@dataclass(order=True)
class Request:
    arrival: float
    rid: int = field(compare=False)
    scene: object = field(compare=False)
    steps: int = field(compare=False)
    slot: int = field(default=-1, compare=False)
    params: object = field(default=None, compare=False)   # what the server runs it with
    admitted: float = field(default=0.0, compare=False)
    done: float = field(default=0.0, compare=False)
    result: Optional[np.ndarray] = field(default=None, compare=False)


def footprint(scene, precision="fp32", max_contacts: int = 32) -> int:
    """Device bytes the scene adds to a batch (an upper bound of what
    dem_batch_device_bytes grows by)."""
    p = scene.params
    cells = 1
    for a in range(3):
        cells *= max(1, int(np.ceil((p.domain_hi[a] - p.domain_lo[a]) / p.cell_size)))
    per = bytes_per_particle(precision, max_contacts, p.resort_interval != 1)
    return per * scene.n + BYTES_PER_CELL * cells


class Server:
    """skin_frac: None runs every request sorting every step (as submitted); a number runs
    every request in list mode with a skin of skin_frac times its largest radius (the
    whole batch sorts when any particle has moved half its scene's skin). max_contacts
    and block_size are the batch's (dem_batch_create)."""

    def __init__(self, hbm_budget: int, precision: str = "fp32", model: str = "practical", chunk: int = 200,
                 device: int = 0, cuda_stream=None, keep_results: bool = False, max_contacts: int = 0,
                 block_size: int = 0, skin_frac=None):
        self.budget = int(hbm_budget)
        self.precision = precision
        self.chunk = int(chunk)
        self.keep = keep_results
        self.max_contacts = int(max_contacts)
        self.skin_frac = skin_frac
        self.b = dem.dem_batch_create(precision=precision, model=model, max_contacts=max_contacts,
                                      block_size=block_size, device=device, cuda_stream=cuda_stream)
        self.waiting: List[Request] = []      # heap by arrival
        self.resident: Dict[int, Request] = {}
        self.finished: List[Request] = []
        self.used = 0
        self.particle_steps = 0

    def run_params(self, scene):
        """The parameters the server runs a scene with."""
        p = scene.params
        if self.skin_frac is None:
            return p
        skin = float(self.skin_frac) * float(np.max(scene.r))
        return p.copy(resort_interval=0, skin=skin, cell_size=p.cell_size + skin)

    def footprint(self, req: Request) -> int:
        sc = req.scene
        return footprint(type(sc)(**dict(sc.__dict__, params=req.params)), self.precision, self.max_contacts or 32)

    def submit(self, req: Request):
        req.params = self.run_params(req.scene)
        heapq.heappush(self.waiting, req)

    def _admit(self, now: float):
        while self.waiting and self.waiting[0].arrival <= now:
            req = self.waiting[0]
            fp = self.footprint(req)
            if self.resident and self.used + fp > self.budget:
                break                                   # wait for memory to free up
            heapq.heappop(self.waiting)
            sc = req.scene
            req.slot = dem.dem_batch_add(self.b, req.params, sc.x, sc.v, sc.w, sc.r, req.steps)
            req.admitted = now
            self.resident[req.slot] = req
            self.used += fp

    def step(self, clock) -> bool:
        """One scheduling round: admit what has arrived and fits, advance the batch by at
        most `chunk` steps, retire finished scenes. Returns False when idle."""
        self._admit(clock())
        if not self.resident:
            return False
        fin = dem.dem_batch_run(self.b, self.chunk)
        now = clock()
        for slot in fin:
            req = self.resident.pop(slot)
            if self.keep:
                req.result = dem.dem_batch_get_state(self.b, slot, req.scene.n)[0]
            dem.dem_batch_remove(self.b, slot)
            req.done = now
            self.used -= self.footprint(req)
            self.particle_steps += req.scene.n * req.steps
            self.finished.append(req)
        return True

    def run(self, requests: List[Request], t0: Optional[float] = None):
        """Serve requests whose `arrival` is seconds after t0 (wall clock)."""
        t0 = time.perf_counter() if t0 is None else t0
        clock = lambda: time.perf_counter() - t0
        for r in requests:
            self.submit(r)
        total = len(requests)
        while len(self.finished) < total:
            busy = self.step(clock)
            if not busy and self.waiting:
                wait = self.waiting[0].arrival - clock()
                if wait > 0:
                    time.sleep(min(wait, 0.05))
        return clock()

    def close(self):
        if self.b:
            dem.dem_batch_destroy(self.b)
            self.b = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def poisson_requests(seed: int, count: int, rate: float, nmin: int, nmax: int, smin: int, smax: int,
                     precision: str = "fp32") -> List[Request]:
    """Seeded request stream: exponential inter-arrival times (mean 1/rate), sizes
    log-uniform in [nmin, nmax], step budgets uniform in [smin, smax], alternating box
    settling and drum scenes."""
    from . import scenes
    gaps = -np.log(1.0 - scenes.uniform(seed, count, 0.0, 1.0)) / rate
    arrivals = np.cumsum(gaps)
    sizes = scenes.loguniform_int(seed + 1, count, nmin, nmax)
    budgets = np.floor(scenes.uniform(seed + 2, count, smin, smax + 1)).astype(int)
    out = []
    for k in range(count):
        n = int(sizes[k])
        if k % 2 == 0:
            sc = scenes.box_lattice_n(seed=seed * 100 + k, n=n, precision=precision)
        else:
            sc = scenes.drum(seed=seed * 100 + k, n=n, precision=precision)
        out.append(Request(arrival=float(arrivals[k]), rid=k, scene=sc, steps=int(budgets[k])))
    return out


def latency_stats(finished: List[Request]):
    lat = np.array([r.done - r.arrival for r in finished])
    return {"p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
            "mean_s": float(lat.mean()), "max_s": float(lat.max())}
