#!/usr/bin/env python
"""Throughput benchmark of the DEM timestep on GB300 (one JSON line on stdout).

Workload (default `drum`): 4,194,304 spheres, radii U[0.9, 1.1] mm, dense bed in a drum
of radius 300 mean radii and length 208 mean radii rotating at 2 rad/s about its
horizontal axis, mu = 0.5, e = 0.7, practical model (Eqs. 2-10), linear stiffness
k_n = 1e4 N/m, k_t = (2/7) k_n, dt = contact time of the smallest pair / 50, FP32
forces with compensated positions. The sort policy and block size are chosen by the
autotuner: in practice the cell sort (Sec. 4.2 steps 2-4) runs only after some particle
has moved half a skin, with neighbour lists built at each sort (sorting every step, as
the paper does, is measured beside it). The bed is built by the seeded deposition
generator and settled on the GPU for `--settle` steps before the warm-up; the working
set (several GB) is far larger than L2, so no flush is needed.

One benchmark step is one timestep of the whole path: the force pass (steps 5-8 and 1)
and, on the steps that sort, the cell sort and new lists. Because a short timed window
may hold no sort, the line also reports an amortized rate over a longer window with the
measured number of steps per sort.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the CPU oracle (the FP64 C statement of the method, one core) on
a bounded sample of the same workload. With N > 1 every rank runs an independent replica
(replicas only: a single scene is not partitioned across GPUs); without torchrun,
--gpus N launches the N ranks itself. Rank 0 prints.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "particle-updates/s (practical model) & % HBM roofline vs simple model; served p50/p99"
UNIT = "particle-updates/s"
FALLBACK_HBM_GBS = 6800.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=50)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=["drum", "rsa", "box"], default="drum")
    ap.add_argument("--n", type=int, default=0, help="particle count (0 = the workload's own)")
    ap.add_argument("--settle", type=int, default=3000,
                    help="accelerated settling steps (input preparation, see settle_bed)")
    ap.add_argument("--relax", type=int, default=1000, help="steps at the real parameters after settling")
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--resort", type=str, default="tune",
                    help="cell-sort policy: 'tune' = autotuned (block size, every step or skin-driven with "
                         "neighbour lists); 1 = every step (Sec. 4.2); 0 = when a particle moved skin/2; K > 1 = "
                         "at least every K steps")
    ap.add_argument("--skin-r", type=float, default=0.1, help="skin in largest radii (used when --resort is 0 or K)")
    ap.add_argument("--max-contacts", type=int, default=24,
                    help="per-particle contact capacity (0 = library default of 32); the drum's largest count is "
                         "reported in the output, and a smaller capacity leaves the force kernel more L1")
    ap.add_argument("--block", type=int, default=0, help="force-kernel block size when not autotuned (0 = default)")
    ap.add_argument("--legacy-stream", action="store_true",
                    help="run the timed handle on the legacy default stream: every kernel is launched on its own "
                         "(no step graphs), for per-kernel launch lists")
    ap.add_argument("--simple-steps", type=int, default=500)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0, help="target CPU time of the oracle sample")
    ap.add_argument("--cpu-procs", type=int, default=0,
                    help="oracle processes of the all-cores baseline (0 = every host core, -1 = skip)")
    ap.add_argument("--amortize-steps", type=int, default=1000,
                    help="steps of the window that measures the steps per sort and the amortized rate (0 = skip)")
    ap.add_argument("--config2-steps", type=int, default=300,
                    help="timed steps of each mode on the 262,144-sphere polydisperse bed (0 = skip)")
    ap.add_argument("--config2-check-steps", type=int, default=50,
                    help="steps compared with the FP64 oracle on that bed")
    ap.add_argument("--batch-scenes", type=int, default=256, help="scenes of the batched run (0 = skip)")
    ap.add_argument("--batch-steps", type=int, default=300)
    ap.add_argument("--batch-seq-scenes", type=int, default=32, help="scenes timed one by one for comparison")
    ap.add_argument("--serve-requests", type=int, default=32, help="requests of each serving run (0 = skip)")
    ap.add_argument("--serve-rate", type=float, default=20.0, help="arrival rate of the saturated run [1/s]")
    ap.add_argument("--serve-nmax", type=int, default=1048576)
    ap.add_argument("--serve-steps", type=str, default="1000,20000", help="step budget range of the requests")
    ap.add_argument("--serve-hbm-gb", type=float, default=64.0)
    ap.add_argument("--serve-load", type=float, default=0.7,
                    help="offered load of the second run, as a fraction of the first run's measured rate (0 = skip)")
    ap.add_argument("--slabs", type=str, default="2,4",
                    help="slab counts of the decomposed runs (sub-domains with halo exchange, sort every step; "
                         "'' = skip)")
    ap.add_argument("--slab-steps", type=int, default=100, help="timed steps of each decomposed run")
    ap.add_argument("--hopper-steps", type=int, default=2000,
                    help="timed steps of the hopper comparison (the paper's own benchmark shape; 0 = skip)")
    ap.add_argument("--hopper-settle", type=int, default=3000, help="fill steps (closed bottom) before the slit opens")
    ap.add_argument("--hopper-drain", type=int, default=20000, help="steps after the slit opens, before timing")
    return ap.parse_args()


# ------------------------------------------------------------------ workload
def make_scene(args, rank=0):
    from paper_1301_1714_gb300 import scenes
    seed = args.seed + 1000 * rank
    if args.workload == "drum":
        return scenes.drum(seed=seed, n=args.n or 4_194_304, precision="fp32")
    if args.workload == "rsa":
        return scenes.box_rsa(seed=seed, n=args.n or 262_144, precision="fp32")
    return scenes.box_lattice(seed=seed, precision="fp64")


def workload_desc(args, sc, p=None, impl="ours"):
    p = p or sc.params
    if args.workload == "drum":
        base = (f"drum: {sc.n:,} spheres r~U[0.9,1.1] mm, drum R=300r L=208r rotating 2 rad/s, mu={p.mu}, e=0.7, "
                f"practical linear kn={p.kn:g} N/m, dt={p.dt:.5e} s")
        if impl == "reference":
            return base + ", FP64 oracle: every step's pairs from the cell grid"
        sort = ("sort every step" if p.resort_interval == 1 else
                f"sort when a particle moved skin/2 (skin {p.skin * 1e3:.2f} mm), neighbour lists")
        return base + f", FP32 forces + compensated positions, {sort}"
    if args.workload == "rsa":
        return f"box settling: {sc.n:,} spheres r~U[0.8,1.2] mm, RSA loose fill, practical linear, FP32"
    return f"box: {sc.n:,} spheres r=1 mm, jittered lattice, practical linear, FP64"


def settle_bed(dem, sc, dev_index, stream, steps, relax):
    """Input preparation: the generated bed rests each sphere on one support only, so it is
    settled before timing. `steps` steps run with dt x 8, g x 4 and e = 0.3 (fast, strongly
    damped compaction; dt x 8 is still below the stability limit of the stiffest contact),
    then the state is handed to the real parameters, which run `relax` further steps in
    the caller's handle. Returns the settled (x, v, w)."""
    from paper_1301_1714_gb300 import scenes
    if steps <= 0:
        return sc.x, sc.v, sc.w
    p = sc.params
    ps = p.copy(dt=8.0 * p.dt, g=tuple(4.0 * gk for gk in p.g), alpha=scenes.alpha_from_e(0.3), resort_interval=1,
                skin=0.0, cell_size=scenes.auto_cell_size(float(sc.r.max())))
    hs = dem.dem_create(dem.config_from_params(ps), dev_index, stream)
    try:
        dem.dem_set_walls(hs, ps.walls)
        dem.dem_set_particles(hs, sc.x, sc.v, sc.w, sc.r)
        dem.dem_step(hs, steps)
        return dem.dem_get_state(hs, sc.n)
    finally:
        dem.dem_destroy(hs)


def run_batch_bench(args, dem, dev_index, stream, block=0):
    """256 independent box-settling scenes (log-uniform 1,024-65,536 spheres, mu ~
    U[0.1, 0.6], e ~ U[0.5, 0.95]) advanced together in one batch, with the block size and
    sort policy the autotuner picks for the batch, against the first scenes advanced one by
    one through their own handles with the same policy."""
    import torch
    from paper_1301_1714_gb300 import autotune, scenes
    mix = scenes.batch_mix(seed=args.seed, count=args.batch_scenes, precision="fp32")
    total = sum(sc.n for sc in mix)
    best, table = autotune.tune_batch(mix, device=dev_index, cuda_stream=stream.cuda_stream,
                                      max_contacts=args.max_contacts)
    params = [autotune.apply(sc.params, float(sc.r.max()), best) for sc in mix]
    b = dem.dem_batch_create(precision="fp32", max_contacts=args.max_contacts, block_size=best.block,
                             device=dev_index, cuda_stream=stream.cuda_stream)
    try:
        for sc, p in zip(mix, params):
            dem.dem_batch_add(b, p, sc.x, sc.v, sc.w, sc.r, args.batch_steps + 3)
        dem.dem_batch_run(b, 3)                      # pack, first sort, graph capture
        torch.cuda.synchronize()
        l0 = dem.dem_batch_launch_count(b)
        t0 = time.perf_counter()
        dem.dem_batch_run(b, args.batch_steps)
        tb = time.perf_counter() - t0
        launches = dem.dem_batch_launch_count(b) - l0
    finally:
        dem.dem_batch_destroy(b)
    seq_n, seq_t = 0, 0.0
    for sc, p in list(zip(mix, params))[:args.batch_seq_scenes]:
        h = dem.dem_create(dem.config_from_params(p, block_size=best.block, max_contacts=args.max_contacts),
                           dev_index, stream.cuda_stream)
        try:
            dem.dem_set_walls(h, p.walls)
            dem.dem_set_particles(h, sc.x, sc.v, sc.w, sc.r)
            dem.dem_step(h, 3)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            dem.dem_step(h, args.batch_steps)
            seq_t += time.perf_counter() - t0
            seq_n += sc.n
        finally:
            dem.dem_destroy(h)
    batched = total * args.batch_steps / tb
    seq = seq_n * args.batch_steps / seq_t if seq_t > 0 else None
    return {"scenes": len(mix), "particles": total, "steps": args.batch_steps, "value": round(batched, 1),
            "unit": UNIT, "ms_per_step": round(tb * 1e3 / args.batch_steps, 4), "gpu_launches": int(launches),
            "autotune": {"choice": {"block": best.block, "resort_interval": best.resort,
                                    "skin_frac_rmax": best.skin_frac},
                         "table": [[c.block, c.resort, c.skin_frac, round(c.ms_per_step, 4)] for c in table]},
            "sequential_value": round(seq, 1) if seq else None,
            "sequential_sample": f"first {min(args.batch_seq_scenes, len(mix))} scenes, one handle each with the "
                                 f"batch's policy, {args.batch_steps} steps",
            "batched_over_sequential": round(batched / seq, 2) if seq else None}


def run_config2(args, dem, dev_index, stream):
    """The 262,144-sphere polydisperse bed (r ~ U[0.8, 1.2] mm, random loose fill in a box
    of 160 x 160 x 400 mean radii) settling under gravity: throughput of the practical
    model with FP32 forces (compensated positions) and in FP64, and of the simple model
    (Eq. 1), each sorting only after a particle moved half a skin of 0.1 r_max; and each
    mode's distance from the FP64 oracle after `config2_check_steps` steps from the same
    start (the oracle runs the whole bed, one core)."""
    import torch
    import oracle
    from paper_1301_1714_gb300 import scenes
    sc = scenes.box_rsa(seed=args.seed, n=262_144, precision="fp32")
    skin = 0.1 * float(sc.r.max())
    listed = lambda q: q.copy(resort_interval=0, skin=skin, cell_size=q.cell_size + skin)
    modes = {"fp32_practical": listed(sc.params), "fp64_practical": listed(sc.params.copy(precision="fp64")),
             "fp32_simple": listed(sc.params.copy(model="simple")), "fp64_simple": listed(
                 sc.params.copy(model="simple", precision="fp64"))}
    ksteps = args.config2_check_steps
    t0 = time.perf_counter()
    refs = {m: oracle.State(sc.params.copy(precision="fp64", model=m), sc.x, sc.v, sc.w, sc.r).run(ksteps)
            for m in ("practical", "simple")}
    t_oracle = time.perf_counter() - t0
    out = {"workload": f"box settling: {sc.n:,} spheres r~U[0.8,1.2] mm, RSA loose fill (phi 0.35) in 160x160x400 "
                       f"mean radii, practical and simple models, skin {skin * 1e3:.3f} mm",
           "n_particles": sc.n, "steps": args.config2_steps, "oracle_check_steps": ksteps,
           "oracle_check_s": round(t_oracle, 1), "modes": {}}
    for name, p in modes.items():
        model = p.model
        ref = refs[model]
        with dem.Simulation(p, sc.x, sc.v, sc.w, sc.r, device=dev_index, cuda_stream=stream.cuda_stream,
                            max_contacts=args.max_contacts) as s:
            s.step(ksteps)
            x, _, _ = s.state()
            err = float(np.max(np.abs(x - ref.x)))
            disp = float(np.max(np.linalg.norm(ref.x - sc.x, axis=1)))
            s.step(20)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            s.step(args.config2_steps)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / args.config2_steps
        out["modes"][name] = {"value": round(sc.n / (ms / 1e3), 1), "ms_per_step": round(ms, 4),
                              "max_abs_dx_vs_oracle_m": err, "oracle_max_displacement_m": disp}
    m = out["modes"]
    out["fp64_over_fp32_slowdown"] = round(m["fp64_practical"]["ms_per_step"] / m["fp32_practical"]["ms_per_step"], 3)
    out["practical_over_simple_slowdown_fp32"] = round(
        m["fp32_practical"]["ms_per_step"] / m["fp32_simple"]["ms_per_step"], 3)
    return out


def run_hopper_bench(args, dem, dev_index, stream, block=0):
    """The paper's benchmark shape (Sec. 5, Table 3): 131,072 equal spheres in a box drain
    through a slit in its bottom onto a floor. The box is filled at rest with the bottom
    closed (accelerated settling), the slit opens, the flow runs `hopper_drain` steps, then
    the practical and the simple model are each timed for `hopper_steps` steps from that
    state (FP32, skin-driven sorting, the drum's tuned block size), and the FP64 oracle on
    a bounded slab of it."""
    import torch
    from paper_1301_1714_gb300 import scenes
    closed = scenes.hopper(seed=args.seed, open_slit=False)
    opened = scenes.hopper(seed=args.seed, open_slit=True)
    N = closed.n
    x, v, w = settle_bed(dem, closed, dev_index, stream.cuda_stream, args.hopper_settle, 0)
    rmax = float(closed.r.max())
    skin = args.skin_r * rmax
    out = {"workload": f"hopper: {N:,} equal spheres r=1 mm, box 134.4 x 67.2 mm filled at rest, slit 12 mm wide "
                       f"across x opened, {args.hopper_drain} steps of flow, then timed",
           "n_particles": N, "steps": args.hopper_steps}
    for model in ("practical", "simple"):
        p = opened.params.copy(model=model, resort_interval=0, skin=skin, cell_size=opened.params.cell_size + skin)
        h = dem.dem_create(dem.config_from_params(p, block_size=block), dev_index, stream.cuda_stream)
        try:
            dem.dem_set_walls(h, p.walls)
            dem.dem_set_particles(h, x, v, w, closed.r)
            if model == "practical":
                dem.dem_step(h, args.hopper_drain)
                xd, vd, wd = dem.dem_get_state(h, N)
                zp = opened.params.walls[6]["p"][2]
                out["below_plate_at_start"] = int(np.count_nonzero(xd[:, 2] < zp))
            else:
                dem.dem_set_particles(h, xd, vd, wd, closed.r)
            dem.dem_step(h, 50)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            dem.dem_step(h, args.hopper_steps)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            d = dict(zip(dem.DIAG_NAMES, dem.dem_get_diagnostics(h)))
            out[model] = {"value": round(N * args.hopper_steps / (ms / 1e3), 1), "unit": UNIT,
                          "ms_per_step": round(ms / args.hopper_steps, 4),
                          "pair_contacts": d["pair_contacts"], "wall_contacts": d["wall_contacts"]}
        finally:
            dem.dem_destroy(h)
    out["practical_over_simple_slowdown"] = round(out["simple"]["value"] / out["practical"]["value"], 3)
    if not args.no_cpu_baseline:
        state = scenes.Scene("hopper_flow", xd, vd, wd, closed.r, opened.params)
        val, desc, _, _ = oracle_sample(args, state, 0.5 * args.cpu_seconds, state="the draining hopper")
        out["cpu_oracle"] = {"value": round(val, 1), "unit": UNIT, "cores": 1, "sample": desc}
        out["gpu_practical_over_cpu"] = round(out["practical"]["value"] / val, 1)
    out["paper_table3_context"] = {"unit": "particles/s", "practical_gpu_opencl_c2050": 2.96e6,
                                   "simple_gpu_cuda_c2050": 2.2359e7, "practical_cpu_x5670_1core": 4.74e5,
                                   "note": "another machine and an unstated geometry: context, not a target"}
    return out


def run_slab_bench(args, dem, dev_index, stream, sc, xs, vs, ws, every):
    """The settled bed divided into slabs along its longest axis (sub-domains with a ghost
    layer, exchange after every force pass, sort every step), against one undivided
    handle in the same mode (`every`). The exchange reads its counts back every step."""
    import torch
    counts = [int(k) for k in args.slabs.split(",") if k.strip()]
    if not counts or args.slab_steps <= 0:
        return None
    N = len(sc.r)
    p = sc.params.copy(resort_interval=1, skin=0.0)
    rows = {}
    for S in counts:
        sl = dem.dem_slabs_create(dem.config_from_params(p, block_size=256, max_contacts=args.max_contacts), S, -1,
                                  dev_index, stream.cuda_stream)
        try:
            dem.dem_slabs_set_walls(sl, p.walls)
            dem.dem_slabs_set_particles(sl, xs, vs, ws, sc.r)
            dem.dem_slabs_step(sl, 3)
            torch.cuda.synchronize(dev_index)
            L0 = dem.dem_slabs_launch_count(sl)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            t0 = time.perf_counter()
            nvtx_push(f"slabs{S}")
            e0.record(stream)
            dem.dem_slabs_step(sl, args.slab_steps)
            e1.record(stream)
            torch.cuda.synchronize(dev_index)
            nvtx_pop()
            wall = time.perf_counter() - t0
            ms = e0.elapsed_time(e1) / args.slab_steps
            info = dem.dem_slabs_info(sl, S)
            rows[str(S)] = {"value": round(N / (ms / 1e3), 1), "ms_per_step": round(ms, 4),
                            "host_ms_per_step": round(wall * 1e3 / args.slab_steps, 4),
                            "ghost_fraction": round(float(info["ghosts"].sum()) / N, 4),
                            "owned_min_max": [int(info["owned"].min()), int(info["owned"].max())],
                            "migrated_per_step": round(info["migrated"] / max(info["steps"], 1), 1),
                            "launches_per_step": round((dem.dem_slabs_launch_count(sl) - L0) / args.slab_steps, 1),
                            "over_undivided": (round((N / (ms / 1e3)) / every["value"], 3) if every else None)}
        finally:
            dem.dem_slabs_destroy(sl)
    return {"unit": UNIT, "steps": args.slab_steps, "block": 256, "rows": rows,
            "note": "one scene as S sub-domains on one GPU: force pass per slab (ghosts included), one exchange "
                    "launch (migration with springs, fresh ghost copies), a host read of the slab counts, a cell "
                    "sort per slab; owned particles are bit-exact against the undivided run"}


def run_serve_bench(args, dem, dev_index, stream):
    """Continuous batching of a Poisson request stream: sizes log-uniform in [1,024,
    serve_nmax], step budgets uniform in serve_steps, box settling and drum scenes
    alternating, every request run in list mode (skin 0.1 r_max) and admitted by its
    device-memory footprint. A fixed count of requests arrives at serve_rate (more work
    than the GPU can do, so the queue grows); then the same count again at serve_load
    times the rate the first run achieved (steady state). Latency = completion - arrival."""
    from paper_1301_1714_gb300 import serve
    smin, smax = (int(t) for t in args.serve_steps.split(","))

    def one_run(rate, seed):
        reqs = serve.poisson_requests(seed, args.serve_requests, rate, 1024, args.serve_nmax, smin, smax)
        work = sum(r.scene.n * r.steps for r in reqs)
        offered = work / max(reqs[-1].arrival, 1e-9)
        with serve.Server(int(args.serve_hbm_gb * 2 ** 30), cuda_stream=stream.cuda_stream, device=dev_index,
                          max_contacts=args.max_contacts, skin_frac=0.1) as srv:
            wall = srv.run(reqs)
            stats = serve.latency_stats(srv.finished)
            done = srv.particle_steps
        return {"requests": len(reqs), "rate_per_s": round(rate, 3), "p50_s": round(stats["p50_s"], 3),
                "p99_s": round(stats["p99_s"], 3), "mean_s": round(stats["mean_s"], 3),
                "value": round(done / wall, 1), "unit": UNIT, "offered": round(offered, 1),
                "achieved_over_offered": round(done / wall / offered, 3), "wall_s": round(wall, 2),
                "particle_steps": int(done)}

    sat = one_run(args.serve_rate, args.seed)
    out = {"n_range": [1024, args.serve_nmax], "step_range": [smin, smax], "hbm_budget_gb": args.serve_hbm_gb,
           "sort_policy": "list mode, skin 0.1 r_max per scene", "saturated": sat}
    if args.serve_load > 0:
        mean_work = sat["particle_steps"] / sat["requests"]
        rate = args.serve_load * sat["value"] / mean_work
        out["steady"] = dict(one_run(rate, args.seed + 7), load_fraction_of_measured=args.serve_load)
    # headline fields of the saturated run
    out.update({k: sat[k] for k in ("p50_s", "p99_s", "value", "unit", "achieved_over_offered")})
    return out


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.proc = None
        self.dev = device_index

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.dev)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [t.strip() for t in line.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                mx = float(f[1])
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if f[4 + k].lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def nvtx_push(name):
    try:
        import torch
        torch.cuda.nvtx.range_push(name)
    except Exception:
        pass


def nvtx_pop():
    try:
        import torch
        torch.cuda.nvtx.range_pop()
    except Exception:
        pass


def physical_gpu_index(local_rank):
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    if vis:
        ids = [v.strip() for v in vis.split(",") if v.strip()]
        if local_rank < len(ids):
            return ids[local_rank]
    return local_rank


# ------------------------------------------------------------------ roofline inputs
def measured_hbm_gbs():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return FALLBACK_HBM_GBS, "fallback"


def kernel_source_hash(list_mode=False):
    """Hash of the sources of the force kernel (list mode or walk), which the committed
    ncu summaries record."""
    h = hashlib.sha256()
    for fn in ("dem_list.cu" if list_mode else "dem_kernels.cu", "dem_policy.cuh", "dem_dev.cuh"):
        with open(os.path.join(ROOT, "paper_1301_1714_gb300", "csrc", fn), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def profiled_traffic_per_particle(list_mode=False):
    """DRAM bytes per particle of the force kernel from the committed ncu summary, if it
    was taken on the current kernel source (else None)."""
    path = os.path.join(ROOT, "profiles", "force_kernel_list_drum.md" if list_mode else "force_kernel_drum.md")
    try:
        txt = open(path).read()
    except OSError:
        return None
    src, bpp = None, None
    for line in txt.splitlines():
        if line.startswith("kernel_source_sha256_16:"):
            src = line.split(":", 1)[1].strip()
        if line.startswith("dram_bytes_per_particle:"):
            try:
                bpp = float(line.split(":", 1)[1].strip())
            except ValueError:
                bpp = None
    return bpp if (src == kernel_source_hash(list_mode) and bpp) else None


# ------------------------------------------------------------------ oracle sample
def oracle_sample(args, sc, target_s, max_steps=None, state="the same seeded workload before settling"):
    """Time the FP64 oracle on a slab of the workload (particles with x below a cut),
    sized so that the steps take about target_s seconds. Returns (value, sample text,
    steps, seconds)."""
    import oracle
    order = np.argsort(sc.x[:, 0], kind="stable")
    # calibrate on a small slab
    n_cal = min(sc.n, 20000)
    sel = np.sort(order[:n_cal])
    t0 = time.perf_counter()
    oracle.State(sc.params.copy(precision="fp64"), sc.x[sel], sc.v[sel], sc.w[sel], sc.r[sel]).run(1)
    per = (time.perf_counter() - t0) / n_cal
    steps = max(1, min(max_steps or 3, 3))
    n_s = int(min(sc.n, max(1000, target_s / (per * steps))))
    sel = np.sort(order[:n_s])
    st = oracle.State(sc.params.copy(precision="fp64"), sc.x[sel], sc.v[sel], sc.w[sel], sc.r[sel])
    t0 = time.perf_counter()
    st.run(steps)
    dt = time.perf_counter() - t0
    value = n_s * steps / dt
    xcut = float(sc.x[sel, 0].max())
    desc = (f"FP64 oracle (C, 1 thread), {steps} step(s) of the {n_s:,} spheres with x <= {xcut:.4f} m of "
            f"{state} (grid pair search), {dt:.1f} s")
    return value, desc, steps, dt


def _oracle_slab_worker(payload):
    """One process of the all-cores baseline: the oracle on its own slab, timed alone."""
    import oracle
    params, x, v, w, r, steps = payload
    st = oracle.State(params, x, v, w, r)
    t0 = time.perf_counter()
    st.run(steps)
    return len(r), steps, time.perf_counter() - t0


def cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo, else the machine type)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.machine()


def oracle_all_cores(args, sc, target_s, procs, state):
    """The FP64 oracle as it stands, one process per host core, each on its own slab of the
    workload (disjoint ranges of x; the oracle's arithmetic is untouched), all started
    together; throughput = every process's particle-steps over the slowest one's time.
    The pool uses the spawn start method, so no process inherits the parent's CUDA state."""
    import multiprocessing as mp
    import oracle
    order = np.argsort(sc.x[:, 0], kind="stable")
    n_cal = min(sc.n, 20000)
    sel = np.sort(order[:n_cal])
    p64 = sc.params.copy(precision="fp64")
    t0 = time.perf_counter()
    oracle.State(p64, sc.x[sel], sc.v[sel], sc.w[sel], sc.r[sel]).run(1)
    per = (time.perf_counter() - t0) / n_cal
    steps = 3
    n_w = int(min(sc.n // procs, max(1000, target_s / (per * steps))))
    payloads = []
    for k in range(procs):
        ids = np.sort(order[k * n_w:(k + 1) * n_w])
        payloads.append((p64, sc.x[ids], sc.v[ids], sc.w[ids], sc.r[ids], steps))
    with mp.get_context("spawn").Pool(procs) as pool:
        res = pool.map(_oracle_slab_worker, payloads)
    dt = max(r_[2] for r_ in res)
    value = sum(r_[0] * r_[1] for r_ in res) / dt
    desc = (f"FP64 oracle (C), {procs} processes at once, each {steps} step(s) of its own slab of {n_w:,} spheres "
            f"(consecutive ranges of x) of {state}; slowest process {dt:.1f} s")
    return value, desc


# ------------------------------------------------------------------ our arm
def run_ours(args):
    import torch
    from paper_1301_1714_gb300 import dem, replicas

    world, rank, local_rank = replicas.rank_env()
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local_rank if world > 1 else 0)
    torch.cuda.set_device(dev)
    stream = torch.cuda.Stream(device=dev)

    sc = make_scene(args, rank)
    N = sc.n
    t_prep = time.perf_counter()
    xs0, vs0, ws0 = settle_bed(dem, sc, dev.index, stream.cuda_stream, args.settle, args.relax)
    if args.relax:
        # relax at the real parameters (sort every step), then start every run from there
        hr = dem.dem_create(dem.config_from_params(sc.params), dev.index, stream.cuda_stream)
        try:
            dem.dem_set_walls(hr, sc.params.walls)
            dem.dem_set_particles(hr, xs0, vs0, ws0, sc.r)
            dem.dem_step(hr, args.relax)
            xs0, vs0, ws0 = dem.dem_get_state(hr, N)
        finally:
            dem.dem_destroy(hr)
    rmax = float(sc.r.max())
    tuned = None
    if args.resort == "tune":
        from paper_1301_1714_gb300 import autotune
        best, table = autotune.tune(sc.params, xs0, vs0, ws0, sc.r, device=dev.index, cuda_stream=stream.cuda_stream,
                                    max_contacts=args.max_contacts)
        p = autotune.apply(sc.params, rmax, best)
        block = best.block
        tuned = {"choice": {"block": best.block, "resort_interval": best.resort, "skin_frac_rmax": best.skin_frac},
                 "table": [[c.block, c.resort, c.skin_frac, round(c.ms_per_step, 4)] for c in table]}
    else:
        k = int(args.resort)
        block = args.block
        p = sc.params if k == 1 else sc.params.copy(resort_interval=k, skin=args.skin_r * rmax,
                                                    cell_size=sc.params.cell_size + args.skin_r * rmax)
    cfg = dem.config_from_params(p, block_size=block, max_contacts=args.max_contacts)
    h = dem.dem_create(cfg, dev.index, None if args.legacy_stream else stream.cuda_stream)
    tstream = torch.cuda.default_stream(dev) if args.legacy_stream else stream   # the timed handle's stream
    try:
        dem.dem_set_walls(h, p.walls)
        dem.dem_set_particles(h, xs0, vs0, ws0, sc.r)
        t_prep = time.perf_counter() - t_prep
        dem.dem_step(h, max(3, args.warmup))
        # ---------------- amortization window: the steps per sort and the rate with the
        # sorts at their natural frequency (the timed window below may be too short to
        # hold one)
        amort = None
        if args.amortize_steps > 0:
            torch.cuda.synchronize(dev)
            dem.dem_set_timing(h, True)
            a_sorts0 = dem.dem_get_diagnostics(h)[14]
            dem.dem_step(h, args.amortize_steps)
            aph = dem.dem_get_phase_times(h)
            a_sorts = dem.dem_get_diagnostics(h)[14] - a_sorts0
            dem.dem_set_timing(h, False)
            a_ms = (aph[0] + aph[1]) / max(aph[2], 1)
            amort = {"steps": args.amortize_steps, "sorts": int(a_sorts),
                     "steps_per_sort": (round(args.amortize_steps / a_sorts, 1) if a_sorts else None),
                     "ms_per_step": round(a_ms, 4), "force_ms": round(aph[0] / max(aph[2], 1), 4),
                     "sort_tail_ms_per_step": round(aph[1] / max(aph[3], 1), 4)}
        # ---------------- timed region (device events on the library's stream)
        if dist:
            dist.barrier()
        torch.cuda.synchronize(dev)
        dem.dem_set_timing(h, True)
        sorts0 = dem.dem_get_diagnostics(h)[14]
        l0 = dem.dem_launch_count(h)
        clk = ClockSampler(physical_gpu_index(local_rank))
        clk.start()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        nvtx_push("timed")                            # lets a profiler select the timed steps
        e0.record(tstream)
        dem.dem_step(h, args.steps)
        e1.record(tstream)
        torch.cuda.synchronize(dev)
        nvtx_pop()
        clocks = clk.stop()
        if dist:
            dist.barrier()
        launches = dem.dem_launch_count(h) - l0
        ms = e0.elapsed_time(e1)
        sorts_timed = dem.dem_get_diagnostics(h)[14] - sorts0
        phase = dem.dem_get_phase_times(h)
        max_seen = dem.dem_max_contacts_seen(h)
        dem.dem_set_timing(h, False)
        diag = dict(zip(dem.DIAG_NAMES, dem.dem_get_diagnostics(h)))
        # the same number of steps again, replayed as the library's step graph (no events
        # between phases; in list mode the sort is a conditional node)
        torch.cuda.synchronize(dev)
        lg0 = dem.dem_launch_count(h)
        g0 = torch.cuda.Event(enable_timing=True)
        g1 = torch.cuda.Event(enable_timing=True)
        g0.record(tstream)
        dem.dem_step(h, args.steps)
        g1.record(tstream)
        torch.cuda.synchronize(dev)
        ms_graph = replicas.reduce_max(g0.elapsed_time(g1), dev)
        graph = {"value": round(replicas.reduce_sum(float(N), dev) * args.steps / (ms_graph / 1e3), 1),
                 "ms_per_step": round(ms_graph / args.steps, 4),
                 "gpu_launches": int(dem.dem_launch_count(h) - lg0)}
        ms = replicas.reduce_max(ms, dev)            # the slowest replica sets the time
        n_total = replicas.reduce_sum(float(N), dev)  # particles advanced by all replicas
        value = n_total * args.steps / (ms / 1e3)

        # ---------------- roofline of the dominant kernel (force pass)
        Z = 2.0 * diag["pair_contacts"] / N
        W = diag["wall_contacts"] / N
        b_force = 104.0 + 20.0 * Z + 40.0 * W
        # the step: the force pass plus the sort's share, (16 c + 16 P + 104) / K bytes per
        # particle (c cells per particle, P = 3 key passes, K steps per sort)
        _, _, gdims = dem.dem_get_grid(h)
        c_cells = float(np.prod(gdims)) / N
        if amort is not None:
            K = (amort["steps"] / amort["sorts"]) if amort["sorts"] else float(amort["steps"])
            b_step = b_force + (16.0 * c_cells + 16.0 * 3 + 104.0) / K
            amort["value"] = round(replicas.reduce_sum(float(N), dev) / (amort["ms_per_step"] / 1e3), 1)
            amort["algorithmic_bytes_per_particle"] = round(b_step, 1)
            amort["cells_per_particle"] = round(c_cells, 3)
            amort["achieved_gbs"] = round(b_step * N / (amort["ms_per_step"] / 1e3) / 1e9, 1)
        force_ms = phase[0] / max(phase[2], 1)
        sort_ms = phase[1] / max(phase[3], 1)
        peak, peak_src = measured_hbm_gbs()
        if amort is not None:
            amort["frac"] = round(amort["achieved_gbs"] / peak, 4)
        achieved = b_force * N / (force_ms / 1e3) / 1e9
        bpp = profiled_traffic_per_particle(p.resort_interval != 1)
        roof = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "traffic": (round(bpp * N) if bpp else None),
                "kernel": "k_list<PF32,practical>" if p.resort_interval != 1 else "k_force<PF32,practical>", "peak_source": f"{peak_src} (MEASURED_PEAKS.json hbm_gbs)",
                "algorithmic_bytes_per_particle": round(b_force, 1), "Z": round(Z, 3), "W": round(W, 4),
                "force_ms": round(force_ms, 4), "sort_ms": round(sort_ms, 4)}

        # ---------------- the paper's policy (sort and walk every step) on the same bed
        xs, vs, ws = dem.dem_get_state(h, N)
        every = None
        if p.resort_interval != 1:
            wblock = block
            if tuned:   # the walk's own best block size among the tuned candidates
                walk = [row for row in tuned["table"] if row[1] == 1]
                if walk:
                    wblock = min(walk, key=lambda row: row[3])[0]
            hk = dem.dem_create(dem.config_from_params(sc.params, block_size=wblock, max_contacts=args.max_contacts),
                                dev.index, stream.cuda_stream)
            try:
                dem.dem_set_walls(hk, sc.params.walls)
                dem.dem_set_particles(hk, xs, vs, ws, sc.r)
                dem.dem_step(hk, 3)
                dem.dem_set_timing(hk, True)
                k0 = torch.cuda.Event(enable_timing=True)
                k1 = torch.cuda.Event(enable_timing=True)
                k0.record(stream)
                dem.dem_step(hk, args.simple_steps or 200)
                k1.record(stream)
                torch.cuda.synchronize(dev)
                kms = k0.elapsed_time(k1) / (args.simple_steps or 200)
                kph = dem.dem_get_phase_times(hk)
                every = {"value": round(N / (kms / 1e3), 1), "ms_per_step": round(kms, 4),
                         "force_ms": round(kph[0] / max(kph[2], 1), 4), "sort_ms": round(kph[1] / max(kph[3], 1), 4)}
            finally:
                dem.dem_destroy(hk)

        # ---------------- the same bed as slabs (sub-domains with halo exchange), sort every step
        slabs = run_slab_bench(args, dem, dev.index, stream, sc, xs, vs, ws, every) if rank == 0 else None

        # ---------------- practical / simple on the same settled bed
        simple = None
        if args.simple_steps > 0:
            hs = dem.dem_create(dem.config_from_params(p.copy(model="simple"), block_size=block,
                                                       max_contacts=args.max_contacts), dev.index, stream.cuda_stream)
            try:
                dem.dem_set_walls(hs, p.walls)
                dem.dem_set_particles(hs, xs, vs, ws, sc.r)
                dem.dem_step(hs, 3)
                torch.cuda.synchronize(dev)
                dem.dem_set_timing(hs, True)
                s0 = torch.cuda.Event(enable_timing=True)
                s1 = torch.cuda.Event(enable_timing=True)
                s0.record(stream)
                dem.dem_step(hs, args.simple_steps)
                s1.record(stream)
                torch.cuda.synchronize(dev)
                sms = s0.elapsed_time(s1)
                sph = dem.dem_get_phase_times(hs)
                simple = {"value": round(N * args.simple_steps / (sms / 1e3), 1),
                          "ms_per_step": round(sms / args.simple_steps, 4),
                          "force_ms": round(sph[0] / max(sph[2], 1), 4),
                          "practical_over_simple_slowdown": round((ms / args.steps) / (sms / args.simple_steps), 3)}
            finally:
                dem.dem_destroy(hs)

        # ---------------- end to end through the C ABI with host buffers
        e2e = None
        if not args.no_e2e:
            pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()
            hx, hv, hw, hr = pin(xs), pin(vs), pin(ws), pin(sc.r)
            ox = torch.empty((N, 3), dtype=torch.float64).pin_memory().numpy()
            ov = torch.empty((N, 3), dtype=torch.float64).pin_memory().numpy()
            ow = torch.empty((N, 3), dtype=torch.float64).pin_memory().numpy()
            he = dem.dem_create(cfg, dev.index, stream.cuda_stream)
            try:
                dem.dem_set_walls(he, p.walls)
                dem.dem_set_particles(he, hx, hv, hw, hr)      # allocate once outside the timed region
                torch.cuda.synchronize(dev)
                if dist:
                    dist.barrier()
                t0 = time.perf_counter()
                dem.dem_set_particles(he, hx, hv, hw, hr)
                dem.dem_step(he, args.steps)
                r_ = dem.lib().dem_get_state(he, dem._ptr(ox), dem._ptr(ov), dem._ptr(ow), dem.DEM_HOST)
                if r_ != 0:
                    raise dem.DemError(r_, dem.dem_last_error(he))
                te = replicas.reduce_max(time.perf_counter() - t0, dev)
            finally:
                dem.dem_destroy(he)
            h2d = N * (3 * 24 + 4)
            d2h = N * 3 * 24
            e2e = {"value": round(n_total * args.steps / te, 1), "unit": UNIT,
                   "h2d_bytes_per_step": round(h2d / args.steps, 1), "d2h_bytes_per_step": round(d2h / args.steps, 1),
                   "note": "one upload of the state, K steps, one download of the state (pinned host buffers), "
                           "through dem_set_particles / dem_step / dem_get_state"}

        batch = run_batch_bench(args, dem, dev.index, stream, block) if args.batch_scenes > 0 else None
        serving = run_serve_bench(args, dem, dev.index, stream) if args.serve_requests > 0 else None
        hopper = (run_hopper_bench(args, dem, dev.index, stream, block)
                  if args.hopper_steps > 0 and rank == 0 and world == 1 else None)
        config2 = (run_config2(args, dem, dev.index, stream)
                   if args.config2_steps > 0 and rank == 0 and world == 1 else None)
        out = {"metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": world, "steps": args.steps,
               "warmup": max(3, args.warmup), "ms_per_step": round(ms / args.steps, 4), "higher_is_better": True,
               "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
               "config": {"workload": workload_desc(args, sc, p), "n_particles": N, "seed": args.seed,
                          "settle_steps": args.settle, "relax_steps": args.relax, "prep_s": round(t_prep, 1),
                          "resort_interval": p.resort_interval, "skin_m": p.skin,
                          "sorts_in_timed_steps": int(sorts_timed),
                          "l2": "inputs larger than L2 (no flush needed)",
                          "device_bytes": dem.dem_device_bytes(h), "parallelism": f"replicas x{world}"},
               "roofline": roof, "amortized": amort, "gpu_launches": int(launches), "clocks": clocks,
               "graph_replay": graph,
               "simple": simple, "e2e": e2e,
               "batch": batch, "serving": serving, "hopper": hopper, "config2": config2, "autotune": tuned,
               "sort_every_step": every,
               "slabs": slabs,
               "diagnostics": dict({k: diag[k] for k in ("pair_contacts", "wall_contacts", "max_overlap", "ke_trans")},
                                   max_contacts_seen=max_seen, max_contacts=cfg.max_contacts or 32)}
    finally:
        dem.dem_destroy(h)

    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        state = "the same seeded workload before settling"
        v1, desc1, steps, dt = oracle_sample(args, sc, args.cpu_seconds, state=state)
        single = {"value": round(v1, 1), "unit": UNIT, "cores": 1, "kind": "oracle", "sample": desc1}
        nproc = os.cpu_count() or 1
        procs = nproc if args.cpu_procs == 0 else args.cpu_procs
        if procs > 1:
            va, desca = oracle_all_cores(args, sc, args.cpu_seconds, procs, state)
            out["cpu_baseline"] = {"value": round(va, 1), "unit": UNIT, "cores": procs, "kind": "oracle",
                                   "sample": desca, "nproc": nproc, "cpu_model": cpu_model(), "single_core": single}
        else:
            out["cpu_baseline"] = dict(single, nproc=nproc, cpu_model=cpu_model())
    elif rank == 0:
        out["cpu_baseline"] = None
    if dist:
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(out), flush=True)


# ------------------------------------------------------------------ reference arm
def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    sc = make_scene(args, 0)
    steps = args.steps + max(3, args.warmup)
    # the whole run (warm-up + timed steps) should take a few minutes: size the sample
    import oracle
    order = np.argsort(sc.x[:, 0], kind="stable")
    n_cal = min(sc.n, 20000)
    sel = np.sort(order[:n_cal])
    t0 = time.perf_counter()
    oracle.State(sc.params.copy(precision="fp64"), sc.x[sel], sc.v[sel], sc.w[sel], sc.r[sel]).run(1)
    per = (time.perf_counter() - t0) / n_cal
    budget = 150.0
    n_s = int(min(sc.n, max(500, budget / (per * steps))))
    sel = np.sort(order[:n_s])
    st = oracle.State(sc.params.copy(precision="fp64"), sc.x[sel], sc.v[sel], sc.w[sel], sc.r[sel])
    st.run(max(3, args.warmup))
    t0 = time.perf_counter()
    st.run(args.steps)
    dt = time.perf_counter() - t0
    value = n_s * args.steps / dt
    desc = (f"FP64 oracle (C, 1 thread) on the {n_s:,} spheres with x <= {float(sc.x[sel, 0].max()):.4f} m of the "
            f"same seeded workload, {args.steps} timed steps after {max(3, args.warmup)} warm-up steps")
    out = {"impl": "reference", "metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": max(3, args.warmup), "ms_per_step": round(dt * 1e3 / args.steps, 3),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": workload_desc(args, sc, impl="reference"), "n_particles": sc.n, "seed": args.seed},
           "cpu_baseline": {"value": round(value, 1), "unit": UNIT, "cores": 1, "kind": "oracle", "sample": desc},
           "e2e": {"value": round(value, 1), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    args = parse()
    from paper_1301_1714_gb300 import replicas
    if args.gpus > 1 and "WORLD_SIZE" not in os.environ:
        # one rank per GPU, launched here when the caller did not use torchrun
        sys.exit(replicas.launch_ranks(args.gpus, [os.path.abspath(__file__), *sys.argv[1:]]))
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
