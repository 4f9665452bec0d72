#!/usr/bin/env python3
"""Benchmark of the Lagrangian-Eulerian coupling step on the many-bubble workload.

One step = one pass of the hot path over the whole point set:
  * locate + interpolate every IBM marker (Peskin-4) and every point particle (trilinear) in
    one persistent launch replayed from a CUDA graph (learned index by default);
  * spread the marker forces back to the cells (deterministic sorted reduction).
value = (markers + particles) / step time, summed over ranks (each rank runs its own
independent copy of the workload: weak scaling, no data-path collective).

Prints ONE JSON line (rank 0).  ``--impl reference`` times the FP64 CPU oracle on the same
workload instead (bounded samples, host cores).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

INDEX_DESC = {"mlp3": "learned: MLP root 1-32-1 -> 4096 linear mid models -> 262144 linear leaf models",
              "mlp2": "learned: MLP root 1-32-1 -> 4096 linear leaf models",
              "linear2": "learned: linear root -> 4096 linear leaf models"}
METRIC = "Lagrangian points located+interpolated/s on 1 GB300 (learned vs plain) at <=1e-5 rel err"
BYTES_PER_POINT = 40   # position 24 B + u 12 B + host 4 B
BYTES_PER_LEAF = 21    # key 8 B + level 1 B + field 12 B


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default="many_bubbles",
                   choices=["many_bubbles", "single_bubble", "learned_index", "tiny", "tracking"])
    p.add_argument("--search", default="auto", choices=["auto", "learned", "binary"],
                   help="form timed for `value`; auto = the faster of the two (both are reported)")
    p.add_argument("--index", default="mlp3", choices=["mlp3", "mlp2", "linear2"],
                   help="mlp3: MLP root -> 4096 mid -> 2^18 leaf models; mlp2: MLP root -> 4096 leaf models")
    p.add_argument("--spread", default="sorted", choices=["sorted", "atomic"])
    p.add_argument("--n-mid", type=int, default=None, help="override the mid model count of mlp3")
    p.add_argument("--n-leaf", type=int, default=None, help="override the leaf model count")
    p.add_argument("--scale", type=float, default=1.0, help="scale point counts (testing only)")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--cpu-seconds", type=float, default=12.0)
    p.add_argument("--launch", default="", help="block,tile,blocks_per_sm[,order_level[,tri_tile,tri_blocks_per_sm]]")
    p.add_argument("--map-level", type=int, default=None, help="level of the level map (default: autotuned)")
    p.add_argument("--no-autotune", action="store_true", help="default launch shape and level map")
    p.add_argument("--no-nomap", action="store_true", help="skip the forms without a level map")
    p.add_argument("--no-mdf", action="store_true", help="skip the multi-direct forcing measurement")
    p.add_argument("--markers-as-generated", action="store_true",
                   help="keep the markers in generation order (default: per bubble, Morton order)")
    p.add_argument("--no-morton-form", action="store_true",
                   help="skip the informative form with the particles stored in Morton order")
    p.add_argument("--no-mates", action="store_true",
                   help="search the trilinear level-mates per query instead of reading the level-mate table")
    return p.parse_args()


def max_over_ranks(value: float, dist, device) -> float:
    """The largest value over all ranks (the job's time is its slowest rank's)."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(points_per_rank: int, world: int, ms_per_step: float) -> float:
    """Whole-job throughput: every rank processes its own batch of points per step."""
    return world * points_per_rank / (ms_per_step / 1e3)


def make_workload(name: str, scale: float, rank: int):
    from paper_2605_20565_gb300 import synth
    if name == "many_bubbles":
        w = synth.many_bubbles(n_markers=int(2_000_000 * scale), n_particles=int(50_000_000 * scale))
    elif name == "single_bubble":
        w = synth.single_bubble(n_markers=int(50_000 * scale), n_particles=int(10_000_000 * scale))
    elif name == "learned_index":
        w = synth.learned_index(n_particles=int(100_000_000 * scale), n_markers=0)
    else:
        w = synth.tiny()
    if rank:  # independent particles per rank (same tree)
        w.particles = synth._uniform_points(w.seed + 1000 * rank, 3, w.particles.shape[1])
    return w


def describe(w, n_leaves, search):
    return {
        "workload": w.name,
        "bubbles": int(w.spheres.shape[0]),
        "levels": [w.lmin, w.lmax],
        "leaves": int(n_leaves),
        "markers_peskin4": int(w.markers.shape[1]),
        "particles_trilinear": int(w.particles.shape[1]),
        "search": search,
        "index": search,
        "spread": "Peskin-4 sorted deterministic",
        "level_map": "top levels staged as a dense level map (level autotuned over 6-8 unless given)",
        "l2": "inputs larger than L2 (tree + field ~0.7 GB, level-mate table 256 B/leaf, points 1.2 GB); "
              "no flush",
    }


BATCH_SOURCES = ("ot_batch.cu", "ot_queue.cuh", "ot_points.cuh", "ot_common.cuh", "ot_pyramid.cu", "ot_mates.cu")


def kernel_sources_hash() -> str:
    """SHA-256 of the batch kernel's sources, to tell whether a stored ncu capture still applies."""
    import hashlib
    h = hashlib.sha256()
    for name in BATCH_SOURCES:
        with open(os.path.join(ROOT, "paper_2605_20565_gb300", "csrc", name), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def batch_traffic(workload: str, form: str, map_level: int, mates: bool):
    """DRAM bytes of one batch graph replay (every kernel in it) from the committed ncu summary,
    when it was taken on this workload, form, level map and level-mate form with the current
    kernel sources; else (None, reason)."""
    path = os.path.join(ROOT, "profiles", f"k_batch_{workload.split('_l')[0]}_traffic.txt")
    if not os.path.exists(path):
        return None, "no capture"
    d = {}
    for line in open(path):
        if ":" in line and not line.startswith("#"):
            k, v = line.split(":", 1)
            d[k.strip()] = v.strip()
    if (d.get("workload") != workload or d.get("form") != form or int(d.get("map_level", -1)) != map_level
            or d.get("level_mates") != ("table" if mates else "searched per query")):
        return None, "capture taken on another workload, form, level map or level-mate form"
    if d.get("kernel_sources_sha256") != kernel_sources_hash():
        return None, "kernel changed since the capture"
    return int(d["bytes_per_replay"]), os.path.relpath(path, ROOT)


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self, index: int):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={index}", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                       "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        rows = [r.split(",") for r in open(self.f.name).read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
                for k, nm in enumerate(names):
                    if r[5 + k].strip().lower() == "active":
                        reasons.add(nm)
            except (ValueError, IndexError):
                continue
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------------------
# CPU oracle timing (cpu_baseline leg and --impl reference)
# ---------------------------------------------------------------------------------------

def oracle_setup(w):
    import oracle
    t0 = time.time()
    ko, lo = oracle.octree_build(w.spheres, w.lmin, w.lmax)
    cen = oracle.leaf_centres(ko, lo)
    from paper_2605_20565_gb300 import synth
    field = synth.fourier_field(w.modes, cen) if w.modes is not None else synth.sin_field(cen)
    return ko, lo, field.astype(np.float32).astype(np.float64), time.time() - t0


def oracle_step(w, ko, lo, field, npart, nmark):
    """locate + interpolate npart particles and nmark markers, spread nmark markers."""
    import oracle
    P = w.particles[:, :npart]
    X = w.markers[:, :nmark]
    t0 = time.perf_counter()
    host = oracle.locate_ub(ko, lo, *P)
    up = oracle.interp_trilinear(ko, lo, field, *P, host)
    um = None
    if nmark:
        um, _ = oracle.interp_delta(ko, lo, w.lmax, 2, field, *X)
        oracle.spread_delta(ko, lo, w.lmax, 2, *X, w.forces[:, :nmark])
    return time.perf_counter() - t0, host, up, um


def size_cpu_sample(w, ko, lo, field, seconds):
    """Points per oracle step so that one step takes about `seconds`."""
    n_p0 = min(200_000, w.particles.shape[1])
    frac = w.markers.shape[1] / max(1, w.n_points)
    n_m0 = min(int(n_p0 * frac), w.markers.shape[1])
    dt, *_ = oracle_step(w, ko, lo, field, n_p0, n_m0)
    k = max(1.0, seconds / max(dt, 1e-3))
    n_p = min(int(n_p0 * k), w.particles.shape[1])
    n_m = min(int(n_m0 * k), w.markers.shape[1])
    return n_p, n_m


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle
    w = make_workload(args.workload, args.scale, 0)
    ko, lo, field, setup_s = oracle_setup(w)
    n_p, n_m = size_cpu_sample(w, ko, lo, field, min(args.cpu_seconds, 20.0) / max(1, args.steps + args.warmup) * 4)
    times = []
    for s in range(args.warmup + args.steps):
        dt, *_ = oracle_step(w, ko, lo, field, n_p, n_m)
        if s >= args.warmup:
            times.append(dt)
    ms = 1e3 * statistics.median(times)
    value = (n_p + n_m) / (ms / 1e3)
    cores = oracle.num_threads()
    sample = (f"{n_p} particles (trilinear) + {n_m} markers (Peskin-4 interp + spread) of {w.name} "
              f"per step; oracle octree build {setup_s:.1f} s untimed")
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": "points/s", "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": describe(w, ko.size, "binary (CPU, FP64)"),
           "cpu_baseline": {"value": value, "unit": "points/s", "cores": cores, "kind": "oracle", "sample": sample},
           "e2e": {"value": value, "unit": "points/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)
    return 0


# ---------------------------------------------------------------------------------------
# GPU path
# ---------------------------------------------------------------------------------------

def run_ours(args):
    import torch
    import paper_2605_20565_gb300 as ot
    from paper_2605_20565_gb300 import _build, synth

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        dist = None
        torch.cuda.set_device(0)
    if rank == 0 or not os.path.exists(_build.LIB):
        _build.build()
    if dist:
        dist.barrier()
    dev = torch.device("cuda", local)

    def barrier():
        if dist:
            dist.barrier()

    w = make_workload(args.workload, args.scale, rank)
    if not args.markers_as_generated:
        synth.order_markers(w)  # the stored marker order: per bubble, Morton order of positions
    t0 = time.time()
    tree = ot.ot_octree_build(w.spheres, w.lmin, w.lmax)
    torch.cuda.synchronize()
    build_s = time.time() - t0
    n_leaves = ot.ot_octree_info(tree)[0]
    if args.map_level is not None:
        ot.ot_octree_set_map_level(tree, args.map_level)
    mates_s = None
    if not args.no_mates:
        t0 = time.time()
        ot.ot_octree_build_mates(tree, True)
        torch.cuda.synchronize()
        mates_s = time.time() - t0
    t0 = time.time()
    root = ot.OT_ROOT_LINEAR if args.index == "linear2" else ot.OT_ROOT_MLP
    n_leaf, n_mid = (1 << 18, 4096) if args.index == "mlp3" else (4096, 0)
    if args.n_leaf:
        n_leaf = args.n_leaf
    if args.n_mid is not None and args.index == "mlp3":
        n_mid = args.n_mid
    ot.ot_index_train(tree, root=root, n_leaf_models=n_leaf, n_mid_models=n_mid, epochs=4, batch=65536, lr=1e-3,
                      seed=1)
    torch.cuda.synchronize()
    train_s = time.time() - t0
    istats = ot.ot_index_get_stats(tree, reset=True)

    if w.modes is not None:
        field = ot.ot_field_fourier(tree, w.modes.n, w.modes.amp, w.modes.phase)
    else:
        cen = ot.ot_octree_centres(tree)
        field = torch.as_tensor(synth.sin_field(cen.T.cpu().numpy()), device=dev).to(torch.float32).contiguous()
        del cen

    def to_dev(a):
        return [torch.as_tensor(np.ascontiguousarray(a[d]), device=dev) for d in range(3)]

    mx, my, mz = to_dev(w.markers)
    px, py, pz = to_dev(w.particles)
    Fm = torch.as_tensor(np.ascontiguousarray(w.forces, dtype=np.float32), device=dev)
    n_m, n_p = w.markers.shape[1], w.particles.shape[1]
    npts = n_m + n_p
    um = torch.empty((3, n_m), dtype=torch.float32, device=dev)
    up = torch.empty((3, n_p), dtype=torch.float32, device=dev)
    f = torch.zeros((n_leaves, 4), dtype=torch.float32, device=dev)
    mode = ot.OT_SORTED if args.spread == "sorted" else ot.OT_ATOMIC
    ws_bytes = ot.ot_spread_workspace_size(tree, ot.OT_PESKIN4, n_m) if mode == ot.OT_SORTED else 0
    ws = torch.empty(max(1, ws_bytes), dtype=torch.uint8, device=dev)
    launch = None
    if args.launch:
        vals = [int(v) for v in args.launch.split(",")]
        launch = dict(zip(("block", "tile", "blocks_per_sm", "order_level", "tri_tile", "tri_blocks_per_sm"), vals))
    groups = [dict(kernel=ot.OT_PESKIN4, x=mx, y=my, z=mz, u=um), dict(kernel=ot.OT_TRILINEAR, x=px, y=py, z=pz, u=up)]
    stream = torch.cuda.current_stream()

    # search forms over the same groups: (search, level-map level, launch shape, level-mate
    # table).  "plain" and "learned" are autotuned (launch shape and level-map level) unless a
    # launch or map level is given; the "_nomap" forms search the whole key array (level map of
    # one cell), the plain one being Algorithm 1's binary search and the learned one the index
    # without any map; "plain_search" searches every trilinear level-mate per query.
    base_level = ot.ot_octree_get_map_level(tree)
    use_mates = not args.no_mates
    forms_cfg, tune = {}, {}
    for name, sv in (("plain", ot.OT_BINARY), ("learned", ot.OT_LEARNED)):
        if launch is None and not args.no_autotune:
            r = ot.ot_batch_autotune(tree, groups, field, search=sv, tune_map_level=args.map_level is None, reps=2)
            tune[name] = r
            forms_cfg[name] = (sv, r["map_level"], r["launch"], use_mates)
        else:
            forms_cfg[name] = (sv, base_level, launch, use_mates)
    if use_mates:
        forms_cfg["plain_search"] = (ot.OT_BINARY,) + forms_cfg["plain"][1:3] + (False,)
    if not args.no_nomap:
        forms_cfg["plain_nomap"] = (ot.OT_BINARY, 0, launch, use_mates)
        forms_cfg["learned_nomap"] = (ot.OT_LEARNED, 0, launch, use_mates)

    def set_form(name):
        sv, lvl, lp, mt = forms_cfg[name]
        if ot.ot_octree_get_map_level(tree) != lvl:
            ot.ot_octree_set_map_level(tree, lvl)
        if ot.ot_octree_has_mates(tree) != mt:
            ot.ot_octree_build_mates(tree, mt)
        return sv, lp

    def make_batch(name):
        sv, lp = set_form(name)
        return ot.ot_batch_create(tree, groups, field, search=sv, launch=lp)

    def step(batch, ev=None):
        if ev:
            ev[0].record(stream)
        ot.ot_batch_run(batch)
        if ev:
            ev[1].record(stream)
        f.zero_()
        ot.ot_spread(tree, ot.OT_PESKIN4, mode, mx, my, mz, Fm, f, workspace=ws)
        if ev:
            ev[2].record(stream)

    def time_steps(batch, k):
        evs_ = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(k)]
        for e in evs_:
            step(batch, e)
        torch.cuda.synchronize()
        li = statistics.mean(e[0].elapsed_time(e[1]) for e in evs_)
        sp = statistics.mean(e[1].elapsed_time(e[2]) for e in evs_)
        return {"step_ms": statistics.mean(e[0].elapsed_time(e[2]) for e in evs_), "locate_interpolate_ms": li,
                "spread_ms": sp}

    def warm(batch):
        for _ in range(max(3, args.warmup)):
            step(batch)
        torch.cuda.synchronize()

    if args.search == "auto":
        cal = {}
        for name in ("plain", "learned"):
            bb = make_batch(name)
            warm(bb)
            cal[name] = time_steps(bb, 3)["step_ms"]
            del bb
        chosen = min(cal, key=cal.get)
    else:
        chosen = "learned" if args.search == "learned" else "plain"
    batch = make_batch(chosen)
    warm(batch)
    assert ot.ot_last_error(tree) & (ot.OT_DEV_STENCIL | ot.OT_DEV_OUTSIDE | ot.OT_DEV_REFINED_CAP) == 0
    ot.ot_index_get_stats(tree, reset=True)

    # timed region: the chosen form
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
    clocks = Clocks(local) if rank == 0 else None
    barrier()
    torch.cuda.synchronize()
    launches0 = ot.ot_launch_count()
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.nvtx.range_push("timed")
    start.record(stream)
    for k in range(args.steps):
        step(batch, evs[k])
    stop.record(stream)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    barrier()
    launches = ot.ot_launch_count() - launches0
    clk = clocks.stop() if clocks else None
    total_ms = max_over_ranks(start.elapsed_time(stop), dist, dev)
    ms_step = total_ms / args.steps
    batch_ms = statistics.mean(e[0].elapsed_time(e[1]) for e in evs)
    spread_ms = statistics.mean(e[1].elapsed_time(e[2]) for e in evs)
    value = job_value(npts, world, ms_step)
    fb = ot.ot_index_get_stats(tree, reset=True)["fallbacks"] if chosen == "learned" else None
    search = forms_cfg[chosen][0]
    # end to end through the public API with host buffers
    e2e = None
    if not args.no_e2e:
        hm = [torch.from_numpy(np.ascontiguousarray(w.markers[d])).pin_memory() for d in range(3)]
        hp = [torch.from_numpy(np.ascontiguousarray(w.particles[d])).pin_memory() for d in range(3)]
        hum = torch.empty((3, n_m), dtype=torch.float32).pin_memory()
        hup = torch.empty((3, n_p), dtype=torch.float32).pin_memory()
        hf = torch.empty((n_leaves, 4), dtype=torch.float32).pin_memory()
        h2d = sum(t.numel() * t.element_size() for t in hm + hp)
        d2h = (hum.numel() + hup.numel() + hf.numel()) * 4

        def e2e_step():
            for d in range(3):
                (mx, my, mz)[d].copy_(hm[d], non_blocking=True)
                (px, py, pz)[d].copy_(hp[d], non_blocking=True)
            step(batch)
            hum.copy_(um, non_blocking=True)
            hup.copy_(up, non_blocking=True)
            hf.copy_(f, non_blocking=True)

        e2e_step()
        torch.cuda.synchronize()
        k_e2e = max(3, min(args.steps, 10))
        barrier()
        t0 = time.perf_counter()
        for _ in range(k_e2e):
            e2e_step()
        torch.cuda.synchronize()
        barrier()
        serial_ms = max_over_ranks(1e3 * (time.perf_counter() - t0) / k_e2e, dist, dev)

        # Pipelined: two slots of device buffers (each with its own batch graph); step k computes
        # on slot k % 2 while step k + 1's inputs go up and step k - 1's results come down on
        # their own streams.  Every step still copies all its inputs and results.
        class Slot:
            pass

        def make_slot(first):
            sl = Slot()
            if first:
                sl.m, sl.p, sl.um, sl.up, sl.f, sl.ws, sl.batch = (mx, my, mz), (px, py, pz), um, up, f, ws, batch
            else:
                sl.m = tuple(torch.empty_like(a_) for a_ in (mx, my, mz))
                sl.p = tuple(torch.empty_like(a_) for a_ in (px, py, pz))
                sl.um, sl.up, sl.f, sl.ws = (torch.empty_like(um), torch.empty_like(up), torch.zeros_like(f),
                                             torch.empty_like(ws))
                sv_, _, lp_, _ = forms_cfg[chosen]
                sl.batch = ot.ot_batch_create(tree, [dict(kernel=ot.OT_PESKIN4, x=sl.m[0], y=sl.m[1], z=sl.m[2], u=sl.um),
                                                     dict(kernel=ot.OT_TRILINEAR, x=sl.p[0], y=sl.p[1], z=sl.p[2],
                                                          u=sl.up)], field, search=sv_, launch=lp_)
            sl.hum = torch.empty((3, n_m), dtype=torch.float32).pin_memory()
            sl.hup = torch.empty((3, n_p), dtype=torch.float32).pin_memory()
            sl.hf = torch.empty((n_leaves, 4), dtype=torch.float32).pin_memory()
            sl.ev_in, sl.ev_comp, sl.ev_out = (torch.cuda.Event(), torch.cuda.Event(), torch.cuda.Event())
            return sl

        slots = [make_slot(True), make_slot(False)]
        s_in, s_out = torch.cuda.Stream(), torch.cuda.Stream()

        def piped_step(k):
            sl = slots[k % 2]
            with torch.cuda.stream(s_in):
                s_in.wait_event(sl.ev_comp)  # the slot's previous step has read its inputs
                for d in range(3):
                    sl.m[d].copy_(hm[d], non_blocking=True)
                    sl.p[d].copy_(hp[d], non_blocking=True)
                sl.ev_in.record(s_in)
            stream.wait_event(sl.ev_in)
            stream.wait_event(sl.ev_out)  # the slot's previous results are on the host
            ot.ot_batch_run(sl.batch)
            sl.f.zero_()
            ot.ot_spread(tree, ot.OT_PESKIN4, mode, sl.m[0], sl.m[1], sl.m[2], Fm, sl.f, workspace=sl.ws)
            sl.ev_comp.record(stream)
            with torch.cuda.stream(s_out):
                s_out.wait_event(sl.ev_comp)
                sl.hum.copy_(sl.um, non_blocking=True)
                sl.hup.copy_(sl.up, non_blocking=True)
                sl.hf.copy_(sl.f, non_blocking=True)
                sl.ev_out.record(s_out)

        for k in range(2):
            piped_step(k)
        torch.cuda.synchronize()
        barrier()
        t0 = time.perf_counter()
        for k in range(k_e2e):
            piped_step(k)
        torch.cuda.synchronize()
        barrier()
        e2e_ms = max_over_ranks(1e3 * (time.perf_counter() - t0) / k_e2e, dist, dev)
        piped_ok = (torch.equal(slots[0].up, slots[1].up) and torch.equal(slots[0].f, slots[1].f)
                    and torch.equal(slots[1].hup, slots[1].up.cpu()))
        del slots
        e2e = {"value": job_value(npts, world, e2e_ms), "unit": "points/s", "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h), "ms_per_step": e2e_ms, "steps": k_e2e,
               "pipeline": "2 slots; inputs up, compute, results down on three streams, overlapped across steps",
               "pipelined_results_identical": bool(piped_ok),
               "serial_ms_per_step": serial_ms, "serial_value": job_value(npts, world, serial_ms)}

    # multi-direct forcing (Sec. 2.2) on the same markers: 3 rounds towards a body at rest
    mdf = None
    if not args.no_mdf and n_m > 0:
        U0 = torch.zeros((3, n_m), dtype=torch.float32, device=dev)
        # marker volumes dV_k = (S_b / N_b) h, the body's surface per marker times the finest cell
        grp = w.marker_group.astype(np.int64)
        nb_k = np.bincount(grp, minlength=w.spheres.shape[0])[grp]
        dv_np = 4.0 * np.pi * w.spheres[grp, 3] ** 2 / nb_k * 2.0 ** -w.lmax
        dV_ = torch.as_tensor(dv_np.astype(np.float32), device=dev)
        um_ = field.clone()
        ot.ot_ibm_mdf(tree, ot.OT_PESKIN4, mx, my, mz, U0, um_, 1.0, 1.0, 3, dV=dV_)
        a_, b_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        um_.copy_(field)
        a_.record(stream)
        _, slip_ = ot.ot_ibm_mdf(tree, ot.OT_PESKIN4, mx, my, mz, U0, um_, 1.0, 1.0, 3, dV=dV_, slip=True)
        b_.record(stream)
        torch.cuda.synchronize()
        mdf_ms = a_.elapsed_time(b_)
        sl = slip_.cpu().numpy()
        mdf = {"rounds": 3, "ms": mdf_ms, "markers_per_s": n_m / (mdf_ms / 1e3),
               "slip_reduction": float(sl[-1] / sl[0]) if sl[0] > 0 else None,
               "note": "dV_k = (S_b / N_b) h; workspace allocation included; field sweeps over all leaves per round"}
        del um_, U0

    # internal-fluid momenta of the bodies (Sec. 2.3): trilinear velocity at the internal markers
    # (a lattice of the finest cell inside each bubble), then the per-body sums
    bodies = None
    if not args.no_mdf and w.extra and "centres" in w.extra:
        hmin = 2.0 ** -w.lmax
        Xi, st_i = synth.internal_markers(w.extra["centres"], w.extra["diameters"], hmin)
        xi, yi, zi = to_dev(Xi)
        d_start = torch.as_tensor(st_i, device=dev)
        xb = torch.as_tensor(np.ascontiguousarray(w.extra["centres"]), device=dev)
        ui = torch.empty((3, Xi.shape[1]), dtype=torch.float32, device=dev)

        def momenta():
            ot.ot_interpolate(tree, ot.OT_TRILINEAR, xi, yi, zi, field, u=ui)
            return ot.ot_body_sums(xi, yi, zi, ui, d_start, xb, 1.0, w=hmin ** 3)

        momenta()
        a_, b_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a_.record(stream)
        for _ in range(3):
            momenta()
        b_.record(stream)
        torch.cuda.synchronize()
        bodies = {"bodies": int(len(st_i) - 1), "internal_markers": int(Xi.shape[1]),
                  "ms": a_.elapsed_time(b_) / 3, "what": "trilinear u at internal markers + per-body P and L"}
        del xi, yi, zi, ui

    # the other forms, same steps (the chosen form's level map is restored afterwards)
    forms = {chosen: {"step_ms": ms_step, "locate_interpolate_ms": batch_ms, "spread_ms": spread_ms}}
    groups_t = {}
    del batch
    for name in forms_cfg:
        if name != chosen:
            bb = make_batch(name)
            warm(bb)
            forms[name] = time_steps(bb, args.steps)
            del bb
        # per-group timing (markers only, particles only) at the form's settings
        for gname, gsel in (("markers", groups[:1]), ("particles", groups[1:])):
            sv, lp = set_form(name)
            bb = ot.ot_batch_create(tree, gsel, field, search=sv, launch=lp)
            for _ in range(2):
                ot.ot_batch_run(bb)
            a_, b_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a_.record(stream)
            for _ in range(5):
                ot.ot_batch_run(bb)
            b_.record(stream)
            torch.cuda.synchronize()
            groups_t[f"{gname}_{name}_ms"] = a_.elapsed_time(b_) / 5
            del bb
    # informative, not `value`: the plain step with the particles stored in Morton order of
    # their level-8 cells (the order the tracking driver keeps them in; sorted once, untimed)
    morton = None
    if not args.no_morton_form and n_p > 0 and forms_cfg["plain"][3]:
        set_form("plain")
        perm = ot.ot_points_morton_order(px, py, pz).long()
        sx, sy, sz = [a_.index_select(0, perm).contiguous() for a_ in (px, py, pz)]
        del perm
        up_m = torch.empty_like(up)  # its own outputs: `up` keeps the timed form's for the parity check
        gs = [groups[0], dict(kernel=ot.OT_TRILINEAR, x=sx, y=sy, z=sz, u=up_m)]
        lp_m = ot.ot_batch_autotune(tree, gs, field, search=ot.OT_BINARY, tune_map_level=False, reps=2)["launch"]
        bb = ot.ot_batch_create(tree, gs, field, search=ot.OT_BINARY, launch=lp_m)
        warm(bb)
        morton = time_steps(bb, args.steps)
        morton.update(points_per_s=npts / (morton["step_ms"] / 1e3),
                      locate_interpolate_points_per_s=npts / (morton["locate_interpolate_ms"] / 1e3), launch=lp_m,
                      map_level=forms_cfg["plain"][1], search="binary", level_mates="table",
                      particle_order="Morton order of level-8 cells")
        del bb, sx, sy, sz, gs, up_m
    for name, v_ in forms.items():
        v_["points_per_s"] = npts / (v_["step_ms"] / 1e3)
        v_["locate_interpolate_points_per_s"] = npts / (v_["locate_interpolate_ms"] / 1e3)
        v_["search"] = "learned" if forms_cfg[name][0] == ot.OT_LEARNED else "binary"
        v_["map_level"] = forms_cfg[name][1]
        v_["launch"] = forms_cfg[name][2]
        v_["level_mates"] = "table" if forms_cfg[name][3] else "searched per query"
    learned_vs_plain = {
        "with_level_map": {
            "locate_interpolate": forms["plain"]["locate_interpolate_ms"] / forms["learned"]["locate_interpolate_ms"],
            "step": forms["plain"]["step_ms"] / forms["learned"]["step_ms"]}}
    if "plain_nomap" in forms:
        # the learned index with its level map against Algorithm 1's binary search of the whole
        # key array (no staging of the top tree levels)
        learned_vs_plain["learned_vs_whole_array_binary"] = {
            "locate_interpolate": forms["plain_nomap"]["locate_interpolate_ms"] /
            forms["learned"]["locate_interpolate_ms"],
            "step": forms["plain_nomap"]["step_ms"] / forms["learned"]["step_ms"]}
        learned_vs_plain["without_level_map"] = {
            "locate_interpolate": forms["plain_nomap"]["locate_interpolate_ms"] /
            forms["learned_nomap"]["locate_interpolate_ms"],
            "step": forms["plain_nomap"]["step_ms"] / forms["learned_nomap"]["step_ms"]}
    if "plain_search" in forms:
        learned_vs_plain["table_vs_search_plain_step"] = forms["plain_search"]["step_ms"] / forms["plain"]["step_ms"]
    if morton:
        forms["plain_particles_morton"] = morton
    set_form(chosen)

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return 0

    peak, peak_kind = measured_peaks()
    alg_bytes = npts * BYTES_PER_POINT + n_leaves * BYTES_PER_LEAF
    achieved = alg_bytes / (batch_ms / 1e3) / 1e9
    traffic, traffic_src = batch_traffic(w.name, chosen, forms_cfg[chosen][1], forms_cfg[chosen][3])
    roof = {"bound": "hbm", "kernel": "batch graph replay (cell means + k_batch delta-kernel launch + k_batch "
                                      "trilinear launch): locate + interpolate of every point",
            "achieved": achieved,
            "peak": peak, "unit": "GB/s", "frac": achieved / peak, "traffic": traffic, "traffic_source": traffic_src,
            "peak_kind": peak_kind, "algorithmic_bytes_per_launch": int(alg_bytes),
            "bytes_rule": f"{BYTES_PER_POINT} B/point + {BYTES_PER_LEAF} B/leaf"}

    cpu = None
    parity = None
    if not args.no_cpu_baseline:
        import oracle
        ko, lo, fref, setup_s = oracle_setup(w)
        kg, lg = ot.ot_octree_copy_leaves(tree)
        tree_exact = bool(np.array_equal(kg.cpu().numpy().view(np.uint64), ko) and
                          np.array_equal(lg.cpu().numpy(), lo))
        n_ps, n_ms = size_cpu_sample(w, ko, lo, fref, args.cpu_seconds)
        dt, host_ref, up_ref, um_ref = oracle_step(w, ko, lo, fref, n_ps, n_ms)
        cpu = {"value": (n_ps + n_ms) / dt, "unit": "points/s", "cores": oracle.num_threads(), "kind": "oracle",
               "sample": f"{n_ps} particles + {n_ms} markers of {w.name} (locate, interpolate, spread), "
                         f"one step, {dt:.1f} s; oracle tree build {setup_s:.1f} s untimed"}
        # sampled parity of the timed launch's outputs (same field values, FP32 inputs)
        fscale = float(np.abs(fref[:, :3]).max())
        hp_gpu = ot.ot_locate(tree, px[:n_ps], py[:n_ps], pz[:n_ps], search=search).cpu().numpy()
        parity = {"octree_bit_exact": tree_exact,
                  "hosts_bit_exact": bool(np.array_equal(hp_gpu, host_ref)),
                  "particles_max_rel_err": float(np.abs(up[:, :n_ps].cpu().numpy() - up_ref).max() / fscale),
                  "markers_max_rel_err": (float(np.abs(um[:, :n_ms].cpu().numpy() - um_ref).max() / fscale)
                                          if n_ms else None),
                  "sampled_points": n_ps + n_ms}

    out = {"metric": METRIC, "value": value, "unit": "points/s", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": dict(describe(w, n_leaves, INDEX_DESC[args.index] if chosen == "learned" else
                                   "plain: level map + binary search"),
                          form=chosen, map_level=forms_cfg[chosen][1], launch=forms_cfg[chosen][2],
                          level_mates="table" if forms_cfg[chosen][3] else "searched per query",
                          marker_order=("as generated (Fibonacci spiral per bubble)" if args.markers_as_generated
                                        else "per bubble, Morton order of level-10 cells"),
                          particle_order="as generated (uniform random)"),
           "roofline": roof, "cpu_baseline": cpu, "e2e": e2e,
           "gpu_launches": int(launches), "clocks": clk,
           "breakdown_ms": {"locate_interpolate": batch_ms, "spread": spread_ms, "step": ms_step},
           "locate_interpolate_points_per_s": world * npts / (batch_ms / 1e3),
           "forms": forms, "learned_vs_plain": learned_vs_plain, "groups_ms": groups_t, "autotune": tune,
           "mdf": mdf, "body_momenta": bodies,
           "index": {"n_mid": n_mid, "n_leaf": n_leaf, "mean_window": istats["mean_window"], "max_window": istats["max_window"],
                     "empty_models": istats["empty_models"], "fallbacks_timed": fb,
                     "mean_probes": istats["mean_probes"],
                     "final_loss": istats["final_loss"], "train_s": train_s},
           "setup_s": {"octree_build": build_s, "index_train": train_s, "level_mate_table": mates_s},
           "parity": parity}
    print(json.dumps(out), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def run_tracking(args):
    """The time-stepped workload: 256 bubbles moving, 200M particles advected by AB2, markers
    spread every step, octree rebuilt and index retrained every 10 steps (all timed)."""
    import torch
    import paper_2605_20565_gb300 as ot
    from paper_2605_20565_gb300 import _build, synth, tracking
    torch.cuda.set_device(0)
    _build.build()
    w = synth.tracking(n_particles=int(200_000_000 * args.scale))
    search = ot.OT_LEARNED if args.search == "learned" else ot.OT_BINARY
    t0 = time.time()
    launch = None
    if args.launch:
        vals = [int(v) for v in args.launch.split(",")]
        launch = dict(zip(("block", "tile", "blocks_per_sm", "order_level", "tri_tile", "tri_blocks_per_sm"), vals))
    tr = tracking.Tracker(w, search=search, rebuild_every=10, mates=not args.no_mates, map_level=args.map_level,
                          launch=launch)
    setup_s = time.time() - t0
    n_leaves = ot.ot_octree_info(tr.tree)[0]
    for _ in range(args.warmup):
        tr.step()
    torch.cuda.synchronize()
    tr.timings = {"rebuild_s": 0.0, "rebuilds": 0}
    clocks = Clocks(0)
    launches0 = ot.ot_launch_count()
    t0 = time.perf_counter()
    pts = 0
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(5)] for _ in range(args.steps)]
    for k in range(args.steps):
        pts += tr.step(evs[k])
    torch.cuda.synchronize()
    el = time.perf_counter() - t0
    parts = {name: statistics.mean(e[i].elapsed_time(e[i + 1]) for e in evs)
             for i, name in enumerate(("batch", "advect", "spread", "markers"))}
    clk = clocks.stop()
    out = {"metric": METRIC, "value": pts / el, "unit": "points/s", "n_gpus": 1, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": w.name, "bubbles": int(w.spheres.shape[0]), "levels": [w.lmin, w.lmax],
                      "leaves": int(n_leaves), "markers_peskin4": int(w.markers.shape[1]),
                      "particles_trilinear": int(w.particles.shape[1]),
                      "search": "learned" if search == ot.OT_LEARNED else "binary",
                      "level_mates": "searched per query" if args.no_mates else "table",
                      "map_level": ot.ot_octree_get_map_level(tr.tree),
                      "launch": tr.launch, "launch_autotuned": launch is None,
                      "step": "locate+interpolate all points, AB2 advect particles, sorted spread of markers; "
                              "octree rebuild + index retrain + field resample every 10 steps",
                      "l2": "inputs larger than L2; no flush"},
           "rebuild": {"rebuilds_timed": tr.timings["rebuilds"], "rebuild_s_timed": tr.timings["rebuild_s"],
                       "parts_s_timed": tr.timings.get("rebuild_parts_s"), "setup_s": setup_s},
           "step_parts_ms": parts,
           "gpu_launches": int(ot.ot_launch_count() - launches0), "clocks": clk,
           "roofline": None, "cpu_baseline": None, "e2e": None}
    print(json.dumps(out), flush=True)
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "tracking":
        return run_tracking(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
