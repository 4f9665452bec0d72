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
    p.add_argument("--launch", default="",
                   help="block,tile,blocks_per_sm[,order_level[,tri_tile,tri_blocks_per_sm[,tri_records]]]")
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
    p.add_argument("--only", action="store_true",
                   help="the headline workload only (no compact lines of the other workloads)")
    p.add_argument("--workloads", default="tiny,single_bubble,learned_index,tracking",
                   help="the other workloads measured after the many-bubble headline (compact lines)")
    p.add_argument("--tracking-steps", type=int, default=100, help="timed steps of the tracking workload")
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
    """DRAM bytes of one replay of the particles' graph (every kernel in it) from the committed
    ncu summary, when it was taken on this workload, form, level map and level-mate form with
    the current kernel sources; else (None, reason)."""
    path = os.path.join(ROOT, "profiles", f"particles_graph_{workload.split('_l')[0]}_traffic.txt")
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

def launch_of(text: str):
    if not text:
        return None
    vals = [int(v) for v in text.split(",")]
    return dict(zip(("block", "tile", "blocks_per_sm", "order_level", "tri_tile", "tri_blocks_per_sm",
                     "tri_records"), vals))


_ORACLE_TREES = {}


def oracle_tree(w):
    """The oracle's octree of a workload's spheres (kept for workloads that share them)."""
    import oracle
    key = (w.spheres.tobytes(), w.lmin, w.lmax)
    if key not in _ORACLE_TREES:
        t0 = time.time()
        ko, lo = oracle.octree_build(w.spheres, w.lmin, w.lmax)
        _ORACLE_TREES[key] = (ko, lo, time.time() - t0)
    return _ORACLE_TREES[key]


def synthetic_field32(w, ko, lo, dev):
    """The workload's velocity field at the oracle's leaf centres, rounded to FP32 once: the one
    array both the GPU path and the oracle read in the parity legs (an input, made by the
    workload generator, not by the library under test)."""
    import torch
    import oracle
    from paper_2605_20565_gb300 import synth
    cen = oracle.leaf_centres(ko, lo)
    if w.modes is None:
        return torch.as_tensor(synth.sin_field(cen), device=dev).to(torch.float32).contiguous()
    f = synth.fourier_field(w.modes, torch.as_tensor(cen, device=dev))
    return f.to(torch.float32).contiguous()


def gpu_numa_cpus(index: int):
    """Host CPUs of the NUMA node the GPU hangs off (empty when the system does not say)."""
    try:
        bus = subprocess.run(["nvidia-smi", f"--id={index}", "--query-gpu=pci.bus_id", "--format=csv,noheader"],
                             capture_output=True, text=True, timeout=20).stdout.strip()
        dom, rest = bus.split(":", 1)
        path = f"/sys/bus/pci/devices/{dom[-4:].lower()}:{rest.lower()}/numa_node"
        node = int(open(path).read().strip())
        if node < 0:
            return node, []
        cpus = []
        for part in open(f"/sys/devices/system/node/node{node}/cpulist").read().strip().split(","):
            a, _, b = part.partition("-")
            cpus.extend(range(int(a), int(b or a) + 1))
        return node, cpus
    except (OSError, ValueError, subprocess.SubprocessError):
        return None, []


class StepBatches:
    """A step's two graphs over the same groups: the delta-kernel (marker) groups and the
    trilinear (particle) groups, each a batch of its own, replayed one after the other."""

    def __init__(self, ot, tree, groups, field, search, launch):
        self.ot = ot
        gm = [g for g in groups if g["kernel"] != ot.OT_TRILINEAR and g["x"].numel() > 0]
        gp = [g for g in groups if g["kernel"] == ot.OT_TRILINEAR and g["x"].numel() > 0]
        self.bm = ot.ot_batch_create(tree, gm, field, search=search, launch=launch) if gm else None
        self.bp = ot.ot_batch_create(tree, gp, field, search=search, launch=launch) if gp else None

    def run_markers(self, stream):
        if self.bm is not None:
            self.ot.ot_batch_run(self.bm, stream=stream)

    def run_particles(self, stream):
        if self.bp is not None:
            self.ot.ot_batch_run(self.bp, stream=stream)


def measure(args, name, light, ctx):
    """One workload through the batched launch: timed steps, e2e with host buffers, the other
    search forms, and the parity and CPU-baseline legs.  Returns the result dict."""
    import torch
    import paper_2605_20565_gb300 as ot
    from paper_2605_20565_gb300 import synth
    dist, world, rank, local, dev = ctx["dist"], ctx["world"], ctx["rank"], ctx["local"], ctx["dev"]
    barrier = ctx["barrier"]

    w = make_workload(name, args.scale, rank)
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
    # every located point's outputs: its velocity (3 planes) and its host leaf
    um = torch.empty((3, n_m), dtype=torch.float32, device=dev)
    up = torch.empty((3, n_p), dtype=torch.float32, device=dev)
    hm = torch.empty(n_m, dtype=torch.int32, device=dev)
    hp = torch.empty(n_p, dtype=torch.int32, device=dev)
    f = torch.zeros((n_leaves, 4), dtype=torch.float32, device=dev)
    mode = ot.OT_SORTED if args.spread == "sorted" else ot.OT_ATOMIC
    ws_bytes = ot.ot_spread_workspace_size(tree, ot.OT_PESKIN4, n_m) if mode == ot.OT_SORTED else 0
    ws = torch.empty(max(1, ws_bytes), dtype=torch.uint8, device=dev)
    launch = launch_of(args.launch)

    def groups_for(m_, p_, um_, up_, hm_, hp_):
        return [dict(kernel=ot.OT_PESKIN4, x=m_[0], y=m_[1], z=m_[2], u=um_, host=hm_),
                dict(kernel=ot.OT_TRILINEAR, x=p_[0], y=p_[1], z=p_[2], u=up_, host=hp_)]

    groups = groups_for((mx, my, mz), (px, py, pz), um, up, hm, hp)
    stream = torch.cuda.current_stream()

    # search forms over the same groups: (search, level-map level, launch shape, level-mate
    # table).  "plain" and "learned" are autotuned (launch shape and level-map level) unless a
    # launch or map level is given; "learned_same_staging" is the learned index with the plain
    # form's level map, table and launch shape (the like-for-like comparison); the "_nomap"
    # forms search the whole key array (a level map of one cell), the plain one being
    # Algorithm 1's binary search; "plain_search" searches every level-mate per query.
    base_level = ot.ot_octree_get_map_level(tree)
    use_mates = not args.no_mates
    forms_cfg, tune = {}, {}
    for fname, sv in (("plain", ot.OT_BINARY), ("learned", ot.OT_LEARNED)):
        if launch is None and not args.no_autotune:
            r = ot.ot_batch_autotune(tree, groups, field, search=sv, tune_map_level=args.map_level is None, reps=2)
            tune[fname] = r
            forms_cfg[fname] = (sv, r["map_level"], r["launch"], use_mates)
        else:
            forms_cfg[fname] = (sv, base_level, launch, use_mates)
    forms_cfg["learned_same_staging"] = (ot.OT_LEARNED,) + forms_cfg["plain"][1:]
    if use_mates and not light:
        forms_cfg["plain_search"] = (ot.OT_BINARY,) + forms_cfg["plain"][1:3] + (False,)
    if not args.no_nomap and not light:
        forms_cfg["plain_nomap"] = (ot.OT_BINARY, 0, launch, use_mates)
        forms_cfg["learned_nomap"] = (ot.OT_LEARNED, 0, launch, use_mates)

    def set_form(fname):
        sv, lvl, lp, mt = forms_cfg[fname]
        if ot.ot_octree_get_map_level(tree) != lvl:
            ot.ot_octree_set_map_level(tree, lvl)
        if ot.ot_octree_has_mates(tree) != mt:
            ot.ot_octree_build_mates(tree, mt)
        return sv, lp

    def make_batch(fname, gs=None):
        """The form's batch over the groups (one graph: delta-kernel and trilinear launches)."""
        sv, lp = set_form(fname)
        return ot.ot_batch_create(tree, gs or groups, field, search=sv, launch=lp)

    def make_step(fname, gs=None):
        """The form's step batches: the markers' and the particles' graphs, replayed one after
        the other, so that each part (the particles' -- cell means, value records and the
        trilinear launch -- is the dominant one) is timed on its own with events."""
        sv, lp = set_form(fname)
        return StepBatches(ot, tree, gs or groups, field, sv, lp)

    def step(sb, ev=None):
        # ev: start, markers located and interpolated, particles located and interpolated, spread
        if ev:
            ev[0].record(stream)
        sb.run_markers(stream)
        if ev:
            ev[1].record(stream)
        sb.run_particles(stream)
        if ev:
            ev[2].record(stream)
        f.zero_()
        ot.ot_spread(tree, ot.OT_PESKIN4, mode, mx, my, mz, Fm, f, workspace=ws)
        if ev:
            ev[3].record(stream)

    def time_steps(sb, k):
        evs_ = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(k)]
        for e in evs_:
            step(sb, e)
        torch.cuda.synchronize()
        mk = statistics.mean(e[0].elapsed_time(e[1]) for e in evs_)
        pt = statistics.mean(e[1].elapsed_time(e[2]) for e in evs_)
        sp = statistics.mean(e[2].elapsed_time(e[3]) for e in evs_)
        return {"step_ms": statistics.mean(e[0].elapsed_time(e[3]) for e in evs_), "locate_interpolate_ms": mk + pt,
                "markers_ms": mk, "particles_ms": pt, "spread_ms": sp}

    def warm(batch):
        for _ in range(max(3, args.warmup)):
            step(batch)
        torch.cuda.synchronize()

    if args.search == "auto":
        cal = {}
        for fname in ("plain", "learned"):
            bb = make_step(fname)
            warm(bb)
            cal[fname] = time_steps(bb, 3)["step_ms"]
            del bb
        chosen = min(cal, key=cal.get)
    else:
        chosen = "learned" if args.search == "learned" else "plain"
    batch = make_step(chosen)
    warm(batch)
    assert ot.ot_last_error(tree) & (ot.OT_DEV_STENCIL | ot.OT_DEV_OUTSIDE | ot.OT_DEV_REFINED_CAP) == 0
    ot.ot_index_get_stats(tree, reset=True)

    # timed region: the chosen form
    steps = args.steps if not light else max(3, min(args.steps, 10))
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(steps)]
    clocks = Clocks(local) if rank == 0 else None
    barrier()
    torch.cuda.synchronize()
    launches0 = ot.ot_launch_count()
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.nvtx.range_push("timed")
    start.record(stream)
    for k in range(steps):
        step(batch, evs[k])
    stop.record(stream)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    barrier()
    launches = ot.ot_launch_count() - launches0
    clk = clocks.stop() if clocks else None
    total_ms = max_over_ranks(start.elapsed_time(stop), dist, dev)
    ms_step = total_ms / steps
    markers_ms = statistics.mean(e[0].elapsed_time(e[1]) for e in evs)
    particles_ms = statistics.mean(e[1].elapsed_time(e[2]) for e in evs)
    spread_ms = statistics.mean(e[2].elapsed_time(e[3]) for e in evs)
    batch_ms = markers_ms + particles_ms
    value = job_value(npts, world, ms_step)
    fb = ot.ot_index_get_stats(tree, reset=True)["fallbacks"] if chosen == "learned" else None

    e2e = None
    if not args.no_e2e:
        e2e = measure_e2e(args, ctx, w, tree, field, forms_cfg[chosen], groups_for, step, batch,
                          (mx, my, mz), (px, py, pz), Fm, um, up, hm, hp, f, ws, mode, npts, light)

    mdf = bodies = None
    if not light:
        mdf, bodies = measure_extras(args, ctx, w, tree, field, (mx, my, mz), to_dev)

    # the other forms, same steps (the chosen form's level map is restored afterwards)
    forms = {chosen: {"step_ms": ms_step, "locate_interpolate_ms": batch_ms, "markers_ms": markers_ms,
                      "particles_ms": particles_ms, "spread_ms": spread_ms}}
    groups_t = {}
    del batch
    for fname in forms_cfg:
        if fname != chosen:
            bb = make_step(fname)
            warm(bb)
            forms[fname] = time_steps(bb, steps)
            del bb
        if light:
            continue
        # per-group timing (markers only, particles only) at the form's settings
        for gname, gsel in (("markers", groups[:1]), ("particles", groups[1:])):
            sv, lp = set_form(fname)
            bb = ot.ot_batch_create(tree, gsel, field, search=sv, launch=lp)
            for _ in range(2):
                ot.ot_batch_run(bb)
            a_, b_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a_.record(stream)
            for _ in range(5):
                ot.ot_batch_run(bb)
            b_.record(stream)
            torch.cuda.synchronize()
            groups_t[f"{gname}_{fname}_ms"] = a_.elapsed_time(b_) / 5
            del bb
    # informative, not `value`: the plain step with the particles stored in Morton order of
    # their level-8 cells (the order the tracking driver keeps them in; sorted once, untimed)
    morton = None
    if not light and not args.no_morton_form and n_p > 0 and forms_cfg["plain"][3]:
        set_form("plain")
        perm = ot.ot_points_morton_order(px, py, pz).long()
        sx, sy, sz = [a_.index_select(0, perm).contiguous() for a_ in (px, py, pz)]
        del perm
        up_m, hp_m = torch.empty_like(up), torch.empty_like(hp)
        gs = [groups[0], dict(kernel=ot.OT_TRILINEAR, x=sx, y=sy, z=sz, u=up_m, host=hp_m)]
        lp_m = ot.ot_batch_autotune(tree, gs, field, search=ot.OT_BINARY, tune_map_level=False, reps=2)["launch"]
        bb = StepBatches(ot, tree, gs, field, ot.OT_BINARY, lp_m)
        warm(bb)
        morton = time_steps(bb, steps)
        morton.update(points_per_s=npts / (morton["step_ms"] / 1e3),
                      locate_interpolate_points_per_s=npts / (morton["locate_interpolate_ms"] / 1e3), launch=lp_m,
                      map_level=forms_cfg["plain"][1], search="binary", level_mates="table",
                      particle_order="Morton order of level-8 cells")
        del bb, sx, sy, sz, gs, up_m, hp_m
    for fname, v_ in forms.items():
        v_["points_per_s"] = npts / (v_["step_ms"] / 1e3)
        v_["locate_interpolate_points_per_s"] = npts / (v_["locate_interpolate_ms"] / 1e3)
        v_["search"] = "learned" if forms_cfg[fname][0] == ot.OT_LEARNED else "binary"
        v_["map_level"] = forms_cfg[fname][1]
        v_["launch"] = forms_cfg[fname][2]
        v_["level_mates"] = "table" if forms_cfg[fname][3] else "searched per query"

    def ratio(a, b):
        return {"locate_interpolate": forms[a]["locate_interpolate_ms"] / forms[b]["locate_interpolate_ms"],
                "step": forms[a]["step_ms"] / forms[b]["step_ms"]}

    # the target: the learned batched form >= 1.5x the plain form, like for like (same level
    # map, table and launch shape); the autotuned pair and the whole-array comparisons are context
    same = ratio("plain", "learned_same_staging")
    learned_vs_plain = {"same_staging": same, "target": 1.5,
                        "target_met": bool(same["locate_interpolate"] >= 1.5),
                        "autotuned_forms": ratio("plain", "learned")}
    if "plain_nomap" in forms:
        learned_vs_plain["context_learned_vs_whole_array_binary"] = ratio("plain_nomap", "learned")
        learned_vs_plain["context_without_level_map"] = ratio("plain_nomap", "learned_nomap")
    if "plain_search" in forms:
        learned_vs_plain["context_table_vs_search_plain_step"] = forms["plain_search"]["step_ms"] / forms["plain"]["step_ms"]
    if morton:
        forms["plain_particles_morton"] = morton
    set_form(chosen)

    peak, peak_kind = measured_peaks()
    # the dominant kernel: the particles' graph replay (cell means of the field, value records,
    # trilinear launch), timed live on its stream in the timed region; the markers' graph beside
    alg_bytes = n_p * BYTES_PER_POINT + n_leaves * BYTES_PER_LEAF
    ms_dom = particles_ms if n_p else markers_ms
    achieved = alg_bytes / (ms_dom / 1e3) / 1e9
    all_bytes = npts * BYTES_PER_POINT + n_leaves * BYTES_PER_LEAF
    traffic, traffic_src = batch_traffic(w.name, chosen, forms_cfg[chosen][1], forms_cfg[chosen][3])
    roof = {"bound": "hbm", "kernel": "particles' graph replay (cell means, value records, trilinear launch): "
                                      "locate + interpolate of every particle",
            "achieved": achieved, "ms": ms_dom,
            "peak": peak, "unit": "GB/s", "frac": achieved / peak, "traffic": traffic, "traffic_source": traffic_src,
            "peak_kind": peak_kind, "algorithmic_bytes_per_launch": int(alg_bytes),
            "bytes_rule": f"{BYTES_PER_POINT} B/particle + {BYTES_PER_LEAF} B/leaf",
            "both_graphs": {"ms": batch_ms, "algorithmic_bytes": int(all_bytes),
                            "achieved": all_bytes / (batch_ms / 1e3) / 1e9,
                            "frac": all_bytes / (batch_ms / 1e3) / 1e9 / peak,
                            "what": "markers' and particles' graphs together, 40 B/point + 21 B/leaf"}}

    cpu = parity = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu, parity = parity_and_baseline(args, w, tree, field, forms_cfg, make_batch, groups_for, chosen,
                                          (mx, my, mz), (px, py, pz), Fm, dev, light)
        set_form(chosen)

    out = {"metric": METRIC, "value": value, "unit": "points/s", "n_gpus": world, "steps": steps,
           "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": dict(describe(w, n_leaves, INDEX_DESC[args.index] if chosen == "learned" else
                                   "plain: level map + subtree descriptors"),
                          form=chosen, map_level=forms_cfg[chosen][1], launch=forms_cfg[chosen][2],
                          level_mates="table" if forms_cfg[chosen][3] else "searched per query",
                          marker_order=("as generated (Fibonacci spiral per bubble)" if args.markers_as_generated
                                        else "per bubble, Morton order of level-10 cells"),
                          particle_order="as generated"),
           "roofline": roof, "cpu_baseline": cpu, "e2e": e2e,
           "gpu_launches": int(launches), "clocks": clk,
           "breakdown_ms": {"locate_interpolate": batch_ms, "markers": markers_ms, "particles": particles_ms,
                            "spread": spread_ms, "step": ms_step},
           "locate_interpolate_points_per_s": world * npts / (batch_ms / 1e3),
           "forms": forms, "learned_vs_plain": learned_vs_plain, "groups_ms": groups_t, "autotune": tune,
           "mdf": mdf, "body_momenta": bodies,
           "index": {"n_mid": n_mid, "n_leaf": n_leaf, "mean_window": istats["mean_window"],
                     "max_window": istats["max_window"], "empty_models": istats["empty_models"],
                     "fallbacks_timed": fb, "mean_probes": istats["mean_probes"],
                     "final_loss": istats["final_loss"], "train_s": train_s},
           "setup_s": {"octree_build": build_s, "index_train": train_s, "level_mate_table": mates_s},
           "parity": parity}
    return out


def measure_e2e(args, ctx, w, tree, field, form_cfg, groups_for, step, batch, M, P, Fm, um, up, hm, hp, f, ws, mode,
                npts, light):
    """The step through the public API with host buffers: every step uploads its marker and
    particle positions and marker forces from pinned host memory and downloads every point's
    velocity and host leaf and the spread force field.  Pinned buffers are first touched by a
    thread bound to the GPU's NUMA node.  Also the copy-only bandwidth of those transfers."""
    import torch
    import paper_2605_20565_gb300 as ot
    dist, world, dev, barrier, local = ctx["dist"], ctx["world"], ctx["dev"], ctx["barrier"], ctx["local"]
    stream = torch.cuda.current_stream()
    node, cpus = gpu_numa_cpus(local)
    old_aff = None
    if cpus:
        try:
            old_aff = os.sched_getaffinity(0)
            os.sched_setaffinity(0, cpus)
        except OSError:
            old_aff = None
    try:
        hmk = [torch.from_numpy(np.ascontiguousarray(w.markers[d])).pin_memory() for d in range(3)]
        hpt = [torch.from_numpy(np.ascontiguousarray(w.particles[d])).pin_memory() for d in range(3)]
        hF = torch.from_numpy(np.ascontiguousarray(w.forces, dtype=np.float32)).pin_memory()
    finally:
        if old_aff is not None:
            os.sched_setaffinity(0, old_aff)
    mx, my, mz = M
    px, py, pz = P
    n_m, n_p = mx.numel(), px.numel()
    n_leaves = f.shape[0]
    h2d = sum(t.numel() * t.element_size() for t in hmk + hpt + [hF])
    d2h = (um.numel() + up.numel() + f.numel()) * 4 + (hm.numel() + hp.numel()) * 4
    k_e2e = max(3, min(args.steps, 10))  # a few steps: one slow host-side step would skew fewer

    def outs_host():
        return (torch.empty((3, n_m), dtype=torch.float32).pin_memory(),
                torch.empty((3, n_p), dtype=torch.float32).pin_memory(),
                torch.empty(n_m, dtype=torch.int32).pin_memory(), torch.empty(n_p, dtype=torch.int32).pin_memory(),
                torch.empty((n_leaves, 4), dtype=torch.float32).pin_memory())

    h_um, h_up, h_hm, h_hp, h_f = outs_host()

    def upload(m_, p_, F_, s=None):
        for d in range(3):
            m_[d].copy_(hmk[d], non_blocking=True)
            p_[d].copy_(hpt[d], non_blocking=True)
        F_.copy_(hF, non_blocking=True)

    def download(dst, src):
        for a_, b_ in zip(dst, src):
            a_.copy_(b_, non_blocking=True)

    # copy-only bandwidth (no compute), each direction alone
    a_, b_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    upload((mx, my, mz), (px, py, pz), Fm)
    torch.cuda.synchronize()
    a_.record(stream)
    for _ in range(3):
        upload((mx, my, mz), (px, py, pz), Fm)
    b_.record(stream)
    torch.cuda.synchronize()
    h2d_gbs = 3 * h2d / (a_.elapsed_time(b_) / 1e3) / 1e9
    a_.record(stream)
    for _ in range(3):
        download((h_um, h_up, h_hm, h_hp, h_f), (um, up, hm, hp, f))
    b_.record(stream)
    torch.cuda.synchronize()
    d2h_gbs = 3 * d2h / (a_.elapsed_time(b_) / 1e3) / 1e9

    def e2e_step():
        upload((mx, my, mz), (px, py, pz), Fm)
        step(batch)
        download((h_um, h_up, h_hm, h_hp, h_f), (um, up, hm, hp, f))


    e2e_step()
    torch.cuda.synchronize()
    barrier()
    t0 = time.perf_counter()
    for _ in range(k_e2e):
        e2e_step()
    torch.cuda.synchronize()
    barrier()
    serial_ms = max_over_ranks(1e3 * (time.perf_counter() - t0) / k_e2e, dist, dev)

    # Pipelined: two slots of device buffers (each with its own batch graph); step k computes
    # on slot k % 2 while step k + 1's inputs go up and step k - 1's results come down on their
    # own streams.  Every step still copies all its inputs and results.
    class Slot:
        pass

    sv_, _, lp_, _ = form_cfg

    def make_slot(first):
        sl = Slot()
        if first:
            sl.m, sl.p, sl.F = (mx, my, mz), (px, py, pz), Fm
            sl.um, sl.up, sl.hm, sl.hp, sl.f, sl.ws, sl.batch = um, up, hm, hp, f, ws, batch
        else:
            sl.m = tuple(torch.empty_like(x_) for x_ in (mx, my, mz))
            sl.p = tuple(torch.empty_like(x_) for x_ in (px, py, pz))
            sl.F = torch.empty_like(Fm)
            sl.um, sl.up, sl.hm, sl.hp = (torch.empty_like(um), torch.empty_like(up), torch.empty_like(hm),
                                          torch.empty_like(hp))
            sl.f, sl.ws = torch.zeros_like(f), torch.empty_like(ws)
            sl.batch = StepBatches(ot, tree, groups_for(sl.m, sl.p, sl.um, sl.up, sl.hm, sl.hp), field, sv_, lp_)
        sl.h = outs_host()
        sl.ev_in, sl.ev_comp, sl.ev_out = (torch.cuda.Event(), torch.cuda.Event(), torch.cuda.Event())
        return sl

    slots = [make_slot(True), make_slot(False)]
    s_in, s_out = torch.cuda.Stream(), torch.cuda.Stream()

    def piped_step(k):
        sl = slots[k % 2]
        with torch.cuda.stream(s_in):
            s_in.wait_event(sl.ev_comp)  # the slot's previous step has read its inputs
            upload(sl.m, sl.p, sl.F)
            sl.ev_in.record(s_in)
        stream.wait_event(sl.ev_in)
        stream.wait_event(sl.ev_out)  # the slot's previous results are on the host
        sl.batch.run_markers(stream)
        sl.batch.run_particles(stream)
        sl.f.zero_()
        ot.ot_spread(tree, ot.OT_PESKIN4, mode, sl.m[0], sl.m[1], sl.m[2], sl.F, sl.f, workspace=sl.ws)
        sl.ev_comp.record(stream)
        with torch.cuda.stream(s_out):
            s_out.wait_event(sl.ev_comp)
            download(sl.h, (sl.um, sl.up, sl.hm, sl.hp, sl.f))
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
                and torch.equal(slots[0].hp, slots[1].hp) and torch.equal(slots[1].h[1], slots[1].up.cpu()))
    del slots
    copy_ms = 1e3 * (h2d / (h2d_gbs * 1e9) + d2h / (d2h_gbs * 1e9))
    return {"value": job_value(npts, world, e2e_ms), "unit": "points/s", "h2d_bytes_per_step": int(h2d),
            "d2h_bytes_per_step": int(d2h), "ms_per_step": e2e_ms, "steps": k_e2e,
            "pipeline": "2 slots; inputs up, compute, results down on three streams, overlapped across steps",
            "pipelined_results_identical": bool(piped_ok),
            "serial_ms_per_step": serial_ms, "serial_value": job_value(npts, world, serial_ms),
            "copy_only": {"h2d_gbs": h2d_gbs, "d2h_gbs": d2h_gbs, "ms_per_step_one_way_each": copy_ms,
                          "pinned_numa_node": node, "pinned_first_touch_cpus": len(cpus)}}


def measure_extras(args, ctx, w, tree, field, M, to_dev):
    """Multi-direct forcing (Sec. 2.2) and the bodies' internal-fluid momenta (Sec. 2.3)."""
    import torch
    import paper_2605_20565_gb300 as ot
    from paper_2605_20565_gb300 import synth
    dev = ctx["dev"]
    stream = torch.cuda.current_stream()
    mx, my, mz = M
    n_m = mx.numel()
    mdf = bodies = None
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
    if not args.no_mdf and w.extra and "centres" in w.extra:
        hmin = 2.0 ** -w.lmax
        Xi, st_i = synth.internal_markers(w.extra["centres"], w.extra["diameters"], hmin)
        xi, yi, zi = to_dev(Xi)
        d_start = torch.as_tensor(st_i, device=dev)
        xb = torch.as_tensor(np.ascontiguousarray(w.extra["centres"]), device=dev)
        ui = torch.empty((3, Xi.shape[1]), dtype=torch.float32, device=dev)
        wsi = torch.empty(max(1, ot.ot_interpolate_workspace_size(tree, ot.OT_TRILINEAR)), dtype=torch.uint8,
                          device=dev)

        def momenta():
            ot.ot_interpolate(tree, ot.OT_TRILINEAR, xi, yi, zi, field, u=ui, workspace=wsi)
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
    return mdf, bodies


def parity_and_baseline(args, w, tree, field, forms_cfg, make_batch, groups_for, chosen, M, P, Fm, dev, light):
    """The oracle against the timed launch on a bounded sample, for BOTH search forms, with
    one FP32 field (the workload's field at the oracle's leaf centres) fed to both sides;
    the octree leaf set compared whole; the timed CPU baseline."""
    import torch
    import oracle
    import paper_2605_20565_gb300 as ot
    ko, lo, setup_s = oracle_tree(w)
    kg, lg = ot.ot_octree_copy_leaves(tree)
    tree_exact = bool(np.array_equal(kg.cpu().numpy().view(np.uint64), ko) and np.array_equal(lg.cpu().numpy(), lo))
    del kg, lg
    f32 = synthetic_field32(w, ko, lo, dev)
    field.copy_(f32)  # the batches read `field`: every form now sees the synthetic FP32 field
    fref = f32.double().cpu().numpy()
    del f32
    fscale = float(np.abs(fref[:, :3]).max())
    n_ps, n_ms = size_cpu_sample(w, ko, lo, fref, args.cpu_seconds * (0.5 if light else 1.0))
    dt, host_ref, up_ref, um_ref = oracle_step(w, ko, lo, fref, n_ps, n_ms)
    cpu = {"value": (n_ps + n_ms) / dt, "unit": "points/s", "cores": oracle.num_threads(), "kind": "oracle",
           "sample": f"{n_ps} particles + {n_ms} markers of {w.name} (locate, interpolate, spread), "
                     f"one step, {dt:.1f} s; oracle tree build {setup_s:.1f} s untimed"}
    mhost_ref = oracle.locate_ub(ko, lo, *w.markers[:, :n_ms]) if n_ms else np.zeros(0, np.int32)
    mx, my, mz = M
    px, py, pz = P
    n_m, n_p = mx.numel(), px.numel()
    res, first = {}, None
    for fname in ("plain", "learned"):
        um_ = torch.empty((3, n_m), dtype=torch.float32, device=dev)
        up_ = torch.empty((3, n_p), dtype=torch.float32, device=dev)
        hm_ = torch.empty(n_m, dtype=torch.int32, device=dev)
        hp_ = torch.empty(n_p, dtype=torch.int32, device=dev)
        b = make_batch(fname, groups_for(M, P, um_, up_, hm_, hp_))
        ot.ot_batch_run(b)
        torch.cuda.synchronize()
        del b
        r = {"hosts_bit_exact": bool(np.array_equal(hp_[:n_ps].cpu().numpy(), host_ref) and
                                     np.array_equal(hm_[:n_ms].cpu().numpy(), mhost_ref)),
             "particles_max_rel_err": float(np.abs(up_[:, :n_ps].cpu().numpy() - up_ref).max() / fscale),
             "markers_max_rel_err": (float(np.abs(um_[:, :n_ms].cpu().numpy() - um_ref).max() / fscale)
                                     if n_ms else None)}
        if first is None:
            first = (up_, hp_, um_, hm_)
        else:  # every point of the full workload: the two forms give the same bits
            r["all_points_equal_plain_form"] = bool(torch.equal(up_, first[0]) and torch.equal(hp_, first[1]) and
                                                    torch.equal(um_, first[2]) and torch.equal(hm_, first[3]))
        res[fname] = r
        del um_, up_, hm_, hp_
    del first
    # spreading of the sampled markers against the oracle's
    spread = None
    if n_ms:
        fs = torch.zeros((tree_leaves(tree), 4), dtype=torch.float32, device=dev)
        ot.ot_spread(tree, ot.OT_PESKIN4, ot.OT_SORTED, mx[:n_ms].contiguous(), my[:n_ms].contiguous(),
                     mz[:n_ms].contiguous(), Fm[:, :n_ms].contiguous(), fs)
        f_ref, _ = oracle.spread_delta(ko, lo, w.lmax, 2, *w.markers[:, :n_ms], w.forces[:, :n_ms].astype(np.float64))
        spread = float(np.abs(fs[:, :3].cpu().numpy() - f_ref[:, :3]).max() / max(np.abs(f_ref[:, :3]).max(), 1e-300))
        del fs
    parity = {"octree_bit_exact": tree_exact, "forms": res, "spread_max_rel_err": spread,
              "sampled_points": n_ps + n_ms, "tolerance": 1e-5,
              "field": "the workload's field at the oracle's leaf centres in FP32, the same array on both sides",
              "all_ok": bool(tree_exact and all(v["hosts_bit_exact"] and v["particles_max_rel_err"] <= 1e-5 and
                                                (v["markers_max_rel_err"] or 0.0) <= 1e-5 and
                                                v.get("all_points_equal_plain_form", True) for v in res.values())
                             and (spread is None or spread <= 1e-5))}
    return cpu, parity


def tree_leaves(tree):
    import paper_2605_20565_gb300 as ot
    return ot.ot_octree_info(tree)[0]


def compact(d):
    """The fields of a secondary workload's line that the headline line carries."""
    keep = ("value", "unit", "ms_per_step", "steps", "config", "roofline", "cpu_baseline", "e2e", "parity",
            "learned_vs_plain", "breakdown_ms", "locate_interpolate_points_per_s", "gpu_launches", "clocks",
            "step_parts_ms", "rebuild")
    out = {k: d[k] for k in keep if k in d}
    if "forms" in d:
        out["forms"] = {k: {kk: v.get(kk) for kk in ("step_ms", "locate_interpolate_ms", "map_level", "search")}
                        for k, v in d["forms"].items()}
    return out


def run_ours(args):
    import torch
    from paper_2605_20565_gb300 import _build

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

    ctx = dict(dist=dist, world=world, rank=rank, local=local, dev=dev, barrier=barrier)
    t_run = time.time()
    out = measure(args, args.workload, False, ctx)
    print(f"[bench] {args.workload}: {time.time() - t_run:.1f} s", file=sys.stderr, flush=True)
    torch.cuda.empty_cache()
    # the other workloads, compact lines in the same run (rank 0 prints them with the headline)
    others = [] if (args.only or args.workload != "many_bubbles" or world > 1) else \
        [x for x in args.workloads.split(",") if x]
    if others:
        out["workloads"] = {}
        for name in others:
            t0 = time.time()
            try:
                if name == "tracking":
                    d = run_tracking(args, light=True, ctx=ctx)
                else:
                    d = measure(args, name, True, ctx)
                d = compact(d)
            except Exception as exc:  # a secondary workload never takes the headline line down
                d = {"error": f"{type(exc).__name__}: {exc}"}
            torch.cuda.empty_cache()
            d["wall_s"] = time.time() - t0
            print(f"[bench] {name}: {d['wall_s']:.1f} s", file=sys.stderr, flush=True)
            out["workloads"][name] = d
    if rank == 0:
        print(json.dumps(out), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def run_tracking(args, light=False, ctx=None):
    """The time-stepped workload: 256 bubbles moving, 200M particles advected by AB2, markers
    spread every step, octree rebuilt (and, for the learned form, the index retrained) every 10
    steps -- all inside the timed region.  Parity: the octree of the last re-adaptation against
    the oracle's octree of the same moved spheres, and the GPU's locate, interpolation, spreading
    and AB2 step on a sample of synthetic points against the oracle on the same inputs."""
    import torch
    import paper_2605_20565_gb300 as ot
    from paper_2605_20565_gb300 import _build, synth, tracking
    if ctx is None:
        torch.cuda.set_device(0)
        _build.build()
    dev = torch.device("cuda", torch.cuda.current_device())
    w = synth.tracking(n_particles=int(200_000_000 * args.scale))
    search = ot.OT_LEARNED if args.search == "learned" else ot.OT_BINARY
    t0 = time.time()
    launch = launch_of(args.launch)
    tr = tracking.Tracker(w, search=search, rebuild_every=10, mates=not args.no_mates, map_level=args.map_level,
                          launch=launch)
    setup_s = time.time() - t0
    n_leaves = ot.ot_octree_info(tr.tree)[0]
    for _ in range(args.warmup):
        tr.step()
    torch.cuda.synchronize()
    tr.timings = {"rebuild_s": 0.0, "rebuilds": 0}
    steps = args.tracking_steps
    clocks = Clocks(0)
    launches0 = ot.ot_launch_count()
    t0 = time.perf_counter()
    pts = 0
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(5)] for _ in range(steps)]
    torch.cuda.nvtx.range_push("timed")  # the steps a profiler's launch list should cover
    for k in range(steps):
        pts += tr.step(evs[k])
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    el = time.perf_counter() - t0
    launches = ot.ot_launch_count() - launches0
    parts = {name: statistics.mean(e[i].elapsed_time(e[i + 1]) for e in evs)
             for i, name in enumerate(("batch", "advect", "spread", "markers"))}
    clk = clocks.stop()
    ms_step = 1e3 * el / steps
    n_p, n_m = tr.x.shape[1], tr.mx.shape[1]
    # e2e: the state stays on the device; each step a host reads the step's results a coupled
    # solver needs -- the marker velocities and the spread force field -- from pinned memory
    h_um = torch.empty_like(tr.um, device="cpu").pin_memory()
    # the leaf count changes at every re-adaptation: a host buffer with room to spare
    h_f = torch.empty((n_leaves + n_leaves // 5 + 1024, 4), dtype=torch.float32).pin_memory()
    k_e2e = 10
    d2h = 0
    t0 = time.perf_counter()
    for _ in range(k_e2e):
        tr.step()
        nl = tr.f.shape[0]
        h_um.copy_(tr.um, non_blocking=True)
        h_f[:nl].copy_(tr.f, non_blocking=True)
        d2h += h_um.numel() * 4 + nl * 16
    torch.cuda.synchronize()
    e2e_ms = 1e3 * (time.perf_counter() - t0) / k_e2e
    e2e = {"value": (n_p + n_m) / (e2e_ms / 1e3), "unit": "points/s", "h2d_bytes_per_step": 0,
           "d2h_bytes_per_step": int(d2h / k_e2e), "ms_per_step": e2e_ms, "steps": k_e2e,
           "what": "state resident on the device (uploaded once); marker velocities and force field read back "
                   "every step; re-adaptations inside"}
    peak, peak_kind = measured_peaks()
    # algorithmic bytes of one step: locate+interpolate (40 B/point + 21 B/leaf), AB2 (read x,
    # v, a_prev, v_prev, u: 72 B; write x, v, a_prev, v_prev: 60 B per particle), spreading
    # (position and force 36 B per marker in; the force field zeroed and accumulated, 16 B per
    # leaf)
    step_bytes = (n_p + n_m) * BYTES_PER_POINT + n_leaves * BYTES_PER_LEAF + n_p * 132 + n_m * 36 + n_leaves * 16
    achieved = step_bytes / (ms_step / 1e3) / 1e9
    roof = {"bound": "hbm", "kernel": "whole tracking step (batch, AB2 advection, sorted spreading, marker "
                                      "motion; re-adaptations amortised)", "achieved": achieved, "peak": peak,
            "unit": "GB/s", "frac": achieved / peak, "traffic": None, "peak_kind": peak_kind,
            "algorithmic_bytes_per_step": int(step_bytes),
            "bytes_rule": "40 B/point + 21 B/leaf + 132 B/particle (AB2) + 36 B/marker + 16 B/leaf (spread)"}
    cpu = parity = None
    if not args.no_cpu_baseline:
        cpu, parity = tracking_parity(args, tr, w, dev, light)
    out = {"metric": METRIC, "value": pts / el, "unit": "points/s", "n_gpus": 1, "steps": steps,
           "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": w.name, "bubbles": int(w.spheres.shape[0]), "levels": [w.lmin, w.lmax],
                      "leaves": int(n_leaves), "markers_peskin4": int(n_m), "particles_trilinear": int(n_p),
                      "search": "learned" if search == ot.OT_LEARNED else "binary",
                      "level_mates": "searched per query" if args.no_mates else "table",
                      "map_level": ot.ot_octree_get_map_level(tr.tree),
                      "launch": tr.launch, "launch_autotuned": launch is None,
                      "step": "locate+interpolate all points, AB2 advect particles, sorted spread of markers; "
                              "octree rebuild (+ index retrain for the learned form) + field resample every 10 steps",
                      "l2": "inputs larger than L2; no flush"},
           "rebuild": {"rebuilds_timed": tr.timings["rebuilds"], "rebuild_s_timed": tr.timings["rebuild_s"],
                       "parts_s_timed": tr.timings.get("rebuild_parts_s"), "setup_s": setup_s},
           "step_parts_ms": parts, "gpu_launches": int(launches), "clocks": clk,
           "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "parity": parity}
    if ctx is None:
        print(json.dumps(out), flush=True)
    return out


def tracking_parity(args, tr, w, dev, light):
    """Oracle checks of the tracking workload's last re-adaptation on inputs that do not come
    from the CUDA path: the moved spheres (octree), synthetic points (locate + trilinear), the
    markers' rigidly moved positions (Peskin-4 interpolation and spreading), the workload's field
    at the oracle's leaf centres in FP32 (both sides), and an AB2 step from a synthetic state."""
    import torch
    import oracle
    import paper_2605_20565_gb300 as ot
    t0 = time.time()
    sph = tr.tree_spheres
    ko, lo = oracle.octree_build(sph, w.lmin, w.lmax)
    build_s = time.time() - t0
    kg, lg = ot.ot_octree_copy_leaves(tr.tree)
    tree_exact = bool(np.array_equal(kg.cpu().numpy().view(np.uint64), ko) and np.array_equal(lg.cpu().numpy(), lo))
    del kg, lg
    fld = synthetic_field32(w, ko, lo, dev)
    fref = fld.double().cpu().numpy()
    fscale = float(np.abs(fref[:, :3]).max())
    # sample: synthetic uniform points and the markers at the re-adaptation's time
    n_s = int(min(w.particles.shape[1], 2_000_000 if not light else 1_000_000))
    P = np.ascontiguousarray(w.particles[:, :n_s])
    Mk = tr.markers_at(tr.tree_time)
    n_ms = int(min(Mk.shape[1], 200_000))
    Mk = np.ascontiguousarray(Mk[:, :n_ms])
    Fk = np.ascontiguousarray(w.forces[:, :n_ms], dtype=np.float32)
    t1 = time.perf_counter()
    host_ref = oracle.locate_ub(ko, lo, *P)
    up_ref = oracle.interp_trilinear(ko, lo, fref, *P, host_ref)
    um_ref, _ = oracle.interp_delta(ko, lo, w.lmax, 2, fref, *Mk)
    f_ref, _ = oracle.spread_delta(ko, lo, w.lmax, 2, *Mk, Fk.astype(np.float64))
    st = {"x": P.copy(), "v": np.zeros_like(P), "a_prev": np.zeros_like(P), "v_prev": np.zeros_like(P)}
    oracle.advect_ab2(st, up_ref, tr.tau, tr.re_coef, tr.dt, True, periodic=True)
    cpu_s = time.perf_counter() - t1
    cpu = {"value": (n_s + n_ms) / cpu_s, "unit": "points/s", "cores": oracle.num_threads(), "kind": "oracle",
           "sample": f"{n_s} particles (locate, trilinear, AB2) + {n_ms} markers (Peskin-4 interpolation and "
                     f"spreading) on the {ko.size}-leaf octree of the last re-adaptation, {cpu_s:.1f} s; oracle "
                     f"octree build {build_s:.1f} s untimed"}
    x, y, z = [torch.as_tensor(P[d], device=dev) for d in range(3)]
    h = torch.empty(n_s, dtype=torch.int32, device=dev)
    u = ot.ot_interpolate(tr.tree, ot.OT_TRILINEAR, x, y, z, fld, host_out=h)
    mx_, my_, mz_ = [torch.as_tensor(Mk[d], device=dev) for d in range(3)]
    um = ot.ot_interpolate(tr.tree, ot.OT_PESKIN4, mx_, my_, mz_, fld)
    fs = torch.zeros_like(fld)
    ot.ot_spread(tr.tree, ot.OT_PESKIN4, ot.OT_SORTED, mx_, my_, mz_, torch.as_tensor(Fk, device=dev), fs)
    # one AB2 step from the same synthetic state with the oracle's velocities
    xs = torch.as_tensor(P, device=dev).contiguous()
    vs = torch.zeros((3, n_s), dtype=torch.float32, device=dev)
    a0, v0 = torch.zeros_like(vs), torch.zeros_like(vs)
    ot.ot_advect_ab2(xs, vs, a0, v0, torch.as_tensor(up_ref.astype(np.float32), device=dev), tr.tau, tr.re_coef,
                     tr.dt, first=True, periodic=True)
    torch.cuda.synchronize()
    dx = np.abs(xs.cpu().numpy() - st["x"])
    dx = np.minimum(dx, 1.0 - dx)
    vscale = max(float(np.abs(st["v"]).max()), 1e-30)
    parity = {"octree_bit_exact": tree_exact, "octree_leaves": int(ko.size),
              "hosts_bit_exact": bool(np.array_equal(h.cpu().numpy(), host_ref)),
              "particles_max_rel_err": float(np.abs(u.cpu().numpy() - up_ref).max() / fscale),
              "markers_max_rel_err": float(np.abs(um.cpu().numpy() - um_ref).max() / fscale),
              "spread_max_rel_err": float(np.abs(fs[:, :3].cpu().numpy() - f_ref[:, :3]).max() /
                                          max(np.abs(f_ref[:, :3]).max(), 1e-300)),
              "ab2_v_max_rel_err": float(np.abs(vs.cpu().numpy() - st["v"]).max() / vscale),
              "ab2_x_max_abs_err": float(dx.max()),
              "sampled_points": n_s + n_ms, "tolerance": 1e-5, "step_of_tree": tr.tree_step}
    parity["all_ok"] = bool(tree_exact and parity["hosts_bit_exact"] and parity["particles_max_rel_err"] <= 1e-5
                            and parity["markers_max_rel_err"] <= 1e-5 and parity["spread_max_rel_err"] <= 1e-5
                            and parity["ab2_v_max_rel_err"] <= 1e-5)
    return cpu, parity


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "tracking":
        run_tracking(args)
        return 0
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
