"""Benchmark of the hemispherical ray-casting hot path on GB300.

One step = one pass of the whole path over one part: BVH build from the
device-resident mesh, area-weighted sampling, hemispherical cast,
directional variability + classification, orthogonal cast, reachability and
setups.  The default workload is the largest single-GPU configuration: the
impeller (hub r = 40 mm, 12 wrapped blades with a 35-degree twist and a
0.8 mm tip gap, ~1.93M triangles), 1,000,000 area-weighted points (seed 0),
2,048 Fibonacci hemisphere directions (2.05e9 rays), origin offset 1e-4 mm,
six-axis orthogonal cast.  The same line carries, under "prismatic", the
prismatic part (150x100x50 mm block with a T-slot, four 20-degree
through-holes and two side pockets, ~203k triangles, 100,000 points x 1,024
directions).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gpu|reference]

Prints one JSON line (rank 0).  ``value`` = occlusion rays cast per second
(hemispherical + orthogonal rays, whole job), timed with CUDA events per
step on the launching stream, L2 flushed (256 MB write) between steps.
``e2e`` = the same metric through ``rc_analyze_part`` with pinned host
buffers, host<->device copies inside the timed region.  ``--impl reference``
times the FP64 CPU oracle on the host cores instead.
Multi-GPU (torchrun): every rank analyses its own copy of the part (replicas;
the path has no exchange step), time = max over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "occlusion rays/s"
UNIT = "rays/s"
L2_FLUSH_BYTES = 256 << 20

WORKLOADS = {
    "prismatic": dict(desc="prismatic part 150x100x50 mm (T-slot, four 20-deg through-holes, two side "
                           "pockets), marching-tetrahedra mesh", n=100_000, n_dirs=1024),
    "pocket": dict(desc="pocket block 100x60x40 mm with a 30x30x15 mm centred pocket", n=1_000, n_dirs=256),
    "impeller": dict(desc="impeller, hub r=40 mm, 12 wrapped blades (35-deg twist, 0.8 mm tip gap)",
                     n=1_000_000, n_dirs=2048),
}


def make_mesh(name):
    import synth
    if name == "prismatic":
        return synth.prismatic()
    if name == "pocket":
        return synth.pocket_block(3)
    if name == "impeller":
        return synth.impeller()
    raise ValueError(name)


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("uuid,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid):
        self.uuid = uuid
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                                          "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, pw, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        rows = [[p.strip() for p in ln.split(",")] for ln in self.lines]
        rows = [r for r in rows if len(r) >= 9]
        mine = [r for r in rows if self.uuid and r[0].lower() == self.uuid.lower()]
        if not mine and len({r[0] for r in rows}) == 1:
            mine = rows
        for parts in mine:
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
                pw.append(float(parts[3]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm), "power_w_max": float(max(pw))}


# ---------------------------------------------------------------------------
# the oracle on the host cores (CPU baseline and the reference arm)
# ---------------------------------------------------------------------------

def oracle_rate(V, F, n_dirs, n_points, seed=0, mesh=None):
    """Time of the FP64 oracle (CPU BVH, all host cores) on the first
    n_points area-weighted points of the workload: (rays, build seconds,
    sampling seconds, cast seconds, cores).  With `mesh` the oracle's BVH is
    reused (build seconds 0)."""
    import oracle
    t0 = time.perf_counter()
    m = mesh if mesh is not None else oracle.Mesh(V, F)
    t1 = time.perf_counter()
    P, Nn, _, _ = oracle.sample_area(V, F, n_points, seed=seed)
    t2 = time.perf_counter()
    m.hemisphere(P, Nn, n_dirs)
    t3 = time.perf_counter()
    return n_points * n_dirs, t1 - t0, t2 - t1, t3 - t2, oracle.num_cores()


def cpu_baseline(V, F, n_dirs, n_points, target_s=12.0):
    """The oracle on a bounded sample of the workload: its first points (the
    sampler draws every point independently from its own counters, so the
    first k are a uniform random subset), as many as about target_s seconds
    of cast take, all of them if fewer.  The rate is the whole workload's
    rays over the oracle's time for it extrapolated from the sample: one
    BVH build plus sampling and cast scaled by n_points / k."""
    import oracle
    oracle.build()
    t0 = time.perf_counter()
    mesh = oracle.Mesh(V, F)
    t_build = time.perf_counter() - t0
    probe = min(500, n_points)
    _, _, _, tc, _ = oracle_rate(V, F, n_dirs, probe, mesh=mesh)
    pts = int(max(probe, min(n_points, probe * target_s / max(tc, 1e-3))))
    rays, _, ts, tc, cores = oracle_rate(V, F, n_dirs, pts, mesh=mesh)
    scale = n_points / pts
    t_full = t_build + (ts + tc) * scale
    kind = "all" if pts == n_points else "a %.1f%% subset" % (100.0 * pts / n_points)
    return {"value": n_points * n_dirs / t_full, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "first %d of the workload's %d area-weighted points (%s) x %d directions (%d rays): CPU BVH "
                      "build %.2f s + sampling %.2f s + cast %.1f s, FP64, all host cores; rate = the workload's "
                      "%d rays over build + (sampling + cast) x %.2f"
                      % (pts, n_points, kind, n_dirs, rays, t_build, ts, tc, n_points * n_dirs, scale)}


def run_reference(args, wl, V, F):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle
    oracle.build()
    n_dirs = wl["n_dirs"]
    rays, tb, ts, tc, cores = oracle_rate(V, F, n_dirs, 200)
    per_step_s = max(1.0, min(10.0, 150.0 / max(1, args.steps + args.warmup)))
    pts = int(max(200, min(wl["n"], 200 * max(0.2, per_step_s - tb) / max(ts + tc, 1e-3))))
    for _ in range(args.warmup):
        oracle_rate(V, F, n_dirs, pts)
    tot_r = tot_t = 0.0
    for _ in range(args.steps):
        r, tb, ts, tc, cores = oracle_rate(V, F, n_dirs, pts)
        tot_r += r
        tot_t += tb + ts + tc
    value = tot_r / tot_t
    sample = ("per step: CPU BVH build + %d of the workload's %d points x %d directions (%d rays), FP64 oracle"
              % (pts, wl["n"], n_dirs, pts * n_dirs))
    out = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_t / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload + ": " + wl["desc"], "tris": int(len(F)), "points": wl["n"],
                   "dirs": n_dirs, "sampled_points_per_step": pts},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out), flush=True)


# ---------------------------------------------------------------------------
# the GPU arm
# ---------------------------------------------------------------------------

def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


# the kernel, the tree it walks and the direction tile order it casts
TRAVERSAL_SOURCES = ("cast.cu", "build.cu", "rc_internal.cuh", "api.cu")


def _code_only(text):
    """C/C++ source without comments, trailing blanks and empty lines (string
    and character literals are kept), so that editing a comment does not
    change the hash of the code."""
    out, i, n = [], 0, len(text)
    while i < n:
        c = text[i]
        if c in "\"'":
            j = i + 1
            while j < n and text[j] != c:
                j += 2 if text[j] == "\\" else 1
            out.append(text[i:j + 1])
            i = j + 1
        elif text.startswith("//", i):
            j = text.find("\n", i)
            i = n if j < 0 else j
        elif text.startswith("/*", i):
            j = text.find("*/", i + 2)
            i = n if j < 0 else j + 2
        else:
            out.append(c)
            i += 1
    lines = [ln.rstrip() for ln in "".join(out).split("\n")]
    return "\n".join(ln for ln in lines if ln)


def traversal_hash():
    """sha256 over the code (comments removed) of the sources that define the
    traversal kernel and the tree layout it walks."""
    h = hashlib.sha256()
    for f in TRAVERSAL_SOURCES:
        h.update(_code_only(open(os.path.join(ROOT, "paper_2609_05467_gb300", "csrc", f)).read()).encode())
    return h.hexdigest()


def committed_profile(workload):
    """Per-ray figures of the traversal kernel from the committed ncu summary
    of this workload (profiles/k_hemisphere_<workload>_ncu.md), if it was
    taken on the current sources (sha256 of their code matches); else a
    note saying why there are none."""
    path = os.path.join(ROOT, "profiles", "k_hemisphere_%s_ncu.md" % workload)
    try:
        txt = open(path).read()
    except OSError:
        return {"source": "no committed ncu summary"}
    m = re.search(r"kernel source sha256:\s*([0-9a-f]{64})", txt)
    if not m:
        return {"source": "ncu summary without a source hash"}
    if m.group(1) != traversal_hash():
        return {"source": "stale ncu summary (kernel sources changed since)"}
    out = {"source": "ncu, profiles/k_hemisphere_%s_ncu.md" % workload}
    for key in ("dram_bytes_per_ray", "l2_bytes_per_ray", "l1_bytes_per_ray", "issue_active", "lanes_per_inst",
                "warp_inst_per_ray"):
        b = re.search(r"%s:\s*([0-9.eE+-]+)" % key, txt)
        out[key] = float(b.group(1)) if b else None
    return out


def job_totals(seconds, units, device):
    """Whole-job figures of replicas: the slowest rank's time and the sum of
    the units all ranks processed (the path has no exchange step, so this is
    the only collective)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([seconds], dtype=torch.float64, device=device)
    u = torch.tensor([units], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def run_gpu(args, name, wl, V, F, cpu=True):
    """The GPU arm on one workload; returns rank 0's JSON object (None on
    the other ranks)."""
    import torch
    import paper_2609_05467_gb300 as rc

    ws, rank, local = dist_env()
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    n, N = wl["n"], wl["n_dirs"]
    W = (N + 31) // 32
    p = rc.rc_params_default(n_dirs=N, seed=rank, tool_length=60.0, always_setups=1)

    Vh = torch.from_numpy(V).pin_memory()
    Fh = torch.from_numpy(F).pin_memory()
    Vd = Vh.to(dev)
    Fd = Fh.to(dev)
    P = torch.empty((n, 3), dtype=torch.float32, device=dev)
    Nn = torch.empty((n, 3), dtype=torch.float32, device=dev)
    face = torch.empty(n, dtype=torch.int32, device=dev)
    bits = torch.empty((n, W), dtype=torch.int32, device=dev)
    cnt = torch.empty(n, dtype=torch.int32, device=dev)
    mask = torch.empty(n, dtype=torch.uint8, device=dev)
    trav = torch.empty((n, 6), dtype=torch.float32, device=dev)
    cls = torch.empty(n, dtype=torch.uint8, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    total_steps = args.warmup + args.steps
    ctr = torch.zeros((total_steps, 2, 4), dtype=torch.int64, device=dev)

    side = torch.cuda.Stream(device=dev)

    def step(k, ev):
        h = rc.rc_build_bvh(Vd, Fd, stream)
        rc.rc_sample_points(h, n, p, P, Nn, face, None, stream)
        ev[0].record(stream)
        rc.rc_hemisphere_cast(h, P, Nn, p, bits, cnt, ctr[k, 0], stream)
        ev[1].record(stream)
        # the orthogonal cast needs only the points: as in rc_analyze_part it
        # runs on a side stream beside the hemispherical cast, issued after
        # it so that the persistent kernel holds the SMs first and the
        # orthogonal cast fills them as it drains
        side.wait_event(ev[0])
        rc.rc_orthogonal_cast(h, P, Nn, p, mask, trav, ctr[k, 1], side)
        ev[2].record(side)
        s = rc.rc_direction_variability(bits, Nn, p, stream=stream)
        label = rc.rc_classify(s, p)
        stream.wait_event(ev[2])
        su = rc.rc_min_setups(h, mask, trav, face, p, cls, stream)
        rc.rc_destroy_bvh(h)
        return s, label, su

    # instrumented traversal (outside any timed region): algorithmic bytes per ray
    h = rc.rc_build_bvh(Vd, Fd, stream)
    info = rc.rc_bvh_get_info(h)
    rc.rc_sample_points(h, n, p, P, Nn, face, None, stream)
    st = torch.zeros(8, dtype=torch.int64, device=dev)
    ps = rc.rc_params_default(n_dirs=N, seed=rank, collect_stats=1)
    rc.rc_hemisphere_cast(h, P, Nn, ps, bits, cnt, st, stream)
    st = st.cpu().numpy()
    rc.rc_destroy_bvh(h)
    rays_cast = float(st[0])
    nodes_per_ray = st[4] / rays_cast
    tris_per_ray = st[5] / rays_cast
    # a 4-wide node fetch reads 7 float4 (four child boxes + child indices),
    # a binary node 4 float4; a triangle record 3 float4
    node_bytes = 64.0 if ps.tree_width == 2 else 112.0
    bytes_per_ray = node_bytes * nodes_per_ray + 48.0 * tris_per_ray + 24.0 / N + 1.0 / 8.0

    # warm-up
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(5)] for _ in range(total_steps)]
    for k in range(args.warmup):
        step(k, evs[k][2:])
    torch.cuda.synchronize()

    props = torch.cuda.get_device_properties(dev)
    uuid = str(getattr(props, "uuid", "") or "")
    if uuid and not uuid.startswith("GPU-"):
        uuid = "GPU-" + uuid
    sampler = ClockSampler(uuid)
    sampler.start()
    time.sleep(0.3)
    launches0 = rc.rc_launch_count()
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    wall0 = time.perf_counter()
    step_ms, cast_ms = [], []
    for k in range(args.warmup, total_steps):
        flush.zero_()                       # L2 flush, outside the step's events
        e = evs[k]
        e[0].record(stream)
        s, label, su = step(k, e[2:])
        e[1].record(stream)
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    wall = time.perf_counter() - wall0
    launches = rc.rc_launch_count() - launches0
    clocks = sampler.stop()
    for k in range(args.warmup, total_steps):
        step_ms.append(evs[k][0].elapsed_time(evs[k][1]))
        cast_ms.append(evs[k][2].elapsed_time(evs[k][3]))
    c = ctr.cpu().numpy()
    rays_per_step = c[args.warmup:, 0, 0] + c[args.warmup:, 1, 0]
    errors = int(c[:, :, 3].sum())
    amb_rays = int(c[args.warmup:, 0, 1].sum() + c[args.warmup:, 1, 1].sum())
    retests = int(c[args.warmup:, 0, 2].sum() + c[args.warmup:, 1, 2].sum())
    t_dev = sum(step_ms) / 1e3
    rays_total = float(rays_per_step.sum())
    if ws > 1:
        t_dev, rays_total = job_totals(t_dev, rays_total, dev)
    value = rays_total / t_dev

    # end to end through rc_analyze_part with pinned host buffers
    hb = torch.empty((n, W), dtype=torch.int32).pin_memory()
    hc = torch.empty(n, dtype=torch.int32).pin_memory()
    hm = torch.empty(n, dtype=torch.uint8).pin_memory()
    hk = torch.empty(n, dtype=torch.uint8).pin_memory()
    for _ in range(0 if args.no_e2e else min(2, args.warmup)):
        rc.rc_analyze_part(Vh, Fh, n, p, hb, hc, hm, hk, stream)
    e2e_steps = 0 if args.no_e2e else max(1, min(args.steps, 20))
    e2e_t, e2e_rays = 0.0, 0.0
    for _ in range(e2e_steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = rc.rc_analyze_part(Vh, Fh, n, p, hb, hc, hm, hk, stream)
        e2e_t += time.perf_counter() - t0
        e2e_rays += r.cast_counters[0] + r.ortho_counters[0]
    if ws > 1:
        e2e_t, e2e_rays = job_totals(e2e_t, e2e_rays, dev)
    h2d = V.nbytes + F.nbytes
    d2h = hb.numel() * 4 + hc.numel() * 4 + hm.numel() + hk.numel() + 2 * 1024

    # roofline of the dominant kernel (the traversal)
    cast_s = float(np.mean(cast_ms)) / 1e3
    rays_cast_step = float(np.mean(c[args.warmup:, 0, 0]))
    roof = roofline(rc, args, name, dev, stream, ps, cast_s, rays_cast_step, nodes_per_ray, tris_per_ray,
                    bytes_per_ray, node_bytes)

    if rank != 0:
        return None
    cpu_line = None
    if cpu and ws == 1 and not args.no_cpu_baseline:
        cpu_line = cpu_baseline(V, F, N, n)
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * t_dev / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": name + ": " + wl["desc"], "tris": int(len(F)), "points": n,
                   "dirs": N, "origin_offset_mm": 1e-4, "sampling": "area-weighted random, seed = rank",
                   "orthogonal": "6 axes, identity frame", "l2": "flushed between steps (256 MB write)",
                   "parallelism": "replicas" if ws > 1 else "single GPU"},
        "e2e": {"value": e2e_rays / e2e_t if e2e_t > 0 else None, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h), "steps": e2e_steps,
                "api": "rc_analyze_part (pinned host mesh in, bits/counts/masks/classes out)"},
        "gpu_launches": int(launches),
        "clocks": clocks,
        "roofline": roof,
        "quality": {"ambiguous_rays": amb_rays, "fp64_retests": retests, "errors": errors,
                    "rays_per_step": float(np.mean(rays_per_step)), "wall_s": wall,
                    "overall_access": s.overall_access, "label": label, "setups_exact": su.setups_exact,
                    "bvh_depth": info.max_depth},
    }
    if cpu_line is not None:
        out["cpu_baseline"] = cpu_line
    return out


def roofline(rc, args, name, dev, stream, ps, cast_s, rays, nodes_per_ray, tris_per_ray, bytes_per_ray,
             node_bytes):
    """Roofline of the traversal kernel (k_hemisphere), the dominant kernel.

    Its tree stays close to the SMs (in L1/L2: the ncu summaries show DRAM
    traffic of a few bytes per ray), so no bandwidth binds it: it is bound
    by instruction issue of a divergent, latency-bound walk.  The reported
    bound is therefore "alu": the algorithmic FP32 work of the walk (the
    node and triangle tests the instrumented traversal counts, at the
    operation counts of their formulas) per CUDA-event second, against the
    FP32 peak from unit counts and clocks (SMs x 128 FP32 lanes x 2 flop x
    maximum SM clock).  The same algorithmic bytes against the measured HBM
    copy bandwidth, the levels and issue figures of the committed ncu
    summary, and this run's probes are reported beside it."""
    import torch
    props = torch.cuda.get_device_properties(dev)
    sm_max = None
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            sm_max = float(json.load(f)["sm_max_mhz"])
    except (OSError, KeyError, ValueError):
        sm_max = 2070.0
    fp32_peak = props.multi_processor_count * 128 * 2 * sm_max * 1e6 / 1e12
    ops_per_ray = 18.0 * (4.0 if ps.tree_width != 2 else 2.0) * nodes_per_ray + 35.0 * tris_per_ray
    fp32_ach = ops_per_ray * rays / cast_s / 1e12
    hbm_peak, peak_src = peaks()
    alg_bytes = bytes_per_ray * rays
    hbm_ach = alg_bytes / cast_s / 1e9
    prof = committed_profile(name)
    traffic = prof["dram_bytes_per_ray"] * rays if prof.get("dram_bytes_per_ray") is not None else None
    # the ceilings of a traversal whose tree stays in L2: random node-sized
    # reads from a 64 MiB L2-resident buffer and FP32 FMA issue (the
    # library's probe kernels, run after the timed region)
    l2_gbs = rc.rc_probe_l2(64 << 20, 128, 256, stream)
    fp32_probe = rc.rc_probe_fp32(4096, stream)
    return {
        "bound": "alu", "achieved": fp32_ach, "peak": fp32_peak, "unit": "TFLOP/s", "frac": fp32_ach / fp32_peak,
        "traffic": traffic,
        "peak_source": "unit counts and clocks: %d SMs x 128 FP32 lanes x 2 flop x %.0f MHz"
                       % (props.multi_processor_count, sm_max),
        "kernel": "k_hemisphere", "kernel_ms": 1e3 * cast_s,
        "binding": "instruction issue of a divergent walk whose dependent fetch -> test -> stack chain is "
                   "latency-bound; no bandwidth binds (see levels)",
        "algorithmic": {"ops_per_ray": ops_per_ray, "bytes_per_ray": bytes_per_ray, "nodes_per_ray": nodes_per_ray,
                        "tris_per_ray": tris_per_ray, "node_bytes": node_bytes,
                        "tree": "4-wide" if ps.tree_width != 2 else "binary",
                        "ops_source": "18 per box test (6 FMA counted as 2 each, 5 min/max, 1 compare), 35 per "
                                      "triangle test (watertight formulas); counts from the instrumented walk"},
        "hbm": {"achieved": hbm_ach, "peak": hbm_peak, "unit": "GB/s", "frac": hbm_ach / hbm_peak,
                "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)" if peak_src == "measured" else peak_src,
                "note": "algorithmic bytes per second; served mostly by L1 and L2, so this can exceed 1"},
        "levels": prof,
        "probes": {"l2_random_128B_gbs": l2_gbs, "fp32_fma_tflops": fp32_probe,
                   "note": "rc_probe_l2 (random 128-byte records from a 64 MiB L2-resident buffer) and "
                           "rc_probe_fp32 (8 FMA chains per thread), measured in this run"},
    }


# ---------------------------------------------------------------------------
# served workload: Poisson arrivals through the server vs one at a time
# ---------------------------------------------------------------------------

def _area(V, F):
    P = V.astype(np.float64)
    c = np.cross(P[F[:, 1]] - P[F[:, 0]], P[F[:, 2]] - P[F[:, 0]])
    return 0.5 * float(np.linalg.norm(c, axis=1).sum())


def served_trace(duration_s, rate, seed=0, n_dirs=512):
    """Seeded request trace: Poisson arrivals; each request a part from one
    of the three families with a triangle count log-uniform in [5e3, 1e6]
    (drawn from a pool of generated parts), n = 2 points per mm^2; 30% are
    re-submissions of an earlier part with one feature moved by 1-5 mm (the
    pocket block keeps its triangle list -> refit; the others are re-meshed
    -> rebuild)."""
    import synth
    rng = np.random.default_rng(seed)
    pool = []
    targets = np.exp(np.linspace(np.log(5e3), np.log(1e6), 8))
    for fam in range(3):
        for t in targets:
            if fam == 0:
                lv = int(min(7, max(3, round(np.log(t / 28.0) / np.log(4)))))
                shift = float(rng.uniform(1, 5))
                base = synth.perturbed_part(lv, 0.0)
                moved = synth.perturbed_part(lv, shift)
            elif fam == 1:
                sc = float(rng.uniform(0.7, 1.3))
                h = 1.67 * sc * float(np.sqrt(203000.0 / t))       # T ~ 203k (1.67 sc / h)^2
                base = synth.prismatic(h=h, scale=sc)
                moved = synth.prismatic(h=h, scale=sc, size=(150.0, 100.0 + float(rng.uniform(1, 5)) / sc, 50.0))
            else:
                sc = float(rng.uniform(0.7, 1.3))
                h = 0.69 * sc * float(np.sqrt(1.93e6 / t))         # T ~ 1.93M (0.69 sc / h)^2
                base = synth.impeller(h=h, scale=sc)
                moved = synth.impeller(h=h, scale=sc, r_tip=70.0 + float(rng.uniform(1, 5)) / sc)
            pool.append((fam, base, moved))
    reqs, t, key = [], 0.0, 0
    while True:
        t += float(rng.exponential(1.0 / rate))
        if t >= duration_s:
            break
        if reqs and rng.uniform() < 0.3:
            prev = reqs[int(rng.integers(len(reqs)))]
            V, F = pool[prev["pool"]][2]
            reqs.append(dict(t=t, key=prev["key"], pool=prev["pool"], V=V, F=F, resub=True))
        else:
            k = int(rng.integers(len(pool)))
            V, F = pool[k][1]
            key += 1
            reqs.append(dict(t=t, key=key, pool=k, V=V, F=F, resub=False))
    for r in reqs:
        r["n"] = int(round(2.0 * _area(r["V"], r["F"])))
    return reqs


def run_served(args):
    import torch
    import paper_2609_05467_gb300 as rc
    rc.load()
    torch.cuda.set_device(0)
    reqs = served_trace(args.duration, args.rate)
    p = rc.rc_params_default(n_dirs=512, tool_length=60.0)
    ps = rc.rc_params_default(n_dirs=512, tool_length=60.0, launch_mode=0 if args.server_persistent else 1)

    def replay(submit, collect):
        import queue as _q
        import threading as _t
        out = [None] * len(reqs)
        done = _q.Queue()
        t0 = time.perf_counter()

        def feeder():
            for k, r in enumerate(reqs):
                dt = r["t"] - (time.perf_counter() - t0)
                if dt > 0:
                    time.sleep(dt)
                done.put((k, submit(r, t0)))
        th = _t.Thread(target=feeder)
        th.start()
        for _ in range(len(reqs)):
            k, h = done.get()
            out[k] = collect(h, reqs[k], t0)
        th.join()
        return out, time.perf_counter() - t0

    # continuous batching through the server
    srv = rc.rc_server_create(ps, slots=args.slots, hbm_budget_bytes=120 << 30, small_rays=int(args.small_rays),
                              incremental=int(args.incremental))
    lat_holder = {}

    def s_submit(r, t0):
        return rc.rc_server_submit(srv, r["key"], r["V"], r["F"], r["n"]), time.perf_counter()

    log = open(args.served_log, "w") if args.served_log else None

    def s_collect(h, r, t0):
        rid, tsub = h
        res = rc.rc_server_wait(srv, rid, timeout_s=600.0)
        if log:
            # one JSON line per request: its timeline on the server and what it cast
            log.write(json.dumps({
                "request": int(res.request_id), "part_key": int(res.part_key), "status": int(res.status),
                "slot": int(res.slot), "priority_level": int(res.priority_level), "rebuilt": int(res.rebuilt),
                "updated": int(res.updated), "arrival_s": float(r["t"]), "t_submit": res.t_submit,
                "t_admit": res.t_admit, "t_start": res.t_start, "t_end": res.t_end, "triangles": int(len(r["F"])),
                "points": int(r["n"]),
                "rays": int(res.result.cast_counters[0] + res.result.ortho_counters[0]),
                "ambiguous_rays": int(res.result.cast_counters[1] + res.result.ortho_counters[1]),
                "retests": int(res.result.cast_counters[2] + res.result.ortho_counters[2]),
                "resident_bytes": int(res.resident_bytes)}) + "\n")
        return dict(lat=res.t_end - res.t_submit, rays=res.result.cast_counters[0] + res.result.ortho_counters[0],
                    rebuilt=res.rebuilt, status=res.status, wait=res.t_start - res.t_submit,
                    level=res.priority_level, tris=len(r["F"]), n=r["n"], arrival=r["t"], updated=res.updated,
                    resub=r["resub"])
    # warm-up pass over a few requests (module load, tables, pools)
    for r in reqs[:3]:
        rc.rc_server_wait(srv, rc.rc_server_submit(srv, 10**9 + r["key"], r["V"], r["F"], r["n"]), 600.0)
    served, wall_s = replay(s_submit, s_collect)
    if log:
        log.close()
    stats = rc.rc_server_get_stats(srv)
    rc.rc_server_destroy(srv)

    # plain path: one request at a time, FIFO, no resident state
    import threading as _t
    lock = _t.Lock()

    def p_submit(r, t0):
        return time.perf_counter()

    def p_collect(tsub, r, t0):
        t_start = time.perf_counter()
        with lock:
            t_run = time.perf_counter()
            res = rc.rc_analyze_part(r["V"], r["F"], r["n"], p)
        t_end = time.perf_counter()
        return dict(lat=t_end - tsub, rays=res.cast_counters[0] + res.ortho_counters[0],
                    rebuilt=1, status=0, wait=t_run - tsub, level=0, tris=len(r["F"]), n=r["n"], arrival=r["t"],
                    resub=r["resub"])
    plain, wall_p = replay(p_submit, p_collect)

    def summ(x, wall):
        lat = np.array([d["lat"] for d in x]) * 1e3
        tr = np.array([d["tris"] for d in x])
        rays = float(sum(d["rays"] for d in x))
        out = {"p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
               "mean_ms": float(lat.mean()), "rays_per_s": rays / wall, "wall_s": wall,
               "failed": int(sum(d["status"] != 0 for d in x))}
        wait = np.array([d["wait"] for d in x]) * 1e3
        out["wait_p99_ms"] = float(np.percentile(wait, 99))
        out["service_p99_ms"] = float(np.percentile(lat - wait, 99))
        slow = np.argsort(-lat)[:6]
        out["slowest"] = [{"lat_ms": round(float(lat[k]), 2), "wait_ms": round(float(wait[k]), 2),
                           "tris": int(x[k]["tris"]), "points": int(x[k]["n"]), "level": int(x[k]["level"]),
                           "rebuilt": int(x[k]["rebuilt"]), "arrival_s": round(float(x[k]["arrival"]), 3)}
                          for k in slow]
        rs = np.array([bool(d["resub"]) for d in x])
        if rs.any():
            out["resubmissions"] = {"requests": int(rs.sum()), "p50_ms": float(np.percentile(lat[rs], 50)),
                                    "p99_ms": float(np.percentile(lat[rs], 99))}
        for name, lo, hi in (("lt_50k", 0, 5e4), ("100k_400k", 1e5, 4e5), ("gt_400k", 4e5, 1e12)):
            sel = lat[(tr >= lo) & (tr < hi)]
            if len(sel):
                out["tris_" + name] = {"requests": int(len(sel)), "p50_ms": float(np.percentile(sel, 50)),
                                       "p99_ms": float(np.percentile(sel, 99))}
        return out
    sv, pl = summ(served, wall_s), summ(plain, wall_p)
    tris = np.array([len(r["F"]) for r in reqs])
    out = {
        "metric": "served p99 part latency", "value": sv["p99_ms"], "unit": "ms", "higher_is_better": False,
        "n_gpus": 1, "steps": len(reqs), "warmup": 3, "ms_per_step": sv["mean_ms"], "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "served: Poisson arrivals %.0f/s for %.0f s, parts from three families, 5k-1M "
                               "triangles log-uniform (median %d), 512 directions, 2 points/mm^2, 30%% "
                               "re-submissions with a feature moved 1-5 mm" % (args.rate, args.duration,
                                                                              int(np.median(tris))),
                   "slots": args.slots, "hbm_budget_gb": 120, "small_rays": args.small_rays,
                   "server_cast": ("persistent grid" if args.server_persistent else "one warp per point (short blocks)")
                                  + ", small requests on high-priority streams",
                   "plain": "rc_analyze_part per request, FIFO, one at a time, persistent grid",
                   "incremental": "re-submissions with the same triangle list keep their points on their faces "
                                  "and cast only what the edit can change" if args.incremental else "off"},
        "served": sv, "plain_one_at_a_time": pl,
        "server_stats": {k: getattr(stats, k) for k in ("completed", "failed", "rejected", "evicted")},
        "refits": int(sum(1 for d in served if d["rebuilt"] == 0)),
        "incremental": bool(args.incremental),
        "incremental_updates": int(sum(1 for d in served if d.get("updated"))),
        "requests": len(reqs),
    }
    print(json.dumps(out), flush=True)


# ---------------------------------------------------------------------------
# batched workload: many parts in one graph-replayed launch
# ---------------------------------------------------------------------------

def run_batched(args):
    import torch
    import synth
    import paper_2609_05467_gb300 as rc
    rc.load()
    torch.cuda.set_device(0)
    rng = np.random.default_rng(0)
    N = 512
    parts = []
    for k in range(args.parts):
        fam = int(rng.integers(3))
        t = float(np.exp(rng.uniform(np.log(1e4), np.log(5e5))))
        V, F = synth.part_family(fam, t, rng)
        n = int(min(200_000, round(2.0 * _area(V, F))))
        parts.append((fam, V, F, n))
    stream = torch.cuda.current_stream()
    p = rc.rc_params_default(n_dirs=N, seed=0)
    items = []
    for fam, V, F, n in parts:
        bvh = rc.Bvh(torch.from_numpy(V).cuda(), torch.from_numpy(F).cuda())
        P = torch.empty((n, 3), dtype=torch.float32, device="cuda")
        Nn = torch.empty_like(P)
        f = torch.empty(n, dtype=torch.int32, device="cuda")
        rc.rc_sample_points(bvh.h, n, p, P, Nn, f)
        bits = torch.empty((n, (N + 31) // 32), dtype=torch.int32, device="cuda")
        cnt = torch.empty(n, dtype=torch.int32, device="cuda")
        ctr = torch.zeros(4, dtype=torch.int64, device="cuda")
        mask = torch.empty(n, dtype=torch.uint8, device="cuda")
        trav = torch.empty((n, 6), dtype=torch.float32, device="cuda")
        octr = torch.zeros(4, dtype=torch.int64, device="cuda")
        items.append(dict(bvh=bvh, P=P, N=Nn, face=f, bits=bits, cnt=cnt, ctr=ctr, n=n, mask=mask, trav=trav,
                          octr=octr))
    rays = float(sum(q["n"] for q in items) * N)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")

    def timed(fn, reps):
        ts = []
        for _ in range(reps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        return float(np.mean(ts))

    # one part at a time (the single-part entry point per part)
    def per_part():
        for q in items:
            rc.rc_hemisphere_cast(q["bvh"].h, q["P"], q["N"], p, q["bits"], q["cnt"], q["ctr"], stream)
    for _ in range(args.warmup):
        per_part()
    t_seq = timed(per_part, args.steps)
    # batched, autotuned, graph replay
    b = rc.rc_batch_create(p)
    for q in items:
        rc.rc_batch_add_part(b, q["bvh"].h, q["P"], q["N"], q["bits"], q["cnt"], q["ctr"])
    t0 = time.perf_counter()
    best = rc.rc_batch_autotune(b, repeats=1, stream=stream)
    tune_s = time.perf_counter() - t0
    for _ in range(args.warmup):
        rc.rc_batch_launch(b, stream)
    launches0 = rc.rc_launch_count()
    t_b = timed(lambda: rc.rc_batch_launch(b, stream), args.steps)
    launches = rc.rc_launch_count() - launches0
    c = torch.stack([q["ctr"] for q in items]).cpu().numpy()
    rc.rc_batch_destroy(b)

    # the whole path of Sections 3.1-3.3 per part (cast, reduction and label,
    # orthogonal cast, classes and covers), one part at a time through the
    # single-part entry points, against the same in one graph-replayed batch
    pw = rc.rc_params_default(n_dirs=N, seed=0, tool_length=60.0, blocks_per_sm=best.blocks_per_sm,
                              points_per_item=best.points_per_item, point_order=best.point_order,
                              tile_mode=best.tile_mode)
    whole_labels = []

    def whole_per_part():
        whole_labels.clear()
        for q in items:
            rc.rc_hemisphere_cast(q["bvh"].h, q["P"], q["N"], pw, q["bits"], q["cnt"], q["ctr"], stream)
            sm = rc.rc_direction_variability(q["bits"], q["N"], pw, stream=stream)
            lab = rc.rc_classify(sm, pw)
            rc.rc_orthogonal_cast(q["bvh"].h, q["P"], q["N"], pw, q["mask"], q["trav"], q["octr"], stream)
            su = rc.rc_min_setups(q["bvh"].h, q["mask"], q["trav"], q["face"], pw, None, stream)
            whole_labels.append((lab, su.setups_exact))
    for _ in range(args.warmup):
        whole_per_part()
    t_wseq = timed(whole_per_part, args.steps)
    bw = rc.rc_batch_create(pw)
    for q in items:
        rc.rc_batch_add_analysis(bw, q["bvh"].h, q["P"], q["N"], q["face"], q["bits"], q["cnt"])
    batch_labels = []

    def whole_batched():
        rc.rc_batch_launch(bw, stream)
        res = rc.rc_batch_results(bw, len(items))
        batch_labels[:] = [(r.label, r.setups.setups_exact) for r in res]
    for _ in range(args.warmup):
        whole_batched()
    wl0 = rc.rc_launch_count()
    t_wb = timed(whole_batched, args.steps)
    wl = rc.rc_launch_count() - wl0
    rc.rc_batch_destroy(bw)
    ortho_rays = float(sum(int(q["octr"][0].item()) for q in items))
    tris = [len(F) for _, _, F, _ in parts]
    out = {
        "metric": METRIC, "value": rays / (t_b / 1e3), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_b, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "batched: %d parts from the three families, %d-%d triangles (log-uniform 10k-500k), "
                               "2 points/mm^2 capped at 200k, 512 directions, one graph-replayed launch"
                               % (len(parts), min(tris), max(tris)),
                   "points": int(sum(q["n"] for q in items)), "rays_per_step": rays,
                   "l2": "flushed between steps (256 MB write)"},
        "one_part_at_a_time": {"value": rays / (t_seq / 1e3), "ms_per_step": t_seq, "launches_per_step": len(items)},
        "autotuned": {"blocks_per_sm": best.blocks_per_sm, "points_per_item": best.points_per_item,
                      "point_order": ["morton", "index"][best.point_order],
                      "tile_mode": ["coherent tiles", "index"][best.tile_mode], "tune_s": tune_s},
        "gpu_launches": int(launches),
        "quality": {"ambiguous_rays": int(c[:, 1].sum()), "errors": int(c[:, 3].sum())},
        "whole_path": {
            "what": "per part: hemispherical cast, reduction + label, orthogonal cast, classes + covers (results on "
                    "the host); hemispherical + orthogonal rays per second",
            "batched_graph": {"value": (rays + ortho_rays) / (t_wb / 1e3), "ms_per_step": t_wb,
                              "graph_launches_per_step": int(wl) // max(1, args.steps)},
            "one_part_at_a_time": {"value": (rays + ortho_rays) / (t_wseq / 1e3), "ms_per_step": t_wseq},
            "same_labels_and_setups": batch_labels == whole_labels,
        },
    }
    print(json.dumps(out), flush=True)
    for q in items:
        q["bvh"].close()


AUTOFRAME_ROTATION = (12.0, -7.0, 25.0)


def run_autoframe(args):
    """Automatic machining frame of the full prismatic part turned off its
    axes: one step = rc_frame_candidates + rc_frame_select (candidate frames,
    one orthogonal cast over all of them, classes and covers per frame)."""
    import torch
    import synth
    import paper_2609_05467_gb300 as rc
    rc.load()
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream()
    V0, F = synth.prismatic()
    V = synth.rotate(V0, synth.rotation(*AUTOFRAME_ROTATION))
    n = args.points if args.points > 0 else 100_000
    p = rc.rc_params_default(tool_length=60.0)
    bvh = rc.Bvh(torch.from_numpy(V).to(dev), torch.from_numpy(F).to(dev))
    P = torch.empty((n, 3), dtype=torch.float32, device=dev)
    Nn = torch.empty_like(P)
    face = torch.empty(n, dtype=torch.int32, device=dev)
    rc.rc_sample_points(bvh.h, n, p, P, Nn, face, None, stream)
    ctr = torch.zeros(4, dtype=torch.int64, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    for _ in range(args.warmup):
        fr = rc.rc_frame_candidates(bvh.h, p, stream)
        rc.rc_frame_select(bvh.h, P, Nn, face, p, fr, ctr, stream)
    torch.cuda.synchronize()
    uuid = str(getattr(torch.cuda.get_device_properties(0), "uuid", "") or "")
    if uuid and not uuid.startswith("GPU-"):
        uuid = "GPU-" + uuid
    clk = ClockSampler(uuid)
    clk.start()
    t_c, t_s, rays = [], [], []
    launches0 = rc.rc_launch_count()
    for _ in range(args.steps):
        flush.zero_()
        e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        e[0].record(stream)
        fr = rc.rc_frame_candidates(bvh.h, p, stream)
        e[1].record(stream)
        rc.rc_frame_select(bvh.h, P, Nn, face, p, fr, ctr, stream)
        e[2].record(stream)
        torch.cuda.synchronize()
        t_c.append(e[0].elapsed_time(e[1]))
        t_s.append(e[1].elapsed_time(e[2]))
        rays.append(int(ctr[0].item()))
    launches = rc.rc_launch_count() - launches0
    clocks = clk.stop()
    ms = float(np.mean(np.array(t_c) + np.array(t_s)))
    c = ctr.cpu().numpy()
    best = fr.best
    # instrumented copy of the same casts (outside the timed region): node
    # fetches and triangle tests per axis ray
    ps = rc.rc_params_default(tool_length=60.0, collect_stats=1)
    cs = torch.zeros(8, dtype=torch.int64, device=dev)
    rc.rc_frame_select(bvh.h, P, Nn, face, ps, rc.rc_frame_candidates(bvh.h, ps, stream), cs, stream)
    cs = cs.cpu().numpy()
    nodes_pr, tris_pr = cs[4] / max(cs[0], 1), cs[5] / max(cs[0], 1)
    bpr = 112.0 * nodes_pr + 48.0 * tris_pr + (24.0 + 1.0 + 24.0 / 6.0) / 6.0
    pk, pk_src = peaks()
    ach = bpr * float(np.mean(rays)) / (float(np.mean(t_s)) / 1e3) / 1e9
    out = {
        "metric": METRIC, "value": float(np.mean(rays)) / (ms / 1e3), "unit": UNIT, "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32 (FP64 moments, boxes and eligibility)",
        "data": "synthetic",
        "config": {"workload": "autoframe: prismatic part (%d triangles) turned by %s deg (x, y, z), %d area-"
                               "weighted points; candidate frames + one orthogonal cast over all candidates + "
                               "classes and covers per frame" % (len(F), AUTOFRAME_ROTATION, n),
                   "tris": int(len(F)), "points": n, "l2": "flushed between steps (256 MB write)"},
        "breakdown_ms": {"candidates": float(np.mean(t_c)), "select": float(np.mean(t_s))},
        "frames": [{"source": int(fr.source[k]), "box_axis": int(fr.box_axis[k]), "box_step": int(fr.box_step[k]),
                    "setups_exact": int(fr.setups[k].setups_exact),
                    "inaccessible_or_over": int(fr.setups[k].class_counts[1] + fr.setups[k].class_counts[2]),
                    "volume_mm3": float(fr.volume[k])} for k in range(fr.k)],
        "best": int(best), "axis_rays_per_step": float(np.mean(rays)),
        "quality": {"ambiguous_rays": int(c[1]), "fp64_retests": int(c[2]), "errors": int(c[3])},
        "gpu_launches": int(launches), "clocks": clocks,
        "roofline": {"bound": "hbm", "achieved": ach, "peak": pk, "unit": "GB/s",
                     "frac": ach / pk, "traffic": None, "peak_source": pk_src + " (MEASURED_PEAKS.json hbm_gbs)",
                     "kernel": "k_orthogonal_axis (all candidate frames in one launch)",
                     "kernel_ms": float(np.mean(t_s)),
                     "kernel_ms_note": "rc_frame_select as a whole (the cast is ~90% of it): achieved is a lower bound",
                     "bytes_per_ray": bpr, "nodes_per_ray": nodes_pr, "tris_per_ray": tris_pr},
    }
    if not args.no_cpu_baseline:
        import oracle
        from oracle import frames as ofr
        oracle.build()
        m = min(n, 20_000)
        Po, No, fo, _ = oracle.sample_area(V, F, m, seed=0)
        t0 = time.perf_counter()
        cands, evals, ob = ofr.auto_frame(V, F, Po, No, fo, 60.0)
        dt = time.perf_counter() - t0
        elig = 0
        for cnd in cands:
            ax = oracle.frame_axes(cnd["frame"]).astype(np.float64)
            elig += int((No.astype(np.float64) @ ax.T >= -oracle.PARALLEL_TOL).sum())
        out["cpu_baseline"] = {"value": elig / dt, "unit": UNIT, "cores": oracle.num_cores(), "kind": "oracle",
                               "sample": "the first %d of the workload's points: oracle candidates (numpy, one "
                                         "core) + FP64 orthogonal casts (all cores) + covers, %.1f s; chose "
                                         "candidate %d" % (m, dt, ob)}
    print(json.dumps(out), flush=True)
    bvh.close()


def run_facelevel(args):
    """The paper's face-level analysis of an STL file: the prismatic part
    written as binary STL, one point per face centroid, 150 directions,
    area-weighted score, orthogonal cast and setups -- rc_analyze_stl, file
    to result, each step."""
    import tempfile
    import struct
    import torch
    import synth
    import paper_2609_05467_gb300 as rc
    rc.load()
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    V, F = synth.prismatic()
    tmp = tempfile.mkdtemp(prefix="rc_stl_")
    path = os.path.join(tmp, "prismatic.stl")
    tri = V[F.astype(np.int64)].reshape(len(F), 9)
    rec = np.zeros(len(F), dtype=np.dtype([("n", "<f4", 3), ("v", "<f4", 9), ("a", "<u2")]))
    rec["v"] = tri
    with open(path, "wb") as f:
        f.write(b"prismatic part".ljust(80, b" "))
        f.write(struct.pack("<I", len(F)))
        f.write(rec.tobytes())
    N = 150
    p = rc.rc_params_default(n_dirs=N, sample_mode=rc.RC_SAMPLE_FACE_CENTROID, always_setups=1, tool_length=60.0)
    for _ in range(args.warmup):
        r = rc.rc_analyze_stl(path, 0, p, stream)
    torch.cuda.synchronize()
    uuid = str(getattr(torch.cuda.get_device_properties(0), "uuid", "") or "")
    if uuid and not uuid.startswith("GPU-"):
        uuid = "GPU-" + uuid
    clk = ClockSampler(uuid)
    clk.start()
    launches0 = rc.rc_launch_count()
    ev_ms, wall = [], []
    for _ in range(args.steps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        t0 = time.perf_counter()
        e0.record(stream)
        r = rc.rc_analyze_stl(path, 0, p, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        wall.append(time.perf_counter() - t0)
        ev_ms.append(e0.elapsed_time(e1))
    launches = rc.rc_launch_count() - launches0
    clocks = clk.stop()
    rays = float(r.cast_counters[0] + r.ortho_counters[0])
    out = {
        "metric": METRIC, "value": rays / (float(np.mean(ev_ms)) / 1e3), "unit": UNIT, "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": float(np.mean(ev_ms)), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "facelevel: prismatic part (%d triangles) as a binary STL file, one point per face "
                               "centroid (area-weighted score), %d directions, six-axis cast and setups; "
                               "rc_analyze_stl from the file each step" % (len(F), N),
                   "tris": int(len(F)), "points": int(len(F)), "dirs": N,
                   "l2": "not flushed: each step re-reads the file and rebuilds everything"},
        "e2e": {"value": rays / float(np.mean(wall)), "unit": UNIT, "file_bytes": os.path.getsize(path),
                "h2d_bytes_per_step": int(V.nbytes + F.nbytes), "d2h_bytes_per_step": 0,
                "api": "rc_analyze_stl (file read, merge, upload, build, cast, summary, setups)"},
        "summary": {"overall_access": r.summary.overall_access,
                    "overall_access_unweighted": r.summary.overall_access_unweighted,
                    "axis_share": list(r.summary.axis_share), "mean_conc": r.summary.mean_conc,
                    "label": ["3-axis", "multi-axis"][r.label], "setups_exact": r.setups.setups_exact,
                    "setups_greedy": r.setups.setups_greedy},
        "gpu_launches": int(launches), "clocks": clocks,
        "quality": {"ambiguous_rays": int(r.cast_counters[1] + r.ortho_counters[1]),
                    "errors": int(r.cast_counters[3] + r.ortho_counters[3])},
    }
    if not args.no_cpu_baseline:
        import oracle
        oracle.build()
        P, Nn, fc, w = oracle.sample_centroid(V, F)
        m = oracle.Mesh(V, F)
        k = 20000
        t0 = time.perf_counter()
        m.hemisphere(P[:k], Nn[:k], N)
        dt = time.perf_counter() - t0
        out["cpu_baseline"] = {"value": k * N / dt, "unit": UNIT, "cores": oracle.num_cores(), "kind": "oracle",
                               "sample": "the first %d face centroids x %d directions, FP64 CPU BVH cast, %.1f s"
                                         % (k, N, dt)}
    os.remove(path)
    os.rmdir(tmp)
    print(json.dumps(out), flush=True)


def run_incremental(args):
    """Re-analysis after an edit that keeps the triangle list: a local bump on
    an impeller blade (default; 200,000 points), or the pocket block refined
    to 458,752 triangles with its pocket deepened or moved (100,000 points);
    1,024 directions.  One step = changed faces + points kept on their faces
    + the update cast; compared with a full re-cast of the edited part at
    the same points."""
    import torch
    import synth
    import paper_2609_05467_gb300 as rc
    rc.load()
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream()
    if args.edit == "bump":
        V0, F = synth.impeller()
        # a 0.3 mm bump of 4 mm radius on a blade, mid-span
        r = np.hypot(V0[:, 0], V0[:, 1])
        c = V0[np.argmin(np.abs(r - 55.0) + np.abs(V0[:, 2] - 25.0))].astype(np.float64)
        V1 = synth.bump(V0, c, 4.0, 0.3, direction=(-c[1], c[0], 0.0))
        edit = "a 0.3 mm bump of 4 mm radius on a blade"
        name = "impeller (%d triangles)" % len(F)
        default_n = 200_000
    else:
        V0, F = synth.perturbed_part(7, 0.0)
        V1, _ = (synth.perturbed_part(7, 0.0, deepen_mm=2.0) if args.edit == "deepen" else synth.perturbed_part(7, 2.5))
        edit = "pocket 2 mm deeper" if args.edit == "deepen" else "pocket moved 2.5 mm"
        name = "pocket block refined to %d triangles" % len(F)
        default_n = 100_000
    n = args.points if args.points > 0 else default_n
    N = 1024
    p = rc.rc_params_default(n_dirs=N, seed=0)
    Vt0, Vt1, Ft = (torch.from_numpy(V0).to(dev), torch.from_numpy(V1).to(dev), torch.from_numpy(F).to(dev))
    b0, b1 = rc.Bvh(Vt0, Ft), rc.Bvh(Vt1, Ft)
    P0 = torch.empty((n, 3), dtype=torch.float32, device=dev)
    N0 = torch.empty_like(P0)
    f = torch.empty(n, dtype=torch.int32, device=dev)
    rc.rc_sample_points(b0.h, n, p, P0, N0, f, None, stream)
    W = (N + 31) // 32
    bits0 = torch.empty((n, W), dtype=torch.int32, device=dev)
    cnt0 = torch.empty(n, dtype=torch.int32, device=dev)
    rc.rc_hemisphere_cast(b0.h, P0, N0, p, bits0, cnt0, None, stream)
    P1, N1 = torch.empty_like(P0), torch.empty_like(P0)
    changed = torch.empty(len(F), dtype=torch.uint8, device=dev)
    bits, cnt = torch.empty_like(bits0), torch.empty_like(cnt0)
    fb, fc = torch.empty_like(bits0), torch.empty_like(cnt0)
    ctr = torch.zeros(4, dtype=torch.int64, device=dev)
    fctr = torch.zeros(4, dtype=torch.int64, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    def update():
        bits.copy_(bits0)
        cnt.copy_(cnt0)
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        nc, box = rc.rc_changed_faces(Vt0, Vt1, Ft, changed, stream)
        rc.rc_sample_points_on_faces(b1.h, p, f, P1, N1, stream)
        rc.rc_hemisphere_update(b1.h, P1, N1, f, changed, box, p, bits, cnt, ctr, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1), nc

    def full():
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        rc.rc_hemisphere_cast(b1.h, P1, N1, p, fb, fc, fctr, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)

    for _ in range(args.warmup):
        update()
        full()
    uuid = str(getattr(torch.cuda.get_device_properties(0), "uuid", "") or "")
    if uuid and not uuid.startswith("GPU-"):
        uuid = "GPU-" + uuid
    clk = ClockSampler(uuid)
    clk.start()
    launches0 = rc.rc_launch_count()
    tu, nc = zip(*[update() for _ in range(args.steps)])
    launches = rc.rc_launch_count() - launches0
    tf = [full() for _ in range(args.steps)]
    clocks = clk.stop()
    same = bool(torch.equal(bits, fb))
    c, fcn = ctr.cpu().numpy(), fctr.cpu().numpy()
    ms = float(np.mean(tu))
    out = {
        "metric": METRIC, "value": n * N / (ms / 1e3), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": "incremental: %s, %s (same triangle list, %d faces changed); %d points kept on "
                               "their faces x %d directions; value = rays of the full result per second of update"
                               % (name, edit, nc[0], n, N),
                   "tris": int(len(F)), "points": n, "dirs": N, "l2": "flushed between steps (256 MB write)"},
        "rays_cast_again": int(c[0]), "rays_total": n * N, "fraction_cast_again": float(c[0]) / (n * N),
        "full_recast_ms": float(np.mean(tf)), "speedup_vs_full_recast": float(np.mean(tf)) / ms,
        "same_bits_as_full_recast": same,
        "quality": {"ambiguous_rays": int(c[1]), "full_ambiguous_rays": int(fcn[1]), "errors": int(c[3])},
        "gpu_launches": int(launches), "clocks": clocks,
    }
    print(json.dumps(out), flush=True)
    b0.close()
    b1.close()


def run_tool(args):
    """Tool-aware accessibility of the prismatic part: 100,000 points, six
    axes, a 3 mm ball-end tool sampled by its axis ray and a ring of 8 rays
    (rc_tool_cast); the thin-ray orthogonal cast of the same points beside it."""
    import torch
    import synth
    import paper_2609_05467_gb300 as rc
    rc.load()
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream()
    V, F = synth.prismatic()
    n = args.points if args.points > 0 else 100_000
    radius, K = 3.0, 8
    p = rc.rc_params_default(tool_length=60.0)
    bvh = rc.Bvh(torch.from_numpy(V).to(dev), torch.from_numpy(F).to(dev))
    P = torch.empty((n, 3), dtype=torch.float32, device=dev)
    Nn = torch.empty_like(P)
    face = torch.empty(n, dtype=torch.int32, device=dev)
    rc.rc_sample_points(bvh.h, n, p, P, Nn, face, None, stream)
    mask = torch.empty(n, dtype=torch.uint8, device=dev)
    thin = torch.empty(n, dtype=torch.uint8, device=dev)
    trav = torch.empty((n, 6), dtype=torch.float32, device=dev)
    ctr = torch.zeros(4, dtype=torch.int64, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    def timed(fn):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)
    tool_fn = lambda: rc.rc_tool_cast(bvh.h, P, Nn, p, radius, K, mask, ctr, stream)
    thin_fn = lambda: rc.rc_orthogonal_cast(bvh.h, P, Nn, p, thin, trav, None, stream)
    for _ in range(args.warmup):
        tool_fn()
        thin_fn()
    launches0 = rc.rc_launch_count()
    tt = [timed(tool_fn) for _ in range(args.steps)]
    launches = rc.rc_launch_count() - launches0
    tn = [timed(thin_fn) for _ in range(args.steps)]
    c = ctr.cpu().numpy()
    m, t = mask.cpu().numpy(), thin.cpu().numpy()
    ms = float(np.mean(tt))
    out = {
        "metric": METRIC, "value": float(c[0]) / (ms / 1e3), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32 (FP64 ray origins)", "data": "synthetic",
        "config": {"workload": "tool: prismatic part (%d triangles), %d area-weighted points, six axes, ball-end "
                               "tool r = %.1f mm sampled by 1 + %d rays per axis" % (len(F), n, radius, K),
                   "tris": int(len(F)), "points": n, "l2": "flushed between steps (256 MB write)"},
        "rays_per_step": int(c[0]), "thin_ray_orthogonal_ms": float(np.mean(tn)),
        "axes_open_thin": int(np.unpackbits(t).sum()), "axes_open_tool": int(np.unpackbits(m).sum()),
        "tool_subset_of_thin": bool(((m & ~t) == 0).all()),
        "quality": {"ambiguous_rays": int(c[1]), "errors": int(c[3])}, "gpu_launches": int(launches),
    }
    print(json.dumps(out), flush=True)
    bvh.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=60)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--workload", default="impeller", choices=list(WORKLOADS) + ["served", "batched", "autoframe",
                                                                                 "facelevel", "incremental", "tool"])
    ap.add_argument("--no-extra", action="store_true",
                    help="default workload: skip the prismatic part's line under \"prismatic\"")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end leg (profiling runs)")
    ap.add_argument("--points", type=int, default=0, help="override the workload's point count (profiling runs)")
    ap.add_argument("--duration", type=float, default=60.0, help="served workload: seconds of arrivals")
    ap.add_argument("--rate", type=float, default=20.0, help="served workload: arrivals per second")
    ap.add_argument("--slots", type=int, default=4, help="served workload: server slots")
    ap.add_argument("--parts", type=int, default=64, help="batched workload: number of parts")
    ap.add_argument("--incremental", action="store_true", help="served workload: incremental re-analysis")
    ap.add_argument("--served-log", default="", help="served workload: write one JSON line per request here")
    ap.add_argument("--server-persistent", action="store_true",
                    help="served workload: the server's casts use the persistent grid (launch_mode 0)")
    ap.add_argument("--edit", default="bump", choices=["bump", "deepen", "shift"],
                    help="incremental workload: the edit")
    ap.add_argument("--small-rays", type=float, default=4e6,
                    help="served workload: rays up to which a request runs at the highest priority")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.workload == "served":
        run_served(args)
        return
    if args.workload == "batched":
        run_batched(args)
        return
    if args.workload == "autoframe":
        run_autoframe(args)
        return
    if args.workload == "facelevel":
        run_facelevel(args)
        return
    if args.workload == "incremental":
        run_incremental(args)
        return
    if args.workload == "tool":
        run_tool(args)
        return
    wl = dict(WORKLOADS[args.workload])
    if args.points > 0:
        wl["n"] = args.points
    V, F = make_mesh(args.workload)
    if args.impl == "reference":
        run_reference(args, wl, V, F)
        return
    import torch
    import paper_2609_05467_gb300 as rc
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1:
        torch.distributed.init_process_group("nccl")
    rc.load(build_if_missing=(rank == 0))
    if ws > 1:
        torch.distributed.barrier()
        rc.load()
    out = run_gpu(args, args.workload, wl, V, F)
    if args.workload == "impeller" and args.points == 0 and not args.no_extra:
        # the prismatic part (100k points x 1,024 directions) in the same run
        V2, F2 = make_mesh("prismatic")
        o2 = run_gpu(args, "prismatic", dict(WORKLOADS["prismatic"]), V2, F2, cpu=False)
        if out is not None:
            out["prismatic"] = {k: o2[k] for k in ("value", "unit", "ms_per_step", "config", "e2e", "quality")}
            out["prismatic"]["roofline"] = {k: o2["roofline"][k] for k in ("bound", "achieved", "peak", "unit", "frac",
                                                                           "kernel_ms", "hbm", "levels")}
    if out is not None:
        print(json.dumps(out), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
