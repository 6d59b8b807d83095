"""Benchmark of the ROCKSTAR hot path on GB300: particles/s through 3D FOF,
the 6D phase-space hierarchy and seed assignment.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--config c3] [--impl ours|reference]

One step = rs_fof3d + rs_group_sort + rs_refine6d + rs_assign over one
synthetic catalogue resident in HBM.  With N > 1 (torchrun, one process per
GPU) every rank runs an independent replica of the workload ("replicas
only": the catalogue is not partitioned); value = all ranks' particles
divided by the slowest rank's time.  Prints one JSON line on rank 0.

``--impl reference`` times the float64 CPU oracle instead, on bounded
samples of the same workload (sub-cubes of the box), on rank 0 only.
"""
from __future__ import annotations

import argparse
import collections
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

from paper_1110_4372_gb300 import synth  # noqa: E402

WORKLOADS = {
    "c1": "32^3=32768 particles, L=10 Mpc/h, 40 NFW halos of 20-4000 particles (dN/dn ~ n^-1.9), uniform background",
    "c2": "128^3=2097152 particles, L=40 Mpc/h, 2500 NFW halos of 20-200k particles with 1-8 subhalos each",
    "c3": "512^3=134217728 particles, L=160 Mpc/h, 150k NFW halos of 20-10^6 particles, subhalos and "
          "sub-subhalos, uniform background; plain 3D FOF b=0.28, 6D refinement f=0.7, min 10 particles",
    "c5": "1024^3=1073741824 particles, L=320 Mpc/h, 1.2M NFW halos of 20-10^6 particles, subhalos and sub-subhalos",
    "c3q": "256^3=16777216 particles, L=80 Mpc/h, 18750 NFW halos of 20-10^6 particles with subhalos "
           "(the 134M workload at 1/8 of its volume; profiling size)",
}
METRIC = "particles/s through 3D FOF + 6D refinement at 134M particles; HBM roofline fraction"

# Algorithmic bytes per unit (the strict minimum each step moves): a 3D FOF
# particle reads 12 B of position and writes a 4 B label; a member of a node
# at one refinement level reads 24 B of position and velocity and writes a
# 4 B label; assignment reads 24 B and writes 4 B per grouped particle.
BYTES_FOF_PER_PARTICLE = 16
BYTES_LEVEL_PER_MEMBER = 28
BYTES_ASSIGN_PER_MEMBER = 28

# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) per unit, from
# one ncu capture of every launch of the kernel in one step of the 16.8M
# workload (profiles/k_bvh_link_c3q_full.md, profiles/k_bvh_nn_c3q_full.md),
# scaled to a step by the units processed.  An entry is dropped when its
# kernel changes.
NCU_TRAFFIC_PER_UNIT = {
    "rf_lvl_link": 325757952 / 8612074,
    "rf_lvl_nn": 241497088 / 8612074,
}

# Which units each kernel processes per step (for its algorithmic bytes).
KERNEL_UNITS = {
    "fof_link": ("particles", BYTES_FOF_PER_PARTICLE),
    "fof_keys": ("particles", BYTES_FOF_PER_PARTICLE),
    "rf_small_subtree": ("small_level_members", BYTES_LEVEL_PER_MEMBER),
    "rf_lvl_nn": ("big_level_members", BYTES_LEVEL_PER_MEMBER),
    "rf_lvl_link": ("big_level_members", BYTES_LEVEL_PER_MEMBER),
    "as_assign": ("members", BYTES_ASSIGN_PER_MEMBER),
}


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock and throttle-reason samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.tmp = None

    def start(self):
        try:
            self.tmp = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.dev}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.tmp,
                                         stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.tmp.flush()
        self.tmp.seek(0)
        rows = [r.split(",") for r in self.tmp.read().strip().splitlines() if r.strip()]
        os.unlink(self.tmp.name)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                smax.append(float(r[2]))
            except ValueError:
                continue
            for k, name in enumerate(names):
                if r[5 + k].lower() in ("active", "0x1", "1"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def cpu_model() -> str:
    """The host CPU's model name (lscpu), or the machine type."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    import platform
    return platform.machine()


def sub_cube(cat, frac_side: float):
    """Particles of the catalogue inside [0, box*frac_side)^3 (a bounded
    sample of the same workload for the CPU oracle)."""
    s = cat.box * frac_side
    m = np.all(cat.pos < s, axis=1)
    return cat.pos[m].copy(), cat.vel[m].copy()


def _oracle_init():
    import oracle  # noqa: F401  (loads the oracle library once per worker)


def _oracle_shard(task):
    """Worker: the oracle's refinement and assignment of one shard of whole
    3D groups (assignment never crosses a 3D group, so shards are
    independent).  Returns the shard's node count."""
    import oracle
    pos, vel, box, mem, off, nn_subset, nn_seed, n_total, nbar = task
    tree = oracle.refine(pos, vel, box, mem, off, 0.7, 10, sub_n=nn_subset, sub_seed=nn_seed)
    oracle.assign(tree, n_total, box, 360.0, nbar)
    return int(tree.n_nodes)


def make_oracle_pool(workers: int):
    """A spawn pool of oracle workers (spawn: safe after CUDA is initialised),
    or None for a single core."""
    if workers <= 1:
        return None
    import multiprocessing as mp
    pool = mp.get_context("spawn").Pool(workers, initializer=_oracle_init)
    pool.map(_oracle_init_probe, range(workers))
    return pool


def _oracle_init_probe(_):
    return 0


def time_oracle_sample(cat, frac_side: float, nn_subset: int = 0, nn_seed: int = 0, pool=None, workers: int = 1):
    """The oracle on the particles of a sub-cube of the workload: 3D FOF on
    one core, then the refinement and assignment of its groups, split over
    `workers` processes in shards of whole groups of about equal member
    count when a pool is given.  Returns (particles, seconds)."""
    import oracle
    pos, vel = sub_cube(cat, frac_side)
    # the linking length of the full catalogue
    l = oracle.linking_length(cat.n, cat.box, 0.28)
    nbar = cat.n / cat.box ** 3
    t0 = time.perf_counter()
    lab, _, _ = oracle.fof3d(pos, cat.box, l=l)
    mem, off = oracle.groups_from_labels(lab, 10)
    if pool is None or workers <= 1 or len(off) <= 2:
        tree = oracle.refine(pos, vel, cat.box, mem, off, 0.7, 10, sub_n=nn_subset, sub_seed=nn_seed)
        oracle.assign(tree, len(pos), cat.box, 360.0, nbar)
    else:
        G = len(off) - 1
        cuts = np.searchsorted(off, np.linspace(0, off[-1], workers + 1)[1:-1])
        bounds = np.unique(np.concatenate([[0], np.clip(cuts, 0, G), [G]]))
        tasks = [(pos, vel, cat.box, mem[off[a]:off[b]], (off[a:b + 1] - off[a]).astype(np.int64), nn_subset,
                  nn_seed, len(pos), nbar) for a, b in zip(bounds[:-1], bounds[1:]) if b > a]
        pool.map(_oracle_shard, tasks)
    return len(pos), time.perf_counter() - t0


def compare_fof(rsgpu, ctx, pos, box, dense_n, reps=3):
    """Sec. 3.1: the plain 3D FOF against the paper's accelerated variant,
    each called alone on the resident workload (one untimed call, then reps
    timed with CUDA events on the context's stream, which is torch's current
    stream)."""
    import torch
    labels = torch.empty(pos.shape[0], dtype=torch.int32, device=pos.device)
    calls = (("plain", lambda: rsgpu.rs_fof3d(ctx, pos, box, 0.28, labels=labels, want_groups=True)),
             ("accel", lambda: rsgpu.rs_fof3d_accel(ctx, pos, box, 0.28, dense_n, labels=labels)))
    out = {"dense_n": dense_n, "reps": reps}
    for name, call in calls:
        r = call()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            r = call()
        e1.record()
        torch.cuda.synchronize()
        out[name + "_ms"] = e0.elapsed_time(e1) / reps
        out[name + "_groups"] = r[1]
        if name == "accel":
            out["centres"] = r[2]
    return out


def sample_groups(sizes, n_sample: int, seed: int):
    """A seeded sample of group indices, ascending: the largest tenth of
    n_sample groups (by size) and the rest drawn at random without
    replacement.  Returns (indices, number taken by size)."""
    G = len(sizes)
    rng = np.random.default_rng(seed)
    k_big = min(G, max(1, n_sample // 10))
    big = np.argsort(sizes, kind="stable")[::-1][:k_big]
    rest = np.setdiff1d(np.arange(G), big)
    extra = rng.choice(rest, min(len(rest), max(0, n_sample - k_big)), replace=False)
    return np.sort(np.concatenate([big, extra]).astype(np.int64)), k_big


def compare_per_group(rsgpu, ctx, pos, vel, box, n_sample, seed=11104372, reps=3):
    """The batched refinement (every group of a level in the same launches)
    against the plain path of one rs_refine6d call per group, on the same
    groups: a seeded sample of n_sample groups of the workload whose tenth
    are its largest groups.  After one untimed call of each, every path is
    timed reps times with CUDA events on the context's stream and the median
    is reported.  The per-group CSR slices are built before the timed region;
    the plain path's time includes the host synchronisation that each
    rs_refine6d call makes (it returns host scalars), which is part of
    launching one call per group.  Both paths must produce the same node
    count, or no speedup is reported."""
    import torch
    p = rsgpu.params()
    labels, _, _ = rsgpu.rs_fof3d(ctx, pos, box, p.b)
    perm, offsets = rsgpu.rs_group_sort(ctx, labels, p.min_n)
    off = offsets.cpu().numpy()
    sizes = np.diff(off)
    G = len(sizes)
    pick, k_big = sample_groups(sizes, n_sample, seed)
    idx = np.concatenate([np.arange(off[g], off[g + 1]) for g in pick])
    sub_perm = perm[torch.from_numpy(idx).to(perm.device)].contiguous()
    sub_sizes = sizes[pick]
    sub_off = np.concatenate([[0], np.cumsum(sub_sizes)]).astype(np.int64)
    sub_off_t = torch.from_numpy(sub_off).to(perm.device)
    one = [(sub_perm[sub_off[k]:sub_off[k + 1]],
            torch.tensor([0, int(sub_sizes[k])], dtype=torch.int64, device=perm.device)) for k in range(len(pick))]

    def batched():
        t = rsgpu.rs_refine6d(ctx, pos, vel, box, sub_perm, sub_off_t, p.f, p.min_n)
        n_nodes = t.info().n_nodes
        t.free()
        return n_nodes

    def plain():
        n_nodes = 0
        for pg, og in one:
            t = rsgpu.rs_refine6d(ctx, pos, vel, box, pg, og, p.f, p.min_n)
            n_nodes += t.info().n_nodes
            t.free()
        return n_nodes

    out = {}
    for name, call in (("batched", batched), ("plain", plain)):
        call()
        torch.cuda.synchronize()
        times, nodes = [], None
        for _ in range(max(1, reps)):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            nodes = call()
            e1.record()
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
        out[name] = (statistics.median(times), times, nodes)
    (b_ms, b_all, nodes_b), (p_ms, p_all, nodes_p) = out["batched"], out["plain"]
    same = nodes_b == nodes_p
    return {"groups": int(len(pick)), "members": int(sub_off[-1]), "largest": int(sub_sizes.max()),
            "batched_ms": b_ms, "plain_per_group_ms": p_ms, "speedup": (p_ms / b_ms) if same else None,
            "batched_ms_all": [round(t, 2) for t in b_all], "plain_ms_all": [round(t, 2) for t in p_all],
            "nodes_batched": int(nodes_b), "nodes_plain": int(nodes_p), "same_nodes": bool(same), "reps": reps,
            "plain_includes": "one host synchronisation per rs_refine6d call",
            "sample": f"{len(pick)} of {G} groups (seed {seed}): the {k_big} largest and the rest at random"}


def time_halo_props(rsgpu, ctx, pos, vel, box, thetas=(0.04, 0.0)):
    """Sec. 3.3-3.5.1 and App. B after the hot path: rs_assign_ex (the halo
    table), rs_halo_props (centres, hosts) and rs_unbind at each theta,
    each timed once with CUDA events on the context's stream after one
    untimed call of the whole sequence."""
    import torch
    p = rsgpu.params()
    n = pos.shape[0]
    labels, _, _ = rsgpu.rs_fof3d(ctx, pos, box, p.b)
    perm, offsets = rsgpu.rs_group_sort(ctx, labels, p.min_n)
    tree = rsgpu.rs_refine6d(ctx, pos, vel, box, perm, offsets, p.f, p.min_n)
    gm = rsgpu.particle_gm(n / box ** 3)

    def timed(fn):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        r = fn()
        e1.record()
        torch.cuda.synchronize()
        return r, e0.elapsed_time(e1)

    out = {"gm": gm}
    for it in range(2):
        (hid, halos), t_as = timed(lambda: rsgpu.rs_assign_ex(ctx, tree, pos, vel, box, p))
        hp, t_hp = timed(lambda: rsgpu.rs_halo_props(ctx, tree, halos, hid))
        ub_t = {}
        for th in thetas:
            if it == 0 and th == 0.0:
                continue  # the direct sum is timed once
            ub, t_ub = timed(lambda: rsgpu.rs_unbind(ctx, tree, halos, hid, hp["host"], pos, vel, gm, 0.0, th))
            ub_t[th] = (t_ub, ub)
    npart = {th: int(u.get("n_part").sum()) for th, (_, u) in ub_t.items()}
    nbound = {th: int(u.get("n_bound").sum()) for th, (_, u) in ub_t.items()}
    sq = {th: float((u.get("n_part").double() ** 2).sum()) for th, (_, u) in ub_t.items()}
    out.update({"halos": halos.n, "assign_ex_ms": t_as, "halo_props_ms": t_hp,
                "unbind": {f"theta={th:g}": {"ms": t, "set_members": npart[th], "bound": nbound[th],
                                              "sum_set_size_sq": sq[th]} for th, (t, _) in ub_t.items()}})
    tree.free()
    return out


# ---- batching stress: independent groups streamed in chunks ----
def plan_chunks(sizes, chunk_particles, task_particles=20_000_000):
    """Chunks of whole consecutive groups with at most chunk_particles
    particles each (a larger group makes a chunk of its own), and inside
    every chunk the drawing tasks of about task_particles particles.
    Returns (chunks [(first, end)], tasks [(first, end)], chunk of each task)."""
    G = len(sizes)
    chunks, a, acc = [], 0, 0
    for g in range(G):
        if acc and acc + sizes[g] > chunk_particles:
            chunks.append((a, g))
            a, acc = g, 0
        acc += int(sizes[g])
    if G:
        chunks.append((a, G))
    tasks, task_chunk = [], []
    for k, (a, b) in enumerate(chunks):
        t0, acc = a, 0
        for g in range(a, b):
            acc += int(sizes[g])
            if acc >= task_particles or g == b - 1:
                tasks.append((t0, g + 1))
                task_chunk.append(k)
                t0, acc = g + 1, 0
    return chunks, tasks, task_chunk


def _draw_groups_to_shm(task):
    """Worker: draws groups first .. first+count-1 of the workload into a
    shared-memory block (pos then vel, float32) and returns its name."""
    from multiprocessing import shared_memory
    name, first, count = task
    g = synth.groups(name, first=first, count=count)
    shm = shared_memory.SharedMemory(create=True, size=max(1, 24 * g.n))
    buf = np.ndarray((2, g.n, 3), np.float32, buffer=shm.buf)
    buf[0] = g.pos
    buf[1] = g.vel
    shm.close()
    return shm.name, g.n


def stream_groups(args, rsgpu, ctx):
    """The batching-stress workload: every group of the independent-group
    recipe, drawn on the host cores (a spawn pool writing into shared memory)
    and refined on the GPU in chunks of whole groups, one rs_refine6d call
    per chunk with the chunk's group offsets (no 3D FOF).  Each chunk's host
    to device copy and refinement are timed with CUDA events; the per-group
    comparison runs on a seeded sample of the first chunk's groups."""
    import multiprocessing as mp
    from multiprocessing import shared_memory
    import torch
    name = args.config
    cfg = synth.GROUP_CONFIGS[name]
    G = min(args.groups or cfg["n_groups"], cfg["n_groups"])
    sizes = synth.group_sizes(name, first=0, count=G)
    chunks, spans, task_chunk = plan_chunks(sizes, args.chunk_particles)
    tasks = [(name, a, b - a) for a, b in spans]
    cap = int(max(sizes[a:b].sum() for a, b in chunks))
    dpos = torch.empty((cap, 3), dtype=torch.float32, device="cuda")
    dvel = torch.empty((cap, 3), dtype=torch.float32, device="cuda")
    hbuf = torch.empty((2, cap, 3), dtype=torch.float32, pin_memory=True)
    perm = torch.arange(cap, dtype=torch.int32, device="cuda")
    p = rsgpu.params()
    box = float(np.float32(synth.GROUP_BOX))
    workers = max(1, (os.cpu_count() or 2) - 1)
    refine_ms = copy_ms = 0.0
    n_nodes = n_levels = 0
    per_group = None
    done_particles = 0
    t_wall = time.perf_counter()
    ctx_mp = mp.get_context("spawn")
    with ctx_mp.Pool(workers) as pool:
        # at most two tasks per worker in flight, so the shared memory the
        # workers fill ahead of the GPU stays bounded
        pending = collections.deque()
        nxt = 0
        ti = 0
        for k, (a, b) in enumerate(chunks):
            m = 0
            while ti < len(tasks) and task_chunk[ti] == k:
                while nxt < len(tasks) and len(pending) < 2 * workers:
                    pending.append(pool.apply_async(_draw_groups_to_shm, (tasks[nxt],)))
                    nxt += 1
                shm_name, nt = pending.popleft().get()
                shm = shared_memory.SharedMemory(name=shm_name)
                src = np.ndarray((2, nt, 3), np.float32, buffer=shm.buf)
                hbuf[0, m:m + nt].numpy()[:] = src[0]
                hbuf[1, m:m + nt].numpy()[:] = src[1]
                del src
                shm.close()
                shm.unlink()
                m += nt
                ti += 1
            off = torch.from_numpy(np.concatenate([[0], np.cumsum(sizes[a:b])]).astype(np.int64)).cuda()
            e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
            e0.record()
            dpos[:m].copy_(hbuf[0, :m], non_blocking=True)
            dvel[:m].copy_(hbuf[1, :m], non_blocking=True)
            e1.record()
            tree = rsgpu.rs_refine6d(ctx, dpos[:m], dvel[:m], box, perm[:m], off, p.f, p.min_n)
            e2.record()
            torch.cuda.synchronize()
            info = tree.info()
            tree.free()
            copy_ms += e0.elapsed_time(e1)
            refine_ms += e1.elapsed_time(e2)
            n_nodes += info.n_nodes
            n_levels = max(n_levels, info.n_levels)
            done_particles += m
            if k == 0 and args.per_group > 0:
                per_group = compare_groups_sample(rsgpu, ctx, dpos[:m], dvel[:m], box, sizes[a:b], args.per_group)
    wall = time.perf_counter() - t_wall
    return {"groups": G, "particles": done_particles, "chunks": len(chunks), "chunk_particles_max": cap,
            "refine_ms": refine_ms, "copy_ms": copy_ms, "wall_s": wall, "n_nodes": n_nodes, "n_levels": n_levels,
            "generation": f"{workers} spawn workers drawing groups into shared memory, overlapped with the GPU",
            "per_group": per_group}


def compare_groups_sample(rsgpu, ctx, pos, vel, box, sizes, n_sample, seed=11104376, reps=3):
    """One rs_refine6d call over a seeded sample of groups (given by their
    sizes, back to back in pos/vel) against one call per group on the same
    groups; medians of reps CUDA-event timings, node counts must agree."""
    import torch
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    pick, k_big = sample_groups(sizes, n_sample, seed)
    idx = np.concatenate([np.arange(off[g], off[g + 1]) for g in pick]).astype(np.int32)
    sub_perm = torch.from_numpy(idx).cuda()
    sub_sizes = sizes[pick]
    sub_off = np.concatenate([[0], np.cumsum(sub_sizes)]).astype(np.int64)
    sub_off_t = torch.from_numpy(sub_off).cuda()
    one = [(sub_perm[sub_off[j]:sub_off[j + 1]],
            torch.tensor([0, int(sub_sizes[j])], dtype=torch.int64, device="cuda")) for j in range(len(pick))]
    p = rsgpu.params()

    def batched():
        t = rsgpu.rs_refine6d(ctx, pos, vel, box, sub_perm, sub_off_t, p.f, p.min_n)
        nn = t.info().n_nodes
        t.free()
        return nn

    def plain():
        nn = 0
        for pg, og in one:
            t = rsgpu.rs_refine6d(ctx, pos, vel, box, pg, og, p.f, p.min_n)
            nn += t.info().n_nodes
            t.free()
        return nn

    res = {}
    for label, call in (("batched", batched), ("plain", plain)):
        call()
        times = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record()
            nn = call()
            e1.record()
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
        res[label] = (statistics.median(times), nn)
    same = res["batched"][1] == res["plain"][1]
    return {"groups": int(len(pick)), "members": int(sub_off[-1]), "largest": int(sub_sizes.max()),
            "batched_ms": res["batched"][0], "plain_per_group_ms": res["plain"][0],
            "speedup": res["plain"][0] / res["batched"][0] if same else None, "same_nodes": bool(same),
            "nodes": int(res["batched"][1]), "reps": reps,
            "plain_includes": "one host synchronisation per rs_refine6d call",
            "sample": f"{len(pick)} of {len(sizes)} groups of the first chunk (seed {seed}): the {k_big} largest "
                      f"and the rest at random"}


def reference_arm(args, cat, cfg_json):
    """The oracle, as it stands, on host cores: each step one bounded sample,
    its groups' refinement spread over the cores."""
    side = args.ref_side
    workers = max(1, args.cpu_workers)
    pool = make_oracle_pool(workers)
    for _ in range(args.warmup):
        time_oracle_sample(cat, side, args.nn_subset, args.nn_seed, pool, workers)
    tot_p, tot_t = 0, 0.0
    for _ in range(args.steps):
        p, t = time_oracle_sample(cat, side, args.nn_subset, args.nn_seed, pool, workers)
        tot_p += p
        tot_t += t
    if pool:
        pool.close()
    v = tot_p / tot_t
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "particles/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": cfg_json,
            "cpu_baseline": {"value": v, "unit": "particles/s", "cores": workers, "kind": "oracle",
                             "host_cores": os.cpu_count(), "cpu_model": cpu_model(),
                             "sample": f"particles in the sub-cube [0, {side:g} L)^3 of the workload "
                                       f"({tot_p // max(args.steps, 1)} per step): 3D FOF on one core, then "
                                       f"refinement + assignment of its groups over {workers} processes, "
                                       f"float64 C oracle"},
            "e2e": {"value": v, "unit": "particles/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---- replicas on N GPUs (one process per GPU, launched by torchrun) ----
def replica_env():
    """(world size, rank, local rank) from the torchrun environment."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def init_replicas(world: int, local: int, backend: str = "nccl"):
    """Process group for the barrier and the max-over-ranks timing; None for
    a single process.  Replicas exchange nothing else: each runs the whole
    workload on its own GPU."""
    if world <= 1:
        return None
    import torch
    import torch.distributed as dist
    if backend == "nccl":
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        dist.init_process_group(backend)
    return dist


def max_over_ranks(x: float, dist, device: str = "cuda") -> float:
    """The largest value of x over all ranks (x itself without a group)."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: int, world: int, seconds: float) -> float:
    """Units all ranks processed divided by the slowest rank's time."""
    return world * units_per_rank / seconds


STRESS_METRIC = "particles/s through 6D refinement of independent co-spatial groups streamed in chunks"


def stress_main(args, world, rank, local):
    """--config c4 / c4s: the batching-stress workload streamed through
    rs_refine6d (one process; replicas run the same stream)."""
    import torch
    from paper_1110_4372_gb300 import rsgpu
    if args.impl == "reference":
        if rank == 0:
            print(json.dumps({"impl": "reference", "unavailable": "the batching-stress workload has no oracle "
                              "timing leg; its parity is tested on its small case"}))
        return
    torch.cuda.set_device(local)
    dist = init_replicas(world, local)
    ctx = rsgpu.Context()
    sampler = ClockSampler(local)
    sampler.start()
    r = stream_groups(args, rsgpu, ctx)
    clocks = sampler.stop()
    if rank != 0:
        return
    cfg = synth.GROUP_CONFIGS[args.config]
    v = r["particles"] / (r["refine_ms"] * 1e-3)
    e = r["particles"] / ((r["refine_ms"] + r["copy_ms"]) * 1e-3)
    line = {"metric": STRESS_METRIC, "value": v, "unit": "particles/s", "n_gpus": world, "steps": 1, "warmup": 0,
            "ms_per_step": r["refine_ms"], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"{r['groups']} independent groups of log-uniform size in [{cfg['nmin']}, "
                                   f"{cfg['nmax']}], NFW hosts with 0-{cfg['max_subs']} co-spatial subhalos "
                                   f"offset by 1-3 sigma in velocity", "name": args.config,
                       "f": 0.7, "min_n": 10, "chunk_particles": args.chunk_particles},
            "e2e": {"value": e, "unit": "particles/s", "h2d_bytes_per_step": 24 * r["particles"],
                    "d2h_bytes_per_step": 0, "note": "host-to-device copy of every chunk plus its refinement"},
            "clocks": clocks, "stream": r}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--config", default="c3", choices=sorted(WORKLOADS) + sorted(synth.GROUP_CONFIGS))
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--nn-subset", type=int, default=0,
                    help="nodes above this size take l from a random subset of this size (Sec. 3.2; 0: exact)")
    ap.add_argument("--nn-seed", type=int, default=11104372, help="seed of those subsets")
    ap.add_argument("--fof-accel", type=int, default=16, metavar="DENSE_N",
                    help="also time the plain 3D FOF against the accelerated variant (Sec. 3.1) alone "
                         "(negative: skip)")
    ap.add_argument("--per-group", type=int, default=2000, metavar="GROUPS",
                    help="also time the batched refinement against one rs_refine6d call per group on a sample "
                         "of this many groups (0: skip)")
    ap.add_argument("--halo-props", action="store_true",
                    help="also time rs_assign_ex, rs_halo_props and rs_unbind (tree and direct sum)")
    ap.add_argument("--groups", type=int, default=None,
                    help="batching-stress workloads (c4, c4s): refine only the first this many groups")
    ap.add_argument("--chunk-particles", type=float, default=1.0e9,
                    help="batching-stress workloads: particles per streamed chunk (whole groups)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-side", type=float, default=1.0 / 6.0, help="sub-cube side for the CPU baseline")
    ap.add_argument("--ref-side", type=float, default=1.0 / 8.0, help="sub-cube side per reference step")
    ap.add_argument("--cpu-workers", type=int, default=os.cpu_count() or 1,
                    help="host processes for the oracle's refinement of the sampled groups")
    args = ap.parse_args()

    world, rank, local = replica_env()
    if args.config in synth.GROUP_CONFIGS:
        return stress_main(args, world, rank, local)

    cfg = synth.CONFIGS[args.config]
    cfg_json = {"workload": WORKLOADS[args.config], "name": args.config, "particles": cfg["n"], "box": cfg["box"],
                "b": 0.28, "f": 0.7, "min_n": 10, "parallelism": "replicas" if world > 1 else "single",
                "l2": "inputs larger than L2 (pos+vel 24 B/particle)"}
    if args.nn_subset:
        cfg_json["nn_subset"] = args.nn_subset
        cfg_json["nn_seed"] = args.nn_seed

    if args.impl == "reference":
        if rank != 0:
            return
        cat = synth.generate(args.config)
        reference_arm(args, cat, cfg_json)
        return

    import torch
    from paper_1110_4372_gb300 import rsgpu

    torch.cuda.set_device(local)
    dist = init_replicas(world, local)

    cat = synth.generate(args.config)
    n = cat.n
    ctx = rsgpu.Context()
    pos = torch.from_numpy(cat.pos).cuda()
    vel = torch.from_numpy(cat.vel).cuda()
    halo = torch.empty(n, dtype=torch.int32, device="cuda")
    p = rsgpu.params(nn_subset=args.nn_subset, nn_seed=args.nn_seed)

    def step():
        _, _, st = rsgpu.rs_find_halos(ctx, pos, vel, cat.box, p, halo_id=halo)
        return st

    for _ in range(max(args.warmup, 0)):
        stats = step()
    torch.cuda.synchronize()

    sampler = ClockSampler(local)
    rsgpu.rs_profile_reset(ctx)
    rsgpu.rs_profile_enable(ctx, True)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    for _ in range(args.steps):
        stats = step()
    ev1.record()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = sampler.stop()
    rsgpu.rs_profile_enable(ctx, False)
    ms = ev0.elapsed_time(ev1) / args.steps
    prof = rsgpu.rs_profile_read(ctx)
    launches = rsgpu.rs_launch_count(ctx) // max(args.steps, 1)
    ms = max_over_ranks(ms, dist)
    value = whole_job_rate(n, world, ms * 1e-3)

    workspace_bytes = rsgpu.rs_workspace_bytes(ctx)

    # ---- the comparisons (rank 0), on the resident inputs ----
    fof_cmp = per_group = halo_props = None
    if rank == 0:
        if args.fof_accel >= 0:
            s = ClockSampler(local)
            s.start()
            fof_cmp = compare_fof(rsgpu, ctx, pos, cat.box, args.fof_accel)
            fof_cmp["clocks"] = s.stop()
        if args.per_group > 0:
            s = ClockSampler(local)
            s.start()
            per_group = compare_per_group(rsgpu, ctx, pos, vel, cat.box, args.per_group)
            per_group["clocks"] = s.stop()
        if args.halo_props:
            s = ClockSampler(local)
            s.start()
            halo_props = time_halo_props(rsgpu, ctx, pos, vel, cat.box)
            halo_props["clocks"] = s.stop()

    # ---- end to end through the C ABI with pinned host buffers ----
    # (the device-resident inputs are released first: this leg has its own
    # device copies inside the library's workspace)
    del pos, vel, halo
    torch.cuda.empty_cache()
    e2e = None
    if not args.no_e2e:
        hp = torch.from_numpy(cat.pos).pin_memory()
        hv = torch.from_numpy(cat.vel).pin_memory()
        hout = torch.empty(n, dtype=torch.int32).pin_memory()
        rsgpu.rs_find_halos(ctx, hp, hv, cat.box, p, halo_id=hout)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        k = max(1, min(args.steps, 3))
        esampler = ClockSampler(local)
        esampler.start()
        calls = []
        t0 = time.perf_counter()
        for _ in range(k):
            t1 = time.perf_counter()
            rsgpu.rs_find_halos(ctx, hp, hv, cat.box, p, halo_id=hout)
            calls.append(1e3 * (time.perf_counter() - t1))
        torch.cuda.synchronize()
        dt = max_over_ranks((time.perf_counter() - t0) / k, dist)
        eclocks = esampler.stop()
        # one more call with the copies bracketed by events (after the timed ones)
        rsgpu.rs_profile_reset(ctx)
        rsgpu.rs_profile_enable(ctx, True)
        rsgpu.rs_find_halos(ctx, hp, hv, cat.box, p, halo_id=hout)
        rsgpu.rs_profile_enable(ctx, False)
        io = {k: round(v[1], 2) for k, v in rsgpu.rs_profile_read(ctx).items() if k.startswith("io_")}
        e2e = {"value": whole_job_rate(n, world, dt), "unit": "particles/s", "h2d_bytes_per_step": 2 * 12 * n,
               "d2h_bytes_per_step": 4 * n, "ms_per_step": 1e3 * dt, "ms_per_call": [round(c, 1) for c in calls],
               "copy_ms_profiled_call": io, "clocks": eclocks}

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return

    # ---- roofline of the dominant kernel ----
    peaks, peak_kind = load_peaks()
    total_ms = sum(v[1] for v in prof.values())
    dom = max(prof.items(), key=lambda kv: kv[1][1])
    dom_name, (dom_launches, dom_ms) = dom
    units = {"particles": n, "members": stats["n_members"], "level_members": stats["sum_level_members"],
             "big_level_members": stats["sum_big_level_members"],
             "small_level_members": stats["sum_level_members"] - stats["sum_big_level_members"]}
    unit_name, per_unit = KERNEL_UNITS.get(dom_name, ("level_members", BYTES_LEVEL_PER_MEMBER))
    bytes_per_step = per_unit * units[unit_name]
    achieved = bytes_per_step * args.steps / (dom_ms * 1e-3) / 1e9
    peak = peaks["hbm_gbs"]
    traffic = None
    if dom_name in NCU_TRAFFIC_PER_UNIT:
        traffic = NCU_TRAFFIC_PER_UNIT[dom_name] * units[unit_name]
    roofline = {"kernel": dom_name, "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": traffic, "traffic_per": "step (all launches)",
                "peak_kind": f"{peak_kind} (hbm_gbs)",
                "algorithmic_bytes_per_step": bytes_per_step, "unit_per_step": f"{units[unit_name]} {unit_name}",
                "ms_per_step": dom_ms / args.steps, "share": dom_ms / total_ms if total_ms else None}
    b_alg = BYTES_FOF_PER_PARTICLE * n + BYTES_LEVEL_PER_MEMBER * stats["sum_level_members"]
    path_frac = b_alg / (ms * 1e-3) / 1e9 / peak

    cpu = None
    if not args.no_cpu_baseline:
        workers = max(1, args.cpu_workers)
        pool = make_oracle_pool(workers)
        npart, t = time_oracle_sample(cat, args.cpu_side, args.nn_subset, args.nn_seed, pool, workers)
        if pool:
            pool.close()
        cpu = {"value": npart / t, "unit": "particles/s", "cores": workers, "kind": "oracle",
               "host_cores": os.cpu_count(), "cpu_model": cpu_model(),
               "sample": f"{npart} particles in the sub-cube [0, {args.cpu_side:.4g} L)^3 of the workload: "
                         f"3D FOF on one core, then refinement + assignment of its groups over {workers} "
                         f"processes, float64 C oracle, {t:.1f} s"}

    stages = {}
    for k, (cnt, t) in prof.items():
        stage = k.split("_")[0]
        stages[stage] = stages.get(stage, 0.0) + t / args.steps
    line = {
        "metric": METRIC, "value": value, "unit": "particles/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": cfg_json,
        "e2e": e2e, "gpu_launches": launches * args.steps, "clocks": clocks, "roofline": roofline,
        "cpu_baseline": cpu,
        "path_hbm_frac": path_frac, "b_alg_bytes_per_step": b_alg,
        "stage_ms": {k: round(v, 3) for k, v in sorted(stages.items(), key=lambda kv: -kv[1])},
        "top_kernels_ms": {k: round(v[1] / args.steps, 3) for k, v in
                           sorted(prof.items(), key=lambda kv: -kv[1][1])[:8]},
        "stats": stats, "workspace_gb": round(workspace_bytes / 1e9, 2),
    }
    if fof_cmp is not None:
        line["fof3d_compare"] = fof_cmp
    if per_group is not None:
        line["refine_per_group_compare"] = per_group
    if halo_props is not None:
        line["halo_props_timing"] = halo_props
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
