"""Launch-choice tuner for the GB300 path (rs_tuning).

    python -m paper_1110_4372_gb300.tune [--config c3] [--reps 3] [--sweeps 2] [--out FILE]

Coordinate descent over the launch choices of ``rs_tuning`` (resident
blocks of the two big-node search kernels, the big-node levels put in k-d
order, the size above which a big node's search is bracketed by a sample,
the size limits of the subtree tiers, and the persistent grid of every
tier), one choice at a time, keeping a candidate only when its median time
of ``rs_find_halos`` on the resident workload beats the best so far by more
than half a percent.  Every candidate's result is checked: its 3D labels and
halo ids must equal those of the library's defaults, or the tuner stops.
The chosen table, every trial and the machine are written to a JSON file.
"""
from __future__ import annotations

import argparse
import json
import statistics
import sys

# candidate values per choice (each inside the range rs_set_tuning accepts)
SPACE = {
    "link_blocks_per_sm": [4, 5, 6],
    "nn_blocks_per_sm": [5, 6, 7],
    "kd_levels": [1, 2, 3],
    "bracket_min": [2048, 4096, 8192, 16384],
    "mid_max": [128, 192, 256],
    "tiny_max": [16, 24, 32],
    "small_ctas_per_sm": [1, 2],
    "mid_ctas_per_sm": [4, 6, 8],
    "tiny_ctas_per_sm": [4, 8, 12, 16],
    "fof_link_ctas_per_sm": [8, 16, 32, 64],
}


def timed_call(rsgpu, ctx, pos, vel, box, halo, labels, reps):
    """Median CUDA-event time (ms) of rs_find_halos over reps calls, after
    one untimed call."""
    import torch
    rsgpu.rs_find_halos(ctx, pos, vel, box, fof_labels=labels, halo_id=halo)
    times = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        rsgpu.rs_find_halos(ctx, pos, vel, box, fof_labels=labels, halo_id=halo)
        e1.record()
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    return statistics.median(times)


def descend(base, space, measure, sweeps=2, log=print, margin=0.995):
    """Coordinate descent from the table `base` over `space` (choice -> its
    candidate values).  measure(table) returns (ms, same_result); a candidate
    becomes the best only when its time is below margin x the best so far, and
    a candidate whose result differs stops the descent.  A sweep that keeps no
    candidate ends it.  Returns (best table, its ms, base ms, trials)."""
    base_ms, same = measure(dict(base))
    if not same:
        raise RuntimeError("the starting table's result differs from the reference")
    best, best_ms = dict(base), base_ms
    trials = [{"tuning": dict(base), "ms": base_ms}]
    log(f"defaults: {base_ms:.2f} ms")
    for sweep in range(sweeps):
        improved = False
        for key, values in space.items():
            for v in values:
                if v == best[key]:
                    continue
                cand = dict(best, **{key: v})
                ms, same = measure(cand)
                trials.append({"tuning": cand, "ms": ms, "same_result": same})
                if not same:
                    raise RuntimeError(f"launch choice {key}={v} changed the result")
                log(f"sweep {sweep} {key}={v}: {ms:.2f} ms (best {best_ms:.2f})")
                if ms < best_ms * margin:
                    best, best_ms, improved = cand, ms, True
        if not improved:
            break
    return best, best_ms, base_ms, trials


def tune(rsgpu, ctx, pos, vel, box, reps=3, sweeps=2, log=print):
    """Coordinate descent from the library's defaults on the resident
    workload; every candidate's 3D labels and halo ids must equal those of
    the defaults.  Returns (best table, its ms, default ms, trials)."""
    import torch
    n = pos.shape[0]
    halo = torch.empty(n, dtype=torch.int32, device=pos.device)
    labels = torch.empty(n, dtype=torch.int32, device=pos.device)
    ref = {}

    def measure(table):
        rsgpu.rs_set_tuning(ctx, **table)
        ms = timed_call(rsgpu, ctx, pos, vel, box, halo, labels, reps)
        if not ref:
            ref["halo"], ref["labels"] = halo.clone(), labels.clone()
            return ms, True
        return ms, bool(torch.equal(halo, ref["halo"]) and torch.equal(labels, ref["labels"]))

    best, best_ms, base_ms, trials = descend(rsgpu.rs_tuning_default(), SPACE, measure, sweeps, log)
    rsgpu.rs_set_tuning(ctx, **best)
    return best, best_ms, base_ms, trials


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--config", default="c3")
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--sweeps", type=int, default=2)
    ap.add_argument("--out", default=None, help="JSON file for the table (default: print only)")
    args = ap.parse_args(argv)
    import torch
    from paper_1110_4372_gb300 import rsgpu, synth
    cat = synth.generate(args.config)
    ctx = rsgpu.Context()
    pos = torch.from_numpy(cat.pos).cuda()
    vel = torch.from_numpy(cat.vel).cuda()
    best, best_ms, base_ms, trials = tune(rsgpu, ctx, pos, vel, cat.box, args.reps, args.sweeps,
                                          log=lambda m: print(m, file=sys.stderr, flush=True))
    rec = {"device": torch.cuda.get_device_name(0), "workload": args.config, "particles": cat.n,
           "default": rsgpu.rs_tuning_default(), "default_ms": base_ms, "tuned": best, "tuned_ms": best_ms,
           "reps": args.reps, "trials": trials}
    text = json.dumps(rec, indent=1)
    if args.out:
        with open(args.out, "w") as fh:
            fh.write(text + "\n")
    print(json.dumps({k: rec[k] for k in ("device", "workload", "default_ms", "tuned_ms", "tuned")}))


if __name__ == "__main__":
    main()
