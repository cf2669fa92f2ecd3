"""Autotuner of the transport's launch and scheduling parameters.

The parameters (rec_tuning: emission and march grids in blocks per SM, the
idle-lane count that triggers a march refill, the packets per march work
chunk, the super-tile side ordering the march queue) change only the speed of
lya_transport: its tallies and counters are identical for every valid setting.
The tuner times the transport of one fixed step (same inputs every trial) for
candidate settings by coordinate descent — one parameter at a time over its
candidates, the others held at the best so far, for a few rounds — and keeps
the fastest.  Results are stored per workload key (side, packets per cell,
precision form, batch or single box) in a JSON table that bench.py and users
apply with `apply_table`.

  python -m paper_2312_11448_gb300.tune --n 256 --packets 100000000 --out table.json
  python -m paper_2312_11448_gb300.tune --batch 64 --out table.json
"""
import json

import numpy as np
import os

FIELDS = ("emit_blocks_per_sm", "march_blocks_per_sm", "march_refill", "march_chunk", "tile", "march_halo")
CANDIDATES = {
    "emit_blocks_per_sm": (2, 3, 4, 5, 6),
    "march_blocks_per_sm": (2, 3, 4, 5),
    "march_refill": (2, 4, 8, 12, 16, 24),
    "march_chunk": (16, 32, 64, 128, 256),
    "tile": (8, 16, 32, 64),
    "march_halo": (0, 8, 16, 32, 64),
}
TABLE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuning_gb300.json")


def workload_key(n, packets, precision, batch=False):
    """Table key: box side, packets per cell rounded to a power of two, form, batch."""
    ppc = max(packets, 1) / float(n ** 3)
    p2 = 1
    while p2 * 2 <= ppc:
        p2 *= 2
    return f"n{n}-ppc{p2}-{precision}-{'batch' if batch else 'single'}"


def batch_key(n_boxes, precision):
    """Table key of the batched workload of n_boxes boxes."""
    return f"batch{n_boxes}-{precision}"


# Fields searched together: the region sweeps change which march grid is best
# (a smaller working set per sweep admits more resident blocks), so one field
# at a time would not leave the grid the plain march prefers.
JOINT = (("march_blocks_per_sm", "march_halo"),)


def coordinate_descent(start, cost, candidates=None, rounds=2, allowed=None, joint=JOINT):
    """Minimise cost(setting) over the candidate grid, one field (or one joint
    pair of fields, every combination) at a time.
    start: dict of FIELDS; allowed(field, value) -> bool filters candidates.
    Returns (best setting, best cost, list of (setting, cost) tried)."""
    cand = dict(CANDIDATES if candidates is None else candidates)
    best = dict(start)
    seen = {}

    def evaluate(s):
        key = tuple(s[f] for f in FIELDS)
        if key not in seen:
            seen[key] = cost(dict(s))
        return seen[key]

    def ok(f, v):
        return allowed is None or allowed(f, v)

    paired = {f for pair in joint for f in pair}
    best_cost = evaluate(best)
    for _ in range(rounds):
        improved = False
        # the joint pairs first: they decide which march variant runs, and the
        # other fields are then tuned for it
        for f1, f2 in joint:
            for v1 in cand.get(f1, (best[f1],)):
                for v2 in cand.get(f2, (best[f2],)):
                    if (v1, v2) == (best[f1], best[f2]) or not ok(f1, v1) or not ok(f2, v2):
                        continue
                    trial = dict(best, **{f1: v1, f2: v2})
                    c = evaluate(trial)
                    if c < best_cost:
                        best, best_cost, improved = trial, c, True
        for f in FIELDS:
            if f in paired:
                continue
            for v in cand.get(f, (best[f],)):
                if v == best[f] or not ok(f, v):
                    continue
                trial = dict(best, **{f: v})
                c = evaluate(trial)
                if c < best_cost:
                    best, best_cost, improved = trial, c, True
        if not improved:
            break
    log = [(dict(zip(FIELDS, k)), c) for k, c in seen.items()]
    return best, best_cost, log


def time_transport(obj, step, z, reps=3):
    """Milliseconds per lya_transport of the same step (CUDA events on the
    context stream, after one untimed call)."""
    import torch
    obj.transport(step, z)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(obj.stream)
    for _ in range(reps):
        obj.transport(step, z)
    e1.record(obj.stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def autotune(obj, step, z, reps=3, rounds=2, candidates=None):
    """Tune a Box or Batch in place for the transport of (step, z); returns
    (best setting, ms per transport, trial log).  The box's tallies change (the
    transport runs repeatedly); its x_e, T and velocities do not."""
    from .rec import RecError
    limits = {}

    def allowed(f, v):
        if f in limits:
            return v <= limits[f]
        return True

    start = obj.tuning()
    # the launch bounds cap the grids: probe the largest accepted values
    for f in ("emit_blocks_per_sm", "march_blocks_per_sm"):
        top = max(c for c in CANDIDATES[f])
        while top > 1:
            try:
                obj.set_tuning(**{f: top})
                break
            except RecError:
                top -= 1
        limits[f] = top
    obj.set_tuning(**start)

    def cost(s):
        try:
            obj.set_tuning(**s)
        except RecError:  # a combination the kernels do not accept (e.g. a grid above a variant's limit)
            return float("inf")
        return time_transport(obj, step, z, reps)

    best, ms, log = coordinate_descent(start, cost, candidates, rounds, allowed)
    obj.set_tuning(**best)
    return best, ms, log


def load_table(path=TABLE):
    if not os.path.exists(path):
        return {}
    with open(path) as f:
        return json.load(f)


def apply_table(obj, key, path=TABLE):
    """Set the tuning stored for `key`, if any; returns the setting or None."""
    entry = load_table(path).get(key)
    if not entry:
        return None
    # a stored grid above the kernels' current residency limit (the defaults
    # after rec_init are those limits) is clamped to it
    cur = obj.tuning()
    # fields the entry predates keep their current value
    setting = {f: entry["setting"].get(f, cur[f]) for f in FIELDS}
    for f in ("emit_blocks_per_sm", "march_blocks_per_sm"):
        setting[f] = min(setting[f], cur[f])
    obj.set_tuning(**setting)
    return setting


def main():
    import argparse
    import torch
    from .inputs import BoxConfig, make_box, z_schedule
    from .rec import Box
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--n", type=int, default=256)
    ap.add_argument("--packets", type=int, default=100_000_000)
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--prep", type=int, default=170, help="steps advanced before tuning (z schedule 1800->600, 400)")
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--out", default=None, help="JSON table to update (default: print only)")
    ap.add_argument("--batch", type=int, default=0,
                    help="tune the batched workload of this many boxes instead (z schedule 1600->700, 200)")
    ap.add_argument("--config", default=None,
                    help="a named single-box workload of inputs.CONFIGS (its fields, packets and z schedule) "
                         "instead of --n/--packets")
    ap.add_argument("--start-z", type=float, default=None,
                    help="start from the Saha state at the schedule node nearest this redshift, then --prep steps")
    ap.add_argument("--rounds", type=int, default=2, help="coordinate-descent rounds")
    a = ap.parse_args()
    if a.batch:
        from .inputs import batched_configs
        from .rec import Batch
        cfgs = batched_configs(7, a.batch)
        zs = z_schedule(1600.0, 700.0, 200)
        boxes = [(c.n, *make_box(c, seed=100 + i), c.n_packets) for i, c in enumerate(cfgs)]
        box = Batch(boxes, precision=a.precision, mixing="tally", seed=7, stream=torch.cuda.Stream())
        del boxes
        prep = min(a.prep, 60)
        key = batch_key(a.batch, a.precision)
    else:
        if a.config:
            from .inputs import CONFIGS
            cfg = CONFIGS[a.config]
            zs = z_schedule(cfg.z_start, cfg.z_end, cfg.n_steps)
        else:
            cfg = BoxConfig("tune", a.n, 0.8, 1.0, a.packets, 400, 1800.0, 600.0, None, a.precision)
            zs = z_schedule(1800.0, 600.0, 400)
        d, U = make_box(cfg, seed=1)
        box = Box(cfg.n, d, U, cfg.n_packets, precision=a.precision, mixing="tally", seed=1,
                  stream=torch.cuda.Stream())
        prep = a.prep
        key = workload_key(cfg.n, cfg.n_packets, a.precision)
    s0 = 0 if a.start_z is None else int(np.argmin(np.abs(zs - a.start_z)))
    box.state_init(zs[s0])
    for s in range(s0, s0 + prep):
        box.transport(s, zs[s])
        box.step(s, zs[s], zs[s + 1])
    prep += s0
    default = box.tuning()
    ms_default = time_transport(box, prep, zs[prep], a.reps)
    best, ms, log = autotune(box, prep, zs[prep], reps=a.reps, rounds=a.rounds)
    entry = {"setting": best, "ms_per_transport": ms, "default": default, "ms_default": ms_default,
             "trials": len(log), "device": torch.cuda.get_device_name(), "step": prep}
    print(json.dumps({key: entry}))
    if a.out:
        table = load_table(a.out)
        table[key] = entry
        with open(a.out, "w") as f:
            json.dump(table, f, indent=1, sort_keys=True)
    box.close()


if __name__ == "__main__":
    main()
