"""The autotuner's search logic on the CPU (a synthetic cost with a known
minimum), its table keys and files."""
import json

from paper_2312_11448_gb300 import tune


def _start():
    return {"emit_blocks_per_sm": 5, "march_blocks_per_sm": 5, "march_refill": 8, "march_chunk": 64, "tile": 32,
            "march_halo": 0}


def test_coordinate_descent_finds_separable_minimum():
    target = {"emit_blocks_per_sm": 3, "march_blocks_per_sm": 4, "march_refill": 16, "march_chunk": 128, "tile": 16,
              "march_halo": 16}

    def cost(s):
        return sum((s[f] - target[f]) ** 2 / (1 + target[f]) for f in tune.FIELDS) + 1.0

    best, c, log = tune.coordinate_descent(_start(), cost)
    assert best == target and c == 1.0
    # every trial is a setting on the candidate grid, none evaluated twice
    keys = [tuple(s[f] for f in tune.FIELDS) for s, _ in log]
    assert len(keys) == len(set(keys))
    for s, _ in log:
        for f in tune.FIELDS:
            assert s[f] in tune.CANDIDATES[f] or s[f] == _start()[f]


def test_coordinate_descent_respects_limits_and_keeps_start_when_best():
    def cost(s):
        return 10.0 - s["march_blocks_per_sm"]  # wants the largest grid

    best, c, _ = tune.coordinate_descent(_start(), cost,
                                         allowed=lambda f, v: not (f == "march_blocks_per_sm" and v > 4))
    assert best["march_blocks_per_sm"] == 5  # the start value stays allowed
    flat, c2, log = tune.coordinate_descent(_start(), lambda s: 1.0)
    assert flat == _start() and c2 == 1.0 and len(log) > 1


def test_workload_keys_and_table(tmp_path):
    assert tune.workload_key(256, 100_000_000, "mixed") == "n256-ppc4-mixed-single"
    assert tune.workload_key(32, 1_000_000, "mixed", batch=True) == "n32-ppc16-mixed-batch"
    assert tune.workload_key(8, 0, "fp64") == "n8-ppc1-fp64-single"
    p = tmp_path / "t.json"
    p.write_text(json.dumps({"k": {"setting": _start()}}))
    old = {f: v for f, v in _start().items() if f != "march_halo"}  # an entry that predates a field
    p_old = tmp_path / "old.json"
    p_old.write_text(json.dumps({"k": {"setting": old}}))
    assert tune.load_table(str(p))["k"]["setting"]["tile"] == 32
    assert tune.load_table(str(tmp_path / "missing.json")) == {}

    class Fake:
        def __init__(self, limit=5):
            self.set = None
            self.limit = limit

        def tuning(self):  # defaults after rec_init: the residency limits
            return dict(_start(), emit_blocks_per_sm=self.limit, march_blocks_per_sm=self.limit)

        def set_tuning(self, **kw):
            self.set = kw

    f = Fake()
    assert tune.apply_table(f, "k", str(p)) == _start() and f.set == _start()
    # a stored grid above the kernels' current limit is clamped to it
    f = Fake(limit=4)
    assert tune.apply_table(f, "k", str(p)) == dict(_start(), emit_blocks_per_sm=4, march_blocks_per_sm=4)
    assert tune.apply_table(f, "absent", str(p)) is None
    # the missing field keeps the context's current value
    f = Fake()
    assert tune.apply_table(f, "k", str(p_old)) == _start()


def test_joint_search_of_march_grid_and_halo():
    """The sweep march admits a grid the plain march does not want: the best
    (grid, halo) pair is reachable only by changing both at once."""
    table = {(4, 0): 6.0, (2, 0): 5.0, (3, 0): 7.0, (3, 32): 1.0, (2, 32): 5.5}

    def cost(s):
        return table.get((s["march_blocks_per_sm"], s["march_halo"]), float("inf"))

    start = dict(_start(), march_blocks_per_sm=4)
    best, c, _ = tune.coordinate_descent(start, cost)
    assert (best["march_blocks_per_sm"], best["march_halo"]) == (3, 32) and c == 1.0
    # one field at a time stops at the plain march's best grid
    best1, c1, _ = tune.coordinate_descent(start, cost, joint=())
    assert (best1["march_blocks_per_sm"], best1["march_halo"]) == (2, 0) and c1 == 5.0
