"""Transport tuning (grids, refill threshold, chunk size, super-tile side)
changes only the speed: tallies and counters must be bit-identical for every
valid setting, single boxes and batches; invalid settings are rejected and
leave the tuning unchanged."""
import numpy as np
import pytest

from gpu_helpers import make_fields, new_box

pytestmark = pytest.mark.gpu


def _settings(t0):
    e, m = t0["emit_blocks_per_sm"], t0["march_blocks_per_sm"]  # defaults are the launch-bound maxima
    return [t0,
            dict(emit_blocks_per_sm=1, march_blocks_per_sm=1, march_refill=1, march_chunk=8, tile=8),
            dict(emit_blocks_per_sm=min(2, e), march_blocks_per_sm=min(3, m), march_refill=32, march_chunk=4096,
                 tile=64),
            dict(emit_blocks_per_sm=e, march_blocks_per_sm=m, march_refill=12, march_chunk=40, tile=16)]


def _zero_tallies(obj, boxes):
    import torch
    obj.stream.synchronize()
    for t in boxes:
        t.zero_()
    torch.cuda.synchronize()


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_single_box_tallies_do_not_depend_on_tuning(precision):
    box = new_box(24, precision, n_packets=200_000, sigma_v=2.0)
    box.state_init(1400.0)
    t0 = box.tuning()
    ref = None
    for s in _settings(t0):
        box.set_tuning(**s)
        assert box.tuning() == s
        _zero_tallies(box, [box.tally])
        box.transport(3, 1390.0)
        got = (box.tally_np().copy(), {k: box.stats()[k] for k in ("emitted", "absorbed", "crossings", "queued")})
        if ref is None:
            ref = got
        else:
            assert np.array_equal(got[0], ref[0]) and got[1] == ref[1], s
    box.close()


def test_batch_tallies_do_not_depend_on_tuning():
    from paper_2312_11448_gb300 import rec
    boxes = []
    for i, (n, npk) in enumerate([(20, 80_000), (13, 30_000), (32, 150_000)]):
        d, U = make_fields(n, 0.7, 1.0, seed=60 + i)
        boxes.append((n, d, U, npk))
    b = rec.Batch(boxes, precision="mixed", seed=3)
    b.state_init(1400.0)
    t0 = b.tuning()
    ref = None
    for s in _settings(t0):
        b.set_tuning(**s)
        _zero_tallies(b, b.tally)
        b.transport(2, 1390.0)
        got = [b.tally_np(i).copy() for i in range(3)]
        st = [(r["absorbed"], r["crossings"], r["queued"]) for r in b.stats()]
        if ref is None:
            ref = (got, st)
        else:
            assert all(np.array_equal(x, y) for x, y in zip(got, ref[0])) and st == ref[1], s
    b.close()


def test_invalid_tuning_rejected():
    from paper_2312_11448_gb300 import rec
    box = new_box(8, "fp64", n_packets=100)
    t0 = box.tuning()
    for bad in (dict(emit_blocks_per_sm=0), dict(emit_blocks_per_sm=4), dict(march_blocks_per_sm=5),
                dict(march_refill=33), dict(march_chunk=4), dict(tile=12)):
        with pytest.raises(rec.RecError):
            box.set_tuning(**bad)
        assert box.tuning() == t0
    box.close()
