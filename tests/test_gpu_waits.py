"""Bounded device-side waits: the bulk-copy stages of the mixed form's
per-cell passes give up when their wait limit runs out, the step returns
cleanly, rec_sync reports REC_ETIMEOUT, and after re-initialising the state
the same context steps again to the same result as a context that never
timed out.  The expiry is provoked with a zero limit (give up whenever a
stage is not complete at the first look); nothing faults or hangs."""
import numpy as np
import pytest

from gpu_helpers import make_fields

pytestmark = pytest.mark.gpu


def _box(seed=7):
    from paper_2312_11448_gb300 import rec
    d, U = make_fields(64, 0.8, 1.0, seed=3)
    return rec.Box(64, d, U, 200_000, precision="mixed", mixing="tally", seed=seed)


def _run(box, z0=1300.0, z1=1295.0):
    box.state_init(z0)
    box.transport(0, z0)
    box.step(0, z0, z1)


def test_wait_expiry_reports_timeout_and_context_recovers():
    from paper_2312_11448_gb300 import rec
    ref = _box()
    _run(ref)
    ref.sync()  # no expiry at the default limit
    x_ref = ref.host("x").copy()
    assert ref.stats()["flags"] & 8 == 0
    ref.close()

    box = _box()
    box.set_wait_limit(0)
    _run(box)
    with pytest.raises(rec.RecError) as ei:
        box.sync()
    assert ei.value.status == rec.REC_ETIMEOUT
    box.sync()  # the expiry was reported once and cleared
    box.set_wait_limit(1 << 22)
    box.tally.zero_()  # a final pass that gave up left some tallies in place
    _run(box)
    box.sync()
    assert box.stats()["flags"] & 8 == 0
    np.testing.assert_array_equal(box.host("x"), x_ref)
    box.close()


def test_sync_without_work_and_rejections():
    from paper_2312_11448_gb300 import rec
    box = _box()
    box.sync()
    box.set_wait_limit(5)
    box.close()


def test_batched_step_is_three_launches_and_its_barriers_are_bounded():
    """A batched step runs as three launches (the persistent allocation +
    emission launch, the march, one persistent launch per rec_step substep),
    whose phases are separated by bounded grid barriers.  With a zero wait
    limit the barriers give up, rec_sync reports REC_ETIMEOUT, and after
    re-initialising the state the same batch reproduces a fresh batch."""
    from paper_2312_11448_gb300 import rec
    sizes = [(16, 0.8, 40_000), (24, 1.2, 90_000), (13, 0.3, 20_001)]

    def batch():
        boxes = []
        for i, (n, sig, npk) in enumerate(sizes):
            d, U = make_fields(n, sig, 1.0, seed=40 + i)
            boxes.append((n, d, U, npk))
        return rec.Batch(boxes, precision="mixed", mixing="tally", seed=9)

    def run(b):
        b.state_init(1400.0)
        b.transport(0, 1400.0)
        b.step(0, 1400.0, 1395.0)

    ref = batch()
    ref.timing(True)
    run(ref)
    ref.sync()
    launches = sum(v[1] for g, v in ref.kernel_times().items() if g != "other")
    assert launches == 3
    xs = [ref.host("x", b).copy() for b in range(len(sizes))]
    ref.close()

    b = batch()
    b.set_wait_limit(0)
    run(b)
    with pytest.raises(rec.RecError) as ei:
        b.sync()
    assert ei.value.status == rec.REC_ETIMEOUT
    b.set_wait_limit(1 << 22)
    for t in b.tally:
        t.zero_()
    run(b)
    b.sync()
    for i in range(len(sizes)):
        np.testing.assert_array_equal(b.host("x", i), xs[i])
    b.close()
