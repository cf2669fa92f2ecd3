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
        assert all(box.tuning()[k] == v for k, v in s.items())
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
    # the defaults are the kernels' residency limits: one block more is rejected
    for bad in (dict(emit_blocks_per_sm=0), dict(emit_blocks_per_sm=t0["emit_blocks_per_sm"] + 1),
                dict(march_blocks_per_sm=t0["march_blocks_per_sm"] + 1),
                dict(march_refill=33), dict(march_chunk=4), dict(tile=12)):
        with pytest.raises(rec.RecError):
            box.set_tuning(**bad)
        assert box.tuning() == t0
    box.close()


def _sweep_case(cosmo, n, Np, precision, settings):
    """Tallies and counters of lya_transport under each (halo, tile) setting
    against the oracle's; returns the statistics records."""
    import oracle as O
    from gpu_helpers import oracle_fields, quantiles, set_state
    box = new_box(n, precision, n_packets=Np, sigma_v=2.0)
    rng = np.random.default_rng(5)
    emis = rng.lognormal(0.0, 1.0, n ** 3)
    T = rng.uniform(2800.0, 3200.0, n ** 3)
    set_state(box, np.full(n ** 3, 0.5), T, tally=np.zeros(n ** 3, np.uint32), emis=emis)
    _, _, v4 = oracle_fields(box)
    prec = "f32" if precision == "mixed" else "f64"
    ref, cnt, _ = O.transport(cosmo, n, 1100.0, 7, 4, Np, box.host("emis"), v4, box.host("T"), quantiles(box),
                              precision=prec)
    limit = box.tuning()["march_blocks_per_sm"]
    out = []
    for halo, tile in settings:
        box.set_tuning(march_halo=halo, tile=tile, march_blocks_per_sm=min(limit, 2))
        _zero_tallies(box, [box.tally])
        box.timing(True)
        box.transport(4, 1100.0)
        kt = box.kernel_times()
        box.timing(False)
        st = box.stats()
        assert np.array_equal(box.tally_np(), ref), (halo, tile)
        assert st["absorbed"] == cnt["absorbed"] == Np and st["crossings"] == cnt["crossings"], (halo, tile)
        if halo:
            assert kt["march"][1] == 22 and st["requeued"] > 0, (halo, tile, kt["march"], st["requeued"])
        else:
            assert kt["march"][1] == 1 and st["requeued"] == 0
        out.append(st)
    box.close()
    return out


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_region_sweeps_match_the_oracle(cosmo, precision):
    """march_halo > 0 (region sweeps) on a 64^3 box: tallies and counters
    bit-identical to the oracle for several halos and super-tile sides; the
    march group runs its eight sweeps and packets are queued again."""
    _sweep_case(cosmo, 64, 400_000, precision, ((4, 8), (8, 16), (0, 32)))


def test_region_sweeps_with_a_full_second_queue(cosmo):
    """A one-cell halo around 8-cell super-tiles on a 256^3 box: about 29 % of
    the packets end outside their first region (oracle per-packet dump), more
    than the second queue holds (n_packets / 4), so packets find it full and
    march on without a limit (flags bit 4); the result is still exact."""
    st = _sweep_case(cosmo, 256, 1_000_000, "mixed", ((1, 8), (0, 32)))
    assert st[0]["flags"] & 16
    assert not st[1]["flags"] & 16  # the flag describes one transport call


def test_region_sweep_settings_rejected():
    from paper_2312_11448_gb300 import rec
    box = new_box(12, "mixed", n_packets=100)  # not a power of two
    with pytest.raises(rec.RecError, match="power-of-two"):
        box.set_tuning(march_halo=4)
    box.close()
    box = new_box(16, "mixed", n_packets=100)
    for bad in (dict(march_halo=-1), dict(march_halo=257)):
        with pytest.raises(rec.RecError):
            box.set_tuning(**bad)
    box.set_tuning(march_halo=4, march_blocks_per_sm=3)
    assert box.tuning()["march_halo"] == 4
    box.close()
    # the FP64 form's sweep march has a lower residency limit (2) than its plain march (3)
    box = new_box(16, "fp64", n_packets=100)
    assert box.tuning()["march_blocks_per_sm"] == 3
    with pytest.raises(rec.RecError, match="march_halo"):
        box.set_tuning(march_halo=4)
    box.set_tuning(march_halo=4, march_blocks_per_sm=2)
    box.close()
