"""GPU transport vs the oracle, element by element: the per-cell tallies must be
bit-identical (integer work) on the same seeded inputs, in both precision
forms, on boxes spanning several allocation chunks and a ragged tail, at the
full 256^3 / 1e8-packet size, and on the degenerate cases."""
import numpy as np
import pytest

import oracle as O
from gpu_helpers import new_box, oracle_fields, quantiles, set_state

pytestmark = pytest.mark.gpu


def _run_both(cosmo, box, emis, T, z, step, n_packets, threads=0):
    n = box.n
    set_state(box, np.full(n ** 3, 0.5), T, tally=np.zeros(n ** 3, np.uint32), emis=emis)
    box.transport(step, z)
    gpu = box.tally_np().copy()
    st = box.stats()
    _, _, v4 = oracle_fields(box)
    prec = "f32" if box.precision == "mixed" else "f64"
    tally, cnt, _ = O.transport(cosmo, n, z, 7, step, n_packets, box.host("emis"), v4, box.host("T"),
                                quantiles(box), precision=prec, threads=threads)
    return gpu, st, tally, cnt


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
@pytest.mark.parametrize("n,Np", [(13, 299_999), (24, 300_000)])
def test_tallies_bit_exact(cosmo, precision, n, Np):
    """n=13: 2197 cells (ragged against every block size) and a packet count
    that leaves a partial warp; n=24: 13824 cells, several allocation chunks."""
    box = new_box(n, precision, n_packets=Np, sigma_v=2.0)
    rng = np.random.default_rng(n)
    emis = rng.lognormal(0.0, 1.5, n ** 3)
    emis[rng.integers(0, n ** 3, 50)] = 0.0
    T = rng.uniform(2500.0, 3500.0, n ** 3)
    gpu, st, tally, cnt = _run_both(cosmo, box, emis, T, 1100.0, 5, Np)
    assert st["emitted"] == cnt["emitted"] == Np
    assert st["absorbed"] == cnt["absorbed"] == Np and st["capped"] == 0
    assert st["crossings"] == cnt["crossings"]
    assert np.array_equal(gpu, tally)
    box.close()


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_steps_and_redshifts_change_streams(cosmo, precision):
    n, Np = 16, 100_000
    box = new_box(n, precision, n_packets=Np)
    rng = np.random.default_rng(2)
    emis = rng.uniform(0.5, 1.5, n ** 3)
    T = np.full(n ** 3, 3000.0)
    for step, z in ((0, 1500.0), (1, 1500.0), (9, 800.0)):
        gpu, st, tally, cnt = _run_both(cosmo, box, emis, T, z, step, Np)
        assert np.array_equal(gpu, tally)
    box.close()


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_degenerate_inputs(cosmo, precision):
    n = 8
    box = new_box(n, precision, n_packets=1000)
    T = np.full(n ** 3, 3000.0)
    # a single emitting cell: every packet starts there
    emis = np.zeros(n ** 3); emis[77] = 2.5
    gpu, st, tally, cnt = _run_both(cosmo, box, emis, T, 1200.0, 3, 1000)
    assert np.array_equal(gpu, tally) and gpu.sum() == 1000
    # no emission at all: the oracle rejects the input, the GPU emits nothing
    # and raises the invalid-weights flag
    with pytest.raises(ValueError):
        _run_both(cosmo, box, np.zeros(n ** 3), T, 1200.0, 3, 1000)
    st = box.stats()
    assert box.tally_np().sum() == 0 and st["emitted"] == 0 and (st["flags"] & 4)
    # a negative weight is invalid input as well
    bad = np.ones(n ** 3); bad[3] = -1.0
    with pytest.raises(ValueError):
        _run_both(cosmo, box, bad, T, 1200.0, 3, 1000)
    st = box.stats()
    assert box.tally_np().sum() == 0 and st["emitted"] == 0 and (st["flags"] & 4)
    box.close()
    # zero packets requested
    box = new_box(n, precision, n_packets=0)
    gpu, st, tally, cnt = _run_both(cosmo, box, np.ones(n ** 3), T, 1200.0, 3, 0)
    assert gpu.sum() == 0 and st["emitted"] == 0
    box.close()


def test_one_cell_box(cosmo):
    box = new_box(1, "fp64", n_packets=500)
    gpu, st, tally, cnt = _run_both(cosmo, box, np.ones(1), np.full(1, 3000.0), 1100.0, 0, 500)
    assert gpu[0] == 500 and np.array_equal(gpu, tally)
    box.close()


@pytest.mark.slow
def test_full_size_256_cubed_1e8_packets(cosmo):
    """The benchmark configuration (256^3, 1e8 packets, binary32 transport):
    all 16.7M tallies bit-exact against the oracle."""
    from paper_2312_11448_gb300.inputs import density_field
    n, Np = 256, 100_000_000
    box = new_box(n, "mixed", n_packets=Np, sigma=0.8, sigma_v=1.0)
    d = density_field(n, 0.8, 1).ravel()
    emis = d * d  # recombination weight of a uniformly ionised box: alpha n_e^2 ~ Delta^2
    T = np.full(n ** 3, 2.7255 * 1101.0) * (1.0 + 0.01 * np.sin(np.arange(n ** 3)))
    gpu, st, tally, cnt = _run_both(cosmo, box, emis, T, 1100.0, 17, Np)
    assert st["emitted"] == cnt["emitted"] == Np and st["absorbed"] == Np
    assert st["crossings"] == cnt["crossings"]
    assert np.array_equal(gpu, tally)
    box.close()


@pytest.mark.slow
def test_full_size_512_cubed_1e8_packets(cosmo):
    """512^3 (the largest configuration's box, sigma_lnrho 1.2, sigma_v 2 km/s),
    1e8 packets, binary32 transport: all 134M tallies bit-exact against the
    oracle (its OpenMP build: the same integers in any order)."""
    import os
    from paper_2312_11448_gb300.inputs import density_field
    n, Np = 512, 100_000_000
    box = new_box(n, "mixed", n_packets=Np, sigma=1.2, sigma_v=2.0)
    d = density_field(n, 1.2, 1).ravel()
    emis = d * d
    T = np.full(n ** 3, 2.7255 * 1101.0) * (1.0 + 0.01 * np.sin(np.arange(n ** 3)))
    gpu, st, tally, cnt = _run_both(cosmo, box, emis, T, 1100.0, 23, Np, threads=os.cpu_count() or 1)
    assert st["emitted"] == cnt["emitted"] == Np and st["absorbed"] == Np
    assert st["crossings"] == cnt["crossings"]
    assert np.array_equal(gpu, tally)
    box.close()
