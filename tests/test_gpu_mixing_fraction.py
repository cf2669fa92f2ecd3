"""The Monte-Carlo mixing fraction f_alpha(D) of Sec. III.B computed behind
the C ABI (lya_mc_mixing_fraction), against its definition written out here
on the same records; and the chain Sec. V builds from it: Monte Carlo at one
redshift -> f_alpha(D) -> partial-mixing share (rec_set_f_alpha) -> one
recombination step, against the oracle's partial-mixing step at that share.

Definition: among photons destroyed in the line (two-photon decay or
photo-ionisation of the n = 2 atom), the fraction destroyed farther than D
from their emission point; photons lost by redshifting do not count, capped
photons are reported separately and bracket the value."""
import numpy as np
import pytest

import oracle as O
from gpu_helpers import oracle_fields, set_state

pytestmark = pytest.mark.gpu


def _definition(recs, D):
    fate = recs["fate"]
    dest = recs["D_kpc"][(fate == 1) | (fate == 2)]
    nc = int((fate == 3).sum())
    B = np.array([(dest > d).sum() for d in D], dtype=np.float64)
    Nd = dest.size
    f = B / Nd if Nd else np.full(len(D), np.nan)
    return f, B / (Nd + nc), (B + nc) / (Nd + nc)


def _x_lost(cp, z, zeta, xe):
    """50 x_50: far enough into the red wing that no photon returns (App. A)."""
    S = O.mc_setup(cp, O.mc_params(z, zeta=zeta))
    n1s = O.background(cp, z)["nH"] * (1 - xe)
    return 50 * (S["sig0"] * S["a"] * n1s / (np.sqrt(np.pi) * S["dxdl"])) ** (1 / 3)


def _uniform_box(n=4, precision="fp64", mixing="full", seed=7):
    from paper_2312_11448_gb300 import rec
    return rec.Box(n, np.ones(n ** 3), np.zeros((n ** 3, 3)), 1000, precision=precision, mixing=mixing, seed=seed)


def test_hand_made_records():
    import torch
    from paper_2312_11448_gb300 import rec
    box = _uniform_box()
    r = np.zeros(8, dtype=rec.MC_PHOTON)
    r["fate"] = [0, 1, 2, 2, 3, 1, 2, 3]
    r["D_kpc"] = [9.0, 0.1, 0.5, 2.0, 9.0, 3.5, 0.5, 0.2]
    dev = torch.as_tensor(r.view(np.uint8)).to(box.x.device)
    D = [0.0, 0.3, 0.5, 1.0, 3.0, 4.0]
    f, fmin, fmax, cnt = box.mixing_fraction(D, records=dev)
    np.testing.assert_array_equal(f, [5 / 5, 4 / 5, 2 / 5, 2 / 5, 1 / 5, 0.0])
    np.testing.assert_array_equal(fmin, [5 / 7, 4 / 7, 2 / 7, 2 / 7, 1 / 7, 0.0])
    np.testing.assert_array_equal(fmax, [7 / 7, 6 / 7, 4 / 7, 4 / 7, 3 / 7, 2 / 7])
    assert list(cnt) == [1, 2, 3, 2]
    # no destroyed photon: NaN, not a division by zero
    r["fate"] = 0
    dev = torch.as_tensor(r.view(np.uint8)).to(box.x.device)
    f, fmin, fmax, cnt = box.mixing_fraction([1.0], records=dev)
    assert np.isnan(f[0]) and np.isnan(fmin[0]) and list(cnt) == [8, 0, 0, 0]
    for bad in ([-1.0], [np.inf], [np.nan], np.zeros(257)):
        with pytest.raises(rec.RecError):
            box.mixing_fraction(bad, records=dev)
    box.close()


@pytest.mark.parametrize("arith", ["fp64", "mixed"])
def test_gpu_records_match_definition(cosmo, arith):
    n, z, xe = 4, 1700.0, 0.5
    box = _uniform_box(n)
    set_state(box, np.full(n ** 3, xe), np.full(n ** 3, 4000.0))
    recs, st = box.scatter_mc(z, 4096, zeta=3e3, lambda2g=3e4, x_lost=_x_lost(cosmo, z, 3e3, xe), arith=arith, max_steps=200_000)
    D = np.concatenate([[0.0], np.logspace(-7, -2, 40)])
    f, fmin, fmax, cnt = box.mixing_fraction(D)
    rf, rmin, rmax = _definition(recs, D)
    np.testing.assert_array_equal(f, rf)
    np.testing.assert_array_equal(fmin, rmin)
    np.testing.assert_array_equal(fmax, rmax)
    assert list(cnt) == st["count"]
    assert f[0] == 1.0 and np.all(np.diff(f) <= 0) and 0.0 < np.median(f) < 1.0
    box.close()


def test_mc_fraction_drives_partial_mixing_step(cosmo):
    """Sec. V's partial mixing with the Monte-Carlo fraction, end to end on the
    GPU: the share comes from lya_mc_mixing_fraction, goes to rec_set_f_alpha,
    and the next step equals the oracle's partial-mixing step at that share.
    (With the accelerated expansion rate that keeps the test short, photons
    travel sub-parsec distances, so the distance is taken where f_alpha is
    between 0.2 and 0.8 rather than at 3 kpc.)"""
    from paper_2312_11448_gb300 import rec
    from gpu_helpers import make_fields
    n, z_mc, xe = 4, 1700.0, 0.5
    mc = _uniform_box(n)
    set_state(mc, np.full(n ** 3, xe), np.full(n ** 3, 4000.0))
    mc.scatter_mc(z_mc, 4096, zeta=3e3, lambda2g=3e4, x_lost=_x_lost(cosmo, z_mc, 3e3, xe), max_steps=200_000)
    D = np.logspace(-7, -2, 60)
    f_all, _, _, _ = mc.mixing_fraction(D)
    j = int(np.argmin(np.abs(f_all - 0.5)))
    f_alpha = float(f_all[j])
    assert 0.2 < f_alpha < 0.8
    mc.close()
    m = 12
    d, U = make_fields(m, 0.8, 3.0, seed=2)
    box = rec.Box(m, d, U, 1000, precision="fp64", mixing="partial", seed=7, f_alpha=1.0)
    box.state_init(1300.0)
    dd, UU, _ = oracle_fields(box)
    x0 = box.host("x")
    T0 = box.host("T").astype(np.float64)
    box.set_f_alpha(f_alpha)
    box.step(0, 1300.0, 1290.0)
    x1, T1, U1, e1, so = O.rec_step(cosmo, m, 1300.0, 1290.0, dd, x0, T0, U=UU, mixing="partial", f_alpha=f_alpha)
    np.testing.assert_allclose(box.host("x"), x1, rtol=1e-9, atol=0)
    np.testing.assert_allclose(box.host("T"), T1, rtol=1e-9, atol=0)
    np.testing.assert_allclose(box.host("vel4")[:, :3], U1, rtol=1e-9, atol=1e-14)
    assert box.stats()["X_e"] == pytest.approx(so["Xe"], rel=1e-9)
    box.close()


def test_volume_stats_start_node(cosmo):
    """rec_volume_stats gives X_e = sum delta x / sum delta of the current state
    (Sec. II.A), as the oracle's history records it at a trajectory's start."""
    from paper_2312_11448_gb300 import rec
    from gpu_helpers import make_fields
    for precision in ("fp64", "mixed"):
        n = 16
        d, U = make_fields(n, 0.8, 1.0, seed=4)
        box = rec.Box(n, d, U, 1000, precision=precision, mixing="full", seed=7)
        box.state_init(1250.0)
        box.volume_stats(0)
        dd = box.host("delta").astype(np.float64)
        x = box.host("x")
        assert box.stats()["X_e"] == pytest.approx(np.dot(dd, x) / dd.sum(), rel=1e-13)
        box.close()
    box = rec.Box(8, d[:512], U[:512], 1000, precision="fp64", mixing="full")
    with pytest.raises(rec.RecError, match="rec_state_init"):
        box.volume_stats(0)
    box.close()
