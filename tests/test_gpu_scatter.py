"""GPU resonant-scattering Monte Carlo (lya_scatter_mc) against the oracle.

Both sides follow the same photons through the same Philox streams with the
same operation order; they differ only in the last bits of the library
functions (exp, log, erf, atan) and of their independently built Voigt
tables.  Per photon, the fate, the number of scatterings and the number of
steps are therefore the same except in the rare case where such a last-bit
difference flips a comparison, and the distance and final frequency agree to
far better than 1e-6.  Checked on a uniform box and on ragged boxes with
density, ionisation and velocity structure, in both storage forms, with the
even allocation and with a caller prefix; plus the Peebles factor of
Fig. Cfact from GPU statistics, independence of the warp scheduling
parameter, the step cap and the rejected arguments."""
import numpy as np
import pytest
from scipy import stats

import oracle as O
from gpu_helpers import make_fields, set_state

pytestmark = pytest.mark.gpu

LAMBDA_A = 6.62607015e-34 * 2.99792458e8 / (0.75 * 13.598434 * 1.602176634e-19)


def _box(n, precision, d, U, seed=7):
    from paper_2312_11448_gb300 import rec
    return rec.Box(n, d, U, 1000, precision=precision, mixing="full", seed=seed)


def _x50(cp, z, zeta, n1s):
    S = O.mc_setup(cp, O.mc_params(z, zeta=zeta))
    return (S["sig0"] * S["a"] * n1s / (np.sqrt(np.pi) * S["dxdl"])) ** (1 / 3)


def _compare(gpu, orc, min_same=0.99):
    assert len(gpu) == len(orc)
    assert np.array_equal(gpu["home"], orc["home"]) and np.array_equal(gpu["j"], orc["j"])
    same = (gpu["fate"] == orc["fate"]) & (gpu["n_scat"] == orc["n_scat"]) & (gpu["n_steps"] == orc["n_steps"])
    assert same.mean() >= min_same, f"only {same.mean():.4f} of the photons agree"
    np.testing.assert_allclose(gpu["D_kpc"][same], orc["D_kpc"][same], rtol=1e-6, atol=1e-15)
    np.testing.assert_allclose(gpu["x_end"][same], orc["x_end"][same], rtol=1e-6, atol=1e-9)
    return same


def _oracle_run(cp, box, z, n_photons, P, seed, **kw):
    d = box.host("delta").astype(np.float64)
    x = box.host("x")
    U = box.host("vel4")[:, :3].astype(np.float64)
    mp = O.mc_params(z, seed=seed, **kw)
    return O.lya_mc(cp, mp, box.n, d, x, P, U=U, threads=8)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_uniform_box_matches_oracle(cosmo, precision):
    n, z, zeta, xe = 4, 1700.0, 3e4, 0.5
    box = _box(n, precision, np.ones(n ** 3), np.zeros((n ** 3, 3)))
    set_state(box, np.full(n ** 3, xe), np.full(n ** 3, 4000.0))
    N = 1024
    x_lost = 50 * _x50(cosmo, z, zeta, O.background(cosmo, z)["nH"] * (1 - xe))
    kw = dict(zeta=zeta, lambda2g=0.0, x_lost=x_lost, max_steps=2_000_000)
    rec, st = box.scatter_mc(z, N, **kw)
    P = (np.arange(n ** 3 + 1) * N // n ** 3).astype(np.uint32)
    orc, cnt = _oracle_run(cosmo, box, z, N, P, seed=7, **kw)
    _compare(rec, orc)
    assert st["count"] == [int(v) for v in np.bincount(rec["fate"], minlength=4)]
    assert st["steps"] == int(rec["n_steps"].sum()) and st["scatterings"] == int(rec["n_scat"].sum())
    assert st["sampler_caps"] == 0 and st["nonfinite"] == 0
    box.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("n,sigma_v", [(8, 20.0), (13, 5.0)])
def test_structured_box_matches_oracle(cosmo, precision, n, sigma_v):
    """Lognormal density, ionisation fraction varying from cell to cell and a
    random velocity field (bulk flows of many Doppler widths); even allocation."""
    z, zeta = 1650.0, 1e4
    d, U = make_fields(n, 0.8, sigma_v, seed=3)
    box = _box(n, precision, d, U)
    rng = np.random.default_rng(n)
    set_state(box, rng.uniform(0.3, 0.7, n ** 3), np.full(n ** 3, 4000.0))
    N = 777
    x_lost = 50 * _x50(cosmo, z, zeta, 0.5 * O.background(cosmo, z)["nH"])
    kw = dict(zeta=zeta, lambda2g=2e4, x_lost=x_lost, step=3, max_steps=2_000_000)
    rec, st = box.scatter_mc(z, N, **kw)
    P = (np.arange(n ** 3 + 1, dtype=np.int64) * N // n ** 3).astype(np.uint32)
    orc, cnt = _oracle_run(cosmo, box, z, N, P, seed=7, **kw)
    _compare(rec, orc)
    assert st["sampler_caps"] == 0
    box.close()


def test_caller_prefix_matches_oracle(cosmo):
    """Photons allocated by the caller in proportion to a weight (the emission
    alpha_e n_e^2 in the paper's box Monte Carlo), some cells without photons."""
    n, z, zeta = 8, 1700.0, 1e4
    d, U = make_fields(n, 1.0, 10.0, seed=5)
    box = _box(n, "fp64", d, U)
    set_state(box, np.full(n ** 3, 0.6), np.full(n ** 3, 4000.0))
    rng = np.random.default_rng(2)
    counts = rng.multinomial(1500, d ** 2 / np.sum(d ** 2))
    P = np.concatenate([[0], np.cumsum(counts)]).astype(np.uint32)
    x_lost = 50 * _x50(cosmo, z, zeta, 0.4 * O.background(cosmo, z)["nH"])
    kw = dict(zeta=zeta, lambda2g=0.0, x_lost=x_lost, max_steps=2_000_000)
    rec, st = box.scatter_mc(z, 1500, prefix=P, **kw)
    orc, _ = _oracle_run(cosmo, box, z, 1500, P, seed=7, **kw)
    _compare(rec, orc)
    assert np.array_equal(np.bincount(rec["home"], minlength=n ** 3), counts)
    box.close()


def test_scheduling_parameter_does_not_change_results(cosmo):
    n, z = 6, 1700.0
    d, U = make_fields(n, 0.5, 3.0, seed=9)
    box = _box(n, "mixed", d, U)
    set_state(box, np.full(n ** 3, 0.5), np.full(n ** 3, 4000.0))
    x_lost = 50 * _x50(cosmo, z, 3e4, 0.5 * O.background(cosmo, z)["nH"])
    runs = [box.scatter_mc(z, 1200, zeta=3e4, x_lost=x_lost, pending=p, max_steps=1_000_000)[0] for p in (1, 12, 32)]
    for r in runs[1:]:
        assert np.array_equal(r, runs[0])
    box.close()


def test_peebles_factor_on_gpu(cosmo):
    """Fig. Cfact with GPU statistics: Lambda_2gamma = 0, C = p_alpha f_z against
    R / (beta + R) at three expansion rates."""
    n, z, xe = 4, 1700.0, 0.5
    box = _box(n, "mixed", np.ones(n ** 3), np.zeros((n ** 3, 3)))
    set_state(box, np.full(n ** 3, xe), np.full(n ** 3, 4000.0))
    bg = O.background(cosmo, z)
    n1s = bg["nH"] * (1 - xe)
    beta = O.rates(cosmo, z, bg["Tg"])["beta"]
    A = O.A_2P1S
    for zeta in (3e3, 1e4, 3e4):
        _, st = box.scatter_mc(z, 8192, records=False, zeta=zeta, lambda2g=0.0,
                               x_lost=50 * _x50(cosmo, z, zeta, n1s), max_steps=2_000_000)
        # The lifetime tail: a few photons in 10^4 outlive the step cap.  They are
        # kept in N and counted as not escaped; whatever their true fate, that
        # moves C by at most p_alpha * capped / N, which widens the band.
        N, capped = 8192, st["count"][3]
        assert capped <= 8 and st["count"][1] == 0
        R = 8 * np.pi * zeta * bg["H"] / (LAMBDA_A ** 3 * n1s)
        C_th = R / (beta + R)
        p_alpha = 3 * A / (beta + 3 * A)
        C_mc = p_alpha * st["count"][0] / N
        band = 4 * np.sqrt(C_th * (1 - C_th) / N) + p_alpha * capped / N
        assert C_mc == pytest.approx(C_th, abs=band), zeta
    box.close()


def test_step_cap(cosmo):
    box = _box(2, "fp64", np.ones(8), np.zeros((8, 3)))
    set_state(box, np.full(8, 0.5), np.full(8, 4000.0))
    rec, st = box.scatter_mc(1500.0, 40, max_steps=500)
    capped = rec["fate"] == 3
    assert capped.sum() >= 39 and st["count"][3] == capped.sum()  # ending within 500 steps: p ~ 1e-3
    assert np.all(rec["n_steps"][capped] == 500) and np.all(rec["n_steps"] <= 500)
    box.close()


def test_rejected_arguments():
    from paper_2312_11448_gb300 import rec
    box = _box(2, "fp64", np.ones(8), np.zeros((8, 3)))
    for bad in (dict(eps=0.0), dict(eps=1.5), dict(zeta=0.0), dict(x_lost=-1.0), dict(pending=33),
                dict(max_steps=0), dict(A_alpha=0.0)):
        with pytest.raises(rec.RecError):
            box.scatter_mc(1500.0, 10, **bad)
    with pytest.raises(rec.RecError):
        box.scatter_mc(1500.0, 0)
    with pytest.raises(rec.RecError):
        box.scatter_mc(-1.0, 10)
    box.close()
    d, U = make_fields(4, 0.5, 1.0, seed=1)
    b = rec.Batch([(4, d, U, 10), (4, d, U, 10)], precision="fp64")
    with pytest.raises(rec.RecError, match="single-box"):
        b._check(rec.lib().lya_scatter_mc(b.ctx, rec.C.byref(rec.mc_params(1500.0, 10)), None, None, None),
                 "lya_scatter_mc")
    b.close()


# ---- mixed-arithmetic form (statistical parity) ---------------------------------


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_mixed_arith_statistics_match_oracle(cosmo, precision):
    """Fate fractions (binomial) and the distributions of scattering counts,
    step counts and distances (two-sample KS) against the oracle on independent
    streams."""
    n, z, zeta = 8, 1650.0, 1e4
    d, U = make_fields(n, 0.8, 10.0, seed=3)
    box = _box(n, precision, d, U)
    set_state(box, np.random.default_rng(1).uniform(0.3, 0.7, n ** 3), np.full(n ** 3, 4000.0))
    N = 4096
    kw = dict(zeta=zeta, lambda2g=2e4, x_lost=50 * _x50(cosmo, z, zeta, 0.5 * O.background(cosmo, z)["nH"]),
              max_steps=2_000_000)
    g, st = box.scatter_mc(z, N, arith="mixed", **kw)
    P = (np.arange(n ** 3 + 1, dtype=np.int64) * N // n ** 3).astype(np.uint32)
    o, _ = _oracle_run(cosmo, box, z, N, P, seed=11, **kw)
    for f in range(3):
        pg, po = np.mean(g["fate"] == f), np.mean(o["fate"] == f)
        assert abs(pg - po) < 5 * np.sqrt(max(po * (1 - po), 1e-4) * 2 / N), f
    for key in ("n_scat", "n_steps", "D_kpc"):
        assert stats.ks_2samp(g[key].astype(float), o[key].astype(float)).pvalue > 1e-3, key
    assert st["sampler_caps"] == 0 and st["nonfinite"] == 0
    box.close()


def test_mixed_arith_peebles_factor(cosmo):
    """Fig. Cfact with the mixed-arithmetic kernel: C = p_alpha f_z from 32768
    photons per expansion rate (a) equals the binary64 kernel's C on
    independent photons (two-sample binomial test, 5 sigma) and (b) follows
    R / (beta + R) of Eq. Cfactor within 4 sigma plus 3 % of C.  At this sample
    size both arithmetic forms resolve a deficit of about 2 % below that
    Sobolev-limit formula at zeta >= 1e4 (the same in both forms, at eps = 0.1
    and 0.03, up to zeta = 1e5), so the allowance is a property of the
    Monte Carlo, not of the arithmetic."""
    n, z, xe = 4, 1700.0, 0.5
    box = _box(n, "mixed", np.ones(n ** 3), np.zeros((n ** 3, 3)))
    set_state(box, np.full(n ** 3, xe), np.full(n ** 3, 4000.0))
    bg = O.background(cosmo, z)
    n1s = bg["nH"] * (1 - xe)
    beta = O.rates(cosmo, z, bg["Tg"])["beta"]
    A = O.A_2P1S
    Np = 32768
    for zeta in (3e3, 1e4, 3e4):
        kw = dict(records=False, zeta=zeta, lambda2g=0.0, x_lost=50 * _x50(cosmo, z, zeta, n1s),
                  max_steps=2_000_000)
        C = {}
        for arith, step in (("mixed", 0), ("fp64", 1)):
            _, st = box.scatter_mc(z, Np, arith=arith, step=step, **kw)
            N = Np - st["count"][3]
            assert st["count"][3] <= 8 and st["count"][1] == 0 and st["nonfinite"] == 0
            C[arith] = (3 * A / (beta + 3 * A) * st["count"][0] / N, N)
        R = 8 * np.pi * zeta * bg["H"] / (LAMBDA_A ** 3 * n1s)
        C_th = R / (beta + R)
        (cm, Nm), (cf, Nf) = C["mixed"], C["fp64"]
        p = 0.5 * (cm + cf)
        assert abs(cm - cf) < 5 * np.sqrt(p * (1 - p) * (1 / Nm + 1 / Nf)), zeta
        assert cm == pytest.approx(C_th, abs=4 * np.sqrt(C_th * (1 - C_th) / Nm) + 0.03 * C_th), zeta
    box.close()
