"""Oracle pins for the second-order TR-BDF2 substep (the row after backward
Euler): convergence at second order to stiff library integrations of the
standard three-level atom (uniform box) and of the two-zone system of
Sec. IV.C with full mixing, far smaller errors than backward Euler at the same
step, tally mode reducing to full mixing when the tallies follow n_1s, and the
end-state identities (lambda, emission weights)."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2312_11448_gb300.inputs import z_schedule
from test_oracle_recombination import PV, _reference


def _history(cosmo, cells, n, zs, n_sub, integrator):
    d = np.asarray(cells, float)
    x = O.saha_xe(cosmo, zs[0], d)
    T = np.full(d.size, O.background(cosmo, zs[0])["Tg"])
    xs, Ts, Xe = [x.copy()], [T.copy()], [float((d * x).sum() / d.sum())]
    for s in range(len(zs) - 1):
        x, T, _, _, st = O.rec_step(cosmo, n, zs[s], zs[s + 1], d, x, T, mixing="full", n_sub=n_sub,
                                    integrator=integrator)
        xs.append(x.copy()); Ts.append(T.copy()); Xe.append(st["Xe"])
    return np.array(xs), np.array(Ts), np.array(Xe)


@pytest.fixture(scope="module")
def uniform(cosmo):
    zs = z_schedule(1700.0, 750.0, 40)
    xr, Tr = _reference(cosmo, [1.0], zs)
    return zs, xr[:, 0], Tr[:, 0]


def test_second_order_convergence_uniform_box(cosmo, uniform):
    zs, xr, Tr = uniform
    ex, eT = {}, {}
    for n_sub in (1, 2, 4):
        x, T, _ = _history(cosmo, [1.0], 1, zs, n_sub, "trbdf2")
        ex[n_sub] = np.max(np.abs(x[:, 0] / xr - 1))
        eT[n_sub] = np.max(np.abs(T[:, 0] / Tr - 1))
    for e in (ex, eT):
        assert 3.6 < e[1] / e[2] < 4.5 and 3.6 < e[2] / e[4] < 4.5
    assert ex[4] < 5e-4 and eT[4] < 1e-6
    # backward Euler with eight times the substeps is still less accurate
    xb, _, _ = _history(cosmo, [1.0], 1, zs, 8, "be")
    assert ex[1] < 0.5 * np.max(np.abs(xb[:, 0] / xr - 1))


def test_second_order_convergence_two_zones(cosmo):
    b = PV["two_zone_b"]["value"]
    dz = [1 + math.sqrt(b), 1 - math.sqrt(b)]
    zs = z_schedule(1600.0, 800.0, 30)
    xr, Tr = _reference(cosmo, dz, zs)
    cells = np.array([dz[0], dz[1]] * 4)
    errs = {}
    for n_sub in (1, 2, 4):
        x, _, Xe = _history(cosmo, cells, 2, zs, n_sub, "trbdf2")
        errs[n_sub] = [np.max(np.abs(x[:, zone] / xr[:, zone] - 1)) for zone in (0, 1)]
    for zone in (0, 1):
        assert 3.5 < errs[1][zone] / errs[2][zone] < 4.6
        assert 3.5 < errs[2][zone] / errs[4][zone] < 4.6
        assert errs[4][zone] < 1e-3


def test_tally_mode_reduces_to_full_mixing(cosmo):
    n = 4
    rng = np.random.default_rng(3)
    d = rng.lognormal(0.0, 0.6, n ** 3)
    z0, z1 = 1300.0, 1280.0
    x = O.saha_xe(cosmo, z0, d) * 0.97
    T = np.full(d.size, O.background(cosmo, z0)["Tg"])
    tally = np.round(1e6 * d * (1 - x)).astype(np.uint32)
    wf = O.rec_step(cosmo, n, z0, z1, d, x, T, mixing="full", n_sub=2, integrator="trbdf2")
    wt = O.rec_step(cosmo, n, z0, z1, d, x, T, tally=tally, mixing="tally", n_sub=2, integrator="trbdf2")
    np.testing.assert_allclose(wt[0], wf[0], rtol=5e-6)  # tallies are rounded to integers
    np.testing.assert_allclose(wt[1], wf[1], rtol=1e-9)


def test_end_state_identities(cosmo):
    n = 3
    rng = np.random.default_rng(5)
    d = rng.lognormal(0.0, 0.8, n ** 3)
    z0, z1 = 1150.0, 1140.0
    x = O.saha_xe(cosmo, z0, d) * rng.uniform(0.8, 1.0, d.size)
    T = O.background(cosmo, z0)["Tg"] * (1 + 0.01 * rng.standard_normal(d.size))
    U = rng.standard_normal((d.size, 3))
    x1, T1, U1, em, st = O.rec_step(cosmo, n, z0, z1, d, x, T, U=U, mixing="full", integrator="trbdf2")
    bg = O.background(cosmo, z1)
    nH = bg["nH"] * d
    al = np.array([O.rates(cosmo, z1, t)["alpha"] for t in T1])
    assert st["lam"] == pytest.approx((al * (nH * x1) ** 2).sum() / (nH * (1 - x1)).sum(), rel=1e-10)
    np.testing.assert_allclose(em, al * (nH * x1) ** 2, rtol=1e-13)
    assert st["Xe"] == pytest.approx((d * x1).sum() / d.sum(), rel=1e-14)
    # drag: the same damping factor for all three components, between the rates at both ends
    fac = U1 / U
    np.testing.assert_allclose(fac, fac[:, :1].repeat(3, axis=1), rtol=1e-14)
    assert np.all((fac > 0) & (fac < 1))


def test_rejects_modes_without_a_global_rate(cosmo):
    d = np.ones(1)
    with pytest.raises(ValueError):
        O.rec_step(cosmo, 1, 1300.0, 1290.0, d, d * 0.5, d * 3000, mixing="local", integrator="trbdf2")


def test_stiff_inhomogeneous_box_self_convergence(cosmo):
    """A lognormal box (sigma 1) near z = 1600, where the per-cell mixing term is
    stiff (gross rates times the step ~ 40) and stage explicit parts go negative,
    started from the state a backward-Euler run from Saha at z = 1800 reaches:
    every step succeeds and the self-convergence against a 64-substep solution
    is second order, with errors far below backward Euler's."""
    from paper_2312_11448_gb300.inputs import density_field
    n = 6
    d = density_field(n, 1.0, 2).ravel()
    zpre = z_schedule(1800.0, 1650.0, 15)
    x = O.saha_xe(cosmo, zpre[0], d)
    T = np.full(d.size, O.background(cosmo, zpre[0])["Tg"])
    for s in range(len(zpre) - 1):
        x, T, _, _, _ = O.rec_step(cosmo, n, zpre[s], zpre[s + 1], d, x, T, mixing="full", n_sub=4)
    zs = z_schedule(1650.0, 1500.0, 6)

    def run(n_sub, integrator="trbdf2"):
        xx, TT = x.copy(), T.copy()
        for s in range(len(zs) - 1):
            xx, TT, _, _, _ = O.rec_step(cosmo, n, zs[s], zs[s + 1], d, xx, TT, mixing="full", n_sub=n_sub,
                                         integrator=integrator)
        return xx

    ref = run(64)
    e = {k: np.max(np.abs(run(k) / ref - 1)) for k in (1, 2, 4)}
    assert 3.5 < e[1] / e[2] < 4.5 and 3.5 < e[2] / e[4] < 4.5
    assert e[1] < 0.01 * np.max(np.abs(run(1, "be") / ref - 1))
