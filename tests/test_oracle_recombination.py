"""Oracle pins for the per-cell recombination step (Sec. III.A, Sec. IV).

The oracle advances x_e by a backward-Euler step whose 2s population comes
from a self-consistent global lambda = <alpha n_e^2>/<n_1s> (Newton).  These
tests check that scheme against independent formulations:
  * a uniform box against the standard three-level atom, Eq. (rec) with
    Eq. (Cfactor), integrated by a stiff library ODE solver;
  * the two-zone model of Sec. IV.C against Eq. (dotne-mix) for each zone,
    integrated the same way;
  * exact algebraic properties (global net rate, mixing term averaging to zero,
    full mixing == tally mode with tallies proportional to n_1s).
"""
import json
import math
import os

import numpy as np
import pytest
from scipy.integrate import solve_ivp

import oracle as O
from paper_2312_11448_gb300.inputs import z_schedule, density_field

GOLD = os.path.join(os.path.dirname(__file__), "golden")
PV = json.load(open(os.path.join(GOLD, "paper_values.json")))
TB = json.load(open(os.path.join(GOLD, "textbook_values.json")))

# Compton coupling written from Eq. (Tb-evolution) with textbook constants:
# gamma_C = 8 sigma_T a_R T^4 x / (3 m_e c (1 + f_He + x)).
_KC0 = 8 * TB["sigma_T_m2"] * TB["a_rad_SI"] / (3 * TB["m_e_kg"] * TB["c_m_s"])
_FHE = 0.24 * 1.00782503 / (0.76 * 4.002602)


def _zone_rhs(cosmo, deltas):
    """d/dy of (x_1..x_k, T_1..T_k), y = ln(1+z), for equal-volume zones with full
    Ly-alpha mixing, Eq. (dotne-mix) per zone:
      n_dot_e = -C (alpha n_e^2 - beta n_1s e_a) - (1-C) alpha (n_e^2 - n_1s <n_e^2>/<n_1s>)
    (with alpha varying per zone, <alpha n_e^2> replaces alpha <n_e^2>), and
    Eq. (Tb-evolution) with the adiabatic term -2 H T."""
    k = len(deltas)
    deltas = np.asarray(deltas, float)

    def rhs(y, s):
        z = math.expm1(y)
        bg = O.background(cosmo, z)
        H, nHb, Tg = bg["H"], bg["nH"], bg["Tg"]
        x, T = s[:k], s[k:]
        rg = O.rates(cosmo, z, Tg)
        al = np.array([O.rates(cosmo, z, t)["alpha"] for t in T])
        nH = nHb * deltas
        ne2 = (x * nH) ** 2
        n1s = (1 - x) * nH
        Rmix = rg["K_R"] / n1s.mean()
        C = (rg["Lambda"] + Rmix) / (rg["beta"] + rg["Lambda"] + Rmix)
        lam = (al * ne2).mean() / n1s.mean()
        ndot = -C * (al * ne2 - rg["beta"] * n1s * rg["e_alpha"]) - (1 - C) * (al * ne2 - n1s * lam)
        dxdt = ndot / nH
        gam = _KC0 * Tg ** 4 * x / (1 + _FHE + x)
        dTdt = -2 * H * T + gam * (Tg - T)
        return -np.concatenate([dxdt, dTdt]) / H

    return rhs


def _reference(cosmo, deltas, zs):
    k = len(deltas)
    x0 = O.saha_xe(cosmo, zs[0], np.asarray(deltas, float))
    T0 = np.full(k, O.background(cosmo, zs[0])["Tg"])
    ys = np.log1p(zs)
    sol = solve_ivp(_zone_rhs(cosmo, deltas), (ys[0], ys[-1]), np.concatenate([x0, T0]), method="Radau",
                    t_eval=ys, rtol=1e-9, atol=1e-12)
    assert sol.success
    return sol.y[:k].T, sol.y[k:].T  # [node, zone]


def _oracle_history(cosmo, cells_delta, n, zs, n_sub):
    d = np.asarray(cells_delta, float)
    x = O.saha_xe(cosmo, zs[0], d)
    T = np.full(d.size, O.background(cosmo, zs[0])["Tg"])
    xs, Ts, Cs, Xe = [x.copy()], [T.copy()], [], [float((d * x).sum() / d.sum())]
    for s in range(len(zs) - 1):
        x, T, _, _, st = O.rec_step(cosmo, n, zs[s], zs[s + 1], d, x, T, mixing="full", n_sub=n_sub)
        xs.append(x.copy()); Ts.append(T.copy()); Cs.append(st["C"]); Xe.append(st["Xe"])
    return np.array(xs), np.array(Ts), np.array(Cs), np.array(Xe)


@pytest.fixture(scope="module")
def uniform_reference(cosmo):
    zs = z_schedule(1700.0, 750.0, 40)
    xr, Tr = _reference(cosmo, [1.0], zs)
    return zs, xr[:, 0], Tr[:, 0]


def test_uniform_box_converges_to_standard_tla(cosmo, uniform_reference):
    """Homogeneous limit: full mixing reduces to Eq. (rec) (Sec. IV.A.2).  The
    backward-Euler history converges to the ODE solution at first order, and
    its Richardson extrapolation matches the ODE closely."""
    zs, xr, Tr = uniform_reference
    ex, eT, hist = {}, {}, {}
    for n_sub in (2, 8, 32):
        x, T, _, _ = _oracle_history(cosmo, [1.0], 1, zs, n_sub)
        hist[n_sub] = (x[:, 0], T[:, 0])
        ex[n_sub] = np.max(np.abs(x[:, 0] / xr - 1))
        eT[n_sub] = np.max(np.abs(T[:, 0] / Tr - 1))
    for e in (ex, eT):
        assert 3.5 < e[2] / e[8] < 4.6 and 3.5 < e[8] / e[32] < 4.6
    x_rich = (4 * hist[32][0] - hist[8][0]) / 3
    T_rich = (4 * hist[32][1] - hist[8][1]) / 3
    assert np.max(np.abs(x_rich / xr - 1)) < 3e-4
    assert np.max(np.abs(T_rich / Tr - 1)) < 1e-6


def test_paper_coarse_values(cosmo):
    """X_e ~ 0.1 at z ~ 1000, ~1e-2 at z ~ 900 (Sec. VI); C ~ 1e-2 near
    z ~ 1100 and C -> 1 below z ~ 800 (Sec. III.A.1)."""
    zs = np.array([1800.0, 1500.0, 1300.0, 1200.0, 1150.0, 1100.0, 1050.0, 1000.0, 950.0, 900.0, 850.0, 800.0, 750.0])
    zs = np.concatenate([z_schedule(a, b, 30)[:-1] for a, b in zip(zs[:-1], zs[1:])] + [zs[-1:]])
    x, T, C, Xe = _oracle_history(cosmo, [1.0], 1, zs, 1)
    at = lambda z0: int(np.argmin(np.abs(zs - z0)))
    lo, hi = PV["Xe_at_1000"]["band"]; assert lo < Xe[at(1000)] < hi
    lo, hi = PV["Xe_at_900"]["band"]; assert lo < Xe[at(900)] < hi
    lo, hi = PV["C_near_1100"]["band"]; assert lo < C[at(1100) - 1] < hi
    lo, hi = PV["C_below_800"]["band"]; assert lo < C[at(790) - 1] <= hi


def test_two_zone_full_mixing(cosmo):
    """Sec. IV.C: equiprobable zones Delta = 1 +- sqrt(b), b = 0.5, full mixing.
    The 2^3 box holds four cells of each zone."""
    b = PV["two_zone_b"]["value"]
    dz = [1 + math.sqrt(b), 1 - math.sqrt(b)]
    zs = z_schedule(1600.0, 800.0, 30)
    xr, Tr = _reference(cosmo, dz, zs)
    cells = np.array([dz[0], dz[1]] * 4)
    x8, _, _, Xe8 = _oracle_history(cosmo, cells, 2, zs, 8)
    x, T, _, Xe = _oracle_history(cosmo, cells, 2, zs, 32)
    x_rich, Xe_rich = (4 * x - x8) / 3, (4 * Xe - Xe8) / 3
    Xr = 0.5 * (dz[0] * xr[:, 0] + dz[1] * xr[:, 1])
    for zone in (0, 1):
        err32 = np.max(np.abs(x[:, zone] / xr[:, zone] - 1))
        err8 = np.max(np.abs(x8[:, zone] / xr[:, zone] - 1))
        assert 3.5 < err8 / err32 < 4.6
        assert np.max(np.abs(x_rich[:, zone] / xr[:, zone] - 1)) < 5e-4
    assert np.max(np.abs(Xe_rich / Xr - 1)) < 5e-4
    # clumping speeds recombination up: X_e below the homogeneous history once x < 0.5
    xu, _, _, Xu = _oracle_history(cosmo, [1.0], 1, zs, 32)
    late = zs < 1150
    assert np.all(Xe[late] < Xu[late])


def _step_check_identities(cosmo, n, d, x, T, z_from, z_to, tally=None, mixing="full"):
    x1, T1, _, em, st = O.rec_step(cosmo, n, z_from, z_to, d, x, T, tally=tally, mixing=mixing)
    bg = O.background(cosmo, z_to)
    nH = bg["nH"] * d
    al = np.array([O.rates(cosmo, z_to, t)["alpha"] for t in T1])
    r = O.rates(cosmo, z_to, bg["Tg"])
    ne2, n1s = (nH * x1) ** 2, nH * (1 - x1)
    # lambda = <alpha n_e^2>/<n_1s> at the end state
    assert st["lam"] == pytest.approx((al * ne2).sum() / n1s.sum(), rel=1e-12)
    # emission weight alpha_e n_e^2
    np.testing.assert_allclose(em, al * ne2, rtol=1e-13)
    return x1, T1, st, nH, al, r, ne2, n1s


def test_global_rate_and_mixing_term_average(cosmo):
    """With full mixing the mixing term of Eq. (dotne-mix) averages to zero
    (Sec. IV.B), so the box-total electron change over the backward-Euler step is
    -C (sum alpha n_e^2 - beta e_a sum n_1s) at the end state."""
    n = 4
    d = density_field(n, 1.0, 3).ravel()
    x = O.saha_xe(cosmo, 1250.0, d) * 0.9
    T = np.full(n ** 3, O.background(cosmo, 1250.0)["Tg"]) * (1 + 0.01 * np.sin(np.arange(n ** 3)))
    x1, T1, st, nH, al, r, ne2, n1s = _step_check_identities(cosmo, n, d, x, T, 1250.0, 1240.0)
    lhs = (nH * (x1 - x)).sum() / st["dt"]
    rhs = -st["C"] * ((al * ne2).sum() - r["beta"] * r["e_alpha"] * n1s.sum())
    assert lhs == pytest.approx(rhs, rel=1e-9)
    mix = (1 - st["C"]) * (al * ne2 - n1s * (al * ne2).sum() / n1s.sum())
    assert abs(mix.sum()) < 1e-12 * np.abs(al * ne2).sum()


def test_tally_mode_equals_full_when_tallies_follow_n1s(cosmo):
    """If absorptions per neutral atom are uniform (tally_i proportional to
    Delta_i (1 - x_i)), the local 2s population is the full-mixing one."""
    n = 2
    d = np.array([0.5, 1.0, 1.5, 2.0, 0.25, 1.25, 0.75, 0.75])
    x = np.full(8, 0.5)
    T = np.full(8, 3500.0)
    tally = (d * 8).astype(np.uint32)  # = 16 Delta (1 - x)
    xf, Tf, _, _, sf = O.rec_step(cosmo, n, 1300.0, 1290.0, d, x, T, mixing="full")
    xt, Tt, _, _, st = O.rec_step(cosmo, n, 1300.0, 1290.0, d, x, T, tally=tally, mixing="tally")
    np.testing.assert_allclose(xt, xf, rtol=1e-13)
    np.testing.assert_allclose(Tt, Tf, rtol=1e-15)
    # only the normalised fractions matter
    x3, _, _, _, _ = O.rec_step(cosmo, n, 1300.0, 1290.0, d, x, T, tally=3 * tally, mixing="tally")
    np.testing.assert_allclose(x3, xt, rtol=1e-13)


def test_tally_mode_local_photoionisation_follows_tallies(cosmo):
    """A cell that absorbed no Ly-alpha packets has no 2s population: it can only
    recombine; a cell with more absorptions per atom stays more ionised."""
    n = 2
    d = np.ones(8)
    x = np.full(8, 0.3)
    T = np.full(8, 3000.0)
    tally = np.array([0, 10, 10, 10, 10, 10, 10, 20], dtype=np.uint32)
    x1, _, _, _, _ = O.rec_step(cosmo, n, 1100.0, 1095.0, d, x, T, tally=tally, mixing="tally")
    assert x1[0] < x1[1] < x1[7]
    # pure recombination in cell 0: backward Euler of dx/dt = -alpha n_H x^2
    bg = O.background(cosmo, 1095.0)
    al = O.rates(cosmo, 1095.0, O.rec_step(cosmo, n, 1100.0, 1095.0, d, x, T, tally=tally)[1][0])["alpha"]
    A = O.dt(cosmo, 1100.0, 1095.0) * al * bg["nH"]
    assert x1[0] == pytest.approx((-1 + math.sqrt(1 + 4 * A * 0.3)) / (2 * A), rel=1e-12)


def test_empty_tallies_fall_back_to_full_mixing(cosmo):
    n = 2
    d = density_field(n, 0.5, 1).ravel()
    x = np.full(8, 0.4)
    T = np.full(8, 3200.0)
    xa, *_ = O.rec_step(cosmo, n, 1200.0, 1190.0, d, x, T, tally=np.zeros(8, np.uint32), mixing="tally")
    xb, *_ = O.rec_step(cosmo, n, 1200.0, 1190.0, d, x, T, mixing="full")
    np.testing.assert_array_equal(xa, xb)
