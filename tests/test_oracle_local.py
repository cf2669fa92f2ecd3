"""Oracle pins for the no-mixing (local) limit of Sec. III.A.2: recombination
per cell by Eq. (rec) with the cell's own n_e, n_1s and the Ly-alpha escape
rate of Eq. (R-alpha) with H -> H + div v / 3.

Checks, none of which re-types the oracle's formulas:
  * the discrete velocity divergence against the closed form for sinusoidal
    fields (each component differentiated along its own axis, periodic wrap,
    comoving-to-physical factor 1 + z);
  * a uniform box: the local and the full-mixing updates are the same equation
    (the full-mixing mode is pinned against the standard TLA elsewhere);
  * locality: a cell's update depends only on its own state and on the
    velocities of its six neighbours;
  * converging flows faster than the expansion: no escape, results independent
    of how strongly the flow converges; diverging flows recombine faster;
  * one cell with a diverging flow against a stiff library ODE integration of
    Eq. (rec) + Eq. (Cfactor) with H + div v/3, Eq. (Tb-evolution) and the
    Compton + Hubble damping of the velocity (first-order convergence of the
    backward-Euler substeps, Richardson extrapolation close to the ODE).
"""
import json
import math
import os

import numpy as np
import pytest
from scipy.integrate import solve_ivp

import oracle as O

GOLD = os.path.join(os.path.dirname(__file__), "golden")
TB = json.load(open(os.path.join(GOLD, "textbook_values.json")))
KPC_M = 3.0856775814913673e19
_KC0 = 8 * TB["sigma_T_m2"] * TB["a_rad_SI"] / (3 * TB["m_e_kg"] * TB["c_m_s"])
_KD0 = 4 * TB["sigma_T_m2"] * TB["a_rad_SI"] * (1 - 0.24) / (3 * TB["c_m_s"] * TB["m_H_kg"])
_FHE = 0.24 * 1.00782503 / (0.76 * 4.002602)


def _grid(n):
    c = np.arange(n ** 3)
    return c % n, (c // n) % n, c // (n * n)


def test_divergence_closed_form(cosmo):
    n, z = 12, 1200.0
    ix, iy, iz = _grid(n)
    h = 24.0 * KPC_M / n
    U = np.zeros((n ** 3, 3))
    a, b, c = 2.0, -1.5, 0.7
    U[:, 0] = a * np.sin(2 * np.pi * 1 * ix / n) + 3.0 * np.sin(2 * np.pi * iy / n)  # plus a shear along y
    U[:, 1] = b * np.cos(2 * np.pi * 2 * iy / n)
    U[:, 2] = c * np.sin(2 * np.pi * 3 * iz / n)
    # sin(k(i+1)) - sin(k(i-1)) = 2 cos(ki) sin(k);  cos(k(i+1)) - cos(k(i-1)) = -2 sin(ki) sin(k)
    k1, k2, k3 = 2 * np.pi / n, 4 * np.pi / n, 6 * np.pi / n
    expect = (1 + z) * 1e3 / h * (a * np.cos(k1 * ix) * np.sin(k1) - b * np.sin(k2 * iy) * np.sin(k2)
                                  + c * np.cos(k3 * iz) * np.sin(k3))
    got = O.divergence(cosmo, n, z, U)
    np.testing.assert_allclose(got, expect, rtol=1e-12, atol=1e-12 * np.abs(expect).max())


@pytest.mark.parametrize("z_from,z_to", [(1500.0, 1480.0), (1100.0, 1090.0), (850.0, 840.0)])
def test_uniform_box_local_equals_full(cosmo, z_from, z_to):
    n = 2
    d = np.ones(n ** 3)
    x = O.saha_xe(cosmo, z_from, d) * 0.98
    T = np.full(n ** 3, O.background(cosmo, z_from)["Tg"])
    out = {m: O.rec_step(cosmo, n, z_from, z_to, d, x, T, U=np.zeros((n ** 3, 3)), mixing=m, n_sub=2)
           for m in ("full", "local")}
    for k in (0, 1, 3):
        np.testing.assert_allclose(out["local"][k], out["full"][k], rtol=2e-11)
    assert out["local"][4]["C"] == pytest.approx(out["full"][4]["C"], rel=1e-12)


def test_cells_are_independent(cosmo):
    n, z0, z1 = 4, 1200.0, 1185.0
    rng = np.random.default_rng(1)
    d = rng.lognormal(0.0, 0.7, n ** 3)
    x = O.saha_xe(cosmo, z0, d) * rng.uniform(0.9, 1.0, n ** 3)
    T = O.background(cosmo, z0)["Tg"] * rng.uniform(0.98, 1.02, n ** 3)
    xb, Tb, _, eb, _ = O.rec_step(cosmo, n, z0, z1, d, x, T, U=np.zeros((n ** 3, 3)), mixing="local")
    for i in (0, 17, 63):  # a one-cell box with the cell's own state
        x1, T1, _, e1, _ = O.rec_step(cosmo, 1, z0, z1, d[i:i + 1], x[i:i + 1], T[i:i + 1],
                                      U=np.zeros((1, 3)), mixing="local")
        assert x1[0] == xb[i] and T1[0] == Tb[i] and e1[0] == eb[i]
    # velocities only matter through the six neighbours of each cell
    U = rng.normal(0.0, 1.0, (n ** 3, 3))
    ref = O.rec_step(cosmo, n, z0, z1, d, x, T, U=U, mixing="local")[0]
    U2 = U.copy()
    ix, iy, iz = _grid(n)
    far = (ix == 2) & (iy == 2) & (iz == 2)  # not a neighbour of cell (0,0,0)
    U2[far] += 5.0
    got = O.rec_step(cosmo, n, z0, z1, d, x, T, U=U2, mixing="local")[0]
    assert got[0] == ref[0]
    changed = np.nonzero(got != ref)[0]
    assert set(changed) <= set(np.nonzero((np.abs(ix - 2) + np.abs(iy - 2) + np.abs(iz - 2)) <= 1)[0]) | {
        int(np.nonzero(far)[0][0])}


def test_converging_and_diverging_flows(cosmo):
    n, z0, z1 = 8, 1100.0, 1095.0
    d = np.ones(n ** 3)
    x = np.full(n ** 3, 0.2)  # well above the equilibrium value: recombining
    T = np.full(n ** 3, O.background(cosmo, z0)["Tg"])
    H = O.background(cosmo, z0)["H"]
    ix = _grid(n)[0]

    def run(amp):
        U = np.zeros((n ** 3, 3))
        U[:, 0] = amp * np.sin(2 * np.pi * ix / n)
        return O.rec_step(cosmo, n, z0, z1, d, x, T, U=U, mixing="local")[0], O.divergence(cosmo, n, z1, U)

    x0, _ = run(0.0)
    xa, div_a = run(40.0)
    xb, div_b = run(80.0)
    clamped = (div_a / 3 < -2 * H) & (div_b / 3 < -2 * H)
    assert clamped.any()
    assert np.array_equal(xa[clamped], xb[clamped])  # no escape either way
    # the net rate is C times the same bracket: no escape is the slowest
    # recombination, a diverging flow speeds it up
    assert np.all(xa[clamped] > x0[clamped])
    out = div_a > 0.3 * H
    assert np.all(xb[out] < xa[out]) and np.all(xa[out] < x0[out])


def test_one_cell_with_flow_against_ode(cosmo):
    """Cell (0,0,0) of an 8^3 box, U_x = A sin(2 pi ix/n): div v = div0 at the
    start of the step, decaying with the velocity as dU/dt = -(alpha_C + H) U."""
    n, z0, z1 = 8, 1150.0, 1100.0
    ix = _grid(n)[0]
    H0 = O.background(cosmo, z0)["H"]
    U = np.zeros((n ** 3, 3))
    A0 = 1.0
    U[:, 0] = A0 * np.sin(2 * np.pi * ix / n)
    div_unit = O.divergence(cosmo, n, 1.0 - 1.0, U)[0]  # (1+z) = 1: div per unit amplitude, comoving
    amp = 6.0 * H0 / (div_unit * (1 + z0))  # div v / 3 = 2 H at the start
    U *= amp
    d = np.ones(n ** 3)
    x0 = O.saha_xe(cosmo, z0, d) * 0.9
    T0 = np.full(n ** 3, O.background(cosmo, z0)["Tg"])

    def rhs(y, s):
        z = math.expm1(y)
        bg = O.background(cosmo, z)
        H, nH, Tg = bg["H"], bg["nH"], bg["Tg"]
        x, T, u = s
        rg = O.rates(cosmo, z, Tg)
        al = O.rates(cosmo, z, T)["alpha"]
        div = div_unit * amp * u * (1 + z)
        Heff = max(H + div / 3, 0.0)
        R = rg["K_R"] * Heff / H / ((1 - x) * nH)  # K_R = 8 pi H / lambda^3 at this z
        C = (rg["Lambda"] + R) / (rg["beta"] + rg["Lambda"] + R)
        dxdt = -C * (al * nH * x * x - rg["beta"] * rg["e_alpha"] * (1 - x))
        dTdt = -2 * H * T + _KC0 * Tg ** 4 * x / (1 + _FHE + x) * (Tg - T)
        dudt = -(_KD0 * Tg ** 4 * x + H) * u
        return -np.array([dxdt, dTdt, dudt]) / H

    sol = solve_ivp(rhs, (math.log1p(z0), math.log1p(z1)), [x0[0], T0[0], 1.0], method="Radau", rtol=1e-11,
                    atol=1e-14)
    assert sol.success
    xr = sol.y[0, -1]
    err, got = {}, {}
    for ns in (4, 16, 64):
        xo = O.rec_step(cosmo, n, z0, z1, d, x0, T0, U=U, mixing="local", n_sub=ns)[0][0]
        got[ns], err[ns] = xo, abs(xo / xr - 1)
    assert 3.3 < err[4] / err[16] < 4.7 and 3.3 < err[16] / err[64] < 4.7
    assert abs(((4 * got[64] - got[16]) / 3) / xr - 1) < 0.05 * err[64]
    # the flow matters: without it the cell ends elsewhere
    xs = O.rec_step(cosmo, n, z0, z1, d, x0, T0, U=np.zeros_like(U), mixing="local", n_sub=64)[0][0]
    assert abs(xs / xr - 1) > 5 * err[64]


# ---- partial mixing: f times the full-mixing rate plus (1 - f) times the local one
def _box_with_flow(n, z, seed):
    rng = np.random.default_rng(seed)
    d = rng.lognormal(0.0, 0.6, n ** 3)
    x = np.clip(O.saha_xe(cosmo_default(), z, d) * rng.uniform(0.8, 1.2, n ** 3), 1e-6, 0.999)
    T = O.background(cosmo_default(), z)["Tg"] * rng.uniform(0.98, 1.02, n ** 3)
    U = rng.normal(0.0, 5.0, (n ** 3, 3))
    return d, x, T, U


def cosmo_default():
    return O.default_cosmo()


def test_partial_mixing_end_points(cosmo):
    """f = 1 is the full-mixing update and f = 0 the local one, exactly."""
    n, z0, z1 = 6, 1250.0, 1240.0
    d, x, T, U = _box_with_flow(n, z0, 3)
    full = O.rec_step(cosmo, n, z0, z1, d, x, T, U=U, mixing="full")
    p1 = O.rec_step(cosmo, n, z0, z1, d, x, T, U=U, mixing="partial", f_alpha=1.0)
    loc = O.rec_step(cosmo, n, z0, z1, d, x, T, U=U, mixing="local")
    p0 = O.rec_step(cosmo, n, z0, z1, d, x, T, U=U, mixing="partial", f_alpha=0.0)
    for k in (0, 1, 2, 3):
        assert np.array_equal(p1[k], full[k]) and np.array_equal(p0[k], loc[k])


def test_partial_mixing_uniform_box(cosmo):
    n = 2
    d = np.ones(n ** 3)
    x = O.saha_xe(cosmo, 1200.0, d) * 0.97
    T = np.full(n ** 3, O.background(cosmo, 1200.0)["Tg"])
    full = O.rec_step(cosmo, n, 1200.0, 1190.0, d, x, T, U=np.zeros((n ** 3, 3)), mixing="full")[0]
    part = O.rec_step(cosmo, n, 1200.0, 1190.0, d, x, T, U=np.zeros((n ** 3, 3)), mixing="partial",
                      f_alpha=0.3)[0]
    np.testing.assert_allclose(part, full, rtol=2e-11)


def test_partial_mixing_two_zones_against_ode(cosmo):
    """Two equal-volume zones Delta = 1 +- 0.7 at rest (div v = 0): each zone's
    rate is f times Eq. (dotne-mix) plus (1 - f) times Eq. (rec) with the zone's
    own n_1s, integrated by a stiff library solver; the backward-Euler history
    converges to it at first order."""
    from paper_2312_11448_gb300.inputs import z_schedule
    f = 0.4
    dz = np.array([1.7, 0.3])
    zs = z_schedule(1400.0, 1000.0, 8)

    def rhs(y, s):
        z = math.expm1(y)
        bg = O.background(cosmo, z)
        H, nHb, Tg = bg["H"], bg["nH"], bg["Tg"]
        x, T = s[:2], s[2:]
        rg = O.rates(cosmo, z, Tg)
        al = np.array([O.rates(cosmo, z, t)["alpha"] for t in T])
        nH = nHb * dz
        ne2, n1s = (x * nH) ** 2, (1 - x) * nH
        Rmix = rg["K_R"] / n1s.mean()
        Cm = (rg["Lambda"] + Rmix) / (rg["beta"] + rg["Lambda"] + Rmix)
        lam = (al * ne2).mean() / n1s.mean()
        full = -Cm * (al * ne2 - rg["beta"] * n1s * rg["e_alpha"]) - (1 - Cm) * (al * ne2 - n1s * lam)
        Rl = rg["K_R"] / n1s
        Cl = (rg["Lambda"] + Rl) / (rg["beta"] + rg["Lambda"] + Rl)
        local = -Cl * (al * ne2 - rg["beta"] * n1s * rg["e_alpha"])
        dxdt = (f * full + (1 - f) * local) / nH
        dTdt = -2 * H * T + _KC0 * Tg ** 4 * x / (1 + _FHE + x) * (Tg - T)
        return -np.concatenate([dxdt, dTdt]) / H

    x0 = O.saha_xe(cosmo, zs[0], dz)
    T0 = np.full(2, O.background(cosmo, zs[0])["Tg"])
    ys = np.log1p(zs)
    sol = solve_ivp(rhs, (ys[0], ys[-1]), np.concatenate([x0, T0]), method="Radau", t_eval=ys, rtol=1e-10,
                    atol=1e-13)
    assert sol.success
    xr = sol.y[:2, -1]
    cells = np.array([dz[0], dz[1]] * 4)  # a 2^3 box, four cells of each zone

    def history(n_sub):
        x = np.array([x0[0], x0[1]] * 4)
        T = np.full(8, T0[0])
        for s in range(len(zs) - 1):
            x, T, _, _, _ = O.rec_step(cosmo, 2, zs[s], zs[s + 1], cells, x, T, U=np.zeros((8, 3)),
                                       mixing="partial", f_alpha=f, n_sub=n_sub)
        return x[:2]

    got = {ns: history(ns) for ns in (4, 16, 64)}
    err = {ns: np.max(np.abs(got[ns] / xr - 1)) for ns in got}
    assert 3.3 < err[4] / err[16] < 4.7 and 3.3 < err[16] / err[64] < 4.7
    assert np.max(np.abs(((4 * got[64] - got[16]) / 3) / xr - 1)) < 0.1 * err[64]
