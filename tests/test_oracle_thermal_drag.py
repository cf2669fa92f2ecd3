"""Oracle pins for the temperature update (Eq. Tb-evolution) and the Compton
drag on the peculiar velocity (Eq. alpha-def, Eq. momentum)."""
import json
import math
import os

import numpy as np
import pytest

import oracle as O
from paper_2312_11448_gb300.inputs import z_schedule

TB = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "textbook_values.json")))


def _run(cosmo, d, x, T, U, zs, n_sub=1, mixing="full"):
    for s in range(len(zs) - 1):
        x, T, U, _, st = O.rec_step(cosmo, 1, zs[s], zs[s + 1], d, x, T, U=U, mixing=mixing, n_sub=n_sub)
    return x, T, U, st


def test_adiabatic_cooling_without_electrons(cosmo):
    """With no free electrons the gas cools adiabatically, T ~ (1+z)^2 for a
    static comoving field (the reading of the adiabatic term of Eq. Tb-evolution)."""
    zs = z_schedule(300.0, 200.0, 20)
    d = np.ones(1)
    x, T, _, _ = _run(cosmo, d, np.zeros(1), np.array([500.0]), None, zs, n_sub=64)
    assert x[0] < 1e-12
    assert T[0] / 500.0 == pytest.approx((201.0 / 301.0) ** 2, rel=2e-3)


def test_compton_lag_matches_tight_coupling(cosmo):
    """Tight coupling: T_b trails T_gamma by (T_gamma - T_b)/T_gamma ~ H / gamma_C,
    gamma_C = 8 sigma_T a_R T^4 x / (3 m_e c (1 + f_He + x)) (Eq. Tb-evolution)."""
    zs = z_schedule(1300.0, 1200.0, 50)
    d = np.ones(1)
    x0 = np.array([0.6])
    T0 = np.array([O.background(cosmo, 1300.0)["Tg"] * 1.2])  # start hot: it must relax
    x, T, _, _ = _run(cosmo, d, x0, T0, None, zs, n_sub=16)
    bg = O.background(cosmo, 1200.0)
    Tg = bg["Tg"]
    gam = 8 * TB["sigma_T_m2"] * TB["a_rad_SI"] * Tg ** 4 * x[0] / (3 * TB["m_e_kg"] * TB["c_m_s"] * (1 + 0.0795 + x[0]))
    lag = (Tg - T[0]) / Tg
    assert lag == pytest.approx(bg["H"] / gam, rel=0.05)


def test_uniform_heating_raises_temperature(cosmo):
    """The uniform heating term 2 Gamma / (3 n_tot) of Eq. (Tb-evolution):
    with negligible Compton coupling the extra temperature over a short interval
    is 2 Gamma dt / (3 k n_tot), diluted adiabatically by ((1+z_end)/(1+z))^2."""
    za, zb = 350.0, 345.0
    zs = z_schedule(za, zb, 4)
    d = np.array([1.0])
    x0 = np.array([1e-9])
    T0 = np.array([800.0])
    heat = 1e-16  # eV/s per H atom
    _, Tn, _, _ = _run(cosmo, d, x0, T0, None, zs, n_sub=16)
    _, Th, _, _ = _run(O.default_cosmo(heating=heat), d, x0, T0, None, zs, n_sub=16)
    tot = O.dt(cosmo, za, zb)
    dil = ((1 + zb) / (1 + 0.5 * (za + zb))) ** 2
    expect = 2 * heat * TB["eV_J"] / (3 * TB["k_B"] * (1 + 0.0795)) * tot * dil
    assert (Th[0] - Tn[0]) == pytest.approx(expect, rel=2e-3)
    # uniform Gamma heats low-density gas more per particle
    _, Tl, _, _ = _run(O.default_cosmo(heating=heat), np.array([0.5]), x0, T0, None, zs, n_sub=16)
    assert (Tl[0] - Tn[0]) == pytest.approx(2 * (Th[0] - Tn[0]), rel=1e-6)


def test_peculiar_velocity_decays_as_one_over_a_without_drag(cosmo):
    zs = z_schedule(300.0, 200.0, 10)
    U = np.array([[1.0, -2.0, 0.5]])
    _, _, U1, _ = _run(cosmo, np.ones(1), np.zeros(1), np.array([600.0]), U, zs, n_sub=64)
    np.testing.assert_allclose(U1 / U, 201.0 / 301.0, rtol=2e-3)


def test_compton_drag_rate_is_eq_alpha_def(cosmo):
    """alpha = (4/3) n_e sigma_T rho_gamma / rho_b (Eq. alpha-def), with rho_gamma
    the photon mass density a_R T^4/c^2 and rho_b = n_H m_H/(1 - Y_p)."""
    za, zb = 1500.0, 1499.0
    d = np.array([2.0])
    x0 = np.array([0.999])
    T0 = np.array([O.background(cosmo, za)["Tg"]])
    U = np.array([[1.0, 0.0, 0.0]])
    x1, _, U1, _, st = O.rec_step(cosmo, 1, za, zb, d, x0, T0, U=U, mixing="full")
    bg = O.background(cosmo, zb)
    nH = bg["nH"] * d[0]
    rho_g = TB["a_rad_SI"] * bg["Tg"] ** 4 / TB["c_m_s"] ** 2
    rho_b = nH * TB["m_H_kg"] / 0.76
    alpha = 4.0 / 3.0 * x1[0] * nH * TB["sigma_T_m2"] * TB["c_m_s"] * rho_g / rho_b  # c = 1 in the paper
    rate = -math.log(U1[0, 0]) / st["dt"]
    assert rate == pytest.approx(alpha + bg["H"], rel=1e-4)
    # before recombination the drag is much faster than the expansion (Sec. IV.A)
    assert alpha > 100 * bg["H"]
