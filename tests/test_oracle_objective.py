"""Oracle pin for the trajectory objectives used by the adjoint checks
(orc_traj_objective): the volume-averaged X_e of Sec. II.A and the visibility
function at the node nearest z*, both written out here from their definitions
with textbook constants, on the X_e history the oracle's own recombination
steps produce.

Definitions (stated reading: the paper names the visibility function without
defining it): X_e = sum_i Delta_i x_i / sum_i Delta_i; g = (d tau/dz) e^{-tau}
at z*, tau(z*) = int_{z_end}^{z*} sigma_T c nbar_H X_e / ((1 + z) H) dz by the
trapezoidal rule on the step nodes."""
import json
import os

import numpy as np
import pytest

import oracle as O
from paper_2312_11448_gb300.inputs import density_field, z_schedule

TB = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "textbook_values.json")))


def _trajectory(cosmo, n=4, seed=3):
    zs = z_schedule(1300.0, 900.0, 24)
    d = density_field(n, 0.8, seed).ravel()
    x0 = O.saha_xe(cosmo, zs[0], d)
    T0 = np.full(n ** 3, O.background(cosmo, zs[0])["Tg"])
    return n, zs, d, x0, T0


def _volume_history(cosmo, n, zs, d, x0, T0):
    """X_e at every node from chained single oracle steps (full mixing)."""
    x, T = x0.copy(), T0.copy()
    out = [np.dot(d, x) / d.sum()]
    for s in range(len(zs) - 1):
        x, T, _, _, _ = O.rec_step(cosmo, n, zs[s], zs[s + 1], d, x, T, mixing="full", want_emis=False)
        out.append(np.dot(d, x) / d.sum())
    return np.array(out)


def _visibility(cosmo, zs, Xe, ks):
    bg = [O.background(cosmo, z) for z in zs]
    f = np.array([TB["sigma_T_m2"] * TB["c_m_s"] * b["nH"] * X / ((1 + z) * b["H"]) for z, b, X in zip(zs, bg, Xe)])
    tau = sum(0.5 * (f[m] + f[m + 1]) * (zs[m] - zs[m + 1]) for m in range(ks, len(zs) - 1))
    return f[ks] * np.exp(-tau), tau


@pytest.mark.parametrize("z_star", [1100.0, 1003.0, 1300.0, 900.0])
def test_objectives_match_definitions_on_oracle_history(cosmo, z_star):
    n, zs, d, x0, T0 = _trajectory(cosmo)
    J1, hist = O.traj_objective(cosmo, n, zs, d, x0, T0, mixing="full", objective=1, z_star=z_star)
    ref = _volume_history(cosmo, n, zs, d, x0, T0)
    np.testing.assert_allclose(hist, ref, rtol=1e-13, atol=0)
    ks = int(np.argmin(np.abs(zs - z_star)))
    assert J1 == hist[ks]
    J2, _ = O.traj_objective(cosmo, n, zs, d, x0, T0, mixing="full", objective=2, z_star=z_star)
    g, tau = _visibility(cosmo, zs, hist, ks)
    # the textbook sigma_T is printed to 8 digits
    assert J2 == pytest.approx(g, rel=2e-8)
    if ks == len(zs) - 1:
        assert tau == 0.0  # optical depth from the last node to itself


def test_visibility_peaks_near_recombination(cosmo):
    """The visibility function over the trajectory has its maximum inside the
    range where X_e falls fastest (Sec. III.A.1: the last-scattering surface
    near z ~ 1100), not at an end of the schedule."""
    n = 4
    zs = z_schedule(1500.0, 800.0, 60)
    d = density_field(n, 0.5, 1).ravel()
    x0 = O.saha_xe(cosmo, zs[0], d)
    T0 = np.full(n ** 3, O.background(cosmo, zs[0])["Tg"])
    g = np.array([O.traj_objective(cosmo, n, zs, d, x0, T0, mixing="full", objective=2, z_star=z)[0]
                  for z in zs[::4]])
    k = int(np.argmax(g))
    assert 0 < k < len(g) - 1
    assert 1000.0 < zs[::4][k] < 1200.0
