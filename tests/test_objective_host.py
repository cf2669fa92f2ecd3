"""The library's host-side objective (rec_objective, no GPU needed) against
its definition written out here with textbook constants, and its gradient
against central differences of itself.

Objectives (stated reading of Sec. II.A and of the visibility function the
paper refers to without defining it): J1 = X_e at the node nearest z*; J2 =
g = (d tau/dz) exp(-tau) at that node, with the Thomson optical depth
tau(z) = int sigma_T c nbar_H X_e / ((1 + z) H) dz accumulated by the
trapezoidal rule from the last node up to z*."""
import json
import os

import numpy as np
import pytest

import oracle as O

TB = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "textbook_values.json")))


def _history():
    from paper_2312_11448_gb300.inputs import z_schedule
    zs = z_schedule(1600.0, 700.0, 60)
    # a smooth, recombination-like X_e history (its exact shape does not matter here)
    Xe = 1.0 / (1.0 + np.exp((1250.0 - zs) / 60.0)) + 2e-4
    return zs, Xe


def _visibility(zs, Xe, z_star):
    cp = O.default_cosmo()
    ks = int(np.argmin(np.abs(zs - z_star)))
    c = np.array([TB["sigma_T_m2"] * TB["c_m_s"] * O.background(cp, z)["nH"] / ((1 + z) * O.background(cp, z)["H"])
                  for z in zs])
    f = c * Xe
    tau = sum(0.5 * (f[m] + f[m + 1]) * (zs[m] - zs[m + 1]) for m in range(ks, len(zs) - 1))
    return f[ks] * np.exp(-tau)


@pytest.mark.parametrize("z_star", [1100.0, 1003.0, 700.0])
def test_objectives_match_their_definitions(z_star):
    from paper_2312_11448_gb300 import rec
    zs, Xe = _history()
    J1, g1 = rec.objective(zs, Xe, objective=1, z_star=z_star)
    ks = int(np.argmin(np.abs(zs - z_star)))
    assert J1 == Xe[ks] and g1[ks] == 1.0 and np.count_nonzero(g1) == 1
    J2, _ = rec.objective(zs, Xe, objective=2, z_star=z_star)
    # the textbook sigma_T is printed to 8 digits
    assert J2 == pytest.approx(_visibility(zs, Xe, z_star), rel=2e-8)


def test_visibility_gradient_matches_central_differences():
    from paper_2312_11448_gb300 import rec
    zs, Xe = _history()
    J, g = rec.objective(zs, Xe, objective=2, z_star=1100.0)
    for k in range(len(zs)):
        h = 1e-6 * Xe[k]
        Xp, Xm = Xe.copy(), Xe.copy()
        Xp[k] += h
        Xm[k] -= h
        fd = (rec.objective(zs, Xp, objective=2, z_star=1100.0)[0] -
              rec.objective(zs, Xm, objective=2, z_star=1100.0)[0]) / (2 * h)
        assert g[k] == pytest.approx(fd, rel=1e-6, abs=1e-12 * abs(J) / Xe[k])


def test_objective_rejects_bad_arguments():
    from paper_2312_11448_gb300 import rec
    zs, Xe = _history()
    with pytest.raises(rec.RecError):
        rec.objective(zs, Xe, objective=3)
