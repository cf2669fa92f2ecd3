"""Oracle pin for the forward-mode tangent used to check the GPU adjoint: the
directional derivative of the volume-averaged X_e (Sec. II.A) and of the
visibility function at z ~ 1100 with respect to per-cell density, initial
temperature and absorbed-Ly-alpha fraction, against central differences."""
import numpy as np
import pytest

import oracle as O
from paper_2312_11448_gb300.inputs import z_schedule, density_field


def _setup(cosmo, n=4, seed=2):
    rng = np.random.default_rng(seed)
    zs = z_schedule(1250.0, 1000.0, 16)
    d = density_field(n, 0.8, seed).ravel()
    x0 = O.saha_xe(cosmo, zs[0], d) * 0.98
    T0 = np.full(n ** 3, O.background(cosmo, zs[0])["Tg"]) * (1 + 0.002 * rng.standard_normal(n ** 3))
    tallies = rng.poisson(30 * d[None, :] ** 1.5, size=(16, n ** 3)).astype(np.uint32)
    return n, zs, d, x0, T0, tallies, rng


@pytest.mark.parametrize("mixing", ["full", "tally"])
@pytest.mark.parametrize("objective", [1, 2])
def test_tangent_matches_central_differences(cosmo, mixing, objective):
    n, zs, d, x0, T0, tallies, rng = _setup(cosmo)
    tl = tallies if mixing == "tally" else None
    dd = d * rng.standard_normal(d.size)
    dT = T0 * 1e-3 * rng.standard_normal(d.size)
    da = rng.standard_normal(d.size) / d.size if mixing == "tally" else None
    J0, Jdot = O.traj_tangent(cosmo, n, zs, d, x0, T0, d_delta=dd, d_T0=dT, d_a=da, tallies=tl, mixing=mixing,
                              objective=objective)
    Jr, _ = O.traj_objective(cosmo, n, zs, d, x0, T0, tallies=tl, mixing=mixing, objective=objective)
    assert J0 == pytest.approx(Jr, rel=1e-13)
    h = 1e-4

    def J(s):
        ap = None if da is None else s * da
        return O.traj_objective(cosmo, n, zs, d + s * dd, x0, T0 + s * dT, tallies=tl, mixing=mixing,
                                objective=objective, a_pert=ap)[0]

    fd = (J(h) - J(-h)) / (2 * h)
    assert Jdot == pytest.approx(fd, rel=2e-6, abs=1e-12 * abs(J0))
    assert abs(Jdot) > 1e-6 * abs(J0)  # the direction actually moves the objective


def test_tangent_components_separately(cosmo):
    """Each input direction on its own (density, temperature, absorbed fraction)."""
    n, zs, d, x0, T0, tallies, rng = _setup(cosmo, seed=7)
    dirs = {"d_delta": d * rng.standard_normal(d.size), "d_T0": T0 * 1e-3 * rng.standard_normal(d.size),
            "d_a": rng.standard_normal(d.size) / d.size}
    for name, v in dirs.items():
        _, Jdot = O.traj_tangent(cosmo, n, zs, d, x0, T0, tallies=tallies, mixing="tally", objective=1, **{name: v})
        # T perturbations are erased by Compton coupling, so that derivative is
        # tiny: use a larger step (the response stays linear)
        h = 1e-1 if name == "d_T0" else 1e-4
        kw = lambda s: dict(delta=d + s * v if name == "d_delta" else d, T0=T0 + s * v if name == "d_T0" else T0,
                            a_pert=s * v if name == "d_a" else None)
        Jp = O.traj_objective(cosmo, n, zs, x0=x0, tallies=tallies, mixing="tally", objective=1, **kw(h))[0]
        Jm = O.traj_objective(cosmo, n, zs, x0=x0, tallies=tallies, mixing="tally", objective=1, **kw(-h))[0]
        J0 = O.traj_objective(cosmo, n, zs, x0=x0, tallies=tallies, mixing="tally", objective=1, **kw(0.0))[0]
        assert Jdot == pytest.approx((Jp - Jm) / (2 * h), rel=5e-6, abs=1e-12 * abs(J0) / h)
