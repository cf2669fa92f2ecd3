"""GPU adjoint (rec_step_adjoint through the sqrt(N)-checkpointed trajectory)
against the oracle's forward-mode tangent and against central finite
differences of the GPU forward, for X_e(z~1100) and the visibility function,
in full-mixing and tally modes."""
import numpy as np
import pytest

import oracle as O
from gpu_helpers import new_box, oracle_fields
from paper_2312_11448_gb300.inputs import z_schedule

pytestmark = pytest.mark.gpu


def _setup(cosmo, mixing, n=8, S=14, seed=4):
    zs = z_schedule(1250.0, 1000.0, S)
    box = new_box(n, "fp64", mixing, sigma=0.8)
    d, U, _ = oracle_fields(box)
    rng = np.random.default_rng(seed)
    x0 = O.saha_xe(cosmo, zs[0], d) * 0.98
    T0 = O.background(cosmo, zs[0])["Tg"] * (1.0 + 0.002 * rng.standard_normal(d.size))
    tallies = rng.poisson(30 * d ** 1.5, size=(S, d.size)).astype(np.uint32) if mixing == "tally" else None
    return zs, box, d, x0, T0, tallies, rng


@pytest.mark.parametrize("mixing", ["full", "tally"])
@pytest.mark.parametrize("objective", [1, 2])
def test_adjoint_vs_tangent_and_finite_differences(cosmo, mixing, objective):
    import torch
    from paper_2312_11448_gb300.autograd import objective_and_gradients
    zs, box, d, x0, T0, tallies, rng = _setup(cosmo, mixing)
    J, g, Xe = objective_and_gradients(box, zs, x0, T0, tallies=tallies, objective=objective, z_star=1100.0,
                                       checkpoint_every=4)
    # the GPU forward objective equals the oracle's
    Jo, hist = O.traj_objective(cosmo, box.n, zs, d, x0, T0, tallies=tallies, mixing=mixing, objective=objective)
    np.testing.assert_allclose(Xe, hist, rtol=1e-9)
    assert J == pytest.approx(Jo, rel=1e-9)
    # adjoint . direction == oracle tangent along the same direction
    dd = d * rng.standard_normal(d.size)
    dT = T0 * 1e-3 * rng.standard_normal(d.size)
    da = rng.standard_normal(d.size) / d.size if mixing == "tally" else None
    _, Jdot = O.traj_tangent(cosmo, box.n, zs, d, x0, T0, d_delta=dd, d_T0=dT, d_a=da, tallies=tallies,
                             mixing=mixing, objective=objective)
    gd, gT, ga = (g[k].cpu().numpy() for k in ("delta", "T0", "a"))
    adj = gd @ dd + gT @ dT + (ga @ da if da is not None else 0.0)
    assert adj == pytest.approx(Jdot, rel=1e-7, abs=1e-12 * abs(J))
    # central differences of the GPU forward along (delta, T0), h = 1e-4
    h = 1e-4
    Jh = []
    for sgn in (1.0, -1.0):
        box.delta.copy_(torch.as_tensor(d + sgn * h * dd))
        Jh.append(objective_and_gradients(box, zs, x0, T0 + sgn * h * dT, tallies=tallies, objective=objective,
                                          z_star=1100.0)[0])
    fd = (Jh[0] - Jh[1]) / (2 * h)
    assert gd @ dd + gT @ dT == pytest.approx(fd, rel=1e-5)
    box.close()


def test_initial_ionisation_gradient(cosmo):
    import torch
    from paper_2312_11448_gb300.autograd import objective_and_gradients
    zs, box, d, x0, T0, tallies, rng = _setup(cosmo, "tally", seed=9)
    J, g, _ = objective_and_gradients(box, zs, x0, T0, tallies=tallies, objective=1)
    dx = x0 * 1e-2 * rng.standard_normal(d.size)
    h = 1e-4
    Jp = objective_and_gradients(box, zs, x0 + h * dx, T0, tallies=tallies, objective=1)[0]
    Jm = objective_and_gradients(box, zs, x0 - h * dx, T0, tallies=tallies, objective=1)[0]
    assert g["x0"].cpu().numpy() @ dx == pytest.approx((Jp - Jm) / (2 * h), rel=1e-5)
    box.close()


def test_autograd_function(cosmo):
    import torch
    from paper_2312_11448_gb300.autograd import recombination_objective
    zs, box, d, x0, T0, tallies, rng = _setup(cosmo, "tally", S=9, seed=2)
    dev = box.x.device
    dt = torch.tensor(d, device=dev, requires_grad=True)
    xt = torch.tensor(x0, device=dev, requires_grad=True)
    Tt = torch.tensor(T0, device=dev, requires_grad=True)
    at = torch.zeros(d.size, dtype=torch.float64, device=dev, requires_grad=True)
    J = recombination_objective(box, zs, dt, xt, Tt, at, tallies=tallies, objective=2)
    J.backward()
    for t in (dt, xt, Tt, at):
        assert t.grad is not None and torch.isfinite(t.grad).all()
    da = rng.standard_normal(d.size) / d.size
    _, Jdot = O.traj_tangent(cosmo, box.n, zs, d, x0, T0, d_a=da, tallies=tallies, mixing="tally", objective=2)
    assert float(at.grad.cpu().numpy() @ da) == pytest.approx(Jdot, rel=1e-7)
    box.close()


@pytest.mark.slow
@pytest.mark.parametrize("objective", [1, 2])
def test_adjoint_at_size_32_cubed_50_steps(cosmo, objective):
    """A 50-step window of the 256^3 run's schedule (z 1800 -> 600 in 400 steps)
    around z* = 1100 on a 32^3 box with its own tallies: adjoint . direction
    against the oracle tangent (1e-7) and against GPU central differences
    (1e-5), checkpoints every ceil(sqrt(50)) = 8 steps."""
    import torch
    from paper_2312_11448_gb300.autograd import objective_and_gradients
    full = z_schedule(1800.0, 600.0, 400)
    k0 = int(np.argmin(np.abs(full - 1100.0))) - 25
    zs = full[k0:k0 + 51]
    n = 32
    box = new_box(n, "fp64", "tally", sigma=0.8)
    d, U, _ = oracle_fields(box)
    rng = np.random.default_rng(11)
    x0 = O.saha_xe(cosmo, zs[0], d) * 0.9
    T0 = O.background(cosmo, zs[0])["Tg"] * (1.0 + 0.002 * rng.standard_normal(d.size))
    tallies = rng.poisson(30 * d ** 1.5, size=(50, d.size)).astype(np.uint32)
    J, g, Xe = objective_and_gradients(box, zs, x0, T0, tallies=tallies, objective=objective, z_star=1100.0)
    Jo, hist = O.traj_objective(cosmo, n, zs, d, x0, T0, tallies=tallies, mixing="tally", objective=objective)
    np.testing.assert_allclose(Xe, hist, rtol=1e-9)
    assert J == pytest.approx(Jo, rel=1e-9)
    dd = d * rng.standard_normal(d.size)
    dT = T0 * 1e-3 * rng.standard_normal(d.size)
    da = rng.standard_normal(d.size) / d.size
    _, Jdot = O.traj_tangent(cosmo, n, zs, d, x0, T0, d_delta=dd, d_T0=dT, d_a=da, tallies=tallies,
                             mixing="tally", objective=objective)
    gd, gT, ga = (g[k].cpu().numpy() for k in ("delta", "T0", "a"))
    assert gd @ dd + gT @ dT + ga @ da == pytest.approx(Jdot, rel=1e-7, abs=1e-12 * abs(J))
    h = 1e-4
    Jh = []
    for sgn in (1.0, -1.0):
        box.delta.copy_(torch.as_tensor(d + sgn * h * dd))
        Jh.append(objective_and_gradients(box, zs, x0, T0 + sgn * h * dT, tallies=tallies, objective=objective,
                                          z_star=1100.0)[0])
    assert gd @ dd + gT @ dT == pytest.approx((Jh[0] - Jh[1]) / (2 * h), rel=1e-5)
    box.close()
