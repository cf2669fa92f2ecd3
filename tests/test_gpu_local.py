"""GPU no-mixing (local) limit against the oracle, element by element: x_e, T,
damped velocities and emission weights within 1e-9 (FP64 form) / 1e-4 (mixed
form) on ragged boxes, with flows strong enough that some cells converge
faster than the expansion (no escape) and others diverge strongly; substeps
and a short trajectory; the cases that are rejected."""
import numpy as np
import pytest

import oracle as O
from gpu_helpers import new_box, oracle_fields, set_state

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-9, "mixed": 1e-4}


def _state(cosmo, d, z, rng):
    x = np.clip(O.saha_xe(cosmo, z, d) * rng.uniform(0.9, 1.3, d.size), 1e-6, 0.999)
    T = O.background(cosmo, z)["Tg"] * (1.0 + 0.01 * rng.standard_normal(d.size))
    return x, T


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("n,sigma_v", [(13, 15.0), (32, 4.0)])
@pytest.mark.parametrize("z_from,z_to,n_sub", [(1500.0, 1490.0, 1), (1150.0, 1140.0, 3), (900.0, 895.0, 1)])
def test_local_step_matches_oracle(cosmo, precision, n, sigma_v, z_from, z_to, n_sub):
    box = new_box(n, precision, "local", sigma_v=sigma_v, n_sub=n_sub)
    rng = np.random.default_rng(n + int(z_from))
    d, U, _ = oracle_fields(box)
    H = O.background(cosmo, z_to)["H"]
    div = O.divergence(cosmo, n, z_to, U)
    assert (div / 3 < -H).any() and (div / 3 > H).any()  # both regimes present
    x0, T0 = _state(cosmo, d, z_from, rng)
    set_state(box, x0, T0, tally=rng.integers(0, 5, n ** 3).astype(np.uint32))
    T_in = box.host("T").astype(np.float64)
    box.refresh(z_from)
    box.step(0, z_from, z_to)
    st = box.stats()
    x1, T1, U1, e1, so = O.rec_step(cosmo, n, z_from, z_to, d, x0, T_in, U=U, mixing="local", n_sub=n_sub)
    tol = TOL[precision]
    np.testing.assert_allclose(box.host("x"), x1, rtol=tol, atol=0)
    np.testing.assert_allclose(box.host("T").astype(np.float64), T1, rtol=tol, atol=0)
    np.testing.assert_allclose(box.host("vel4")[:, :3].astype(np.float64), U1, rtol=tol, atol=1e-12)
    np.testing.assert_allclose(box.host("emis").astype(np.float64), e1, rtol=3 * max(tol, 1e-6), atol=0)
    assert st["X_e"] == pytest.approx(so["Xe"], rel=tol)
    assert st["C"] == pytest.approx(so["C"], rel=tol)
    assert st["lam"] == pytest.approx(so["lam"], rel=10 * tol)
    assert st["newton_passes"] == 0 and st["flags"] == 0
    assert box.tally_np().sum() == 0  # tallies unused, reset at the end of the step
    box.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_local_trajectory_with_transport(cosmo, precision):
    """Ten steps with transport between them (tallies play no part in the local
    update): the GPU state stays within the tolerance of the oracle started
    from the same Saha state, and the transport keeps conserving packets."""
    from paper_2312_11448_gb300.inputs import z_schedule
    n = 16
    box = new_box(n, precision, "local", n_packets=50_000, sigma_v=3.0)
    zs = z_schedule(1300.0, 1200.0, 10)
    d, U, _ = oracle_fields(box)
    box.state_init(zs[0])
    x = O.saha_xe(cosmo, zs[0], d)
    T = np.full(n ** 3, O.background(cosmo, zs[0])["Tg"])
    for s in range(10):
        box.transport(s, zs[s])
        st = box.stats()
        assert st["emitted"] == st["absorbed"] + st["capped"] == 50_000
        box.step(s, zs[s], zs[s + 1])
        x, T, U, _, _ = O.rec_step(cosmo, n, zs[s], zs[s + 1], d, x, T, U=U, mixing="local")
    tol = 10 * TOL[precision]
    np.testing.assert_allclose(box.host("x"), x, rtol=tol, atol=0)
    np.testing.assert_allclose(box.host("T").astype(np.float64), T, rtol=tol, atol=0)
    box.close()


def test_local_mode_rejections():
    from gpu_helpers import make_fields
    from paper_2312_11448_gb300 import rec
    d, U = make_fields(8, 0.5, 1.0, seed=2)
    with pytest.raises(rec.RecError, match="single-box"):
        rec.Batch([(8, d, U, 10), (8, d, U, 10)], precision="fp64", mixing="local")
    box = new_box(8, "fp64", "local")
    with pytest.raises(rec.RecError, match="tally and full"):
        box.step_noalloc(1400.0, 1390.0)
    x = box.x
    with pytest.raises(rec.RecError, match="tally and full"):
        box.xe_adjoint(x, 1.0, x.clone(), x.clone())
    box.close()


# ---- partial mixing: f_alpha of the full-mixing rate plus the rest local
def _partial_box(n, precision, f, sigma_v, n_sub=1):
    from gpu_helpers import make_fields
    from paper_2312_11448_gb300 import rec
    d, U = make_fields(n, 0.8, sigma_v, seed=1)
    return rec.Box(n, d, U, 1000, precision=precision, mixing="partial", seed=7, n_sub=n_sub, f_alpha=f)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("f", [0.0, 0.3, 0.8, 1.0])
@pytest.mark.parametrize("n,sigma_v,n_sub", [(13, 15.0, 1), (32, 4.0, 2)])
def test_partial_step_matches_oracle(cosmo, precision, f, n, sigma_v, n_sub):
    box = _partial_box(n, precision, f, sigma_v, n_sub)
    rng = np.random.default_rng(n + int(10 * f))
    d, U, _ = oracle_fields(box)
    z_from, z_to = 1200.0, 1190.0
    x0, T0 = _state(cosmo, d, z_from, rng)
    set_state(box, x0, T0, tally=rng.integers(0, 5, n ** 3).astype(np.uint32))
    T_in = box.host("T").astype(np.float64)
    box.refresh(z_from)
    box.step(0, z_from, z_to)
    st = box.stats()
    x1, T1, U1, e1, so = O.rec_step(cosmo, n, z_from, z_to, d, x0, T_in, U=U, mixing="partial", f_alpha=f,
                                    n_sub=n_sub)
    tol = TOL[precision]
    np.testing.assert_allclose(box.host("x"), x1, rtol=tol, atol=0)
    np.testing.assert_allclose(box.host("T").astype(np.float64), T1, rtol=tol, atol=0)
    np.testing.assert_allclose(box.host("vel4")[:, :3].astype(np.float64), U1, rtol=tol, atol=1e-12)
    assert st["X_e"] == pytest.approx(so["Xe"], rel=tol)
    assert st["flags"] & 1 == 0
    box.close()


def test_partial_mode_rejections():
    from gpu_helpers import make_fields
    from paper_2312_11448_gb300 import rec
    d, U = make_fields(8, 0.5, 1.0, seed=2)
    with pytest.raises(rec.RecError, match="single-box"):
        rec.Batch([(8, d, U, 10), (8, d, U, 10)], precision="fp64", mixing="partial", f_alpha=0.5)
    with pytest.raises(rec.RecError, match="f_alpha"):
        rec.Box(8, d, U, 10, precision="fp64", mixing="partial", f_alpha=1.5)
    box = _partial_box(8, "fp64", 0.5, 1.0)
    with pytest.raises(rec.RecError, match="tally and full"):
        box.step_noalloc(1400.0, 1390.0)
    box.close()


@pytest.mark.parametrize("f_new", [0.4, 0.0, 1.0])
def test_set_f_alpha_equals_a_context_made_with_it(cosmo, f_new):
    """Changing the partial-mixing share on a context gives the step of a
    context created with that share (Sec. V's redshift-dependent f_alpha),
    including the two ends: 0 (the local limit) and 1 (full mixing)."""
    from gpu_helpers import make_fields
    from paper_2312_11448_gb300 import rec
    d, U = make_fields(12, 0.8, 3.0, seed=1)
    a = rec.Box(12, d, U, 1000, precision="fp64", mixing="partial", seed=7, f_alpha=0.9)
    b = rec.Box(12, d, U, 1000, precision="fp64", mixing="partial", seed=7, f_alpha=f_new)
    for box in (a, b):
        box.state_init(1300.0)
    a.step(0, 1300.0, 1295.0)
    b.set_f_alpha(0.9)
    b.step(0, 1300.0, 1295.0)
    a.set_f_alpha(f_new)
    b.set_f_alpha(f_new)
    a.step(1, 1295.0, 1290.0)
    b.step(1, 1295.0, 1290.0)
    for name in ("x", "T", "vel4", "emis"):
        assert np.array_equal(a.host(name), b.host(name)), name
    # and against the oracle's partial step at the new share
    c = rec.Box(12, d, U, 1000, precision="fp64", mixing="partial", seed=7, f_alpha=f_new)
    c.state_init(1300.0)
    dd, UU, _ = oracle_fields(c)
    x0 = c.host("x")
    T0 = c.host("T").astype(np.float64)
    c.close()
    x1, T1, U1, e1, so = O.rec_step(cosmo, 12, 1300.0, 1295.0, dd, x0, T0, U=UU, mixing="partial", f_alpha=0.9)
    x2, T2, U2, e2, so = O.rec_step(cosmo, 12, 1295.0, 1290.0, dd, x1, T1, U=U1, mixing="partial", f_alpha=f_new)
    np.testing.assert_allclose(a.host("x"), x2, rtol=TOL["fp64"], atol=0)
    np.testing.assert_allclose(a.host("T"), T2, rtol=TOL["fp64"], atol=0)
    with pytest.raises(rec.RecError, match="0, 1"):
        a.set_f_alpha(1.2)
    full = rec.Box(8, d[:512], U[:512], 10, precision="fp64", mixing="full")
    with pytest.raises(rec.RecError, match="partial"):
        full.set_f_alpha(0.5)
    for box in (a, b, full):
        box.close()
