"""Host side of the library's scattering Monte Carlo (no GPU needed): the
Voigt function it interpolates, against the library Faddeeva function of
scipy and against closed forms, and the argument checks of lya_voigt."""
import numpy as np
import pytest
from scipy.special import erfcx, wofz


@pytest.mark.parametrize("a", [1e-4, 8.6e-4, 1e-2, 0.1])
def test_library_voigt_matches_faddeeva(a):
    from paper_2312_11448_gb300 import rec
    y = np.concatenate([np.random.default_rng(1).uniform(-14, 14, 20000), np.logspace(1, 6, 200),
                        -np.logspace(0, 4, 50), [0.0, 9.999999, 10.0, 10.000001]])
    got = rec.voigt(a, y)
    ref = wofz(y + 1j * a).real
    assert np.max(np.abs(got / ref - 1)) < 3e-8


def test_library_voigt_closed_forms():
    from paper_2312_11448_gb300 import rec
    for a in (1e-4, 1e-2, 0.5):
        assert rec.voigt(a, [0.0])[0] == pytest.approx(erfcx(a), rel=1e-9)  # exp(a^2) erfc(a)
    a = 8.6e-4
    y = np.array([60.0, 500.0, 4e4])
    np.testing.assert_allclose(rec.voigt(a, y), a / (np.sqrt(np.pi) * y * y), rtol=1e-3)


def test_library_voigt_rejects_bad_arguments():
    from paper_2312_11448_gb300 import rec
    with pytest.raises(rec.RecError):
        rec.voigt(0.0, [1.0])
    with pytest.raises(rec.RecError):
        rec.voigt(-1e-3, [1.0])


@pytest.mark.parametrize("z,zeta,lam,n", [(1100.0, 1.0, -1.0, 256), (1700.0, 3e4, 0.0, 4), (1400.0, 10.0, 5e3, 33)])
def test_library_mc_scalars_match_oracle(z, zeta, lam, n):
    """The snapshot scalars the GPU Monte Carlo uses equal the oracle's (the two
    compute them independently from the same definitions)."""
    import oracle as O
    from paper_2312_11448_gb300 import rec
    lib = rec.mc_scalars(z, n=n, zeta=zeta, lambda2g=lam)
    orc = O.mc_setup(O.default_cosmo(), O.mc_params(z, zeta=zeta, lambda2g=lam), n)
    for key, v in orc.items():
        assert lib[key] == pytest.approx(v, rel=1e-13), key


# ---- the mixed form's redistribution, run on the host from the kernel source ----
def _moments(a, y):
    w = wofz(y + 1j * a)
    H, K = w.real, w.imag
    Es = a * K / H
    Es2 = a / (np.sqrt(np.pi) * H) - a * a
    Ep = y - Es
    Ep2 = y * y - 2 * y * Es + Es2
    return Ep, Ep2, -Ep, 4.0 / 3.0 * Ep2 + 1.0 / 3.0


@pytest.mark.parametrize("y", [0.0, 0.4, 1.0, 2.2, 3.0, 4.5, 20.0, -5.0, 300.0])
def test_mixed_form_redistribution_moments(y):
    """Mean and second moment of the atom's parallel velocity and of the
    frequency change against their closed forms in the Faddeeva function
    (binary32 arithmetic: the statistical error dominates)."""
    from paper_2312_11448_gb300 import rec
    a, m = 8.6e-4, 200_000
    pp, dy, _, caps = rec.mc_redistribution_mixed(a, y, seed=11, m=m)
    assert caps == 0
    Ep, Ep2, Edy, Edy2 = _moments(a, y)
    tol_rel = 3e-6 * max(1.0, abs(y))  # binary32 rounding of y and p near |y|
    assert abs(pp.mean() - Ep) < 5 * np.sqrt(max(Ep2 - Ep * Ep, 1e-12) / m) + tol_rel
    assert abs(dy.mean() - Edy) < 5 * np.sqrt(max(Edy2 - Edy * Edy, 1e-12) / m) + tol_rel
    assert abs(np.mean(dy ** 2) - Edy2) < 5 * np.std(dy ** 2) / np.sqrt(m) + tol_rel * abs(Edy2)


@pytest.mark.parametrize("y", [0.5, 1.6, 3.5, 12.0])
def test_mixed_form_atom_velocity_density_ks(y):
    from scipy import stats
    from paper_2312_11448_gb300 import rec
    a = 1e-2
    pp, _, _, _ = rec.mc_redistribution_mixed(a, y, seed=5, m=40_000)
    grid = np.sort(np.concatenate([np.linspace(-6, 6 + y, 60001), y + a * np.tan(np.linspace(-1.55, 1.55, 4001))]))
    f = np.exp(-grid ** 2) / ((y - grid) ** 2 + a * a)
    cdf = np.concatenate([[0], np.cumsum(0.5 * (f[1:] + f[:-1]) * np.diff(grid))])
    cdf /= cdf[-1]
    assert stats.kstest(pp, lambda p: np.interp(p, grid, cdf)).pvalue > 1e-3


@pytest.mark.parametrize("kin", [(0.0, 0.0, 1.0), (0.0, 0.0, -1.0), (0.48, -0.6, 0.64)])
def test_mixed_form_outgoing_direction_isotropic(kin):
    from scipy import stats
    from paper_2312_11448_gb300 import rec
    m = 60_000
    _, _, ko, _ = rec.mc_redistribution_mixed(8.6e-4, 0.3, seed=17, m=m, kin=kin)
    np.testing.assert_allclose(np.linalg.norm(ko, axis=1), 1.0, rtol=1e-6)
    mu = ko @ np.asarray(kin)
    assert stats.kstest(mu, stats.uniform(loc=-1, scale=2).cdf).pvalue > 1e-3
    assert np.all(np.abs(ko.mean(axis=0)) < 5 * np.sqrt(1 / 3 / m))
    np.testing.assert_allclose(ko.T @ ko / m, np.eye(3) / 3, atol=5 * np.sqrt(2 / 15 / m))


@pytest.mark.parametrize("a", [1e-4, 8.6e-4, 1e-2])
def test_mixed_form_voigt(a):
    """The binary32 Voigt evaluation of the mixed form: relative error at the
    binary32 level over the table and the wing series."""
    from paper_2312_11448_gb300 import rec
    y = np.concatenate([np.random.default_rng(2).uniform(-14, 14, 20000), np.logspace(1, 5, 200), [9.99999, 10.0]])
    got = rec.voigt(a, y, mixed=True)
    ref = wofz(y.astype(np.float32).astype(np.float64) + 1j * np.float32(a)).real
    assert np.max(np.abs(got / ref - 1)) < 2e-6
