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
