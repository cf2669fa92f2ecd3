"""Oracle pins for the resonant-scattering Ly-alpha Monte Carlo (Appendix A).

- Voigt / Faddeeva function against the library Faddeeva function and closed
  forms; the table the Monte Carlo interpolates against the function.
- The thermally averaged cross-section against direct quadrature of Eq. MC.
- The paper's wing estimate: x_50 of about 60 and a comoving mean free path
  of about 0.1 kpc there at z = 1100.
- The redistribution of Eq. inout: mean and second moment of the atom's
  parallel velocity and of the frequency change against closed forms in the
  Faddeeva function, the paper's wing statement (shift -1/x, unit width) and
  the exact density of the atom velocity (KS).
- The first-flight law of steps (3)-(5) (geometric number of steps of eps
  mean free paths, comoving distance).
- Galilean invariance under a uniform bulk flow.
- Escape and destruction fractions against the Sobolev escape probability:
  the Peebles C factor for a range of expansion rates zeta H with
  Lambda_2gamma = 0 (Fig. Cfact), and the two-photon fraction.
"""
import os

import numpy as np
import pytest
from scipy import integrate, stats
from scipy.special import erfcx, wofz

import json

import oracle as O

PV = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))

# Independent constants for the checks (SI, CODATA 2018).
C_LIGHT = 2.99792458e8
K_B = 1.380649e-23
M_H = 1.00782503223 * 1.66053906660e-27
LAMBDA_A = 6.62607015e-34 * C_LIGHT / (0.75 * 13.598434 * 1.602176634e-19)
KPC = 3.0856775814913673e19
THREADS = max(1, min(8, os.cpu_count() or 1))


# ---- Voigt function ----------------------------------------------------------
@pytest.mark.parametrize("a", [1e-4, 8.6e-4, 1e-2, 0.3])
def test_faddeeva_matches_library(a):
    ys = np.concatenate([np.linspace(-12, 12, 481), np.logspace(1, 5, 60), -np.logspace(1, 5, 7)])
    for y in ys:
        w = O.faddeeva(y, a)
        ref = wofz(y + 1j * a)
        assert w.real == pytest.approx(ref.real, rel=2e-9), (a, y)
        assert w.imag == pytest.approx(ref.imag, rel=2e-9, abs=1e-300), (a, y)


def test_voigt_closed_forms():
    for a in (1e-4, 1e-3, 0.1, 1.0):
        assert O.faddeeva(0.0, a).real == pytest.approx(erfcx(a), rel=1e-10)  # exp(a^2) erfc(a)
    for y in (0.0, 0.5, 1.7, 3.0):
        assert O.faddeeva(y, 1e-7).real == pytest.approx(np.exp(-y * y), rel=1e-5, abs=2e-7)
    a = 8.6e-4
    for y in (50.0, 300.0, 3e4):  # Lorentzian wing a / (sqrt(pi) y^2)
        assert O.faddeeva(y, a).real == pytest.approx(a / (np.sqrt(np.pi) * y * y), rel=2e-3)
    # normalisation of the profile: integral of H over y is sqrt(pi)
    y = np.concatenate([np.linspace(0, 10, 20001), np.logspace(1, 7, 20001)[1:]])
    H = O.voigt_table(a, y)
    tot = 2 * (integrate.trapezoid(H, y) + a / (np.sqrt(np.pi) * 1e7))
    assert tot == pytest.approx(np.sqrt(np.pi), rel=1e-6)


@pytest.mark.parametrize("a", [1e-4, 8.6e-4, 1e-2])
def test_voigt_table_interpolation(a):
    y = np.random.default_rng(3).uniform(-14, 14, 20000)
    got = O.voigt_table(a, y)
    ref = wofz(y + 1j * a).real
    assert np.max(np.abs(got / ref - 1)) < 3e-8


# ---- Eq. MC normalisation and the wing estimate -----------------------------------
def _setup(z=1100.0, **kw):
    cp = O.default_cosmo()
    return cp, O.mc_setup(cp, O.mc_params(z, **kw))


def test_cross_section_is_the_thermal_average_of_eq_mc():
    """<sigma>(y) = (1/sqrt pi) int dp exp(-p^2) sigma_0 Gamma^2 /
    (omega_a^2 v_th^2 (y - p)^2 + Gamma^2/4), sigma_0 = 3 lambda^2 / 8 pi,
    integrated directly with the physical constants, against sig0 H(a, y)."""
    cp, S = _setup()
    Tg = O.background(cp, 1100.0)["Tg"]
    vth = np.sqrt(2 * K_B * Tg / M_H) / C_LIGHT
    assert S["vth"] == pytest.approx(vth, rel=1e-12)
    G = O.A_2P1S
    om = 2 * np.pi * C_LIGHT / LAMBDA_A
    sigma0 = 3 * LAMBDA_A ** 2 / (8 * np.pi)
    for y in (0.0, 0.7, 2.5, 30.0):
        f = lambda p: np.exp(-p * p) * sigma0 * G * G / (om * om * vth * vth * (y - p) ** 2 + G * G / 4)
        pts = sorted({y, 0.0})
        direct = integrate.quad(f, -12, 12, points=pts, limit=2000, epsabs=0, epsrel=1e-12)[0] / np.sqrt(np.pi)
        if abs(y) > 12:  # far wing: add the Lorentzian tails outside the Gaussian core
            direct = integrate.quad(f, -12, 12, limit=2000, epsabs=0, epsrel=1e-12)[0] / np.sqrt(np.pi)
        model = S["sig0"] * O.voigt_table(S["a"], [y])[0]
        assert model == pytest.approx(direct, rel=1e-6), y


def test_wing_balance_x50_and_mean_free_path():
    """Appendix A: where the redshift per mean free path H l / v_th equals the
    restoring drift 1/x of the wing random walk, x_50 is about 60, with a
    comoving mean free path of about 0.1 kpc (z = 1100, mostly neutral)."""
    cp, S = _setup()
    n1s = 0.85 * S["nH"]
    xs = np.logspace(0.5, 4, 4000)
    sigma = S["sig0"] * O.voigt_table(S["a"], xs)
    lhs = S["dxdl"] / (sigma * n1s)      # H l / v_th per mean free path
    x50 = xs[np.argmin(np.abs(lhs - 1.0 / xs))]
    lo, hi = PV["x50"]["band"]
    assert lo < x50 < hi
    l_com_kpc = (1.0 + 1100.0) / (S["sig0"] * O.voigt_table(S["a"], [x50])[0] * n1s) / KPC
    lo, hi = PV["mfp_at_x50_kpc"]["band"]
    assert lo < l_com_kpc < hi


def test_escape_and_two_photon_fractions_at_1100():
    """Sec. III.B: without bulk flows about 5e-3 of the Ly-alpha photons are lost
    by redshifting and about 1.5e-2 to two-photon decay at z ~ 1100.  The
    Sobolev chain of the Monte Carlo's branching (an absorbed photon's atom is
    photo-ionised, decays by two photons or re-emits with weights
    beta : Lambda : 3 A; each emission escapes with P = R_alpha / (3 A)) on the
    homogeneous full-mixing history gives both."""
    from paper_2312_11448_gb300.inputs import z_schedule
    cp = O.default_cosmo()
    zs = z_schedule(1700.0, 1100.0, 120)
    d = np.ones(1)
    x = O.saha_xe(cp, zs[0], d)
    T = np.full(1, O.background(cp, zs[0])["Tg"])
    for s in range(len(zs) - 1):
        x, T, _, _, _ = O.rec_step(cp, 1, zs[s], zs[s + 1], d, x, T, mixing="full", n_sub=4)
    S = O.mc_setup(cp, O.mc_params(1100.0))
    n1s = S["nH"] * (1 - x[0])
    R = O.rates(cp, 1100.0, T[0])["K_R"] / n1s
    A = O.A_2P1S
    Pe = R / (3 * A)
    pa = 1 - S["p_ion"] - S["p_2g"]
    den = 1 - (1 - Pe) * pa
    fz, f2 = Pe / den, (1 - Pe) * S["p_2g"] / den
    lo, hi = PV["f_z_at_1100"]["band"]
    assert lo < fz < hi
    lo, hi = PV["f_2gamma_at_1100"]["band"]
    assert lo < f2 < hi


# ---- redistribution (Eq. inout) ------------------------------------------------
def _moments(a, y):
    w = wofz(y + 1j * a)
    H, K = w.real, w.imag
    Es = a * K / H                       # mean of y - p under exp(-p^2) L(y - p)
    Es2 = a / (np.sqrt(np.pi) * H) - a * a
    Ep = y - Es
    Ep2 = y * y - 2 * y * Es + Es2
    # y_out - y = -p (1 - mu) + p_perp sqrt(1 - mu^2) cos beta, mu uniform:
    # E = -E[p]; E[.^2] = (4/3) E[p^2] + E[p_perp^2] (2/3)(1/2) = (4/3) E[p^2] + 1/3
    return Ep, Ep2, -Ep, 4.0 / 3.0 * Ep2 + 1.0 / 3.0


@pytest.mark.parametrize("y", [0.0, 0.4, 1.0, 2.2, 3.0, 4.5, 20.0, -5.0, 300.0])
def test_redistribution_moments(y):
    a = 8.6e-4
    m = 200_000
    pp, dy = O.mc_redistribution(a, y, seed=11, m=m)
    Ep, Ep2, Edy, Edy2 = _moments(a, y)
    se = np.sqrt(max(Ep2 - Ep * Ep, 1e-12) / m)
    assert abs(pp.mean() - Ep) < 5 * se
    assert abs(dy.mean() - Edy) < 5 * np.sqrt(max(Edy2 - Edy * Edy, 1e-12) / m)
    assert abs(np.mean(dy ** 2) - Edy2) < 5 * np.std(dy ** 2) / np.sqrt(m)
    assert abs(np.mean(pp ** 2) - Ep2) < 5 * np.std(pp ** 2) / np.sqrt(m)


def test_wing_redistribution_as_stated():
    """On the wing x_out is about Gaussian of unit width centred on x_in - 1/x_in."""
    pp, dy = O.mc_redistribution(8.6e-4, 25.0, seed=3, m=200_000)
    assert dy.mean() == pytest.approx(-1 / 25.0, abs=0.01)
    assert dy.var() == pytest.approx(1.0, rel=0.02)
    assert abs(stats.skew(dy)) < 0.1


@pytest.mark.parametrize("kin", [(0.0, 0.0, 1.0), (0.0, 0.0, -1.0), (0.48, -0.6, 0.64), (1.0, 0.0, 0.0)])
def test_outgoing_direction_isotropic(kin):
    """Isotropic scattering: k_out is a unit vector, k_in . k_out is uniform on
    [-1, 1], and k_out is isotropic (zero mean, covariance I/3)."""
    m = 60_000
    _, _, ko = O.mc_redistribution(8.6e-4, 0.3, seed=17, m=m, kin=kin, want_k=True)
    np.testing.assert_allclose(np.linalg.norm(ko, axis=1), 1.0, rtol=1e-14)
    mu = ko @ np.asarray(kin)
    assert stats.kstest(mu, stats.uniform(loc=-1, scale=2).cdf).pvalue > 1e-3
    assert np.all(np.abs(ko.mean(axis=0)) < 5 * np.sqrt(1 / 3 / m))
    cov = ko.T @ ko / m
    np.testing.assert_allclose(cov, np.eye(3) / 3, atol=5 * np.sqrt(2 / 15 / m))


@pytest.mark.parametrize("y", [0.5, 1.6, 3.5, 12.0])
def test_atom_velocity_density_ks(y):
    """The sampled parallel velocity follows exp(-p^2) / ((y - p)^2 + a^2) (KS
    against the numerically integrated CDF)."""
    a = 1e-2
    pp, _ = O.mc_redistribution(a, y, seed=5, m=40_000)
    grid = np.sort(np.concatenate([np.linspace(-6, 6 + y, 60001), y + a * np.tan(np.linspace(-1.55, 1.55, 4001))]))
    f = np.exp(-grid ** 2) / ((y - grid) ** 2 + a * a)
    cdf = np.concatenate([[0], np.cumsum(0.5 * (f[1:] + f[:-1]) * np.diff(grid))])
    cdf /= cdf[-1]
    res = stats.kstest(pp, lambda p: np.interp(p, grid, cdf))
    assert res.pvalue > 1e-3


# ---- the Monte Carlo proper ------------------------------------------------------
def _uniform_box(n, nph):
    P = (np.arange(n ** 3 + 1, dtype=np.uint64) * (nph // n ** 3)).astype(np.uint32)
    return np.ones(n ** 3), P


def _x50(S, n1s):
    return (S["sig0"] * S["a"] * n1s / (np.sqrt(np.pi) * S["dxdl"])) ** (1 / 3)


def test_first_flight_law():
    """Lambda_2gamma huge: every photon ends at its first scattering.  Its step
    count is geometric with success probability 1 - exp(-eps) and the comoving
    distance is steps x eps x l(line centre) x (1 + z)."""
    cp = O.default_cosmo()
    z, eps, xe = 1200.0, 0.1, 0.3
    mp = O.mc_params(z, eps=eps, lambda2g=1e30, seed=4)
    S = O.mc_setup(cp, mp, 4)
    d, P = _uniform_box(4, 20_000)
    rec, cnt = O.lya_mc(cp, mp, 4, d, np.full(64, xe), P, threads=THREADS)
    assert cnt[1] == len(rec) and np.all(rec["n_scat"] == 1)
    n1s = S["nH"] * (1 - xe)
    l0 = 1.0 / (S["sig0"] * O.voigt_table(S["a"], [0.0])[0] * n1s)
    D_unit = eps * l0 * (1 + z) / KPC
    # positions are absolute (box of 24 kpc): each step rounds them by about
    # one ulp of a few cells, 1e-14 kpc, against flights of 1e-9 kpc
    np.testing.assert_allclose(rec["D_kpc"], rec["n_steps"] * D_unit, rtol=1e-9,
                               atol=2e-14 * (rec["n_steps"].max() + 1))
    q = 1 - np.exp(-eps)
    k = rec["n_steps"].astype(float)
    assert k.mean() == pytest.approx(1 / q, rel=5 * np.sqrt((1 - q) / len(k)) * q)
    # P(K > 20) = exp(-20 eps)
    assert np.mean(k > 20) == pytest.approx(np.exp(-20 * eps), abs=5 * np.sqrt(np.exp(-2) / len(k)))


def test_galilean_invariance_uniform_flow():
    cp = O.default_cosmo()
    mp = O.mc_params(1700.0, zeta=3e4, lambda2g=0.0, seed=9)
    S = O.mc_setup(cp, mp, 2)
    mp.x_lost = 50 * _x50(S, 0.5 * S["nH"])
    d, P = _uniform_box(2, 800)
    xe = np.full(8, 0.5)
    U0 = np.tile([30.0, -20.0, 10.0], (8, 1))
    r0, _ = O.lya_mc(cp, mp, 2, d, xe, P, threads=THREADS)
    r1, _ = O.lya_mc(cp, mp, 2, d, xe, P, U=U0, threads=THREADS)
    same = (r0["fate"] == r1["fate"]) & (r0["n_scat"] == r1["n_scat"])
    assert same.mean() > 0.98
    np.testing.assert_allclose(r1["D_kpc"][same], r0["D_kpc"][same], rtol=1e-6)


@pytest.mark.parametrize("zeta", [3e3, 3e4])
def test_peebles_factor_with_expansion_rate(zeta):
    """Fig. Cfact: with Lambda_2gamma = 0 the Monte-Carlo C = p_alpha f_z (a fresh
    n = 2 atom re-emits with probability p_alpha = 3A/(beta + 3A), the photon is
    then lost by redshifting with probability f_z) equals the Peebles factor
    R / (beta + R), R = 8 pi zeta H / (lambda^3 n_1s)."""
    cp = O.default_cosmo()
    z, xe = 1700.0, 0.5
    mp = O.mc_params(z, zeta=zeta, lambda2g=0.0, seed=21)
    S = O.mc_setup(cp, mp, 4)
    n1s = S["nH"] * (1 - xe)
    mp.x_lost = 50 * _x50(S, n1s)
    d, P = _uniform_box(4, 2048)
    rec, cnt = O.lya_mc(cp, mp, 4, d, np.full(64, xe), P, threads=THREADS)
    assert cnt[3] == 0 and cnt[4] == 0 and cnt[1] == 0
    N = len(rec)
    beta = O.rates(cp, z, O.background(cp, z)["Tg"])["beta"]
    H = zeta * O.background(cp, z)["H"]
    R = 8 * np.pi * H / (LAMBDA_A ** 3 * n1s)
    A = O.A_2P1S
    p_alpha = 3 * A / (beta + 3 * A)
    fz = cnt[0] / N
    C_th = R / (beta + R)
    C_mc = p_alpha * fz
    assert C_mc == pytest.approx(C_th, abs=4 * np.sqrt(C_th * (1 - C_th) / N))


def test_two_photon_and_escape_fractions():
    """Lambda_2gamma comparable to beta: per-photon fractions against the chain
    of Sobolev escapes, f_z = P / (1 - (1-P) p_a) and
    f_2g = (1-P) p_2g / (1 - (1-P) p_a), P = R / (3 A)."""
    cp = O.default_cosmo()
    z, xe, lam = 1700.0, 0.5, 5e4
    mp = O.mc_params(z, zeta=1e3, lambda2g=lam, seed=33)
    S = O.mc_setup(cp, mp, 4)
    n1s = S["nH"] * (1 - xe)
    mp.x_lost = 50 * _x50(S, n1s)
    d, P = _uniform_box(4, 2048)
    rec, cnt = O.lya_mc(cp, mp, 4, d, np.full(64, xe), P, threads=THREADS)
    N = len(rec)
    beta = O.rates(cp, z, O.background(cp, z)["Tg"])["beta"]
    A = O.A_2P1S
    R = 8 * np.pi * 1e3 * O.background(cp, z)["H"] / (LAMBDA_A ** 3 * n1s)
    Pe = R / (3 * A)
    tot = beta + lam + 3 * A
    pa, p2 = 3 * A / tot, lam / tot
    den = 1 - (1 - Pe) * pa
    fz, f2 = Pe / den, (1 - Pe) * p2 / den
    assert cnt[0] / N == pytest.approx(fz, abs=4 * np.sqrt(fz * (1 - fz) / N))
    assert cnt[1] / N == pytest.approx(f2, abs=4 * np.sqrt(f2 * (1 - f2) / N))
    assert cnt[2] + cnt[1] + cnt[0] == N


def test_loss_threshold_is_past_the_point_of_no_return():
    """Photons past 20 x_50 on the red wing never come back: the fates do not
    change between a loss threshold of 20 x_50 and 100 x_50."""
    cp = O.default_cosmo()
    mp = O.mc_params(1700.0, zeta=1e4, lambda2g=0.0, seed=8)
    S = O.mc_setup(cp, mp, 2)
    x50 = _x50(S, 0.5 * S["nH"])
    d, P = _uniform_box(2, 400)
    out = []
    for fac in (20, 100):
        mp.x_lost = fac * x50
        rec, _ = O.lya_mc(cp, mp, 2, d, np.full(8, 0.5), P, threads=THREADS)
        out.append(rec)
    assert np.array_equal(out[0]["fate"], out[1]["fate"])
    # lost photons still scatter now and then far on the wing (each step has
    # the same scattering probability) without coming back; the others are
    # untouched
    kept = out[0]["fate"] != 0
    assert np.array_equal(out[0]["n_scat"][kept], out[1]["n_scat"][kept])
    assert np.all(out[1]["n_scat"] >= out[0]["n_scat"])


def test_max_steps_caps_photons():
    cp = O.default_cosmo()
    mp = O.mc_params(1500.0, zeta=1.0, max_steps=1000, seed=2)
    d, P = _uniform_box(2, 16)
    rec, cnt = O.lya_mc(cp, mp, 2, d, np.full(8, 0.5), P)
    assert cnt[3] == 16 and np.all(rec["n_steps"] == 1000)


def test_openmp_build_gives_the_same_photons():
    """The tests run the Monte Carlo in the oracle's OpenMP build (photons are
    independent); its records equal the plain build's."""
    cp = O.default_cosmo()
    mp = O.mc_params(1700.0, zeta=3e4, lambda2g=2e4, seed=12)
    S = O.mc_setup(cp, mp, 2)
    mp.x_lost = 50 * _x50(S, 0.5 * S["nH"])
    d, P = _uniform_box(2, 64)
    a, _ = O.lya_mc(cp, mp, 2, d, np.full(8, 0.5), P)
    b, _ = O.lya_mc(cp, mp, 2, d, np.full(8, 0.5), P, threads=4)
    assert np.array_equal(a, b)
