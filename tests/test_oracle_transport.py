"""Oracle pins for the counter-based generator, the packet allocation and the
ballistic Ly-alpha transport (Appendix A steps (1), (4); Eq. for omega_r).

Checks: statistical quality of Philox4x32-10; exact totals and per-cell
expectations of the allocation; the closed-form resonance cell for a uniform
Hubble flow; packet conservation; a brute-force crossing enumeration against
the incremental traversal; and the emitted distributions (position, direction,
frequency).
"""
import math

import numpy as np
import pytest
from scipy import stats
from scipy.special import erf

import oracle as O
from paper_2312_11448_gb300.inputs import doppler_quantiles, pack_vel4


# ---- Philox -------------------------------------------------------------------
def _philox_many(n, key=(123, 456), block=0):
    out = np.empty((n, 4), dtype=np.uint32)
    for i in range(n):
        out[i] = O.philox4x32_10([i, 7, block, 1], key)
    return out


def test_philox_uniformity_and_bit_balance():
    w = _philox_many(8192).astype(np.uint64)
    for col in range(4):
        top = (w[:, col] >> 24).astype(np.int64)
        counts = np.bincount(top, minlength=256)
        chi2 = ((counts - 32.0) ** 2 / 32.0).sum()
        assert stats.chi2.sf(chi2, 255) > 1e-4
    bits = ((w[:, :, None] >> np.arange(32, dtype=np.uint64)) & 1).reshape(-1, 32)
    frac = bits.mean(axis=0)
    assert np.all(np.abs(frac - 0.5) < 5 * 0.5 / math.sqrt(bits.shape[0]))


def test_philox_avalanche_on_counter_and_key():
    rng = np.random.default_rng(5)
    flips = []
    for _ in range(300):
        ctr = rng.integers(0, 2 ** 32, size=4, dtype=np.uint64).astype(np.uint32)
        key = rng.integers(0, 2 ** 32, size=2, dtype=np.uint64).astype(np.uint32)
        base = O.philox4x32_10(ctr, key)
        for which in ("ctr", "key"):
            c2, k2 = ctr.copy(), key.copy()
            b = int(rng.integers(0, 32))
            if which == "ctr":
                c2[int(rng.integers(0, 4))] ^= np.uint32(1 << b)
            else:
                k2[int(rng.integers(0, 2))] ^= np.uint32(1 << b)
            d = O.philox4x32_10(c2, k2) ^ base
            flips.append(sum(bin(int(v)).count("1") for v in d) / 128.0)
    f = np.array(flips)
    assert abs(f.mean() - 0.5) < 0.01
    assert f.min() > 0.25


# ---- allocation -----------------------------------------------------------------
def test_allocation_exact_total_and_expectation():
    n = 8
    rng = np.random.default_rng(1)
    r = rng.lognormal(0.0, 1.5, n ** 3)
    r[rng.integers(0, n ** 3, 20)] = 0.0
    N = 123457
    for dtype in (np.float32, np.float64):
        P = O.allocate(n, r.astype(dtype), N, seed=99, step=3)
        cnt = np.diff(P.astype(np.int64))
        assert P[0] == 0 and P[-1] == N and np.all(cnt >= 0)
        expect = N * r / r.sum()
        assert np.max(np.abs(cnt - expect)) < 1.0 + 1e-3
        assert np.all(cnt[r == 0] == 0)


def test_allocation_unbiased_over_steps():
    n = 4
    r = np.linspace(0.1, 1.0, n ** 3)
    N = 1000
    acc = np.zeros(n ** 3)
    S = 400
    for s in range(S):
        acc += np.diff(O.allocate(n, r, N, seed=5, step=s).astype(np.int64))
    expect = N * r / r.sum()
    frac = expect - np.floor(expect)
    sd = np.sqrt(np.maximum(frac * (1 - frac), 1e-12) / S)
    assert np.all(np.abs(acc / S - expect) < 5 * sd + 1e-9)


def test_allocation_edge_cases():
    n = 2
    z = np.zeros(8)
    with pytest.raises(ValueError):
        O.allocate(n, z, 10, 1, 0)
    P = O.allocate(n, z, 0, 1, 0)
    assert np.all(P == 0)
    r = z.copy(); r[5] = 3.0
    P = O.allocate(n, r, 77, 1, 0)
    assert np.array_equal(np.diff(P.astype(np.int64)), np.array([0, 0, 0, 0, 0, 77, 0, 0]))
    r[2] = np.nan
    with pytest.raises(ValueError):
        O.allocate(n, r, 10, 1, 0)


# ---- transport ------------------------------------------------------------------
def _inputs(n, sigma_v, seed=3, precision="f32"):
    rng = np.random.default_rng(seed)
    emis = rng.uniform(0.2, 2.0, n ** 3)
    U = rng.normal(0.0, sigma_v, (n ** 3, 3)) if sigma_v > 0 else np.zeros((n ** 3, 3))
    T = rng.uniform(2800.0, 3200.0, n ** 3)
    dt = np.float32 if precision == "f32" else np.float64
    return emis.astype(dt), pack_vel4(U, dt), T.astype(dt), doppler_quantiles().astype(dt)


def _cell_xyz(c, n):
    return np.stack([c % n, (c // n) % n, c // (n * n)], axis=1)


@pytest.mark.parametrize("precision,eps", [("f32", 2e-3), ("f64", 1e-9)])
def test_resonance_cell_closed_form_uniform_hubble_flow(cosmo, precision, eps):
    """With no peculiar flow a packet emitted at point p with frequency offset xi
    comes back into resonance after a path kappa xi v_th (cells); it is absorbed
    in the cell containing p + n_hat * u0, or at home if xi <= 0."""
    n = 8
    emis, vel4, T, q = _inputs(n, 0.0, precision=precision)
    Np = 20000
    tally, cnt, pk = O.transport(cosmo, n, 1100.0, 17, 2, Np, emis, vel4, T, q, precision=precision, dump=Np)
    assert cnt == dict(emitted=Np, absorbed=Np, capped=0, crossings=cnt["crossings"])
    home = _cell_xyz(pk["home"], n)
    end = home + pk["f"] + pk["dir"] * np.maximum(pk["u0"], 0.0)[:, None]
    near = np.abs(end - np.round(end)) < eps
    ok = ~near.any(axis=1) | (pk["u0"] <= 0)
    expect = np.where(pk["u0"][:, None] > 0, np.floor(end).astype(np.int64) % n, home)
    ec = (expect[:, 2] * n + expect[:, 1]) * n + expect[:, 0]
    assert ok.mean() > 0.97
    assert np.array_equal(pk["absorb"][ok], ec[ok])
    # the resonance distance is kappa xi v_th (no flow)
    kappa, cth = O.transport_params(cosmo, n, 1100.0)
    vt = np.sqrt(T.astype(np.float64)[pk["home"]] * cth)
    np.testing.assert_allclose(pk["u0"], pk["xi"] * vt, rtol=1e-5 if precision == "f32" else 1e-13, atol=1e-5)
    assert np.array_equal(np.bincount(pk["absorb"], minlength=n ** 3), tally)


def _brute_force_absorb(p, n, vel, kappa):
    """Enumerate every face crossing of the ray up to the largest possible
    resonance distance, sort them, and walk the cells (independent of the
    incremental traversal).  Returns (cell, crossings, margin)."""
    home = np.array([p["home"] % n, (p["home"] // n) % n, p["home"] // (n * n)])
    d = p["dir"]
    f = p["f"]
    umax = p["u0"] + kappa * np.abs(vel).max() * math.sqrt(3) + 2.0
    events = []
    for a in range(3):
        if d[a] > 0:
            k = np.arange(1, int(umax * d[a] + 3))
            events += [((kk - f[a]) / d[a], a, 1) for kk in k]
        elif d[a] < 0:
            k = np.arange(0, int(umax * -d[a] + 3))
            events += [((f[a] + kk) / -d[a], a, -1) for kk in k]
    events.sort()
    cell = home.copy()
    margin = np.inf
    for i, (t, a, s) in enumerate(events):
        c = (cell[2] * n + cell[1]) * n + cell[0]
        res = p["u0"] - kappa * float(np.dot(d, vel[c]))
        margin = min(margin, abs(res - t), (events[i + 1][0] - t) if i + 1 < len(events) else np.inf)
        if res <= t:
            return c, i, margin
        cell[a] = (cell[a] + s) % n
    raise AssertionError("ray did not resonate")


def test_brute_force_crossings_with_flow(cosmo):
    n = 8
    emis, vel4, T, q = _inputs(n, 3.0, seed=11, precision="f64")
    Np = 3000
    tally, cnt, pk = O.transport(cosmo, n, 1100.0, 5, 9, Np, emis, vel4, T, q, precision="f64", dump=Np)
    assert cnt["emitted"] == Np and cnt["absorbed"] == Np and tally.sum() == Np
    kappa, _ = O.transport_params(cosmo, n, 1100.0)
    vel = vel4[:, :3].astype(np.float64)
    checked = 0
    for i in range(0, Np, 3):
        p = {k: pk[k][i] for k in pk}
        c, ncross, margin = _brute_force_absorb(p, n, vel, kappa)
        if margin < 1e-9:
            continue
        assert p["absorb"] == c and p["crossings"] == ncross
        checked += 1
    assert checked > 900


@pytest.mark.parametrize("precision", ["f32", "f64"])
def test_emission_distributions(cosmo, precision):
    n = 8
    emis, vel4, T, q = _inputs(n, 0.0, seed=2, precision=precision)
    Np = 20000
    _, _, pk = O.transport(cosmo, n, 1200.0, 8, 1, Np, emis, vel4, T, q, precision=precision, dump=Np)
    # positions uniform inside the cell
    for a in range(3):
        assert stats.kstest(pk["f"][:, a], "uniform").pvalue > 1e-3
    # isotropic directions: unit norm, zero mean, <n_a^2> = 1/3, n_z uniform in (-1, 1)
    nrm = np.linalg.norm(pk["dir"], axis=1)
    np.testing.assert_allclose(nrm, 1.0, rtol=1e-6 if precision == "f32" else 1e-14)
    assert np.all(np.abs(pk["dir"].mean(axis=0)) < 5 / math.sqrt(3 * Np))
    assert np.all(np.abs((pk["dir"] ** 2).mean(axis=0) - 1 / 3) < 0.02)
    assert stats.kstest((pk["dir"][:, 2] + 1) / 2, "uniform").pvalue > 1e-3
    # frequency offsets follow the Doppler profile exp(-x^2)/sqrt(pi) (tails beyond the table cut)
    assert stats.kstest(pk["xi"], lambda x: (1 + erf(x)) / 2).pvalue > 1e-3
    assert np.abs(pk["xi"]).max() <= q.max() + 1e-6


def test_precisions_agree_statistically(cosmo):
    n = 16
    out = {}
    for prec in ("f32", "f64"):
        emis, vel4, T, q = _inputs(n, 1.0, seed=4, precision=prec)
        tally, cnt, _ = O.transport(cosmo, n, 1100.0, 21, 0, 200000, emis, vel4, T, q, precision=prec)
        out[prec] = (tally.astype(np.float64), cnt["crossings"] / cnt["emitted"])
    assert out["f32"][1] == pytest.approx(out["f64"][1], rel=0.02)
    # the f32 and f64 paths draw different random streams, but the absorbed
    # distributions agree within shot noise
    a, b = out["f32"][0], out["f64"][0]
    z = (a - b) / np.sqrt(np.maximum(a + b, 1.0))
    assert abs(z.mean()) < 0.1 and z.std() < 1.2


@pytest.mark.parametrize("precision", ["f32", "f64"])
def test_openmp_build_same_integers(cosmo, precision):
    """The OpenMP build (used only to time the oracle on all host cores) gives
    the same tallies and counters as the plain build: integer sums in any order."""
    n = 16
    emis, vel4, T, q = _inputs(n, 1.0, seed=9, precision=precision)
    t1, c1, _ = O.transport(cosmo, n, 1150.0, 5, 3, 150000, emis, vel4, T, q, precision=precision)
    t4, c4, _ = O.transport(cosmo, n, 1150.0, 5, 3, 150000, emis, vel4, T, q, precision=precision, threads=4)
    assert np.array_equal(t1, t4) and c1 == c4
    assert O.lib().orc_threads(0) == 1 and O.lib(openmp=True).orc_threads(4) == 4


# ---- the emission-frame Doppler term (omega_r = omega (1 - U_par), App. A) ------------
def _closed_form_cell(pk, n, s, eps):
    """Cell containing p + n_hat s per packet, and a mask of the points that lie
    farther than eps (cells) from every face."""
    home = _cell_xyz(pk["home"], n)
    end = home + pk["f"] + pk["dir"] * s[:, None]
    ok = ~(np.abs(end - np.round(end)) < eps).any(axis=1)
    cell = np.floor(end).astype(np.int64) % n
    return (cell[:, 2] * n + cell[:, 1]) * n + cell[:, 0], ok


@pytest.mark.parametrize("precision,eps", [("f32", 2e-3), ("f64", 1e-9)])
def test_galilean_invariance_uniform_flow(cosmo, precision, eps):
    """A bulk flow that is the same in every cell is a change of frame: in the
    gas frame every packet is emitted and absorbed exactly as with no flow, so
    the absorbing cells must equal the zero-flow ones.  The home-cell Doppler
    term (emission frame) and the per-cell term (absorption frame) must cancel;
    a sign error in either moves most packets by kappa n.U ~ 2 cells here."""
    n, z, Np = 16, 1100.0, 20000
    emis, vel4, T, q = _inputs(n, 0.0, seed=5, precision=precision)
    U = np.array([3.0, -4.0, 2.5])  # km/s, along no axis
    vel_u = pack_vel4(np.tile(U, (n ** 3, 1)), vel4.dtype)
    t0, c0, p0 = O.transport(cosmo, n, z, 29, 4, Np, emis, vel4, T, q, precision=precision, dump=Np)
    t1, c1, p1 = O.transport(cosmo, n, z, 29, 4, Np, emis, vel_u, T, q, precision=precision, dump=Np)
    # same random draws: positions, directions and frequencies are frame independent
    assert np.array_equal(p0["f"], p1["f"]) and np.array_equal(p0["dir"], p1["dir"])
    assert np.array_equal(p0["xi"], p1["xi"])
    kappa, _ = O.transport_params(cosmo, n, z)
    assert kappa * np.linalg.norm(U) > 2.0  # the flow shifts resonance by more than two cells
    _, ok = _closed_form_cell(p0, n, np.maximum(p0["u0"], 0.0), eps)
    ok &= ~(np.abs(p0["u0"]) < eps)  # absorbed-at-home boundary
    assert ok.mean() > 0.97
    assert np.array_equal(p1["absorb"][ok], p0["absorb"][ok])
    assert c1["absorbed"] == Np and c0["absorbed"] == Np
    assert np.abs(t1.astype(np.int64) - t0.astype(np.int64)).sum() <= 2 * (~ok).sum()


def _slab_walk(pk, n, s0, shift, sig):
    """Absorption distance along each ray in a two-slab flow, U_z = +V for
    iz < n/2 and -V above, derived from the physics rather than from the
    traversal: the packet is emitted at gas-frame offset xi in its home cell,
    so in the Hubble frame its resonance distance is s0 = kappa xi v_th plus
    kappa n.U_home (emitter moving along n blue-shifts the packet); in a cell
    moving with U_c the resonance point is kappa n.U_c earlier.  In a segment
    of the other slab the distance is therefore s0 + 2 kappa V n_z sigma_home
    (shift = 2 kappa V n_z sigma_home); a packet entering a segment already past
    its resonance point is absorbed in the first cell it enters.  Returns
    (s, boundary-safe mask)."""
    half = n // 2
    z0 = (pk["home"] // (n * n)) + pk["f"][:, 2]
    nz = pk["dir"][:, 2]
    out = np.full(len(z0), np.nan)
    safe = np.ones(len(z0), dtype=bool)
    for i in range(len(z0)):
        zz, d = z0[i], nz[i]
        s_start = 0.0
        # the boundaries the ray meets, in order
        nxt = (np.floor(zz / half) + 1) * half if d > 0 else np.floor(zz / half) * half
        seg_sig = sig[i]
        for _ in range(64):
            s_end = (nxt - zz) / d if d != 0 else np.inf
            r = s0[i] if seg_sig == sig[i] else s0[i] + shift[i]
            if r <= s_end:
                s_hit = max(r, s_start)
                if abs(r - s_start) < 1e-6 or abs(r - s_end) < 1e-6:
                    safe[i] = False
                if s_hit == s_start and s_start > 0:
                    s_hit = s_start + 1e-7  # just inside the entered cell
                out[i] = s_hit
                break
            s_start = s_end
            seg_sig = -seg_sig
            nxt = nxt + half if d > 0 else nxt - half
        else:
            safe[i] = False
    return out, safe


@pytest.mark.parametrize("precision,eps", [("f32", 2e-3), ("f64", 1e-9)])
def test_two_slab_flow_closed_form(cosmo, precision, eps):
    """Closed-form absorbing cells in a flow with a velocity jump: every packet
    has the same frequency offset xi0 (a one-point profile table) and uniform
    temperature, so its resonance distance follows from the slab it is in and
    its direction alone.  Pins the sign and the frame of the home-cell
    Doppler term independently of the traversal code."""
    n, z, Np, V, xi0, T0 = 16, 1100.0, 6000, 8.0, 1.5, 3000.0
    R = np.float32 if precision == "f32" else np.float64
    emis = np.random.default_rng(3).uniform(0.5, 1.5, n ** 3).astype(R)
    iz = np.arange(n ** 3) // (n * n)
    Uz = np.where(iz < n // 2, V, -V)
    vel4 = pack_vel4(np.stack([np.zeros(n ** 3), np.zeros(n ** 3), Uz], axis=1), R)
    T = np.full(n ** 3, T0, dtype=R)
    q = np.full(8, xi0, dtype=R)
    tally, cnt, pk = O.transport(cosmo, n, z, 41, 6, Np, emis, vel4, T, q, precision=precision, dump=Np)
    assert cnt["absorbed"] == Np
    kappa, cth = O.transport_params(cosmo, n, z)
    s0 = np.full(Np, xi0 * math.sqrt(T0 * cth))  # kappa xi0 v_th, in cells
    assert s0[0] > 3.0 and 2 * kappa * V > 5.0
    sig = np.where(pk["home"] // (n * n) < n // 2, 1.0, -1.0)
    shift = 2.0 * kappa * V * pk["dir"][:, 2] * sig
    s, safe = _slab_walk(pk, n, s0, shift, sig)
    home = _cell_xyz(pk["home"], n)
    end = home + pk["f"] + pk["dir"] * s[:, None]
    cell = np.floor(end).astype(np.int64) % n
    cell = (cell[:, 2] * n + cell[:, 1]) * n + cell[:, 0]
    # away from x and y faces; z faces only matter where the packet resonates
    # inside a segment (an entered cell's point sits on its z face by construction)
    ok = safe & ~(np.abs(end[:, :2] - np.round(end[:, :2])) < eps).any(axis=1)
    inside = np.isclose(s, s0) | np.isclose(s, s0 + shift)
    ok &= ~(inside & (np.abs(end[:, 2] - np.round(end[:, 2])) < eps))
    assert ok.mean() > 0.9
    assert np.array_equal(pk["absorb"][ok], cell[ok])
    # the flow matters: the zero-flow cells, and the cells a reversed home-cell
    # term would give, both disagree with the oracle for many packets
    c_noflow, _ = _closed_form_cell(pk, n, s0, eps)
    assert (c_noflow[ok] != pk["absorb"][ok]).mean() > 0.2
    s_wrong, _ = _slab_walk(pk, n, s0 - shift, shift, sig)
    c_wrong, _ = _closed_form_cell(pk, n, np.maximum(np.nan_to_num(s_wrong), 0.0), eps)
    assert (c_wrong[ok] != pk["absorb"][ok]).mean() > 0.2


@pytest.mark.parametrize("precision", ["f32", "f64"])
def test_packets_at_or_below_line_centre_end_at_home(cosmo, precision):
    """Emitted at or below the line centre (xi <= 0), a packet is resonant in its
    home cell whatever its direction and the flow: in the gas frame its
    frequency is already at or below resonance (u0 - kappa n.U_home = xi v_th
    <= 0 up to rounding, which cannot make it positive).  The oracle's packets
    with xi <= 0, in strong random flows of 20 km/s, all end in their home cell
    without crossing a face, while most of those above the line centre leave."""
    n, z, Np = 16, 1100.0, 40000
    emis, _, T, q = _inputs(n, 0.0, seed=9, precision=precision)
    rng = np.random.default_rng(13)
    vel4 = pack_vel4(rng.normal(0.0, 20.0, (n ** 3, 3)), emis.dtype)
    _, cnt, pk = O.transport(cosmo, n, z, 31, 2, Np, emis, vel4, T, q, precision=precision, dump=Np)
    low = pk["xi"] <= 0.0
    assert 0.4 < low.mean() < 0.6
    assert np.array_equal(pk["absorb"][low], pk["home"][low]) and not pk["crossings"][low].any()
    assert (pk["crossings"][~low] > 0).mean() > 0.75
