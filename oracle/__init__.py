"""Oracle for the recombination hot path (TEST INFRASTRUCTURE ONLY).

A plain single-threaded FP64 C++ restatement of what the GPU path computes,
written from Jedamzik, Abel & Ali-Haimoud, arXiv:2312.11448 (Sec. II.A
Eqs. alpha-def and Tb-evolution; Sec. III.A Eqs. rec0, n2s-sol, Cfactor,
R-alpha; Sec. IV Eq. dotne-mix; Appendix A for the Ly-alpha transport).  Only
tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may import it.
It shares no code with the CUDA library.

This module is argument marshalling over liboracle.so (numpy in, numpy out).
"""
import ctypes as C
import os

import numpy as np

from . import build as _build

_lib = None


class Cosmo(C.Structure):
    """Mirror of orc_cosmo (oracle.h)."""
    _fields_ = [("h", C.c_double), ("omega_b_h2", C.c_double), ("omega_c_h2", C.c_double),
                ("Y_p", C.c_double), ("T_cmb0", C.c_double), ("N_eff", C.c_double),
                ("L_box_kpc", C.c_double), ("fudge", C.c_double), ("heating", C.c_double)]


class Packet(C.Structure):
    """Mirror of orc_packet (oracle.h)."""
    _fields_ = [("home", C.c_uint32), ("j", C.c_uint32), ("absorb", C.c_uint32), ("crossings", C.c_uint32),
                ("f", C.c_double * 3), ("dir", C.c_double * 3), ("xi", C.c_double), ("u0", C.c_double)]


class McParams(C.Structure):
    """Mirror of orc_mc_params (oracle.h)."""
    _fields_ = [("z", C.c_double), ("eps", C.c_double), ("x_lost", C.c_double), ("zeta", C.c_double),
                ("lambda2g", C.c_double), ("A_alpha", C.c_double), ("seed", C.c_uint64), ("step", C.c_uint32),
                ("box", C.c_uint32), ("max_steps", C.c_uint64)]


class McPhoton(C.Structure):
    """Mirror of orc_mc_photon (oracle.h)."""
    _fields_ = [("home", C.c_uint32), ("j", C.c_uint32), ("fate", C.c_int32), ("n_scat", C.c_uint64),
                ("n_steps", C.c_uint64), ("D_kpc", C.c_double), ("x_end", C.c_double)]


MC_FATES = ("lost", "two_photon", "ionised", "capped")
# 2p -> 1s decay rate (NIST, 6.2649e8 /s; the paper quotes about 6.3e8 /s).
A_2P1S = 6.2649e8


def mc_params(z, eps=0.1, x_lost=1.0e4, zeta=1.0, lambda2g=-1.0, A_alpha=A_2P1S, seed=1, step=0, box=0,
              max_steps=10 ** 9) -> McParams:
    return McParams(z=z, eps=eps, x_lost=x_lost, zeta=zeta, lambda2g=lambda2g, A_alpha=A_alpha, seed=seed,
                    step=step, box=box, max_steps=max_steps)


def default_cosmo(**kw) -> Cosmo:
    """Sec. II.C defaults (h, Omega_b h^2, Omega_c h^2, Y_p) and the 24 kpc box."""
    p = dict(h=0.67, omega_b_h2=0.0224, omega_c_h2=0.12, Y_p=0.24, T_cmb0=2.7255, N_eff=3.046,
             L_box_kpc=24.0, fudge=1.14, heating=0.0)
    p.update(kw)
    return Cosmo(**p)


_lib_omp = None


def lib(openmp=False):
    """liboracle.so; openmp=True: the OpenMP build of the same source (timing only)."""
    global _lib, _lib_omp
    if openmp:
        if _lib_omp is None:
            _lib_omp = _bind(C.CDLL(_build.build(openmp=True)))
        return _lib_omp
    if _lib is None:
        _lib = _bind(C.CDLL(_build.build()))
    return _lib


def _bind(L):
    d, i64, u32, u64, i = C.c_double, C.c_int64, C.c_uint32, C.c_uint64, C.c_int
    P = C.POINTER
    L.orc_background.argtypes = [P(Cosmo), d, P(d)]
    L.orc_dt.argtypes = [P(Cosmo), d, d]
    L.orc_dt.restype = d
    L.orc_rates.argtypes = [P(Cosmo), d, d, P(d)]
    L.orc_saha_xe.argtypes = [P(Cosmo), d, i64, P(d), P(d)]
    L.orc_rec_step.argtypes = [P(Cosmo), i, i, i, d, d, P(d), P(d), P(d), P(d), P(u32), P(d), P(d), d]
    L.orc_philox4x32_10.argtypes = [P(u32), P(u32), P(u32)]
    L.orc_philox4x32_10.restype = None
    L.orc_transport_params.argtypes = [P(Cosmo), i, d, P(d)]
    L.orc_allocate_f32.argtypes = [i, P(C.c_float), u64, u64, u32, u32, P(u32)]
    L.orc_allocate_f64.argtypes = [i, P(d), u64, u64, u32, u32, P(u32)]
    for name, R in (("orc_transport_f32", C.c_float), ("orc_transport_f64", d)):
        getattr(L, name).argtypes = [P(Cosmo), i, d, u64, u32, u32, u64, P(R), P(R), P(R), P(R), i,
                                     P(u32), P(u64), P(Packet), i64]
    L.orc_traj_objective.argtypes = [P(Cosmo), i, i, i, i, P(d), P(u32), P(d), P(d), P(d), P(d), i, d,
                                     P(d), P(d)]
    L.orc_traj_tangent.argtypes = [P(Cosmo), i, i, i, i, P(d), P(u32), P(d), P(d), P(d), P(d), P(d), P(d),
                                   i, d, P(d)]
    L.orc_threads.argtypes = [i]
    L.orc_divergence.argtypes = [P(Cosmo), i, d, P(d), P(d)]
    L.orc_rec_step_trbdf2.argtypes = [P(Cosmo), i, i, i, d, d, P(d), P(d), P(d), P(d), P(u32), P(d), P(d)]
    L.orc_faddeeva.argtypes = [d, d, P(d)]
    L.orc_voigt_table.argtypes = [d, i64, P(d), P(d)]
    L.orc_mc_setup.argtypes = [P(Cosmo), P(McParams), i, P(d)]
    L.orc_mc_redistribution.argtypes = [d, d, P(d), u64, i64, P(d), P(d), P(d)]
    L.orc_lya_mc.argtypes = [P(Cosmo), P(McParams), i, P(d), P(d), P(d), P(u32), u64, u64, P(McPhoton),
                             P(u64)]
    return L


def _p(a, ctype):
    if a is None:
        return None
    return a.ctypes.data_as(C.POINTER(ctype))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _check(rc, what):
    if rc != 0:
        raise ValueError(f"oracle {what} failed with code {rc}")


def background(cp: Cosmo, z: float) -> dict:
    out = np.zeros(5)
    _check(lib().orc_background(C.byref(cp), z, _p(out, C.c_double)), "background")
    return dict(H=out[0], nH=out[1], Tg=out[2], Omega_r=out[3], Omega_L=out[4])


def dt(cp: Cosmo, z_from: float, z_to: float) -> float:
    return lib().orc_dt(C.byref(cp), z_from, z_to)


def rates(cp: Cosmo, z: float, T_b: float) -> dict:
    out = np.zeros(6)
    _check(lib().orc_rates(C.byref(cp), z, T_b, _p(out, C.c_double)), "rates")
    return dict(alpha=out[0], beta=out[1], e_alpha=out[2], Lambda=out[3], K_R=out[4], saha=out[5])


def saha_xe(cp: Cosmo, z: float, delta) -> np.ndarray:
    d = _f64(delta).ravel()
    x = np.empty_like(d)
    _check(lib().orc_saha_xe(C.byref(cp), z, d.size, _p(d, C.c_double), _p(x, C.c_double)), "saha")
    return x.reshape(np.shape(delta))


def rec_step(cp: Cosmo, n: int, z_from: float, z_to: float, delta, x, T, U=None, tally=None, mixing="tally",
             n_sub=1, want_emis=True, f_alpha=1.0, integrator="be"):
    """One step; returns (x', T', U', emis, stats).  Inputs are not modified.
    integrator: "be" (backward Euler) or "trbdf2" (second order; tally and full mixing)."""
    if integrator == "trbdf2":
        return _rec_step_trbdf2(cp, n, z_from, z_to, delta, x, T, U, tally, mixing, n_sub, want_emis)
    d = _f64(delta).ravel()
    x1 = _f64(x).ravel().copy()
    T1 = _f64(T).ravel().copy()
    U1 = None if U is None else _f64(U).reshape(-1, 3).copy()
    t = None if tally is None else np.ascontiguousarray(tally, dtype=np.uint32).ravel()
    em = np.empty_like(d) if want_emis else None
    st = np.zeros(6)
    mix = {"tally": 0, "full": 1, "local": 2, "partial": 3}[mixing]
    rc = lib().orc_rec_step(C.byref(cp), n, mix, n_sub, z_from, z_to, _p(d, C.c_double), _p(x1, C.c_double),
                            _p(T1, C.c_double), _p(U1, C.c_double), _p(t, C.c_uint32), _p(em, C.c_double),
                            _p(st, C.c_double), float(f_alpha))
    _check(rc, "rec_step")
    stats = dict(lam=st[0], C=st[1], Xe=st[2], iters=int(st[3]), S1s=st[4], dt=st[5])
    return x1, T1, U1, em, stats


def divergence(cp: Cosmo, n: int, z: float, U) -> np.ndarray:
    """Physical velocity divergence per cell (1/s) as the local mode uses it."""
    u = _f64(U).reshape(-1, 3)
    out = np.zeros(u.shape[0])
    _check(lib().orc_divergence(C.byref(cp), n, z, _p(u, C.c_double), _p(out, C.c_double)), "divergence")
    return out


def philox4x32_10(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(_p(c, C.c_uint32), _p(k, C.c_uint32), _p(out, C.c_uint32))
    return out


def transport_params(cp: Cosmo, n: int, z: float):
    out = np.zeros(2)
    _check(lib().orc_transport_params(C.byref(cp), n, z, _p(out, C.c_double)), "transport_params")
    return out[0], out[1]


def allocate(n, emis, n_packets, seed, step, box=0):
    e = np.ascontiguousarray(emis).ravel()
    P = np.zeros(e.size + 1, dtype=np.uint32)
    if e.dtype == np.float32:
        rc = lib().orc_allocate_f32(n, _p(e, C.c_float), n_packets, seed, step, box, _p(P, C.c_uint32))
    else:
        e = _f64(e)
        rc = lib().orc_allocate_f64(n, _p(e, C.c_double), n_packets, seed, step, box, _p(P, C.c_uint32))
    _check(rc, "allocate")
    return P


def transport(cp: Cosmo, n: int, z: float, seed: int, step: int, n_packets: int, emis, vel4, T, quant, box=0,
              precision="f32", dump=0, threads=0):
    """Ballistic transport; returns (tally, counters dict, packets or None).

    precision "f32" runs the binary32 operation sequence, "f64" the binary64 one.
    vel4 is [n^3, 4] (Ux, Uy, Uz, unused) in km/s.  threads > 0 runs the OpenMP
    build on that many threads (same results; host-cores timing only).
    """
    R, ct = (np.float32, C.c_float) if precision == "f32" else (np.float64, C.c_double)
    e = np.ascontiguousarray(emis, dtype=R).ravel()
    v = np.ascontiguousarray(vel4, dtype=R).reshape(-1, 4)
    TT = np.ascontiguousarray(T, dtype=R).ravel()
    q = np.ascontiguousarray(quant, dtype=R).ravel()
    tally = np.zeros(e.size, dtype=np.uint32)
    cnt = np.zeros(4, dtype=np.uint64)
    pk = (Packet * dump)() if dump > 0 else None
    L = lib(openmp=threads > 0)
    if threads > 0:
        L.orc_threads(int(threads))
    fn = L.orc_transport_f32 if precision == "f32" else L.orc_transport_f64
    rc = fn(C.byref(cp), n, z, seed, step, box, n_packets, _p(e, ct), _p(v, ct), _p(TT, ct), _p(q, ct), q.size,
            _p(tally, C.c_uint32), _p(cnt, C.c_uint64), pk, dump)
    _check(rc, "transport")
    counters = dict(emitted=int(cnt[0]), absorbed=int(cnt[1]), capped=int(cnt[2]), crossings=int(cnt[3]))
    packets = None
    if dump > 0:
        m = min(dump, counters["emitted"])
        packets = dict(
            home=np.array([pk[i].home for i in range(m)], dtype=np.int64),
            j=np.array([pk[i].j for i in range(m)], dtype=np.int64),
            absorb=np.array([pk[i].absorb for i in range(m)], dtype=np.int64),
            crossings=np.array([pk[i].crossings for i in range(m)], dtype=np.int64),
            f=np.array([list(pk[i].f) for i in range(m)]).reshape(m, 3),
            dir=np.array([list(pk[i].dir) for i in range(m)]).reshape(m, 3),
            xi=np.array([pk[i].xi for i in range(m)]),
            u0=np.array([pk[i].u0 for i in range(m)]))
    return tally, counters, packets


def traj_objective(cp, n, zs, delta, x0, T0, tallies=None, mixing="tally", n_sub=1, objective=1, z_star=1100.0,
                   a_pert=None):
    zs = _f64(zs)
    d, x, T = _f64(delta).ravel(), _f64(x0).ravel(), _f64(T0).ravel()
    t = None if tallies is None else np.ascontiguousarray(tallies, dtype=np.uint32).ravel()
    ap = None if a_pert is None else _f64(a_pert).ravel()
    J = np.zeros(1)
    hist = np.zeros(zs.size)
    rc = lib().orc_traj_objective(C.byref(cp), n, {"tally": 0, "full": 1}[mixing], n_sub, zs.size - 1,
                                  _p(zs, C.c_double), _p(t, C.c_uint32), _p(d, C.c_double), _p(x, C.c_double),
                                  _p(T, C.c_double), _p(ap, C.c_double), objective, z_star, _p(J, C.c_double),
                                  _p(hist, C.c_double))
    _check(rc, "traj_objective")
    return J[0], hist


def traj_tangent(cp, n, zs, delta, x0, T0, d_delta=None, d_T0=None, d_a=None, tallies=None, mixing="tally",
                 n_sub=1, objective=1, z_star=1100.0):
    zs = _f64(zs)
    d, x, T = _f64(delta).ravel(), _f64(x0).ravel(), _f64(T0).ravel()
    t = None if tallies is None else np.ascontiguousarray(tallies, dtype=np.uint32).ravel()
    dd = None if d_delta is None else _f64(d_delta).ravel()
    dT = None if d_T0 is None else _f64(d_T0).ravel()
    da = None if d_a is None else _f64(d_a).ravel()
    J = np.zeros(2)
    rc = lib().orc_traj_tangent(C.byref(cp), n, {"tally": 0, "full": 1}[mixing], n_sub, zs.size - 1,
                                _p(zs, C.c_double), _p(t, C.c_uint32), _p(d, C.c_double), _p(x, C.c_double),
                                _p(T, C.c_double), _p(dd, C.c_double), _p(dT, C.c_double), _p(da, C.c_double),
                                objective, z_star, _p(J, C.c_double))
    _check(rc, "traj_tangent")
    return J[0], J[1]


def _rec_step_trbdf2(cp, n, z_from, z_to, delta, x, T, U, tally, mixing, n_sub, want_emis):
    d = _f64(delta).ravel()
    x1 = _f64(x).ravel().copy()
    T1 = _f64(T).ravel().copy()
    U1 = None if U is None else _f64(U).reshape(-1, 3).copy()
    t = None if tally is None else np.ascontiguousarray(tally, dtype=np.uint32).ravel()
    em = np.empty_like(d) if want_emis else None
    st = np.zeros(6)
    if mixing not in ("tally", "full"):
        raise ValueError("the TR-BDF2 step covers tally and full mixing")
    mix = {"tally": 0, "full": 1}[mixing]
    rc = lib().orc_rec_step_trbdf2(C.byref(cp), n, mix, n_sub, z_from, z_to, _p(d, C.c_double), _p(x1, C.c_double),
                                   _p(T1, C.c_double), _p(U1, C.c_double), _p(t, C.c_uint32), _p(em, C.c_double),
                                   _p(st, C.c_double))
    _check(rc, "rec_step_trbdf2")
    stats = dict(lam=st[0], C=st[1], Xe=st[2], iters=int(st[3]), S1s=st[4], dt=st[5])
    return x1, T1, U1, em, stats


# ---- resonant-scattering Ly-alpha Monte Carlo (Appendix A) ----------------------
def faddeeva(y: float, a: float) -> complex:
    out = np.zeros(2)
    _check(lib().orc_faddeeva(float(y), float(a), _p(out, C.c_double)), "faddeeva")
    return complex(out[0], out[1])


def voigt_table(a: float, y) -> np.ndarray:
    yy = _f64(y).ravel()
    H = np.empty_like(yy)
    _check(lib().orc_voigt_table(float(a), yy.size, _p(yy, C.c_double), _p(H, C.c_double)), "voigt_table")
    return H


def mc_setup(cp: Cosmo, mp: McParams, n: int = 1) -> dict:
    out = np.zeros(12)
    _check(lib().orc_mc_setup(C.byref(cp), C.byref(mp), n, _p(out, C.c_double)), "mc_setup")
    keys = ("a", "vth", "sig0", "dxdl", "p_ion", "p_2g", "beta", "Lambda", "H", "nH", "Tg", "cells_per_m")
    return dict(zip(keys, out))


def mc_redistribution(a: float, y: float, seed: int, m: int, kin=(0.0, 0.0, 1.0), want_k=False):
    """(p_par, y_out - y[, k_out]) of m independent isotropic scatterings at
    offset y of a photon travelling along kin."""
    pp = np.empty(m)
    dy = np.empty(m)
    ko = np.empty((m, 3)) if want_k else None
    k = _f64(kin)
    _check(lib().orc_mc_redistribution(float(a), float(y), _p(k, C.c_double), seed, m, _p(pp, C.c_double),
                                       _p(dy, C.c_double), _p(ko, C.c_double)), "mc_redistribution")
    return (pp, dy, ko) if want_k else (pp, dy)


def lya_mc(cp: Cosmo, mp: McParams, n: int, delta, xe, P, U=None, k0=0, k1=None, threads=0):
    """Photons k0..k1-1 of the allocation prefix P through the Monte Carlo.
    Returns (records, counters): records is a numpy structured array with
    home, j, fate, n_scat, n_steps, D_kpc, x_end; counters = photons per fate
    (lost, two_photon, ionised, capped) and the sampler-cap count.  threads > 0
    uses the OpenMP build (same per-photon results)."""
    d = _f64(delta).ravel()
    x = _f64(xe).ravel()
    if x.size == 1:
        x = np.full_like(d, x[0])
    Pa = np.ascontiguousarray(P, dtype=np.uint32).ravel()
    U1 = None if U is None else _f64(U).reshape(-1, 3)
    if k1 is None:
        k1 = int(Pa[-1])
    recs = (McPhoton * max(k1 - k0, 1))()
    cnt = np.zeros(5, dtype=np.uint64)
    L = lib(openmp=threads > 0)
    if threads > 0:
        L.orc_threads(int(threads))
    rc = L.orc_lya_mc(C.byref(cp), C.byref(mp), n, _p(d, C.c_double), _p(x, C.c_double), _p(U1, C.c_double),
                      _p(Pa, C.c_uint32), k0, k1, recs, _p(cnt, C.c_uint64))
    _check(rc, "lya_mc")
    dt = np.dtype([("home", np.uint32), ("j", np.uint32), ("fate", np.int32), ("n_scat", np.uint64),
                   ("n_steps", np.uint64), ("D_kpc", np.float64), ("x_end", np.float64)], align=True)
    arr = np.frombuffer(recs, dtype=dt, count=k1 - k0).copy()
    return arr, cnt
