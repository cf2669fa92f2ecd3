"""Thin Python binding of the C ABI in include/rec.h (argument marshalling only).

Device buffers are torch tensors on the current CUDA device; every step of
the path runs in the CUDA kernels of librec.so.  There is no CPU fallback:
constructing a Box without a CUDA device or without the built library raises.

    box = Box(n, delta, U, n_packets, precision="mixed")   # uploads the fields
    box.state_init(z0)                                     # Saha x_e, T = T_gamma
    for s, (za, zb) in enumerate(zip(zs[:-1], zs[1:])):
        box.transport(s, za)                               # Ly-alpha packets -> tallies
        box.step(s, za, zb)                                # x_e, T, U update
    stats = box.stats()                                    # last rec_stats record
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

REC_OK, REC_EINVAL, REC_ENOMEM, REC_ECUDA, REC_ETIMEOUT, REC_ESTATE = range(6)
PREC = {"fp64": 0, "mixed": 1}
MIXING = {"tally": 0, "full": 1, "local": 2, "partial": 3}
_lib = None


class Params(C.Structure):
    _fields_ = [("h", C.c_double), ("omega_b_h2", C.c_double), ("omega_c_h2", C.c_double), ("Y_p", C.c_double),
                ("T_cmb0", C.c_double), ("N_eff", C.c_double), ("L_box_kpc", C.c_double), ("fudge", C.c_double),
                ("heating", C.c_double), ("seed", C.c_uint64), ("n_sub", C.c_int32), ("precision", C.c_int32),
                ("mixing", C.c_int32), ("n_quantiles", C.c_int32),
                ("emission_quantiles", C.POINTER(C.c_double)), ("f_alpha", C.c_double)]


class BoxDesc(C.Structure):
    _fields_ = [("n", C.c_int32), ("delta", C.c_void_p), ("vel4", C.c_void_p), ("x_e", C.c_void_p),
                ("T", C.c_void_p), ("tally", C.c_void_p), ("emis", C.c_void_p), ("n_packets", C.c_uint64)]


class Stats(C.Structure):
    _fields_ = [("emitted", C.c_uint64), ("absorbed", C.c_uint64), ("capped", C.c_uint64),
                ("crossings", C.c_uint64), ("queued", C.c_uint64), ("X_e", C.c_double), ("lambda_", C.c_double), ("C_mix", C.c_double),
                ("S1s", C.c_double), ("newton_passes", C.c_int32), ("flags", C.c_int32), ("requeued", C.c_uint64)]


class Tuning(C.Structure):
    """rec_tuning: transport launch and scheduling parameters (speed only)."""
    _fields_ = [("emit_blocks_per_sm", C.c_int32), ("march_blocks_per_sm", C.c_int32), ("march_refill", C.c_int32),
                ("march_chunk", C.c_int32), ("tile", C.c_int32), ("march_halo", C.c_int32)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class McParams(C.Structure):
    """lya_mc_params: one resonant-scattering Monte-Carlo run (Appendix A)."""
    _fields_ = [("z", C.c_double), ("eps", C.c_double), ("x_lost", C.c_double), ("zeta", C.c_double),
                ("lambda2g", C.c_double), ("A_alpha", C.c_double), ("n_photons", C.c_uint64),
                ("max_steps", C.c_uint64), ("step", C.c_int32), ("pending", C.c_int32), ("arith", C.c_int32),
                ("reserved", C.c_int32)]


class McStats(C.Structure):
    _fields_ = [("count", C.c_uint64 * 4), ("sampler_caps", C.c_uint64), ("steps", C.c_uint64),
                ("scatterings", C.c_uint64), ("nonfinite", C.c_uint64)]


# lya_mc_photon as a numpy record
MC_PHOTON = np.dtype([("home", np.uint32), ("j", np.uint32), ("fate", np.int32), ("reserved", np.uint32),
                      ("n_scat", np.uint64), ("n_steps", np.uint64), ("D_kpc", np.float64), ("x_end", np.float64)])
MC_FATES = ("lost", "two_photon", "ionised", "capped")
A_2P1S = 6.2649e8  # 2p -> 1s decay rate, 1/s


class RecError(RuntimeError):
    """A failed call; .status is the rec_status it returned (None for binding-side checks)."""

    def __init__(self, msg, status=None):
        super().__init__(msg)
        self.status = status


def lib():
    """Load (building first if needed) the in-tree CUDA library."""
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        P, d, i32, u32, vp = C.POINTER, C.c_double, C.c_int32, C.c_uint32, C.c_void_p
        L.rec_init.argtypes = [P(Params), P(BoxDesc), i32, vp, P(vp)]
        L.rec_state_init.argtypes = [vp, d]
        L.rec_refresh.argtypes = [vp, d]
        L.lya_transport.argtypes = [vp, i32, d, vp]
        L.rec_step.argtypes = [vp, i32, d, d, vp]
        L.rec_step_noalloc.argtypes = [P(Params), P(BoxDesc), d, d, vp, vp]
        L.rec_graph_step.argtypes = [vp, i32, d, d, vp]
        L.rec_get_tuning.argtypes = [vp, P(Tuning)]
        L.rec_set_tuning.argtypes = [vp, P(Tuning)]
        L.rec_step_adjoint.argtypes = [vp, i32, d, d, vp, vp, vp, vp, vp, vp, vp, vp, vp, d]
        L.rec_xe_adjoint.argtypes = [vp, vp, d, vp, vp]
        L.rec_transport_params.argtypes = [P(Params), i32, d, P(d)]
        L.rec_objective.argtypes = [P(Params), P(d), P(d), i32, i32, d, P(d), P(d)]
        L.rec_timing.argtypes = [vp, i32]
        L.rec_kernel_times.argtypes = [vp, P(d), P(C.c_int64)]
        L.rec_step_trbdf2.argtypes = [vp, i32, d, d, vp]
        L.rec_set_f_alpha.argtypes = [vp, d]
        L.lya_scatter_mc.argtypes = [vp, P(McParams), vp, vp, vp]
        L.lya_voigt.argtypes = [d, C.c_int64, P(d), P(d)]
        L.lya_voigt_mixed.argtypes = [d, C.c_int64, P(d), P(d)]
        L.lya_mc_scalars.argtypes = [P(Params), P(McParams), i32, P(d)]
        L.lya_mc_redistribution_host.argtypes = [d, d, P(d), C.c_uint64, C.c_int64, P(d), P(d), P(d),
                                                 P(C.c_uint64)]
        L.lya_mc_mixing_fraction.argtypes = [vp, vp, C.c_uint64, P(d), i32, vp, vp]
        L.rec_volume_stats.argtypes = [vp, vp]
        L.rec_set_wait_limit.argtypes = [vp, u32]
        L.rec_sync.argtypes = [vp]
        L.rec_free.argtypes = [vp]
        L.rec_free.restype = None
        L.rec_last_error.argtypes = [vp]
        L.rec_last_error.restype = C.c_char_p
        for f in ("rec_init", "rec_state_init", "rec_refresh", "lya_transport", "rec_step", "rec_step_noalloc", "rec_graph_step", "rec_get_tuning", "rec_set_tuning",
                  "rec_step_adjoint", "rec_xe_adjoint", "rec_transport_params", "rec_objective", "rec_timing", "rec_kernel_times",
                  "lya_scatter_mc", "lya_voigt", "rec_step_trbdf2", "lya_mc_scalars",
                  "lya_mc_redistribution_host", "lya_voigt_mixed", "rec_set_f_alpha", "lya_mc_mixing_fraction",
                  "rec_volume_stats", "rec_set_wait_limit", "rec_sync"):
            getattr(L, f).restype = C.c_int
        _lib = L
    return _lib


def make_params(precision="mixed", mixing="tally", seed=1, n_sub=1, quantiles=None, **cosmo) -> tuple:
    """rec_params with the Sec. II.C defaults; returns (Params, quantile array kept alive)."""
    if quantiles is None:
        from .inputs import doppler_quantiles
        quantiles = doppler_quantiles()
    q = np.ascontiguousarray(quantiles, dtype=np.float64)
    base = dict(h=0.67, omega_b_h2=0.0224, omega_c_h2=0.12, Y_p=0.24, T_cmb0=2.7255, N_eff=3.046, L_box_kpc=24.0,
                fudge=1.14, heating=0.0, f_alpha=1.0)
    base.update(cosmo)
    p = Params(**base, seed=seed, n_sub=n_sub, precision=PREC[precision], mixing=MIXING[mixing],
               n_quantiles=q.size, emission_quantiles=q.ctypes.data_as(C.POINTER(C.c_double)))
    return p, q


def transport_params(n: int, z: float, **kw):
    """(kappa, cth) as the library computes them (host only)."""
    p, _q = make_params(**kw)
    out = (C.c_double * 2)()
    rc = lib().rec_transport_params(C.byref(p), n, z, out)
    if rc != REC_OK:
        raise RecError(lib().rec_last_error(None).decode())
    return out[0], out[1]


def objective(zs, Xe, objective=1, z_star=1100.0, **kw):
    """(J, dJ/dX_e per node) of an X_e history (host computation in the library)."""
    p, _q = make_params(**kw)
    z = np.ascontiguousarray(zs, dtype=np.float64)
    X = np.ascontiguousarray(Xe, dtype=np.float64)
    J = C.c_double()
    dJ = np.zeros(z.size)
    dp = lambda a: a.ctypes.data_as(C.POINTER(C.c_double))
    rc = lib().rec_objective(C.byref(p), dp(z), dp(X), z.size, int(objective), float(z_star), C.byref(J), dp(dJ))
    if rc != REC_OK:
        raise RecError(lib().rec_last_error(None).decode())
    return J.value, dJ


def voigt(a: float, y, mixed=False) -> np.ndarray:
    """H(a, y) as the scattering Monte Carlo evaluates it (host computation);
    mixed=True: the binary32 evaluation of the mixed-arithmetic form."""
    yy = np.ascontiguousarray(y, dtype=np.float64).ravel()
    H = np.empty_like(yy)
    dp = lambda v: v.ctypes.data_as(C.POINTER(C.c_double))
    fn = lib().lya_voigt_mixed if mixed else lib().lya_voigt
    rc = fn(float(a), yy.size, dp(yy), dp(H))
    if rc != REC_OK:
        raise RecError(lib().rec_last_error(None).decode())
    return H


MC_ARITH = {"fp64": 0, "mixed": 1}


def mc_redistribution_mixed(a, y, seed, m, kin=(0.0, 0.0, 1.0)):
    """The mixed form's redistribution run on the host: (p_par, y_out - y, k_out, caps)."""
    dp = lambda v: v.ctypes.data_as(C.POINTER(C.c_double))
    k = np.ascontiguousarray(kin, dtype=np.float64)
    pp, dy, ko = np.empty(m), np.empty(m), np.empty((m, 3))
    caps = C.c_uint64(0)
    rc = lib().lya_mc_redistribution_host(float(a), float(y), dp(k), int(seed), int(m), dp(pp), dp(dy), dp(ko),
                                          C.byref(caps))
    if rc != REC_OK:
        raise RecError(lib().rec_last_error(None).decode())
    return pp, dy, ko, caps.value


def mc_scalars(z, n=1, **kw) -> dict:
    """Monte-Carlo snapshot scalars as lya_scatter_mc uses them (host only).
    kw: lya_mc_params fields (zeta, lambda2g, eps, A_alpha, ...) and
    cosmology overrides of make_params."""
    mkeys = {"eps", "x_lost", "zeta", "lambda2g", "A_alpha", "max_steps", "step", "pending", "arith"}
    mp = mc_params(z, 1, **{k: v for k, v in kw.items() if k in mkeys})
    p, _q = make_params(**{k: v for k, v in kw.items() if k not in mkeys})
    out = (C.c_double * 12)()
    rc = lib().lya_mc_scalars(C.byref(p), C.byref(mp), int(n), out)
    if rc != REC_OK:
        raise RecError(lib().rec_last_error(None).decode())
    keys = ("a", "vth", "sig0", "dxdl", "p_ion", "p_2g", "beta", "Lambda", "H", "nH", "Tg", "cells_per_m")
    return dict(zip(keys, list(out)))


def mc_params(z, n_photons, eps=0.1, x_lost=1.0e4, zeta=1.0, lambda2g=-1.0, A_alpha=A_2P1S, max_steps=10 ** 9,
              step=0, pending=0, arith="fp64") -> McParams:
    return McParams(z=z, eps=eps, x_lost=x_lost, zeta=zeta, lambda2g=lambda2g, A_alpha=A_alpha,
                    n_photons=int(n_photons), max_steps=int(max_steps), step=int(step), pending=int(pending),
                    arith=MC_ARITH[arith], reserved=0)


class Batch:
    """Several boxes in one context (n_boxes > 1): every phase of a call is one
    launch over all boxes.  boxes: list of (n, delta, U, n_packets).  Fields live
    in per-box torch CUDA tensors; statistics have one record per box."""

    def __init__(self, boxes, precision="mixed", mixing="tally", seed=1, n_sub=1, quantiles=None, stream=None,
                 **cosmo):
        import torch
        if not torch.cuda.is_available():
            raise RecError("a CUDA device is required (there is no CPU fallback)")
        if len(boxes) < 2:
            raise RecError("a batch needs at least two boxes (use Box for one)")
        self.torch = torch
        self.precision = precision
        self.mixing = mixing
        fdt = torch.float32 if precision == "mixed" else torch.float64
        dev = torch.device("cuda", torch.cuda.current_device())
        self.stream = stream or torch.cuda.current_stream(dev)
        self.n = [int(b[0]) for b in boxes]
        self.n_packets = [int(b[3]) for b in boxes]
        self.delta, self.vel4, self.x, self.T, self.tally, self.emis = [], [], [], [], [], []
        with torch.cuda.stream(self.stream):
            for (n, delta, U, _npk) in boxes:
                n3 = int(n) ** 3
                d = torch.as_tensor(np.asarray(delta).ravel(), dtype=torch.float64)
                if d.numel() != n3:
                    raise RecError("delta must have n^3 cells")
                u = torch.as_tensor(np.asarray(U).reshape(-1, 3), dtype=torch.float64)
                v4 = torch.zeros(n3, 4, dtype=torch.float64)
                v4[:, :3] = u
                self.delta.append(d.to(dev, fdt))
                self.vel4.append(v4.to(dev, fdt).contiguous())
                self.x.append(torch.zeros(n3, dtype=torch.float64, device=dev))
                self.T.append(torch.zeros(n3, dtype=fdt, device=dev))
                self.tally.append(torch.zeros(n3, dtype=torch.int32, device=dev))
                self.emis.append(torch.zeros(n3, dtype=fdt, device=dev))
            self._stats = torch.zeros(len(boxes), C.sizeof(Stats), dtype=torch.uint8, device=dev)
        self._params, self._q = make_params(precision, mixing, seed, n_sub, quantiles, **cosmo)
        descs = (BoxDesc * len(boxes))()
        for i in range(len(boxes)):
            descs[i] = BoxDesc(self.n[i], self.delta[i].data_ptr(), self.vel4[i].data_ptr(), self.x[i].data_ptr(),
                               self.T[i].data_ptr(), self.tally[i].data_ptr(), self.emis[i].data_ptr(),
                               self.n_packets[i])
        ctx = C.c_void_p()
        self.stream.synchronize()
        rc = lib().rec_init(C.byref(self._params), descs, len(boxes), C.c_void_p(self.stream.cuda_stream),
                            C.byref(ctx))
        if rc != REC_OK:
            raise RecError(f"rec_init: {lib().rec_last_error(None).decode()} (status {rc})")
        self.ctx = ctx

    def _check(self, rc, what):
        if rc != REC_OK:
            raise RecError(f"{what}: {lib().rec_last_error(self.ctx).decode()} (status {rc})", rc)

    def state_init(self, z):
        self._check(lib().rec_state_init(self.ctx, z), "rec_state_init")

    def refresh(self, z):
        self._check(lib().rec_refresh(self.ctx, z), "rec_refresh")

    def transport(self, step, z):
        self._check(lib().lya_transport(self.ctx, int(step), z, C.c_void_p(self._stats.data_ptr())), "lya_transport")

    def step(self, step, z_from, z_to):
        self._check(lib().rec_step(self.ctx, int(step), z_from, z_to, C.c_void_p(self._stats.data_ptr())), "rec_step")

    def graph_step(self, step, z_from, z_to):
        self._check(lib().rec_graph_step(self.ctx, int(step), z_from, z_to, C.c_void_p(self._stats.data_ptr())),
                    "rec_graph_step")

    def set_wait_limit(self, polls):
        self._check(lib().rec_set_wait_limit(self.ctx, int(polls)), "rec_set_wait_limit")

    def sync(self):
        self._check(lib().rec_sync(self.ctx), "rec_sync")

    def volume_stats(self):
        """rec_volume_stats: X_e, lambda and S1s of every box's current state into the records."""
        self._check(lib().rec_volume_stats(self.ctx, C.c_void_p(self._stats.data_ptr())), "rec_volume_stats")

    def timing(self, enable=True):
        self._check(lib().rec_timing(self.ctx, 1 if enable else 0), "rec_timing")

    def tuning(self) -> dict:
        return _get_tuning(self)

    def set_tuning(self, **kw):
        _set_tuning(self, **kw)

    def kernel_times(self) -> dict:
        ms = (C.c_double * 7)()
        ln = (C.c_int64 * 7)()
        self._check(lib().rec_kernel_times(self.ctx, ms, ln), "rec_kernel_times")
        return {g: (ms[i], ln[i]) for i, g in enumerate(Box.TIMER_GROUPS)}

    def stats(self) -> list:
        """One statistics record per box."""
        self.stream.synchronize()
        return [_stats_dict(Stats.from_buffer_copy(row.tobytes())) for row in self._stats.cpu().numpy()]

    def tally_np(self, b) -> np.ndarray:
        self.stream.synchronize()
        return self.tally[b].cpu().numpy().view(np.uint32)

    def host(self, name, b) -> np.ndarray:
        self.stream.synchronize()
        return getattr(self, name)[b].cpu().numpy()

    def close(self):
        if getattr(self, "ctx", None):
            lib().rec_free(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _get_tuning(obj) -> dict:
    t = Tuning()
    obj._check(lib().rec_get_tuning(obj.ctx, C.byref(t)), "rec_get_tuning")
    return t.as_dict()


def _set_tuning(obj, **kw):
    t = Tuning()
    obj._check(lib().rec_get_tuning(obj.ctx, C.byref(t)), "rec_get_tuning")
    for k, v in kw.items():
        setattr(t, k, int(v))
    obj._check(lib().rec_set_tuning(obj.ctx, C.byref(t)), "rec_set_tuning")


def _stats_dict(s) -> dict:
    return dict(emitted=s.emitted, absorbed=s.absorbed, capped=s.capped, crossings=s.crossings, queued=s.queued,
                X_e=s.X_e, lam=s.lambda_, C=s.C_mix, S1s=s.S1s, newton_passes=s.newton_passes, flags=s.flags,
                requeued=s.requeued)


class Box:
    """One periodic box and its context.  Fields live in torch CUDA tensors."""

    def __init__(self, n, delta, U, n_packets, precision="mixed", mixing="tally", seed=1, n_sub=1, quantiles=None,
                 stream=None, n_stats=1, **cosmo):
        import torch
        if not torch.cuda.is_available():
            raise RecError("a CUDA device is required (there is no CPU fallback)")
        self.torch = torch
        self.n = int(n)
        self.n3 = self.n ** 3
        self.precision = precision
        self.mixing = mixing
        fdt = torch.float32 if precision == "mixed" else torch.float64
        dev = torch.device("cuda", torch.cuda.current_device())
        self.stream = stream or torch.cuda.current_stream(dev)
        d = torch.as_tensor(np.asarray(delta).ravel(), dtype=torch.float64)
        if d.numel() != self.n3:
            raise RecError("delta must have n^3 cells")
        u = torch.as_tensor(np.asarray(U).reshape(-1, 3), dtype=torch.float64)
        v4 = torch.zeros(self.n3, 4, dtype=torch.float64)
        v4[:, :3] = u
        with torch.cuda.stream(self.stream):
            self.delta = d.to(dev, fdt)
            self.vel4 = v4.to(dev, fdt).contiguous()
            self.x = torch.zeros(self.n3, dtype=torch.float64, device=dev)
            self.T = torch.zeros(self.n3, dtype=fdt, device=dev)
            self.tally = torch.zeros(self.n3, dtype=torch.int32, device=dev)  # read as uint32
            self.emis = torch.zeros(self.n3, dtype=fdt, device=dev)
            self._stats = torch.zeros(max(1, int(n_stats)), C.sizeof(Stats), dtype=torch.uint8, device=dev)
        self.n_packets = int(n_packets)
        self._params, self._q = make_params(precision, mixing, seed, n_sub, quantiles, **cosmo)
        desc = BoxDesc(self.n, self.delta.data_ptr(), self.vel4.data_ptr(), self.x.data_ptr(), self.T.data_ptr(),
                       self.tally.data_ptr(), self.emis.data_ptr(), self.n_packets)
        ctx = C.c_void_p()
        self.stream.synchronize()
        rc = lib().rec_init(C.byref(self._params), C.byref(desc), 1, C.c_void_p(self.stream.cuda_stream),
                            C.byref(ctx))
        if rc != REC_OK:
            raise RecError(f"rec_init: {lib().rec_last_error(None).decode()} (status {rc})")
        self.ctx = ctx
        self.mc_records = None

    # ---- calls -----------------------------------------------------------------------
    def _check(self, rc, what):
        if rc != REC_OK:
            raise RecError(f"{what}: {lib().rec_last_error(self.ctx).decode()} (status {rc})", rc)

    def state_init(self, z):
        self._check(lib().rec_state_init(self.ctx, z), "rec_state_init")

    def refresh(self, z):
        self._check(lib().rec_refresh(self.ctx, z), "rec_refresh")

    def ensure_stats(self, n_slots):
        """Grow the device statistics array to at least n_slots records."""
        if self._stats.shape[0] < n_slots:
            self.stream.synchronize()
            new = self.torch.zeros(n_slots, C.sizeof(Stats), dtype=self.torch.uint8, device=self._stats.device)
            new[: self._stats.shape[0]] = self._stats
            self._stats = new

    def _slot(self, slot):
        return C.c_void_p(self._stats[int(slot)].data_ptr())

    def transport(self, step, z, slot=0):
        self._check(lib().lya_transport(self.ctx, int(step), z, self._slot(slot)), "lya_transport")

    def step(self, step, z_from, z_to, slot=0):
        self._check(lib().rec_step(self.ctx, int(step), z_from, z_to, self._slot(slot)), "rec_step")

    def graph_step(self, step, z_from, z_to, slot=0):
        """transport(step, z_from) + step(step, z_from, z_to) as one CUDA graph launch."""
        self._check(lib().rec_graph_step(self.ctx, int(step), z_from, z_to, self._slot(slot)), "rec_graph_step")

    def set_wait_limit(self, polls):
        """rec_set_wait_limit: polls before a bounded device-side wait gives up."""
        self._check(lib().rec_set_wait_limit(self.ctx, int(polls)), "rec_set_wait_limit")

    def sync(self):
        """rec_sync: wait for the stream; raises RecError (status REC_ETIMEOUT) if a
        bounded device-side wait expired since the last sync."""
        self._check(lib().rec_sync(self.ctx), "rec_sync")

    def volume_stats(self, slot=0):
        """rec_volume_stats: X_e, lambda and S1s of the current state into record `slot`."""
        self._check(lib().rec_volume_stats(self.ctx, self._slot(slot)), "rec_volume_stats")

    def set_f_alpha(self, f_alpha):
        """Partial mixing: the share of the full-mixing rate for the following steps."""
        self._check(lib().rec_set_f_alpha(self.ctx, float(f_alpha)), "rec_set_f_alpha")

    def step_trbdf2(self, step, z_from, z_to, slot=0):
        """rec_step_trbdf2: the second-order (TR-BDF2) step (FP64 form, tally or full mixing)."""
        self._check(lib().rec_step_trbdf2(self.ctx, int(step), z_from, z_to, self._slot(slot)), "rec_step_trbdf2")

    def step_noalloc(self, z_from, z_to, slot=0):
        """rec_step_noalloc on this machine's fields and parameters (the context is not used)."""
        desc = BoxDesc(self.n, self.delta.data_ptr(), self.vel4.data_ptr(), self.x.data_ptr(), self.T.data_ptr(),
                       self.tally.data_ptr(), self.emis.data_ptr(), self.n_packets)
        rc = lib().rec_step_noalloc(C.byref(self._params), C.byref(desc), z_from, z_to,
                                    C.c_void_p(self.stream.cuda_stream), self._slot(slot))
        if rc != REC_OK:
            raise RecError(f"rec_step_noalloc: {lib().rec_last_error(None).decode()} (status {rc})")

    def step_adjoint(self, step, z_from, z_to, x_in, T_in, vel4_in, tally_in, xbar, Tbar, Ubar, g_delta, g_a,
                     Xe_bar_out=0.0):
        ptr = lambda t: None if t is None else C.c_void_p(t.data_ptr())
        self._check(lib().rec_step_adjoint(self.ctx, int(step), z_from, z_to, ptr(x_in), ptr(T_in), ptr(vel4_in),
                                           ptr(tally_in), ptr(xbar), ptr(Tbar), ptr(Ubar), ptr(g_delta), ptr(g_a),
                                           float(Xe_bar_out)), "rec_step_adjoint")

    def xe_adjoint(self, x, Xe_bar, xbar, g_delta):
        self._check(lib().rec_xe_adjoint(self.ctx, C.c_void_p(x.data_ptr()), float(Xe_bar),
                                         C.c_void_p(xbar.data_ptr()), C.c_void_p(g_delta.data_ptr())),
                    "rec_xe_adjoint")

    def scatter_mc(self, z, n_photons, prefix=None, records=True, **kw):
        """Resonant-scattering Monte Carlo (lya_scatter_mc) in this box's fields.
        prefix: photons per cell as an exclusive prefix (n^3 + 1 integers), or
        None for the even allocation.  kw: the other lya_mc_params fields.
        Returns (records or None, stats dict); synchronises."""
        torch = self.torch
        mp = mc_params(z, n_photons, **kw)
        dev = self.x.device
        with torch.cuda.stream(self.stream):
            pre = None
            if prefix is not None:
                pa = np.ascontiguousarray(prefix, dtype=np.int64).ravel()
                if pa.size != self.n3 + 1:
                    raise RecError("prefix must have n^3 + 1 entries")
                pre = torch.as_tensor(pa.astype(np.uint32).view(np.int32)).to(dev)
            rec = torch.empty(int(n_photons) * MC_PHOTON.itemsize if records else 0, dtype=torch.uint8, device=dev)
            st = torch.zeros(C.sizeof(McStats), dtype=torch.uint8, device=dev)
        ptr = lambda t: None if t is None or t.numel() == 0 else C.c_void_p(t.data_ptr())
        self._check(lib().lya_scatter_mc(self.ctx, C.byref(mp), ptr(pre), ptr(rec), ptr(st)), "lya_scatter_mc")
        self.mc_records = rec if records else None  # device copy, for mixing_fraction
        self.stream.synchronize()
        s = McStats.from_buffer_copy(st.cpu().numpy().tobytes())
        stats = dict(count=[int(v) for v in s.count], sampler_caps=int(s.sampler_caps), steps=int(s.steps),
                     scatterings=int(s.scatterings), nonfinite=int(s.nonfinite))
        out = rec.cpu().numpy().view(MC_PHOTON) if records else None
        return out, stats

    def mixing_fraction(self, D_kpc, records=None):
        """f_alpha(D) of Sec. III.B (lya_mc_mixing_fraction) from the device records
        of the last scatter_mc call (or a device uint8 tensor of records).
        Returns (f, f_min, f_max, counts): f excludes capped photons, [f_min, f_max]
        is the range their unknown fates allow, counts the photons per fate."""
        torch = self.torch
        recs = self.mc_records if records is None else records
        if recs is None or recs.numel() == 0:
            raise RecError("no device Monte-Carlo records: run scatter_mc(records=True) first")
        n_ph = recs.numel() // MC_PHOTON.itemsize
        D = np.ascontiguousarray(np.atleast_1d(D_kpc), dtype=np.float64)
        with torch.cuda.stream(self.stream):
            out = torch.empty(3 * D.size, dtype=torch.float64, device=recs.device)
            cnt = torch.empty(4, dtype=torch.int64, device=recs.device)
        self._check(lib().lya_mc_mixing_fraction(self.ctx, C.c_void_p(recs.data_ptr()), int(n_ph),
                                                 D.ctypes.data_as(C.POINTER(C.c_double)), int(D.size),
                                                 C.c_void_p(out.data_ptr()), C.c_void_p(cnt.data_ptr())),
                    "lya_mc_mixing_fraction")
        self.stream.synchronize()
        o = out.cpu().numpy().reshape(3, D.size)
        return o[0], o[1], o[2], cnt.cpu().numpy().astype(np.uint64)

    TIMER_GROUPS = ("alloc", "emit", "march", "transport_end", "rec_step", "adjoint", "other")

    def tuning(self) -> dict:
        return _get_tuning(self)

    def set_tuning(self, **kw):
        _set_tuning(self, **kw)

    def timing(self, enable=True):
        self._check(lib().rec_timing(self.ctx, 1 if enable else 0), "rec_timing")

    def kernel_times(self) -> dict:
        """{group: (ms, launches)} since timing(True)."""
        ms = (C.c_double * 7)()
        ln = (C.c_int64 * 7)()
        self._check(lib().rec_kernel_times(self.ctx, ms, ln), "rec_kernel_times")
        return {g: (ms[i], ln[i]) for i, g in enumerate(self.TIMER_GROUPS)}

    # ---- host views (synchronising) -------------------------------------------------------
    def stats(self, slot=0) -> dict:
        return self.stats_all()[int(slot)]

    def stats_all(self) -> list:
        self.stream.synchronize()
        raw = self._stats.cpu().numpy()
        out = []
        for row in raw:
            out.append(_stats_dict(Stats.from_buffer_copy(row.tobytes())))
        return out

    def tally_np(self) -> np.ndarray:
        self.stream.synchronize()
        return self.tally.cpu().numpy().view(np.uint32)

    def host(self, name) -> np.ndarray:
        self.stream.synchronize()
        return getattr(self, name).cpu().numpy()

    def close(self):
        if getattr(self, "ctx", None):
            lib().rec_free(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
