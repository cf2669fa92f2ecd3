"""Gradients of the recombination history through the hand-written adjoint.

A trajectory runs rec_step over node redshifts zs[0..S] with the Monte-Carlo
tallies of every step held fixed (given, or produced by lya_transport in the
forward run and stored).  The reverse sweep replays segments of
ceil(sqrt(S)) steps from stored checkpoints and calls rec_step_adjoint step by
step, so memory holds about 2 sqrt(S) states instead of S.  Objectives are the
volume-averaged X_e at a node (Sec. II.A) or the visibility function there
(rec_objective); gradients are with respect to the per-cell overdensity, the
initial temperature and ionisation fraction, and the absorbed-Ly-alpha
fraction a_i = tally_i / sum(tally) (the same perturbation at every step).

FP64 form only (the adjoint is binary64).  The box's buffers are overwritten
by the replays.
"""
from __future__ import annotations

import math

import numpy as np

from . import rec


class Trajectory:
    def __init__(self, box: "rec.Box", zs, tallies=None, run_transport=False, checkpoint_every=None):
        import torch
        if box.precision != "fp64":
            raise rec.RecError("the adjoint trajectory needs the FP64 form")
        self.torch = torch
        self.box = box
        self.zs = np.asarray(zs, dtype=np.float64)
        self.S = self.zs.size - 1
        self.k = int(checkpoint_every or max(1, math.ceil(math.sqrt(self.S))))
        self.given = tallies
        self.run_transport = run_transport
        dev = box.x.device
        # every buffer of the trajectory is made on the box's stream, where the
        # library's kernels read and write it
        with torch.cuda.stream(box.stream):
            self.tallies = torch.zeros(self.S, box.n3, dtype=torch.int32, device=dev)
            self._v4_0 = box.vel4.clone()  # velocity at the first node
        self.ckpt = {}
        box.ensure_stats(self.S + 1)

    def _set_state(self, x, T, v4):
        b = self.box
        b.x.copy_(x)
        b.T.copy_(T)
        b.vel4.copy_(v4)

    def _snapshot(self):
        b = self.box
        return b.x.clone(), b.T.clone(), b.vel4.clone()

    def _prepare_tally(self, s, z):
        b = self.box
        if self.given is not None:
            t = self.given[s]
            t = t if hasattr(t, "data_ptr") else self.torch.as_tensor(np.asarray(t, np.uint32).view(np.int32))
            b.tally.copy_(t.to(b.tally.device))
        elif self.run_transport:
            b.tally.zero_()
            b.refresh(z)
            b.transport(s, z)
        else:
            b.tally.zero_()
        self.tallies[s].copy_(b.tally)

    def forward(self, x0, T0) -> np.ndarray:
        """Runs the S steps from (x0, T0); returns X_e at every node."""
        torch, b = self.torch, self.box
        with torch.cuda.stream(b.stream):
            self._set_state(torch.as_tensor(x0, dtype=torch.float64, device=b.x.device),
                            torch.as_tensor(T0, dtype=torch.float64, device=b.x.device), b.vel4)
            self.x0 = b.x.clone()
            b.vel4.copy_(self._v4_0)
            self.ckpt = {}
            for s in range(self.S):
                if s % self.k == 0:
                    self.ckpt[s] = self._snapshot()
                self._prepare_tally(s, self.zs[s])
                b.tally.copy_(self.tallies[s])
                b.refresh(self.zs[s])
                if s == 0:
                    b.volume_stats(slot=0)  # X_e of the start node
                b.step(s, self.zs[s], self.zs[s + 1], slot=s + 1)
        st = b.stats_all()
        return np.array([st[s]["X_e"] for s in range(self.S + 1)])

    def backward(self, dJ_dXe):
        """Reverse sweep for weights dJ/dX_e at every node.
        Returns (g_delta, g_T0, g_x0, g_a) as float64 CUDA tensors."""
        torch, b = self.torch, self.box
        w = np.asarray(dJ_dXe, dtype=np.float64)
        dev = b.x.device
        z = lambda: torch.zeros(b.n3, dtype=torch.float64, device=dev)
        with torch.cuda.stream(b.stream):
            xbar, Tbar, g_delta, g_a = z(), z(), z(), z()
            for s0 in reversed(range(0, self.S, self.k)):
                s1 = min(s0 + self.k, self.S)
                states = [self.ckpt[s0]]
                self._set_state(*self.ckpt[s0])
                for s in range(s0, s1 - 1):
                    b.tally.copy_(self.tallies[s])
                    b.refresh(self.zs[s])
                    b.step(s, self.zs[s], self.zs[s + 1])
                    states.append(self._snapshot())
                for s in reversed(range(s0, s1)):
                    x_s, T_s, v_s = states[s - s0]
                    tal = self.tallies[s] if b.mixing == "tally" else None
                    b.step_adjoint(s, self.zs[s], self.zs[s + 1], x_s, T_s, v_s, tal, xbar, Tbar, None, g_delta, g_a,
                                   Xe_bar_out=float(w[s + 1]))
            if w[0] != 0.0:
                b.xe_adjoint(self.x0, float(w[0]), xbar, g_delta)
        return g_delta, Tbar, xbar, g_a


def objective_and_gradients(box, zs, x0, T0, tallies=None, run_transport=False, objective=1, z_star=1100.0,
                            checkpoint_every=None):
    """J and its gradients (dict) for one trajectory."""
    traj = Trajectory(box, zs, tallies, run_transport, checkpoint_every)
    Xe = traj.forward(x0, T0)
    J, dJ = rec.objective(zs, Xe, objective, z_star)
    g_delta, g_T0, g_x0, g_a = traj.backward(dJ)
    return J, dict(delta=g_delta, T0=g_T0, x0=g_x0, a=g_a), Xe


def recombination_objective(box, zs, delta, x0, T0, a_pert, tallies=None, objective=1, z_star=1100.0):
    """torch.autograd entry point: J(delta, x0, T0, a_pert) with the tallies held
    fixed; a_pert (zeros) is the perturbation of the absorbed fraction at every
    step, present so that autograd returns its gradient."""
    import torch

    class _Fn(torch.autograd.Function):
        @staticmethod
        def forward(ctx, delta_t, x0_t, T0_t, a_t):
            box.delta.copy_(delta_t.to(box.delta.device, box.delta.dtype))
            traj = Trajectory(box, zs, tallies)
            Xe = traj.forward(x0_t, T0_t)
            J, dJ = rec.objective(zs, Xe, objective, z_star)
            ctx.traj, ctx.dJ = traj, dJ
            return torch.tensor(J, dtype=torch.float64, device=delta_t.device)

        @staticmethod
        def backward(ctx, gJ):
            g_delta, g_T0, g_x0, g_a = ctx.traj.backward(ctx.dJ * float(gJ))
            return g_delta, g_x0, g_T0, g_a

    return _Fn.apply(delta, x0, T0, a_pert)
