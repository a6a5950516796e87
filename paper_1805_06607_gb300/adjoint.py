"""PyTorch autograd functions over the library's discrete adjoint (FP64 systems).

Each function's forward and backward run in the library's CUDA kernels through the C ABI
(``sbp_rhs_eval`` / ``sbp_rhs_eval_vjp``, ``sbp_overset_interp`` / ``sbp_overset_interp_vjp``,
``sbp_adjoint_probe``); PyTorch only chains them with whatever the caller computes around
them (for example the far-field state as a function of the free-stream Mach number).

The far-field state ``qinf`` (4 values) is an explicit input of every function so that its
gradient can flow; it is written into the system before each library call.
"""
from __future__ import annotations

import torch


def _set_qinf(system, qinf):
    system.set_freestream([float(v) for v in qinf.detach().cpu().reshape(4)])


class RhsEval(torch.autograd.Function):
    """dq/dt of one mesh (Sec. 2.2 eq. (int)) as a function of both meshes' states and qinf."""

    @staticmethod
    def forward(ctx, system, k, q_self, q_other, qinf):
        _set_qinf(system, qinf)
        out = system.rhs_eval(k, q_self, q_other)
        ctx.system, ctx.k = system, k
        ctx.qinf = qinf.detach().clone()
        ctx.save_for_backward(q_self, q_other)
        return out

    @staticmethod
    def backward(ctx, g):
        q_self, q_other = ctx.saved_tensors
        _set_qinf(ctx.system, ctx.qinf)
        lq_s, lq_o, lqinf = ctx.system.rhs_eval_vjp(ctx.k, q_self, q_other, g.contiguous())
        gq = torch.as_tensor(lqinf, dtype=ctx.qinf.dtype, device=ctx.qinf.device)
        return None, None, lq_s, lq_o, gq


class OversetInterp(torch.autograd.Function):
    """Receiver values (states, viscous fluxes) of mesh ``recv`` from the donor state (Sec. 2.2)."""

    @staticmethod
    def forward(ctx, system, recv, q_donor):
        qhat, fvhat = system.overset_interp(recv, q_donor, viscous_fluxes=True)
        ctx.system, ctx.recv = system, recv
        ctx.save_for_backward(q_donor)
        return qhat.clone(), fvhat.clone()

    @staticmethod
    def backward(ctx, gq, gfv):
        (q_donor,) = ctx.saved_tensors
        lq = ctx.system.overset_interp_vjp(ctx.recv, q_donor, gq.contiguous(),
                                           gfv.contiguous() if gfv is not None else None)
        return None, None, lq


class ProbeObjective(torch.autograd.Function):
    """J = H sum_n sum_p p_p(t_n)^2 over an MRAB run (bootstrap + n_steps macro steps) from the
    initial states q0_0, q0_1, as a function of them and of qinf. The gradient comes from the
    library's checkpointed reverse sweep, computed together with J when any input needs it."""

    @staticmethod
    def forward(ctx, system, probe_xy, n_steps, H, n_snapshots, q0_0, q0_1, qinf):
        _set_qinf(system, qinf)
        need = any(ctx.needs_input_grad[5:8])
        r = system.adjoint_probe((q0_0, q0_1), probe_xy, n_steps, H, n_snapshots=n_snapshots, grad=need)
        if need:
            ctx.grads = (r["dq0"][0], r["dq0"][1],
                         torch.as_tensor(r["dqinf"], dtype=qinf.dtype, device=qinf.device))
        ctx.forward_steps = r["forward_steps"]
        return torch.tensor(r["J"], dtype=torch.float64)

    @staticmethod
    def backward(ctx, g):
        g0, g1, gq = ctx.grads
        s = float(g)
        return None, None, None, None, None, g0 * s, g1 * s, gq * s


def probe_objective(system, q0, qinf, probe_xy, n_steps, H, n_snapshots=None):
    """Convenience wrapper of ProbeObjective.apply."""
    return ProbeObjective.apply(system, probe_xy, n_steps, H, n_snapshots, q0[0], q0[1], qinf)


def freestream_state(mach, gamma, alpha=0.0):
    """Far-field conserved state (rho = 1, c = 1) as a differentiable function of the Mach number."""
    mach = torch.as_tensor(mach, dtype=torch.float64)
    ca, sa = torch.cos(torch.as_tensor(alpha, dtype=torch.float64)), torch.sin(torch.as_tensor(alpha, dtype=torch.float64))
    u, v = mach * ca, mach * sa
    E = 1.0 / (gamma * (gamma - 1.0)) + 0.5 * (u * u + v * v)
    return torch.stack([torch.ones_like(mach), u, v, E])
