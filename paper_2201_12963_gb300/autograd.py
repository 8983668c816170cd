"""Differentiable constant-potential energy and electrode charge (torch.autograd.Function).

CPMEnergy(xyz, dpsi, system) -> H per replica, the constant-potential energy
H = U - dpsi q^T v (+ dpsi/L_z sum_j Q_j Z_j for the finite field) at the charges q solved in the
forward pass (Eq. 3, with the field term of Eqs. 10-11 and the potentials of Eq. 5).  Because q
minimises the energy under the neutrality constraints (Eqs. 6-7, 12), dH/dq is
parallel to the constraints and the charge response drops out of every derivative (envelope
theorem):
    dH/dR_j   = -F_j                  (the electrostatic force; backward launches cpm_forces)
    dH/d dpsi = -q^T v (+ sum Q_j Z_j / L_z)

CPMCharge(dpsi, system) -> Q_+ per replica, the total charge of the side +1 electrode, with
dQ_+/d dpsi = e_+^T S v (cpm_capacitance; S of Eqs. 8-9 / 13-15), the differential capacitance of
the cell (Sec. IV.D).

Both functions drive the C ABI through a driver.System whose electrolyte charges and replica
layout stay fixed; only positions and potential differences are inputs.
"""
from __future__ import annotations

import torch

from . import cpm_capacitance, cpm_forces, cpm_step


def _load_inputs(system, xyz, dpsi):
    n = xyz.shape[0]
    system.xyzq[:n, :3].copy_(xyz.detach())
    system.dpsi.copy_(dpsi.detach())


class CPMEnergy(torch.autograd.Function):
    """H (float64 [n_rep]) of the electrolyte positions xyz (float64 [N_l, 3], replica-major as
    in system.offsets) and the potential differences dpsi (float64 [n_rep])."""

    @staticmethod
    def forward(ctx, xyz, dpsi, system):
        _load_inputs(system, xyz, dpsi)
        cpm_step(system.ctx, system.n_rep, system.offsets, system.xyzq, system.dpsi, system.q,
                 energy=system.energy)
        e = system.energy.view(system.n_rep, 4)
        ctx.system = system
        ctx.save_for_backward(system.xyzq.clone(), system.dpsi.clone(), system.q.clone(), e[:, 2].clone())
        return e[:, 1].clone()

    @staticmethod
    def backward(ctx, g_h):
        s = ctx.system
        xyzq, dpsi, q, dh_ddpsi = ctx.saved_tensors
        grad_xyz = grad_dpsi = None
        if ctx.needs_input_grad[0]:
            f = torch.zeros_like(s.f_elyt)
            cpm_forces(s.ctx, s.n_rep, s.offsets, xyzq, dpsi, q, f_elyt=f)
            counts = (s.offsets[1:] - s.offsets[:-1]).long()
            nl = int(counts.sum().item())
            scale = torch.repeat_interleave(g_h.to(f.dtype), counts, output_size=nl)   # chain rule per replica
            grad_xyz = -f[: 3 * nl].view(nl, 3) * scale[:, None]
        if ctx.needs_input_grad[1]:
            grad_dpsi = g_h * dh_ddpsi
        return grad_xyz, grad_dpsi, None


class CPMCharge(torch.autograd.Function):
    """Q_+ (float64 [n_rep]) as a function of dpsi for the electrolyte loaded in `system`.
    Its derivative with respect to dpsi is the constant e_+^T S v."""

    @staticmethod
    def forward(ctx, dpsi, system):
        system.dpsi.copy_(dpsi.detach())
        cpm_step(system.ctx, system.n_rep, system.offsets, system.xyzq, system.dpsi, system.q,
                 energy=system.energy)
        ctx.cap = cpm_capacitance(system.ctx)
        return system.energy.view(system.n_rep, 4)[:, 3].clone()

    @staticmethod
    def backward(ctx, g_q):
        return g_q * ctx.cap, None


def energy(xyz, dpsi, system):
    return CPMEnergy.apply(xyz, dpsi, system)


def electrode_charge(dpsi, system):
    return CPMCharge.apply(dpsi, system)
