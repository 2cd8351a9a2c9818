"""torch.autograd Functions over the fastpod C ABI.

``PODEnergy``  E(pos, c) of the linear POD model (Eq. 57a, 58a).
               Backward: dE/dpos = -F (the adjoint forces of Eq. 24c / 26c),
               dE/dc = G, the global descriptors.
``PODForces``  F(pos, c) = -dE/dpos.  Backward with respect to c only: the
               forces are linear in c, F = -sum_m c_m dG_m/dr, so for a loss
               L(F) the gradient is dL/dc_m = -sum_k dG_m/dr_k . dL/dF_k, one
               forward-mode pass (pod_descriptors_jvp).  Second derivatives
               with respect to positions are not provided.

Positions may be (N, 3) or (3, N) float64 CUDA tensors; gradients come back in
the caller's layout.  All arithmetic runs in the library's kernels.
"""
from __future__ import annotations

import torch


def _layout_N3(pos):
    return pos.dim() == 2 and pos.shape[1] == 3 and not (pos.shape[0] == 3 and pos.shape[1] != 3)


class PODEnergy(torch.autograd.Function):
    @staticmethod
    def forward(ctx, pos, c, pod, box, pbc=(1, 1, 1)):
        out = pod.energy_forces(pos.detach(), box, c.detach(), pbc, atom_energies=False, virial=False)
        G = pod.global_descriptors(pos.detach(), box, pbc)[0] if ctx.needs_input_grad[1] else None
        ctx.n3 = _layout_N3(pos)
        ctx.save_for_backward(out["F"], G if G is not None else torch.empty(0, device=pos.device))
        return out["E"][0].clone()

    @staticmethod
    def backward(ctx, gE):
        F, G = ctx.saved_tensors  # F is (N, 3)
        gpos = None
        if ctx.needs_input_grad[0]:
            gpos = -F * gE
            if not ctx.n3:
                gpos = gpos.t().contiguous()
        gc = G * gE if ctx.needs_input_grad[1] else None
        return gpos, gc, None, None, None


class PODForces(torch.autograd.Function):
    @staticmethod
    def forward(ctx, pos, c, pod, box, pbc=(1, 1, 1)):
        out = pod.energy_forces(pos.detach(), box, c.detach(), pbc, atom_energies=False, virial=False)
        ctx.pod, ctx.box, ctx.pbc = pod, box, pbc
        ctx.save_for_backward(pos.detach())
        F = out["F"].contiguous()  # (N, 3)
        return F if _layout_N3(pos) else F.t().contiguous()

    @staticmethod
    def backward(ctx, gF):
        if ctx.needs_input_grad[0]:
            raise NotImplementedError("second derivatives of the POD energy with respect to positions are not provided")
        (pos,) = ctx.saved_tensors
        gc = None
        if ctx.needs_input_grad[1]:
            v = gF.to(torch.float64)
            gc = -ctx.pod.descriptors_jvp(pos, ctx.box, v, ctx.pbc)[0]
        return None, gc, None, None, None


def pod_energy(pos, c, pod, box, pbc=(1, 1, 1)):
    return PODEnergy.apply(pos, c, pod, box, pbc)


def pod_forces(pos, c, pod, box, pbc=(1, 1, 1)):
    return PODForces.apply(pos, c, pod, box, pbc)
