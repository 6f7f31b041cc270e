"""Differentiable flow refinement on the GPU (a build extension, not a step of
the paper).

The energy at pyramid level l of two full-resolution planes T0, J0 and a flow
u on level l is

    E(u) = sum_p (J_l(p + u(p)) - T_l(p))^2 + alpha * sum_p |forward differences of u|^2,

with T_l, J_l the level-l REDUCE images of T0, J0 (the LK pyramid of the flow
path) and J_l sampled by the same bilinear clamp-to-edge sampler. The energy
and every gradient come from the library's kernels (``pano_energy_grad`` and
the REDUCE transpose ``pano_stage_pyr_down_adjoint``). ``PyramidEnergy``
stores only T0, J0 and u: the backward pass rebuilds the pyramid levels
instead of keeping them.
"""
from __future__ import annotations

from typing import List, Optional, Tuple

import torch

from . import binding


def _levels(img: torch.Tensor, level: int) -> List[torch.Tensor]:
    """[level 0 (img), level 1, ..., level `level`] with the library REDUCE."""
    out = [img]
    for _ in range(level):
        out.append(binding.stage_pyr_down(out[-1]))
    return out


def _reduce_transpose(g: torch.Tensor, shapes: List[Tuple[int, int]]) -> torch.Tensor:
    """Carry a gradient at the coarsest of `shapes` back to the finest one."""
    for h, w in reversed(shapes[:-1]):
        g = binding.stage_pyr_down_adjoint(g.contiguous(), h, w)
    return g


class PyramidEnergy(torch.autograd.Function):
    """E at pyramid level `level` of T0, J0 for the flow u (float64 scalar)."""

    @staticmethod
    def forward(ctx, T0, J0, u, level: int, alpha: float):
        T = _levels(T0, level)[-1]
        J = _levels(J0, level)[-1]
        E, _, _, _ = binding.energy_grad(T.contiguous(), J.contiguous(), u.contiguous(), alpha,
                                         want_u=False, want_T=False, want_J=False)
        ctx.save_for_backward(T0, J0, u)
        ctx.level, ctx.alpha = level, alpha
        return E

    @staticmethod
    def backward(ctx, gE):
        T0, J0, u = ctx.saved_tensors
        need_T, need_J, need_u = ctx.needs_input_grad[:3]
        Tl = _levels(T0, ctx.level)          # rebuilt, not stored
        Jl = _levels(J0, ctx.level)
        shapes = [tuple(t.shape) for t in Tl]
        _, gu, gt, gj = binding.energy_grad(Tl[-1].contiguous(), Jl[-1].contiguous(), u.contiguous(), ctx.alpha,
                                            want_energy=False, want_u=need_u, want_T=need_T, want_J=need_J)
        s = gE.to(torch.float32)
        dT = _reduce_transpose(gt, shapes) * s if need_T else None
        dJ = _reduce_transpose(gj, shapes) * s if need_J else None
        du = gu * s if need_u else None
        return dT, dJ, du, None, None


def pyramid_energy(T0, J0, u, level: int = 0, alpha: float = 0.05):
    return PyramidEnergy.apply(T0, J0, u, level, alpha)


def refine_flow(T0: torch.Tensor, J0: torch.Tensor, levels: int, steps: int = 30, lr: float = 0.05,
                alpha: float = 0.05, u_init: Optional[torch.Tensor] = None):
    """Coarse-to-fine refinement of the flow from T0 to J0 by Adam steps on
    the energy at each level; the result of a level, upsampled by the
    library's coarse-to-fine kernel, starts the next finer one.

    Returns (flow at level 0, list of (level, first energy, last energy)).
    """
    shapes = [tuple(t.shape) for t in _levels(T0, levels - 1)]
    dev = T0.device
    u = None
    trace = []
    for l in range(levels - 1, -1, -1):
        h, w = shapes[l]
        if u is None:
            u0 = u_init if (u_init is not None and tuple(u_init.shape[:2]) == (h, w)) else \
                torch.zeros((h, w, 2), dtype=torch.float32, device=dev)
        else:
            z = torch.zeros((h, w), dtype=torch.float32, device=dev)
            u0 = binding.stage_lk(z, z, u.contiguous(), upsample=True, iters=0)   # 2 * bilinear upsampling
        u = u0.clone().requires_grad_(True)
        opt = torch.optim.Adam([u], lr=lr)
        first = last = None
        for _ in range(steps):
            opt.zero_grad()
            E = pyramid_energy(T0, J0, u, l, alpha)
            E.backward()
            opt.step()
            e = float(E.detach())
            first = e if first is None else first
            last = e
        u = u.detach()
        trace.append((l, first, last))
    return u, trace
