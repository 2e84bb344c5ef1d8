"""torch.autograd wrappers of the winding-number kernels (differentiable voxelization, §1, §2.4).

``winding_number(verts, module)`` returns w(q) for the module's grid or query list and
back-propagates through ``dv_winding_backward``; with ``kind="dipole"`` it uses the Eq. (4)
dipole surrogate (``dv_dipole_winding`` / ``dv_dipole_backward``), which the paper uses for
morphing because the exact winding number of a closed mesh is almost binary and its gradient
vanishes away from the surface. All arithmetic runs in the CUDA library; this file only wires
tensors to it.
"""
from __future__ import annotations

import torch

from . import dv


class _WindingFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, verts, mesh, grid, queries, precision, kind, adjoint):
        v = verts.detach().contiguous()
        dv.dv_mesh_update_verts(mesh, v)
        if kind == "exact":
            w = dv.dv_winding(mesh, queries=queries, grid=grid, precision=precision)
        elif kind == "dipole":
            w = dv.dv_dipole_winding(mesh, queries=queries, grid=grid)
        else:
            raise ValueError(f"unknown kind {kind!r}")
        ctx.mesh, ctx.grid, ctx.queries, ctx.kind, ctx.adjoint = mesh, grid, queries, kind, adjoint
        ctx.save_for_backward(v)
        return w

    @staticmethod
    def backward(ctx, grad_w):
        (v,) = ctx.saved_tensors
        # re-pack from the vertices of this forward (another forward may have moved the mesh since)
        dv.dv_mesh_update_verts(ctx.mesh, v)
        g = grad_w.detach().to(torch.float32).contiguous()
        if ctx.kind == "dipole":
            fn = dv.dv_dipole_backward
        else:
            fn = dv.dv_winding_backward_boundary if ctx.adjoint == "boundary" else dv.dv_winding_backward
        dV = fn(ctx.mesh, g, queries=ctx.queries, grid=ctx.grid)
        return dV, None, None, None, None, None, None


class WindingNumber(torch.nn.Module):
    """Differentiable w(q) of a mesh with fixed faces over a grid or a fixed query list.

    verts [nv,3] float32 CUDA tensor -> w [nq] float32. ``kind`` is "exact" (Eq. (5)/(7), with
    ``precision`` "fp32" | "kahan" | "mixed") or "dipole" (Eq. (4)). For "exact", ``adjoint``
    selects the face-by-face derivative ("faces") or the same derivative from the mesh's boundary
    edges ("boundary", dv_winding_backward_boundary)."""

    def __init__(self, verts, faces, grid: dv.Grid | None = None, queries=None, precision: str = "mixed",
                 kind: str = "exact", adjoint: str = "faces"):
        super().__init__()
        self.mesh = dv.dv_mesh_create(verts.detach().contiguous(), faces.contiguous())
        if grid is not None:
            dv.dv_mesh_reserve(self.mesh, grid)
        self.grid = grid
        self.queries = queries
        self.precision = precision
        self.kind = kind
        if adjoint not in ("faces", "boundary"):
            raise ValueError(f"unknown adjoint {adjoint!r}")
        self.adjoint = adjoint

    def forward(self, verts):
        return _WindingFn.apply(verts, self.mesh, self.grid, self.queries, self.precision, self.kind, self.adjoint)


def winding_number(verts, module: WindingNumber):
    return module(verts)
