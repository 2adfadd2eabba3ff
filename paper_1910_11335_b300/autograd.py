"""Differentiable S_N solve: a torch.autograd.Function around dts_solve (forward)
and dts_solve_adjoint (backward).

Inputs are the per-voxel multipliers of sigma_t and sigma_s (float64 tensors,
[V]); the output is the total scalar fluence [G][V] of one source. The
backward pass is the library's discrete adjoint: per-group forward moments
are kept by the forward solve, angular fluxes and fixup sets are recomputed
group by group, and the transposed sweeps run on the GPU. Any loss built from
the fluence with torch operations (for example a detector response) then
differentiates through it.
"""
from __future__ import annotations

import numpy as np
import torch

from . import dts, inputs


class DtsSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, scale_t, scale_s, w: inputs.Workload, source_index: int, tol: float,
                max_iters: int):
        st = scale_t.detach().cpu().numpy().astype(np.float64)
        ss = scale_s.detach().cpu().numpy().astype(np.float64)
        dev = scale_t.device if scale_t.is_cuda else torch.device("cuda", 0)
        p = dts.Problem(nx=w.nx, ny=w.ny, nz=w.nz, dx=w.dx, dy=w.dy, dz=w.dz, x0=w.x0, y0=w.y0,
                        z0=w.z0, n_groups=w.n_groups, sn_order=w.sn_order,
                        legendre_order=w.legendre_order, batch=1, precision=dts.PREC_FP64,
                        tol=tol, max_iters=max_iters, keep_moments=True,
                        device=dev.index or 0, stream=torch.cuda.current_stream(dev).cuda_stream)
        p.set_materials(w.sigma_t, w.sigma_s, w.mat_id.reshape(-1), st, ss)
        p.set_source(0, w.sources[source_index])
        p.solve(allow_not_converged=True)
        out = torch.empty(w.n_groups * w.n_voxels, dtype=torch.float64, device=dev)
        p.fluence(0, dts.TOTAL, out=out)
        ctx.problem = p
        return out.view(w.n_groups, w.n_voxels)

    @staticmethod
    def backward(ctx, grad_out):
        p = ctx.problem
        gt, gs = p.adjoint(0, grad_out.contiguous())
        return gt, gs, None, None, None, None


def solve(scale_t, scale_s, w: inputs.Workload, source_index: int = 0, tol: float = 1e-10,
          max_iters: int = 2000):
    """Total scalar fluence [G][V] of source `source_index` of workload w with
    per-voxel multipliers scale_t, scale_s (float64 tensors of length V)."""
    return DtsSolve.apply(scale_t, scale_s, w, source_index, tol, max_iters)


def detector_response(phi, w: inputs.Workload, bin_size: int = 2):
    """R_p = sum_g E_g sum_{v in pixel p} phi^g(v) over the far y layer of the
    grid (source on the -y side), binned bin_size x bin_size in (x, z)."""
    pix, n_pix = inputs.detector_layout(w, bin_size)
    G = w.n_groups
    e = torch.as_tensor(w.group_energy_kev, dtype=phi.dtype, device=phi.device)
    layer = phi.view(G, w.nz, w.ny, w.nx)[:, :, w.ny - 1, :]          # [G][nz][nx]
    weighted = (e[:, None, None] * layer).sum(0).reshape(-1)          # [nz*nx]
    idx = torch.as_tensor(pix.reshape(-1), device=phi.device)
    return torch.zeros(n_pix, dtype=phi.dtype, device=phi.device).index_add_(0, idx, weighted)
