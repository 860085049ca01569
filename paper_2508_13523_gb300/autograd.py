"""torch.autograd.Function wrappers of the hand-written adjoint kernels.

``lj_forces(x, eps, sigma, md)`` -- forces of Eq. 1 (arXiv 2508.13523,
Sec. 4) at positions x with per-type-pair tables eps, sigma; backward is
``md_force_vjp``.

``lj_trajectory_forces(x0, v0, eps, sigma, md, nsteps, every)`` -- forces at
the end of nsteps velocity-Verlet steps from (x0, v0); backward is
``md_traj_vjp`` (checkpoints every ``every`` steps, recomputed segment by
segment).

Both run entirely in libmd.so; these classes only move tensors across the C
ABI.  ``md`` is an ``LJMD`` context whose state they overwrite.  eps and
sigma are symmetric (nt, nt) tables used as (T + T^T)/2: the gradient puts
half of an unordered pair's derivative in each off-diagonal entry, so a table
built symmetrically from independent pair parameters receives the right
gradient through autograd.  The cutoffs are constants.
"""
from __future__ import annotations

import numpy as np
import torch


def _table_grad(g_unordered: np.ndarray, like: torch.Tensor) -> torch.Tensor:
    g = np.array(g_unordered, dtype=np.float64)
    off = ~np.eye(g.shape[0], dtype=bool)
    g[off] *= 0.5
    return torch.as_tensor(g, dtype=like.dtype, device=like.device)


class LJForces(torch.autograd.Function):
    @staticmethod
    def forward(fctx, x, eps, sigma, md):
        md.set_lj(eps, sigma)
        md.set_state(x.detach(), torch.zeros_like(x))
        _, _, f = md.get_state()
        fctx.md = md
        fctx.save_for_backward(x, eps, sigma)
        return f

    @staticmethod
    def backward(fctx, gF):
        x, eps, sigma = fctx.saved_tensors
        md = fctx.md
        md.set_lj(eps, sigma)
        md.set_state(x.detach(), torch.zeros_like(x))
        xbar, g = md.force_vjp(gF.contiguous())
        return xbar, _table_grad(g[0], eps), _table_grad(g[1], sigma), None


class LJTrajectoryForces(torch.autograd.Function):
    @staticmethod
    def forward(fctx, x0, v0, eps, sigma, md, nsteps, every):
        md.set_lj(eps, sigma)
        ckx, ckv, fK = md.traj_forward(x0.detach(), v0.detach(), nsteps, every)
        fctx.md = md
        fctx.nsteps, fctx.every = int(nsteps), int(every)
        fctx.save_for_backward(ckx, ckv, eps, sigma)
        return fK

    @staticmethod
    def backward(fctx, gF):
        ckx, ckv, eps, sigma = fctx.saved_tensors
        md = fctx.md
        md.set_lj(eps, sigma)
        x0b, v0b, g = md.traj_vjp(fctx.nsteps, fctx.every, ckx, ckv, gF.contiguous())
        return (x0b, v0b, _table_grad(g[0], eps), _table_grad(g[1], sigma), None, None, None)


def lj_forces(x, eps, sigma, md):
    return LJForces.apply(x, eps, sigma, md)


def lj_trajectory_forces(x0, v0, eps, sigma, md, nsteps, every):
    return LJTrajectoryForces.apply(x0, v0, eps, sigma, md, nsteps, every)
