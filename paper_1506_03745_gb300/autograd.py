"""torch.autograd wrapper of the solve + energy (forward) and the adjoint
gradients (backward) of libpgb.

    fe = FreeEnergy(ctx, bodies)            # ctx from pgb_create + pgb_mesh_load
    F = fe(q, bc, t)                        # total free energy (kcal/mol)
    F.backward()                            # q.grad, bc.grad, t.grad via pgb_grad

q: all charges of the dielectric bodies concatenated in load order (e);
bc: one value per body (sigma0 in C/m^2 or phi0 in V for surfaces, ignored
for molecules); t: (n_bodies, 3) translations of the bodies' rigid poses
(rotations as last set with pgb_set_pose, identity by default).  Every step
runs in the CUDA library; this module only marshals arguments.
"""
import numpy as np
import torch

from . import _lib as L


class _FreeEnergy(torch.autograd.Function):
    @staticmethod
    def forward(fctx, helper, q, bc, t):
        F, x = helper._forward(q.detach().cpu().double().numpy(), bc.detach().cpu().double().numpy(),
                               t.detach().cpu().double().numpy())
        fctx.helper = helper
        fctx.x = x
        fctx.shapes = (q.shape, bc.shape, t.shape)
        return torch.tensor(F, dtype=torch.float64)

    @staticmethod
    def backward(fctx, gF):
        dq, dbc, dt = fctx.helper._backward(fctx.x)
        g = float(gF)
        return (None, torch.tensor(dq * g).reshape(fctx.shapes[0]), torch.tensor(dbc * g).reshape(fctx.shapes[1]),
                torch.tensor(dt * g).reshape(fctx.shapes[2]))


class FreeEnergy:
    """Differentiable total free energy of a loaded context.

    kinds: list of body kinds (L.PGB_DIELECTRIC, ...), n_charges: list of the
    charge counts per body, R: optional list of per-body rotations.
    frozen_lists: after the first forward, later forwards keep its
    interaction lists (pgb_tree_refresh instead of pgb_tree_build), so that
    finite differences in t see no change of the near/far split."""

    def __init__(self, ctx, kinds, n_charges, R=None, mode=L.PGB_FP32_REFINE, tol=1e-6,
                 grad_precision=L.PGB_FP32, grad_tol=1e-6, max_iter=2000, restart=100, frozen_lists=False):
        self.ctx = ctx
        self.kinds = list(kinds)
        self.nq = list(n_charges)
        self.R = [np.eye(3) for _ in kinds] if R is None else [np.asarray(r, dtype=float) for r in R]
        self.mode, self.tol = mode, tol
        self.gp, self.gtol = grad_precision, grad_tol
        self.max_iter, self.restart = max_iter, restart
        self.frozen, self._built = frozen_lists, False

    def __call__(self, q, bc, t):
        return _FreeEnergy.apply(self, q, bc, t)

    def _forward(self, q, bc, t):
        off = 0
        for b, kind in enumerate(self.kinds):
            if kind == L.PGB_DIELECTRIC and self.nq[b]:
                L.pgb_set_charges(self.ctx, b, q[off:off + self.nq[b]])
                off += self.nq[b]
            elif kind != L.PGB_DIELECTRIC:
                L.pgb_set_bc(self.ctx, b, bc[b])
            L.pgb_set_pose(self.ctx, b, self.R[b], t[b])
        if self.frozen and self._built:
            L.pgb_tree_refresh(self.ctx)
        else:
            L.pgb_tree_build(self.ctx)
            self._built = True
        x = torch.empty(L.pgb_num_unknowns(self.ctx), dtype=torch.float64, device="cuda")
        code, st = L.pgb_solve(self.ctx, self.mode, self.tol, self.max_iter, self.restart, x)
        if code != L.PGB_OK:
            raise L.PgbError(code, f"solve did not converge: {st}")
        return L.pgb_energy(self.ctx, x)["total"], x

    def _backward(self, x):
        code, dq, dbc, dt, st = L.pgb_grad(self.ctx, x, sum(self.nq), len(self.kinds), self.gp, self.gtol,
                                           self.max_iter, self.restart)
        if code != L.PGB_OK:
            raise L.PgbError(code, f"adjoint solve did not converge: {st}")
        return dq, dbc, dt
