"""torch.autograd wrapper (paper_1506_03745_gb300.autograd.FreeEnergy):
forward = solve + energy, backward = adjoint gradients, checked against
finite differences of the forward."""
import numpy as np
import pytest

import synth
from problems import gpu_context

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no GPU", allow_module_level=True)

import paper_1506_03745_gb300 as pgb  # noqa: E402
from paper_1506_03745_gb300.autograd import FreeEnergy  # noqa: E402


def _setup():
    v, f = synth.star_surface(9, 5, 4.0)
    rng = np.random.default_rng(3)
    q = rng.uniform(-1, 1, 5)
    mol = dict(kind="dielectric", verts=v, tris=f, eps_in=4.0, qxyz=rng.uniform(-1.2, 1.2, (5, 3)), q=q, bc=0.0)
    v2, f2 = synth.icosphere(2, 3.0)
    srf = dict(kind="sigma", verts=v2, tris=f2, eps_in=1.0, qxyz=np.zeros((0, 3)), q=np.zeros(0), bc=-0.05)
    ctx = gpu_context([mol, srf], theta=0.5, P=6, leaf_size=16)
    fe = FreeEnergy(ctx, [pgb.PGB_DIELECTRIC, pgb.PGB_SET_CHARGE], [5, 0], mode=pgb.PGB_FP64, tol=1e-11,
                    grad_precision=pgb.PGB_FP64, grad_tol=1e-11, frozen_lists=True)
    return ctx, fe, q


def test_forward_backward_against_finite_differences():
    ctx, fe, q0 = _setup()
    try:
        q = torch.tensor(q0, requires_grad=True)
        bc = torch.tensor([0.0, -0.05], dtype=torch.float64, requires_grad=True)
        t = torch.tensor([[0.0, 0.0, 0.0], [11.0, 0.5, 0.0]], dtype=torch.float64, requires_grad=True)
        F = fe(q, bc, t)
        F.backward()
        # finite differences of the forward itself
        def f(qq, bb, tt):
            return float(fe(torch.tensor(qq), torch.tensor(bb), torch.tensor(tt)))
        qn, bn, tn = q0.copy(), bc.detach().numpy().copy(), t.detach().numpy().copy()
        h = 1e-4
        for k in (0, 4):
            a, b = qn.copy(), qn.copy()
            a[k] += h
            b[k] -= h
            assert q.grad[k].item() == pytest.approx((f(a, bn, tn) - f(b, bn, tn)) / (2 * h), rel=1e-5)
        a, b = bn.copy(), bn.copy()
        a[1] += 1e-4
        b[1] -= 1e-4
        assert bc.grad[1].item() == pytest.approx((f(qn, a, tn) - f(qn, b, tn)) / 2e-4, rel=1e-5)
        assert bc.grad[0].item() == 0.0
        # translations: central differences with h = 1e-3 A on the lists of the
        # base pose (reading G20), within 1e-4 of the gradient's norm
        fd = np.zeros(3)
        for ax in range(3):
            a, b = tn.copy(), tn.copy()
            a[1, ax] += 1e-3
            b[1, ax] -= 1e-3
            fd[ax] = (f(qn, bn, a) - f(qn, bn, b)) / 2e-3
        assert np.abs(t.grad[1].numpy() - fd).max() <= 1e-4 * np.linalg.norm(fd)
        np.testing.assert_allclose(t.grad[0].numpy(), -t.grad[1].numpy(), rtol=1e-5, atol=1e-9)
    finally:
        pgb.pgb_destroy(ctx)
