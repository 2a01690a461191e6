"""The 512x512 constant-gradient source-inversion workload (c = 1 + 0.5 z,
w = 2 pi 64): loss ||P u(s) - d||^2 over 256 seeded receivers P, data d
from a point source, autograd backward through the adjoint apply, at full
size in the mixed precision.

The exact gradient is 2 h^2 K^H P^T (P K (h^2 s) - d) (Sec. 3.1 operator;
the loss is quadratic in s).  The oracle computes the receiver rows of the
dense sum and the gradient on 2048 seeded cells from K[P, cells]; 32 seeded
directions are checked by central differences, exact for a quadratic loss at
any step (here a step of the size of s)."""
import numpy as np
import pytest

from paper_2210_02698_gb300 import workloads as W
from tests._common import gpu_op, oracle_op


@pytest.mark.gpu
@pytest.mark.slow
def test_c4_gradient_at_full_size():
    import torch
    from paper_2210_02698_gb300 import binding
    from paper_2210_02698_gb300.autograd import hb_apply
    from oracle import dense
    w = W.WORKLOADS["grad512"]
    g = w.grid
    rng = np.random.default_rng(512)
    P = np.sort(rng.choice(g.Nv, 256, replace=False))
    j0 = int(rng.integers(g.Nv))
    cells = np.sort(rng.choice(g.Nv, 2048, replace=False))
    s0 = W.complex_normal_sources(g.Nv, 1, 5120)[:, 0]
    s_ref = W.point_source(g, j0 % g.N, j0 // g.N)[:, 0]

    # oracle: d = P u(s_ref), residual r = P u(s0) - d, gradient on the sampled cells
    og = oracle_op(w)
    d = og.block(P, [j0])[:, 0] * (g.h ** 2 * s_ref[j0])
    r = dense.apply(og, s0, rows=P, chunk=8192)[:, 0] - d
    g_ref = 2 * g.h ** 2 * (og.block(P, cells).conj().T @ r)

    gp = gpu_op(w, precision=binding.HB_MIXED_BF16X3)
    gp.build()
    Pd = torch.from_numpy(P).cuda()
    d_dev = torch.from_numpy(d).cuda()

    def loss(x):
        return (hb_apply(x, gp)[:, Pd] - d_dev).abs().pow(2).sum()

    s = torch.from_numpy(s0[None, :].copy()).cuda().requires_grad_(True)
    L = loss(s)
    L.backward()
    grad = s.grad.detach()
    got = grad[0, torch.from_numpy(cells).cuda()].cpu().numpy()
    assert np.linalg.norm(got - g_ref) <= 1e-4 * np.linalg.norm(g_ref)

    s_t = s.detach()
    with torch.no_grad():
        for k in range(32):
            dl = torch.from_numpy(W.complex_normal_sources(g.Nv, 1, 6000 + k).T.copy()).cuda()
            t = float(s_t.norm() / dl.norm())
            fd = (loss(s_t + t * dl) - loss(s_t - t * dl)) / (2 * t)
            pred = torch.real(torch.vdot(grad.reshape(-1), dl.reshape(-1)))
            assert abs(float(fd - pred)) <= 1e-4 * float(grad.norm() * dl.norm())
    gp.close()
