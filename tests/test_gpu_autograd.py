"""The torch.autograd form (Eq. 3 forward, per-brick recomputing backward).

Workload: a 256^3 Gaussian random field with a k^-5/3 spectrum and 65,536
Gaussians from the analytic allocation.  The gradient is checked against the
FP64 oracle (relative L2 <= 1e-4 on 64 sampled Gaussians) and against central
finite differences with h = 1e-3 of the CUDA forward at 5 sigma truncation
(where crossing the truncation surface moves the field by at most
e^-12.5 of a contribution), and a torch training loop over the Function
matches the library's fused refinement.
"""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2608_14112_b300 import gve, inputs
from paper_2608_14112_b300.autograd import gaussian_field

pytestmark = pytest.mark.gpu


def rel_l2(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.fixture(scope="module")
def grf256():
    V = inputs.grf(256, seed=2)
    prm, _, st, status = O.allocate(V, 65536, seed=2)
    assert status == 0
    ids = np.sort(np.random.default_rng(3).choice(65536, 64, replace=False))
    return V, prm.astype(np.float32), ids


def test_autograd_gradient_matches_oracle(grf256):
    V, p32, ids = grf256
    Vd = torch.from_numpy(V).cuda()
    P = torch.from_numpy(p32).cuda().requires_grad_(True)
    vt = gaussian_field(P, V.shape)
    loss = ((vt - Vd) ** 2).mean()
    loss.backward()
    g = P.grad.cpu().numpy()[ids]
    ref = O.grad_subset(p32.astype(np.float64), V, ids)
    assert rel_l2(g, ref) <= 1e-4
    for sl in (slice(0, 3), slice(3, 6), slice(6, 10), slice(10, 11), slice(11, 12)):
        assert rel_l2(g[:, sl], ref[:, sl]) <= 3e-4, sl


def test_autograd_central_differences(grf256):
    V, p32, ids = grf256
    opts = gve.EvalOptions(trunc_k=5.0)
    rng = np.random.default_rng(7)
    U = torch.from_numpy(rng.standard_normal(V.shape).astype(np.float32)).cuda()
    P = torch.from_numpy(p32).cuda().requires_grad_(True)
    vt = gaussian_field(P, V.shape, opts)
    (vt * U).sum().backward()
    g = P.grad.cpu().numpy()[ids].astype(np.float64)
    h = 1e-3
    Ud = U.double()

    def L(Q):
        return float((gve.gve_evaluate(Q, V.shape, opts).double() * Ud).sum())

    fd = np.zeros_like(g)
    base = torch.from_numpy(p32).cuda()
    for r, i in enumerate(ids):
        for j in range(12):
            Qp = base.clone()
            Qm = base.clone()
            Qp[i, j] += h
            Qm[i, j] -= h
            fd[r, j] = (L(Qp) - L(Qm)) / (2 * h)
    assert rel_l2(g, fd) <= 1e-2
    for sl in (slice(0, 3), slice(3, 6), slice(6, 10), slice(10, 11), slice(11, 12)):
        assert rel_l2(g[:, sl], fd[:, sl]) <= 3e-2, sl


def test_torch_training_loop_matches_fused_refine():
    V = inputs.blobs(64, seed=1)
    prm, _, _, status = O.allocate(V, 4096, seed=0)
    p32 = prm.astype(np.float32)
    Vd = torch.from_numpy(V).cuda()
    P = torch.from_numpy(p32).cuda().requires_grad_(True)
    opt = torch.optim.Adam([P], lr=1e-2, betas=(0.9, 0.999), eps=1e-15)
    losses = []
    for _ in range(10):
        opt.zero_grad()
        loss = ((gaussian_field(P, V.shape) - Vd) ** 2).mean()
        loss.backward()
        opt.step()
        losses.append(loss.item())
    Q = torch.from_numpy(p32).cuda()
    trace = torch.zeros(10, dtype=torch.float64, device="cuda")
    gve.gve_refine(Q, Vd, iters=10, lr=1e-2, eps=1e-15, trace=trace)
    np.testing.assert_allclose(losses, trace.cpu().numpy(), rtol=1e-4)
    assert rel_l2(P.detach().cpu().numpy(), Q.cpu().numpy()) <= 1e-5
