"""Stratified-sample refinement (Sec. III-F, Table III) against the FP64
oracle: the draw is bit-exact (points, targets and voxels: the same Philox
words, integer class indexing and FP64 trilinear targets on both sides);
Eq. 3 at the points, the sampled loss and its gradient within the voxel
path's tolerances (relative L2 1e-5 on values, 1e-4 on gradients); a short
refinement within the dense refinement's bars (per-iteration losses 2e-3
relative, final full-grid PSNR 0.05 dB)."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2608_14112_b300 import gve, inputs

pytestmark = pytest.mark.gpu


def rel_l2(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _prims(rng, n, dims, lo=0.8, hi=2.5):
    p = np.zeros((n, 12), np.float64)
    p[:, 0:3] = rng.uniform(-1.0, 1.0, (n, 3)) + rng.uniform(0, 1, (n, 3)) * (np.array(dims) - 1)
    p[:, 3:6] = np.log(rng.uniform(lo, hi, (n, 3)))
    p[:, 6:10] = rng.normal(size=(n, 4))
    p[:, 10] = rng.uniform(0.05, 1.0, n)
    p[:, 11] = rng.uniform(-2.5, 1.5, n)
    return p.astype(np.float32)


FIELDS = {
    "blobs": lambda: inputs.blobs(40, seed=3)[:, :36, :28].copy(),
    "grf": lambda: inputs.grf((37, 29, 45), seed=9),
    "no_high": lambda: (0.3 * inputs.grf((24, 24, 24), seed=4)).astype(np.float32),
}


@pytest.mark.parametrize("name", list(FIELDS))
@pytest.mark.parametrize("S,it", [(3072, 0), (3072, 17), (1000, 3), (1, 2)])
def test_draw_is_bit_exact(name, S, it):
    V = np.ascontiguousarray(FIELDS[name](), np.float32)
    pts, vals, vox = O.draw_samples(V, S, seed=123, it=it)
    g, gv = gve.gve_draw_samples(dev(V), S, seed=123, it=it, want_voxels=True)
    g = g.cpu().numpy()
    np.testing.assert_array_equal(gv.cpu().numpy(), vox)
    np.testing.assert_array_equal(g[:, :3], pts)
    np.testing.assert_array_equal(g[:, 3], vals)


@pytest.mark.parametrize("S", [3072, 2500, 1])
@pytest.mark.parametrize("k", [3.0, 5.0])
def test_sample_loss_grad_matches_oracle(S, k):
    V = inputs.grf((40, 36, 28), seed=21)
    shape = V.shape
    dims = (shape[2], shape[1], shape[0])
    rng = np.random.default_rng(S + int(k))
    p = _prims(rng, 400, dims)
    pts, vals, _ = O.draw_samples(V, S, seed=5, it=1)
    L, g, vt = O.sample_loss_grad(p.astype(np.float64), pts, vals, k=k)
    P4 = dev(np.concatenate([pts, vals[:, None]], 1).astype(np.float32))
    loss, gg, gvt = gve.gve_sample_loss_grad(dev(p), shape, P4, gve.EvalOptions(trunc_k=k))
    assert abs(loss.item() - L) <= 1e-5 * max(L, 1e-30)
    assert rel_l2(gvt.cpu().numpy(), vt) <= 1e-5
    if S > 1:
        assert rel_l2(gg.cpu().numpy(), g) <= 1e-4


def test_refine_sampled_matches_oracle():
    V = inputs.blobs(48, seed=2)
    prm, _, _, status = O.allocate(V, 2000, seed=1)
    assert status == 0
    p32 = prm.astype(np.float32)
    iters, S = 20, 3072
    ref, losses = O.refine_sampled(p32.astype(np.float64), V, iters, S=S, seed=7)
    P = dev(p32)
    trace = torch.zeros(iters, dtype=torch.float64, device="cuda")
    st = gve.gve_refine_sampled(P, dev(V), iters, S=S, seed=7, trace=trace)
    np.testing.assert_allclose(trace.cpu().numpy(), losses, rtol=2e-3)
    M = V.size
    psnr_ref = O.psnr_from_sse(O.loss_grad(ref.astype(np.float32).astype(np.float64), V, want_grad=False)[2], M)
    psnr_gpu = O.psnr_from_sse(O.loss_grad(P.cpu().numpy().astype(np.float64), V, want_grad=False)[2], M)
    assert abs(psnr_gpu - psnr_ref) <= 0.05
    # the call's own full-grid PSNR is that of its final records
    assert abs(st["psnr_final"] - psnr_gpu) <= 1e-3
    assert st["iters_done"] == iters and st["loss_first"] > st["loss_last"]


def test_sampled_invalid_arguments():
    V = dev(inputs.blobs(16, seed=1))
    P = torch.zeros((8, 12), device="cuda")
    for S in (0, 8193):
        with pytest.raises(gve.GveError):
            gve.gve_refine_sampled(P, V, 1, S=S)
        with pytest.raises(gve.GveError):
            gve.gve_draw_samples(V, S, seed=1, it=0)
    with pytest.raises(gve.GveError):
        gve.gve_refine_sampled(P, V, 1, S=64, opts=gve.EvalOptions(normalized=False))
