"""The full sampled objective (Sec. III-F: value term plus the density,
smoothness, anchor, anisotropy and scale-cap regularisers) against the
oracle.  Partners are bit-exact (the same Philox words and float32
arithmetic); the objective and its terms agree to 1e-5 relative and the
gradient to 1e-4 relative L2 (float32 sums and atomics on the device, FP64
in the oracle, as for the value term alone); a regularised refinement
follows the oracle's losses to 2e-3 and its final PSNR to 0.05 dB."""
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


def _prims(rng, n, dims):
    p = np.zeros((n, 12), np.float64)
    p[:, 0:3] = rng.uniform(0, 1, (n, 3)) * (np.array(dims) - 1)
    p[:, 3:6] = np.log(rng.lognormal(np.log(1.4), 0.7, (n, 3)))
    p[:, 6:10] = rng.normal(size=(n, 4))
    p[:, 10] = rng.uniform(0.05, 1.0, n)
    p[:, 11] = rng.uniform(-2.5, 1.5, n)
    return p.astype(np.float32)


@pytest.mark.parametrize("S,it,radius", [(3072, 0, 1.0), (1000, 9, 0.5), (1, 2, 2.0)])
def test_partners_are_bit_exact(S, it, radius):
    V = inputs.grf((37, 29, 45), seed=9)
    pts, vals, _ = O.draw_samples(V, S, seed=11, it=it)
    ref = O.draw_partners(pts, V.shape, seed=11, it=it, radius=radius)
    P4 = dev(np.concatenate([pts, vals[:, None]], 1).astype(np.float32))
    got = gve.gve_draw_partners(P4, V.shape, seed=11, it=it, radius=radius).cpu().numpy()
    np.testing.assert_array_equal(got[:, :3], ref)
    np.testing.assert_array_equal(got[:, 3], -1.0)


REGS = [
    dict(rho=0.3, sm=0.5, anc=0.2, aniso=0.1, cap=0.4, r_max=2.0, s_lo=0.8, s_hi=2.5),
    dict(rho=1e-3, sm=0.0, anc=1e-3, aniso=1e-3, cap=1e-3, r_max=3.0, s_lo=0.3, s_hi=2.0),
    dict(rho=0.0, sm=2.0, anc=0.0, aniso=0.0, cap=0.0, r_max=3.0, s_lo=0.3, s_hi=100.0),
]


@pytest.mark.parametrize("reg", REGS)
@pytest.mark.parametrize("k", [3.0, 5.0])
def test_objective_and_gradient_match_oracle(reg, k):
    V = inputs.grf((40, 36, 28), seed=21)
    dims = (V.shape[2], V.shape[1], V.shape[0])
    rng = np.random.default_rng(int(k * 10) + len(str(reg)))
    p = _prims(rng, 500, dims)
    S = 2000
    pts, vals, _ = O.draw_samples(V, S, seed=5, it=1)
    smooth = reg["sm"] > 0
    allp = np.concatenate([pts, O.draw_partners(pts, V.shape, seed=5, it=1, radius=1.0)]) if smooth else pts
    L, g, terms = O.sample_objective(p.astype(np.float64), allp, vals, field=V, reg=reg, smooth=smooth, k=k)
    tgt = np.concatenate([vals, -np.ones(S, np.float32)]) if smooth else vals
    P4 = dev(np.concatenate([allp, tgt[:, None]], 1).astype(np.float32))
    ro = gve.RegOptions(lambda_rho=reg["rho"], lambda_sm=reg["sm"], lambda_sm_end=0.0, anneal_iters=0,
                        lambda_anc=reg["anc"], lambda_aniso=reg["aniso"], lambda_cap=reg["cap"],
                        aniso_max=reg["r_max"], s_lo=reg["s_lo"], s_hi=reg["s_hi"])
    loss, gg, _, tt = gve.gve_sample_loss_grad(dev(p), V.shape, P4, gve.EvalOptions(trunc_k=k), reg=ro, field=dev(V),
                                               want_terms=True)
    assert abs(loss.item() - L) <= 1e-5 * abs(L)
    np.testing.assert_allclose(tt.cpu().numpy(), terms, rtol=1e-5, atol=1e-12)
    assert rel_l2(gg.cpu().numpy(), g) <= 1e-4


def test_regularised_refinement_matches_oracle():
    V = inputs.blobs(48, seed=2)
    prm, _, _, status = O.allocate(V, 2000, seed=1)
    assert status == 0
    p32 = prm.astype(np.float32)
    iters, S = 20, 2048
    reg = dict(rho=1e-2, sm0=5e-2, sm1=1e-3, anneal=10, anc=1e-2, aniso=1e-2, cap=1e-2, r_max=3.0, s_lo=0.3,
               s_hi=3.0, radius=1.0)
    ref, losses = O.refine_sampled_reg(p32.astype(np.float64), V, iters, reg, S=S, seed=7)
    P = dev(p32)
    trace = torch.zeros(iters, dtype=torch.float64, device="cuda")
    ro = gve.RegOptions(lambda_rho=1e-2, lambda_sm=5e-2, lambda_sm_end=1e-3, anneal_iters=10, lambda_anc=1e-2,
                        lambda_aniso=1e-2, lambda_cap=1e-2, partner_radius=1.0, aniso_max=3.0, s_lo=0.3, s_hi=3.0)
    st = gve.gve_refine_sampled(P, dev(V), iters, S=S, seed=7, trace=trace, reg=ro)
    np.testing.assert_allclose(trace.cpu().numpy(), losses, rtol=2e-3)
    M = V.size
    psnr_ref = O.psnr_from_sse(O.loss_grad(ref.astype(np.float32).astype(np.float64), V, want_grad=False)[2], M)
    psnr_gpu = O.psnr_from_sse(O.loss_grad(P.cpu().numpy().astype(np.float64), V, want_grad=False)[2], M)
    assert abs(psnr_gpu - psnr_ref) <= 0.05
    assert st["iters_done"] == iters and st["loss_first"] > st["loss_last"]


def test_objective_invalid_arguments():
    V = dev(inputs.blobs(16, seed=1))
    P = torch.zeros((8, 12), device="cuda")
    P[:, 6] = 1.0
    with pytest.raises(gve.GveError):                       # partners double the points
        gve.gve_refine_sampled(P, V, 1, S=5000, reg=gve.RegOptions())
    with pytest.raises(gve.GveError):
        gve.gve_refine_sampled(P, V, 1, S=64, reg=gve.RegOptions(lambda_rho=-1.0))
    with pytest.raises(gve.GveError):
        gve.gve_refine_sampled(P, V, 1, S=64, reg=gve.RegOptions(s_lo=5.0, s_hi=2.0))
    pts = torch.zeros((8, 4), device="cuda")
    with pytest.raises(gve.GveError):                       # the anchor needs the field
        gve.gve_sample_loss_grad(P, V.shape, pts, reg=gve.RegOptions(lambda_sm=0.0, lambda_anc=1.0))
