"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Bars: bit-exact for the brick binning (counts, sorted keys, Gaussian ids,
ranges) and the kept-pair count; relative L2 <= 1e-5 on fields; <= 1e-4 on
gradients; <= 0.05 dB on PSNR after a fixed schedule.  Cases span several
bricks with ragged tails, Gaussian lists longer than one shared-memory chunk,
empty and degenerate inputs.
"""
import math
import os

import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2608_14112_b300 import gve, inputs

pytestmark = pytest.mark.gpu

FIELD_TOL = 1e-5
GRAD_TOL = 1e-4
PSNR_TOL = 0.05


def rel_l2(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))


def rand_prims(rng, n, dims, s_lo=0.8, s_hi=2.5):
    p = np.zeros((n, 12), np.float64)
    p[:, 0:3] = rng.uniform(-1.0, 1.0, (n, 3)) + rng.uniform(0, 1, (n, 3)) * (np.array(dims) - 1)
    p[:, 3:6] = np.log(rng.uniform(s_lo, s_hi, (n, 3)))
    p[:, 6:10] = rng.normal(size=(n, 4))
    p[:, 10] = rng.uniform(0.05, 1.0, n)
    p[:, 11] = rng.uniform(-2.5, 1.5, n)
    return p.astype(np.float32)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


CASES = {
    # name: (dims (nx,ny,nz), n, s_lo, s_hi, seed)
    "ragged": ((37, 29, 21), 300, 0.8, 3.0, 1),
    "long_lists": ((16, 16, 16), 420, 4.0, 6.0, 2),      # > 64 Gaussians per brick: several staged chunks
    "thin": ((45, 33, 1), 120, 0.6, 2.5, 3),
    "small_gauss": ((24, 24, 24), 500, 0.2, 0.6, 4),
}


@pytest.mark.parametrize("case", list(CASES))
def test_binning_bit_exact(case):
    dims, n, lo, hi, seed = CASES[case]
    p = rand_prims(np.random.default_rng(seed), n, dims, lo, hi)
    counts, sk, sg, start, end = O.bin_sorted(p, dims, 3.0, 8)
    gc, gk, gg, gs, ge = gve.gve_bin(dev(p), (dims[2], dims[1], dims[0]))
    np.testing.assert_array_equal(gc.numpy(), counts.astype(np.int64))
    np.testing.assert_array_equal(gk.numpy(), sk.astype(np.int64))
    np.testing.assert_array_equal(gg.numpy(), sg.astype(np.int64))
    np.testing.assert_array_equal(gs.numpy(), start.astype(np.int64))
    np.testing.assert_array_equal(ge.numpy(), end.astype(np.int64))


MASK_CASES = dict(CASES, aniso=((40, 36, 30), 200, 0.4, 9.0, 7))


@pytest.mark.parametrize("brick", [4, 8, 16])
@pytest.mark.parametrize("case", list(MASK_CASES))
def test_subbrick_masks_cover_kept_voxels(case, brick):
    """The evaluator's sub-brick masks contain every sub-brick in which the
    oracle's float32 keep test keeps a voxel (they may hold more)."""
    dims, n, lo, hi, seed = MASK_CASES[case]
    shape = (dims[2], dims[1], dims[0])
    p = rand_prims(np.random.default_rng(seed + 40), n, dims, lo, hi)
    _, gk, gg, _, _, gm = gve.gve_bin(dev(p), shape, gve.EvalOptions(brick=brick), with_masks=True)
    ref = O.kept_submasks(p, dims, gk.numpy().astype(np.uint32), gg.numpy().astype(np.uint32), 3.0, brick)
    got = gm.numpy()
    assert got.shape == ref.shape and ref.any()
    missing = ref & ~got
    assert not missing.any(), np.nonzero(missing)[0][:10]


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("normalized", [True, False])
def test_evaluate_parity(case, normalized):
    dims, n, lo, hi, seed = CASES[case]
    p = rand_prims(np.random.default_rng(seed), n, dims, lo, hi)
    _, _, vt = O.eval_region(p, dims, k=3.0, normalized=normalized)
    out = gve.gve_evaluate(dev(p), (dims[2], dims[1], dims[0]), gve.EvalOptions(normalized=normalized))
    assert rel_l2(out.cpu().numpy(), vt) <= FIELD_TOL


@pytest.mark.parametrize("case", list(CASES))
def test_kept_pairs_bit_exact(case):
    """The float32 keep decision agrees pair for pair in count, and the
    candidate count is what the brick lists imply."""
    dims, n, lo, hi, seed = CASES[case]
    p = rand_prims(np.random.default_rng(seed), n, dims, lo, hi)
    kept, cand = gve.gve_count_pairs(dev(p), (dims[2], dims[1], dims[0]))
    assert kept == O.count_kept(p, dims, 3.0)
    assert cand >= kept


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("mask", [-1.0, 0.3])
def test_loss_grad_parity(case, mask):
    dims, n, lo, hi, seed = CASES[case]
    rng = np.random.default_rng(seed + 10)
    p = rand_prims(rng, n, dims, lo, hi)
    field = rng.uniform(0, 1, (dims[2], dims[1], dims[0])).astype(np.float32)
    L, g, sse = O.loss_grad(p.astype(np.float64), field, mask_thresh=mask)
    gg, gsse = gve.gve_loss_grad(dev(p), dev(field), mask_thresh=mask)
    gg = gg.cpu().numpy()
    M = field.size
    assert abs(gsse[1].item() - sse) <= 1e-5 * sse
    assert abs(gsse[0].item() / M - L) <= 1e-5 * L
    assert rel_l2(gg, g) <= GRAD_TOL
    for sl in (slice(0, 3), slice(3, 6), slice(6, 10), slice(10, 11), slice(11, 12)):
        assert rel_l2(gg[:, sl], g[:, sl]) <= 3 * GRAD_TOL, sl


def test_backward_upstream_parity():
    dims, n, lo, hi, seed = CASES["ragged"]
    rng = np.random.default_rng(77)
    p = rand_prims(rng, n, dims, lo, hi)
    U = rng.normal(size=(dims[2], dims[1], dims[0])).astype(np.float32)
    g = O.backward(p.astype(np.float64), U.astype(np.float64))
    gg = gve.gve_backward(dev(p), dev(U)).cpu().numpy()
    assert rel_l2(gg, g) <= GRAD_TOL


def test_target_rows_at_any_alignment():
    """The target (loss) and upstream (backward) rows reach the evaluator by
    16-byte copies when a row starts 16-byte aligned and by 4-byte copies
    otherwise: a field starting 4 bytes past an aligned address gives the
    same SSE (bit for bit) and the same gradients as an aligned copy."""
    dims, n, lo, hi, seed = CASES["long_lists"]
    rng = np.random.default_rng(seed + 30)
    p = dev(rand_prims(rng, n, dims, lo, hi))
    shape = (dims[2], dims[1], dims[0])
    buf = torch.empty(int(np.prod(shape)) + 4, dtype=torch.float32, device="cuda")
    for values in (rng.uniform(0, 1, shape), rng.normal(size=shape)):
        a = dev(values.astype(np.float32))
        b = buf[1:1 + a.numel()].view(shape)
        b.copy_(a)
        assert a.data_ptr() % 16 == 0 and b.data_ptr() % 16 == 4
        ga, sa = gve.gve_loss_grad(p, a)
        gb, sb = gve.gve_loss_grad(p, b)
        assert torch.equal(sa, sb)
        assert rel_l2(gb.cpu().numpy(), ga.cpu().numpy()) <= 1e-6
        ua, ub = gve.gve_backward(p, a), gve.gve_backward(p, b)
        assert rel_l2(ub.cpu().numpy(), ua.cpu().numpy()) <= 1e-6


def test_empty_and_degenerate_inputs():
    dims = (20, 12, 9)
    shape = (9, 12, 20)
    # no Gaussians: field is zero, gradient empty
    out = gve.gve_evaluate(torch.zeros((0, 12), device="cuda"), shape)
    assert float(out.abs().max()) == 0.0
    # Gaussians outside the grid, non-finite records, zero quaternion: contribute nothing
    p = rand_prims(np.random.default_rng(5), 6, dims)
    p[0, 0:3] = [-50.0, 5.0, 5.0]
    p[1, 2] = np.nan
    p[2, 6:10] = 0.0
    p[3, 3] = np.inf
    _, _, vt = O.eval_region(p[4:].astype(np.float64), dims)
    out = gve.gve_evaluate(dev(p), shape).cpu().numpy()
    assert rel_l2(out, vt) <= FIELD_TOL
    field = np.random.default_rng(1).uniform(0, 1, shape).astype(np.float32)
    gg, _ = gve.gve_loss_grad(dev(p), dev(field))
    gg = gg.cpu().numpy()
    assert np.isfinite(gg).all()
    assert (gg[:4] == 0).all()


def test_invalid_arguments_raise():
    p = torch.zeros((4, 12), device="cuda")
    with pytest.raises(gve.GveError):
        gve.gve_evaluate(p, (8, 8, 8), gve.EvalOptions(brick=5))
    with pytest.raises(gve.GveError):
        gve.gve_evaluate(p, (8, 8, 8), gve.EvalOptions(trunc_k=-1.0))
    # an axis beyond 2^14 voxels lies outside the brick cover's float32 margins
    with pytest.raises(gve.GveError):
        gve.gve_evaluate(p, (1, 1, (1 << 14) + 1))
    with pytest.raises(ValueError):
        gve.gve_evaluate(p.double(), (8, 8, 8))


@pytest.fixture(scope="module")
def small_workload():
    V = inputs.blobs(64, seed=1)
    prm, vox, st, status = O.allocate(V, 4096, seed=0)
    assert status == 0
    return V, prm


def test_refine_psnr_parity_small(small_workload):
    """64^3 blobs, 4,096 Gaussians from the analytic allocation, 20 Adam
    iterations at lr 1e-2, 3-sigma truncation: final PSNR within 0.05 dB."""
    V, prm = small_workload
    p32 = prm.astype(np.float32)
    ref, losses, sse = O.refine(p32.astype(np.float64), V, iters=20, lr=1e-2, eps=1e-15)
    psnr_ref = O.psnr_from_sse(sse, V.size)
    P = dev(p32)
    trace = torch.zeros(20, dtype=torch.float64, device="cuda")
    st = gve.gve_refine(P, dev(V), iters=20, lr=1e-2, eps=1e-15, trace=trace)
    assert abs(st["psnr_final"] - psnr_ref) <= PSNR_TOL
    np.testing.assert_allclose(trace.cpu().numpy(), losses, rtol=2e-3)
    assert st["psnr_final"] > O.psnr_from_sse(O.loss_grad(p32.astype(np.float64), V, want_grad=False)[2], V.size)


def test_refine_resumes_with_adam_state(small_workload):
    """Two calls of 10 iterations with carried Adam moments equal one call of 20."""
    V, prm = small_workload
    p32 = prm.astype(np.float32)
    A = dev(p32)
    gve.gve_refine(A, dev(V), iters=20)
    B = dev(p32)
    state = torch.zeros((2, p32.shape[0], 12), device="cuda")
    gve.gve_refine(B, dev(V), iters=10, adam_state=state)
    gve.gve_refine(B, dev(V), iters=10, adam_state=state, step0=10)
    assert rel_l2(B.cpu().numpy(), A.cpu().numpy()) <= 1e-5


def test_allocate_matches_oracle(small_workload):
    V, prm = small_workload
    P, info = gve.gve_allocate(dev(V), 4096, seed=0)
    P = P.cpu().numpy()
    # same seeds in the same order: centres agree to float32 rounding of c + u
    np.testing.assert_allclose(P[:, 0:3], prm[:, 0:3], rtol=0, atol=1e-5)
    np.testing.assert_allclose(P[:, 3:6], prm[:, 3:6], rtol=0, atol=1e-5)
    # quaternions up to sign
    dots = np.abs(np.sum(P[:, 6:10] * prm[:, 6:10], axis=1))
    assert (dots > 1 - 1e-5).mean() > 0.999
    np.testing.assert_allclose(P[:, 10:12], prm[:, 10:12], rtol=1e-5, atol=1e-6)
    assert info["n_detail"] == 2253 and info["n_coverage"] == 4096 - 2253


@pytest.mark.parametrize("kind,occ", [("grf", 0.02), ("fbm", 0.02), ("fbm", 0.5)])
def test_two_level_draws_match_full_keys(kind, occ):
    """Both draws select on 32-bit surrogates of their keys first and compute
    the full keys (FP64 for the detail draw) only for the voxels near the
    threshold; the allocation equals the one drawn from full keys at every
    voxel bit for bit, from small budgets to the largest one the field
    supports (thresholds among the largest keys), with most voxels occupied
    or about half of them."""
    dev_ = torch.device("cuda", 0)
    V = inputs.grf(96, seed=21, device=dev_) if kind == "grf" else inputs.fbm_fronts(96, seed=22, device=dev_)
    try:
        gve.gve_allocate(V, 10 ** 9, seed=5, occ_thresh=occ)
        raise AssertionError("a budget of 10^9 on 96^3 voxels must be infeasible")
    except gve.BudgetError as e:
        fmax = e.feasible_max
    # 20,000: a few candidates; a quarter of the voxels: about as many
    # candidates as fit beside the surrogates; fmax: the full-key fallback
    for budget in (20_000, V.numel() // 4, fmax):
        P, info = gve.gve_allocate(V, budget, seed=5, occ_thresh=occ)
        os.environ["GVE_TEST_DRAW_FULL"] = "1"
        try:
            Q, info_q = gve.gve_allocate(V, budget, seed=5, occ_thresh=occ)
        finally:
            del os.environ["GVE_TEST_DRAW_FULL"]
        assert torch.equal(P, Q), budget
        assert info == info_q


def test_allocate_grf_and_budget_error():
    V = inputs.grf((40, 36, 28), seed=12)
    ref, vox, st, status = O.allocate(V, 3000, seed=9)
    P, info = gve.gve_allocate(dev(V), 3000, seed=9)
    P = P.cpu().numpy()
    np.testing.assert_allclose(P[:, 0:3], ref[:, 0:3], rtol=0, atol=1e-5)
    np.testing.assert_allclose(P[:, 3:6], ref[:, 3:6], atol=1e-5)
    assert info["n_occupied"] == st["n_occupied"] and info["n_eligible"] == st["n_eligible"]
    assert info["gbar"] == st["gbar"]
    assert info["h_detail"] == st["h_detail"] and info["h_coverage"] == st["h_coverage"]
    # infeasible: a field with few occupied voxels
    W = np.zeros((16, 16, 16), np.float32)
    W[6:10, 6:10, 6:10] = 1.0
    _, _, st2, status2 = O.allocate(W, 1000, seed=1)
    assert status2 == 2
    with pytest.raises(gve.BudgetError) as ei:
        gve.gve_allocate(dev(W), 1000, seed=1)
    assert ei.value.feasible_max == st2["feasible_max"]


BRICK_VARIANTS = [(4, 0), (16, 0), (8, 32), (4, 32), (16, 32)]


@pytest.mark.parametrize("brick,chunk", BRICK_VARIANTS)
@pytest.mark.parametrize("case", ["ragged", "long_lists", "small_gauss"])
def test_brick_variants_bin_eval_grad(case, brick, chunk):
    """Other brick edges and chunk sizes: bit-exact binning and kept-pair
    counts, the same field and gradient tolerances."""
    dims, n, lo, hi, seed = CASES[case]
    shape = (dims[2], dims[1], dims[0])
    rng = np.random.default_rng(seed + 20)
    p = rand_prims(rng, n, dims, lo, hi)
    opts = gve.EvalOptions(brick=brick, gaussians_per_block=chunk)
    counts, sk, sg, start, end = O.bin_sorted(p, dims, 3.0, brick)
    gc, gk, gg, gs, ge = gve.gve_bin(dev(p), shape, opts)
    np.testing.assert_array_equal(gc.numpy(), counts.astype(np.int64))
    np.testing.assert_array_equal(gk.numpy(), sk.astype(np.int64))
    np.testing.assert_array_equal(gg.numpy(), sg.astype(np.int64))
    np.testing.assert_array_equal(gs.numpy(), start.astype(np.int64))
    np.testing.assert_array_equal(ge.numpy(), end.astype(np.int64))
    kept, cand = gve.gve_count_pairs(dev(p), shape, opts)
    assert kept == O.count_kept(p, dims, 3.0)
    _, _, vt = O.eval_region(p, dims)
    assert rel_l2(gve.gve_evaluate(dev(p), shape, opts).cpu().numpy(), vt) <= FIELD_TOL
    field = rng.uniform(0, 1, shape).astype(np.float32)
    L, g, sse = O.loss_grad(p.astype(np.float64), field)
    gg2, gsse = gve.gve_loss_grad(dev(p), dev(field), opts)
    assert abs(gsse[1].item() - sse) <= 1e-5 * sse
    assert rel_l2(gg2.cpu().numpy(), g) <= GRAD_TOL


# sparse grids with more than 2^16 bricks (17-18 bit brick keys): thousands
# of tiles of 4^3 bricks, and tile lists spread over many radix-sort tiles
# (more than 4,096 tile pairs)
SCALE_CASES = {
    # name: (dims (nx, ny, nz), brick, n, s_lo, s_hi, seed)
    "b4_18bit": ((1040, 520, 16), 4, 6000, 0.6, 2.5, 31),
    "b8_17bit": ((1024, 1024, 40), 8, 12000, 0.8, 3.0, 32),
}


@pytest.mark.parametrize("case", list(SCALE_CASES))
def test_binning_bit_exact_large_sparse_grids(case):
    dims, brick, n, lo, hi, seed = SCALE_CASES[case]
    nb = np.prod([(d + brick - 1) // brick for d in dims])
    assert nb > 2 ** 16
    p = rand_prims(np.random.default_rng(seed), n, dims, lo, hi)
    counts, sk, sg, start, end = O.bin_sorted(p, dims, 3.0, brick)
    assert sk.size > 8 * 4096
    gc, gk, gg, gs, ge = gve.gve_bin(dev(p), (dims[2], dims[1], dims[0]), gve.EvalOptions(brick=brick))
    np.testing.assert_array_equal(gc.numpy(), counts.astype(np.int64))
    np.testing.assert_array_equal(gk.numpy(), sk.astype(np.int64))
    np.testing.assert_array_equal(gg.numpy(), sg.astype(np.int64))
    np.testing.assert_array_equal(gs.numpy(), start.astype(np.int64))
    np.testing.assert_array_equal(ge.numpy(), end.astype(np.int64))


@pytest.mark.parametrize("case", ["ragged", "small_gauss", "long_lists"])
def test_kept_pair_sets_equal(case):
    """The kept (voxel, Gaussian) pairs themselves, not only their number:
    the set the evaluator keeps equals the oracle's float32 keep rule."""
    dims, n, lo, hi, seed = CASES[case]
    p = rand_prims(np.random.default_rng(seed), n, dims, lo, hi)
    ref = O.list_kept(p, dims, 3.0)
    got = gve.gve_kept_pairs(dev(p), (dims[2], dims[1], dims[0])).numpy()
    assert got.shape == ref.shape
    np.testing.assert_array_equal(got, ref)
