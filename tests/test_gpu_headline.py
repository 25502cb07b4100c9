"""Parity at the headline configuration: the 1024^3 fBm + fronts field
(4.3 GB) with 1,400,000 Gaussians, the size at which every throughput number
is measured.

Only this size exercises the 21-bit brick keys (2.1 M bricks in 32,768 tiles
of 4^3 bricks, about 1.4e8 brick pairs written from per-brick counts, over
10^7 tile pairs sorted in thousands of radix-sort tiles), Gaussian lists of
1.4 M records and the allocator's selections over 10^9 voxels.  The FP64 oracle
cannot refine at this size, so it checks what it can compute exactly:

* allocation (Sec. III-E, S1a-S1e): the split, distinct and eligible seeds,
  an exhaustive census over all 10^9 voxels showing that the detail and
  coverage sets are exactly the Nd / Nc smallest keys, the lower-median
  gbar, both group spacings, and the records of 4,096 sampled seeds;
* Eq. 3 on 64 seeded random 32^3 sub-blocks (relative L2 <= 1e-5 each) and
  the loss gradient of 64 seeded Gaussians (relative L2 <= 1e-4, whole record
  and each parameter group), at the allocation and again after 5 refinement
  iterations on the GPU (parameters that have moved off the allocation).
"""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2608_14112_b300 import gve, inputs

pytestmark = pytest.mark.gpu

N = 1_400_000
SEED = 4
EDGE = 1024
FIELD_TOL = 1e-5
GRAD_TOL = 1e-4
GROUPS = {"mu": slice(0, 3), "log_s": slice(3, 6), "q": slice(6, 10), "a": slice(10, 11), "w_logit": slice(11, 12)}


def rel_l2(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))


@pytest.fixture(scope="module")
def headline():
    torch.cuda.set_device(0)
    V = inputs.fbm_fronts(EDGE, seed=SEED, device="cuda")
    Vh = V.cpu().numpy()
    prims, info = gve.gve_allocate(V, N, seed=SEED)
    torch.cuda.synchronize()
    yield V, Vh, prims, info
    del V, prims
    torch.cuda.empty_cache()


def _seed_voxels(P, info):
    """Voxel index of every seed: c = mu - u with u the seed's own jitter."""
    Nd, Nc = info["n_detail"], info["n_coverage"]
    u = np.concatenate([O.jitter_many(Nd, 0, SEED), O.jitter_many(Nc, 1, SEED)]).astype(np.float64)
    c = np.rint(P[:, 0:3].astype(np.float64) - u).astype(np.int64)
    assert np.abs(P[:, 0:3] - (c + u)).max() <= 1e-4   # float32 rounding of c + u
    return (c[:, 2] * EDGE + c[:, 1]) * EDGE + c[:, 0]


def test_headline_allocation_census(headline):
    V, Vh, prims, info = headline
    P = prims.cpu().numpy()
    Nd, Nc = info["n_detail"], info["n_coverage"]
    assert (Nd, Nc) == (770_000, 630_000)
    vox = _seed_voxels(P, info)
    vd, vc = vox[:Nd], vox[Nd:]
    # distinct within each draw, in ascending voxel order
    assert (np.diff(vd) > 0).all() and (np.diff(vc) > 0).all()
    flat = Vh.reshape(-1)
    gd = O.grad_mag32_at(Vh, vd)
    assert (flat[vd] > np.float32(0.02)).all() and (gd > 0).all()
    assert (flat[vc] > np.float32(0.02)).all()
    # the largest (key, index) of each selected set ...
    kd = O.detail_keys(vd, gd, SEED)
    jd = np.lexsort((vd, kd))[-1]
    ku = O.coverage_keys(vc, SEED)
    ju = np.lexsort((vc, ku))[-1]
    cen = O.draw_census(Vh, SEED, kd[jd], int(vd[jd]), int(ku[ju]), int(vc[ju]), info["gbar"])
    assert cen["n_occupied"] == info["n_occupied"] and cen["n_eligible"] == info["n_eligible"]
    # ... bounds exactly Nd (Nc) keys over the whole grid: each set is the
    # Nd (Nc) smallest keys (Efraimidis-Spirakis for the detail draw)
    assert cen["detail_at_most"] == Nd
    assert cen["coverage_at_most"] == Nc
    # gbar is the lower median of |grad V| over the occupied voxels
    k = (cen["n_occupied"] - 1) // 2
    assert cen["g_below"] <= k < cen["g_at_most"]
    # S1c: both group spacings
    dims = (EDGE, EDGE, EDGE)
    hd = O.group_spacing(vd, dims, info["n_occupied"], N)
    hc = O.group_spacing(vc, dims, info["n_occupied"], N)
    assert abs(info["h_detail"] - hd) <= 1e-12 * hd and abs(info["h_coverage"] - hc) <= 1e-12 * hc
    # S1d + S1e: the records of 4,096 sampled seeds
    rng = np.random.default_rng(77)
    ids = np.sort(rng.choice(N, 4096, replace=False))
    grp = (ids >= Nd).astype(np.int32)
    gi = np.where(grp == 0, ids, ids - Nd)
    ref = O.assemble_seeds(Vh, vox[ids], gi, grp, SEED, info["h_detail"], info["h_coverage"], info["gbar"])
    got = P[ids]
    np.testing.assert_allclose(got[:, 0:3], ref[:, 0:3], rtol=0, atol=1e-4)
    np.testing.assert_allclose(got[:, 3:6], ref[:, 3:6], rtol=0, atol=1e-5)
    dots = np.abs(np.sum(got[:, 6:10] * ref[:, 6:10], axis=1))
    assert (dots > 1 - 1e-5).mean() > 0.999
    np.testing.assert_allclose(got[:, 10:12], ref[:, 10:12], rtol=1e-5, atol=1e-6)


def _blocks(rng, count=64, size=32):
    return rng.integers(0, EDGE - size + 1, size=(count, 3))


def _check_field_and_gradients(V, Vh, prims, tag):
    P = prims.cpu().numpy().astype(np.float64)
    rng = np.random.default_rng({"allocation": 5, "refined": 6}[tag])
    corners = _blocks(rng)
    out = gve.gve_evaluate(prims, Vh.shape)
    got = torch.stack([out[z:z + 32, y:y + 32, x:x + 32] for x, y, z in corners]).cpu().numpy()
    del out
    ref = O.eval_blocks(P, (EDGE, EDGE, EDGE), corners, (32, 32, 32))
    per_block = [rel_l2(got[b], ref[b]) for b in range(len(corners))]
    assert max(per_block) <= FIELD_TOL, (tag, max(per_block))
    ids = np.sort(rng.choice(P.shape[0], 64, replace=False))
    g_gpu, _ = gve.gve_loss_grad(prims, V)
    gg = g_gpu[torch.from_numpy(ids).cuda()].cpu().numpy()
    gr = O.grad_subset(P, Vh, ids)
    assert rel_l2(gg, gr) <= GRAD_TOL, (tag, rel_l2(gg, gr))
    for name, sl in GROUPS.items():
        assert rel_l2(gg[:, sl], gr[:, sl]) <= GRAD_TOL, (tag, name, rel_l2(gg[:, sl], gr[:, sl]))


def test_headline_field_and_gradients_at_allocation(headline):
    V, Vh, prims, _ = headline
    _check_field_and_gradients(V, Vh, prims, "allocation")


def test_headline_field_and_gradients_after_refinement(headline):
    V, Vh, prims, _ = headline
    P = prims.clone()
    st = gve.gve_refine(P, V, iters=5, lr=1e-2)
    assert st["retries"] >= 0 and np.isfinite(st["psnr_final"])
    assert st["brick_pairs"] > 50_000_000       # 21-bit brick keys, tile lists over thousands of sort tiles
    moved = (P - prims).abs().max().item()
    assert moved > 1e-3
    _check_field_and_gradients(V, Vh, P, "refined")
