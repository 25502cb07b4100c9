"""Pins of the FP64 CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: published
known-answer vectors, closed forms, library routines solving the same
mathematical problem (numpy/scipy/torch autograd), brute force on tiny grids,
exact invariants, and numbers printed in the paper (arxiv 2608.14112).
"""
import math
import os

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

from oracle import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rand_prims(rng, n, dims, s_lo=0.8, s_hi=2.5, aniso=True):
    """Random raw records: mu inside the grid, log-scales, random quaternion,
    a in [0.1, 1], w_logit around logit(0.1..0.9)."""
    p = np.zeros((n, 12))
    p[:, 0:3] = rng.uniform(0, 1, (n, 3)) * (np.array(dims) - 1)
    s = rng.uniform(s_lo, s_hi, (n, 3)) if aniso else np.repeat(rng.uniform(s_lo, s_hi, (n, 1)), 3, 1)
    p[:, 3:6] = np.log(s)
    p[:, 6:10] = rng.normal(size=(n, 4)) * rng.uniform(0.5, 2.0, (n, 1))
    p[:, 10] = rng.uniform(0.1, 1.0, n)
    p[:, 11] = rng.uniform(-2.0, 2.0, n)
    return p


def _dense_numpy(prm, dims, rho0=0.05, normalized=True):
    """Untruncated Eq. 3 written with scipy's rotation and numpy's inverse:
    independent of the oracle's R(q) and conic."""
    nx, ny, nz = dims
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    P = np.stack([x, y, z], -1).astype(np.float64)
    num = np.zeros((nz, ny, nx))
    den = np.zeros((nz, ny, nx))
    for r in prm:
        q = r[6:10]
        Rm = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()  # scipy: (x,y,z,w)
        S = np.diag(np.exp(2 * r[3:6]))
        Sig = Rm @ S @ Rm.T
        Ci = np.linalg.inv(Sig)
        d = P - r[0:3]
        m = np.einsum("...i,ij,...j->...", d, Ci, d)
        G = np.exp(-0.5 * m)
        w = 1 / (1 + np.exp(-r[11]))
        num += w * r[10] * G
        den += w * G
    vt = num / np.maximum(den, rho0) if normalized else num
    return num, den, vt, P


# ------------------------------------------------------------------------
# Philox4x32-10: published known-answer vectors
# ------------------------------------------------------------------------
def test_philox_known_answers():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(t, 16) for t in r]
        out = O.philox4x32_10(v[0:4], v[4:6])
        assert [int(o) for o in out] == v[6:10]


# ------------------------------------------------------------------------
# Field, Eq. 3
# ------------------------------------------------------------------------
def test_dense_matches_independent_numpy():
    rng = np.random.default_rng(11)
    dims = (13, 11, 9)
    prm = _rand_prims(rng, 6, dims)
    num, den, vt = O.eval_region(prm, dims, truncated=False)
    n2, d2, v2, _ = _dense_numpy(prm, dims)
    np.testing.assert_allclose(num, n2, rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(den, d2, rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(vt, v2, rtol=1e-12, atol=1e-14)
    _, _, vp = O.eval_region(prm, dims, truncated=False, normalized=False)
    np.testing.assert_allclose(vp, n2, rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("k", [3.0, 5.0])
def test_single_gaussian_closed_form(k):
    """One Gaussian: Vt = a where wG >= rho0, a wG/rho0 where wG < rho0,
    and 0 outside the truncation ellipsoid (Eq. 3 with N = 1)."""
    dims = (24, 24, 24)
    rng = np.random.default_rng(5)
    p = _rand_prims(rng, 1, dims, s_lo=1.5, s_hi=3.0)
    p[0, 0:3] = [11.3, 12.6, 11.9]
    num, den, vt = O.eval_region(p, dims, k=k)
    _, _, _, P = _dense_numpy(p, dims)
    r = p[0]
    Rm = Rotation.from_quat([r[7], r[8], r[9], r[6]]).as_matrix()
    Ci = np.linalg.inv(Rm @ np.diag(np.exp(2 * r[3:6])) @ Rm.T)
    d = P - r[0:3]
    m = np.einsum("...i,ij,...j->...", d, Ci, d)
    w = 1 / (1 + np.exp(-r[11]))
    wG = w * np.exp(-0.5 * m)
    expect = np.where(wG >= 0.05, r[10], r[10] * wG / 0.05)
    expect = np.where(m < k * k, expect, 0.0)
    away = np.abs(m - k * k) > 1e-4 * k * k   # the float32 decision is exact away from the surface
    np.testing.assert_allclose(vt[away], expect[away], rtol=1e-12, atol=1e-15)
    assert (vt[m > k * k * 1.0001] == 0).all()
    assert (vt[m < k * k * 0.9999] != 0).all()
    # plain (unnormalised) mode: w a G
    _, _, vp = O.eval_region(p, dims, k=k, normalized=False)
    np.testing.assert_allclose(vp[away], np.where(m < k * k, r[10] * wG, 0)[away], rtol=1e-12, atol=1e-15)


def test_float32_decision_agrees_with_fp64_away_from_surface():
    rng = np.random.default_rng(3)
    dims = (30, 30, 30)
    prm = _rand_prims(rng, 20, dims, s_lo=0.5, s_hi=4.0)
    T = O.pred_threshold(3.0)
    assert T < 0
    for r in prm:
        p32 = r.astype(np.float32)
        r64 = p32.astype(np.float64)
        Rm = Rotation.from_quat([r64[7], r64[8], r64[9], r64[6]]).as_matrix()
        Ci = np.linalg.inv(Rm @ np.diag(np.exp(2 * r64[3:6])) @ Rm.T)
        for _ in range(60):
            v = rng.integers(0, 30, 3)
            d = v - r64[0:3]
            m = d @ Ci @ d
            t = O.pred_t(p32, *v)
            # t is -0.5*log2(e)*m in float32
            assert abs(t - (-0.5 / math.log(2)) * m) <= 1e-5 * max(1.0, m)
            if abs(m - 9.0) > 1e-4 * 9.0:
                assert (t > T) == (m < 9.0)


def test_truncation_error_bounded_and_k20_is_dense():
    """|Vt_k - Vt_inf| <= (|N_o| + |Vt_k| D_o)/rho0, where N_o, D_o are the
    omitted parts of the sums, each a priori <= sum_i w_i max(|a_i|,1) e^{-k^2/2}."""
    rng = np.random.default_rng(7)
    dims = (20, 18, 16)
    prm = _rand_prims(rng, 12, dims)
    nI, dI, vI, _ = _dense_numpy(prm, dims)
    w = 1 / (1 + np.exp(-prm[:, 11]))
    for k in (2.0, 3.0, 5.0):
        nk, dk, vk = O.eval_region(prm, dims, k=k)
        No, Do = nI - nk, dI - dk
        assert (Do >= -1e-15).all()
        apriori = np.sum(w * np.maximum(np.abs(prm[:, 10]), 1.0)) * math.exp(-k * k / 2)
        assert np.abs(No).max() <= apriori * 1.0001 + 1e-15
        assert Do.max() <= apriori * 1.0001 + 1e-15
        bound = (np.abs(No) + np.abs(vk) * Do) / 0.05
        assert (np.abs(vI - vk) <= bound * (1 + 1e-9) + 1e-13).all()
    _, _, v20 = O.eval_region(prm, dims, k=20.0)
    np.testing.assert_allclose(v20, vI, rtol=1e-12, atol=1e-14)


def test_region_evaluation_matches_full_grid():
    rng = np.random.default_rng(8)
    dims = (19, 23, 17)
    prm = _rand_prims(rng, 15, dims)
    _, _, vt = O.eval_region(prm, dims)
    _, _, sub = O.eval_region(prm, dims, region=((3, 5, 2), (9, 7, 11)))
    np.testing.assert_array_equal(sub, vt[2:13, 5:12, 3:12])


# ------------------------------------------------------------------------
# Loss, PSNR and gradient
# ------------------------------------------------------------------------
def test_psnr_textbook():
    """No Gaussians: Vt = 0, so against a constant field c MSE = c^2 and
    PSNR = 10 log10(1/c^2) (Sec. IV-C definition with V_max = 1)."""
    f = np.full((4, 5, 6), 0.25, np.float32)
    L, _, sse = O.loss_grad(np.zeros((0, 12)), f, want_grad=False)
    assert L == pytest.approx(0.0625, rel=1e-15)
    assert O.psnr_from_sse(sse, f.size) == pytest.approx(-20 * math.log10(0.25), rel=1e-12)


def _fd_case(seed=21):
    rng = np.random.default_rng(seed)
    dims = (12, 11, 10)
    prm = _rand_prims(rng, 5, dims, s_lo=1.0, s_hi=2.2)
    field = rng.uniform(0, 1, (10, 11, 12)).astype(np.float32)
    return prm, field


@pytest.mark.parametrize("normalized", [True, False])
@pytest.mark.parametrize("mask", [-1.0, 0.3])
def test_gradient_central_differences_frozen_membership(normalized, mask):
    """Central differences of the FP64 loss with membership frozen at the
    unperturbed parameters (the kept set is piecewise constant in mu, s, q);
    a and w_logit do not move the truncation surface at all.  h = 3e-5 keeps
    both the O(h^2) error and the summation round-off near 1e-7 (the density
    floor max(den, rho0) is a kink, so much larger steps may straddle it)."""
    prm, field = _fd_case()
    L0, g, _ = O.loss_grad(prm, field, normalized=normalized, mask_thresh=mask)
    h = 3e-5
    for i in range(prm.shape[0]):
        for j in range(12):
            pp, pm = prm.copy(), prm.copy()
            pp[i, j] += h
            pm[i, j] -= h
            Lp, _, _ = O.loss_grad(pp, field, normalized=normalized, mask_thresh=mask,
                                   pred_prm=prm, want_grad=False)
            Lm, _, _ = O.loss_grad(pm, field, normalized=normalized, mask_thresh=mask,
                                   pred_prm=prm, want_grad=False)
            fd = (Lp - Lm) / (2 * h)
            assert abs(fd - g[i, j]) <= 1e-6 * max(abs(fd), 1e-4), (i, j, fd, g[i, j])


def test_gradient_matches_torch_autograd_dense():
    """Untruncated loss differentiated by torch autograd (float64): an
    independent derivation of the chain rule through Eq. 3 and Eq. 2."""
    torch = pytest.importorskip("torch")
    prm, field = _fd_case(seed=4)
    _, g, _ = O.loss_grad(prm, field, truncated=False)
    P = torch.tensor(prm, dtype=torch.float64, requires_grad=True)
    nz, ny, nx = field.shape
    zz, yy, xx = torch.meshgrid(torch.arange(nz), torch.arange(ny), torch.arange(nx), indexing="ij")
    X = torch.stack([xx, yy, zz], -1).double()
    num = torch.zeros(nz, ny, nx, dtype=torch.float64)
    den = torch.zeros_like(num)
    for i in range(P.shape[0]):
        r = P[i]
        q = r[6:10] / torch.linalg.norm(r[6:10])
        w_, x_, y_, z_ = q
        Rm = torch.stack([
            torch.stack([1 - 2 * (y_ ** 2 + z_ ** 2), 2 * (x_ * y_ - w_ * z_), 2 * (x_ * z_ + w_ * y_)]),
            torch.stack([2 * (x_ * y_ + w_ * z_), 1 - 2 * (x_ ** 2 + z_ ** 2), 2 * (y_ * z_ - w_ * x_)]),
            torch.stack([2 * (x_ * z_ - w_ * y_), 2 * (y_ * z_ + w_ * x_), 1 - 2 * (x_ ** 2 + y_ ** 2)])])
        Sig = Rm @ torch.diag(torch.exp(2 * r[3:6])) @ Rm.T
        Ci = torch.linalg.inv(Sig)
        d = X - r[0:3]
        m = torch.einsum("...i,ij,...j->...", d, Ci, d)
        G = torch.exp(-0.5 * m)
        w = torch.sigmoid(r[11])
        num = num + w * r[10] * G
        den = den + w * G
    vt = num / torch.clamp(den, min=0.05)
    loss = ((vt - torch.tensor(field, dtype=torch.float64)) ** 2).mean()
    loss.backward()
    np.testing.assert_allclose(g, P.grad.numpy(), rtol=1e-9, atol=1e-13)


def test_gradient_subset_matches_full():
    prm, field = _fd_case(seed=9)
    _, g, _ = O.loss_grad(prm, field)
    ids = np.array([3, 0, 4])
    gs = O.grad_subset(prm, field, ids)
    np.testing.assert_allclose(gs, g[ids], rtol=1e-12, atol=1e-16)


def test_adam_matches_torch_optim():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(2)
    p0 = rng.normal(size=24)
    grads = [rng.normal(size=24) * 10 ** rng.uniform(-8, 0) for _ in range(6)]
    p, m, v = p0.copy(), np.zeros(24), np.zeros(24)
    for t, g in enumerate(grads, 1):
        O.adam_step(p, m, v, g, t, lr=1e-2, eps=1e-15)
    T = torch.tensor(p0, dtype=torch.float64, requires_grad=True)
    opt = torch.optim.Adam([T], lr=1e-2, betas=(0.9, 0.999), eps=1e-15)
    for g in grads:
        opt.zero_grad()
        T.grad = torch.tensor(g, dtype=torch.float64)
        opt.step()
    np.testing.assert_allclose(p, T.detach().numpy(), rtol=1e-12, atol=1e-14)


def test_refine_decreases_loss_and_reports_final_sse():
    rng = np.random.default_rng(12)
    dims = (16, 16, 16)
    prm = _rand_prims(rng, 30, dims, s_lo=1.2, s_hi=2.5)
    field = np.asarray(O.eval_region(_rand_prims(rng, 10, dims), dims)[2], np.float32)
    out, losses, sse = O.refine(prm, field, iters=8, lr=2e-2)
    assert losses[-1] < losses[0]
    L, _, sse2 = O.loss_grad(out, field, want_grad=False)
    assert sse == pytest.approx(sse2, rel=1e-15)


# ------------------------------------------------------------------------
# Brick binning: every kept pair is covered
# ------------------------------------------------------------------------
@pytest.mark.parametrize("B", [4, 8])
def test_binning_covers_every_kept_pair(B):
    rng = np.random.default_rng(100 + B)
    dims = (21, 17, 13)
    prm = np.concatenate([_rand_prims(rng, 25, dims, s_lo=0.3, s_hi=3.0),
                          _rand_prims(rng, 10, dims, s_lo=0.5, s_hi=1.0, aniso=False)])
    # strongly anisotropic ones too
    prm[:5, 3] = np.log(6.0)
    prm[:5, 4] = np.log(0.4)
    p32 = prm.astype(np.float32)
    counts, keys, gids = O.bin_pairs(p32, dims, 3.0, B)
    nbx, nby = (dims[0] + B - 1) // B, (dims[1] + B - 1) // B
    listed = {}
    for kk, gg in zip(keys, gids):
        listed.setdefault(int(gg), set()).add(int(kk))
    T = O.pred_threshold(3.0)
    kept_bricks = 0
    for i in range(prm.shape[0]):
        need = set()
        for z in range(dims[2]):
            for y in range(dims[1]):
                for x in range(dims[0]):
                    if O.pred_t(p32[i], x, y, z) > T:
                        need.add((z // B * nby + y // B) * nbx + x // B)
        assert need <= listed.get(i, set()), i
        kept_bricks += len(need)
        assert counts[i] == len(listed.get(i, set()))
    # emission order: Gaussian-major, bricks ascending within a Gaussian
    assert (np.diff(gids.astype(np.int64)) >= 0).all()
    for i in range(prm.shape[0]):
        kk = keys[gids == i]
        assert (np.diff(kk.astype(np.int64)) > 0).all()
    # conservative but not wasteful
    assert keys.size <= 3 * kept_bricks + 8


def test_binning_sorted_ranges_consistent():
    rng = np.random.default_rng(5)
    dims = (33, 20, 9)
    p32 = _rand_prims(rng, 40, dims).astype(np.float32)
    counts, sk, sg, start, end = O.bin_sorted(p32, dims, 3.0, 8)
    assert (np.diff(sk.astype(np.int64)) >= 0).all()
    for b in range(start.size):
        seg = sg[start[b]:end[b]]
        assert (sk[start[b]:end[b]] == b).all()
        assert (np.diff(seg.astype(np.int64)) > 0).all()
    assert int((end - start).sum()) == sk.size == int(counts.sum())


# ------------------------------------------------------------------------
# Allocation (Sec. III-E, Table I S1a..S1e, Sec. V-B)
# ------------------------------------------------------------------------
def test_detail_coverage_split_golden():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "nd_split.txt"))
            if l.strip() and not l.startswith("#")]
    for N, Nd, Nc in ((int(a), int(b), int(c)) for a, b, c in rows):
        assert O.feasible_max(N, 0.55, N, N) == N
        # the split itself: feasible with exactly Nd eligible, infeasible with Nd-1
        assert O.feasible_max(N, 0.55, Nd, Nc) == N
        assert O.feasible_max(N, 0.55, Nd - 1, N) < N
        assert O.feasible_max(N, 0.55, N, Nc - 1) < N


def test_seed_limit_matches_paper():
    row = [l.split() for l in open(os.path.join(GOLDEN, "seed_limit.txt"))
           if l.strip() and not l.startswith("#")][0]
    elig, frac, approx, tol = int(row[0]), float(row[1]), int(row[2]), float(row[3])
    fm = O.feasible_max(10_000_000, frac, elig, 10 ** 9)
    assert abs(fm - approx) <= tol * approx
    assert fm == 228704  # floor(0.55 N + 1/2) <= 125787 <=> N <= 228704


def test_gradient_magnitude_ramp():
    nz, ny, nx = 9, 10, 11
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    a, b, c = 0.0125, -0.03125, 0.0078125   # dyadic: every difference exact in float32
    V = (a * x + b * y + c * z + 0.5).astype(np.float32)
    g = O.grad_mag32(V)
    np.testing.assert_allclose(g, math.sqrt(a * a + b * b + c * c), rtol=2e-6)


def test_structure_tensor_ramp_closed_form():
    nz, ny, nx = 16, 16, 16
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    gv = np.array([0.25, -0.5, 0.125])
    V = (gv[0] * x + gv[1] * y + gv[2] * z).astype(np.float32)
    outer = np.outer(gv, gv)
    expect6 = lambda n: n * np.array([outer[0, 0], outer[1, 1], outer[2, 2], outer[0, 1], outer[0, 2], outer[1, 2]])
    np.testing.assert_allclose(O.struct_tensor(V, (8, 7, 9)), expect6(343), rtol=1e-12)
    # corner: window clipped to 4^3
    np.testing.assert_allclose(O.struct_tensor(V, (0, 0, 0)), expect6(64), rtol=1e-12)
    # ramp: the tangent (smallest eigenvalue) is orthogonal to the gradient
    ev, vec = O.jacobi3(O.struct_tensor(V, (8, 7, 9)))
    assert abs(vec[:, 0] @ gv) < 1e-9
    assert abs(abs(vec[:, 2] @ gv) / np.linalg.norm(gv) - 1) < 1e-12


def test_jacobi_matches_numpy_eigh():
    rng = np.random.default_rng(0)
    for _ in range(200):
        A = rng.normal(size=(3, 3))
        S = A @ A.T + rng.uniform(0, 1) * np.eye(3)
        ev, vec = O.jacobi3([S[0, 0], S[1, 1], S[2, 2], S[0, 1], S[0, 2], S[1, 2]])
        ev2, vec2 = np.linalg.eigh(S)
        np.testing.assert_allclose(ev, ev2, rtol=1e-11, atol=1e-12)
        for c in range(3):
            if min(abs(ev2[c] - ev2[(c + 1) % 3]), abs(ev2[c] - ev2[(c + 2) % 3])) > 1e-6:
                assert abs(abs(vec[:, c] @ vec2[:, c]) - 1) < 1e-9
        np.testing.assert_allclose(vec.T @ vec, np.eye(3), atol=1e-12)


def test_plane_and_cylinder_orientation():
    n = 24
    z, y, x = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    nv = np.array([1.0, 2.0, 2.0]) / 3.0
    plane = np.tanh((nv[0] * (x - 12) + nv[1] * (y - 12) + nv[2] * (z - 12)) / 2).astype(np.float32)
    ev, vec = O.jacobi3(O.struct_tensor(plane, (12, 12, 12)))
    assert abs(abs(vec[:, 2] @ nv) - 1) < 1e-3       # normal = largest eigenvalue
    assert abs(vec[:, 0] @ nv) < 1e-3                # tangent lies in the plane
    axis = np.array([2.0, -1.0, 2.0]) / 3.0
    P = np.stack([x - 12.0, y - 12.0, z - 12.0], -1)
    r = np.linalg.norm(P - (P @ axis)[..., None] * axis, axis=-1)
    cyl = np.exp(-(r / 5.0) ** 2).astype(np.float32)
    ev, vec = O.jacobi3(O.struct_tensor(cyl, (15, 12, 12)))
    assert abs(abs(vec[:, 0] @ axis) - 1) < 2e-2    # tangent along the axis


def test_quaternion_from_rotation_all_branches():
    rots = list(Rotation.random(200, random_state=1))
    for ax in ([1, 0, 0], [0, 1, 0], [0, 0, 1]):  # near-180 degree turns exercise every branch
        rots.append(Rotation.from_rotvec(np.array(ax) * (math.pi - 1e-3)))
    for R in rots:
        M = R.as_matrix()
        q = O.quat_from_R(M)
        assert q[0] >= 0 and abs(np.linalg.norm(q) - 1) < 1e-12
        M2 = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()
        np.testing.assert_allclose(M2, M, atol=1e-12)


def test_canonical_frame_is_proper_rotation():
    rng = np.random.default_rng(4)
    for _ in range(50):
        Q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
        R = O.canonical_frame(Q)
        np.testing.assert_allclose(R.T @ R, np.eye(3), atol=1e-12)
        assert np.linalg.det(R) == pytest.approx(1.0, abs=1e-12)
        for c in range(2):
            assert abs(abs(R[:, c] @ Q[:, c]) - 1) < 1e-12
            assert R[np.argmax(np.abs(R[:, c])), c] > 0


def test_trilinear_exact_on_linear_field():
    nz, ny, nx = 7, 8, 9
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    V = (0.1 * x + 0.2 * y - 0.05 * z + 1).astype(np.float32).astype(np.float64)
    Vf = V.astype(np.float32)
    for p in [(1.25, 2.5, 3.75), (0.0, 0.0, 0.0), (7.9, 6.1, 5.5)]:
        expect = 0.1 * p[0] + 0.2 * p[1] - 0.05 * p[2] + 1
        assert O.trilinear(Vf, p) == pytest.approx(expect, abs=1e-6)
    assert O.trilinear(Vf, (-3, -3, -3)) == pytest.approx(float(Vf[0, 0, 0]))


def test_group_spacing_regular_lattice():
    dims = (30, 30, 30)
    vox = [((z * 30 + y) * 30 + x) for z in range(0, 30, 3) for y in range(0, 30, 3) for x in range(0, 30, 3)]
    assert O.group_spacing(sorted(vox), dims, 27000, 1000) == 3.0


def test_detail_draw_is_weighted_without_replacement():
    """Efraimidis-Spirakis: with k = 1 the winner is i with probability
    g_i / sum g (exponential race)."""
    g = np.array([0.5, 1.0, 2.0, 4.5], np.float32)
    wins = np.zeros(4)
    S = 20000
    for s in range(S):
        keys = [O.detail_key(v, s, g[v]) for v in range(4)]
        wins[int(np.argmin(keys))] += 1
    p = g / g.sum()
    chi2 = float(((wins - S * p) ** 2 / (S * p)).sum())
    assert chi2 < 16.3   # 3 d.o.f., p = 0.001
    wins = np.zeros(5)
    for s in range(S):
        wins[int(np.argmin([O.coverage_key(v, s) for v in range(5)]))] += 1
    chi2 = float(((wins - S / 5) ** 2 / (S / 5)).sum())
    assert chi2 < 18.5   # 4 d.o.f.


def test_jitter_range_and_determinism():
    for i in range(100):
        u = O.jitter(i, i % 2, 77)
        assert (u >= -0.5).all() and (u < 0.5).all()
        np.testing.assert_array_equal(u, O.jitter(i, i % 2, 77))


@pytest.fixture(scope="module")
def blobs64():
    from paper_2608_14112_b300 import inputs
    return inputs.blobs(64, seed=1)


def test_allocation_invariants(blobs64):
    V = blobs64
    N = 4096
    prm, vox, st, status = O.allocate(V, N, seed=3)
    assert status == 0 and prm.shape == (N, 12)
    Nd = st["n_detail"]
    assert Nd == 2253 and st["n_coverage"] == N - Nd
    g = O.grad_mag32(V).reshape(-1)
    Vf = V.reshape(-1)
    dv, cv = vox[:Nd], vox[Nd:]
    assert len(set(dv.tolist())) == Nd and len(set(cv.tolist())) == N - Nd
    assert (Vf[dv] > np.float32(0.02)).all() and (g[dv] > 0).all()
    assert (Vf[cv] > np.float32(0.02)).all()
    assert st["n_occupied"] == int((Vf > np.float32(0.02)).sum())
    c = np.stack([vox % 64, (vox // 64) % 64, vox // 4096], -1)
    assert (np.abs(prm[:, 0:3] - c) <= 0.5).all()
    np.testing.assert_allclose(np.linalg.norm(prm[:, 6:10], axis=1), 1.0, atol=1e-12)
    s = np.exp(prm[:, 3:6])
    assert (s >= 0.3 - 1e-12).all() and (s <= 4.0 + 1e-12).all()
    ratio = s[:, 0] / s[:, 1]
    assert (ratio >= 1 - 1e-12).all() and (ratio <= 3 + 1e-12).all()
    np.testing.assert_allclose(prm[:, 11], math.log(0.1 / 0.9), rtol=1e-15)
    # detail seeds are tighter than coverage seeds (Sec. III-E)
    assert st["h_detail"] <= st["h_coverage"]
    # the allocated model is already a meaningful reconstruction (S1x)
    L, _, sse = O.loss_grad(prm, V, want_grad=False)
    assert O.psnr_from_sse(sse, V.size) > 10.0


def test_allocation_detail_prefers_high_gradient(blobs64):
    V = blobs64
    prm, vox, st, _ = O.allocate(V, 4096, seed=3)
    g = O.grad_mag32(V).reshape(-1)
    occ = V.reshape(-1) > np.float32(0.02)
    assert g[vox[:st["n_detail"]]].mean() > 1.5 * g[occ].mean()


def test_allocation_infeasible_reports_shortfall():
    V = np.zeros((16, 16, 16), np.float32)
    V[6:10, 6:10, 6:10] = 1.0      # 64 occupied voxels, all with g > 0
    prm, vox, st, status = O.allocate(V, 1000, seed=1)
    assert status == 2
    fm = st["feasible_max"]
    assert fm == O.feasible_max(1000, 0.55, st["n_eligible"], st["n_occupied"])
    prm, vox, st2, status = O.allocate(V, fm, seed=1)
    assert status == 0 and prm.shape[0] == fm


def test_backward_upstream_central_differences():
    """dL/dtheta for L = sum_p U(p) Vt(p), U arbitrary: central differences
    of the frozen-membership field (the backward of Eq. 3 alone)."""
    rng = np.random.default_rng(31)
    dims = (10, 9, 11)
    prm = _rand_prims(rng, 4, dims, s_lo=1.0, s_hi=2.0)
    U = rng.normal(size=(11, 9, 10))
    g = O.backward(prm, U)
    h = 3e-5
    for i in range(prm.shape[0]):
        for j in range(12):
            pp, pm = prm.copy(), prm.copy()
            pp[i, j] += h
            pm[i, j] -= h
            Lp = float((U * O.eval_region(pp, dims, pred_prm=prm)[2]).sum())
            Lm = float((U * O.eval_region(pm, dims, pred_prm=prm)[2]).sum())
            fd = (Lp - Lm) / (2 * h)
            assert abs(fd - g[i, j]) <= 2e-6 * max(abs(fd), 1e-3), (i, j, fd, g[i, j])


def test_count_kept_brute_force():
    rng = np.random.default_rng(6)
    dims = (9, 8, 7)
    p32 = _rand_prims(rng, 6, dims).astype(np.float32)
    T = O.pred_threshold(3.0)
    brute = sum(O.pred_t(p32[i], x, y, z) > T for i in range(6)
                for z in range(7) for y in range(8) for x in range(9))
    assert O.count_kept(p32, dims, 3.0) == brute


def test_binning_empty_bricks_are_zero_ranges():
    """Bricks with no pair get [0, 0), wherever they sit in the key order."""
    dims = (40, 8, 8)
    p = np.zeros((2, 12))
    p[:, 3:6] = np.log(0.5)
    p[:, 6] = 1.0
    p[:, 10] = 0.5
    p[0, 0:3] = [2.0, 4.0, 4.0]
    p[1, 0:3] = [37.0, 4.0, 4.0]
    _, sk, sg, start, end = O.bin_sorted(p.astype(np.float32), dims, 3.0, 4)
    occupied = set(sk.tolist())
    for b in range(start.size):
        if b not in occupied:
            assert start[b] == 0 and end[b] == 0
    assert len(occupied) >= 2


def test_mlp_reference_gradient_central_differences():
    """The FP64 MLP reference: analytic gradient against central differences."""
    from oracle import mlp as M
    rng = np.random.default_rng(5)
    params = rng.normal(size=M.P) * 0.2
    mean, istd = rng.normal(size=16) * 0.1, rng.uniform(0.5, 2.0, 16)
    X = rng.normal(size=(9, 16))
    T = rng.normal(size=(9, 4)) * 0.3
    L, g = M.loss_grad(params, mean, istd, X, T)
    h = 1e-6
    for idx in rng.choice(M.P, 60, replace=False).tolist() + [M.P - 1, 0, 1100, 9400]:
        pp, pm = params.copy(), params.copy()
        pp[idx] += h
        pm[idx] -= h
        fd = (M.loss_grad(pp, mean, istd, X, T)[0] - M.loss_grad(pm, mean, istd, X, T)[0]) / (2 * h)
        assert abs(fd - g[idx]) <= 1e-6 * max(abs(fd), 1e-3), idx


def test_mlp_reference_gelu_closed_form():
    from oracle import mlp as M
    assert M.gelu(np.array(0.0)) == 0.0
    x = np.linspace(-4, 4, 81)
    # GELU(x) - GELU(-x) = x (odd part of x * Phi(x))
    np.testing.assert_allclose(M.gelu(x) - M.gelu(-x), x, atol=1e-15)
    h = 1e-6
    np.testing.assert_allclose(M.gelu_d(x), (M.gelu(x + h) - M.gelu(x - h)) / (2 * h), atol=1e-8)


def test_mlp_reference_backward_matches_mse_gradient_and_differences():
    """backward() with an arbitrary upstream gradient: a linear functional
    sum(C * y) has gradient backward(C), checked by central differences."""
    from oracle import mlp as M
    rng = np.random.default_rng(8)
    params = rng.normal(size=M.P) * 0.2
    mean, istd = rng.normal(size=16) * 0.1, rng.uniform(0.5, 2.0, 16)
    X = rng.normal(size=(7, 16))
    C = rng.normal(size=(7, 4))
    g = M.backward(params, mean, istd, X, C)
    h = 1e-6
    for idx in rng.choice(M.P, 40, replace=False).tolist() + [M.P - 1, 9664, 0]:
        pp, pm = params.copy(), params.copy()
        pp[idx] += h
        pm[idx] -= h
        fd = ((M.forward(pp, mean, istd, X)[0] * C).sum() - (M.forward(pm, mean, istd, X)[0] * C).sum()) / (2 * h)
        assert abs(fd - g[idx]) <= 1e-6 * max(abs(fd), 1e-3), idx


def test_proposal_chain_central_differences_and_clamp():
    """The end-to-end chain theta -> y -> corrected records -> sum(G * records):
    backward(upstream(...)) against central differences; a record whose
    log-scales sit at the clamp passes no log-scale gradient."""
    from oracle import mlp as M
    rng = np.random.default_rng(9)
    params = rng.normal(size=M.P) * 0.1
    mean, istd = np.zeros(16), np.ones(16)
    n, dims = 6, (64, 48, 40)
    X = rng.normal(size=(n, 16))
    prm = rng.normal(size=(n, 12))
    prm[:, 3:6] = rng.uniform(-0.5, 0.5, (n, 3))
    prm[2, 3:6] = 5.0          # far above log(64/16): clamped whatever the correction
    G = rng.normal(size=(n, 12))

    def L(th):
        y, _ = M.forward(th, mean, istd, X)
        return float((G * M.apply(prm, y, dims)).sum())

    y, _ = M.forward(params, mean, istd, X)
    pc = M.apply(prm, y, dims)
    lo, hi = M.ls_bounds(dims)
    assert np.all(pc[2, 3:6] == hi) and abs(hi - np.log(4.0)) < 1e-6 and abs(lo - np.log(0.3)) < 1e-6
    dY = M.upstream(pc, G, y, dims)
    assert np.all(dY[2, 1:] == 0.0) and dY[2, 0] == G[2, 10]
    g = M.backward(params, mean, istd, X, dY)
    h = 1e-5
    for idx in rng.choice(M.P, 40, replace=False).tolist() + [9408, 9664, 9667]:
        pp, pm = params.copy(), params.copy()
        pp[idx] += h
        pm[idx] -= h
        fd = (L(pp) - L(pm)) / (2 * h)
        assert abs(fd - g[idx]) <= 1e-6 * max(abs(fd), 1e-2), idx


def test_proposal_features_linear_field_closed_form():
    """On a linear field V = a x + b y + c z every feature has a closed form:
    central and one-sided differences both give the exact gradient g, so the
    7^3 structure tensor is cnt * g g^T (eigenvalues 0, 0, cnt |g|^2); the 5^3
    window's mean is V at its centre, its spread |g| sqrt(2) (variance of
    a uniform offset in {-2..2} is 2 per axis), its extremes V -+ 2 sum|g_k|."""
    from oracle import mlp as M
    gx, gy, gz = 0.004, -0.003, 0.0015
    nx, ny, nz = 20, 18, 16
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    V = (0.3 + gx * x + gy * y + gz * z).astype(np.float32)
    prm = np.zeros((3, 12), np.float32)
    prm[0, :3] = (9.2, 8.7, 7.9)        # interior seed (9, 9, 8)
    prm[1, :3] = (0.2, 1.1, 15.4)       # border seed (0, 1, 15): clipped windows
    prm[2, :3] = (10.0, 10.0, 10.0)
    prm[:, 3:6] = (0.1, -0.2, 0.3)
    prm[:, 10] = 0.5
    gbar = 0.01
    F = M.features(V, prm, 1, gbar)
    g2 = gx * gx + gy * gy + gz * gz
    c = np.array([9, 9, 8])
    Vc = float(np.float32(0.3 + gx * 9 + gy * 9 + gz * 8))
    np.testing.assert_allclose(F[0, 0:2], 0.0, atol=1e-8)   # float32 field: differences exact to ~1e-7
    np.testing.assert_allclose(F[0, 2], np.log1p(343 * g2 / (343 * gbar * gbar)), rtol=1e-5)
    np.testing.assert_allclose(F[0, 3], np.sqrt(g2) / gbar, rtol=1e-5)
    np.testing.assert_allclose(F[0, 4], Vc, atol=1e-6)
    np.testing.assert_allclose(F[0, 5], np.sqrt(2.0 * g2), rtol=1e-4)
    span = 2 * (abs(gx) + abs(gy) + abs(gz))
    np.testing.assert_allclose(F[0, 6:8], [Vc - span, Vc + span], atol=1e-6)
    np.testing.assert_allclose(F[0, 8:11], [0.1, -0.2, 0.3], atol=1e-7)
    assert F[0, 11] == np.float32(0.5) and F[0, 12] == 1.0 and F[1, 12] == 0.0
    assert F[0, 13] == 1.0 and abs(F[0, 14]) < 1e-6 and abs(F[0, 15] - Vc) < 1e-7
    # border seed: the 7^3 window holds 4*5*4 voxels, the gradient is still exact
    cnt = 4 * 5 * 4
    np.testing.assert_allclose(F[1, 2], np.log1p(cnt * g2 / (343 * gbar * gbar)), rtol=1e-5)
    np.testing.assert_allclose(F[1, 3], np.sqrt(g2) / gbar, rtol=1e-5)
    w = V[13:16, 0:4, 0:3].astype(np.float64)   # 5^3 window clipped to 3 x 4 x 3
    np.testing.assert_allclose(F[1, 4:8], [w.mean(), w.std(), w.min(), w.max()], atol=1e-7)
    assert c.sum() == 26


def test_bf16_round_nearest_even():
    """bfloat16 keeps 8 significant bits: spacing 2^-7 on [1, 2).  Halfway
    cases go to the even neighbour, others to the nearest."""
    from oracle import mlp as M
    x = np.array([1.0, 1 + 2.0 ** -8, 1 + 3 * 2.0 ** -8, 1 + 2.0 ** -8 + 2.0 ** -20, -(1 + 2.0 ** -8), 3.0e-3, 0.0],
                 np.float32)
    r = M.bf16_round(x)
    assert r[0] == 1.0 and r[1] == 1.0 and r[2] == 1 + 2.0 ** -6 and r[3] == 1 + 2.0 ** -7 and r[4] == -1.0
    assert r[6] == 0.0 and abs(r[5] - 3.0e-3) <= 3.0e-3 * 2.0 ** -8
    y = np.random.default_rng(3).normal(size=1000).astype(np.float32)
    ry = M.bf16_round(y)
    # nearest: no representable bf16 (8 significant bits) lies closer
    e = np.floor(np.log2(np.abs(y.astype(np.float64))))
    ulp = 2.0 ** (e - 7)
    assert np.all(np.abs(ry - y) <= ulp / 2 + 1e-30)
    assert np.all(np.mod(ry / ulp, 1.0) == 0.0)


def test_kept_submasks_brute_force():
    """Kept sub-bricks of listed bricks, against a voxel-by-voxel scan with
    the oracle's own keep exponent (pred_t), for every brick edge."""
    rng = np.random.default_rng(12)
    dims = (21, 18, 13)
    p = np.zeros((6, 12), np.float32)
    p[:, 0:3] = rng.uniform(2, 16, (6, 3))
    p[:, 3:6] = np.log(rng.uniform(0.6, 2.5, (6, 3)))
    p[:, 6:10] = rng.normal(size=(6, 4))
    p[:, 10] = 1.0
    for B in (4, 8, 16):
        _, keys, gids = O.bin_pairs(p, dims, 3.0, B)
        got = O.kept_submasks(p, dims, keys, gids, 3.0, B)
        T = O.pred_threshold(3.0)
        nbx, nby = -(-dims[0] // B), -(-dims[1] // B)
        for kk, gg, m in zip(keys.tolist(), gids.tolist(), got.tolist()):
            bx, by, bz = kk % nbx, (kk // nbx) % nby, kk // (nbx * nby)
            want = 0
            for z in range(bz * B, min(bz * B + B, dims[2])):
                for y in range(by * B, min(by * B + B, dims[1])):
                    for x in range(bx * B, min(bx * B + B, dims[0])):
                        if O.pred_t(p[gg], x, y, z) > T:
                            want |= 1 << ((y - by * B) // (B // 2) + 2 * ((z - bz * B) // (B // 4)))
            assert m == want, (B, kk, gg)
        assert got.any() and not got.all()


# ---------------------------------------------------------------------------
# Stratified-sample refinement (Sec. III-F, Table III)
# ---------------------------------------------------------------------------
def _sample_field(n=20, seed=3):
    rng = np.random.default_rng(seed)
    V = rng.uniform(0, 1, (n, n - 2, n - 4)).astype(np.float32) ** 2
    V[:, :3, :] = 0.0      # an empty region
    return V


def test_sample_classes_and_split():
    V = _sample_field()
    hi, mid = O.sample_classes(V)
    flat = V.reshape(-1)
    np.testing.assert_array_equal(hi, np.nonzero(flat > np.float32(0.4))[0])
    np.testing.assert_array_equal(mid, np.nonzero((flat > np.float32(0.02)) & (flat <= np.float32(0.4)))[0])
    np.testing.assert_array_equal(O.sample_split(3072), [1075, 1229, 768])   # Table III: 35 / 40 / 25 %
    for S in (1, 7, 100, 4096):
        sp = O.sample_split(S)
        assert sp.sum() == S and sp[0] == int(np.floor(0.35 * S + 0.5)) and sp[1] == int(np.floor(0.4 * S + 0.5))


def test_draw_samples_classes_jitter_targets():
    from scipy.ndimage import map_coordinates
    V = _sample_field()
    nz, ny, nx = V.shape
    hi, mid = O.sample_classes(V)
    S = 3072
    pts, vals, vox = O.draw_samples(V, S, seed=11, it=5)
    nh, nm, _ = O.sample_split(S)
    assert np.isin(vox[:nh], hi).all() and np.isin(vox[nh:nh + nm], mid).all()
    assert ((vox >= 0) & (vox < V.size)).all()
    c = np.stack([vox % nx, (vox // nx) % ny, vox // (nx * ny)], 1).astype(np.float64)
    assert np.all(np.abs(pts.astype(np.float64) - c) <= 0.5)
    # targets: trilinear interpolation, edge-clamped (scipy, order 1, nearest)
    q = np.clip(pts.astype(np.float64), 0, np.array([nx - 1, ny - 1, nz - 1]))
    ref = map_coordinates(V.astype(np.float64), [q[:, 2], q[:, 1], q[:, 0]], order=1, mode="nearest")
    np.testing.assert_allclose(vals, ref, rtol=1e-6, atol=1e-7)
    # deterministic per (seed, iteration), different across iterations
    p2, v2, x2 = O.draw_samples(V, S, seed=11, it=5)
    assert np.array_equal(pts, p2) and np.array_equal(vox, x2)
    p3, _, _ = O.draw_samples(V, S, seed=11, it=6)
    assert not np.array_equal(pts, p3)
    # a class without voxels hands its samples to the uniform draw
    Z = np.full_like(V, 0.1)
    _, _, xz = O.draw_samples(Z, S, seed=1, it=0)
    assert len(O.sample_classes(Z)[0]) == 0 and len(np.unique(xz[:nh])) > nh // 2


def test_draw_samples_uniform_within_class():
    """Chi-square: the high-class draws spread evenly over its voxels."""
    from scipy.stats import chisquare
    V = np.zeros((6, 6, 6), np.float32)
    V[1:5, 2:4, 1:4] = 0.9            # 24 high voxels
    hi, _ = O.sample_classes(V)
    counts = np.zeros(V.size, np.int64)
    nh = O.sample_split(1024)[0]
    for it in range(40):
        _, _, vox = O.draw_samples(V, 1024, seed=5, it=it)
        np.add.at(counts, vox[:nh], 1)
    assert counts[hi].sum() == 40 * nh
    assert chisquare(counts[hi]).pvalue > 1e-3


def test_sample_eval_at_voxel_centres_equals_voxel_eval():
    rng = np.random.default_rng(21)
    dims = (14, 12, 10)
    p = np.zeros((25, 12))
    p[:, 0:3] = rng.uniform(0, 1, (25, 3)) * (np.array(dims) - 1)
    p[:, 3:6] = np.log(rng.uniform(0.7, 2.2, (25, 3)))
    p[:, 6:10] = rng.normal(size=(25, 4))
    p[:, 10] = rng.uniform(0.1, 1.0, 25)
    p[:, 11] = rng.uniform(-2, 1, 25)
    p = p.astype(np.float32).astype(np.float64)
    _, _, vt = O.eval_region(p, dims)
    idx = rng.integers(0, np.prod(dims), 300)
    nx, ny = dims[0], dims[1]
    pts = np.stack([idx % nx, (idx // nx) % ny, idx // (nx * ny)], 1).astype(np.float32)
    _, _, vs = O.sample_loss_grad(p, pts, np.zeros(300, np.float32), want_grad=False)
    np.testing.assert_allclose(vs, vt.reshape(-1)[idx], rtol=1e-12, atol=1e-14)


def test_sample_eval_single_gaussian_closed_form():
    """One Gaussian at continuous points: Vt = a where w G >= rho0, a w G / rho0
    below, 0 outside the truncation (m computed here from R, s)."""
    q = np.array([0.9, 0.2, -0.3, 0.25])
    p = np.array([[5.3, 6.1, 4.7, np.log(1.5), np.log(0.8), np.log(2.0), *q, 0.7, 0.4]])
    p = p.astype(np.float32).astype(np.float64)
    w = 1 / (1 + np.exp(-p[0, 11]))
    qn = p[0, 6:10] / np.linalg.norm(p[0, 6:10])
    a_, b_, c_, d_ = qn
    R = np.array([[1 - 2 * (c_ * c_ + d_ * d_), 2 * (b_ * c_ - a_ * d_), 2 * (b_ * d_ + a_ * c_)],
                  [2 * (b_ * c_ + a_ * d_), 1 - 2 * (b_ * b_ + d_ * d_), 2 * (c_ * d_ - a_ * b_)],
                  [2 * (b_ * d_ - a_ * c_), 2 * (c_ * d_ + a_ * b_), 1 - 2 * (b_ * b_ + c_ * c_)]])
    C = R @ np.diag(np.exp(-2 * p[0, 3:6])) @ R.T
    pts = (p[0, :3] + np.random.default_rng(2).normal(0, 2.5, (200, 3))).astype(np.float32)
    _, _, vt = O.sample_loss_grad(p, pts, np.zeros(200, np.float32), want_grad=False)
    d = pts.astype(np.float64) - p[0, :3]
    m = np.einsum("si,ij,sj->s", d, C, d)
    G = np.exp(-0.5 * m)
    away = np.abs(m - 9.0) > 1e-3          # the float32 keep test decides at the surface itself
    want = np.where(m < 9.0, np.where(w * G >= 0.05, p[0, 10], p[0, 10] * w * G / 0.05), 0.0)
    np.testing.assert_allclose(vt[away], want[away], rtol=1e-12, atol=1e-15)
    assert (m < 9).any() and (m > 9).any() and (w * G[m < 9] < 0.05).any()


def test_sample_loss_gradient_central_differences():
    """k = 20: no pair near the truncation surface, the loss is smooth."""
    rng = np.random.default_rng(31)
    n, S = 6, 120
    p = np.zeros((n, 12))
    p[:, 0:3] = rng.uniform(3, 7, (n, 3))
    p[:, 3:6] = np.log(rng.uniform(0.8, 1.8, (n, 3)))
    p[:, 6:10] = rng.normal(size=(n, 4))
    p[:, 10] = rng.uniform(0.2, 1.0, n)
    p[:, 11] = rng.uniform(-1, 1, n)
    pts = rng.uniform(2, 8, (S, 3)).astype(np.float32)
    vals = rng.uniform(0.03, 0.9, S).astype(np.float32)
    L, g, _ = O.sample_loss_grad(p, pts, vals, k=20.0)
    h = 3e-5
    for i in range(n):
        for j in range(12):
            pp, pm = p.copy(), p.copy()
            pp[i, j] += h
            pm[i, j] -= h
            fd = (O.sample_loss_grad(pp, pts, vals, k=20.0, want_grad=False)[0]
                  - O.sample_loss_grad(pm, pts, vals, k=20.0, want_grad=False)[0]) / (2 * h)
            assert abs(fd - g[i, j]) <= 1e-5 * max(abs(fd), 1e-4), (i, j, fd, g[i, j])


# ---------------------------------------------------------------------------
# Pre-encoding structure statistics (Sec. V-F, Table VI)
# ---------------------------------------------------------------------------
def test_structure_stats_linear_ramp_closed_form():
    """V = 0.1 + a x on nx x ny x nz: every voxel occupied, |grad V| = a at
    every voxel (one-sided differences are exact on a ramp), so the top 10 %
    hold exactly ceil(0.1 M) / M of the mass; S(l) = a^2 l^2 along x and 0
    along y, z, so S(1) / S(16) = 1 / 256."""
    nz, ny, nx = 20, 24, 40              # every axis longer than the lag 16
    a = np.float32(0.02)
    x = np.arange(nx, dtype=np.float32)
    V = np.broadcast_to(np.float32(0.1) + a * x, (nz, ny, nx)).astype(np.float32)
    st = O.structure_stats(V)
    M = V.size
    assert st["occupancy"] == 1.0
    assert abs(st["grad_top10"] - np.ceil(0.1 * M) / M) < 1e-6     # float32 ramp values
    dx = np.diff(V[0, 0, :].astype(np.float64))
    s1 = float(np.mean(dx ** 2)) / 3.0
    np.testing.assert_allclose(st["S1"], s1, rtol=1e-12)
    np.testing.assert_allclose(st["S1_over_S16"], 1 / 256, rtol=1e-5)


def test_structure_stats_step_and_empty_fields():
    """A single plane jump: the gradient mass sits on the two planes beside
    the jump; a constant field has no gradient mass and no structure."""
    V = np.zeros((20, 20, 20), np.float32) + 0.5
    V[:, :, 10:] = 0.9
    st = O.structure_stats(V)
    # central differences: |grad| = 0.2 on the planes x = 9, 10, zero elsewhere:
    # 800 voxels hold all of the mass, the top 10 % (800 voxels) hold all of it
    assert abs(st["grad_top10"] - 1.0) < 1e-12
    # at lag l, min(l, 20 - l) of the 20 - l pairs of each x row cross the
    # jump (y, z rows never do): S(l) = min(l, 20 - l) / (20 - l) d^2 / 3 with
    # d = 0.9 - 0.5 in float32; at l = 16 all 4 pairs cross
    d2 = float(np.float32(0.9) - np.float32(0.5)) ** 2
    np.testing.assert_allclose(st["S1"], d2 / 19 / 3, rtol=1e-12)
    np.testing.assert_allclose(st["S16"], d2 / 3, rtol=1e-12)
    np.testing.assert_allclose(st["S1_over_S16"], 1 / 19, rtol=1e-12)
    C = np.full((8, 8, 8), 0.3, np.float32)
    sc = O.structure_stats(C)
    assert sc["grad_top10"] == 0.0 and sc["S1"] == 0.0 and sc["S1_over_S16"] == 0.0
    Z = np.zeros((8, 8, 8), np.float32)
    assert O.structure_stats(Z)["occupancy"] == 0.0


def test_structure_function_kolmogorov_scaling():
    """A random field with shell spectrum E(k) ~ k^-5/3 has S(l) ~ l^(2/3) in
    the inertial range, so S(1)/S(16) lies near 16^(-2/3) = 0.157 (the range
    of the paper's Table VI)."""
    from paper_2608_14112_b300 import inputs
    V = inputs.grf(96, seed=3)
    r = O.structure_stats(V)["S1_over_S16"]
    assert 0.08 < r < 0.3


# --------------------------------------------------------------------------
# Mixture-field ray marching (Sec. III-A: transfer function applied to the
# value of Eq. 3 at ray samples, composited front to back)
# --------------------------------------------------------------------------
def _axis_camera(cx, cy, z0, th, W=5, H=5):
    """Camera at (cx, cy, z0) looking along +z; the central pixel of an odd
    image has the exact direction (0, 0, 1)."""
    f = lambda *v: np.array(v, np.float32)
    return (f(cx, cy, z0), f(1, 0, 0), f(0, 1, 0), f(0, 0, 1), th)


def test_render_constant_transfer_function_closed_form():
    """With a constant table every sample has the same opacity: the central
    ray enters the 13 x 15 x 20 box at z = -0.5 and leaves at 19.5, so at
    spacing 0.5 it takes 40 samples, and the pixel is c (1 - 0.9^20) +
    bg 0.9^20 (opacity 0.1 per voxel).  A ray that misses shows the
    background; early termination at 0.5 stops after the 14th sample."""
    dims = (20, 15, 13)
    rng = np.random.default_rng(3)
    prm = np.zeros((3, 12))
    prm[:, :3] = rng.uniform(2, 10, (3, 3))
    prm[:, 6] = 1.0
    tf = np.tile(np.array([[0.2, 0.5, 0.9, 0.1]], np.float32), (4, 1))
    cam = _axis_camera(6.0, 7.0, -10.0, float(np.float32(np.tan(np.radians(60)))))
    bg = (0.3, 0.1, 0.05)
    img, _ = O.render(prm, dims, cam, 5, 5, tf, dict(step=0.5, ref_step=1.0, background=bg))
    c = tf[0].astype(np.float64)                     # the table and background are float32
    bg64 = np.array(bg, np.float32).astype(np.float64)
    a = 1.0 - (1.0 - c[3]) ** 20
    np.testing.assert_allclose(img[2, 2, :3], c[:3] * a + bg64 * (1 - a), rtol=1e-12)
    assert img[2, 2, 3] == pytest.approx(a, rel=1e-12)
    hit, d, t0, t1 = O.ray_setup(cam, 5, 5, 2, 2, dims)
    assert hit and tuple(d) == (0.0, 0.0, 1.0) and (t0, t1) == (9.5, 29.5)
    assert not O.ray_setup(cam, 5, 5, 0, 0, dims)[0]
    np.testing.assert_allclose(img[0, 0], [*bg64, 0.0], atol=0)
    img_t, _ = O.render(prm, dims, cam, 5, 5, tf, dict(step=0.5, ref_step=1.0, term=0.5))
    assert img_t[2, 2, 3] == pytest.approx(1.0 - (1.0 - c[3]) ** 7, rel=1e-12)


def _axis_gaussian(a=0.8, w_logit=0.0, mu=(6.0, 7.0, 9.0)):
    p = np.zeros((1, 12))
    p[0, :3] = mu
    p[0, 3:6] = np.float32(np.log(2.0))
    p[0, 6] = 1.0
    p[0, 10] = a
    p[0, 11] = w_logit
    return p


def _axis_expect(prm, normalized, alpha0, shade=None, rho0=0.05, step=0.5, nz=20):
    """Front-to-back sum along the z axis through the Gaussian's centre,
    written from the definitions: samples at z = -0.5 + (k + 1/2) step,
    kept within 3 sigma, Vt = w a G / max(w G, rho0) or w a G, a grayscale
    table (colour = value), opacity alpha0 per voxel."""
    s = float(np.exp(np.float64(np.float32(np.log(2.0)))))   # the record holds float32(ln 2)
    a, w = prm[0, 10], 1.0 / (1.0 + np.exp(-prm[0, 11]))
    mz = prm[0, 2]
    a_s = 1.0 - (1.0 - float(np.float32(alpha0))) ** step
    Tr, C = 1.0, 0.0
    for k in range(int(np.ceil(nz / step - 0.5))):
        z = -0.5 + (k + 0.5) * step
        G = np.exp(-0.5 * (z - mz) ** 2 / s ** 2) if abs(z - mz) < 3 * s else 0.0
        v = w * a * G / max(w * G, rho0) if normalized else w * a * G
        c = v
        if shade is not None:
            ka, kd, ks = shade
            c = c * (ka + kd) + ks if G > 0 else c * ka   # |n . l| = 1 on the axis, 0 where grad = 0
        C += Tr * a_s * c
        Tr *= 1.0 - a_s
    return C, 1.0 - Tr


@pytest.mark.parametrize("normalized", [True, False])
def test_render_axis_gaussian_closed_form(normalized):
    dims = (20, 15, 13)
    prm = _axis_gaussian()
    tf = np.array([[0, 0, 0, 0.2], [1, 1, 1, 0.2]], np.float32)
    cam = _axis_camera(6.0, 7.0, -10.0, 0.5)
    img, kept = O.render(prm, dims, cam, 5, 5, tf, dict(step=0.5), normalized=normalized)
    C, A = _axis_expect(prm, normalized, 0.2)
    np.testing.assert_allclose(img[2, 2, :3], [C, C, C], rtol=1e-12, atol=1e-15)
    assert img[2, 2, 3] == pytest.approx(A, rel=1e-12)


def test_render_axis_shading_closed_form():
    """Plain sum, headlight shading: on the axis grad Vt is parallel to the
    ray, so |n . l| = 1 wherever the Gaussian is kept (gfloor below every
    gradient there) and the shaded colour is c (ka + kd) + ks."""
    dims = (20, 15, 13)
    prm = _axis_gaussian()
    tf = np.array([[0, 0, 0, 0.2], [1, 1, 1, 0.2]], np.float32)
    cam = _axis_camera(6.0, 7.0, -10.0, 0.5)
    opts = dict(step=0.5, shade=True, ka=0.25, kd=0.6, ks=0.15, shininess=8.0, gfloor=1e-12)
    img, _ = O.render(prm, dims, cam, 5, 5, tf, opts, normalized=False)
    C, _ = _axis_expect(prm, False, 0.2, shade=tuple(float(np.float32(x)) for x in (0.25, 0.6, 0.15)))
    np.testing.assert_allclose(img[2, 2, :3], [C, C, C], rtol=1e-12)


@pytest.mark.parametrize("w_logit,normalized", [(3.0, True), (-7.0, True), (0.0, False)])
def test_field_gradient_central_differences(w_logit, normalized):
    """grad Vt against central differences of Vt at float32 points (steps of
    2^-10 are exact there); k = 20 so truncation does not enter.  w_logit 3
    keeps the denominator above rho0 near the centres (quotient rule), -7
    keeps it below (grad N / rho0)."""
    rng = np.random.default_rng(11)
    n = 12
    prm = np.zeros((n, 12))
    prm[:, :3] = rng.uniform(6, 10, (n, 3))
    prm[:, 3:6] = np.log(rng.uniform(1.0, 2.5, (n, 3)))
    prm[:, 6:10] = rng.normal(size=(n, 4))
    prm[:, 10] = rng.uniform(0.1, 1.0, n)
    prm[:, 11] = w_logit
    h = 2.0 ** -10
    for _ in range(6):
        p = np.round(rng.uniform(6.5, 9.5, 3) * 16) / 16
        v, g, _ = O.field_at(prm, p, k=20.0, normalized=normalized)
        fd = np.zeros(3)
        for a in range(3):
            e = np.zeros(3)
            e[a] = h
            fd[a] = (O.field_at(prm, p + e, k=20.0, normalized=normalized)[0]
                     - O.field_at(prm, p - e, k=20.0, normalized=normalized)[0]) / (2 * h)
        np.testing.assert_allclose(g, fd, rtol=1e-4, atol=1e-7 * max(1.0, abs(v)))


def test_render_candidate_index_drops_nothing():
    """The renderer's candidate index only skips Gaussians that cannot be
    kept: marching the same rays with a brute-force field (every Gaussian)
    and compositing in numpy gives the same pixels and kept-pair count."""
    from paper_2608_14112_b300 import inputs
    dims = (40, 37, 45)
    rng = np.random.default_rng(21)
    n = 60
    prm = np.zeros((n, 12))
    prm[:, :3] = rng.uniform(-2, 1, (n, 3)) + rng.uniform(0, 1, (n, 3)) * np.array([44, 36, 39])
    prm[:, 3:6] = np.log(rng.uniform(1.0, 6.0, (n, 3)))
    prm[:, 6:10] = rng.normal(size=(n, 4))
    prm[:, 10] = rng.uniform(0.1, 1.0, n)
    prm[:, 11] = rng.uniform(-3, 2, n)
    cam = inputs.orbit_camera(dims, 35.0, 25.0, 1.4, 45.0)
    tf = inputs.transfer_function(16, seed=2)
    W, H, step = 7, 5, 0.75
    img, kept = O.render(prm, dims, cam, W, H, tf, dict(step=step))
    tot = 0
    for j in range(H):
        for i in range(W):
            hit, d, t0, t1 = O.ray_setup(cam, W, H, i, j, dims)
            Tr, C = 1.0, np.zeros(3)
            if hit:
                k = 0
                while True:
                    t = np.float32(t0) + (np.float32(k) + np.float32(0.5)) * np.float32(step)
                    if not t < np.float32(t1):
                        break
                    p = cam[0] + t * d                     # float32, one rounding per operation
                    v, _, kp = O.field_at(prm, p)
                    tot += kp
                    u = min(max(v, 0.0), 1.0) * 15
                    i0 = min(int(np.floor(u)), 14)
                    c = tf[i0].astype(np.float64) * (1 - (u - i0)) + tf[i0 + 1].astype(np.float64) * (u - i0)
                    a_s = 1.0 - (1.0 - min(max(c[3], 0.0), 1.0)) ** (step / 1.0)
                    C += Tr * a_s * c[:3]
                    Tr *= 1.0 - a_s
                    k += 1
            np.testing.assert_allclose(img[j, i], [*C, 1.0 - Tr], rtol=1e-12, atol=1e-14)
    assert tot == kept and kept > 0


# --------------------------------------------------------------------------
# Full objective (Sec. III-F): value term plus the five regularisers
# --------------------------------------------------------------------------
def _one_gaussian(mu=(5.0, 6.0, 7.0), logs=(0.0, 0.0, 0.0), a=0.7, w_logit=0.0):
    p = np.zeros((1, 12))
    p[0, :3] = mu
    p[0, 3:6] = logs
    p[0, 6] = 1.0
    p[0, 10] = a
    p[0, 11] = w_logit
    return p


def test_regulariser_closed_forms():
    far = np.array([[50.0, 50.0, 50.0]], np.float32)     # a sample no Gaussian reaches
    v0 = np.array([0.0], np.float32)
    # anisotropy: log-scales (0, 0, ln 4) exceed 3:1 on two axis pairs
    p = _one_gaussian(logs=(0.0, 0.0, np.log(4.0)))
    u = np.log(4.0) - np.log(3.0)
    L, g, t = O.sample_objective(p, far, v0, reg=dict(aniso=0.5), k=3.0)
    assert t[4] == pytest.approx(2 * u * u, rel=1e-12) and L == pytest.approx(0.5 * 2 * u * u, rel=1e-12)
    np.testing.assert_allclose(g[0, 3:6], 0.5 * 2 * u * np.array([-1.0, -1.0, 2.0]), rtol=1e-12)
    # scale cap: s = 0.1 below s_lo = 0.3, s = 20 above s_hi = 10
    p = _one_gaussian(logs=(np.log(0.1), 0.0, np.log(20.0)))
    L, g, t = O.sample_objective(p, far, v0, reg=dict(cap=0.25, s_lo=0.3, s_hi=10.0, r_max=1e9), k=3.0)
    assert t[5] == pytest.approx(np.log(3.0) ** 2 + np.log(2.0) ** 2, rel=1e-12)
    np.testing.assert_allclose(g[0, 3:6], 0.25 * 2 * np.array([-np.log(3.0), 0.0, np.log(2.0)]), rtol=1e-12)
    # anchor: the Gaussian sits on voxel (5, 6, 7) of a field, gradient into a only
    field = np.random.default_rng(1).uniform(0, 1, (12, 11, 10)).astype(np.float32)
    p = _one_gaussian(a=0.9)
    L, g, t = O.sample_objective(p, far, v0, field=field, reg=dict(anc=2.0), k=3.0)
    r = 0.9 - float(field[7, 6, 5])
    assert t[3] == pytest.approx(r * r, rel=1e-12)
    assert g[0, 10] == pytest.approx(2.0 * 2 * r, rel=1e-12)
    np.testing.assert_array_equal(g[0, :10], 0.0)
    # density: one occupied sample at the centre has rho = w (and Vt = a)
    p = _one_gaussian(a=0.6, w_logit=0.5)
    w = 1.0 / (1.0 + np.exp(-0.5))
    at = np.array([[5.0, 6.0, 7.0]], np.float32)
    L, g, t = O.sample_objective(p, at, np.array([0.6], np.float32), reg=dict(rho=1.0), k=3.0)
    r0 = 0.6 - float(np.float32(0.6))                      # the target is float32
    assert t[0] == pytest.approx(r0 * r0, rel=1e-9) and t[1] == pytest.approx((w - 1.0) ** 2, rel=1e-12)
    # smoothness: partner one voxel along x from the centre (unit scales)
    pair = np.array([[5.0, 6.0, 7.0], [6.0, 6.0, 7.0]], np.float32)
    L, g, t = O.sample_objective(p, pair, np.array([0.0], np.float32), reg=dict(sm=1.0), smooth=True, k=3.0)
    assert t[2] == pytest.approx((w - w * np.exp(-0.5)) ** 2, rel=1e-12)


def test_objective_gradient_central_differences():
    """Every term but the anchor (whose target V(mu) carries no gradient by
    the reading) against central differences of L; k = 20 so membership
    does not move."""
    from paper_2608_14112_b300 import inputs
    V = inputs.grf((16, 18, 20), seed=4)
    rng = np.random.default_rng(7)
    n = 30
    prm = np.zeros((n, 12))
    prm[:, :3] = rng.uniform(2, 13, (n, 3))
    prm[:, 3:6] = np.log(rng.lognormal(np.log(1.5), 0.6, (n, 3)))
    prm[:, 6:10] = rng.normal(size=(n, 4))
    prm[:, 10] = rng.uniform(0.1, 1.0, n)
    prm[:, 11] = rng.uniform(-2, 2, n)
    pts, vals, _ = O.draw_samples(V, 96, seed=3, it=2)
    both = np.concatenate([pts, O.draw_partners(pts, V.shape, seed=3, it=2, radius=1.0)])
    reg = dict(rho=0.3, sm=0.7, anc=0.0, aniso=0.2, cap=0.4, r_max=2.0, s_lo=0.8, s_hi=2.5)
    L, g, _ = O.sample_objective(prm, both, vals, reg=reg, smooth=True, k=20.0)
    h = 1e-6
    for i, j in [(0, 0), (3, 2), (5, 3), (7, 4), (9, 5), (11, 6), (13, 8), (17, 9), (19, 10), (23, 11), (29, 1)]:
        e = np.zeros_like(prm)
        e[i, j] = h
        fd = (O.sample_objective(prm + e, both, vals, reg=reg, smooth=True, k=20.0, want_grad=False)[0]
              - O.sample_objective(prm - e, both, vals, reg=reg, smooth=True, k=20.0, want_grad=False)[0]) / (2 * h)
        assert g[i, j] == pytest.approx(fd, rel=2e-5, abs=1e-10), (i, j)


def test_smoothness_schedule_and_partners():
    assert O.lambda_sm(1e-2, 1e-4, 100, 0) == pytest.approx(1e-2, rel=1e-15)
    assert O.lambda_sm(1e-2, 1e-4, 100, 50) == pytest.approx(1e-3, rel=1e-12)
    assert O.lambda_sm(1e-2, 1e-4, 100, 400) == pytest.approx(1e-4, rel=1e-15)
    assert O.lambda_sm(1e-2, 1e-4, 0, 50) == 1e-2
    from scipy import stats
    rng = np.random.default_rng(2)
    pts = rng.uniform(3, 17, (4000, 3)).astype(np.float32)
    q = O.draw_partners(pts, (20, 20, 20), seed=9, it=4, radius=1.5)
    d = (q - pts).astype(np.float64)
    assert np.abs(d).max() <= 1.5
    assert stats.kstest(d.ravel(), stats.uniform(loc=-1.5, scale=3.0).cdf).pvalue > 1e-3
    edge = np.zeros((50, 3), np.float32)
    assert O.draw_partners(edge, (20, 20, 20), seed=9, it=4).min() >= 0.0
    assert not np.array_equal(q, O.draw_partners(pts, (20, 20, 20), seed=9, it=5, radius=1.5))


def test_regularised_refinement_reduces_to_plain():
    from paper_2608_14112_b300 import inputs
    V = inputs.blobs(24, seed=4)
    prm, _, _, status = O.allocate(V, 150, seed=1)
    assert status == 0
    zero = dict(rho=0.0, sm0=0.0, sm1=0.0, anneal=0, anc=0.0, aniso=0.0, cap=0.0, r_max=3.0, s_lo=0.3,
                s_hi=1.5, radius=1.0)
    a, la = O.refine_sampled_reg(prm, V, 4, zero, S=256, seed=5)
    b, lb = O.refine_sampled(prm, V, 4, S=256, seed=5)
    np.testing.assert_array_equal(a, b)
    np.testing.assert_array_equal(la, lb)


def test_exp_fixed_against_exp():
    """The float32 exponential of the keep coefficients' scales: within
    2^-22 relative of exp over the range log-scales and weight logits take,
    exact at 0, monotone, and infinite / zero beyond the float range."""
    xs = np.concatenate([np.linspace(-30, 30, 20001), np.random.default_rng(1).uniform(-80, 80, 20000)])
    got = np.array([O.exp_fixed(float(np.float32(x))) for x in xs])
    ref = np.exp(xs.astype(np.float32).astype(np.float64))
    assert np.max(np.abs(got - ref) / ref) < 2.0 ** -22
    assert O.exp_fixed(0.0) == 1.0
    g = np.array([O.exp_fixed(float(x)) for x in np.linspace(-5, 5, 4001).astype(np.float32)])
    assert np.all(np.diff(g) >= 0)
    assert O.exp_fixed(100.0) == float("inf") and O.exp_fixed(-200.0) == 0.0


# ------------------------------------------------------------------------
# S1e shape assembly pinned on closed forms (Sec. III-E, Table I S1e)
# ------------------------------------------------------------------------
def _slope_field(two_slopes: bool, nx=64, ny=24, nz=20):
    """V(x) = 1/4 + x/256, and with two_slopes the slope triples after column
    31.  Every value is a multiple of 2^-8, so every central difference is
    exact in float32: |grad V| = 1/256 on columns 0..30, 2/256 on column 31
    (the kink) and 3/256 on columns 32..63 (one-sided at both borders)."""
    x = np.arange(nx, dtype=np.float64)
    if two_slopes:
        v = np.where(x <= 31, 0.25 + x / 256.0, 0.25 + 31 / 256.0 + 3.0 * (x - 31) / 256.0)
    else:
        v = 0.25 + x / 256.0
    return np.broadcast_to(v.astype(np.float32), (nz, ny, nx)).copy()


@pytest.mark.parametrize("two_slopes", [False, True])
def test_allocation_shape_closed_form_on_ramps(two_slopes):
    """On V = c + alpha x every voxel is occupied, |grad V| = alpha and the
    lower median gbar = alpha, so every seed gets s_t / s_perp = 1 + 1 = 2,
    s_perp = h_g / 2 on both perpendicular axes, and its long axis
    perpendicular to e_x (the structure tensor is rank one along e_x, so the
    tangent -- the smallest eigenvalue's eigenvector -- lies in the y-z
    plane).  With two slopes (31 columns at alpha, the kink column at 2 alpha,
    32 columns at 3 alpha) the lower median of |grad V| is the kink's 2 alpha
    (the upper median would be 3 alpha), so the ratios are 1.5, 2 and 2.5 by
    column.  The covariance Sigma = R diag(s^2) R^T is checked, not the
    record's axis order: e_x must be an eigenvector with eigenvalue s_perp^2
    and the largest eigenvalue must be s_t^2."""
    V = _slope_field(two_slopes)
    nz, ny, nx = V.shape
    N = 2000
    prm, vox, st, status = O.allocate(V, N, seed=11)
    assert status == 0
    alpha = 1.0 / 256.0
    assert st["gbar"] == (2 * alpha if two_slopes else alpha)
    assert st["n_occupied"] == V.size
    Nd = st["n_detail"]
    cap_hi, cap_lo = max(nx, ny, nz) / 16.0, 0.3
    xs = vox % nx
    if two_slopes:
        ratio = np.where(xs <= 30, 1.5, np.where(xs == 31, 2.0, 2.5))
    else:
        ratio = np.full(N, 2.0)
    sig = np.where(np.arange(N) < Nd, 0.5 * st["h_detail"], 0.5 * st["h_coverage"])
    # the design keeps every scale inside the caps, so no clamp hides a mistake
    assert (ratio * sig < cap_hi).all() and (sig > cap_lo).all()
    s = np.exp(prm[:, 3:6])
    rot = Rotation.from_quat(np.concatenate([prm[:, 7:10], prm[:, 6:7]], 1)).as_matrix()
    Sig = np.einsum("nij,nj,nkj->nik", rot, s * s, rot)
    ex = np.array([1.0, 0.0, 0.0])
    np.testing.assert_allclose(Sig @ ex, (sig ** 2)[:, None] * ex[None, :], rtol=0, atol=1e-9 * sig.max() ** 2)
    ev = np.linalg.eigvalsh(Sig)
    np.testing.assert_allclose(ev[:, 2], (ratio * sig) ** 2, rtol=1e-9)
    np.testing.assert_allclose(ev[:, 0], sig ** 2, rtol=1e-9)
    np.testing.assert_allclose(ev[:, 1], sig ** 2, rtol=1e-9)
    # the record's own convention: the first scale is the elongated one
    np.testing.assert_allclose(s[:, 0], ratio * sig, rtol=1e-12)
    np.testing.assert_allclose(s[:, 1], sig, rtol=1e-12)
    np.testing.assert_allclose(s[:, 2], sig, rtol=1e-12)


# ------------------------------------------------------------------------
# Brick lists worked out by hand (the binning rule's own pin)
# ------------------------------------------------------------------------
def _record(mu, scales, q=(1.0, 0.0, 0.0, 0.0), a=0.5, w_logit=0.0):
    r = np.zeros(12, np.float32)
    r[0:3] = mu
    r[3:6] = np.log(np.asarray(scales, np.float64))
    r[6:10] = q
    r[10], r[11] = a, w_logit
    return r


def test_binning_hand_computed_brick_lists():
    """Two Gaussians whose brick lists follow from the rule on paper (k = 3).

    (1) Isotropic, s = 1, mu = (5.5, 5.5, 5.5) on a 16^3 grid, B = 8: the box
    radius is kb + 0.01 with kb = 3 (1.0001 + 1e-5) = 3.00033, so the voxel box
    is [3, 8]^3 and touches all 8 bricks.  The whitened brick test compares
    sum_j max(0, |c_j - mu_j| - 3.51)^2 with K2 = kb^2 1.0001 + 1e-4 = 9.0029,
    c the brick centre (3.5 or 11.5 per axis): one far axis gives 2.49^2 =
    6.2 (kept), two give 12.4 (dropped).  So the list is bricks (0,0,0),
    (1,0,0), (0,1,0), (0,0,1): keys (bz 2 + by) 2 + bx = 0, 1, 2, 4.  The
    dropped bricks indeed hold no kept voxel: their nearest voxel centre, e.g.
    (8, 8, 5), is at squared distance 12.75 > 9.

    (2) Axis-aligned, s = (3, 0.5, 0.5), mu = (20.2, 4, 4) on 40 x 8 x 8:
    cond = 36, kb = 3 (1.0001 + 3.6e-4) = 3.00138; x radius 9.014 gives voxels
    12..29 (bricks 1..3), y and z radius 1.511 give voxels 3..5 (brick 0).
    The whitened test passes all three (x offsets 2.9 and 2.43 against a
    half-extent of 3.51 / 3), so the keys are 1, 2, 3.  Swapped axes would
    give a single brick."""
    p1 = _record((5.5, 5.5, 5.5), (1.0, 1.0, 1.0))
    counts, keys, gids = O.bin_pairs(p1[None, :], (16, 16, 16), 3.0, 8)
    assert counts.tolist() == [4]
    assert keys.tolist() == [0, 1, 2, 4] and gids.tolist() == [0, 0, 0, 0]
    p2 = _record((20.2, 4.0, 4.0), (3.0, 0.5, 0.5))
    counts, keys, gids = O.bin_pairs(p2[None, :], (40, 8, 8), 3.0, 8)
    assert counts.tolist() == [3] and keys.tolist() == [1, 2, 3]
    # both at once: Gaussian-major emission, then the stable sort by brick
    both = np.stack([p1, p1])
    # the mirror image of (1) across the brick boundary x = 7.5 keeps bricks
    # (1,0,0), (0,0,0), (1,1,0), (1,0,1): keys 0, 1, 3, 5
    both[1, 0:3] = (9.5, 5.5, 5.5)
    counts, sk, sg, start, end = O.bin_sorted(both, (16, 16, 16), 3.0, 8)
    assert counts.tolist() == [4, 4]
    assert sk.tolist() == [0, 0, 1, 1, 2, 3, 4, 5]
    assert sg.tolist() == [0, 1, 0, 1, 0, 1, 0, 1]
    assert start.tolist()[:6] == [0, 2, 4, 5, 6, 7] and end.tolist()[:6] == [2, 4, 5, 6, 7, 8]
    # (1) shifted by half a voxel along x: box [3, 9] in x; the far x brick
    # gives (5.5 - 3.51)^2 = 3.96 alone (kept) and 3.96 + 6.2 with a far y or
    # z offset (dropped), so the list of (1) is unchanged
    counts, keys, _ = O.bin_pairs(_record((6.0, 5.5, 5.5), (1.0, 1.0, 1.0))[None, :], (16, 16, 16), 3.0, 8)
    assert keys.tolist() == [0, 1, 2, 4]


# ------------------------------------------------------------------------
# Stage P: normalisation to [0, 1] (Sec. III-B)
# ------------------------------------------------------------------------
def test_normalize_closed_forms():
    """A dyadic ramp V = 3/8 + x/64 (every difference exact) maps to the
    correctly rounded x / (nx - 1): numpy's float32 division is the IEEE
    operation, so equality is bit for bit; the extremes map to exactly 0 and
    1; a constant field maps to 0; a non-finite value is refused; and the
    result does not depend on where the values sit in the grid."""
    nz, ny, nx = 3, 5, 37
    x = np.arange(nx, dtype=np.float32)
    V = np.broadcast_to((np.float32(0.375) + x / np.float32(64.0)).astype(np.float32), (nz, ny, nx)).copy()
    out, (mn, mx) = O.normalize(V)
    assert (mn, mx) == (0.375, 0.375 + 36 / 64.0)
    want = (x / np.float32(nx - 1)).astype(np.float32)
    np.testing.assert_array_equal(out, np.broadcast_to(want, V.shape))
    assert out.min() == 0.0 and out.max() == 1.0
    z, _ = O.normalize(np.full((4, 4, 4), 0.7, np.float32))
    assert (z == 0).all()
    bad = V.copy()
    bad[1, 2, 3] = np.inf
    with pytest.raises(ValueError):
        O.normalize(bad)
    rng = np.random.default_rng(3)
    R = rng.normal(size=(9, 8, 7)).astype(np.float32)
    perm = rng.permutation(R.size)
    a, _ = O.normalize(R)
    b, _ = O.normalize(R.reshape(-1)[perm].reshape(R.shape))
    np.testing.assert_array_equal(a.reshape(-1)[perm], b.reshape(-1))
    # scaling by a power of two and shifting by a dyadic constant change
    # nothing (every rounding is the same)
    c, _ = O.normalize((R * np.float32(4.0)).astype(np.float32))
    np.testing.assert_array_equal(a, c)


def test_list_kept_matches_count_and_keep_rule():
    """The listed kept pairs are the count of the keep rule, each one kept by
    the float32 test and no pair listed twice."""
    rng = np.random.default_rng(8)
    dims = (19, 14, 11)
    p = _rand_prims(rng, 25, dims, s_lo=0.4, s_hi=2.5).astype(np.float32)
    L = O.list_kept(p, dims)
    assert L.shape[0] == O.count_kept(p, dims)
    assert np.unique(L, axis=0).shape[0] == L.shape[0]
    T = O.pred_threshold(3.0)
    for v, i in L[:: max(1, L.shape[0] // 200)]:
        x, y, z = v % dims[0], (v // dims[0]) % dims[1], v // (dims[0] * dims[1])
        assert O.pred_t(p[i], int(x), int(y), int(z)) > T


@pytest.mark.parametrize("B", [4, 8, 16])
def test_binning_covers_kept_pairs_at_large_coordinates_and_anisotropy(B):
    """The float32 cover stays conservative where float32 rounding is
    largest: centres near x = 2^14 - 1 (the evaluation limit, where one ulp is
    2^-10 voxel) and near the low border, anisotropy up to 12:1 in random
    orientations.  Every kept pair's brick must be listed for its Gaussian."""
    rng = np.random.default_rng(400 + B)
    dims = (16384, 24, 20)
    n = 60
    p = np.zeros((n, 12), np.float64)
    p[:, 0] = np.where(np.arange(n) % 2 == 0, rng.uniform(16360, 16383.5, n), rng.uniform(-1.0, 20.0, n))
    p[:, 1] = rng.uniform(-1.0, 24.0, n)
    p[:, 2] = rng.uniform(-1.0, 20.0, n)
    sc = rng.uniform(0.3, 1.0, (n, 3))
    sc[:, 0] *= rng.uniform(1.0, 12.0, n)
    p[:, 3:6] = np.log(sc)
    p[:, 6:10] = rng.normal(size=(n, 4))
    p[:, 10] = 0.5
    p32 = p.astype(np.float32)
    kept = O.list_kept(p32, dims, 3.0)
    assert kept.shape[0] > 1000
    _, keys, gids = O.bin_pairs(p32, dims, 3.0, B)
    listed = set(zip(keys.tolist(), gids.tolist()))
    nbx, nby = (dims[0] + B - 1) // B, (dims[1] + B - 1) // B
    v, i = kept[:, 0], kept[:, 1]
    x, y, z = v % dims[0], (v // dims[0]) % dims[1], v // (dims[0] * dims[1])
    bk = (z // B * nby + y // B) * nbx + x // B
    missing = [(int(a), int(b)) for a, b in zip(bk, i) if (int(a), int(b)) not in listed]
    assert not missing, missing[:5]
