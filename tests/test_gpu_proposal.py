"""Learned proposal kernels against the FP64 reference in oracle/mlp.py:
features, MLP forward (BF16 weights, FP32 accumulation), the MSE gradient,
Adam with the BF16 refresh, the correction of the records, the end-to-end
gradient through the encoder's loss; then the trained proposal against the
plain analytic allocation on held-out fields.

Tolerances: features relative 1e-5 (FP64 on both sides, float32 outputs);
forward relative L2 1e-5 (FP32 sums of 64 products, float erf against
scipy's); gradients relative L2 1e-4 (float atomics across CTAs).
"""
import numpy as np
import pytest
import torch

from oracle import mlp as M
from paper_2608_14112_b300 import gve, inputs, proposal

pytestmark = pytest.mark.gpu

SHAPE = (40, 36, 28)


def rel_l2(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.fixture(scope="module")
def alloc():
    V = torch.from_numpy(inputs.grf(SHAPE, seed=71)).cuda()
    P, info = gve.gve_allocate(V, 700, seed=5)
    return V, P, info


def _model(seed=1, rows=None):
    """A proposal with every layer random (last layer included) and a
    non-trivial input normalisation."""
    m = proposal.Proposal("cuda", seed=seed)
    rng = np.random.default_rng(seed)
    flat = m.model[:M.P].cpu().numpy()
    flat[9408:9668] = rng.normal(0.0, 0.05, 260)
    flat[M.P - 4:] = rng.normal(0.0, 0.05, 4)
    for name, lo, n in (("b1", 1024, 64), ("b2", 5184, 64), ("b3", 9344, 64)):
        flat[lo:lo + n] = rng.normal(0.0, 0.1, n)
    m.model[:M.P] = torch.from_numpy(flat).cuda()
    m.model[3 * M.P:3 * M.P + 16] = torch.from_numpy(rng.normal(0, 0.2, 16).astype(np.float32)).cuda()
    m.model[3 * M.P + 16:3 * M.P + 32] = torch.from_numpy(rng.uniform(0.5, 2.0, 16).astype(np.float32)).cuda()
    m._quantise()
    return m


def _ref_params(m):
    host = m.model.cpu().numpy()
    return (M.bf16_round(host[:M.P]), host[3 * M.P:3 * M.P + 16].astype(np.float64),
            host[3 * M.P + 16:3 * M.P + 32].astype(np.float64))


def test_features_match_oracle(alloc):
    V, P, info = alloc
    F = proposal.features(V, P, info["n_detail"], info["gbar"])
    ref = M.features(V.cpu().numpy(), P.cpu().numpy(), info["n_detail"], info["gbar"])
    assert F.shape == (P.shape[0], 16)
    np.testing.assert_allclose(F.cpu().numpy(), ref, rtol=1e-5, atol=1e-6)


def test_quantise_is_round_to_nearest_even():
    m = _model(seed=2)
    host = m.model.cpu().numpy()
    np.testing.assert_array_equal(M.bf16_params(host), M.bf16_round(host[:M.P]))


@pytest.mark.parametrize("rows", [1, 127, 1000, 4096 + 37])
def test_mlp_forward_matches_oracle(rows):
    m = _model(seed=3)
    X = torch.from_numpy(np.random.default_rng(rows).normal(size=(rows, 16)).astype(np.float32)).cuda()
    Y = m.forward(X).cpu().numpy()
    W, mean, istd = _ref_params(m)
    ref, _ = M.forward(W, mean, istd, X.cpu().numpy())
    assert rel_l2(Y, ref) <= 1e-5
    np.testing.assert_allclose(Y, ref, rtol=1e-4, atol=1e-6)


@pytest.mark.parametrize("rows", [128, 1000 + 13])
def test_mlp_grad_matches_oracle(rows):
    m = _model(seed=4)
    rng = np.random.default_rng(10 + rows)
    X = torch.from_numpy(rng.normal(size=(rows, 16)).astype(np.float32)).cuda()
    T = torch.from_numpy(rng.normal(0, 0.3, size=(rows, 4)).astype(np.float32)).cuda()
    dP, loss = m.grad(X, T)
    W, mean, istd = _ref_params(m)
    ref_loss, ref = M.loss_grad(W, mean, istd, X.cpu().numpy(), T.cpu().numpy())
    assert rel_l2(dP.cpu().numpy(), ref) <= 1e-4
    assert abs(float(loss.item()) - ref_loss) <= 1e-5 * ref_loss


def test_mlp_adam_step_matches_definition():
    m = _model(seed=5)
    rng = np.random.default_rng(6)
    mom = rng.normal(0, 1e-3, M.P).astype(np.float32)
    vel = rng.uniform(0, 1e-5, M.P).astype(np.float32)
    m.model[M.P:2 * M.P] = torch.from_numpy(mom).cuda()
    m.model[2 * M.P:3 * M.P] = torch.from_numpy(vel).cuda()
    g = rng.normal(0, 1e-3, M.P).astype(np.float32)
    w0 = m.model[:M.P].cpu().numpy().astype(np.float64)
    m.step = 2
    lr, b1, b2, eps = 1e-3, 0.9, 0.999, 1e-8
    m.adam(torch.from_numpy(g).cuda(), lr, b1, b2, eps)
    mm = b1 * mom + (1 - b1) * g.astype(np.float64)
    vv = b2 * vel + (1 - b2) * g.astype(np.float64) ** 2
    w = w0 - lr * (mm / (1 - b1 ** 3)) / (np.sqrt(vv / (1 - b2 ** 3)) + eps)
    host = m.model.cpu().numpy()
    # float32 rounding of terms of size ~1e-3 (first moment), ~1e-5 (second)
    np.testing.assert_allclose(host[M.P:2 * M.P], mm, rtol=1e-5, atol=1e-9)
    np.testing.assert_allclose(host[2 * M.P:3 * M.P], vv, rtol=1e-5, atol=1e-11)
    np.testing.assert_allclose(host[:M.P], w, rtol=1e-6, atol=lr * 1e-4)
    np.testing.assert_array_equal(M.bf16_params(host), M.bf16_round(host[:M.P]))


def test_apply_and_end_to_end_gradient_match_oracle(alloc):
    V, P, info = alloc
    m = _model(seed=7)
    F = proposal.features(V, P, info["n_detail"], info["gbar"])
    W, mean, istd = _ref_params(m)
    Fh = F.cpu().numpy()
    Yref, _ = M.forward(W, mean, istd, Fh)
    Pc = P.clone()
    m.apply(F, Pc, V.shape)
    dims = (SHAPE[0], SHAPE[1], SHAPE[2])
    Pref = M.apply(P.cpu().numpy(), Yref, dims)
    np.testing.assert_allclose(Pc.cpu().numpy(), Pref, rtol=0, atol=2e-5)
    G = torch.from_numpy(np.random.default_rng(8).normal(size=(P.shape[0], 12)).astype(np.float32)).cuda()
    dP = m.backward(F, Pc, G, V.shape)
    ref = M.backward(W, mean, istd, Fh, M.upstream(Pref, G.cpu().numpy(), Yref, dims))
    assert rel_l2(dP.cpu().numpy(), ref) <= 1e-4
    # accumulate = adds to what dP holds
    dP2 = m.backward(F, Pc, G, V.shape, dP.clone(), accumulate=True)
    assert rel_l2(dP2.cpu().numpy(), 2 * ref) <= 1e-4


def test_untrained_proposal_is_identity(alloc):
    V, P, info = alloc
    m = proposal.Proposal("cuda", seed=0)
    F = proposal.features(V, P, info["n_detail"], info["gbar"])
    m.set_normalisation(F)
    m._quantise()
    Pc = P.clone()
    m.apply(F, Pc, V.shape)
    assert torch.equal(Pc, P)


def test_proposal_invalid_arguments(alloc):
    V, P, info = alloc
    m = proposal.Proposal("cuda", seed=0)
    with pytest.raises(gve.GveError):
        proposal.features(V, P, P.shape[0] + 1, info["gbar"])
    F = proposal.features(V, P, info["n_detail"], info["gbar"])
    with pytest.raises(gve.GveError):
        m.backward(F[:0], P[:0], P[:0], V.shape)


def test_trained_proposal_beats_plain_allocation():
    """End-to-end training on 12 seeded fields raises the PSNR of the
    allocation on held-out fields, and the head start survives the first
    refinement iterations."""
    n_tr, n_te = 96, 96
    tr = [inputs.grf(n_tr, seed=s, device="cuda") for s in range(300, 312)]
    te = [inputs.grf(n_te, seed=s, device="cuda") for s in (400, 401)]
    btr, bte = n_tr ** 3 // 671, n_te ** 3 // 671
    m = proposal.Proposal("cuda", seed=0)
    log = m.train_e2e(tr, proposal.allocations(tr, btr), epochs=30, lr=3e-3, fields_per_step=2)
    assert log.losses[-1] < log.losses[0]
    for V in te:
        _, t_plain, _ = proposal.encode(V, bte, 10, None)
        _, t_prop, _ = proposal.encode(V, bte, 10, m)
        gain = 10 * torch.log10(t_plain / t_prop).cpu().numpy()
        assert gain[0] > 0.1, gain
        assert gain[5] > 0.0, gain


def test_pairs_proposal_step_is_judged_by_refinement():
    """The allocation -> refined pairs trainer and its refinement-judged step:
    the chosen step's mean PSNR after refinement is the best of the
    candidates, zero (the plain allocation) among them, and the folded
    network predicts that multiple of its unscaled corrections."""
    tr = [inputs.grf(96, seed=s, device="cuda") for s in range(300, 308)]
    b = 96 ** 3 // 671
    X, T = proposal.make_pairs(tr, b, iters=50, seed=0)
    Ts, sc = proposal.scale_targets(T)
    m = proposal.Proposal("cuda", seed=0)
    m.train(X, Ts, epochs=10, lr=1e-3, tscale=sc)
    y0 = m.forward(X[:512])
    assert y0.abs().max().item() > 0
    scores = m.calibrate(tr[:4], b, iters=30)
    assert set(scores) == {float(g) for g in proposal.CAL_GAMMAS}
    assert scores[m.gamma] == max(scores.values()) and scores[m.gamma] >= scores[0.0]
    y1 = m.forward(X[:512])
    torch.testing.assert_close(y1, m.gamma * y0, rtol=1e-2, atol=1e-5)


def test_standardise_matches_column_moments():
    """gve_mlp_standardise: column means and sample spreads (ddof 1) of the
    training features, inverse spread 0 for a feature whose spread is at
    most 1e-3 (1 + |mean|)."""
    rng = np.random.default_rng(17)
    X = rng.normal(size=(5003, 16)) * rng.uniform(0.1, 3.0, 16) + rng.normal(0, 2, 16)
    X[:, 12] = 0.0                       # constant: dead
    X[:, 13] = 5.0 + 1e-5 * rng.normal(size=5003)   # negligible spread: dead
    X = X.astype(np.float32)
    m = proposal.Proposal("cuda", seed=0)
    m.set_normalisation(torch.from_numpy(X).cuda())
    host = m.model.cpu().numpy()
    mean, istd = host[3 * M.P:3 * M.P + 16], host[3 * M.P + 16:3 * M.P + 32]
    X64 = X.astype(np.float64)
    mu, sd = X64.mean(0), X64.std(0, ddof=1)
    live = sd > 1e-3 * (1 + np.abs(mu))
    assert live.tolist().count(False) == 2 and not live[12] and not live[13]
    np.testing.assert_allclose(mean, mu.astype(np.float32), rtol=1e-6, atol=1e-7)
    np.testing.assert_allclose(istd[live], (1.0 / sd[live]).astype(np.float32), rtol=1e-6)
    assert (istd[~live] == 0).all()


def test_targets_scale_and_fold():
    """Targets refined - allocated (exact float32 differences), their
    division by the column spreads (numpy float32 division of the same
    spreads), and the fold of the spreads into the last layer (exact float32
    products, BF16 copies refreshed)."""
    rng = np.random.default_rng(18)
    n = 3001
    p0 = rng.normal(size=(n, 12)).astype(np.float32)
    p1 = (p0 + rng.normal(0, [0.1] * 3 + [0.05, 0.2, 0.01] + [0.1] * 4 + [0.3, 0.0], (n, 12))).astype(np.float32)
    T = proposal.targets(torch.from_numpy(p0).cuda(), torch.from_numpy(p1).cuda()).cpu().numpy()
    want = np.stack([p1[:, 10] - p0[:, 10], p1[:, 3] - p0[:, 3], p1[:, 4] - p0[:, 4], p1[:, 5] - p0[:, 5]], 1)
    np.testing.assert_array_equal(T, want)
    Ts, sc = proposal.scale_targets(torch.from_numpy(T).cuda())
    sc = sc.cpu().numpy()
    sd = np.maximum(T.astype(np.float64).std(0, ddof=1), 1e-6).astype(np.float32)
    np.testing.assert_allclose(sc, sd, rtol=1e-6)
    np.testing.assert_array_equal(Ts.cpu().numpy(), (T / sc).astype(np.float32))
    m = _model(seed=3)
    before = m.model[:M.P].cpu().numpy().copy()
    scale = torch.tensor([2.0, 0.5, 3.0, 0.25], device="cuda")
    gve._check(proposal._lib().gve_mlp_fold_output_scale(m._ctx(), proposal._p(m.model), proposal._p(scale),
                                                         gve._stream(m.device)), m._ctx())
    after = m.model.cpu().numpy()
    s = np.array([2.0, 0.5, 3.0, 0.25], np.float32)
    np.testing.assert_array_equal(after[9408:9664].reshape(4, 64), before[9408:9664].reshape(4, 64) * s[:, None])
    np.testing.assert_array_equal(after[9664:9668], before[9664:9668] * s)
    np.testing.assert_array_equal(after[:9408], before[:9408])
    np.testing.assert_array_equal(M.bf16_params(after), M.bf16_round(after[:M.P]))
