"""Batched allocation (all volumes concurrently), batched refinement (one
binning of all volumes, then one persistent cooperative kernel for the
evaluation and update of all volumes, one CUDA graph launch per iteration)
and the launch-shape autotuner.

The batched allocation must write, volume by volume, exactly the records
gve_allocate writes for that volume alone (bit for bit), and report a volume
whose field cannot support its budget by name.

A batch of uneven volumes must give, volume by volume, what the FP64 oracle's
refinement gives (final PSNR within 0.05 dB, losses within 2e-3 relative, the
bars of the single-volume parity test), and what gve_refine gives alone: the
same loss traces (relative 1e-4) and final PSNR (1e-3 dB).  The parameters
agree to relative L2 1e-3 only: gradient sums are accumulated with float
atomics, whose order varies run to run, and Adam with eps = 1e-15 turns a
gradient that is zero up to rounding into a step of +-lr.  The
capacity-overflow replay is exercised by forcing a small logical pair
capacity through the library's test hook; the bounded grid-wide wait by the
host fault-injection hook GVE_FAULT=timeout (the barrier then waits for one
CTA more than the grid holds and gives up after a few milliseconds: no GPU
fault, no hang), and the out-of-memory status by GVE_FAULT=alloc.
"""
import ctypes
import os

import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2608_14112_b300 import batched, gve, inputs

pytestmark = pytest.mark.gpu

SHAPES = [(40, 36, 28), (24, 24, 24), (64, 20, 12), (33, 17, 45)]


def rel_l2(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.fixture(scope="module")
def batch():
    fields, counts, parts = [], [], []
    for i, shp in enumerate(SHAPES):
        V = torch.from_numpy(inputs.grf(shp, seed=50 + i)).cuda()
        n = max(64, (shp[0] * shp[1] * shp[2]) // 48)
        P, _ = gve.gve_allocate(V, n, seed=i)
        fields.append(V)
        counts.append(n)
        parts.append(P)
    return fields, counts, torch.cat(parts, 0).contiguous()


def _single(fields, counts, prims, iters, opts=None):
    outs, psnr, traces = [], [], []
    off = 0
    for f, n in zip(fields, counts):
        P = prims[off:off + n].clone()
        tr = torch.zeros(iters, dtype=torch.float64, device="cuda")
        st = gve.gve_refine(P, f, iters=iters, trace=tr, opts=opts)
        outs.append(P)
        psnr.append(st["psnr_final"])
        traces.append(tr)
        off += n
    return torch.cat(outs, 0), psnr, torch.stack(traces, 1)


@pytest.mark.parametrize("brick,gpb", [(8, 0), (4, 0), (16, 0), (8, 32)])
def test_batch_matches_per_volume_refine(batch, brick, gpb):
    fields, counts, prims = batch
    iters = 6
    opts = gve.EvalOptions(brick=brick, gaussians_per_block=gpb)
    ref, ref_psnr, ref_trace = _single(fields, counts, prims, iters, opts)
    P = prims.clone()
    trace = torch.zeros(iters * len(fields), dtype=torch.float64, device="cuda")
    psnr, st = gve.gve_refine_batch(P, fields, counts, iters, opts=opts, trace=trace)
    assert rel_l2(P.cpu().numpy(), ref.cpu().numpy()) <= 1e-3
    np.testing.assert_allclose(psnr, ref_psnr, atol=1e-3)
    np.testing.assert_allclose(trace.view(iters, len(fields)).cpu().numpy(), ref_trace.cpu().numpy(), rtol=1e-4)
    assert st["iters_done"] == iters and st["retries"] == 0


def test_overflow_replay_gives_the_same_result(batch):
    fields, counts, prims = batch
    iters = 5
    ref, ref_psnr, _ = _single(fields, counts, prims, iters)
    refb = prims.clone()
    gve.gve_refine_batch(refb, fields, counts, iters)
    os.environ["GVE_TEST_PAIR_CAP"] = "1000"
    try:
        P = prims.clone()
        psnr, st = gve.gve_refine_batch(P, fields, counts, iters)
        Q = prims[:counts[0]].clone()
        st1 = gve.gve_refine(Q, fields[0], iters=iters)
    finally:
        del os.environ["GVE_TEST_PAIR_CAP"]
    assert st["retries"] >= 1 and st1["retries"] >= 1
    assert rel_l2(P.cpu().numpy(), refb.cpu().numpy()) <= 1e-3
    assert rel_l2(Q.cpu().numpy(), ref[:counts[0]].cpu().numpy()) <= 1e-3
    np.testing.assert_allclose(psnr, ref_psnr, atol=1e-3)


def test_autotune_and_encode_batch(batch):
    fields, counts, prims = batch
    best, table = gve.gve_autotune(prims, fields, counts)
    assert best.brick in (4, 8, 16) and best.gaussians_per_block in (32, 64)
    assert len(table) == 6 and all(v > 0 for v in table.values())
    assert table[(best.brick, best.gaussians_per_block)] == min(table.values())
    res = batched.encode_batch(fields, counts, iters=4, seed=1)
    assert len(res.psnr) == len(fields) and all(np.isfinite(res.psnr))
    assert sum(p.shape[0] for p in res.prims) == sum(counts)


def test_batch_matches_oracle_refine():
    """An uneven batch of three small volumes from the oracle's own
    allocations, 10 iterations: each volume's final PSNR within 0.05 dB of
    the oracle's refinement of that volume alone, losses within 2e-3."""
    shapes = [(20, 24, 28), (32, 16, 24), (18, 30, 14)]
    fields, counts, recs, refs = [], [], [], []
    for i, shp in enumerate(shapes):
        V = inputs.grf(shp, seed=300 + i)
        n = (shp[0] * shp[1] * shp[2]) // 40
        prm, _, _, status = O.allocate(V, n, seed=10 + i)
        assert status == 0
        p32 = prm.astype(np.float32)
        _, losses, sse = O.refine(p32.astype(np.float64), V, iters=10, lr=1e-2, eps=1e-15)
        refs.append((O.psnr_from_sse(sse, V.size), losses))
        fields.append(torch.from_numpy(V).cuda())
        counts.append(n)
        recs.append(p32)
    P = torch.from_numpy(np.concatenate(recs)).cuda()
    trace = torch.zeros(10 * len(shapes), dtype=torch.float64, device="cuda")
    psnr, st = gve.gve_refine_batch(P, fields, counts, 10, lr=1e-2, eps=1e-15, trace=trace)
    tr = trace.view(10, len(shapes)).cpu().numpy()
    for v, (psnr_ref, losses) in enumerate(refs):
        assert abs(psnr[v] - psnr_ref) <= 0.05, (v, psnr[v], psnr_ref)
        np.testing.assert_allclose(tr[:, v], losses, rtol=2e-3)


def test_batch_barrier_timeout_returns_status(batch):
    """A grid-wide wait that runs out ends the call with GVE_E_TIMEOUT and
    leaves the records as they were; the next call is unaffected."""
    fields, counts, prims = batch
    P = prims.clone()
    os.environ["GVE_FAULT"] = "timeout"
    try:
        with pytest.raises(gve.GveError) as ei:
            gve.gve_refine_batch(P, fields, counts, 3)
    finally:
        del os.environ["GVE_FAULT"]
    assert ei.value.status == gve.GVE_E_TIMEOUT
    assert torch.equal(P, prims)
    ref, ref_psnr, _ = _single(fields, counts, prims, 3)
    psnr, st = gve.gve_refine_batch(P, fields, counts, 3)
    np.testing.assert_allclose(psnr, ref_psnr, atol=1e-3)


def test_alloc_fault_returns_nomem_and_context_recovers():
    """An allocation failure (injected on the host) is a status, not a crash:
    a fresh context cannot grow its scratch, returns GVE_E_NOMEM, and works
    once allocation succeeds again."""
    L = gve.lib()
    ctx = ctypes.c_void_p()
    assert L.gve_ctx_create(ctypes.byref(ctx), torch.cuda.current_device()) == gve.GVE_OK
    try:
        rng = np.random.default_rng(4)
        p = np.zeros((50, 12), np.float32)
        p[:, 0:3] = rng.uniform(0, 15, (50, 3))
        p[:, 6] = 1.0
        p[:, 10] = 0.5
        P = torch.from_numpy(p).cuda()
        out = torch.zeros((16, 16, 16), device="cuda")
        o = gve.EvalOptions().c()
        args = (ctx, ctypes.c_void_p(P.data_ptr()), 50, gve.Dims(16, 16, 16), ctypes.byref(o),
                ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        os.environ["GVE_FAULT"] = "alloc"
        try:
            assert L.gve_evaluate(*args) == gve.GVE_E_NOMEM
        finally:
            del os.environ["GVE_FAULT"]
        assert L.gve_evaluate(*args) == gve.GVE_OK
        torch.cuda.synchronize()
        ref = gve.gve_evaluate(P, (16, 16, 16))
        assert torch.allclose(out, ref, rtol=1e-6, atol=1e-7)
    finally:
        L.gve_ctx_destroy(ctx)


def test_allocate_batch_matches_single_volume_allocation():
    """Twelve uneven volumes (more than the eight allocation workers): every
    volume's records and summary equal gve_allocate's on it alone."""
    shapes = SHAPES * 3
    fields = [torch.from_numpy(inputs.grf(shp, seed=60 + i)).cuda() for i, shp in enumerate(shapes)]
    budgets = [max(64, (s[0] * s[1] * s[2]) // 40) for s in shapes]
    P, infos = gve.gve_allocate_batch(fields, budgets, seed=3)
    torch.cuda.synchronize()
    off = 0
    for f, n, info in zip(fields, budgets, infos):
        ref, rinfo = gve.gve_allocate(f, n, seed=3)
        assert torch.equal(P[off:off + n], ref)
        assert info == rinfo
        off += n


def test_allocate_batch_reports_the_infeasible_volume():
    fields = [torch.from_numpy(inputs.grf(shp, seed=70 + i)).cuda() for i, shp in enumerate(SHAPES)]
    budgets = [64, 64, 10 ** 6, 64]          # volume 2 holds fewer voxels than its budget
    with pytest.raises(gve.GveError) as e:
        gve.gve_allocate_batch(fields, budgets, seed=0)
    assert e.value.status == gve.GVE_E_BUDGET and "volume 2" in str(e.value)

