"""Pre-encoding structure statistics (Sec. V-F, Table VI) against the oracle.

The occupancy is an integer count and must match exactly.  The other values
are sums of float32 terms that the oracle forms in FP64.  The device rounds
each difference to float32 (its square then within 2u, u = 2^-24), sums a
few terms per lane in float32 (fused multiply-adds: <= 3u for the four of
the 16-byte layout), and adds those partials in compensated float32 (<= 2u),
folded in FP64.  The terms are non-negative, so each sum is within 7u ~ 4e-7
of the oracle's; the test allows 1e-6 relative.  Rows whose length is a
multiple of 4 take the 16-byte layout (four voxels per lane), the others
and unaligned fields the one-voxel-per-lane layout; both give the same
gradient bits, so the same top-10 % decision.
"""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2608_14112_b300 import gve, inputs

pytestmark = pytest.mark.gpu

FIELDS = {
    "blobs": lambda: inputs.blobs(48, seed=5),
    "grf": lambda: inputs.grf((70, 41, 33), seed=8),
    "sparse": lambda: np.where(inputs.blobs(40, seed=2) > 0.3, inputs.blobs(40, seed=2), 0).astype(np.float32),
    "thin": lambda: inputs.grf((64, 20, 1), seed=1),
    "constant": lambda: np.full((17, 18, 19), 0.3, np.float32),
    "grf256": lambda: inputs.grf(256, seed=3),
    "x12": lambda: inputs.grf((9, 7, 12), seed=4),          # rows of 4-voxel lanes, no x + 16 pairs
    "x20": lambda: inputs.grf((23, 17, 20), seed=6),        # one x + 16 pair per lane group
    "x132": lambda: inputs.grf((6, 18, 132), seed=7),       # a full 128-voxel chunk and a 4-voxel tail
    # fewer than 4 voxels (only the streaming sweep's tail), exactly one
    # 16-byte vector of bits, one 4-voxel row of the 16-byte layout; K = 1
    "tiny3": lambda: np.float32([[[0.05, 0.22, 0.39]]]),
    "tiny4": lambda: np.float32([[[0.05, 0.22], [0.39, 0.56]]]),
    "tiny4v": lambda: (np.arange(8, dtype=np.float32).reshape(2, 1, 4) * np.float32(0.17) + np.float32(0.05)),
}


@pytest.mark.parametrize("name", list(FIELDS))
def test_structure_stats_match_oracle(name):
    V = np.ascontiguousarray(FIELDS[name](), np.float32)
    ref = O.structure_stats(V)
    got = gve.gve_structure_stats(torch.from_numpy(V).cuda())
    assert got["occupancy"] == ref["occupancy"]
    for k in ("grad_top10", "S1", "S16", "S1_over_S16"):
        np.testing.assert_allclose(got[k], ref[k], rtol=1e-6, atol=1e-300, err_msg=k)


def test_structure_unaligned_field_matches_aligned():
    """A field starting 4 bytes past a 16-byte boundary takes the
    one-voxel-per-lane layout: the same occupancy and top-10 % share (the
    same gradient bits), and both agree with the oracle."""
    V = np.ascontiguousarray(inputs.grf((21, 30, 64), seed=12), np.float32)
    ref = O.structure_stats(V)
    buf = torch.zeros(V.size + 4, device="cuda")
    view = buf[1:1 + V.size].view(V.shape)
    view.copy_(torch.from_numpy(V).cuda())
    assert view.data_ptr() % 16 == 4
    a = gve.gve_structure_stats(torch.from_numpy(V).cuda())
    b = gve.gve_structure_stats(view)
    assert a["occupancy"] == b["occupancy"] == ref["occupancy"]
    for k in ("grad_top10", "S1", "S16", "S1_over_S16"):
        np.testing.assert_allclose(a[k], ref[k], rtol=1e-6, atol=1e-300, err_msg=k)
        np.testing.assert_allclose(b[k], ref[k], rtol=1e-6, atol=1e-300, err_msg=k)


def test_structure_stage_times_and_invalid_arguments():
    V = torch.from_numpy(inputs.grf(64, seed=2)).cuda()
    res = gve.gve_structure_stats(V, want_stage_ms=True)
    assert res["ms_sweep1"] > 0 and res["ms_sweep2"] > 0
    assert res["ms_total"] >= res["ms_sweep1"] and res["launches"] >= 2
    with pytest.raises(gve.GveError):
        gve.gve_structure_stats(V[:0])
