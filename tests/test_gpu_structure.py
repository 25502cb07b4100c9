"""Pre-encoding structure statistics (Sec. V-F, Table VI) against the oracle.

The occupancy is an integer count and must match exactly.  The other values
are sums of float32 terms that the oracle forms in FP64.  The device rounds
each difference and square to float32 (relative error <= 3u, u = 2^-24) and
adds them in compensated float32 partials (<= 2u of the partial sum), folded
in FP64.  The terms are non-negative, so each sum is within 5u ~ 3e-7 of the
oracle's; the test allows 1e-6 relative.
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
}


@pytest.mark.parametrize("name", list(FIELDS))
def test_structure_stats_match_oracle(name):
    V = np.ascontiguousarray(FIELDS[name](), np.float32)
    ref = O.structure_stats(V)
    got = gve.gve_structure_stats(torch.from_numpy(V).cuda())
    assert got["occupancy"] == ref["occupancy"]
    for k in ("grad_top10", "S1", "S16", "S1_over_S16"):
        np.testing.assert_allclose(got[k], ref[k], rtol=1e-6, atol=1e-300, err_msg=k)


def test_structure_stage_times_and_invalid_arguments():
    V = torch.from_numpy(inputs.grf(64, seed=2)).cuda()
    res = gve.gve_structure_stats(V, want_stage_ms=True)
    assert res["ms_sweep1"] > 0 and res["ms_sweep2"] > 0
    assert res["ms_total"] >= res["ms_sweep1"] and res["launches"] >= 2
    with pytest.raises(gve.GveError):
        gve.gve_structure_stats(V[:0])
