"""Pre-encoding structure statistics (Sec. V-F, Table VI) against the oracle:
the occupancy exactly (an integer count), the top-10 % gradient-mass share
and the structure-function values to 1e-9 relative (FP64 sums of the same
float32 gradient magnitudes and values, in another order)."""
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
        np.testing.assert_allclose(got[k], ref[k], rtol=1e-9, atol=1e-300), k
