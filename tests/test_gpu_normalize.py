"""Stage P on the device (Sec. III-B): gve_normalize against the oracle's
float32 definition, bit for bit (an integer-exact decision per voxel: one
correctly rounded subtraction and division), on raw fields with ragged tails
(sizes not a multiple of 4), an unaligned view (the scalar path), in place,
on a constant field and with a non-finite value (refused, output untouched)."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2608_14112_b300 import gve, inputs

pytestmark = pytest.mark.gpu


def _raw(shape, seed):
    rng = np.random.default_rng(seed)
    return (rng.normal(size=shape) * 3.7 + 11.0).astype(np.float32)


@pytest.mark.parametrize("shape", [(37, 29, 21), (64, 64, 64), (1, 1, 7), (5, 3, 1)])
def test_normalize_bit_exact(shape):
    V = _raw(shape, sum(shape))
    ref, (mn, mx) = O.normalize(V)
    out, (gmn, gmx) = gve.gve_normalize(torch.from_numpy(V).cuda())
    assert (gmn, gmx) == (mn, mx)
    np.testing.assert_array_equal(out.cpu().numpy(), ref)


def test_normalize_unaligned_in_place_and_large():
    V = _raw((33, 31, 29), 5)
    big = torch.from_numpy(np.concatenate([[0.0], V.reshape(-1)]).astype(np.float32)).cuda()
    view = big[1:].view(V.shape)                     # 4-byte offset: the scalar path
    ref, _ = O.normalize(V)
    gve.gve_normalize(view, out=view)               # in place
    np.testing.assert_array_equal(view.cpu().numpy(), ref)
    # the headline field recipe before its own scaling: a 256^3 slab of raw values
    W = inputs.grf((256, 256, 256), seed=2) * np.float32(7.0) - np.float32(2.5)
    W = W.astype(np.float32)
    refW, _ = O.normalize(W)
    outW, _ = gve.gve_normalize(torch.from_numpy(W).cuda())
    np.testing.assert_array_equal(outW.cpu().numpy(), refW)


def test_normalize_constant_and_non_finite():
    C = torch.full((9, 10, 11), 0.3, device="cuda")
    out, mm = gve.gve_normalize(C)
    assert (out == 0).all() and mm == (pytest.approx(0.3), pytest.approx(0.3))
    V = _raw((12, 12, 12), 9)
    V[3, 4, 5] = np.nan
    Vd = torch.from_numpy(V).cuda()
    out = torch.full_like(Vd, -7.0)
    with pytest.raises(gve.GveError) as ei:
        gve.gve_normalize(Vd, out=out)
    assert ei.value.status == gve.GVE_E_INVALID
    assert (out == -7.0).all()
