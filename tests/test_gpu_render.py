"""Mixture-field ray marcher (Sec. III-A rendering path) against the oracle.

Both sides place the same float32 samples (ray setup and positions in one
fixed float32 order) and take the same float32 keep decisions, so the number
of kept (sample, Gaussian) pairs must match exactly.  Values differ by the
arithmetic: the device sums Eq. 3 in float32 with exp2 approximated to 2
ulp and composites in float32; the oracle is FP64.  A sample value is then
within ~1e-5 of the oracle's, the table's slope (at most (n - 1) times the
largest step between entries, ~4 here) turns that into ~4e-5 of colour,
and ~200 float32 compositing steps add ~1e-5: pixels are compared to 2e-4
(5e-4 with shading, whose normal divides by |grad Vt| >= gfloor) and the
mean error to 1e-5.
"""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2608_14112_b300 import gve, inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def model():
    V = inputs.blobs(40, seed=3)[:, :37, :]          # (40, 37, 40): ragged cells
    prm, _, _, status = O.allocate(V, 1500, seed=2)
    assert status == 0
    return V.shape, prm.astype(np.float32)


def _gpu(prims32, shape, cam, W, H, tf, ro, normalized=True, k=3.0):
    P = torch.from_numpy(np.ascontiguousarray(prims32)).cuda()
    gve.gve_render_prepare(P, shape, gve.EvalOptions(trunc_k=k, normalized=normalized))
    img, kept = gve.gve_render(cam, W, H, torch.from_numpy(tf).cuda(), ro, want_kept=True)
    return img.cpu().numpy().astype(np.float64), kept


def _ro(**kw):
    return gve.RenderOptions(**kw)


def _od(ro):
    return dict(step=ro.step, term=ro.term, ref_step=ro.ref_step, background=ro.background, shade=ro.shade,
                ka=ro.ka, kd=ro.kd, ks=ro.ks, shininess=ro.shininess, gfloor=ro.gfloor)


CASES = [
    # (azimuth, elevation, distance, W, H, step, shade, normalized)
    (30.0, 20.0, 1.6, 50, 37, 0.5, False, True),
    (200.0, -35.0, 1.3, 33, 24, 0.7, False, False),
    (110.0, 60.0, 1.8, 40, 40, 0.5, True, True),
    (300.0, 5.0, 1.5, 17, 29, 1.0, True, False),
]


@pytest.mark.parametrize("az,el,dist,W,H,step,shade,normalized", CASES)
def test_render_matches_oracle(model, az, el, dist, W, H, step, shade, normalized):
    shape, prm = model
    cam = inputs.orbit_camera(shape, az, el, dist, 40.0)
    tf = inputs.transfer_function(64, seed=int(az))
    ro = _ro(step=step, shade=shade, background=(0.1, 0.2, 0.3), ka=0.3, kd=0.6, ks=0.25, shininess=12.0)
    img, kept = _gpu(prm, shape, cam, W, H, tf, ro, normalized)
    ref, kept_ref = O.render(prm.astype(np.float64), shape, cam, W, H, tf, _od(ro), normalized=normalized)
    assert kept == kept_ref and kept > 0
    tol = 5e-4 if shade else 2e-4
    err = np.abs(img - ref)
    assert err.max() <= tol, err.max()
    assert err.mean() <= 1e-5, err.mean()
    assert ref[..., 3].max() > 0.2          # the rays cross material


def test_render_inside_volume_and_misses(model):
    """Eye inside the box (rays start at t = 0); a camera looking away from
    the box shows only the background; a 1 x 1 image."""
    shape, prm = model
    nz, ny, nx = shape
    f = lambda *v: np.array(v, np.float32)
    tf = inputs.transfer_function(32, seed=5)
    ro = _ro(step=0.5, background=(0.5, 0.25, 0.125))
    inside = (f((nx - 1) / 2, (ny - 1) / 2, (nz - 1) / 2), f(1, 0, 0), f(0, 0, 1), f(0, 1, 0), 0.8)
    img, kept = _gpu(prm, shape, inside, 21, 13, tf, ro)
    ref, kept_ref = O.render(prm.astype(np.float64), shape, inside, 21, 13, tf, _od(ro))
    assert kept == kept_ref
    assert np.abs(img - ref).max() <= 2e-4
    away = (f(-30, -30, -30), f(0, 1, 0), f(0, 0, 1), f(-1, 0, 0), 0.2)
    img, kept = _gpu(prm, shape, away, 9, 7, tf, ro)
    assert kept == 0
    np.testing.assert_array_equal(img[..., :3], np.broadcast_to(np.float32([0.5, 0.25, 0.125]), (7, 9, 3)))
    np.testing.assert_array_equal(img[..., 3], 0.0)
    cam = inputs.orbit_camera(shape, 45.0, 30.0, 1.5, 30.0)
    img, kept = _gpu(prm, shape, cam, 1, 1, tf, ro)
    ref, kept_ref = O.render(prm.astype(np.float64), shape, cam, 1, 1, tf, _od(ro))
    assert kept == kept_ref and np.abs(img - ref).max() <= 2e-4


def test_render_empty_and_huge_primitives(model):
    """No primitives: every sample has value 0 and the table's entry 0 is
    composited; one Gaussian larger than the grid is listed in every cell."""
    shape, _ = model
    tf = inputs.transfer_function(8, seed=1)
    tf[0, 3] = 0.05
    cam = inputs.orbit_camera(shape, 10.0, 10.0, 1.5, 40.0)
    ro = _ro(step=0.8)
    empty = np.zeros((0, 12), np.float32)
    img, kept = _gpu(empty, shape, cam, 16, 8, tf, ro)
    ref, _ = O.render(np.zeros((0, 12)), shape, cam, 16, 8, tf, _od(ro))
    assert kept == 0 and np.abs(img - ref).max() <= 2e-4
    big = np.zeros((1, 12), np.float32)
    big[0, :3] = (20, 18, 20)
    big[0, 3:6] = np.log(40.0)
    big[0, 6] = 1.0
    big[0, 10] = 0.9
    img, kept = _gpu(big, shape, cam, 16, 8, tf, ro)
    ref, kept_ref = O.render(big.astype(np.float64), shape, cam, 16, 8, tf, _od(ro))
    assert kept == kept_ref and kept > 0 and np.abs(img - ref).max() <= 2e-4


def test_early_termination_bound(model):
    """Stopping a ray once its transmittance falls below `term` changes a
    pixel by at most term times the largest colour (here <= 1 + background)."""
    shape, prm = model
    cam = inputs.orbit_camera(shape, 75.0, 15.0, 1.4, 40.0)
    tf = inputs.transfer_function(64, seed=9, max_alpha=0.9)
    full, _ = _gpu(prm, shape, cam, 40, 32, tf, _ro(step=0.5, background=(1, 1, 1)))
    cut, _ = _gpu(prm, shape, cam, 40, 32, tf, _ro(step=0.5, term=0.02, background=(1, 1, 1)))
    assert np.abs(full - cut).max() <= 0.02 * 2 + 1e-6
    assert (full[..., 3] > 0.98).mean() > 0.05      # termination did happen
    ref, _ = O.render(prm.astype(np.float64), shape, cam, 40, 32, tf,
                      dict(step=0.5, term=0.02, background=(1, 1, 1)))
    assert np.abs(cut - ref).max() <= 0.02 * 2 + 1e-6


def test_render_headline_size_sampled_pixels():
    """1.4 M Gaussians over a 1024^3 grid (allocation-like scales), 256 x 256
    image at step 0.5, the launch configuration of the benchmark: 12 pixels
    recomputed by the oracle one by one."""
    n, N = 1024, 1_400_000
    rng = np.random.default_rng(4)
    prm = np.zeros((N, 12), np.float32)
    prm[:, :3] = rng.uniform(0, n - 1, (N, 3))
    prm[:, 3:6] = np.log(rng.lognormal(np.log(3.0), 0.4, (N, 3)))
    prm[:, 6:10] = rng.normal(size=(N, 4))
    prm[:, 10] = rng.uniform(0.0, 1.0, N)
    prm[:, 11] = rng.normal(-2.2, 0.5, N)
    shape = (n, n, n)
    cam = inputs.orbit_camera(shape, 40.0, 25.0, 1.7, 40.0)
    tf = inputs.transfer_function(256, seed=4, max_alpha=0.05)
    ro = _ro(step=0.5)
    img, _ = _gpu(prm, shape, cam, 256, 256, tf, ro)
    pix = rng.choice(256 * 256, 12, replace=False)
    ref, _ = O.render(prm.astype(np.float64), shape, cam, 256, 256, tf, _od(ro), pixels=pix)
    got = img.reshape(-1, 4)[pix]
    assert np.abs(got - ref).max() <= 5e-4
    assert ref[:, 3].max() > 0.1


def test_render_invalid_arguments(model):
    shape, prm = model
    P = torch.from_numpy(prm).cuda()
    gve.gve_render_prepare(P, shape)
    tf = torch.from_numpy(inputs.transfer_function(8, seed=1)).cuda()
    cam = inputs.orbit_camera(shape, 0.0, 0.0, 1.5, 40.0)
    with pytest.raises(gve.GveError):
        gve.gve_render(cam, 8, 8, tf, _ro(step=1.0 / 128))
    with pytest.raises(gve.GveError):
        gve.gve_render(cam, 8, 8, tf[:1].contiguous(), _ro())
    with pytest.raises(gve.GveError):
        gve.gve_render(cam, 0, 8, tf, _ro())
    bad = (cam[0], cam[1], cam[2], np.array([np.nan, 0, 1], np.float32), cam[4])
    with pytest.raises(gve.GveError):
        gve.gve_render(bad, 8, 8, tf, _ro())
