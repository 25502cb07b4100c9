"""The evaluation entry point that allocates no device memory.

It exists for callers that cannot call cudaMalloc -- code that runs inside a
memory pool or arena owning the whole device, a service whose device
footprint must stay fixed after start-up, or a call path that must not take
the allocator's locks.  Its scratch is a fixed array inside the library, so
this file checks, through the C ABI, that two calls in a row (the second one
finding the first one's leftovers in that array) give the same field as the
ordinary gve_evaluate and as the FP64 oracle, within the field tolerance of
the other parity tests; that oversized requests are refused before anything
runs; that a pair count beyond the array's capacity, found on the device,
returns GVE_E_CAPACITY with the output untouched and leaves the next call
unharmed; that pointers of another memory space are refused; and that the
Python wrapper gives the same field.

The file name sorts last so that a run stopping at the first failure has
already run every other test.
"""
import ctypes

import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2608_14112_b300 import gve

pytestmark = pytest.mark.gpu

FIELD_TOL = 1e-5


def _prims(rng, n, dims, s_lo, s_hi):
    p = np.zeros((n, 12), np.float64)
    p[:, 0:3] = rng.uniform(0, 1, (n, 3)) * (np.array(dims) - 1)
    p[:, 3:6] = np.log(rng.uniform(s_lo, s_hi, (n, 3)))
    p[:, 6:10] = rng.normal(size=(n, 4))
    p[:, 10] = rng.uniform(0.05, 1.0, n)
    p[:, 11] = rng.uniform(-2.5, 1.5, n)
    return torch.from_numpy(p.astype(np.float32)).cuda()


def _noalloc_status(prims, shape, out_ptr, chunk=0):
    nz, ny, nx = shape
    opts = gve.EvalOpts(3.0, 0.05, 1, 8, chunk)
    return gve.lib().gve_evaluate_noalloc(ctypes.c_void_p(prims.data_ptr()), prims.shape[0], gve.Dims(nx, ny, nz),
                                          ctypes.byref(opts), out_ptr,
                                          ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


def _call_noalloc(prims, shape, out):
    """Direct C-ABI call: raw device pointers and the current stream."""
    nz, ny, nx = shape
    opts = gve.EvalOpts(3.0, 0.05, 1, 8)
    s = gve.lib().gve_evaluate_noalloc(ctypes.c_void_p(prims.data_ptr()), prims.shape[0], gve.Dims(nx, ny, nz),
                                       ctypes.byref(opts), ctypes.c_void_p(out.data_ptr()),
                                       ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return s


def _rel(a, b):
    a = a.double().cpu()
    b = b.double().cpu()
    return float((a - b).norm() / b.norm())


def test_noalloc_matches_evaluate_on_two_calls_in_a_row():
    rng = np.random.default_rng(2024)
    cases = [((37, 29, 21), 700, 0.8, 3.0), ((24, 40, 33), 1500, 0.5, 2.0)]
    for dims, n, lo, hi in cases:
        nx, ny, nz = dims
        shape = (nz, ny, nx)
        p = _prims(rng, n, dims, lo, hi)
        ref = gve.gve_evaluate(p, shape)
        out = torch.full(shape, float("nan"), device="cuda")
        assert _call_noalloc(p, shape, out) == gve.GVE_OK
        torch.cuda.synchronize()
        assert torch.isfinite(out).all()
        assert _rel(out, ref) <= FIELD_TOL
        _, _, vt = O.eval_region(p.cpu().numpy().astype(np.float64), dims)
        assert _rel(out, torch.from_numpy(vt)) <= FIELD_TOL


def test_noalloc_capacity_overflow_leaves_output_and_next_call_intact():
    """8,192 primitives with scales near 20 voxels on a 128^3 grid need far
    more than the array's 524,288 (brick, Gaussian) pairs: the count is found
    on the device, the call returns GVE_E_CAPACITY and writes nothing.  The
    sticky overflow flag it leaves in the shared array is cleared by the next
    call, which must succeed."""
    rng = np.random.default_rng(7)
    shape = (128, 128, 128)
    big = _prims(rng, 8192, (128, 128, 128), 15.0, 25.0)
    out = torch.full(shape, float("nan"), device="cuda")
    assert _noalloc_status(big, shape, ctypes.c_void_p(out.data_ptr())) == gve.GVE_E_CAPACITY
    torch.cuda.synchronize()
    assert torch.isnan(out).all()
    small_shape = (21, 29, 37)
    p = _prims(rng, 600, (37, 29, 21), 0.8, 3.0)
    out2 = torch.full(small_shape, float("nan"), device="cuda")
    assert _noalloc_status(p, small_shape, ctypes.c_void_p(out2.data_ptr()), chunk=32) == gve.GVE_OK
    torch.cuda.synchronize()
    assert _rel(out2, gve.gve_evaluate(p, small_shape)) <= FIELD_TOL


def test_noalloc_refuses_host_pointers_and_bad_options():
    rng = np.random.default_rng(8)
    p = _prims(rng, 50, (16, 16, 16), 1.0, 2.0)
    host_out = torch.zeros((16, 16, 16))          # pageable host memory
    assert _noalloc_status(p, (16, 16, 16), ctypes.c_void_p(host_out.data_ptr())) == gve.GVE_E_INVALID
    out = torch.zeros((16, 16, 16), device="cuda")
    assert _noalloc_status(p, (16, 16, 16), ctypes.c_void_p(out.data_ptr()), chunk=48) == gve.GVE_E_INVALID


def test_noalloc_python_wrapper_matches_evaluate():
    rng = np.random.default_rng(9)
    shape = (20, 24, 28)
    p = _prims(rng, 900, (28, 24, 20), 0.7, 2.5)
    got = gve.gve_evaluate_noalloc(p, shape)
    assert _rel(got, gve.gve_evaluate(p, shape)) <= FIELD_TOL


def test_noalloc_rejects_sizes_beyond_its_limits():
    shape_big = (264, 256, 256)   # more than 32,768 bricks of 8^3
    p = torch.zeros((4, 12), device="cuda")
    out = torch.zeros((1, 1, 1), device="cuda")
    nz, ny, nx = shape_big
    opts = gve.EvalOpts(3.0, 0.05, 1, 8)
    s = gve.lib().gve_evaluate_noalloc(ctypes.c_void_p(p.data_ptr()), 4, gve.Dims(nx, ny, nz), ctypes.byref(opts),
                                       ctypes.c_void_p(out.data_ptr()), None)
    assert s == gve.GVE_E_INVALID
    long_axis = gve.Dims((1 << 14) + 8, 1, 1)     # few bricks, but an axis beyond 2^14 voxels
    s = gve.lib().gve_evaluate_noalloc(ctypes.c_void_p(p.data_ptr()), 4, long_axis, ctypes.byref(opts),
                                       ctypes.c_void_p(out.data_ptr()), None)
    assert s == gve.GVE_E_INVALID
    too_many = torch.zeros((8193, 12), device="cuda")
    s = gve.lib().gve_evaluate_noalloc(ctypes.c_void_p(too_many.data_ptr()), 8193, gve.Dims(8, 8, 8),
                                       ctypes.byref(opts), ctypes.c_void_p(out.data_ptr()), None)
    assert s == gve.GVE_E_INVALID
