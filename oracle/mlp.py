"""FP64 reference of the learned proposal's MLP and features.

TEST INFRASTRUCTURE ONLY (like the rest of this package): it checks the CUDA
MLP kernels and the feature kernel.  Plain numpy, written from the
definitions: four affine layers 16-64-64-64-4 with the erf form of GELU
between them, inputs standardised by a stored mean and inverse standard
deviation and clipped to [-6, 6], mean squared error over rows and outputs.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erf

from . import oracle as O

P = 9668
MODEL_FLOATS = 33870
IN_CLIP = 6.0            # standardised inputs are clipped to [-6, 6]
SHAPES = [("W1", (64, 16)), ("b1", (64,)), ("W2", (64, 64)), ("b2", (64,)), ("W3", (64, 64)), ("b3", (64,)),
          ("W4", (4, 64)), ("b4", (4,))]


def unpack(flat: np.ndarray) -> dict:
    out, o = {}, 0
    for name, shp in SHAPES:
        n = int(np.prod(shp))
        out[name] = np.asarray(flat[o:o + n], np.float64).reshape(shp)
        o += n
    return out


def bf16_round(x) -> np.ndarray:
    """float32 -> bfloat16 with round-to-nearest-even on the 16 dropped bits
    (finite inputs), returned as float64."""
    u = np.ascontiguousarray(np.asarray(x, np.float32)).view(np.uint32).astype(np.uint64)
    r = (u + 0x7FFF + ((u >> 16) & 1)) >> 16
    return ((r << 16).astype(np.uint32)).view(np.float32).astype(np.float64)


def bf16_params(model: np.ndarray) -> np.ndarray:
    """The BF16 copies stored in the model buffer, as float64."""
    raw = np.ascontiguousarray(model[3 * P + 32: 3 * P + 32 + P // 2]).view(np.uint16)[:P]
    return (raw.astype(np.uint32) << 16).view(np.float32).astype(np.float64)


def gelu(x):
    return 0.5 * x * (1.0 + erf(x / math.sqrt(2.0)))


def gelu_d(x):
    return 0.5 * (1.0 + erf(x / math.sqrt(2.0))) + x * np.exp(-0.5 * x * x) / math.sqrt(2.0 * math.pi)


def forward(params: np.ndarray, mean, istd, X):
    W = unpack(params)
    x = np.clip((np.asarray(X, np.float64) - mean) * istd, -IN_CLIP, IN_CLIP)
    z1 = x @ W["W1"].T + W["b1"]
    a1 = gelu(z1)
    z2 = a1 @ W["W2"].T + W["b2"]
    a2 = gelu(z2)
    z3 = a2 @ W["W3"].T + W["b3"]
    a3 = gelu(z3)
    y = a3 @ W["W4"].T + W["b4"]
    return y, (x, z1, a1, z2, a2, z3, a3)


def backward(params: np.ndarray, mean, istd, X, dY):
    """Gradient w.r.t. the flat params for the upstream gradient dY = dL/dy
    (back-propagation through the four layers)."""
    W = unpack(params)
    _, (x, z1, a1, z2, a2, z3, a3) = forward(params, mean, istd, X)
    d4 = np.asarray(dY, np.float64)
    g = {"W4": d4.T @ a3, "b4": d4.sum(0)}
    d3 = (d4 @ W["W4"]) * gelu_d(z3)
    g["W3"], g["b3"] = d3.T @ a2, d3.sum(0)
    d2 = (d3 @ W["W3"]) * gelu_d(z2)
    g["W2"], g["b2"] = d2.T @ a1, d2.sum(0)
    d1 = (d2 @ W["W2"]) * gelu_d(z1)
    g["W1"], g["b1"] = d1.T @ x, d1.sum(0)
    return np.concatenate([g[name].reshape(-1) for name, _ in SHAPES])


def loss_grad(params: np.ndarray, mean, istd, X, T):
    """MSE over rows and outputs and its gradient w.r.t. the flat params."""
    y, _ = forward(params, mean, istd, X)
    diff = y - np.asarray(T, np.float64)
    loss = float((diff ** 2).mean())
    return loss, backward(params, mean, istd, X, 2.0 * diff / diff.size)


def ls_bounds(dims) -> tuple:
    """Clamp interval of the corrected log-scales: the allocator's scale caps
    [0.3, max dim / 16], logarithms in float64 rounded once to float32."""
    return float(np.float32(math.log(0.3))), float(np.float32(math.log(max(dims) / 16.0)))


def apply(prm: np.ndarray, Y: np.ndarray, dims) -> np.ndarray:
    """Corrected records: a + dA, clamp(log s + dLS); rows with a non-finite
    output are left as they are."""
    lo, hi = ls_bounds(dims)
    out = np.array(prm, np.float64, copy=True)
    for i in range(out.shape[0]):
        if not np.all(np.isfinite(Y[i])):
            continue
        out[i, 10] += Y[i, 0]
        out[i, 3:6] = np.clip(out[i, 3:6] + Y[i, 1:4], lo, hi)
    return out


def upstream(prm_corrected: np.ndarray, grad_prims: np.ndarray, Y: np.ndarray, dims) -> np.ndarray:
    """dL/dY from dL/d(corrected records): the amplitude gradient passes
    through, a log-scale gradient only where the clamp was inactive."""
    lo, hi = ls_bounds(dims)
    p = np.asarray(prm_corrected, np.float64)
    g = np.asarray(grad_prims, np.float64)
    dY = np.zeros((p.shape[0], 4))
    ok = np.all(np.isfinite(Y), axis=1)
    dY[:, 0] = np.where(ok, g[:, 10], 0.0)
    inside = (p[:, 3:6] > lo) & (p[:, 3:6] < hi)
    dY[:, 1:4] = np.where(ok[:, None] & inside, g[:, 3:6], 0.0)
    return dY


def features(field: np.ndarray, prm: np.ndarray, n_detail: int, gbar: float, occ: float = 0.02) -> np.ndarray:
    """The 16 features of each record (seed voxel = round(mu), windows
    clipped at the borders)."""
    V = np.asarray(field, np.float32)
    nz, ny, nx = V.shape
    out = np.zeros((prm.shape[0], 16), np.float64)
    for i, p in enumerate(np.asarray(prm, np.float64)):
        c = [int(min(max(math.floor(np.float32(p[j]) + np.float32(0.5)), 0), d - 1)) for j, d in enumerate((nx, ny, nz))]
        J = O.struct_tensor(V, c)
        ev, _ = O.jacobi3(J)
        gb2 = gbar * gbar * 343.0 + 1e-30
        out[i, 0:3] = np.log1p(np.maximum(ev, 0.0) / gb2)
        gv = np.zeros(3)
        for ax, (lo, hi, n) in enumerate(((c[0], c[0], nx), (c[1], c[1], ny), (c[2], c[2], nz))):
            a, b, scale = c[ax] + 1, c[ax] - 1, 0.5
            if b < 0:
                b, scale = c[ax], 1.0
            if a > n - 1:
                a, scale = c[ax], 1.0
            ia, ib = list(c), list(c)
            ia[ax], ib[ax] = a, b
            gv[ax] = 0.0 if n < 2 else scale * (float(V[ia[2], ia[1], ia[0]]) - float(V[ib[2], ib[1], ib[0]]))
        out[i, 3] = min(math.sqrt((gv ** 2).sum()) / (gbar + 1e-30), 10.0)
        w = V[max(c[2] - 2, 0):c[2] + 3, max(c[1] - 2, 0):c[1] + 3, max(c[0] - 2, 0):c[0] + 3].astype(np.float64)
        out[i, 4] = w.mean()
        out[i, 5] = math.sqrt(max((w ** 2).mean() - w.mean() ** 2, 0.0))
        out[i, 6] = w.min()
        out[i, 7] = w.max()
        out[i, 8:11] = p[3:6]
        out[i, 11] = p[10]
        out[i, 12] = 1.0 if i < n_detail else 0.0
        out[i, 13] = (w > np.float32(occ)).mean()
        out[i, 14] = (ev[1] - ev[0]) / (max(ev[2], 0.0) + 1e-30)
        out[i, 15] = V[c[2], c[1], c[0]]
    return out
