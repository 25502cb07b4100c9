"""Seeded synthetic scalar volumes.

This module holds no arithmetic of the encoder: it only draws the test and
benchmark fields, so that the CUDA path and the CPU oracle are fed the very
same bytes.  Every field is float32, shaped ``(nz, ny, nx)`` (x fastest) and
min-max normalised to [0, 1] (Sec. III-B of the paper).

The paper evaluates on five simulation/scan volumes (Table II) that are not
available here; these generators stand in for them with the shapes, sizes and
structure of the workloads named below:

* ``blobs``      -- sum of random anisotropic Gaussian blobs plus a weak
  low-frequency sinusoidal background (small dense field, 64^3).
* ``grf``        -- Gaussian random field with a k^-5/3 shell energy spectrum
  (turbulence-like; amplitude |F(k)| ~ k^-11/6, random phases, F(0) = 0).
* ``fbm_fronts`` -- six-octave value-noise fBm plus three sharp tanh fronts
  of width 2 voxels (multiscale gigavoxel stand-in).
"""
from __future__ import annotations

import math

import numpy as np

try:  # torch is plumbing here: fast separable upsampling on any device
    import torch
except Exception:  # pragma: no cover
    torch = None


def _normalise(a: np.ndarray) -> np.ndarray:
    a = a.astype(np.float64)
    lo, hi = float(a.min()), float(a.max())
    if hi <= lo:
        return np.zeros_like(a, dtype=np.float32)
    return ((a - lo) / (hi - lo)).astype(np.float32)


def _random_rotation(rng: np.random.Generator) -> np.ndarray:
    """Uniform random rotation (Shoemake's subgroup algorithm)."""
    u1, u2, u3 = rng.random(3)
    a, b = math.sqrt(1 - u1), math.sqrt(u1)
    qx, qy = a * math.sin(2 * math.pi * u2), a * math.cos(2 * math.pi * u2)
    qz, qw = b * math.sin(2 * math.pi * u3), b * math.cos(2 * math.pi * u3)
    return np.array([
        [1 - 2 * (qy * qy + qz * qz), 2 * (qx * qy - qw * qz), 2 * (qx * qz + qw * qy)],
        [2 * (qx * qy + qw * qz), 1 - 2 * (qx * qx + qz * qz), 2 * (qy * qz - qw * qx)],
        [2 * (qx * qz - qw * qy), 2 * (qy * qz + qw * qx), 1 - 2 * (qx * qx + qy * qy)]])


def blobs(n: int = 64, n_blobs: int = 40, seed: int = 1, shape=None) -> np.ndarray:
    """Sum of ``n_blobs`` anisotropic Gaussian blobs (centres U[0,n)^3,
    amplitudes U[0.2,1], per-axis sigma U[1.5,8] voxels, uniform random
    rotations) plus 0.05 sin(2 pi f.p / n + phi), f in {1,2}^3."""
    rng = np.random.Generator(np.random.PCG64(seed))
    nx, ny, nz = (n, n, n) if shape is None else shape
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    P = np.stack([x, y, z], axis=-1).astype(np.float64)
    V = np.zeros((nz, ny, nx), np.float64)
    for _ in range(n_blobs):
        c = rng.random(3) * np.array([nx, ny, nz])
        amp = rng.uniform(0.2, 1.0)
        sig = rng.uniform(1.5, 8.0, size=3)
        R = _random_rotation(rng)
        d = (P - c) @ R  # coordinates in the blob frame
        V += amp * np.exp(-0.5 * np.sum((d / sig) ** 2, axis=-1))
    f = rng.integers(1, 3, size=3)
    phi = rng.uniform(0, 2 * np.pi)
    V += 0.05 * np.sin(2 * np.pi * (f[0] * x / nx + f[1] * y / ny + f[2] * z / nz) + phi)
    return _normalise(V)


def grf(shape, seed: int, device=None):
    """Gaussian random field, shell spectrum E(k) ~ k^-5/3 (so |F(k)| ~
    k^-11/6), white-noise phases, zero mean mode.  ``shape`` = (nx, ny, nz)
    or an int for a cube.  With ``device`` the spectral filtering runs in
    torch there and a float32 tensor is returned (same white noise)."""
    if isinstance(shape, int):
        shape = (shape, shape, shape)
    nx, ny, nz = shape
    rng = np.random.Generator(np.random.PCG64(seed))
    noise = rng.standard_normal((nz, ny, nx)).astype(np.float64)
    if device is not None:
        t = torch.from_numpy(noise).to(device)
        F = torch.fft.rfftn(t)
        kz = torch.fft.fftfreq(nz, device=device, dtype=torch.float64) * nz
        ky = torch.fft.fftfreq(ny, device=device, dtype=torch.float64) * ny
        kx = torch.fft.rfftfreq(nx, device=device, dtype=torch.float64) * nx
        K = torch.sqrt(kz[:, None, None] ** 2 + ky[None, :, None] ** 2 + kx[None, None, :] ** 2)
        K[0, 0, 0] = 1.0
        F = F * K.pow(-11.0 / 6.0)
        F[0, 0, 0] = 0.0
        V = torch.fft.irfftn(F, s=(nz, ny, nx))
        lo, hi = V.min(), V.max()
        return ((V - lo) / (hi - lo)).float().contiguous()
    F = np.fft.rfftn(noise)
    kz = np.fft.fftfreq(nz) * nz
    ky = np.fft.fftfreq(ny) * ny
    kx = np.fft.rfftfreq(nx) * nx
    K = np.sqrt(kz[:, None, None] ** 2 + ky[None, :, None] ** 2 + kx[None, None, :] ** 2)
    K[0, 0, 0] = 1.0
    F *= K ** (-11.0 / 6.0)
    F[0, 0, 0] = 0.0
    return _normalise(np.fft.irfftn(F, s=(nz, ny, nx), axes=(0, 1, 2)))


def _interp_matrix(n: int, L: int, dtype, device):
    """(n, L) linear interpolation from an L-point lattice spanning [0, n-1]."""
    u = torch.arange(n, dtype=torch.float64, device=device) * ((L - 1) / max(n - 1, 1))
    i0 = torch.clamp(torch.floor(u).long(), 0, L - 2)
    f = u - i0.double()
    W = torch.zeros((n, L), dtype=torch.float64, device=device)
    W[torch.arange(n, device=device), i0] = 1.0 - f
    W[torch.arange(n, device=device), i0 + 1] += f
    return W.to(dtype)


def fbm_fronts(n: int = 1024, seed: int = 4, octaves: int = 6, device="cpu",
               as_numpy: bool = False, region=None):
    """Six-octave value-noise fBm (lattice (4*2^o+1)^3 of iid U[-1,1], gain
    1/2, trilinear upsampling) plus three fronts 0.5 tanh(n_j.(p - p_j)/2)
    with n_j uniform on the sphere and p_j in U[n/4, 3n/4)^3, min-max
    normalised.  Returns a float32 torch tensor on ``device`` (numpy if
    ``as_numpy``).  ``region = ((x0, y0, z0), (sx, sy, sz))`` draws only that
    sub-box of the n^3 field (same lattices and fronts), normalised by its own
    min and max."""
    if torch is None:
        raise RuntimeError("fbm_fronts needs torch")
    rng = np.random.Generator(np.random.PCG64(seed))
    dev = torch.device(device)
    dt = torch.float32
    if region is None:
        r0, rs = (0, 0, 0), (n, n, n)
    else:
        r0, rs = tuple(int(v) for v in region[0]), tuple(int(v) for v in region[1])
    x0, y0, z0 = r0
    sx, sy, sz = rs
    V = torch.zeros((sz, sy, sx), dtype=dt, device=dev)
    amp = 1.0
    for o in range(octaves):
        L = 4 * 2 ** o + 1
        lat = torch.from_numpy(rng.uniform(-1.0, 1.0, size=(L, L, L))).to(dev, dt)  # (z, y, x)
        W = _interp_matrix(n, L, dt, dev)
        Wx, Wy, Wz = W[x0:x0 + sx], W[y0:y0 + sy], W[z0:z0 + sz]
        t = torch.matmul(lat, Wx.T)                                   # (Lz, Ly, sx)
        t = torch.matmul(Wy, t)                                       # (Lz, sy, sx)
        t = torch.matmul(Wz, t.reshape(L, sy * sx)).reshape(sz, sy, sx)
        V.add_(t, alpha=amp)
        del t
        amp *= 0.5
    for _ in range(3):
        nv = rng.standard_normal(3)
        nv /= np.linalg.norm(nv)
        pj = rng.uniform(n / 4, 3 * n / 4, size=3)
        sxv = (torch.arange(x0, x0 + sx, dtype=dt, device=dev) - float(pj[0])) * float(nv[0])
        syv = (torch.arange(y0, y0 + sy, dtype=dt, device=dev) - float(pj[1])) * float(nv[1])
        szv = (torch.arange(z0, z0 + sz, dtype=dt, device=dev) - float(pj[2])) * float(nv[2])
        for zi in range(0, sz, 64):
            arg = szv[zi:zi + 64, None, None] + syv[None, :, None] + sxv[None, None, :]
            V[zi:zi + 64].add_(torch.tanh(arg * 0.5), alpha=0.5)
    lo, hi = V.min(), V.max()
    V.sub_(lo).div_(hi - lo)
    if as_numpy:
        return V.cpu().numpy()
    return V


# Workload table: the five evaluation configurations.
BATCHED_SHAPES = [(96, 96, 96), (128, 128, 128), (160, 160, 160), (192, 192, 192),
                  (224, 224, 224), (256, 256, 256), (320, 320, 320), (384, 384, 384),
                  (512, 256, 128), (640, 320, 64), (384, 192, 96), (448, 224, 112),
                  (512, 128, 64), (320, 160, 80), (256, 256, 64), (576, 288, 72)]
BATCHED_SEEDS = list(range(100, 116))


def batched_budget(shape) -> int:
    """1/64 of the voxel count rounded half-up to a multiple of 1024."""
    v = shape[0] * shape[1] * shape[2] / 64.0
    return int(math.floor(v / 1024.0 + 0.5)) * 1024


WORKLOADS = {
    "small": dict(kind="blobs", n=64, seed=1, budget=4096, iters=20, lr=1e-2, k=3.0),
    "autograd": dict(kind="grf", n=256, seed=2, budget=65536, iters=500, lr=1e-2, k=3.0),
    # the paper's Adam learning rate (8e-3) at the headline size
    "headline": dict(kind="fbm_fronts", n=1024, seed=4, budget=1_400_000, iters=2000,
                     iters_reduced=300, lr=8e-3, k=3.0),
}


# --------------------------------------------------------------------------
# Rendering inputs: cameras and transfer functions
# --------------------------------------------------------------------------
def orbit_camera(shape, azimuth_deg: float, elevation_deg: float, distance: float = 2.0, fovy_deg: float = 40.0):
    """Pinhole camera on a sphere around the grid centre, looking at it, in
    voxel coordinates (voxel centres at integers).  shape = (nz, ny, nx);
    distance in units of the longest axis.  Returns float32 (eye, right, up,
    forward) and tan(fovy / 2), the tuple the renderers take."""
    nz, ny, nx = shape
    c = np.array([(nx - 1) / 2.0, (ny - 1) / 2.0, (nz - 1) / 2.0])
    az, el = math.radians(azimuth_deg), math.radians(elevation_deg)
    off = np.array([math.cos(el) * math.cos(az), math.cos(el) * math.sin(az), math.sin(el)])
    eye = c + distance * max(nx, ny, nz) * off
    fwd = c - eye
    fwd /= np.linalg.norm(fwd)
    world_up = np.array([0.0, 0.0, 1.0]) if abs(fwd[2]) < 0.99 else np.array([0.0, 1.0, 0.0])
    right = np.cross(fwd, world_up)
    right /= np.linalg.norm(right)
    up = np.cross(right, fwd)
    f32 = lambda a: np.asarray(a, np.float32)
    return f32(eye), f32(right), f32(up), f32(fwd), float(np.float32(math.tan(math.radians(fovy_deg) / 2.0)))


def transfer_function(n: int = 256, seed: int = 0, max_alpha: float = 0.35) -> np.ndarray:
    """(n, 4) float32 RGBA table over V in [0, 1]: colours from 9 random
    control points (PCG64 seed), opacity rising as V^1.5 with two random
    bumps, scaled to max_alpha."""
    rng = np.random.Generator(np.random.PCG64(seed))
    x = np.linspace(0.0, 1.0, n)
    ctrl = np.linspace(0.0, 1.0, 9)
    rgb = np.stack([np.interp(x, ctrl, rng.uniform(0.05, 1.0, 9)) for _ in range(3)], axis=1)
    a = x ** 1.5
    for _ in range(2):
        m, w = rng.uniform(0.2, 0.9), rng.uniform(0.03, 0.1)
        a = a + 0.8 * np.exp(-0.5 * ((x - m) / w) ** 2)
    a = max_alpha * a / a.max()
    return np.ascontiguousarray(np.concatenate([rgb, a[:, None]], axis=1), np.float32)
