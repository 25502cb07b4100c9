"""ctypes shim over the FP64 CPU oracle (gve_oracle.c).

TEST INFRASTRUCTURE ONLY: the test-suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers.  Nothing in the product
package imports this module, and this module imports nothing from the product
package.

Every function states the paper passage it follows (arxiv 2608.14112); the C
source holds the arithmetic.  Arrays: fields are float32 ``(nz, ny, nx)``
(x fastest, voxel (i,j,k) centred at (i,j,k), Sec. III-B); primitive records
are ``(N, 12)`` in the order ``mu(3), log s(3), q(w,x,y,z), a, w_logit``
(Sec. III-C, Eq. 2; 48 bytes per primitive in float32, Sec. III-J).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from pathlib import Path

import numpy as np

_HERE = Path(__file__).resolve().parent
_SRC = _HERE / "gve_oracle.c"
_BUILD = _HERE / "_build"
_SO = _BUILD / "libgve_oracle.so"
_lock = threading.Lock()
_lib = None

CFLAGS = ["-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
          "-fexcess-precision=standard", "-std=gnu11"]


def build(force: bool = False) -> Path:
    """Compile the oracle with gcc (no FMA contraction: float32 decisions must
    follow the written operation order)."""
    _BUILD.mkdir(exist_ok=True)
    if force or not _SO.exists() or _SO.stat().st_mtime < _SRC.stat().st_mtime:
        tmp = _SO.with_suffix(f".{os.getpid()}.tmp.so")
        subprocess.check_call(["gcc", *CFLAGS, "-o", str(tmp), str(_SRC), "-lm"])
        os.replace(tmp, _SO)
    return _SO


class AllocStats(ctypes.Structure):
    _fields_ = [("n_occupied", ctypes.c_int64), ("n_eligible", ctypes.c_int64),
                ("n_detail", ctypes.c_int64), ("n_coverage", ctypes.c_int64),
                ("feasible_max", ctypes.c_int64), ("gbar", ctypes.c_double),
                ("h_detail", ctypes.c_double), ("h_coverage", ctypes.c_double)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(str(build()))
            P = ctypes.c_void_p
            i64, i32, f32, f64, u64, u32 = (ctypes.c_int64, ctypes.c_int, ctypes.c_float,
                                            ctypes.c_double, ctypes.c_uint64, ctypes.c_uint32)
            L.or_philox4x32_10.argtypes = [P, P, P]
            L.or_pred_t.argtypes = [P, i32, i32, i32]
            L.or_pred_t.restype = f32
            L.or_exp_fixed.argtypes = [f32]
            L.or_exp_fixed.restype = f32
            L.or_pred_threshold.argtypes = [f32]
            L.or_pred_threshold.restype = f32
            L.or_eval_region.argtypes = [P, P, i64, P, P, P, f32, f64, i32, i32, P, P, P]
            L.or_eval_region.restype = i32
            L.or_loss_grad.argtypes = [P, P, i64, P, P, f32, f64, i32, i32, f64, P, P]
            L.or_loss_grad.restype = f64
            L.or_grad_subset.argtypes = [P, i64, P, P, f32, f64, i32, f64, P, i64, P]
            L.or_grad_subset.restype = i32
            L.or_backward.argtypes = [P, i64, P, P, f32, f64, i32, P]
            L.or_backward.restype = i32
            L.or_count_kept.argtypes = [P, i64, P, f32]
            L.or_count_kept.restype = i64
            L.or_adam.argtypes = [P, P, P, P, i64, i32, f64, f64, f64, f64]
            L.or_refine.argtypes = [P, i64, P, P, f32, f64, i32, f64, i32, f64, f64, f64, f64, P]
            L.or_refine.restype = f64
            L.or_bin_count.argtypes = [P, i64, P, f32, i32, P]
            L.or_bin_count.restype = i64
            L.or_bin_emit.argtypes = [P, i64, P, f32, i32, P, P]
            L.or_bin_emit.restype = i64
            L.or_sample_classes.argtypes = [P, P, P, P, P, P]
            L.or_sample_classes.restype = None
            L.or_sample_split.argtypes = [i64, P]
            L.or_sample_split.restype = None
            L.or_draw_samples.argtypes = [P, P, P, i64, P, i64, i64, u64, u32, P, P, P]
            L.or_draw_samples.restype = None
            L.or_sample_loss_grad.argtypes = [P, i64, P, P, i64, f32, f64, f64, P, P]
            L.or_sample_loss_grad.restype = f64
            L.or_refine_sampled.argtypes = [P, i64, P, P, i64, u64, i32, f32, f64, f64, i32, f64, f64, f64, f64, P]
            L.or_refine_sampled.restype = i32
            L.or_kept_submasks.argtypes = [P, P, f32, i32, i64, P, P, P]
            L.or_kept_submasks.restype = None
            L.or_draw_partners.argtypes = [P, i64, P, u64, u32, f32, P]
            L.or_draw_partners.restype = None
            L.or_lambda_sm.argtypes = [f64, f64, i32, i32]
            L.or_lambda_sm.restype = f64
            L.or_sample_objective.argtypes = [P, i64, P, P, i64, i32, P, P, P, f32, f64, f64, P, P]
            L.or_sample_objective.restype = f64
            L.or_refine_sampled_reg.argtypes = [P, i64, P, P, i64, u64, i32, f32, f64, f64, i32, f64, f64, f64, f64,
                                                P, P]
            L.or_refine_sampled_reg.restype = i32
            L.or_ray_setup.argtypes = [P, i32, i32, i32, i32, P, P, P, P]
            L.or_ray_setup.restype = i32
            L.or_field_at.argtypes = [P, i64, f32, f64, i32, P, P, P, P]
            L.or_field_at.restype = i32
            L.or_render.argtypes = [P, i64, P, f32, f64, i32, P, i32, i32, P, P, i32, P, i64, P, P, P]
            L.or_render.restype = i32
            L.or_grad_mag32.argtypes = [P, P, P]
            L.or_struct_tensor.argtypes = [P, P, i32, i32, i32, P]
            L.or_jacobi3.argtypes = [P, P, P]
            L.or_quat_from_R.argtypes = [P, P]
            L.or_canonical_frame.argtypes = [P, P]
            L.or_trilinear.argtypes = [P, P, f64, f64, f64]
            L.or_trilinear.restype = f64
            L.or_feasible_max.argtypes = [i64, f64, i64, i64]
            L.or_feasible_max.restype = i64
            L.or_detail_key.argtypes = [u64, u64, f32]
            L.or_detail_key.restype = f64
            L.or_coverage_key.argtypes = [u64, u64]
            L.or_coverage_key.restype = u64
            L.or_jitter.argtypes = [u64, u32, u64, P]
            L.or_group_spacing.argtypes = [P, i64, P, i64, i64]
            L.or_group_spacing.restype = f64
            L.or_allocate.argtypes = [P, P, i64, f64, f32, f64, u64, P, P, ctypes.POINTER(AllocStats)]
            L.or_allocate.restype = i32
            L.or_eval_blocks.argtypes = [P, i64, P, i64, P, P, f32, f64, i32, P]
            L.or_eval_blocks.restype = i32
            L.or_grad_mag32_at.argtypes = [P, P, P, i64, P]
            L.or_grad_mag32_at.restype = None
            L.or_assemble_seeds.argtypes = [P, P, P, P, P, i64, u64, f64, f64, f64, f64, P]
            L.or_assemble_seeds.restype = None
            L.or_draw_census.argtypes = [P, P, f32, u64, f64, i64, u64, i64, f32, P]
            L.or_draw_census.restype = None
            L.or_detail_keys.argtypes = [P, P, i64, u64, P]
            L.or_detail_keys.restype = None
            L.or_coverage_keys.argtypes = [P, i64, u64, P]
            L.or_coverage_keys.restype = None
            L.or_jitter_many.argtypes = [i64, u32, u64, P]
            L.or_jitter_many.restype = None
            L.or_list_kept.argtypes = [P, i64, P, f32, P, i64]
            L.or_list_kept.restype = i64
            L.or_normalize.argtypes = [P, i64, P, P]
            L.or_normalize.restype = i32
            _lib = L
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _dims(field_or_dims):
    if isinstance(field_or_dims, np.ndarray) and field_or_dims.ndim == 3:
        nz, ny, nx = field_or_dims.shape
        return np.array([nx, ny, nz], dtype=np.int32)
    return np.asarray(field_or_dims, dtype=np.int32).reshape(3)


def _prm64(prm) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(prm, dtype=np.float64).reshape(-1, 12))


def _f32c(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float32))


# --------------------------------------------------------------------------
# Random numbers: Philox4x32-10 (Salmon et al., SC'11)
# --------------------------------------------------------------------------
def philox4x32_10(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(np.asarray(ctr, dtype=np.uint32).reshape(4))
    k = np.ascontiguousarray(np.asarray(key, dtype=np.uint32).reshape(2))
    out = np.zeros(4, dtype=np.uint32)
    lib().or_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


# --------------------------------------------------------------------------
# Field (Sec. III-C, Eq. 3)
# --------------------------------------------------------------------------
def pred_threshold(k: float) -> float:
    """float32 threshold T of the kept-pair test t > T."""
    return float(lib().or_pred_threshold(float(k)))


def exp_fixed(x: float) -> float:
    """The float32 exponential both sides use for the scales of the keep
    coefficients (a fixed sequence of correctly rounded operations)."""
    return float(lib().or_exp_fixed(float(x)))


def pred_t(p32_record, x: int, y: int, z: int) -> float:
    """float32 exponent t of the kept-pair test for one voxel."""
    r = _f32c(p32_record).reshape(12)
    return float(lib().or_pred_t(_ptr(r), int(x), int(y), int(z)))


def eval_region(prm, dims, region=None, k=3.0, rho0=0.05, normalized=True, truncated=True,
                pred_prm=None):
    """Eq. 3 on a sub-box ``region = ((x0,y0,z0), (sx,sy,sz))`` (whole grid by
    default).  Returns (num, den, vtilde) as float64 ``(sz, sy, sx)``."""
    d = _dims(dims)
    if region is None:
        r0, rs = np.zeros(3, np.int32), d.copy()
    else:
        r0 = np.asarray(region[0], np.int32).reshape(3)
        rs = np.asarray(region[1], np.int32).reshape(3)
    p = _prm64(prm)
    pp = _prm64(pred_prm) if pred_prm is not None else None
    shape = (int(rs[2]), int(rs[1]), int(rs[0]))
    num = np.zeros(shape, np.float64)
    den = np.zeros(shape, np.float64)
    vt = np.zeros(shape, np.float64)
    rc = lib().or_eval_region(_ptr(p), _ptr(pp) if pp is not None else None, p.shape[0], _ptr(d),
                              _ptr(r0), _ptr(rs), float(k), float(rho0), int(bool(normalized)),
                              int(bool(truncated)), _ptr(num), _ptr(den), _ptr(vt))
    if rc != 0:
        raise MemoryError("oracle eval failed")
    return num, den, vt


def eval_blocks(prm, dims, corners, size, k=3.0, rho0=0.05, normalized=True):
    """Eq. 3 on many regions of one size: ``corners`` (B, 3) as (x0, y0, z0),
    ``size`` (sx, sy, sz); the records are activated once for all regions.
    Returns vtilde float64 (B, sz, sy, sx)."""
    d = _dims(dims)
    c = np.ascontiguousarray(np.asarray(corners, np.int32).reshape(-1, 3))
    rs = np.ascontiguousarray(np.asarray(size, np.int32).reshape(3))
    p = _prm64(prm)
    vt = np.zeros((c.shape[0], int(rs[2]), int(rs[1]), int(rs[0])), np.float64)
    rc = lib().or_eval_blocks(_ptr(p), p.shape[0], _ptr(d), c.shape[0], _ptr(c), _ptr(rs), float(k), float(rho0),
                              int(bool(normalized)), _ptr(vt))
    if rc != 0:
        raise MemoryError("oracle eval failed")
    return vt


def loss_grad(prm, field, k=3.0, rho0=0.05, normalized=True, truncated=True, mask_thresh=-1.0,
              pred_prm=None, want_grad=True):
    """Full-grid MSE (Eq. 6 value term, mean over voxels), its analytic
    gradient w.r.t. the raw records, and the unmasked SSE.  Returns
    (loss, grad (N,12) or None, sse)."""
    f = _f32c(field)
    d = _dims(f)
    p = _prm64(prm)
    pp = _prm64(pred_prm) if pred_prm is not None else None
    g = np.zeros_like(p) if want_grad else None
    sse = ctypes.c_double(0.0)
    L = lib().or_loss_grad(_ptr(p), _ptr(pp) if pp is not None else None, p.shape[0], _ptr(f),
                           _ptr(d), float(k), float(rho0), int(bool(normalized)),
                           int(bool(truncated)), float(mask_thresh),
                           _ptr(g) if g is not None else None, ctypes.byref(sse))
    return float(L), g, float(sse.value)


def grad_subset(prm, field, ids, k=3.0, rho0=0.05, normalized=True, mask_thresh=-1.0):
    """Gradient of the full-grid loss for the Gaussians ``ids`` only."""
    f = _f32c(field)
    d = _dims(f)
    p = _prm64(prm)
    ids = np.ascontiguousarray(np.asarray(ids, np.int64))
    g = np.zeros((ids.size, 12), np.float64)
    lib().or_grad_subset(_ptr(p), p.shape[0], _ptr(f), _ptr(d), float(k), float(rho0),
                         int(bool(normalized)), float(mask_thresh), _ptr(ids), ids.size, _ptr(g))
    return g


def backward(prm, upstream, k=3.0, rho0=0.05, normalized=True):
    """Gradient w.r.t. the raw records for an arbitrary upstream dL/dVtilde
    (float64 array shaped like the field)."""
    u = np.ascontiguousarray(np.asarray(upstream, np.float64))
    nz, ny, nx = u.shape
    d = np.array([nx, ny, nz], np.int32)
    p = _prm64(prm)
    g = np.zeros_like(p)
    lib().or_backward(_ptr(p), p.shape[0], _ptr(u), _ptr(d), float(k), float(rho0), int(bool(normalized)), _ptr(g))
    return g


def count_kept(p32, dims, k=3.0) -> int:
    """Number of kept (voxel, Gaussian) pairs of one truncated evaluation."""
    p = _f32c(p32).reshape(-1, 12)
    return int(lib().or_count_kept(_ptr(p), p.shape[0], _ptr(_dims(dims)), float(k)))


def list_kept(p32, dims, k=3.0) -> np.ndarray:
    """The kept (voxel, Gaussian) pairs of one truncated evaluation, (K, 2)
    int64 (voxel index (z ny + y) nx + x, Gaussian index), sorted."""
    p = _f32c(p32).reshape(-1, 12)
    d = _dims(dims)
    total = int(lib().or_list_kept(_ptr(p), p.shape[0], _ptr(d), float(k), None, 0))
    if total < 0:
        raise MemoryError("oracle pair listing failed")
    out = np.zeros(max(total, 1), np.uint64)
    lib().or_list_kept(_ptr(p), p.shape[0], _ptr(d), float(k), _ptr(out), total)
    v = np.sort(out[:total].astype(np.int64))
    return np.stack([v >> 24, v & ((1 << 24) - 1)], 1)


def psnr_from_sse(sse: float, M: int) -> float:
    """PSNR = 10 log10(1/MSE) for a field normalised to [0,1] (Sec. IV-C)."""
    return float(10.0 * np.log10(M / sse)) if sse > 0 else float("inf")


# --------------------------------------------------------------------------
# Optimiser (Sec. III-E: Adam)
# --------------------------------------------------------------------------
def adam_step(p, m, v, g, t, lr=1e-2, b1=0.9, b2=0.999, eps=1e-15):
    """One Adam step in place on float64 arrays (t is 1-based)."""
    for a in (p, m, v):
        assert a.dtype == np.float64 and a.flags.c_contiguous
    g = np.ascontiguousarray(g, np.float64)
    lib().or_adam(_ptr(p), _ptr(m), _ptr(v), _ptr(g), p.size, int(t), float(lr), float(b1),
                  float(b2), float(eps))


def refine(prm, field, iters, lr=1e-2, b1=0.9, b2=0.999, eps=1e-15, k=3.0, rho0=0.05,
           normalized=True, mask_thresh=-1.0):
    """Fixed-budget refinement (Sec. III-E): returns (refined records (N,12)
    float64, per-iteration losses, SSE of one extra evaluation afterwards)."""
    f = _f32c(field)
    d = _dims(f)
    p = _prm64(prm).copy()
    losses = np.zeros(max(int(iters), 1), np.float64)
    sse = lib().or_refine(_ptr(p), p.shape[0], _ptr(f), _ptr(d), float(k), float(rho0),
                          int(bool(normalized)), float(mask_thresh), int(iters), float(lr),
                          float(b1), float(b2), float(eps), _ptr(losses))
    return p, losses[:int(iters)], float(sse)


# --------------------------------------------------------------------------
# Brick binning (conservative cover of every kept pair)
# --------------------------------------------------------------------------
def bin_pairs(p32, dims, k=3.0, B=8):
    """Per-Gaussian brick counts and the (brick key, gid) pairs in
    Gaussian-major emission order."""
    p = _f32c(p32).reshape(-1, 12)
    d = _dims(dims)
    counts = np.zeros(p.shape[0], np.uint32)
    total = lib().or_bin_count(_ptr(p), p.shape[0], _ptr(d), float(k), int(B), _ptr(counts))
    keys = np.zeros(max(total, 1), np.uint32)
    gids = np.zeros(max(total, 1), np.uint32)
    n = lib().or_bin_emit(_ptr(p), p.shape[0], _ptr(d), float(k), int(B), _ptr(keys), _ptr(gids))
    assert n == total
    return counts, keys[:total], gids[:total]


def bin_sorted(p32, dims, k=3.0, B=8):
    """Pairs stably sorted by brick key, plus per-brick [start, end)."""
    d = _dims(dims)
    counts, keys, gids = bin_pairs(p32, d, k, B)
    order = np.argsort(keys, kind="stable")
    sk, sg = keys[order], gids[order]
    nb = int(np.prod([(int(d[j]) + B - 1) // B for j in range(3)]))
    start = np.searchsorted(sk, np.arange(nb, dtype=np.uint32), side="left").astype(np.uint32)
    end = np.searchsorted(sk, np.arange(nb, dtype=np.uint32), side="right").astype(np.uint32)
    empty = start == end          # empty bricks are reported as [0, 0)
    start[empty] = 0
    end[empty] = 0
    return counts, sk, sg, start, end


def kept_submasks(p32, dims, keys, gids, k=3.0, B=8) -> np.ndarray:
    """Per listed (brick, Gaussian) pair, the 8-bit set of sub-bricks
    (B x B/2 x B/4; bit = y half + 2 * z quarter) holding a kept voxel."""
    p = _f32c(p32).reshape(-1, 12)
    d = _dims(dims)
    kk = np.ascontiguousarray(keys, np.uint32)
    gg = np.ascontiguousarray(gids, np.uint32)
    out = np.zeros(max(kk.size, 1), np.uint8)
    lib().or_kept_submasks(_ptr(p), _ptr(d), float(k), int(B), int(kk.size), _ptr(kk), _ptr(gg), _ptr(out))
    return out[:kk.size]


# --------------------------------------------------------------------------
# Pre-encoding structure statistics (Sec. V-F, Table VI)
# --------------------------------------------------------------------------
def structure_function(field, lag: int) -> float:
    """S(lag): mean over the grid axes (those longer than lag) of the mean
    squared difference (V(x + lag e_a) - V(x))^2 over all voxel pairs."""
    V = np.asarray(field, np.float64)
    vals = []
    for axis in (2, 1, 0):              # x, y, z of a [nz][ny][nx] array
        n = V.shape[axis]
        if n <= lag:
            continue
        a = np.take(V, np.arange(lag, n), axis=axis)
        b = np.take(V, np.arange(0, n - lag), axis=axis)
        vals.append(float(np.mean((a - b) ** 2)))
    return float(np.mean(vals)) if vals else 0.0


def structure_stats(field, occ_thresh=0.02):
    """Table VI statistics: occupancy (V > 0.02), the share of the occupied
    voxels' gradient-magnitude mass held by the ceil(n_occ / 10) largest
    (integer ceiling), and S(1) / S(16) of the second-order structure
    function."""
    f = _f32c(field)
    occ = f > np.float32(occ_thresh)
    n_occ = int(occ.sum())
    g = grad_mag32(f)[occ].astype(np.float64)
    tot = float(g.sum())
    if n_occ and tot > 0:
        K = -(-n_occ // 10)
        top = float(np.sort(g)[n_occ - K:].sum()) / tot
    else:
        top = 0.0
    s1, s16 = structure_function(f, 1), structure_function(f, 16)
    return {"occupancy": n_occ / f.size, "grad_top10": top, "S1": s1, "S16": s16,
            "S1_over_S16": s1 / s16 if s16 > 0 else 0.0}


# --------------------------------------------------------------------------
# Stratified-sample refinement (Sec. III-F; Table III: 3,072 points per
# iteration, 35 / 40 / 25 %)
# --------------------------------------------------------------------------
def sample_classes(field):
    """(high, mid) voxel index lists: V > 0.4 and 0.02 < V <= 0.4."""
    f = _f32c(field)
    d = _dims(f)
    nh, nm = ctypes.c_int64(0), ctypes.c_int64(0)
    lib().or_sample_classes(_ptr(f), _ptr(d), None, ctypes.byref(nh), None, ctypes.byref(nm))
    hi = np.zeros(max(nh.value, 1), np.int64)
    mid = np.zeros(max(nm.value, 1), np.int64)
    lib().or_sample_classes(_ptr(f), _ptr(d), _ptr(hi), ctypes.byref(nh), _ptr(mid), ctypes.byref(nm))
    return hi[:nh.value], mid[:nm.value]


def sample_split(S: int) -> np.ndarray:
    out = np.zeros(3, np.int64)
    lib().or_sample_split(int(S), _ptr(out))
    return out


def draw_samples(field, S: int, seed: int, it: int, classes=None):
    """(points (S,3) float32, targets (S,) float32, voxel indices (S,))."""
    f = _f32c(field)
    d = _dims(f)
    hi, mid = classes if classes is not None else sample_classes(f)
    hi = np.ascontiguousarray(hi, np.int64)
    mid = np.ascontiguousarray(mid, np.int64)
    pts = np.zeros((S, 3), np.float32)
    vals = np.zeros(S, np.float32)
    vox = np.zeros(S, np.int64)
    lib().or_draw_samples(_ptr(f), _ptr(d), _ptr(hi) if hi.size else None, hi.size,
                          _ptr(mid) if mid.size else None, mid.size, int(S), int(seed), int(it),
                          _ptr(pts), _ptr(vals), _ptr(vox))
    return pts, vals, vox


def sample_loss_grad(prm, pts, vals, k=3.0, rho0=0.05, occ=0.02, want_grad=True):
    """(sampled loss, gradient (N,12) or None, Vt at the points (S,))."""
    p = _prm64(prm)
    pts = np.ascontiguousarray(pts, np.float32)
    vals = np.ascontiguousarray(vals, np.float32)
    S = vals.size
    g = np.zeros_like(p) if want_grad else None
    vt = np.zeros(S, np.float64)
    L = lib().or_sample_loss_grad(_ptr(p), p.shape[0], _ptr(pts), _ptr(vals), S, float(k), float(rho0),
                                  float(occ), _ptr(g) if g is not None else None, _ptr(vt))
    return float(L), g, vt


def refine_sampled(prm, field, iters, S=3072, seed=0, step0=0, lr=1e-2, b1=0.9, b2=0.999, eps=1e-15, k=3.0,
                   rho0=0.05, occ=0.02):
    """Stratified-sample refinement from zero Adam moments; returns the
    refined records and the per-iteration sampled losses."""
    p = _prm64(prm).copy()
    f = _f32c(field)
    losses = np.zeros(max(iters, 1), np.float64)
    st = lib().or_refine_sampled(_ptr(p), p.shape[0], _ptr(f), _ptr(_dims(f)), int(S), int(seed), int(step0),
                                 float(k), float(rho0), float(occ), int(iters), float(lr), float(b1), float(b2),
                                 float(eps), _ptr(losses))
    if st != 0:
        raise RuntimeError("oracle sampled refinement failed")
    return p, losses[:iters]


# --------------------------------------------------------------------------
# The full objective (Sec. III-F): value term plus five regularisers
# --------------------------------------------------------------------------
def draw_partners(pts, dims_zyx, seed, it, radius=1.0):
    """Jittered partners (float32, clamped to the grid) of the points
    pts (S, 3): Philox stream 5, counter (j, it)."""
    q = np.ascontiguousarray(np.asarray(pts, np.float32).reshape(-1, 3))
    nz, ny, nx = dims_zyx
    out = np.zeros_like(q)
    lib().or_draw_partners(_ptr(q), q.shape[0], _ptr(np.array([nx, ny, nz], np.int32)), int(seed), int(it),
                           float(radius), _ptr(out))
    return out


def lambda_sm(l0, l1, anneal, t):
    return lib().or_lambda_sm(float(l0), float(l1), int(anneal), int(t))


def sample_objective(prm, pts, vals, field=None, reg=None, smooth=False, k=3.0, rho0=0.05, occ=0.02,
                     want_grad=True):
    """(L, grad, terms) of the regularised sampled objective.  pts holds S
    samples and, with smooth, their S partners after them.  reg = dict with
    rho, sm (this iteration's weight), anc, aniso, cap, r_max, s_lo, s_hi."""
    q = _prm64(prm)
    pt = np.ascontiguousarray(np.asarray(pts, np.float32).reshape(-1, 3))
    vv = np.ascontiguousarray(np.asarray(vals, np.float32).ravel())
    S = vv.size
    r = dict(rho=0.0, sm=0.0, anc=0.0, aniso=0.0, cap=0.0, r_max=3.0, s_lo=0.3, s_hi=1e30)
    r.update(reg or {})
    regv = np.array([r["rho"], r["sm"], r["anc"], r["aniso"], r["cap"], r["r_max"], r["s_lo"], r["s_hi"]],
                    np.float64)
    f = None if field is None else _f32c(field)
    g = np.zeros_like(q) if want_grad else None
    terms = np.zeros(6, np.float64)
    L = lib().or_sample_objective(_ptr(q), q.shape[0], _ptr(pt), _ptr(vv), S, int(bool(smooth)),
                                  None if f is None else _ptr(f), None if f is None else _ptr(_dims(f)), _ptr(regv),
                                  float(k), float(rho0), float(occ), None if g is None else _ptr(g), _ptr(terms))
    return L, g, terms


def refine_sampled_reg(prm, field, iters, reg, S=3072, seed=0, step0=0, lr=1e-2, b1=0.9, b2=0.999, eps=1e-15,
                       k=3.0, rho0=0.05, occ=0.02):
    """Regularised stratified-sample refinement; reg = dict with rho, sm0,
    sm1, anneal, anc, aniso, cap, r_max, s_lo, s_hi, radius."""
    p = _prm64(prm).copy()
    f = _f32c(field)
    regp = np.array([reg["rho"], reg["sm0"], reg["sm1"], reg["anneal"], reg["anc"], reg["aniso"], reg["cap"],
                     reg["r_max"], reg["s_lo"], reg["s_hi"], reg["radius"]], np.float64)
    losses = np.zeros(max(iters, 1), np.float64)
    st = lib().or_refine_sampled_reg(_ptr(p), p.shape[0], _ptr(f), _ptr(_dims(f)), int(S), int(seed), int(step0),
                                     float(k), float(rho0), float(occ), int(iters), float(lr), float(b1), float(b2),
                                     float(eps), _ptr(regp), _ptr(losses))
    if st != 0:
        raise RuntimeError("oracle regularised refinement failed")
    return p, losses[:iters]


# --------------------------------------------------------------------------
# Mixture-field ray marching (Sec. III-A: the transfer function maps the
# value of Eq. 3 at each sample to colour and opacity, composited along the
# ray; grad Vt shades the sample)
# --------------------------------------------------------------------------
RENDER_DEFAULTS = dict(step=0.5, term=0.0, ref_step=1.0, background=(0.0, 0.0, 0.0), shade=False, ka=0.3,
                       kd=0.7, ks=0.2, shininess=16.0, gfloor=1e-3)


def _cam13(cam) -> np.ndarray:
    """cam = (eye, right, up, forward, tan_half_fovy) -> float32[13]."""
    eye, right, up, fwd, th = cam
    out = np.concatenate([np.asarray(eye, np.float32).ravel(), np.asarray(right, np.float32).ravel(),
                          np.asarray(up, np.float32).ravel(), np.asarray(fwd, np.float32).ravel(),
                          np.asarray([th], np.float32)])
    return np.ascontiguousarray(out, np.float32)


def _opt12(opts) -> np.ndarray:
    o = dict(RENDER_DEFAULTS, **(opts or {}))
    bg = tuple(o["background"])
    return np.array([o["step"], o["term"], o["ref_step"], bg[0], bg[1], bg[2], 1.0 if o["shade"] else 0.0,
                     o["ka"], o["kd"], o["ks"], o["shininess"], o["gfloor"]], np.float32)


def ray_setup(cam, W, H, i, j, dims_zyx):
    """(hit, unit direction, tmin, tmax) of the ray through pixel (i, j),
    float32 in the renderer's fixed order; dims_zyx = field shape."""
    c = _cam13(cam)
    nz, ny, nx = dims_zyx
    d = np.zeros(3, np.float32)
    t0, t1 = ctypes.c_float(0), ctypes.c_float(0)
    hit = lib().or_ray_setup(_ptr(c), int(W), int(H), int(i), int(j), _ptr(np.array([nx, ny, nz], np.int32)),
                             _ptr(d), ctypes.byref(t0), ctypes.byref(t1))
    return bool(hit), d, t0.value, t1.value


def field_at(prm, p, k=3.0, rho0=0.05, normalized=True):
    """Eq. 3 at a float32 point and its gradient (FP64; float32 membership),
    plus the number of kept Gaussians."""
    q = _prm64(prm)
    pt = np.ascontiguousarray(np.asarray(p, np.float32).reshape(3))
    v = ctypes.c_double(0)
    g = np.zeros(3, np.float64)
    kept = ctypes.c_int64(0)
    if lib().or_field_at(_ptr(q), q.shape[0], float(k), float(rho0), int(bool(normalized)), _ptr(pt),
                         ctypes.byref(v), _ptr(g), ctypes.byref(kept)) != 0:
        raise RuntimeError("oracle field evaluation failed")
    return v.value, g, kept.value


def render(prm, dims_zyx, cam, W, H, tf, opts=None, k=3.0, rho0=0.05, normalized=True, pixels=None,
           timing=None):
    """RGBA image (H, W, 4) in FP64 and the number of kept (sample,
    Gaussian) pairs.  tf: (n, 4) float32 table of RGBA over V in [0, 1].
    pixels (optional): flat indices j W + i; then the result is (len, 4).
    timing (optional dict) receives the seconds of the pixel loop alone."""
    q = _prm64(prm)
    c = _cam13(cam)
    o = _opt12(opts)
    t = np.ascontiguousarray(np.asarray(tf, np.float32).reshape(-1, 4))
    nz, ny, nx = dims_zyx
    pix = None if pixels is None else np.ascontiguousarray(np.asarray(pixels, np.int64).ravel())
    img = np.zeros((H, W, 4) if pix is None else (pix.size, 4), np.float64)
    kept = ctypes.c_int64(0)
    secs = ctypes.c_double(0)
    if lib().or_render(_ptr(q), q.shape[0], _ptr(np.array([nx, ny, nz], np.int32)), float(k), float(rho0),
                       int(bool(normalized)), _ptr(c), int(W), int(H), _ptr(o), _ptr(t), t.shape[0],
                       None if pix is None else _ptr(pix), 0 if pix is None else pix.size, _ptr(img),
                       ctypes.byref(kept), ctypes.byref(secs)) != 0:
        raise RuntimeError("oracle render failed (bad table, image size or step)")
    if timing is not None:
        timing["pixel_seconds"] = secs.value
    return img, kept.value


# --------------------------------------------------------------------------
# Allocation (Sec. III-E, Table I S1a..S1e, Eq. 4; Sec. V-B)
# --------------------------------------------------------------------------
def grad_mag32(field) -> np.ndarray:
    f = _f32c(field)
    g = np.zeros_like(f)
    lib().or_grad_mag32(_ptr(f), _ptr(_dims(f)), _ptr(g))
    return g


def struct_tensor(field, c) -> np.ndarray:
    """7^3 structure tensor at integer voxel c: [Jxx Jyy Jzz Jxy Jxz Jyz]."""
    f = _f32c(field)
    J = np.zeros(6, np.float64)
    lib().or_struct_tensor(_ptr(f), _ptr(_dims(f)), int(c[0]), int(c[1]), int(c[2]), _ptr(J))
    return J


def jacobi3(J6):
    J = np.ascontiguousarray(np.asarray(J6, np.float64).reshape(6))
    ev = np.zeros(3, np.float64)
    vec = np.zeros(9, np.float64)
    lib().or_jacobi3(_ptr(J), _ptr(ev), _ptr(vec))
    return ev, vec.reshape(3, 3)


def canonical_frame(evecs) -> np.ndarray:
    e = np.ascontiguousarray(np.asarray(evecs, np.float64).reshape(9))
    R = np.zeros(9, np.float64)
    lib().or_canonical_frame(_ptr(e), _ptr(R))
    return R.reshape(3, 3)


def quat_from_R(R) -> np.ndarray:
    r = np.ascontiguousarray(np.asarray(R, np.float64).reshape(9))
    q = np.zeros(4, np.float64)
    lib().or_quat_from_R(_ptr(r), _ptr(q))
    return q


def trilinear(field, p) -> float:
    f = _f32c(field)
    return float(lib().or_trilinear(_ptr(f), _ptr(_dims(f)), float(p[0]), float(p[1]), float(p[2])))


def feasible_max(N: int, detail_frac: float, n_eligible: int, n_occupied: int) -> int:
    return int(lib().or_feasible_max(int(N), float(detail_frac), int(n_eligible), int(n_occupied)))


def detail_key(v: int, seed: int, g: float) -> float:
    return float(lib().or_detail_key(int(v), int(seed), float(g)))


def coverage_key(v: int, seed: int) -> int:
    return int(lib().or_coverage_key(int(v), int(seed)))


def jitter(i: int, group: int, seed: int) -> np.ndarray:
    u = np.zeros(3, np.float32)
    lib().or_jitter(int(i), int(group), int(seed), _ptr(u))
    return u


def group_spacing(vox, dims, n_occupied, N) -> float:
    v = np.ascontiguousarray(np.asarray(vox, np.int64))
    return float(lib().or_group_spacing(_ptr(v), v.size, _ptr(_dims(dims)), int(n_occupied), int(N)))


def grad_mag32_at(field, vox) -> np.ndarray:
    """The allocator's float32 |grad V| (S1a) at listed voxel indices."""
    f = _f32c(field)
    v = np.ascontiguousarray(np.asarray(vox, np.int64))
    out = np.zeros(v.size, np.float32)
    lib().or_grad_mag32_at(_ptr(f), _ptr(_dims(f)), _ptr(v), v.size, _ptr(out))
    return out


def detail_keys(vox, g, seed: int) -> np.ndarray:
    """Efraimidis-Spirakis keys of the detail draw at listed voxels."""
    v = np.ascontiguousarray(np.asarray(vox, np.int64))
    gg = _f32c(g).reshape(-1)
    out = np.zeros(v.size, np.float64)
    lib().or_detail_keys(_ptr(v), _ptr(gg), v.size, int(seed), _ptr(out))
    return out


def coverage_keys(vox, seed: int) -> np.ndarray:
    """Philox keys of the coverage draw at listed voxels."""
    v = np.ascontiguousarray(np.asarray(vox, np.int64))
    out = np.zeros(v.size, np.uint64)
    lib().or_coverage_keys(_ptr(v), v.size, int(seed), _ptr(out))
    return out


def jitter_many(n: int, group: int, seed: int) -> np.ndarray:
    """Jitter (Eq. 4) of seeds 0..n-1 of a group: (n, 3) float32."""
    out = np.zeros((int(n), 3), np.float32)
    lib().or_jitter_many(int(n), int(group), int(seed), _ptr(out))
    return out


def draw_census(field, seed: int, kd: float, kd_idx: int, ku: int, ku_idx: int, gbar: float,
                occ_thresh: float = 0.02) -> dict:
    """Exhaustive counts over the whole grid for checking a draw made
    elsewhere (S1b): occupied and eligible voxels, eligible voxels whose
    (detail key, index) is at most (kd, kd_idx), occupied voxels whose
    (coverage key, index) is at most (ku, ku_idx), and occupied voxels with
    |grad V| below / at most gbar."""
    f = _f32c(field)
    out = np.zeros(6, np.int64)
    lib().or_draw_census(_ptr(f), _ptr(_dims(f)), float(np.float32(occ_thresh)), int(seed), float(kd), int(kd_idx),
                         int(ku), int(ku_idx), float(np.float32(gbar)), _ptr(out))
    return dict(zip(("n_occupied", "n_eligible", "detail_at_most", "coverage_at_most", "g_below", "g_at_most"),
                    (int(x) for x in out)))


def assemble_seeds(field, vox, gi, grp, seed: int, h_detail: float, h_coverage: float, gbar: float,
                   w0: float = 0.1) -> np.ndarray:
    """S1d + S1e of listed seeds (voxel, index within its group, group 0 =
    detail / 1 = coverage) with given group spacings and median: the records
    the allocation gives those seeds, (n, 12) float64."""
    f = _f32c(field)
    v = np.ascontiguousarray(np.asarray(vox, np.int64))
    i = np.ascontiguousarray(np.asarray(gi, np.int64))
    g = np.ascontiguousarray(np.asarray(grp, np.int32))
    out = np.zeros((v.size, 12), np.float64)
    lib().or_assemble_seeds(_ptr(f), _ptr(_dims(f)), _ptr(v), _ptr(i), _ptr(g), v.size, int(seed), float(h_detail),
                            float(h_coverage), float(gbar), float(w0), _ptr(out))
    return out


def normalize(field):
    """Stage P (Sec. III-B): (V - min) / (max - min) in float32, correctly
    rounded per operation (a constant field maps to 0).  Returns (field,
    (min, max)); raises ValueError on a non-finite value."""
    f = _f32c(field)
    out = np.empty_like(f)
    mm = np.zeros(2, np.float32)
    if lib().or_normalize(_ptr(f), f.size, _ptr(out), _ptr(mm)) != 0:
        raise ValueError("non-finite value in the field")
    return out, (float(mm[0]), float(mm[1]))


def allocate(field, N, detail_frac=0.55, occ_thresh=0.02, w0=0.1, seed=0):
    """Analytic fixed-budget allocation.  Returns (records (N,12) float64,
    chosen voxel indices (N,), stats dict, status) with status 0 = ok,
    2 = infeasible budget (records empty, stats['feasible_max'] set)."""
    f = _f32c(field)
    d = _dims(f)
    prm = np.zeros((max(int(N), 1), 12), np.float64)
    vox = np.zeros(max(int(N), 1), np.int64)
    st = AllocStats()
    rc = lib().or_allocate(_ptr(f), _ptr(d), int(N), float(detail_frac), float(np.float32(occ_thresh)),
                           float(w0), int(seed), _ptr(prm), _ptr(vox), ctypes.byref(st))
    stats = {name: getattr(st, name) for name, _ in AllocStats._fields_}
    if rc == 1:
        raise MemoryError("oracle allocation failed")
    if rc == 2:
        return np.zeros((0, 12)), np.zeros(0, np.int64), stats, 2
    return prm[:int(N)], vox[:int(N)], stats, 0
