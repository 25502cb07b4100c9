"""Thin Python binding of libgve (include/gve.h) -- argument marshalling only.

Every step of the encoder runs in the CUDA kernels of ``libgve.so``; this
module only checks tensor shapes, dtypes and devices, passes raw device
pointers and the current torch stream through ctypes, and turns status codes
into exceptions.  There is no CPU fallback: without the built library or a
CUDA device every call raises.

Names follow the C ABI: ``gve_allocate``, ``gve_evaluate``, ``gve_loss_grad``,
``gve_backward``, ``gve_refine``, ``gve_bin``, ``gve_count_pairs``.
Primitive records are float32 ``(N, 12)`` tensors in the order
``mu(3), log s(3), q(w,x,y,z), a, w_logit`` (48 bytes each, Eq. 2 / Eq. 7 of
arxiv 2608.14112); fields are float32 ``(nz, ny, nx)``, x fastest.
"""
from __future__ import annotations

import ctypes
import threading
from dataclasses import dataclass
from pathlib import Path

import torch

_HERE = Path(__file__).resolve().parent
LIB_PATH = _HERE / "libgve.so"

GVE_OK, GVE_E_INVALID, GVE_E_BUDGET, GVE_E_NOMEM, GVE_E_CUDA, GVE_E_TIMEOUT, GVE_E_CAPACITY, GVE_E_INTERNAL = range(8)


class GveError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"libgve status {status}: {msg}")
        self.status = status


class BudgetError(GveError):
    """The field cannot support the requested budget (paper Sec. V-B)."""

    def __init__(self, msg: str, feasible_max: int):
        super().__init__(GVE_E_BUDGET, msg)
        self.feasible_max = feasible_max


class Dims(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32)]


class EvalOpts(ctypes.Structure):
    _fields_ = [("trunc_k", ctypes.c_float), ("rho0", ctypes.c_float), ("normalized", ctypes.c_int32),
                ("brick", ctypes.c_int32), ("gaussians_per_block", ctypes.c_int32)]


class AllocOpts(ctypes.Structure):
    _fields_ = [("detail_frac", ctypes.c_double), ("w0", ctypes.c_double), ("occ_thresh", ctypes.c_float),
                ("reserved", ctypes.c_int32), ("seed", ctypes.c_uint64)]


class Schedule(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int32), ("lr", ctypes.c_float), ("beta1", ctypes.c_float),
                ("beta2", ctypes.c_float), ("eps", ctypes.c_float), ("mask_thresh", ctypes.c_float),
                ("step0", ctypes.c_int32), ("eval", EvalOpts)]


class Stats(ctypes.Structure):
    _fields_ = [("loss_first", ctypes.c_double), ("loss_last", ctypes.c_double), ("sse_final", ctypes.c_double),
                ("psnr_final", ctypes.c_double), ("brick_pairs", ctypes.c_int64), ("launches", ctypes.c_int64),
                ("iters_done", ctypes.c_int32), ("retries", ctypes.c_int32), ("ms_total", ctypes.c_float),
                ("ms_brick", ctypes.c_float), ("ms_bin", ctypes.c_float), ("ms_fwd", ctypes.c_float)]


class Volume(ctypes.Structure):
    _fields_ = [("field_dev", ctypes.c_void_p), ("dims", Dims), ("n", ctypes.c_int64)]


class AllocInfo(ctypes.Structure):
    _fields_ = [("n_occupied", ctypes.c_int64), ("n_eligible", ctypes.c_int64), ("n_detail", ctypes.c_int64),
                ("n_coverage", ctypes.c_int64), ("gbar", ctypes.c_double), ("h_detail", ctypes.c_double),
                ("h_coverage", ctypes.c_double)]


_lock = threading.Lock()
_lib = None
_ctx = {}


def lib():
    """Load libgve.so (raises if it was not built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not LIB_PATH.exists():
                raise RuntimeError(f"{LIB_PATH} is missing: run paper_2608_14112_b300/build.py (no CPU fallback)")
            L = ctypes.CDLL(str(LIB_PATH))
            P, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
            st = ctypes.c_int
            L.gve_ctx_create.argtypes = [ctypes.POINTER(P), i32]
            L.gve_ctx_create.restype = st
            L.gve_ctx_destroy.argtypes = [P]
            L.gve_ctx_destroy.restype = None
            L.gve_status_str.argtypes = [st]
            L.gve_status_str.restype = ctypes.c_char_p
            L.gve_last_error.argtypes = [P]
            L.gve_last_error.restype = ctypes.c_char_p
            L.gve_allocate.argtypes = [P, P, Dims, i64, ctypes.POINTER(AllocOpts), P, ctypes.POINTER(i64),
                                       ctypes.POINTER(AllocInfo), P]
            L.gve_evaluate.argtypes = [P, P, i64, Dims, ctypes.POINTER(EvalOpts), P, P]
            L.gve_loss_grad.argtypes = [P, P, i64, P, Dims, ctypes.POINTER(EvalOpts), ctypes.c_float, P, P, P]
            L.gve_backward.argtypes = [P, P, i64, Dims, ctypes.POINTER(EvalOpts), P, P, P]
            L.gve_refine.argtypes = [P, P, i64, P, Dims, ctypes.POINTER(Schedule), P, P, ctypes.POINTER(Stats), P]
            L.gve_render_prepare.argtypes = [P, P, i64, Dims, P, P]
            L.gve_render_prepare.restype = st
            L.gve_render.argtypes = [P, P, P, P, P, P, P]
            L.gve_render.restype = st
            L.gve_structure_stats.argtypes = [P, P, Dims, P, P, P]
            L.gve_structure_stats.restype = st
            L.gve_draw_samples.argtypes = [P, P, Dims, i64, ctypes.c_uint64, ctypes.c_uint32, P, P, P]
            L.gve_draw_samples.restype = st
            L.gve_draw_partners.argtypes = [P, P, i64, Dims, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_float, P, P]
            L.gve_draw_partners.restype = st
            L.gve_sample_loss_grad.argtypes = [P, P, i64, Dims, ctypes.POINTER(EvalOpts), P, i64, ctypes.c_float,
                                               P, P, P, P, P, P, P]
            L.gve_sample_loss_grad.restype = st
            L.gve_refine_sampled.argtypes = [P, P, i64, P, Dims, ctypes.POINTER(Schedule), i64, ctypes.c_uint64, P,
                                             P, P, P, P]
            L.gve_refine_sampled.restype = st
            L.gve_bin.argtypes = [P, P, i64, Dims, ctypes.POINTER(EvalOpts), P, P, P, P, i64, P, ctypes.POINTER(i64), P]
            L.gve_count_pairs.argtypes = [P, P, i64, Dims, ctypes.POINTER(EvalOpts), ctypes.POINTER(i64),
                                          ctypes.POINTER(i64), P]
            L.gve_evaluate_noalloc.argtypes = [P, i64, Dims, ctypes.POINTER(EvalOpts), P, P]
            L.gve_kept_pairs.argtypes = [P, P, i64, Dims, ctypes.POINTER(EvalOpts), P, i64, ctypes.POINTER(i64), P]
            L.gve_normalize.argtypes = [P, P, Dims, P, P, P]
            L.gve_peak_bench.argtypes = [i32, i64, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_float), P]
            L.gve_refine_batch.argtypes = [P, i32, ctypes.POINTER(Volume), P, ctypes.POINTER(Schedule), P, P, P,
                                           ctypes.POINTER(Stats), P]
            L.gve_autotune.argtypes = [P, i32, ctypes.POINTER(Volume), P, ctypes.POINTER(EvalOpts), P, P]
            L.gve_allocate_batch.argtypes = [P, i32, ctypes.POINTER(Volume), ctypes.POINTER(AllocOpts), P,
                                             ctypes.POINTER(AllocInfo), P]
            L.gve_allocate_batch.restype = st
            for f in ("gve_allocate", "gve_evaluate", "gve_loss_grad", "gve_backward", "gve_refine", "gve_bin",
                      "gve_count_pairs", "gve_evaluate_noalloc", "gve_refine_batch", "gve_autotune", "gve_kept_pairs",
                      "gve_normalize", "gve_peak_bench"):
                getattr(L, f).restype = st
            _lib = L
    return _lib


def context(device: int | None = None) -> ctypes.c_void_p:
    """Per-device library context (created on first use)."""
    if not torch.cuda.is_available():
        raise RuntimeError("libgve needs a CUDA device (no CPU fallback)")
    dev = torch.cuda.current_device() if device is None else int(device)
    with _lock:
        c = _ctx.get(dev)
    if c is None:
        h = ctypes.c_void_p()
        s = lib().gve_ctx_create(ctypes.byref(h), dev)
        if s != GVE_OK:
            raise GveError(s, "gve_ctx_create failed")
        with _lock:
            _ctx[dev] = h
        c = h
    return c


def _check(s: int, ctx) -> None:
    if s != GVE_OK:
        raise GveError(s, lib().gve_last_error(ctx).decode())


def _ptr(t: torch.Tensor | None):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _stream(dev: torch.device):
    return ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream)


def _prims(p: torch.Tensor) -> torch.Tensor:
    if p.dtype != torch.float32 or p.dim() != 2 or p.shape[1] != 12 or not p.is_cuda or not p.is_contiguous():
        raise ValueError("primitives must be a contiguous CUDA float32 tensor of shape (N, 12)")
    return p


def _field(f: torch.Tensor) -> torch.Tensor:
    if f.dtype != torch.float32 or f.dim() != 3 or not f.is_cuda or not f.is_contiguous():
        raise ValueError("field must be a contiguous CUDA float32 tensor of shape (nz, ny, nx)")
    return f


def _dims(shape) -> Dims:
    nz, ny, nx = (int(s) for s in shape)
    return Dims(nx, ny, nz)


@dataclass
class EvalOptions:
    trunc_k: float = 3.0
    rho0: float = 0.05
    normalized: bool = True
    brick: int = 8
    gaussians_per_block: int = 0

    def c(self) -> EvalOpts:
        return EvalOpts(float(self.trunc_k), float(self.rho0), int(bool(self.normalized)), int(self.brick),
                        int(self.gaussians_per_block))


def gve_evaluate(prims: torch.Tensor, shape, opts: EvalOptions | None = None, out: torch.Tensor | None = None):
    """Eq. 3 at every voxel centre of a grid of ``shape = (nz, ny, nx)``."""
    prims = _prims(prims)
    o = (opts or EvalOptions()).c()
    if out is None:
        out = torch.empty(tuple(int(s) for s in shape), dtype=torch.float32, device=prims.device)
    _field(out)
    c = context(prims.device.index)
    _check(lib().gve_evaluate(c, _ptr(prims), prims.shape[0], _dims(out.shape), ctypes.byref(o), _ptr(out),
                              _stream(prims.device)), c)
    return out


def gve_loss_grad(prims: torch.Tensor, field: torch.Tensor, opts: EvalOptions | None = None,
                  mask_thresh: float = -1.0):
    """(dL/dprims (N,12), sse (2,) float64 = {masked, unmasked}) of the
    full-grid mean squared error at the current parameters."""
    prims, field = _prims(prims), _field(field)
    o = (opts or EvalOptions()).c()
    grad = torch.empty_like(prims)
    sse = torch.empty(2, dtype=torch.float64, device=prims.device)
    c = context(prims.device.index)
    _check(lib().gve_loss_grad(c, _ptr(prims), prims.shape[0], _ptr(field), _dims(field.shape), ctypes.byref(o),
                               float(mask_thresh), _ptr(grad), _ptr(sse), _stream(prims.device)), c)
    return grad, sse


def gve_backward(prims: torch.Tensor, grad_field: torch.Tensor, opts: EvalOptions | None = None):
    """dL/dprims for an arbitrary upstream dL/dVtilde (recomputes per brick)."""
    prims, grad_field = _prims(prims), _field(grad_field)
    o = (opts or EvalOptions()).c()
    grad = torch.empty_like(prims)
    c = context(prims.device.index)
    _check(lib().gve_backward(c, _ptr(prims), prims.shape[0], _dims(grad_field.shape), ctypes.byref(o),
                              _ptr(grad_field), _ptr(grad), _stream(prims.device)), c)
    return grad


def gve_refine(prims: torch.Tensor, field: torch.Tensor, iters: int, lr: float = 1e-2, beta1: float = 0.9,
               beta2: float = 0.999, eps: float = 1e-15, mask_thresh: float = -1.0, step0: int = 0,
               opts: EvalOptions | None = None, adam_state: torch.Tensor | None = None,
               trace: torch.Tensor | None = None, want_stats: bool = True):
    """Fixed-budget refinement in place on ``prims``.  Returns a dict of the
    host statistics (or None when ``want_stats`` is False: no synchronisation
    beyond the capacity checks)."""
    prims, field = _prims(prims), _field(field)
    sched = Schedule(int(iters), float(lr), float(beta1), float(beta2), float(eps), float(mask_thresh), int(step0),
                     (opts or EvalOptions()).c())
    if adam_state is not None:
        if adam_state.shape != (2, prims.shape[0], 12) or adam_state.dtype != torch.float32 or not adam_state.is_contiguous():
            raise ValueError("adam_state must be float32 (2, N, 12)")
    if trace is not None and (trace.dtype != torch.float64 or trace.numel() < iters or not trace.is_cuda):
        raise ValueError("trace must be a CUDA float64 tensor with >= iters entries")
    st = Stats()
    c = context(prims.device.index)
    _check(lib().gve_refine(c, _ptr(prims), prims.shape[0], _ptr(field), _dims(field.shape), ctypes.byref(sched),
                            _ptr(adam_state), _ptr(trace), ctypes.byref(st) if want_stats else None,
                            _stream(prims.device)), c)
    if not want_stats:
        return None
    return {name: getattr(st, name) for name, _ in Stats._fields_}


class Camera(ctypes.Structure):
    _fields_ = [("eye", ctypes.c_float * 3), ("right", ctypes.c_float * 3), ("up", ctypes.c_float * 3),
                ("forward", ctypes.c_float * 3), ("tan_half_fovy", ctypes.c_float), ("width", ctypes.c_int32),
                ("height", ctypes.c_int32)]


class RenderOpts(ctypes.Structure):
    _fields_ = [("step", ctypes.c_float), ("term", ctypes.c_float), ("ref_step", ctypes.c_float),
                ("background", ctypes.c_float * 3), ("shade", ctypes.c_int32), ("ka", ctypes.c_float),
                ("kd", ctypes.c_float), ("ks", ctypes.c_float), ("shininess", ctypes.c_float),
                ("gfloor", ctypes.c_float), ("tf_dev", ctypes.c_void_p), ("tf_n", ctypes.c_int32)]


@dataclass
class RenderOptions:
    step: float = 0.5
    term: float = 0.0
    ref_step: float = 1.0
    background: tuple = (0.0, 0.0, 0.0)
    shade: bool = False
    ka: float = 0.3
    kd: float = 0.7
    ks: float = 0.2
    shininess: float = 16.0
    gfloor: float = 1e-3


def gve_render_prepare(prims: torch.Tensor, shape, opts: EvalOptions | None = None) -> None:
    """Builds the ray marcher's cell lists for a primitive set on a grid of
    ``shape = (nz, ny, nx)`` (the context keeps its own copy)."""
    prims = _prims(prims)
    o = (opts or EvalOptions()).c()
    c = context(prims.device.index)
    _check(lib().gve_render_prepare(c, _ptr(prims), prims.shape[0], _dims(shape), ctypes.byref(o),
                                    _stream(prims.device)), c)


def gve_render(camera, width: int, height: int, tf: torch.Tensor, opts: RenderOptions | None = None,
               device=None, out: torch.Tensor | None = None, want_kept: bool = False, want_tested: bool = False):
    """RGBA image (height, width, 4) of the prepared set.  camera = (eye,
    right, up, forward, tan_half_fovy) in voxel coordinates; tf = (n, 4)
    float32 CUDA tensor over V in [0, 1].  With want_kept the kept (sample,
    Gaussian) pairs follow the image, with want_tested also the tested
    pairs."""
    o = opts or RenderOptions()
    if tf.dtype != torch.float32 or tf.dim() != 2 or tf.shape[1] != 4 or not tf.is_cuda or not tf.is_contiguous():
        raise ValueError("tf must be a contiguous CUDA float32 tensor of shape (n, 4)")
    dev = tf.device if device is None else torch.device(device)
    eye, right, up, fwd, th = camera
    cam = Camera((ctypes.c_float * 3)(*map(float, eye)), (ctypes.c_float * 3)(*map(float, right)),
                 (ctypes.c_float * 3)(*map(float, up)), (ctypes.c_float * 3)(*map(float, fwd)), float(th),
                 int(width), int(height))
    ro = RenderOpts(float(o.step), float(o.term), float(o.ref_step), (ctypes.c_float * 3)(*map(float, o.background)),
                    int(bool(o.shade)), float(o.ka), float(o.kd), float(o.ks), float(o.shininess), float(o.gfloor),
                    tf.data_ptr(), int(tf.shape[0]))
    if out is None:
        out = torch.empty((int(height), int(width), 4), dtype=torch.float32, device=dev)
    kept, tested = ctypes.c_int64(0), ctypes.c_int64(0)
    want_kept = want_kept or want_tested
    c = context(dev.index)
    _check(lib().gve_render(c, ctypes.byref(cam), ctypes.byref(ro), _ptr(out),
                            ctypes.byref(kept) if want_kept else None,
                            ctypes.byref(tested) if want_tested else None, _stream(dev)), c)
    if want_tested:
        return out, kept.value, tested.value
    return (out, kept.value) if want_kept else out


def gve_structure_stats(field: torch.Tensor, want_stage_ms: bool = False) -> dict:
    """Table VI statistics of a field: occupancy, top-10 % gradient-mass
    share, S(1), S(16) and their ratio (plus the device time of the two
    sweeps and of the whole pass when asked)."""
    field = _field(field)
    out = (ctypes.c_double * 5)()
    ms = (ctypes.c_double * 4)()
    c = context(field.device.index)
    _check(lib().gve_structure_stats(c, _ptr(field), _dims(field.shape), ctypes.cast(out, ctypes.c_void_p),
                                     ctypes.cast(ms, ctypes.c_void_p) if want_stage_ms else None,
                                     _stream(field.device)), c)
    res = dict(zip(("occupancy", "grad_top10", "S1", "S16", "S1_over_S16"), list(out)))
    if want_stage_ms:
        res.update(ms_sweep1=ms[0], ms_sweep2=ms[1], ms_total=ms[2], launches=int(ms[3]))
    return res


def gve_draw_samples(field: torch.Tensor, S: int, seed: int, it: int, want_voxels: bool = False):
    """The stratified points of iteration ``it``: (S, 4) float32 (x, y, z,
    target) on the field's device, plus the voxel indices when asked."""
    field = _field(field)
    pts = torch.empty((S, 4), dtype=torch.float32, device=field.device)
    vox = torch.empty(S, dtype=torch.int64, device=field.device) if want_voxels else None
    c = context(field.device.index)
    _check(lib().gve_draw_samples(c, _ptr(field), _dims(field.shape), int(S), int(seed), int(it), _ptr(pts),
                                  _ptr(vox), _stream(field.device)), c)
    return (pts, vox) if want_voxels else pts


class RegOpts(ctypes.Structure):
    _fields_ = [("lambda_rho", ctypes.c_float), ("lambda_sm", ctypes.c_float), ("lambda_sm_end", ctypes.c_float),
                ("anneal_iters", ctypes.c_int32), ("lambda_anc", ctypes.c_float), ("lambda_aniso", ctypes.c_float),
                ("lambda_cap", ctypes.c_float), ("partner_radius", ctypes.c_float), ("aniso_max", ctypes.c_float),
                ("s_lo", ctypes.c_float), ("s_hi", ctypes.c_float)]


@dataclass
class RegOptions:
    """Weights and bounds of the five regularisers of the full objective.
    The paper gives no values; these defaults were chosen by a sweep on the
    1024^3, 1.4M-Gaussian sampled schedule (1,500 iterations): the per-
    Gaussian terms are means over N, so their weights are large; the density
    term costs PSNR at any weight that moves it and is kept small."""
    lambda_rho: float = 1e-5
    lambda_sm: float = 1e-4
    lambda_sm_end: float = 1e-6
    anneal_iters: int = 1500
    lambda_anc: float = 30.0
    lambda_aniso: float = 30.0
    lambda_cap: float = 30.0
    partner_radius: float = 1.0
    aniso_max: float = 3.0
    s_lo: float = 0.3
    s_hi: float = 0.0          # <= 0: the allocator's cap (longest axis / 16)

    def c(self) -> RegOpts:
        return RegOpts(float(self.lambda_rho), float(self.lambda_sm), float(self.lambda_sm_end),
                       int(self.anneal_iters), float(self.lambda_anc), float(self.lambda_aniso),
                       float(self.lambda_cap), float(self.partner_radius), float(self.aniso_max), float(self.s_lo),
                       float(self.s_hi))


def gve_draw_partners(pts: torch.Tensor, shape, seed: int, it: int, radius: float = 1.0) -> torch.Tensor:
    """Smoothness partners (S, 4) = (x', y', z', -1) of points (S, 4)."""
    if pts.dtype != torch.float32 or pts.dim() != 2 or pts.shape[1] != 4 or not pts.is_contiguous():
        raise ValueError("points must be a contiguous float32 (S, 4) tensor")
    out = torch.empty_like(pts)
    c = context(pts.device.index)
    _check(lib().gve_draw_partners(c, _ptr(pts), pts.shape[0], _dims(shape), int(seed), int(it), float(radius),
                                   _ptr(out), _stream(pts.device)), c)
    return out


def gve_sample_loss_grad(prims: torch.Tensor, shape, pts: torch.Tensor, opts: EvalOptions | None = None,
                         occ: float = 0.02, want_grad: bool = True, reg: RegOptions | None = None,
                         field: torch.Tensor | None = None, want_terms: bool = False):
    """(objective (float64 tensor), dL/dprims (N,12) or None, Vt per sample
    [, the six unweighted terms]) at caller-given points (x, y, z, target):
    S samples, followed by S partners when reg.lambda_sm > 0."""
    prims = _prims(prims)
    if pts.dtype != torch.float32 or pts.dim() != 2 or pts.shape[1] != 4 or not pts.is_contiguous():
        raise ValueError("points must be a contiguous float32 (S, 4) tensor")
    o = (opts or EvalOptions()).c()
    smooth = reg is not None and reg.lambda_sm > 0
    if smooth and pts.shape[0] % 2:
        raise ValueError("with partners the points are S samples then S partners")
    S = pts.shape[0] // 2 if smooth else pts.shape[0]
    grad = torch.empty_like(prims) if want_grad else None
    loss = torch.zeros(1, dtype=torch.float64, device=prims.device)
    terms = torch.zeros(6, dtype=torch.float64, device=prims.device)
    vt = torch.empty(S, dtype=torch.float32, device=prims.device)
    r = reg.c() if reg is not None else None
    if field is not None:
        _field(field)
    c = context(prims.device.index)
    _check(lib().gve_sample_loss_grad(c, _ptr(prims), prims.shape[0], _dims(shape), ctypes.byref(o), _ptr(pts), S,
                                      float(occ), ctypes.byref(r) if r is not None else None, _ptr(field),
                                      _ptr(grad), _ptr(loss), _ptr(terms), _ptr(vt), _stream(prims.device)), c)
    return (loss, grad, vt, terms) if want_terms else (loss, grad, vt)


def gve_refine_sampled(prims: torch.Tensor, field: torch.Tensor, iters: int, S: int = 3072, seed: int = 0,
                       lr: float = 1e-2, beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-15,
                       occ: float = 0.02, step0: int = 0, opts: EvalOptions | None = None,
                       adam_state: torch.Tensor | None = None, trace: torch.Tensor | None = None,
                       want_stats: bool = True, reg: RegOptions | None = None):
    """Stratified-sample refinement in place on ``prims`` (the paper's training
    regime; ``reg`` adds the five regularisers of the full objective).  With
    ``want_stats`` the result includes the full-grid PSNR after the last
    step."""
    prims, field = _prims(prims), _field(field)
    sched = Schedule(int(iters), float(lr), float(beta1), float(beta2), float(eps), float(occ), int(step0),
                     (opts or EvalOptions()).c())
    if adam_state is not None:
        if adam_state.shape != (2, prims.shape[0], 12) or adam_state.dtype != torch.float32 or not adam_state.is_contiguous():
            raise ValueError("adam_state must be float32 (2, N, 12)")
    if trace is not None and (trace.dtype != torch.float64 or trace.numel() < iters or not trace.is_cuda):
        raise ValueError("trace must be a CUDA float64 tensor with >= iters entries")
    st = Stats()
    r = reg.c() if reg is not None else None
    c = context(prims.device.index)
    _check(lib().gve_refine_sampled(c, _ptr(prims), prims.shape[0], _ptr(field), _dims(field.shape),
                                    ctypes.byref(sched), int(S), int(seed), ctypes.byref(r) if r is not None else None,
                                    _ptr(adam_state), _ptr(trace), ctypes.byref(st) if want_stats else None,
                                    _stream(prims.device)), c)
    if not want_stats:
        return None
    return {name: getattr(st, name) for name, _ in Stats._fields_}


def _volumes(fields, counts):
    vols = (Volume * len(fields))()
    for i, (f, n) in enumerate(zip(fields, counts)):
        _field(f)
        vols[i] = Volume(ctypes.c_void_p(f.data_ptr()), _dims(f.shape), int(n))
    return vols


def gve_refine_batch(prims: torch.Tensor, fields, counts, iters: int, lr: float = 1e-2, beta1: float = 0.9,
                     beta2: float = 0.999, eps: float = 1e-15, mask_thresh: float = -1.0, step0: int = 0,
                     opts: EvalOptions | None = None, adam_state: torch.Tensor | None = None,
                     trace: torch.Tensor | None = None):
    """Batched refinement of ``len(fields)`` volumes whose records are
    concatenated in ``prims`` (``counts[v]`` rows each, volume order), one
    CUDA graph launch per iteration.  Returns (per-volume final PSNR list,
    stats dict)."""
    prims = _prims(prims)
    if sum(int(n) for n in counts) != prims.shape[0]:
        raise ValueError("counts must add up to the number of records")
    vols = _volumes(fields, counts)
    sched = Schedule(int(iters), float(lr), float(beta1), float(beta2), float(eps), float(mask_thresh), int(step0),
                     (opts or EvalOptions()).c())
    if adam_state is not None and (adam_state.shape != (2, prims.shape[0], 12) or not adam_state.is_contiguous()):
        raise ValueError("adam_state must be float32 (2, N, 12)")
    if trace is not None and (trace.dtype != torch.float64 or trace.numel() < iters * len(fields)):
        raise ValueError("trace must be float64 with iters * nvol entries")
    psnr = (ctypes.c_double * len(fields))()
    st = Stats()
    c = context(prims.device.index)
    _check(lib().gve_refine_batch(c, len(fields), vols, _ptr(prims), ctypes.byref(sched), _ptr(adam_state),
                                  _ptr(trace), psnr, ctypes.byref(st), _stream(prims.device)), c)
    return list(psnr), {name: getattr(st, name) for name, _ in Stats._fields_}


def gve_autotune(prims: torch.Tensor, fields, counts, opts: EvalOptions | None = None):
    """Fastest (brick, gaussians_per_block) for this batch; returns
    (EvalOptions, {(brick, chunk): ms})."""
    prims = _prims(prims)
    vols = _volumes(fields, counts)
    base = opts or EvalOptions()
    o = base.c()
    ms = (ctypes.c_float * 6)()
    c = context(prims.device.index)
    _check(lib().gve_autotune(c, len(fields), vols, _ptr(prims), ctypes.byref(o), ms, _stream(prims.device)), c)
    table = {}
    k = 0
    for b in (4, 8, 16):
        for ch in (32, 64):
            table[(b, ch)] = float(ms[k])
            k += 1
    best = EvalOptions(trunc_k=base.trunc_k, rho0=base.rho0, normalized=base.normalized, brick=int(o.brick),
                       gaussians_per_block=int(o.gaussians_per_block))
    return best, table


def gve_allocate(field: torch.Tensor, budget: int, detail_frac: float = 0.55, occ_thresh: float = 0.02,
                 w0: float = 0.1, seed: int = 0, out: torch.Tensor | None = None):
    """Analytic fixed-budget allocation (Sec. III-E).  Returns (prims (N,12),
    info dict); raises BudgetError (with ``feasible_max``) when the field
    cannot support the budget."""
    field = _field(field)
    if out is None:
        out = torch.empty((int(budget), 12), dtype=torch.float32, device=field.device)
    _prims(out)
    o = AllocOpts(float(detail_frac), float(w0), float(occ_thresh), 0, int(seed) & (2 ** 64 - 1))
    fm = ctypes.c_int64(0)
    info = AllocInfo()
    c = context(field.device.index)
    s = lib().gve_allocate(c, _ptr(field), _dims(field.shape), int(budget), ctypes.byref(o), _ptr(out),
                           ctypes.byref(fm), ctypes.byref(info), _stream(field.device))
    if s == GVE_E_BUDGET:
        raise BudgetError(lib().gve_last_error(c).decode(), int(fm.value))
    _check(s, c)
    return out, {name: getattr(info, name) for name, _ in AllocInfo._fields_}


def gve_allocate_batch(fields, budgets, detail_frac: float = 0.55, occ_thresh: float = 0.02, w0: float = 0.1,
                       seed: int = 0, out: torch.Tensor | None = None):
    """Allocation of every volume of a batch, run concurrently
    (gve_allocate_batch): volume v's ``budgets[v]`` records land in rows
    [sum(budgets[:v]), sum(budgets[:v + 1])) of one (sum(budgets), 12)
    tensor, each exactly as gve_allocate would write them.  Returns (prims,
    list of info dicts); raises GveError naming the first failing volume."""
    dev = fields[0].device
    total = int(sum(int(n) for n in budgets))
    if out is None:
        out = torch.empty((total, 12), dtype=torch.float32, device=dev)
    _prims(out)
    if out.shape[0] != total:
        raise ValueError("out must hold sum(budgets) records")
    vols = _volumes(fields, budgets)
    o = AllocOpts(float(detail_frac), float(w0), float(occ_thresh), 0, int(seed) & (2 ** 64 - 1))
    infos = (AllocInfo * len(fields))()
    c = context(dev.index)
    _check(lib().gve_allocate_batch(c, len(fields), vols, ctypes.byref(o), _ptr(out), infos, _stream(dev)), c)
    return out, [{name: getattr(inf, name) for name, _ in AllocInfo._fields_} for inf in infos]


def gve_bin(prims: torch.Tensor, shape, opts: EvalOptions | None = None, cap: int | None = None,
            with_masks: bool = False):
    """The (brick, Gaussian) pairs of the binner: (counts (N,), keys, gids,
    start, end) as int64 CPU tensors for inspection, plus the sub-brick
    masks (uint8) when ``with_masks``."""
    prims = _prims(prims)
    o = (opts or EvalOptions()).c()
    d = _dims(shape)
    B = int(o.brick)
    nb = ((d.nx + B - 1) // B) * ((d.ny + B - 1) // B) * ((d.nz + B - 1) // B)
    c = context(prims.device.index)
    dev = prims.device
    n = prims.shape[0]
    counts = torch.empty(max(n, 1), dtype=torch.int32, device=dev)
    ranges = torch.empty(2 * nb, dtype=torch.int32, device=dev)
    npairs = ctypes.c_int64(0)
    if cap is None:
        kk = torch.empty(1, dtype=torch.int32, device=dev)
        s = lib().gve_bin(c, _ptr(prims), n, d, ctypes.byref(o), _ptr(counts), _ptr(kk), _ptr(kk), None, 0,
                          _ptr(ranges), ctypes.byref(npairs), _stream(dev))
        if s not in (GVE_OK, GVE_E_CAPACITY):
            _check(s, c)
        cap = int(npairs.value)
    keys = torch.empty(max(cap, 1), dtype=torch.int32, device=dev)
    gids = torch.empty(max(cap, 1), dtype=torch.int32, device=dev)
    masks = torch.empty(max(cap, 1), dtype=torch.uint8, device=dev) if with_masks else None
    _check(lib().gve_bin(c, _ptr(prims), n, d, ctypes.byref(o), _ptr(counts), _ptr(keys), _ptr(gids),
                         _ptr(masks) if masks is not None else None, cap, _ptr(ranges), ctypes.byref(npairs),
                         _stream(dev)), c)
    m = int(npairs.value)
    u32 = lambda t: t.cpu().to(torch.int64) & 0xFFFFFFFF
    out = (u32(counts[:n]), u32(keys[:m]), u32(gids[:m]), u32(ranges[:nb]), u32(ranges[nb:]))
    return out + (masks[:m].cpu(),) if with_masks else out


def gve_count_pairs(prims: torch.Tensor, shape, opts: EvalOptions | None = None):
    """(kept pairs, candidate pairs) of one evaluation."""
    prims = _prims(prims)
    o = (opts or EvalOptions()).c()
    kept, cand = ctypes.c_int64(0), ctypes.c_int64(0)
    c = context(prims.device.index)
    _check(lib().gve_count_pairs(c, _ptr(prims), prims.shape[0], _dims(shape), ctypes.byref(o), ctypes.byref(kept),
                                 ctypes.byref(cand), _stream(prims.device)), c)
    return int(kept.value), int(cand.value)


def gve_kept_pairs(prims: torch.Tensor, shape, opts: EvalOptions | None = None, cap: int | None = None):
    """The kept (voxel, Gaussian) pairs of one evaluation as an int64 CPU
    tensor (K, 2) of (voxel index, Gaussian index), sorted."""
    prims = _prims(prims)
    o = (opts or EvalOptions()).c()
    c = context(prims.device.index)
    npairs = ctypes.c_int64(0)
    if cap is None:
        cap = gve_count_pairs(prims, shape, opts)[0]
    buf = torch.empty(max(int(cap), 1), dtype=torch.int64, device=prims.device)
    _check(lib().gve_kept_pairs(c, _ptr(prims), prims.shape[0], _dims(shape), ctypes.byref(o), _ptr(buf), int(cap),
                                ctypes.byref(npairs), _stream(prims.device)), c)
    v = buf[:npairs.value].cpu()
    v, _ = torch.sort(v)
    return torch.stack([v >> 24, v & ((1 << 24) - 1)], 1)


def gve_normalize(field: torch.Tensor, out: torch.Tensor | None = None):
    """Stage P (Sec. III-B): (V - min) / (max - min) on the device.  Returns
    (normalised field, (min, max)); ``out`` may be ``field`` (in place)."""
    field = _field(field)
    if out is None:
        out = torch.empty_like(field)
    _field(out)
    if out.shape != field.shape or out.device != field.device:
        raise ValueError("output must match the field's shape and device")
    mm = (ctypes.c_float * 2)()
    c = context(field.device.index)
    _check(lib().gve_normalize(c, _ptr(field), _dims(field.shape), _ptr(out), ctypes.cast(mm, ctypes.c_void_p),
                               _stream(field.device)), c)
    return out, (float(mm[0]), float(mm[1]))


PEAK_KINDS = {"ffma": 0, "ffma2": 1, "ex2": 2}


def gve_peak_bench(kind: str, iters: int, device=None):
    """(lane-operations per second, kernel ms) of one throughput
    microbenchmark: 'ffma', 'ffma2' (two operations per packed FMA) or 'ex2'."""
    if device is None:
        dev = torch.device("cuda", torch.cuda.current_device())
    elif isinstance(device, torch.device):
        dev = torch.device("cuda", device.index if device.index is not None else torch.cuda.current_device())
    else:
        dev = torch.device("cuda", int(device))
    ops = ctypes.c_double(0.0)
    ms = ctypes.c_float(0.0)
    with torch.cuda.device(dev):
        s = lib().gve_peak_bench(PEAK_KINDS[kind], int(iters), ctypes.byref(ops), ctypes.byref(ms), _stream(dev))
    if s != GVE_OK:
        raise GveError(s, lib().gve_status_str(s).decode())
    return ops.value, ms.value


def gve_evaluate_noalloc(prims: torch.Tensor, shape, opts: EvalOptions | None = None,
                         out: torch.Tensor | None = None):
    """Eq. 3 at every voxel centre through the entry point that allocates no
    device memory, for callers that cannot call cudaMalloc (sizes are capped:
    see include/gve.h).  ``out`` may be preallocated by the caller."""
    prims = _prims(prims)
    o = (opts or EvalOptions()).c()
    if out is None:
        out = torch.empty(tuple(int(s) for s in shape), dtype=torch.float32, device=prims.device)
    _field(out)
    if out.device != prims.device:
        raise ValueError("primitives and output must be on the same device")
    with torch.cuda.device(prims.device):
        s = lib().gve_evaluate_noalloc(_ptr(prims), prims.shape[0], _dims(out.shape), ctypes.byref(o), _ptr(out),
                                       _stream(prims.device))
    if s != GVE_OK:
        raise GveError(s, lib().gve_status_str(s).decode())
    return out
