"""Batched encode: many volumes (or timesteps) of uneven shapes encoded
together -- analytic allocation of each volume's budget (all volumes
concurrently, ``gve_allocate_batch``), one autotuning pass of the
evaluator's launch shape, then refinement of all volumes with one CUDA graph
launch per iteration (``gve_refine_batch``: one binning of all volumes, then
one persistent kernel over the bricks of every volume for evaluation and
update).  Each volume is encoded exactly as it would be alone (Sec. III-E of
arxiv 2608.14112)."""
from __future__ import annotations

import time
from dataclasses import dataclass

import torch

from . import gve


@dataclass
class BatchResult:
    prims: list            # per-volume (N_v, 12) views into one concatenated tensor
    psnr: list             # final PSNR per volume
    options: gve.EvalOptions
    tune_ms: dict
    alloc_s: float
    refine_s: float
    stats: dict


def encode_batch(fields, budgets, iters: int, lr: float = 1e-2, seed: int = 0, autotune: bool = True,
                 opts: gve.EvalOptions | None = None) -> BatchResult:
    """Allocate ``budgets[v]`` Gaussians in each ``fields[v]`` (CUDA float32,
    shape (nz, ny, nx)) and refine all volumes for ``iters`` iterations."""
    dev = fields[0].device
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    prims, _ = gve.gve_allocate_batch(fields, budgets, seed=seed)
    torch.cuda.synchronize(dev)
    alloc_s = time.perf_counter() - t0
    views, off = [], 0
    for n in budgets:
        views.append(prims[off:off + n])
        off += n
    o = opts or gve.EvalOptions()
    table = {}
    if autotune:
        o, table = gve.gve_autotune(prims, fields, budgets, o)
    t0 = time.perf_counter()
    psnr, stats = gve.gve_refine_batch(prims, fields, budgets, iters, lr=lr, opts=o)
    torch.cuda.synchronize(dev)
    refine_s = time.perf_counter() - t0
    return BatchResult(views, psnr, o, table, alloc_s, refine_s, stats)
