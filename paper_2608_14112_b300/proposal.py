"""Learned proposal: a small MLP that corrects each allocated Gaussian's
initial amplitude and log-scales from its local structure statistics.

The network (16 -> 64 -> 64 -> 64 -> 4, GELU, BF16 weights, FP32
accumulation) runs and trains in the library's own kernels
(``gve_proposal_features``, ``gve_mlp_forward``, ``gve_mlp_grad``,
``gve_mlp_adam``, ``gve_proposal_apply``).  Training pairs come from the
encoder itself: features of an analytic allocation (Sec. III-E of arxiv
2608.14112) against the change that full refinement made to a and log s.
The last layer starts at zero, so an untrained model leaves the allocation
unchanged -- plain allocation is the fallback, and refinement judges the
result: after the regression, one step size for all corrections is chosen
among a few candidates (zero, the plain allocation, included) by the PSNR
that refinement reaches from the corrected allocations of training fields
(``Proposal.calibrate``).
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import numpy as np
import torch

from . import gve

P = 9668
MODEL_FLOATS = 33870
LAYERS = [("W1", (64, 16)), ("b1", (64,)), ("W2", (64, 64)), ("b2", (64,)), ("W3", (64, 64)), ("b3", (64,)),
          ("W4", (4, 64)), ("b4", (4,))]


def _lib():
    L = gve.lib()
    if not hasattr(L, "_proposal_typed"):
        Pp, i64, i32, f = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_float
        L.gve_proposal_features.argtypes = [Pp, Pp, gve.Dims, Pp, i64, i64, f, f, Pp, Pp]
        L.gve_mlp_forward.argtypes = [Pp, Pp, Pp, i64, Pp, Pp, Pp]
        L.gve_mlp_grad.argtypes = [Pp, Pp, Pp, Pp, i64, Pp, Pp, Pp]
        L.gve_mlp_adam.argtypes = [Pp, Pp, Pp, f, f, f, f, i32, Pp]
        L.gve_mlp_quantise.argtypes = [Pp, Pp, Pp]
        L.gve_proposal_apply.argtypes = [Pp, Pp, Pp, Pp, i64, gve.Dims, Pp]
        L.gve_proposal_backward.argtypes = [Pp, Pp, Pp, Pp, Pp, i64, gve.Dims, i32, Pp, Pp]
        L.gve_mlp_standardise.argtypes = [Pp, Pp, Pp, i64, Pp]
        L.gve_proposal_targets.argtypes = [Pp, Pp, Pp, i64, Pp, Pp]
        L.gve_mlp_scale_targets.argtypes = [Pp, Pp, i64, Pp, Pp]
        L.gve_mlp_fold_output_scale.argtypes = [Pp, Pp, Pp, Pp]
        for fn in ("gve_proposal_features", "gve_mlp_forward", "gve_mlp_grad", "gve_mlp_adam", "gve_mlp_quantise",
                   "gve_proposal_apply", "gve_proposal_backward", "gve_mlp_standardise", "gve_proposal_targets",
                   "gve_mlp_scale_targets", "gve_mlp_fold_output_scale"):
            getattr(L, fn).restype = ctypes.c_int
        L._proposal_typed = True
    return L


def _p(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def features(field: torch.Tensor, prims: torch.Tensor, n_detail: int, gbar: float, occ: float = 0.02):
    """(N, 16) float32 features of the allocated records."""
    gve._field(field)
    gve._prims(prims)
    out = torch.empty((prims.shape[0], 16), dtype=torch.float32, device=prims.device)
    c = gve.context(prims.device.index)
    gve._check(_lib().gve_proposal_features(c, _p(field), gve._dims(field.shape), _p(prims), prims.shape[0],
                                            int(n_detail), float(gbar), float(occ), _p(out),
                                            gve._stream(prims.device)), c)
    return out


# candidate step sizes of Proposal.calibrate (0 = plain allocation)
CAL_GAMMAS = (0.0, 0.125, 0.25, 0.375, 0.5, 0.75, 1.0)


@dataclass
class TrainLog:
    losses: list
    epochs: int
    rows: int


class Proposal:
    """Model buffer (see include/gve.h) plus host-side training loop."""

    def __init__(self, device="cuda", seed: int = 0):
        self.device = torch.device(device)
        rng = np.random.Generator(np.random.PCG64(seed))
        flat = []
        for name, shp in LAYERS:
            if name.startswith("b") or name == "W4":
                flat.append(np.zeros(int(np.prod(shp))))
            else:
                fan_in = shp[1]
                flat.append(rng.normal(0.0, np.sqrt(2.0 / fan_in), size=shp).reshape(-1))
        model = np.zeros(MODEL_FLOATS, np.float32)
        model[:P] = np.concatenate(flat).astype(np.float32)
        model[3 * P + 16: 3 * P + 32] = 1.0          # inverse standard deviation
        self.model = torch.from_numpy(model).to(self.device)
        self.step = 0
        self.gamma = 1.0
        self._quantise()

    def _ctx(self):
        return gve.context(self.device.index)

    def _quantise(self):
        c = self._ctx()
        gve._check(_lib().gve_mlp_quantise(c, _p(self.model), gve._stream(self.device)), c)

    def set_normalisation(self, X: torch.Tensor):
        """Input standardisation from training features (gve_mlp_standardise:
        column means and spreads on the device; a feature whose spread is
        negligible against its magnitude carries nothing to learn from and
        gets weight 0, so that it cannot swing the network on data where it
        does vary)."""
        X = X.contiguous()
        c = self._ctx()
        gve._check(_lib().gve_mlp_standardise(c, _p(self.model), _p(X), X.shape[0], gve._stream(self.device)), c)

    def forward(self, X: torch.Tensor) -> torch.Tensor:
        Y = torch.empty((X.shape[0], 4), dtype=torch.float32, device=self.device)
        c = self._ctx()
        gve._check(_lib().gve_mlp_forward(c, _p(self.model), _p(X.contiguous()), X.shape[0], _p(Y), None,
                                          gve._stream(self.device)), c)
        return Y

    def grad(self, X: torch.Tensor, T: torch.Tensor):
        dP = torch.empty(P, dtype=torch.float32, device=self.device)
        loss = torch.zeros(1, dtype=torch.float64, device=self.device)
        c = self._ctx()
        gve._check(_lib().gve_mlp_grad(c, _p(self.model), _p(X.contiguous()), _p(T.contiguous()), X.shape[0],
                                       _p(dP), _p(loss), gve._stream(self.device)), c)
        return dP, loss

    def adam(self, dP: torch.Tensor, lr: float, beta1=0.9, beta2=0.999, eps=1e-8):
        self.step += 1
        c = self._ctx()
        gve._check(_lib().gve_mlp_adam(c, _p(self.model), _p(dP), float(lr), float(beta1), float(beta2),
                                       float(eps), self.step, gve._stream(self.device)), c)

    def train(self, X: torch.Tensor, T: torch.Tensor, epochs: int = 20, batch: int = 4096, lr: float = 1e-3,
              seed: int = 0, tscale: torch.Tensor | None = None) -> TrainLog:
        """Minibatch Adam on the mean squared error of the corrections.  The
        targets come from ``make_pairs`` divided by their spreads ``tscale``
        (device float32 [4]); the scale is folded back into the last layer
        afterwards (gve_mlp_fold_output_scale), so the trained network
        predicts the corrections themselves."""
        self.set_normalisation(X)
        self._quantise()
        g = torch.Generator(device=self.device)
        g.manual_seed(seed)
        losses = []
        R = X.shape[0]
        for _ in range(epochs):
            perm = torch.randperm(R, generator=g, device=self.device)
            total = torch.zeros(1, dtype=torch.float64, device=self.device)
            nb = 0
            for s in range(0, R, batch):
                idx = perm[s:s + batch]
                dP, loss = self.grad(X.index_select(0, idx), T.index_select(0, idx))
                self.adam(dP, lr)
                total += loss
                nb += 1
            losses.append(float(total.item()) / nb)
        if tscale is not None:
            c = self._ctx()
            gve._check(_lib().gve_mlp_fold_output_scale(c, _p(self.model), _p(tscale), gve._stream(self.device)),
                       c)
        return TrainLog(losses, epochs, R)

    def scale_outputs(self, factors) -> None:
        """Multiplies the network's four outputs by ``factors`` (folded into
        the last layer by gve_mlp_fold_output_scale, BF16 copies refreshed)."""
        sc = torch.as_tensor(factors, dtype=torch.float32, device=self.device).reshape(4).contiguous()
        c = self._ctx()
        gve._check(_lib().gve_mlp_fold_output_scale(c, _p(self.model), _p(sc), gve._stream(self.device)), c)

    def calibrate(self, fields, budget: int, iters: int = 150, gammas=CAL_GAMMAS, seed: int = 0, lr: float = 1e-2,
                  opts: gve.EvalOptions | None = None) -> dict:
        """Step size of the corrections, judged by refinement itself.  For
        each gamma the corrections gamma * (predicted change) are applied to
        the analytic allocations of ``fields`` (seeds seed + i), all fields
        are refined ``iters`` iterations together (gve_refine_batch), and the
        gamma with the highest mean final PSNR is folded into the last layer;
        gamma 0 is the plain allocation, so the result is never worse than
        plain on these fields.  Returns {gamma: mean PSNR (dB)}."""
        allocs, feats = [], []
        for i, f in enumerate(fields):
            Pv, info = gve.gve_allocate(f, budget, seed=seed + i)
            allocs.append(Pv)
            feats.append(features(f, Pv, info["n_detail"], info["gbar"]))
        base = self.model.clone()
        scores = {}
        for gam in gammas:
            Pc = [p.clone() for p in allocs]
            if gam != 0.0:
                self.model = base.clone()
                self.scale_outputs([gam] * 4)
                for f, x, p in zip(fields, feats, Pc):
                    self.apply(x, p, f.shape)
            psnr, _ = gve.gve_refine_batch(torch.cat(Pc, 0).contiguous(), fields, [budget] * len(fields), iters,
                                           lr=lr, opts=opts)
            scores[float(gam)] = float(np.mean(psnr))
        best = max(scores, key=lambda g: (scores[g], -g))
        self.model = base
        self.scale_outputs([best] * 4)
        self.gamma = best
        return scores

    def apply(self, feats: torch.Tensor, prims: torch.Tensor, shape):
        """Correct the allocated records in place."""
        c = self._ctx()
        gve._check(_lib().gve_proposal_apply(c, _p(self.model), _p(feats.contiguous()), _p(prims),
                                             prims.shape[0], gve._dims(shape), gve._stream(self.device)), c)
        return prims

    def backward(self, feats: torch.Tensor, prims_corrected: torch.Tensor, grad_prims: torch.Tensor, shape,
                 dP: torch.Tensor | None = None, accumulate: bool = False) -> torch.Tensor:
        """dL/dtheta from dL/dprims at the corrected records (end-to-end)."""
        if dP is None:
            dP = torch.empty(P, dtype=torch.float32, device=self.device)
        c = self._ctx()
        gve._check(_lib().gve_proposal_backward(c, _p(self.model), _p(feats.contiguous()), _p(prims_corrected),
                                                _p(grad_prims), prims_corrected.shape[0], gve._dims(shape),
                                                int(bool(accumulate)), _p(dP), gve._stream(self.device)), c)
        return dP

    def train_e2e(self, fields, allocs, epochs: int = 20, lr: float = 1e-3, fields_per_step: int = 4,
                  seed: int = 0, opts: gve.EvalOptions | None = None) -> TrainLog:
        """Trains the proposal through the encoder's own objective: each step
        corrects the analytic allocations of a few fields, evaluates the
        full-grid MSE of the corrected records (Eq. 3) and its gradient, and
        back-propagates dL/d(a, log s) into the network.  ``allocs`` holds
        (features, allocated records) per field.  The per-epoch log is the
        mean MSE of the corrected allocations."""
        self.set_normalisation(torch.cat([x for x, _ in allocs], 0))
        self._quantise()
        g = torch.Generator()
        g.manual_seed(seed)
        dP = torch.empty(P, dtype=torch.float32, device=self.device)
        losses = []
        for _ in range(epochs):
            order = torch.randperm(len(fields), generator=g).tolist()
            tot = torch.zeros((), dtype=torch.float64, device=self.device)
            for s in range(0, len(order), fields_per_step):
                for j, fi in enumerate(order[s:s + fields_per_step]):
                    X, P0 = allocs[fi]
                    f = fields[fi]
                    Pc = P0.clone()
                    self.apply(X, Pc, f.shape)
                    grad, sse = gve.gve_loss_grad(Pc, f, opts)
                    tot += sse[1] / f.numel()
                    self.backward(X, Pc, grad, f.shape, dP, accumulate=j > 0)
                self.adam(dP, lr)
            losses.append(float(tot.item()) / len(fields))
        return TrainLog(losses, epochs, sum(int(x.shape[0]) for x, _ in allocs))

    def state_dict(self):
        return {"model": self.model.cpu(), "step": self.step}

    def load_state_dict(self, sd):
        self.model = sd["model"].to(self.device)
        self.step = int(sd["step"])
        self._quantise()


def targets(prims0: torch.Tensor, prims1: torch.Tensor) -> torch.Tensor:
    """Training targets (gve_proposal_targets): refined minus allocated (a,
    log s0, log s1, log s2)."""
    n = prims0.shape[0]
    T = torch.empty((n, 4), dtype=torch.float32, device=prims0.device)
    c = gve.context(prims0.device.index)
    gve._check(_lib().gve_proposal_targets(c, _p(prims0.contiguous()), _p(prims1.contiguous()), n, _p(T),
                                           gve._stream(prims0.device)), c)
    return T


def make_pairs(fields, budget: int, iters: int, seed: int = 0, lr: float = 1e-2, chunk: int = 32):
    """Allocation -> refined pairs from the encoder itself: features of each
    field's analytic allocation and the corrections refinement applied
    (unscaled; ``scale_targets`` divides them by their spreads).  Fields are
    refined in batches with gve_refine_batch."""
    X, T = [], []
    for s in range(0, len(fields), chunk):
        group = fields[s:s + chunk]
        allocs, infos = [], []
        for i, f in enumerate(group):
            Pv, info = gve.gve_allocate(f, budget, seed=seed + s + i)
            allocs.append(Pv)
            infos.append(info)
        feats = [features(f, Pv, info["n_detail"], info["gbar"]) for f, Pv, info in zip(group, allocs, infos)]
        P0 = torch.cat(allocs, 0).contiguous()
        P1 = P0.clone()
        gve.gve_refine_batch(P1, group, [budget] * len(group), iters, lr=lr)
        X.append(torch.cat(feats, 0))
        T.append(targets(P0, P1))
    return torch.cat(X, 0).contiguous(), torch.cat(T, 0).contiguous()


def scale_targets(T: torch.Tensor):
    """(a copy of T with each column divided by its spread, the spreads
    (device float32 [4])), computed by gve_mlp_scale_targets."""
    Ts = T.clone().contiguous()
    sc = torch.empty(4, dtype=torch.float32, device=T.device)
    c = gve.context(T.device.index)
    gve._check(_lib().gve_mlp_scale_targets(c, _p(Ts), Ts.shape[0], _p(sc), gve._stream(T.device)), c)
    return Ts, sc


def allocations(fields, budget: int, seed: int = 0):
    """(features, allocated records) of each field's analytic allocation."""
    out = []
    for i, f in enumerate(fields):
        Pv, info = gve.gve_allocate(f, budget, seed=seed + i)
        out.append((features(f, Pv, info["n_detail"], info["gbar"]), Pv))
    return out


def encode(field: torch.Tensor, budget: int, iters: int, model: Proposal | None = None, seed: int = 0,
           lr: float = 1e-2):
    """Allocate (optionally corrected by ``model``) and refine; returns
    (records, per-iteration loss trace (float64 tensor), final stats)."""
    Pv, info = gve.gve_allocate(field, budget, seed=seed)
    if model is not None:
        f = features(field, Pv, info["n_detail"], info["gbar"])
        model.apply(f, Pv, field.shape)
    trace = torch.zeros(max(iters, 1), dtype=torch.float64, device=field.device)
    st = gve.gve_refine(Pv, field, iters=iters, lr=lr, trace=trace)
    return Pv, trace[:iters], st
