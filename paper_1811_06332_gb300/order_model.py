"""Training and calibration of the per-pair M2L order model of learned_p
plans (an addition to the paper, which fixes one order per run).

Sequencing only: pair features and labels, training, FMM evaluations and the
direct sums all run in the library's kernels (fmm_pair_data, fmm_mlp_train,
fmm_evaluate, fmm_direct); this module draws the seeded random numbers
(initial weights, sample order, sampled targets) and passes them in.

Parameter blob layout (FMM_MLP_NBLOB floats, include/fmm_gb300.h):
header {6332, 2, 12, 64, 9, 2, log10 kappa, 0}, 12 means, 12 deviations,
W1 (64x12), b1, W2 (64x64), b2, W3 (64x64), b3, W4 (9x64), b4.
"""
from __future__ import annotations

import numpy as np
import torch

from . import fmm as F
from . import inputs

NF, H, NOUT = 12, 64, 9
HDR, OFF_PAR = 8, 8 + 2 * 12
SHAPES = [(H, NF), (H,), (H, H), (H,), (H, H), (H,), (NOUT, H), (NOUT,)]
NBLOB = OFF_PAR + sum(int(np.prod(s)) for s in SHAPES)
assert NBLOB == F.MLP_NBLOB


def init_blob(seed: int, log10_kappa: float = 0.0) -> np.ndarray:
    """He-uniform weights U(-sqrt(6/fan_in), +sqrt(6/fan_in)) from the seeded
    generator, zero biases, identity feature normalisation."""
    b = np.zeros(NBLOB)
    b[:HDR] = [6332.0, 2.0, NF, H, NOUT, 2.0, log10_kappa, 0.0]
    b[HDR + NF:HDR + 2 * NF] = 1.0
    o = OFF_PAR
    for k, shp in enumerate(SHAPES):
        cnt = int(np.prod(shp))
        if len(shp) == 2:
            lim = np.sqrt(6.0 / shp[1])
            b[o:o + cnt] = (inputs.u01(seed, k, cnt) * 2.0 - 1.0) * lim
        o += cnt
    return b.astype(np.float32)


def pair_samples(sets, max_leaf: int, theta: float, device=None):
    """Features and labels (float32 device tensors) of the M2L pairs of each
    particle set (x, y, z, q numpy arrays), from FP64 plans at order 10."""
    dev = device or torch.device("cuda", torch.cuda.current_device())
    feats, labs = [], []
    for X in sets:
        plan = F.Plan(p=10, basis=F.BASIS_SYM, prec=F.FP64, adaptive=True, max_leaf=max_leaf, theta=theta)
        Xd = [torch.from_numpy(np.ascontiguousarray(a)).to(dev) for a in X]
        plan.fmm_build_tree(*Xd)
        f, lab = plan.pair_data(labels=True)
        feats.append(f)
        labs.append(lab.float())
        torch.cuda.synchronize()
        plan.close()
    return torch.cat(feats), torch.cat(labs)


def train(feat, lab, seed: int, epochs: int = 20, batch: int = 1024, lr: float = 2e-3, blob=None):
    """Trains on the GPU (fmm_mlp_train); returns (blob, per-epoch losses)."""
    n = feat.shape[0]
    order = torch.from_numpy(np.argsort(inputs.u01(seed, 7, n)).astype(np.int32)).to(feat.device)
    b0 = init_blob(seed) if blob is None else blob
    return F.fmm_mlp_train(b0, feat, lab, order, epochs=epochs, batch=batch, lr=lr, fit_moments=True)


def force_error(acc, Xd, nsample: int, seed: int) -> float:
    """Relative force error sqrt(sum |a - a_ref|^2 / sum |a_ref|^2) on
    nsample seeded targets against the FP64 direct sum (fmm_direct)."""
    n = Xd[0].shape[0]
    sel = np.unique((inputs.u01(seed, 95, nsample) * n).astype(np.int64))
    t = torch.from_numpy(sel).to(Xd[0].device)
    ref = torch.empty((4, len(sel)), dtype=torch.float64, device=Xd[0].device)
    F.fmm_direct(Xd[0], Xd[1], Xd[2], Xd[3], ref[0], ref[1], ref[2], ref[3], targets=t)
    a = acc[:, t]
    return float(torch.sqrt(((a - ref[1:]) ** 2).sum() / (ref[1:] ** 2).sum()).item())


def calibrate(blob, X, p: int, max_leaf: int, theta: float, target: float, prec=F.FP32,
              grid=tuple(-1.0 + 0.25 * k for k in range(13)), margin: float = 0.8, seed: int = 5):
    """Largest log10 kappa of the grid (tried in increasing order, stopping at
    the first miss) whose learned FMM on the set X meets margin * target.
    The budget per pair is target * kappa / sqrt(K_B) (fmm_config); kappa
    absorbs what that scaling leaves out (correlated pair errors, the near
    field).  Returns (blob with that kappa, [(log10 kappa, error, mean
    order)])."""
    dev = torch.device("cuda", torch.cuda.current_device())
    Xd = [torch.from_numpy(np.ascontiguousarray(a)).to(dev) for a in X]
    best = None
    log = []
    for k in grid:
        b = np.array(blob, dtype=np.float32)
        b[6] = k
        plan = F.Plan(p=p, basis=F.BASIS_SYM, prec=prec, adaptive=True, max_leaf=max_leaf, theta=theta,
                      learned_p=True, target_rel_err=target)
        plan.set_mlp(b)
        _, acc = plan.evaluate(*Xd)
        err = force_error(acc, Xd, 4096, seed)
        cnt = np.array(plan.stats()["pairs_per_order"], dtype=np.float64)
        plan.close()
        mean_p = float((cnt * np.arange(len(cnt))).sum() / max(cnt.sum(), 1))
        log.append((k, err, mean_p))
        if err <= margin * target:
            best = b
        else:
            break
    if best is None:
        best = np.array(blob, dtype=np.float32)
        best[6] = grid[0]
    return best, log
