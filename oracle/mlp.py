"""FP64 oracle of the order-choosing MLP (an addition to the paper, which
fixes one expansion order per run).

TEST INFRASTRUCTURE ONLY (same rules as the rest of ``oracle/``).

The model maps the 12 per-pair features of ``oracle.adaptive_pairs`` to the
predicted log10 force error of the pair's M2L at orders 2..10:

    z0 = (f - mu) / sd
    h1 = relu(W1 z0 + b1)          W1: 64 x 12
    h2 = relu(W2 h1 + b2)          W2: 64 x 64
    h3 = relu(W3 h2 + b3)          W3: 64 x 64
    y  = W4 h3 + b4                W4:  9 x 64

and the pair takes the lowest order p in 2..P whose prediction is at most
``log10(target) + log10(kappa) - log10(K_B)/2``, or P when none is; K_B is
the number of M2L pairs of the target and its ancestors (independent pair
errors add in quadrature at a target).  The BF16 form rounds
the weights and every layer input (z0, h1, h2, h3) to bfloat16 (round to
nearest even) and accumulates in FP32; this module emulates that rounding
exactly and accumulates in FP64.

Parameter blob (float32, 9769 values):
    [0:8]   header: tag 6332, version 2, NF=12, H=64, NOUT=9, p_lo=2,
            log10 kappa, 0
    [8:20]  mu,  [20:32] sd
    [32:]   W1 (row-major, 64x12), b1, W2, b2, W3, b3, W4 (9x64), b4
The trainable parameters are blob[32:].

Loss for training: L = mean over samples and the 9 outputs of (y - t)^2.
Adam (Kingma & Ba): m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2,
theta -= lr (m / (1-b1^t)) / (sqrt(v / (1-b2^t)) + eps).
"""
from __future__ import annotations

import numpy as np

NF, H, NOUT, P_LO = 12, 64, 9, 2
HDR = 8
OFF_MU = HDR
OFF_SD = HDR + NF
OFF_PAR = HDR + 2 * NF
SHAPES = [("W1", (H, NF)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)), ("W3", (H, H)), ("b3", (H,)),
          ("W4", (NOUT, H)), ("b4", (NOUT,))]
NPAR = sum(int(np.prod(s)) for _, s in SHAPES)
NBLOB = OFF_PAR + NPAR


def unpack(blob):
    blob = np.asarray(blob, dtype=np.float64)
    assert blob.shape == (NBLOB,), blob.shape
    out = {"hdr": blob[:HDR], "mu": blob[OFF_MU:OFF_MU + NF], "sd": blob[OFF_SD:OFF_SD + NF]}
    o = OFF_PAR
    for name, shp in SHAPES:
        k = int(np.prod(shp))
        out[name] = blob[o:o + k].reshape(shp)
        o += k
    return out


def pack(d):
    parts = [np.asarray(d["hdr"], dtype=np.float64), np.asarray(d["mu"]), np.asarray(d["sd"])]
    parts += [np.asarray(d[name], dtype=np.float64).reshape(-1) for name, _ in SHAPES]
    return np.concatenate(parts).astype(np.float32)


def header(log10_kappa=0.0):
    return np.array([6332.0, 2.0, NF, H, NOUT, P_LO, log10_kappa, 0.0])


def bf16_round(a):
    """Round to the nearest bfloat16 (ties to even), returned as float64.
    Works on the float32 bit pattern: add 0x7fff plus the lowest kept bit,
    then clear the 16 dropped bits (finite inputs)."""
    f = np.ascontiguousarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def forward(blob, feat, bf16=False, keep=False):
    """Predictions (n, 9).  With keep=True also returns the activations."""
    d = unpack(blob)
    f = np.asarray(feat, dtype=np.float64)
    z0 = (f - d["mu"]) / d["sd"]
    Ws = [d["W1"], d["W2"], d["W3"], d["W4"]]
    bs = [d["b1"], d["b2"], d["b3"], d["b4"]]
    if bf16:
        # the normalised input is formed in FP32 before rounding
        z0 = bf16_round(((f.astype(np.float32) - d["mu"].astype(np.float32)) / d["sd"].astype(np.float32)))
        Ws = [bf16_round(W) for W in Ws]
    acts = [z0]
    h = z0
    for k in range(3):
        a = h @ Ws[k].T + bs[k]
        h = np.maximum(a, 0.0)
        if bf16:
            h = bf16_round(h)
        acts.append(h)
    y = h @ Ws[3].T + bs[3]
    return (y, acts) if keep else y


def loss_grad(blob, feat, lab):
    """Loss and its gradient with respect to the trainable parameters
    (a vector of NPAR values in blob order), FP64, no rounding."""
    d = unpack(blob)
    y, acts = forward(blob, feat, keep=True)
    t = np.asarray(lab, dtype=np.float64)
    n = y.shape[0]
    r = y - t
    loss = float(np.mean(r * r))
    g_y = 2.0 * r / (n * NOUT)
    Ws = [d["W1"], d["W2"], d["W3"], d["W4"]]
    grads = {}
    g = g_y
    for k in (3, 2, 1, 0):
        grads["W%d" % (k + 1)] = g.T @ acts[k]
        grads["b%d" % (k + 1)] = g.sum(0)
        if k > 0:
            g = (g @ Ws[k]) * (acts[k] > 0.0)
    vec = np.concatenate([grads[name].reshape(-1) for name, _ in SHAPES])
    return loss, vec


def adam_step(theta, g, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (step number t >= 1); returns new (theta, m, v)."""
    m = b1 * m + (1.0 - b1) * g
    v = b2 * v + (1.0 - b2) * g * g
    mh = m / (1.0 - b1 ** t)
    vh = v / (1.0 - b2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v


def select(pred, log10_target, log10_kappa, p_max=10, log10_k=None):
    """Lowest order p in 2..p_max with pred[p-2] <= threshold, else p_max.
    threshold = log10_target + log10_kappa - log10(K_B)/2 with log10_k the
    per-pair log10 K_B (the M2L pairs of the target and its ancestors), or
    without that term when log10_k is None."""
    pred = np.asarray(pred)
    thr = log10_target + log10_kappa - (0.0 if log10_k is None else 0.5 * np.asarray(log10_k))
    thr = np.broadcast_to(thr, (pred.shape[0],))
    out = np.full(pred.shape[0], p_max, dtype=np.int8)
    for p in range(p_max, P_LO - 1, -1):
        ok = pred[:, p - P_LO] <= thr
        out[ok] = p
    return out


def chain_pairs(tgt, parent):
    """K_B per node: the number of M2L pairs whose target is the node or one
    of its ancestors (parents precede children in the node numbering)."""
    cnt = np.bincount(np.asarray(tgt), minlength=len(parent)).astype(np.float64)
    K = np.zeros(len(parent))
    for c in range(len(parent)):
        K[c] = cnt[c] + (K[parent[c]] if parent[c] >= 0 else 0.0)
    return K
