"""FP64 numpy oracle of the learned initialiser's network and loss.

TEST INFRASTRUCTURE ONLY (imported by tests/ and the smoke check, never by
the product package).  It restates, in plain FP64 numpy, the set encoder the
CUDA library trains: per-point ReLU layers, mean pooling, ReLU head layers
and a linear output giving a diagonal mixture (softmax hefts, means,
variances exp(r) + var_floor), with the loss

    NLL  = -(1/P) sum_p log sum_g w_g N(x_p | m_g, v_g)          (Eqs. 1, 2, 16)
    PULL = lambda sum_k w~_k min_g sum_d (m_gd - m~_kd)^2 / v~_kd

averaged over the sets of a batch, and its gradient by hand-written reverse
mode.  Weight layout: per layer W [out][in] then b [out], layers in order.
"""
from __future__ import annotations

import numpy as np

LOG_2PI = np.log(2.0 * np.pi)


def layer_shapes(D, G, Hp, Hh, Lp, Lh):
    shapes = []
    for l in range(Lp + Lh + 1):
        fan_in = D if l == 0 else (Hp if l <= Lp else Hh)
        out = Hp if l < Lp else (Hh if l < Lp + Lh else G * (1 + 2 * D))
        shapes.append((out, fan_in))
    return shapes


def unpack(w, shapes):
    out, o = [], 0
    for (fo, fi) in shapes:
        W = w[o:o + fo * fi].reshape(fo, fi)
        o += fo * fi
        b = w[o:o + fo]
        o += fo
        out.append((W, b))
    assert o == w.size
    return out


def mixture_from_output(out, G, D, var_floor):
    a = out[:G]
    m = out[G:G + G * D].reshape(G, D)
    r = out[G + G * D:].reshape(G, D)
    w = np.exp(a - a.max())
    w /= w.sum()
    return w, m, np.exp(r) + var_floor, r


def set_loss_and_grad(out, x, G, D, var_floor, tgt=None, lam=0.0):
    """Loss of one set and d loss / d out (FP64)."""
    w, m, v, r = mixture_from_output(out, G, D, var_floor)
    diff = x[:, None, :] - m[None]                       # [P][G][D]
    logits = np.log(w)[None] - 0.5 * (D * LOG_2PI + np.log(v).sum(1))[None] - 0.5 * (diff ** 2 / v[None]).sum(2)
    mx = logits.max(1, keepdims=True)
    lse = mx[:, 0] + np.log(np.exp(logits - mx).sum(1))
    P = x.shape[0]
    nll = -lse.mean()
    gam = np.exp(logits - lse[:, None])                   # Eq. 3
    S0 = gam.sum(0)
    S1 = (gam[:, :, None] * diff).sum(0)
    S2 = (gam[:, :, None] * diff ** 2).sum(0)
    d = np.zeros_like(out)
    d[:G] = w - S0 / P
    d[G:G + G * D] = (-S1 / v / P).ravel()
    d[G + G * D:] = (-0.5 * (S2 / v - S0[:, None]) * np.exp(r) / v / P).ravel()
    pull = 0.0
    if tgt is not None and lam > 0.0:
        tm, tv, tw = tgt
        for k in range(G):
            q = ((m - tm[k]) ** 2 / tv[k]).sum(1)
            g = int(np.argmin(q))
            pull += lam * tw[k] * q[g]
            d[G + g * D:G + (g + 1) * D] += 2.0 * lam * tw[k] * (m[g] - tm[k]) / tv[k]
    return nll + pull, d


def loss_and_grad(w, pts, G, D, Hp, Hh, Lp, Lh, var_floor, targets=None, lam=0.0):
    """Batch-mean loss and its gradient w.r.t. the flat weights.
    pts: [B][P][D]; targets: (means [B][G][D], dcovs [B][G][D], hefts [B][G])."""
    shapes = layer_shapes(D, G, Hp, Hh, Lp, Lh)
    layers = unpack(np.asarray(w, np.float64), shapes)
    B, P, _ = pts.shape
    X = pts.reshape(B * P, D).astype(np.float64)
    acts = [X]
    for l in range(Lp):
        W, b = layers[l]
        acts.append(np.maximum(acts[-1] @ W.T + b, 0.0))
    pooled = acts[-1].reshape(B, P, -1).mean(1)
    hacts = [pooled]
    for l in range(Lh):
        W, b = layers[Lp + l]
        hacts.append(np.maximum(hacts[-1] @ W.T + b, 0.0))
    Wo, bo = layers[-1]
    out = hacts[-1] @ Wo.T + bo
    total, dout = 0.0, np.zeros_like(out)
    for s in range(B):
        tgt = None if targets is None else (targets[0][s], targets[1][s], targets[2][s])
        ls, ds = set_loss_and_grad(out[s], pts[s].astype(np.float64), G, D, var_floor, tgt, lam)
        total += ls / B
        dout[s] = ds / B
    grads = [None] * len(layers)
    grads[-1] = (dout.T @ hacts[-1], dout.sum(0))
    dh = dout @ Wo
    for l in range(Lh - 1, -1, -1):
        W, b = layers[Lp + l]
        dz = dh * (hacts[l + 1] > 0)
        grads[Lp + l] = (dz.T @ hacts[l], dz.sum(0))
        dh = dz @ W
    dh = np.repeat(dh[:, None, :], P, axis=1).reshape(B * P, -1) / P   # mean-pool backward
    for l in range(Lp - 1, -1, -1):
        W, b = layers[l]
        dz = dh * (acts[l + 1] > 0)
        grads[l] = (dz.T @ acts[l], dz.sum(0))
        dh = dz @ W
    flat = np.concatenate([np.concatenate([gW.ravel(), gb]) for gW, gb in grads])
    return total, flat, out
