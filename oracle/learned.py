"""Learned smoother network (oracle, FP64).  Not in the paper: a systems
extension of its multigrid (Sec. 4.3), defined here in full.

Network on one macro-face's lattice, an image X[c, j, i] over the padded
square 0 <= i, j <= N (lattice point (i, j); zero where i + j > N):
  h1 = M * relu(conv(X,  W1) + b1)      3 -> 16 channels
  h2 = M * relu(conv(h1, W2) + b2)      16 -> 16
  d  = Mi * (conv(h2, W3) + b3)         16 -> 1
conv is a 3x3 cross-correlation over (i +- 1, j +- 1) with zeros outside the
array: out[o, j, i] = sum_{c, dj, di} W[o, c, dj + 1, di + 1] x[c, j + dj, i + di].
M masks the closed triangle (i + j <= N), Mi the face interior (i, j >= 1,
i + j <= N - 1).  Input channels: D^-1 r (residual over the operator
diagonal), log k of the upward and of the downward micro-triangle (i, j)
(0 where the downward one does not exist).  The residual channel enters
divided by its RMS sigma over the face's closed lattice and d is multiplied
by sigma (per crop in training), so the step is homogeneous of degree 1 in
the residual.  The smoother step is x += d.

Training pair: a crop of the lattice, target e = x* - x; loss per crop
||d - e||^2 / ||e||^2 over the crop's loss mask; Adam (Kingma & Ba 2015).
The backward pass is derived by hand and pinned against central finite
differences.
"""
from __future__ import annotations

import numpy as np

SHAPES = {"W1": (16, 3, 3, 3), "b1": (16,), "W2": (16, 16, 3, 3), "b2": (16,),
          "W3": (1, 16, 3, 3), "b3": (1,)}
ORDER = ["W1", "b1", "W2", "b2", "W3", "b3"]


def n_params():
    return int(sum(np.prod(SHAPES[k]) for k in ORDER))


def init_params(seed=0):
    """He-style initialisation from a seeded normal draw."""
    rng = np.random.default_rng(seed)
    p = {}
    for k in ORDER:
        shp = SHAPES[k]
        if k.startswith("W"):
            fan_in = shp[1] * 9
            p[k] = rng.normal(0.0, np.sqrt(2.0 / fan_in), size=shp)
        else:
            p[k] = np.zeros(shp)
    p["W3"] *= 0.1
    return p


def flatten(p):
    return np.concatenate([np.asarray(p[k], dtype=np.float64).ravel() for k in ORDER])


def unflatten(v):
    p, o = {}, 0
    for k in ORDER:
        n = int(np.prod(SHAPES[k]))
        p[k] = np.asarray(v[o:o + n], dtype=np.float64).reshape(SHAPES[k])
        o += n
    return p


def shift(x, dj, di):
    """y[..., j, i] = x[..., j + dj, i + di] with zeros outside."""
    y = np.zeros_like(x)
    H, W = x.shape[-2], x.shape[-1]
    js, je = max(0, -dj), min(H, H - dj)
    is_, ie = max(0, -di), min(W, W - di)
    y[..., js:je, is_:ie] = x[..., js + dj:je + dj, is_ + di:ie + di]
    return y


def conv(x, W, b):
    out = np.zeros((W.shape[0],) + x.shape[1:])
    for dj in (-1, 0, 1):
        for di in (-1, 0, 1):
            xs = shift(x, dj, di)
            out += np.einsum("oc,cji->oji", W[:, :, dj + 1, di + 1], xs)
    return out + b[:, None, None]


def conv_backward(x, W, gout):
    """Gradients of sum(gout * conv(x, W, b)) w.r.t. x, W, b."""
    gW = np.zeros_like(W)
    gx = np.zeros_like(x)
    for dj in (-1, 0, 1):
        for di in (-1, 0, 1):
            xs = shift(x, dj, di)
            gW[:, :, dj + 1, di + 1] = np.einsum("oji,cji->oc", gout, xs)
            # x[c, j+dj, i+di] feeds out[o, j, i]: move gout back by (-dj, -di)
            gx += shift(np.einsum("oc,oji->cji", W[:, :, dj + 1, di + 1], gout), -dj, -di)
    gb = gout.sum(axis=(1, 2))
    return gx, gW, gb


def bf16(x):
    """Round to bfloat16 (8 significant bits, round to nearest even) and back:
    the float32 bit pattern rounded at bit 16."""
    b = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def forward(p, X, M, Mi, round_bf16=False):
    """round_bf16: weights, biases and hidden activations rounded to BF16
    where the GPU kernels round them (the FP64 network otherwise)."""
    if round_bf16:
        p = {k: bf16(v) for k, v in p.items()}
    r = bf16 if round_bf16 else (lambda v: v)
    a1 = conv(X, p["W1"], p["b1"])
    h1 = r(M * np.maximum(a1, 0.0))
    a2 = conv(h1, p["W2"], p["b2"])
    h2 = r(M * np.maximum(a2, 0.0))
    d = Mi * conv(h2, p["W3"], p["b3"])[0]
    return d, (X, a1, h1, a2, h2)


def loss_and_grad(p, X, M, Mi, e, Ml):
    """Relative squared error over the loss mask Ml and its gradient."""
    d, (X, a1, h1, a2, h2) = forward(p, X, M, Mi)
    den = float(np.sum(Ml * e * e))
    diff = Ml * (d - e)
    L = float(np.sum(diff * diff)) / den
    gd = (2.0 / den) * diff * Mi
    g3x, gW3, gb3 = conv_backward(h2, p["W3"], gd[None])
    g2 = g3x * M * (a2 > 0)
    g2x, gW2, gb2 = conv_backward(h1, p["W2"], g2)
    g1 = g2x * M * (a1 > 0)
    _, gW1, gb1 = conv_backward(X, p["W1"], g1)
    return L, {"W1": gW1, "b1": gb1, "W2": gW2, "b2": gb2, "W3": gW3, "b3": gb3}


def adam_step(v, g, m, s, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update of the flat parameter vector v (t counts from 1)."""
    m = b1 * m + (1 - b1) * g
    s = b2 * s + (1 - b2) * g * g
    mh = m / (1 - b1 ** t)
    sh = s / (1 - b2 ** t)
    return v - lr * mh / (np.sqrt(sh) + eps), m, s


def masks(N, i0=0, j0=0, H=None, W=None):
    """Closed-triangle mask M, interior mask Mi for the window [j0, j0+H) x
    [i0, i0+W) of a face lattice with N intervals."""
    H = N + 1 if H is None else H
    W = N + 1 if W is None else W
    j = np.arange(j0, j0 + H)[:, None]
    i = np.arange(i0, i0 + W)[None, :]
    inside = (i >= 0) & (j >= 0) & (i + j <= N)
    interior = (i >= 1) & (j >= 1) & (i + j <= N - 1)
    return inside.astype(np.float64), interior.astype(np.float64)


def face_images(level, s, k_elem=None):
    """Per macro-face input image X (3, N+1, N+1) and masks (M, Mi) from a
    canonical vector s (the scaled residual) and the per-element coefficient
    in canonical element order (None: k = 1).  Returns a list over faces of
    (X, M, Mi, G, sigma): X with its residual channel divided by sigma, the
    face's residual RMS; G the lattice -> canonical id map."""
    N = level.N
    M, Mi = masks(N)
    out = []
    for f, G in enumerate(level.face_ids):
        X = np.zeros((3, N + 1, N + 1))
        ok = G >= 0
        X[0][ok] = s[G[ok]]
        sig = np.sqrt(np.sum(X[0][ok] ** 2) / ((N + 1) * (N + 2) / 2))
        if k_elem is not None:
            kf = np.asarray(k_elem)[f * N * N:(f + 1) * N * N]
            r = 0
            for j in range(N):
                for i in range(N - j):
                    X[1, j, i] = np.log(kf[r])
                    r += 1
            for j in range(N - 1):
                for i in range(N - 1 - j):
                    X[2, j, i] = np.log(kf[r])
                    r += 1
        if sig > 0:
            X[0] /= sig
        out.append((X * M, M, Mi, G, sig))
    return out


# ------------------------------------------------------------------ residual loss
def edge_weights(cot, ku, kd):
    """Off-diagonal magnitudes of the P1 rows on a lattice window: for each
    point p = (i, j) and each of its six neighbours, w = 1/2 cot(opposite
    angle) (k_T1 + k_T2) over the two micro-triangles sharing the edge (the
    cotangent form, face angles t0, t1, t2 at v0, v1, v2).  ku, kd: (H, W)
    images of the upward / downward micro-triangle coefficients at (i, j)
    (0 where absent).  Returns {offset (di, dj): (H, W) weights}."""
    c0, c1, c2 = cot
    sh = lambda a, dj, di: shift(a[None], dj, di)[0]
    u, uw, us = ku, sh(ku, 0, -1), sh(ku, -1, 0)                 # up(i,j), up(i-1,j), up(i,j-1)
    ds, dw, dsw = sh(kd, -1, 0), sh(kd, 0, -1), sh(kd, -1, -1)   # down(i,j-1), down(i-1,j), down(i-1,j-1)
    return {(1, 0): 0.5 * c2 * (u + ds), (-1, 0): 0.5 * c2 * (uw + dsw),
            (0, 1): 0.5 * c1 * (u + dw), (0, -1): 0.5 * c1 * (us + dsw),
            (1, -1): 0.5 * c0 * (us + ds), (-1, 1): 0.5 * c0 * (uw + dw)}


def scaled_operator(d, wts):
    """(D^-1 A d)_p = d_p - sum_q (w_pq / diag_p) d_q on the window (zeros
    outside), diag_p = sum_q w_pq."""
    diag = sum(wts.values())
    acc = np.zeros_like(d)
    for (di, dj), w in wts.items():
        acc += w * shift(d[None], dj, di)[0]
    with np.errstate(divide="ignore", invalid="ignore"):
        return d - np.where(diag > 0, acc / diag, 0.0)


def residual_loss_and_grad(p, X, M, Mi, shat, Ml, wts, round_bf16=False):
    """Loss ||Ml (shat - D^-1 A d)||^2 / ||Ml shat||^2 of the smoother step d
    on the normalised scaled residual shat, and its gradient (w.r.t. the
    weights as used: rounded ones under round_bf16)."""
    d, (X, a1, h1, a2, h2) = forward(p, X, M, Mi, round_bf16)
    if round_bf16:
        p = {k: bf16(v) for k, v in p.items()}
    den = float(np.sum(Ml * shat * shat))
    res = Ml * (shat - scaled_operator(d, wts))
    L = float(np.sum(res * res)) / den
    # d/dd_q of -sum_p res_p (D^-1 A d)_p: -(res_q - sum_p (w_pq/diag_p) res_p)
    diag = sum(wts.values())
    with np.errstate(divide="ignore", invalid="ignore"):
        v = np.where(diag > 0, res / diag, 0.0)
    back = np.zeros_like(d)
    for (di, dj), w in wts.items():
        # p = q - (di, dj) has q as its (di, dj) neighbour with weight w(p)
        back += shift((w * v)[None], -dj, -di)[0]
    gd = -(2.0 / den) * (res - back) * Mi
    g3x, gW3, gb3 = conv_backward(h2, p["W3"], gd[None])
    g2 = g3x * M * (a2 > 0)
    g2x, gW2, gb2 = conv_backward(h1, p["W2"], g2)
    g1 = g2x * M * (a1 > 0)
    _, gW1, gb1 = conv_backward(X, p["W1"], g1)
    return L, {"W1": gW1, "b1": gb1, "W2": gW2, "b2": gb2, "W3": gW3, "b3": gb3}
