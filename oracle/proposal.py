"""CPU FP64 reference of the learned head proposal network (oracle; test-only).

The network is a spec addition (the paper trains no model; it only
notes that neural operators consume the generated data). Definition, as
documented in the library header:

* input: per coarse node (32 x 32) the mean of log a over its 4 x 4 block of the
  s x s node field, and the node coordinates ((I + 1/2)/32, (J + 1/2)/32);
* lift v0 = in Wl + bl (3 -> 32 channels);
* 4 Fourier layers: a = Re(G (R (F v))) + v Wp + bp, v' = gelu(a) (no gelu after
  the last), where F keeps the DFT modes k1 in {0..11, 20..31}, k2 in {0..11}
  (e^{-i theta}, theta = 2 pi (k1 x + k2 y)/32), R multiplies each mode by its
  own complex 32 x 32 matrix, and G maps back with e^{+i theta}, weight 1 for
  k2 = 0 and 2 for k2 > 0, divided by 1024;
* heads: Y = gelu(v Wh + bh) Wy (1024 x 64 coarse block through a 128-wide hidden
  layer, so the block can have full rank), s = mean_nodes(v) Wb + bb;
* loss terms, batch means: sub = 64 - tr((G + delta I)^-1 C^T C) with G = Y^T Y,
  C = Q^T Y (the sum of squared sines of the principal angles between span Y and
  span Q as delta -> 0), orth = |G - I|_F^2, bounds = |s - t|^2; the training
  objective is sub + mu orth + bounds, delta = 1e-3, mu = 0.01.

Parameters are one flat vector: Wl [3][32], bl [32], then per layer Rr [288][32][32],
Ri [288][32][32], Wp [32][32], bp [32], then Wh [32][128], bh [128], Wy [128][64],
Wb [32][2], bb [2]; every
block starts at a multiple of 64 entries. gelu is the tanh form
0.5 x (1 + tanh(sqrt(2/pi) (x + 0.044715 x^3))).
"""
from __future__ import annotations

import numpy as np

S, W, MODES, L, KY, H, CIN = 32, 32, 12, 4, 64, 128, 3
DELTA, MU = 1e-3, 0.01
K1 = np.concatenate([np.arange(MODES), np.arange(S - MODES, S)])
K2 = np.arange(MODES)
M = len(K1) * len(K2)


def layout():
    off = {}
    o = 0

    def take(name, n):
        nonlocal o
        off[name] = (o, n)
        o += (n + 63) // 64 * 64

    take("Wl", CIN * W)
    take("bl", W)
    for l in range(L):
        take(f"Rr{l}", M * W * W)
        take(f"Ri{l}", M * W * W)
        take(f"Wp{l}", W * W)
        take(f"bp{l}", W)
    take("Wh", W * H)
    take("bh", H)
    take("Wy", H * KY)
    take("Wb", W * 2)
    take("bb", 2)
    return off, o


OFFSETS, COUNT = layout()


def unpack(params):
    def g(name, shape):
        a, n = OFFSETS[name]
        return np.asarray(params[a:a + n], dtype=np.float64).reshape(shape)
    p = {"Wl": g("Wl", (CIN, W)), "bl": g("bl", (W,)), "Wh": g("Wh", (W, H)),
         "bh": g("bh", (H,)), "Wy": g("Wy", (H, KY)),
         "Wb": g("Wb", (W, 2)), "bb": g("bb", (2,))}
    for l in range(L):
        p[f"R{l}"] = g(f"Rr{l}", (M, W, W)) + 1j * g(f"Ri{l}", (M, W, W))
        p[f"Wp{l}"] = g(f"Wp{l}", (W, W))
        p[f"bp{l}"] = g(f"bp{l}", (W,))
    return p


def gelu(x):
    return 0.5 * x * (1.0 + np.tanh(np.sqrt(2.0 / np.pi) * (x + 0.044715 * x ** 3)))


def inverse_matrix():
    """G [1024, M]: e^{+i theta} with weights 1 (k2 = 0) or 2 (k2 > 0), over 1024."""
    x, y = np.meshgrid(np.arange(S), np.arange(S), indexing="ij")
    x, y = x.ravel(), y.ravel()
    kk1, kk2 = np.meshgrid(K1, K2, indexing="ij")
    kk1, kk2 = kk1.ravel(), kk2.ravel()
    theta = 2 * np.pi * (np.outer(x, kk1) + np.outer(y, kk2)) / S
    w = np.where(kk2 == 0, 1.0, 2.0) / (S * S)
    return np.exp(1j * theta) * w[None, :]


G_INV = inverse_matrix()


def spectral_conv(v, R):
    """Re(G (R (F v))) for v [B, 1024, w] (node-major) and R [M, w, w'] complex."""
    B, w = v.shape[0], v.shape[2]
    spec = np.fft.fft2(v.reshape(B, S, S, w), axes=(1, 2))            # e^{-i theta}
    Vhat = spec[:, K1][:, :, K2].reshape(B, M, w)
    Uhat = np.einsum("bmw,mwo->bmo", Vhat, R)
    return np.real(np.einsum("pm,bmo->bpo", G_INV, Uhat))


def block_terms(Y, Q):
    """(sub, orth) for one block Y [P, 64] and orthonormal targets Q [P, 64]."""
    G = Y.T @ Y
    C = Q.T @ Y
    Minv = np.linalg.inv(G + DELTA * np.eye(Y.shape[1]))
    sub = Y.shape[1] - np.trace(Minv @ C.T @ C)
    orth = np.sum((G - np.eye(Y.shape[1])) ** 2)
    return float(sub), float(orth)


def forward(params, fields):
    """(s [B, 2], Y [B, 1024, 64]) for fields [B, s, s] of positive coefficients."""
    p = unpack(params)
    B, s = fields.shape[0], fields.shape[1]
    f = s // S
    pooled = np.log(fields).reshape(B, S, f, S, f).mean(axis=(2, 4))
    xs = (np.arange(S) + 0.5) / S
    X, Yc = np.meshgrid(xs, xs, indexing="ij")
    inp = np.stack([pooled, np.broadcast_to(X, pooled.shape), np.broadcast_to(Yc, pooled.shape)],
                   axis=-1).reshape(B, S * S, CIN)
    v = inp @ p["Wl"] + p["bl"]
    for l in range(L):
        a = spectral_conv(v, p[f"R{l}"]) + v @ p[f"Wp{l}"] + p[f"bp{l}"]
        v = gelu(a) if l + 1 < L else a
    Yb = gelu(v @ p["Wh"] + p["bh"]) @ p["Wy"]
    sb = v.mean(axis=1) @ p["Wb"] + p["bb"]
    return sb, Yb


def loss(params, fields, t_bounds, t_Q):
    """Batch means of the three loss terms: (sub, orth, bounds)."""
    sb, Yb = forward(params, fields)
    B = fields.shape[0]
    l1 = l2 = 0.0
    for b in range(B):
        e1, e2 = block_terms(Yb[b], t_Q[b])
        l1 += e1
        l2 += e2
    l3 = np.sum((sb - t_bounds) ** 2)
    return l1 / B, l2 / B, l3 / B


def bf16_round(x):
    """Round FP32 values to the nearest BF16 (round to nearest even), as FP64."""
    x32 = np.asarray(x, dtype=np.float32)
    u = x32.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    u = (u + 0x7FFF + lsb) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def matrix_mask():
    """True for entries used in BF16 (all matrices), False for the FP32 biases."""
    mask = np.zeros(COUNT, dtype=bool)
    for name, (a, n) in OFFSETS.items():
        if not name.startswith("b"):
            mask[a:a + n] = True
    return mask


def objective(params, fields, t_bounds, t_Q):
    """The trained scalar: sub + mu orth + bounds."""
    l1, l2, l3 = loss(params, fields, t_bounds, t_Q)
    return l1 + MU * l2 + l3
