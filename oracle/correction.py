"""Plain FP64 numpy oracle of the learned sub-mesh force correction.

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the CPU leg of the
benchmark may import this module; the library never does.  It shares no code
with the CUDA path.  The paper itself has no learned component: the
network, its inputs and its target are the readings written out below.

Mesh arrays are [C][z][y][x] (x fastest), periodic, vertex-centred.

* Convolution (3^3, periodic cross-correlation, offsets d in {-1,0,1}^3,
  index d = 9 (dz+1) + 3 (dy+1) + (dx+1)):
      y[co](c) = b[co] + sum_d sum_ci W[d, co, ci] x[ci](c + d)
* Network: 2 -> 16 -> 16 -> 16 -> 3 channels, ReLU after the first three
  layers, none after the last.
* Loss: mean over cells and the 3 output channels of (out - target)^2.
* Backward of one layer, with g = dL/dy masked by the ReLU (y > 0):
      dW[d, co, ci] = sum_c g[co](c) x[ci](c + d),   db[co] = sum_c g[co](c),
      dx[ci](c)     = sum_d sum_co W[d, co, ci] g[co](c - d).
* Force on a mesh: F_a(i) = -(phi(i + e_a) - phi(i - e_a)) N / 2.
* Restriction of a 2N mesh field to the N mesh (vertex 2i of the fine mesh
  sits on vertex i of the coarse one): full weighting with weights
  1/2 (offset 0) and 1/4 (offsets +-1) per axis.
* Adam (Kingma & Ba 2015) with bias correction.
"""
from __future__ import annotations

import itertools

import numpy as np

OFFSETS = [(dz, dy, dx) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]
LAYERS = [(2, 16, True), (16, 16, True), (16, 16, True), (16, 3, False)]   # (c_in, c_out, relu)


def shift(x, d):
    """x(c + d) for every cell c of a [C][z][y][x] (or [z][y][x]) array, periodic."""
    dz, dy, dx = d
    return np.roll(x, (-dz, -dy, -dx), axis=(-3, -2, -1))


def conv(x, W, b):
    """3^3 periodic cross-correlation, x [ci][n][n][n], W [27][co][ci], b [co]."""
    out = np.zeros((W.shape[1],) + x.shape[1:])
    for k, d in enumerate(OFFSETS):
        out += np.einsum("oi,izyx->ozyx", W[k], shift(x, d))
    return out + b[:, None, None, None]


def conv_backward(x, W, g):
    """Gradients of sum(g * conv(x, W, b)) with respect to W, b and x."""
    dW = np.zeros_like(W)
    for k, d in enumerate(OFFSETS):
        dW[k] = np.einsum("ozyx,izyx->oi", g, shift(x, d))
    db = g.sum(axis=(1, 2, 3))
    dx = np.zeros_like(x)
    for k, d in enumerate(OFFSETS):
        dx += np.einsum("oi,ozyx->izyx", W[k], shift(g, tuple(-e for e in d)))
    return dW, db, dx


def forward(params, x):
    """params: list of (W, b) per layer.  Returns the output and the list of layer inputs and outputs."""
    acts = [x]
    for (W, b), (_, _, relu) in zip(params, LAYERS):
        y = conv(acts[-1], W, b)
        acts.append(np.maximum(y, 0.0) if relu else y)
    return acts[-1], acts


def loss_and_grads(params, x, target):
    out, acts = forward(params, x)
    m = out.size
    loss = float(np.mean((out - target) ** 2))
    g = 2.0 * (out - target) / m
    grads = [None] * len(params)
    for l in range(len(params) - 1, -1, -1):
        if LAYERS[l][2]:
            g = g * (acts[l + 1] > 0)
        dW, db, dx = conv_backward(acts[l], params[l][0], g)
        grads[l] = (dW, db)
        g = dx
    return loss, grads


def force(phi):
    n = phi.shape[-1]
    return np.stack([-(np.roll(phi, -1, axis=ax) - np.roll(phi, 1, axis=ax)) * n / 2.0 for ax in (2, 1, 0)])


def restrict(fine):
    """Full-weighting restriction of [..][2n][2n][2n] to [..][n][n][n]."""
    acc = 0.0
    for e in itertools.product((-1, 0, 1), repeat=3):
        w = np.prod([0.5 if a == 0 else 0.25 for a in e])
        acc = acc + w * shift(fine, e)
    return acc[..., ::2, ::2, ::2]


def cic_interp(field, pos):
    """Trilinear (CIC) value of a vertex field [n][n][n] at positions pos [np][3] in [0,1)."""
    n = field.shape[-1]
    s = pos * n
    i = np.floor(s).astype(np.int64)
    f = s - i
    out = np.zeros(len(pos))
    for dz, dy, dx in itertools.product((0, 1), repeat=3):
        w = (f[:, 0] if dx else 1 - f[:, 0]) * (f[:, 1] if dy else 1 - f[:, 1]) * (f[:, 2] if dz else 1 - f[:, 2])
        out += w * field[(i[:, 2] + dz) % n, (i[:, 1] + dy) % n, (i[:, 0] + dx) % n]
    return out


def adam(theta, g, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step at step count t (1-based); returns the new (theta, m, v)."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v
