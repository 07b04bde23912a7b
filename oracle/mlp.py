"""The selector network in float64 numpy: forward, masked squared error,
backward and one Adam step, in the flat parameter layout of the library
(W1[H][IN] b1[H] W2[H][H] b2[H] W3[OUT][H] b3[OUT]).

TEST INFRASTRUCTURE ONLY (see the package docstring).  Written from the
definitions: a two-hidden-layer ReLU perceptron, the loss
sum(mask*(out-target)^2)/max(1, sum(mask)), back-propagation by the chain
rule, and Adam (Kingma and Ba, "Adam: a method for stochastic optimization",
ICLR 2015, Algorithm 1).
"""
from __future__ import annotations

import numpy as np

IN, H, OUT = 22, 64, 15


def unpack(p):
    p = np.asarray(p, dtype=np.float64)
    shapes = [(H, IN), (H,), (H, H), (H,), (OUT, H), (OUT,)]
    out, o = [], 0
    for s in shapes:
        k = int(np.prod(s))
        out.append(p[o:o + k].reshape(s))
        o += k
    assert o == p.size
    return out


def pack(parts):
    return np.concatenate([np.asarray(a, dtype=np.float64).ravel() for a in parts])


def forward(p, x):
    W1, b1, W2, b2, W3, b3 = unpack(p)
    x = np.asarray(x, dtype=np.float64)
    z1 = x @ W1.T + b1
    h1 = np.maximum(z1, 0)
    z2 = h1 @ W2.T + b2
    h2 = np.maximum(z2, 0)
    out = h2 @ W3.T + b3
    return out, (x, h1, h2)


def loss(out, target, mask):
    c = max(float(np.sum(mask)), 1.0)
    d = np.asarray(mask, dtype=np.float64) * (out - target)
    return float(np.sum(d * d) / c), 2.0 * d / c


def backward(p, cache, dout):
    W1, b1, W2, b2, W3, b3 = unpack(p)
    x, h1, h2 = cache
    gW3 = dout.T @ h2
    gb3 = dout.sum(0)
    dz2 = (dout @ W3) * (h2 > 0)
    gW2 = dz2.T @ h1
    gb2 = dz2.sum(0)
    dz1 = (dz2 @ W2) * (h1 > 0)
    gW1 = dz1.T @ x
    gb1 = dz1.sum(0)
    return pack([gW1, gb1, gW2, gb2, gW3, gb3])


def adam_step(p, g, m, v, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** step)
    vh = v / (1 - b2 ** step)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v
