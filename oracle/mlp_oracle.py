"""CPU fp64 reference of the planner network -- TEST INFRASTRUCTURE ONLY.

Network: x -> relu(W1 x + b1) -> relu(W2 h1 + b2) -> W3 h2 + b3.
Loss: sum(mask * (y - t)^2) / sum(mask).  Parameters are one flat vector in
the layout W1[h][f], b1[h], W2[h][h], b2[h], W3[o][h], b3[o].  Written from
the definitions (chain rule by hand); pinned by central finite differences in
tests/test_mlp_cpu.py.
"""
import numpy as np


def unpack(p, nfeat, hidden, nout):
    p = np.asarray(p, dtype=np.float64)
    i = 0
    def take(n, shape):
        nonlocal i
        a = p[i:i + n].reshape(shape)
        i += n
        return a
    W1 = take(hidden * nfeat, (hidden, nfeat))
    b1 = take(hidden, (hidden,))
    W2 = take(hidden * hidden, (hidden, hidden))
    b2 = take(hidden, (hidden,))
    W3 = take(nout * hidden, (nout, hidden))
    b3 = take(nout, (nout,))
    assert i == p.size
    return W1, b1, W2, b2, W3, b3


def forward(p, X, nfeat, hidden, nout):
    W1, b1, W2, b2, W3, b3 = unpack(p, nfeat, hidden, nout)
    X = np.asarray(X, dtype=np.float64)
    z1 = X @ W1.T + b1
    h1 = np.maximum(z1, 0)
    z2 = h1 @ W2.T + b2
    h2 = np.maximum(z2, 0)
    y = h2 @ W3.T + b3
    return y, (X, z1, h1, z2, h2)


def loss_grad(p, X, T, M, nfeat, hidden, nout):
    W1, b1, W2, b2, W3, b3 = unpack(p, nfeat, hidden, nout)
    y, (X, z1, h1, z2, h2) = forward(p, X, nfeat, hidden, nout)
    T = np.asarray(T, dtype=np.float64)
    M = np.asarray(M, dtype=np.float64)
    cnt = max(M.sum(), 1.0)
    loss = float((M * (y - T) ** 2).sum() / cnt)
    dy = 2.0 * M * (y - T) / cnt
    gW3 = dy.T @ h2
    gb3 = dy.sum(0)
    dh2 = dy @ W3
    dz2 = dh2 * (z2 > 0)
    gW2 = dz2.T @ h1
    gb2 = dz2.sum(0)
    dh1 = dz2 @ W2
    dz1 = dh1 * (z1 > 0)
    gW1 = dz1.T @ X
    gb1 = dz1.sum(0)
    g = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3.ravel(), gb3])
    return loss, g
