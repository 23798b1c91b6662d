"""CPU fp64 reference of the planner network -- TEST INFRASTRUCTURE ONLY.

Network: x -> relu(W1 x + b1) -> relu(W2 h1 + b2) -> W3 h2 + b3.
Loss: sum(mask * (y - t)^2) / sum(mask).  Parameters are one flat vector in
the layout W1[h][f], b1[h], W2[h][h], b2[h], W3[o][h], b3[o].  Written from
the definitions (chain rule by hand); pinned by central finite differences in
tests/test_mlp_cpu.py.  The optimiser step is Adam (Kingma and Ba, 2015,
their Algorithm 1), pinned there by its closed forms and by torch.optim.Adam.
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


def adam_step(p, g, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update at step t >= 1 (Kingma and Ba, 2015, Algorithm 1), fp64:
    moving averages of g and g^2, each divided by its bias correction
    1 - beta^t, then p <- p - lr * mhat / (sqrt(vhat) + eps).
    Returns (p, m, v) as new arrays."""
    p, g, m, v = (np.asarray(a, dtype=np.float64) for a in (p, g, m, v))
    m = b1 * m + (1.0 - b1) * g
    v = b2 * v + (1.0 - b2) * g * g
    mhat = m / (1.0 - b1 ** t)
    vhat = v / (1.0 - b2 ** t)
    return p - lr * mhat / (np.sqrt(vhat) + eps), m, v
