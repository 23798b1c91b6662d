"""Pins of the fp64 planner-network reference (CPU): its analytic gradient
against central finite differences of its own loss, on a network small
enough to check every parameter."""
import numpy as np

from oracle import mlp_oracle


def test_reference_gradient_matches_finite_differences():
    rng = np.random.default_rng(0)
    nf, h, no, n = 5, 7, 3, 11
    npar = h * nf + h + h * h + h + no * h + no
    p = rng.standard_normal(npar) * 0.5
    X = rng.standard_normal((n, nf))
    T = rng.standard_normal((n, no))
    M = (rng.random((n, no)) < 0.8).astype(np.float64)
    _, g = mlp_oracle.loss_grad(p, X, T, M, nf, h, no)
    eps = 1e-6
    fd = np.zeros_like(p)
    for i in range(npar):
        pp = p.copy(); pp[i] += eps
        pm = p.copy(); pm[i] -= eps
        fd[i] = (mlp_oracle.loss_grad(pp, X, T, M, nf, h, no)[0] -
                 mlp_oracle.loss_grad(pm, X, T, M, nf, h, no)[0]) / (2 * eps)
    assert np.max(np.abs(fd - g)) <= 1e-6 * max(1.0, np.max(np.abs(g)))


def test_reference_loss_is_masked_mse():
    nf, h, no = 2, 3, 2
    p = np.zeros(h * nf + h + h * h + h + no * h + no)
    p[-no:] = [1.0, 2.0]  # b3: constant predictions
    X = np.ones((2, nf))
    T = np.array([[0.0, 0.0], [1.0, 5.0]])
    M = np.array([[1.0, 0.0], [1.0, 1.0]])
    loss, _ = mlp_oracle.loss_grad(p, X, T, M, nf, h, no)
    assert abs(loss - (1.0 + 0.0 + 9.0) / 3.0) < 1e-15
