"""GPU checks of the planner network's own kernels against the fp64 CPU
reference: forward outputs, loss and every gradient (<= 1e-4 relative),
training that lowers the loss, and installation as the batch planner."""
import numpy as np
import pytest

from oracle import mlp_oracle
from paper_2410_06770_gb300 import batch as gb

pytestmark = pytest.mark.gpu

NF, H, NO = gb.NFEAT, 128, 4


def data(n, seed):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((n, NF)).astype(np.float32)
    W = rng.standard_normal((NF, NO))
    T = (np.tanh(X @ W) + 0.1 * rng.standard_normal((n, NO))).astype(np.float32)
    M = (rng.random((n, NO)) < 0.9).astype(np.float32)
    return X, T, M


def test_forward_matches_reference():
    m = gb.MLP(NF, H, NO, seed=1)
    X, _, _ = data(64, 0)
    y = m.predict(X)
    ref, _ = mlp_oracle.forward(m.get_params(), X, NF, H, NO)
    assert np.max(np.abs(y - ref)) <= 1e-4 * max(1.0, np.max(np.abs(ref)))


@pytest.mark.parametrize("n", [1, 37, 256])
def test_gradients_match_reference(n):
    m = gb.MLP(NF, H, NO, seed=2)
    X, T, M = data(n, n)
    loss, g = m.loss_grad(X, T, M)
    rloss, rg = mlp_oracle.loss_grad(m.get_params(), X, T, M, NF, H, NO)
    assert abs(loss - rloss) <= 1e-4 * max(1.0, abs(rloss))
    assert np.linalg.norm(g - rg) <= 1e-4 * max(1e-6, np.linalg.norm(rg))
    assert np.max(np.abs(g - rg)) <= 1e-4 * max(1e-6, np.max(np.abs(rg)))


def test_adam_steps_match_reference():
    """Three Adam steps of gett_mlp_fit (one sample, so the minibatch order
    cannot change the gradient) against the fp64 Adam step fed the same GPU
    gradient: parameters within fp32 rounding of the update, and the reported
    loss that of the parameters before the step."""
    m = gb.MLP(NF, H, NO, seed=9)
    X, T, M = data(1, 11)
    p = m.get_params().astype(np.float64)
    mom = np.zeros_like(p)
    vel = np.zeros_like(p)
    lr = 1e-3
    for t in range(1, 4):
        loss, g = m.loss_grad(X, T, M)
        fit_loss = m.fit(X, T, M, epochs=1, batch=1, lr=lr, seed=t)
        assert fit_loss == loss
        p, mom, vel = mlp_oracle.adam_step(p, g.astype(np.float64), mom, vel, t, lr)
        got = m.get_params().astype(np.float64)
        # fp32 rounding of p at each step, and the fp32 betas and bias
        # corrections (relative 1.3e-5 on 1 - beta2) on an update of at most
        # about 3 lr
        assert np.all(np.abs(got - p) <= 4 * t * 2.0 ** -24 * np.abs(p) + 1e-4 * t * lr)


def test_training_reduces_loss_and_is_deterministic():
    X, T, M = data(2000, 5)
    losses = []
    params = []
    for _ in range(2):
        m = gb.MLP(NF, H, NO, seed=3)
        l0, _ = m.loss_grad(X[:512], T[:512], M[:512])
        lf = m.fit(X, T, M, epochs=20, batch=128, lr=1e-3, seed=4)
        losses.append((l0, lf))
        params.append(m.get_params())
    assert losses[0][1] < 0.5 * losses[0][0]
    assert np.array_equal(params[0], params[1])


def test_installed_model_drives_host_prediction():
    m = gb.MLP(NF, H, NO, seed=6)
    p = m.get_params()
    mean = np.zeros(NF, dtype=np.float32)
    std = np.ones(NF, dtype=np.float32)
    gb.install_model(p, mean, std, H, NO)
    X, _, _ = data(8, 1)
    L = gb._bind()
    ref, _ = mlp_oracle.forward(p, X, NF, H, NO)
    for i in range(8):
        out = np.zeros(NO, dtype=np.float32)
        assert L.gett_learn_predict(gb._f(np.ascontiguousarray(X[i])), gb._f(out)) == 0
        assert np.max(np.abs(out - ref[i])) <= 1e-4 * max(1.0, np.max(np.abs(ref[i])))
    gb.clear_model()
