"""Pins of the fp64 planner-network reference (CPU): its analytic gradient
against central finite differences of its own loss, on a network small
enough to check every parameter; its Adam step against closed forms and
torch.optim.Adam.  Host logic of the learned planner: inference of an
installed model against the reference forward, and the feature vector's
definition and invariances."""
import numpy as np
import pytest

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


# --- Adam (Kingma and Ba, 2015, Algorithm 1): pins of the oracle's step ---

def test_adam_first_step_closed_form():
    """Step 1: mhat = g and vhat = g^2, so p moves by lr * g / (|g| + eps);
    a zero gradient does not move p."""
    rng = np.random.default_rng(1)
    p0 = rng.standard_normal(50)
    g = rng.standard_normal(50) * 10.0 ** rng.uniform(-12, 2, 50)
    g[:5] = 0.0
    lr = 1e-3
    p1, m, v = mlp_oracle.adam_step(p0, g, np.zeros(50), np.zeros(50), 1, lr)
    assert np.allclose(p1, p0 - lr * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)
    assert np.array_equal(p1[:5], p0[:5])
    assert np.allclose(m, 0.1 * g, rtol=1e-14, atol=0) and np.allclose(v, 0.001 * g * g, rtol=1e-14, atol=0)


def test_adam_constant_gradient_moves_lr_per_step():
    """A constant gradient keeps mhat = g and vhat = g^2 at every step (the bias
    corrections divide out exactly), so t steps move p by t * lr * g / (|g| + eps)."""
    rng = np.random.default_rng(2)
    p = p0 = rng.standard_normal(20)
    g = rng.standard_normal(20)
    m = v = np.zeros(20)
    lr = 3e-3
    for t in range(1, 51):
        p, m, v = mlp_oracle.adam_step(p, g, m, v, t, lr)
    assert np.allclose(p, p0 - 50 * lr * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-12)


def test_adam_matches_torch_optim():
    """Twenty steps on a random gradient sequence against torch.optim.Adam
    (fp64, default betas and eps), a library implementation of the same update."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(3)
    p0 = rng.standard_normal(64)
    grads = rng.standard_normal((20, 64)) * 10.0 ** rng.uniform(-6, 1, (20, 64))
    w = torch.tensor(p0, dtype=torch.float64, requires_grad=True)
    opt = torch.optim.Adam([w], lr=1e-2)
    p, m, v = p0, np.zeros(64), np.zeros(64)
    for t in range(1, 21):
        w.grad = torch.tensor(grads[t - 1], dtype=torch.float64)
        opt.step()
        p, m, v = mlp_oracle.adam_step(p, grads[t - 1], m, v, t, 1e-2)
    assert np.max(np.abs(p - w.detach().numpy())) <= 1e-14


# --- host inference of an installed model and the planner's features ---

def _lib():
    from paper_2410_06770_gb300 import batch as gb
    from paper_2410_06770_gb300 import build
    build.build()
    return gb


def test_host_inference_matches_reference():
    """gett_learn_predict normalises the raw features with the installed mean
    and std and runs the network on the host: the fp64 reference forward on the
    normalised input, to fp32 rounding."""
    gb = _lib()
    L = gb._bind()
    nf, h, no = gb.NFEAT, 16, 4
    rng = np.random.default_rng(4)
    npar = h * nf + h + h * h + h + no * h + no
    p = (rng.standard_normal(npar) * 0.3).astype(np.float32)
    mean = rng.standard_normal(nf).astype(np.float32)
    std = rng.uniform(0.5, 2.0, nf).astype(np.float32)
    std[3] = 0.0  # a zero deviation leaves that feature unscaled
    gb.install_model(p, mean, std, h, no)
    try:
        X = rng.standard_normal((6, nf)).astype(np.float32) * 3
        Z = (X.astype(np.float64) - mean) / np.where(std > 0, std, 1.0).astype(np.float64)
        ref, _ = mlp_oracle.forward(p, Z, nf, h, no)
        for i in range(6):
            out = np.zeros(no, dtype=np.float32)
            assert L.gett_learn_predict(gb._f(np.ascontiguousarray(X[i])), gb._f(out)) == 0
            assert np.max(np.abs(out - ref[i])) <= 1e-5 * max(1.0, np.max(np.abs(ref[i])))
        # a parameter set that predicts a non-finite time is rejected
        bad = p.copy()
        bad[-1] = np.inf
        gb.install_model(bad, mean, std, h, no)
        out = np.zeros(no, dtype=np.float32)
        assert L.gett_learn_predict(gb._f(np.ascontiguousarray(X[0])), gb._f(out)) != 0
    finally:
        gb.clear_model()
    out = np.zeros(no, dtype=np.float32)
    assert L.gett_learn_predict(gb._f(np.zeros(nf, dtype=np.float32)), gb._f(out)) != 0  # no model


def _gemm4():
    # C[a,b,i,j] += A[a,b,c,d] B[c,d,i,j], column-major: fuses to M = 6, N = 6, K = 20
    return dict(EXTA=(2, 3, 4, 5), INCA=(1, 2, 6, 24), EXTB=(4, 5, 3, 2), INCB=(1, 4, 20, 60),
                CONTA=(2, 3), CONTB=(0, 1), PERM=(0, 1, 2, 3), INCC=(1, 2, 6, 18))


def test_features_of_a_gemm():
    """M, N, K are the products of the free and contracted extents; a
    column-major problem fuses to one mode per class."""
    gb = _lib()
    f = gb.features(_gemm4(), "f32").astype(np.float64)
    lg = lambda x: np.log2(x + 1.0)
    assert np.allclose(f[:4], [lg(6), lg(6), lg(20), lg(6 * 6 * 20) / 3], rtol=1e-6)
    assert list(f[4:7]) == [1, 1, 1]
    assert f[19] == 0 and f[23] == 1
    assert np.allclose(f[20:23], [6 / 32, 6 / 32, 20 % 16 / 16])


def test_features_invariant_under_fusion_squeeze_and_reversal():
    """The features describe the planned problem: the fused two-mode GEMM, the
    same problem with an extent-1 mode inserted (any increment), and the problem
    with index b running backwards in every tensor holding it all give the same
    vector; the operand type changes only its own entry."""
    gb = _lib()
    base = gb.features(_gemm4(), "f32")
    fused = dict(EXTA=(6, 20), INCA=(1, 6), EXTB=(20, 6), INCB=(1, 20), CONTA=(1,), CONTB=(0,),
                 PERM=(0, 1), INCC=(1, 6))
    unit = dict(EXTA=(2, 1, 3, 4, 5), INCA=(1, 1000, 2, 6, 24), EXTB=(4, 5, 3, 2), INCB=(1, 4, 20, 60),
                CONTA=(3, 4), CONTB=(0, 1), PERM=(0, 1, 2, 3, 4), INCC=(1, 7777, 2, 6, 18))
    rev = _gemm4()
    rev["INCA"] = (1, -2, 6, 24)
    rev["INCC"] = (1, -2, 6, 18)
    for other in (fused, unit, rev):
        assert np.array_equal(gb.features(other, "f32"), base)
    b16 = gb.features(_gemm4(), "bf16")
    assert b16[19] == 1 and np.array_equal(np.delete(b16, 19), np.delete(base, 19))


def test_features_of_an_empty_problem_and_bad_arguments():
    gb = _lib()
    from paper_2410_06770_gb300 import gett
    empty = _gemm4()
    empty["EXTA"] = (2, 0, 4, 5)
    assert not np.any(gb.features(empty, "f32"))
    bad = _gemm4()
    bad["PERM"] = (0, 1, 1, 3)
    with pytest.raises(gett.GettError):
        gb.features(bad, "f32")
