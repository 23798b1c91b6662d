"""Pins for the oracle's scaled form C <- alpha * S + beta * C (the ALPHA and
BETA of xGEMM / xGEMV, Sec. 2.3.1; S the contraction of Sec. 2.2).

References: numpy's BLAS matmul and int64 einsum on the logical tensors,
never the oracle itself.  BLAS conventions pinned: beta == 0 does not read C
(NaN there does not propagate); alpha == 0 does not form the product."""
import numpy as np
import pytest

import oracle
from paper_2410_06770_gb300 import synth
from tests._einsum_ref import einsum_spec

SCALES = [(2.5, -0.75), (-1.0, 0.0), (0.3, 1.0), (1.0, 0.0), (0.0, 2.0)]


def _logical(p, buf):
    return synth.logical(p.lc, buf)


@pytest.mark.parametrize("alpha,beta", SCALES)
@pytest.mark.parametrize("conta,contb,perm", [(0, 0, (0, 1)), (1, 1, (1, 0)), (1, 0, (0, 1))])
def test_scaled_gemm_matches_blas(alpha, beta, conta, contb, perm):
    """Rank-2 x rank-2, one contraction: xGEMM's C <- alpha op(A) op(B) + beta C
    (Sec. 2.3.1), op chosen by the contracted modes, PERM (1, 0) transposing
    the product.  numpy sums in another order: agreement to 1e-14."""
    m, k, n = 23, 31, 19
    rng = np.random.default_rng(300 + 4 * conta + 2 * contb + perm[0])
    exta = (k, m) if conta == 0 else (m, k)
    extb = (k, n) if contb == 0 else (n, k)
    sig = synth.Signature(exta, extb, (conta,), (contb,), perm)
    p = synth.make_problem(sig, rng, np.float64, "uniform", ("padded", "negative", "padded"), "uniform")
    Am = synth.logical(p.la, p.A)
    Bm = synth.logical(p.lb, p.B)
    prod = (Am.T if conta == 0 else Am) @ (Bm if contb == 0 else Bm.T)
    if perm == (1, 0):
        prod = prod.T
    ref = alpha * prod + beta * synth.logical(p.lc, p.C)
    got = _logical(p, oracle.gett_scaled(p, alpha, beta))
    assert np.linalg.norm(got - ref) <= 1e-14 * max(np.linalg.norm(ref), 1e-300)


@pytest.mark.parametrize("seed", range(3))
def test_scaled_complex_gemm_matches_blas(seed):
    """Complex alpha and beta (prefix z): products not conjugated."""
    rng = np.random.default_rng(400 + seed)
    sig = synth.Signature((17, 13), (13, 11), (1,), (0,), (0, 1))
    p = synth.make_problem(sig, rng, np.complex128, "uniform", ("contig", "padded", "negative"), "uniform")
    alpha, beta = 0.5 - 1.25j, -0.3 + 0.7j
    ref = alpha * (synth.logical(p.la, p.A) @ synth.logical(p.lb, p.B)) + beta * synth.logical(p.lc, p.C)
    got = _logical(p, oracle.gett_scaled(p, alpha, beta))
    assert np.linalg.norm(got - ref) <= 1e-14 * np.linalg.norm(ref)


@pytest.mark.parametrize("family", synth.THESIS_TESTS)
def test_scaled_integer_exact_vs_einsum(family):
    """Integer data, alpha = 2, beta = -3: every value is an exact double, so
    the result equals int64 2 * einsum - 3 * C0 exactly, and C's gaps keep
    their values."""
    p = synth.thesis_problem(family, 3000, np.float64, "int", c_dist="int")
    E = np.einsum(einsum_spec(p.sig), synth.logical(p.la, p.A).astype(np.int64),
                  synth.logical(p.lb, p.B).astype(np.int64))
    ref = 2 * E - 3 * synth.logical(p.lc, p.C).astype(np.int64)
    out = oracle.gett_scaled(p, 2.0, -3.0)
    assert np.array_equal(_logical(p, out), ref.astype(np.float64)), einsum_spec(p.sig)
    gaps = synth.gap_mask(p.lc)
    assert np.array_equal(out[gaps], p.C[gaps], equal_nan=True)


def test_beta_zero_does_not_read_c():
    """beta == 0: C may hold NaN; the result is alpha * S, finite."""
    p = synth.thesis_problem("basic", 3100, np.float64, "int", c_dist="int")
    q = p.copy()
    pos = oracle.output_positions(q.sig.extc(), q.args()["INCC"], q.lc.off)
    q.C[pos] = np.nan
    got = _logical(q, oracle.gett_scaled(q, -2.0, 0.0))
    E = np.einsum(einsum_spec(p.sig), synth.logical(p.la, p.A).astype(np.int64),
                  synth.logical(p.lb, p.B).astype(np.int64))
    assert np.array_equal(got, (-2 * E).astype(np.float64))


def test_alpha_zero_scales_c_only():
    """alpha == 0: C <- beta * C exactly, A and B not used (NaN there is
    harmless); beta == 0 as well gives zeros."""
    p = synth.thesis_problem("basic", 3200, np.float64, "int", c_dist="int")
    q = p.copy()
    q.A[:] = np.nan
    C0 = synth.logical(p.lc, p.C)
    assert np.array_equal(_logical(q, oracle.gett_scaled(q, 0.0, -1.5)), -1.5 * C0)
    assert np.array_equal(_logical(q, oracle.gett_scaled(q, 0.0, 0.0)), np.zeros_like(C0))


def test_one_one_is_alg1_accumulation():
    """alpha = beta = 1 equals Alg. 1's C + S (bit-exact on integer data)."""
    p = synth.thesis_problem("commutativity", 3300, np.float64, "int", c_dist="int")
    assert np.array_equal(_logical(p, oracle.gett_scaled(p, 1.0, 1.0)), _logical(p, oracle.gett_problem(p)))


def test_empty_sum_scales_c():
    """A contracted extent 0: S = 0, so C <- beta * C."""
    sig = synth.Signature((3, 0), (0, 4), (1,), (0,), (0, 1))
    p = synth.make_problem(sig, np.random.default_rng(5), np.float64, "int", c_dist="int")
    C0 = synth.logical(p.lc, p.C)
    assert np.array_equal(_logical(p, oracle.gett_scaled(p, 3.0, 2.0)), 2 * C0)
