"""GPU parity of the scaled form C <- alpha * A.B + beta * C (xGEMM's ALPHA
and BETA, Sec. 2.3.1) through the C ABI against the oracle's scaled form, for
every kernel family and precision form.

Float data: each element within 2 (K + 3) u (|alpha| sum |A||B| + |beta||C0|)
and the normwise tolerance of the form; integer data with integer alpha,
beta: bit-exact.  beta == 0 runs on a C full of NaN (it must not be read)."""
import numpy as np
import pytest

import oracle
from paper_2410_06770_gb300 import gett, synth
from tests._gpu_util import TOL, UNIT, problem_for, run_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2410_06770_gb300 import build
    build.build()
    gett.lib()


def _nan_c(p):
    """The same problem with NaN in every logical C element."""
    q = p.copy()
    pos = oracle.output_positions(q.sig.extc(), q.args()["INCC"], q.lc.off)
    q.C = q.C.copy()
    q.C[pos] = np.nan
    return q


def compare_scaled(prefix, p, got, alpha, beta, exact=False, tol=None):
    ref_buf = oracle.gett_scaled(p, alpha, beta, "z" if np.iscomplexobj(p.A) else "f64")
    gaps = synth.gap_mask(p.lc)
    assert np.array_equal(got[gaps].view(np.uint8), p.C[gaps].view(np.uint8)), "C gaps were modified"
    g = synth.gather(p.lc, got).astype(np.complex128 if np.iscomplexobj(got) else np.float64)
    r = synth.gather(p.lc, ref_buf)
    if exact:
        assert np.array_equal(g, r), f"max |diff| {np.max(np.abs(g - r)) if g.size else 0}"
        return 0.0
    assert np.all(np.isfinite(g)), "non-finite output"
    # |alpha| sum |A||B| + |beta| |C0| per element
    q = p.copy()
    q.A = np.abs(oracle.widen(p.A)).astype(np.float64)
    q.B = np.abs(oracle.widen(p.B)).astype(np.float64)
    C0 = np.abs(oracle.widen(p.C)).astype(np.float64)
    q.C = np.zeros_like(C0)
    s_abs = synth.gather(p.lc, oracle.gett_problem(q, "f64"))
    c_abs = synth.gather(p.lc, C0) if beta != 0 else 0.0
    bound = abs(alpha) * s_abs + abs(beta) * c_abs
    K = max(1, int(np.prod([p.sig.exta[m] for m in p.sig.conta], dtype=np.int64)))
    factor = 2.0 * (K + 3) * UNIT[prefix] * (2.0 if np.iscomplexobj(got) else 1.0)
    err = np.abs(g - r)
    assert np.all(err <= factor * bound + 1e-300), f"element error {np.max(err - factor * bound)} above the bound"
    nr = np.linalg.norm(r)
    rel = np.linalg.norm(g - r) / nr if nr > 0 else np.linalg.norm(g - r)
    assert rel <= (tol if tol is not None else TOL[prefix]), f"normwise error {rel}"
    return rel


SHAPES = {
    # family forced: signature, layouts
    "dense": (synth.Signature((70, 33, 9), (9, 45, 3), (2,), (0,), (1, 2, 0, 3)), ("padded", "negative", "padded")),
    "outer": (synth.Signature((37, 129), (3, 67), (), (), (2, 0, 3, 1)), ("padded", "negative", "padded")),
    "reduce": (synth.Signature((3, 1001, 17), (17, 1001), (1, 2), (1, 0), (0,)), ("padded", "negative", "padded")),
    "skinny": (synth.Signature((700, 3000), (3000, 3), (1,), (0,), (0, 1)), ("padded", "contig", "negative")),
    "short_sum": (synth.Signature((300, 3, 40), (3, 25), (1,), (0,), (0, 2, 1)), ("contig", "padded", "contig")),
}
FAMILY = {"dense": "dense", "outer": "outer", "reduce": "reduce", "skinny": "skinny", "short_sum": "outer"}
REAL_SCALES = [(2.5, -0.75), (-1.5, 0.0), (0.0, 2.0), (1.0, 1.0)]
COMPLEX_SCALES = [(0.5 - 1.25j, -0.3 + 0.7j), (2j, 0.0), (1.0, -1.0)]


def _problem(name, prefix, seed=0, dist="uniform"):
    sig, kinds = SHAPES[name]
    rng = np.random.default_rng(900 + seed + sum(map(ord, name)))
    dtype = np.complex128 if prefix in ("z", "c") else np.float64
    return problem_for(prefix, synth.make_problem(sig, rng, dtype, dist, kinds, dist))


@pytest.mark.parametrize("prefix", ("d", "s", "z", "c", "sb"))
@pytest.mark.parametrize("name", sorted(SHAPES))
def test_scaled_families(prefix, name):
    scales = COMPLEX_SCALES + REAL_SCALES if prefix in ("z", "c") else REAL_SCALES
    for alpha, beta in scales:
        p = _problem(name, prefix)
        if beta == 0:
            p = _nan_c(p)
        got, rep = run_gpu(prefix, p, mode="scaled", opts=gett.options(family=FAMILY[name]), alpha=alpha, beta=beta)
        if alpha != 0:
            assert rep["family_name"] == FAMILY[name]
        compare_scaled(prefix, p, got, alpha, beta)


@pytest.mark.parametrize("split_k", (1, 4))
@pytest.mark.parametrize("prefix", ("d", "z"))
def test_scaled_dense_split_k(prefix, split_k):
    p = _problem("dense", prefix, seed=1)
    for alpha, beta in ((2.5, -0.75), (-1.5, 0.0)):
        q = _nan_c(p) if beta == 0 else p
        got, rep = run_gpu(prefix, q, mode="scaled", opts=gett.options(family="dense", config=1, split_k=split_k),
                           alpha=alpha, beta=beta)
        compare_scaled(prefix, q, got, alpha, beta)


@pytest.mark.parametrize("prefix", ("d", "s", "z", "c"))
@pytest.mark.parametrize("family", synth.THESIS_TESTS)
def test_scaled_integer_exact(prefix, family):
    """alpha = 2, beta = -3 on integer data: bit-exact on every family the
    selector picks."""
    dtype = np.complex128 if prefix in ("z", "c") else np.float64
    p = problem_for(prefix, synth.thesis_problem(family, 600, dtype, "int", c_dist="int"))
    got, _ = run_gpu(prefix, p, mode="scaled", alpha=2.0, beta=-3.0)
    compare_scaled(prefix, p, got, 2.0, -3.0, exact=True)


def test_scaled_one_one_equals_plain():
    """alpha = beta = 1 runs Alg. 1's accumulation: bitwise the plain call."""
    p = synth.cfg_small_dgett()
    a, _ = run_gpu("d", p)
    b, _ = run_gpu("d", p, mode="scaled", alpha=1.0, beta=1.0)
    assert np.array_equal(a, b)


@pytest.mark.parametrize("prefix", ("d", "z"))
def test_scaled_empty_sum_and_alpha_zero(prefix):
    dtype = np.complex128 if prefix == "z" else np.float64
    sig = synth.Signature((3, 0, 5), (0, 4), (1,), (0,), (2, 0, 1))
    p = synth.make_problem(sig, np.random.default_rng(3), dtype, "int", ("padded", "contig", "padded"), "int")
    for beta in (2.0, 0.0, 1.0):
        q = _nan_c(p) if beta == 0 else p
        got, _ = run_gpu(prefix, q, mode="scaled", alpha=3.0, beta=beta)
        compare_scaled(prefix, q, got, 3.0, beta, exact=True)
    # alpha == 0: A, B not read (NaN there), C <- beta C
    q = synth.thesis_problem("basic", 71, dtype, "int", c_dist="int")
    q.A = q.A.copy()
    q.A[:] = np.nan
    got, rep = run_gpu(prefix, q, mode="scaled", alpha=0.0, beta=-2.0)
    compare_scaled(prefix, q, got, 0.0, -2.0, exact=True)
    got, _ = run_gpu(prefix, _nan_c(q), mode="scaled", alpha=0.0, beta=0.0)
    compare_scaled(prefix, _nan_c(q), got, 0.0, 0.0, exact=True)


# ---- tensor-core forms ----------------------------------------------------
def _tc_problem(prefix, dist="uniform", seed=0):
    sig = synth.Signature((520, 300), (300, 530), (1,), (0,), (0, 1))
    rng = np.random.default_rng(1200 + seed)
    dtype = np.complex128 if prefix == "z" else np.float64
    return problem_for(prefix, synth.make_problem(sig, rng, dtype, dist, ("contig", "padded", "contig"), dist))


@pytest.mark.parametrize("alpha,beta", [(2.5, -0.75), (-1.5, 0.0)])
def test_scaled_bf16_tensor_cores(alpha, beta):
    p = _tc_problem("sb")
    p = _nan_c(p) if beta == 0 else p
    got, rep = run_gpu("sb", p, mode="scaled", opts=gett.options(family="tc"), alpha=alpha, beta=beta)
    assert rep["family_name"] == "tc"
    compare_scaled("sb", p, got, alpha, beta)


@pytest.mark.parametrize("algo", ("bf16x6",))
@pytest.mark.parametrize("alpha,beta", [(2.5, -0.75), (-1.5, 0.0)])
def test_scaled_sgett_split(algo, alpha, beta):
    p = _tc_problem("s")
    p = _nan_c(p) if beta == 0 else p
    got, rep = run_gpu("s", p, mode="scaled", opts=gett.options(algo=algo), alpha=alpha, beta=beta)
    assert rep["family_name"] == "tc"
    compare_scaled("s", p, got, alpha, beta)


@pytest.mark.parametrize("alpha,beta", [(2.5, -0.75), (-1.5, 0.0), (1.0, 1.0)])
def test_scaled_dgett_split_precision(alpha, beta):
    p = _tc_problem("d")
    p = _nan_c(p) if beta == 0 else p
    got, rep = run_gpu("d", p, mode="scaled", opts=gett.options(algo="ozaki_bf16"), alpha=alpha, beta=beta)
    assert rep["family_name"] == "tc" and rep["moduli"] > 0
    compare_scaled("d", p, got, alpha, beta)


@pytest.mark.parametrize("alpha,beta", [(2.5, -0.75), (0.5 - 1.25j, -0.3 + 0.7j), (2j, 0.0), (-1.0, 1j)])
def test_scaled_zgett_split_precision(alpha, beta):
    """Real alpha, beta act on each part in the recombination; a non-real one
    goes through the staged product."""
    sig = synth.Signature((130, 90), (90, 70), (1,), (0,), (0, 1))
    rng = np.random.default_rng(1300)
    p = synth.make_problem(sig, rng, np.complex128, "uniform", ("padded", "negative", "contig"), "uniform")
    p = _nan_c(p) if beta == 0 else p
    got, rep = run_gpu("z", p, mode="scaled", opts=gett.options(algo="ozaki_bf16"), alpha=alpha, beta=beta)
    assert rep["family_name"] == "tc" and rep["moduli"] > 0
    compare_scaled("z", p, got, alpha, beta)


def test_scaled_integer_exact_split_precision():
    p = _tc_problem("d", dist="int", seed=2)
    got, _ = run_gpu("d", p, mode="scaled", opts=gett.options(algo="ozaki_bf16"), alpha=2.0, beta=-3.0)
    compare_scaled("d", p, got, 2.0, -3.0, exact=True)
