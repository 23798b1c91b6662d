"""GPU parity: the CUDA path through the C ABI against the CPU oracle,
element by element, on the same seeded inputs.

Float data: each element within the rounding bound of any summation order
(2 (K+2) u (|C0| + sum |A||B|)), and the normwise error within the form's
tolerance (1e-13 for d/z, 1e-5 for s/c and bf16 inputs).  Integer data:
bit-exact.  C's gaps (sub-tensor padding) must keep their sentinel bits."""
import numpy as np
import pytest

import oracle
from paper_2410_06770_gb300 import gett, synth
from tests._gpu_util import compare, oracle_ref, problem_for, run_gpu

pytestmark = pytest.mark.gpu

PREFIXES = ("d", "s", "z", "c", "sb")


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2410_06770_gb300 import build
    build.build()
    gett.lib()


@pytest.mark.parametrize("prefix", PREFIXES)
@pytest.mark.parametrize("family", synth.THESIS_TESTS)
@pytest.mark.parametrize("seed", range(3))
def test_thesis_families(prefix, family, seed):
    dtype = np.complex128 if prefix in ("z", "c") else np.float64
    p = synth.thesis_problem(family, 100 + seed, dtype, "uniform", c_dist="uniform")
    q = problem_for(prefix, p)
    got, _ = run_gpu(prefix, q)
    compare(prefix, q, got, oracle_ref(q))


@pytest.mark.parametrize("prefix", PREFIXES)
@pytest.mark.parametrize("family", synth.THESIS_TESTS)
def test_thesis_families_integer_exact(prefix, family):
    dtype = np.complex128 if prefix in ("z", "c") else np.float64
    p = synth.thesis_problem(family, 500, dtype, "int", c_dist="int")
    q = problem_for(prefix, p)
    got, _ = run_gpu(prefix, q)
    compare(prefix, q, got, oracle_ref(q), exact=True)


@pytest.mark.parametrize("prefix", ("d", "s", "z"))
@pytest.mark.parametrize("family", ("dense", "outer", "reduce"))
@pytest.mark.parametrize("seed", range(2))
def test_forced_families_multi_tile(prefix, family, seed):
    """Sizes that span several tiles with ragged tails, each family forced."""
    rng = np.random.default_rng(700 + seed)
    dtype = np.complex128 if prefix == "z" else np.float64
    if family == "outer":
        sig = synth.Signature((37, 129), (3, 67), (), (), (2, 0, 3, 1))
    elif family == "reduce":
        sig = synth.Signature((3, 1001, 17), (17, 1001), (1, 2), (1, 0), (0,))
    else:
        sig = synth.Signature((70, 33, 9), (9, 45, 3), (2,), (0,), (1, 2, 0, 3))
    p = synth.make_problem(sig, rng, dtype, "uniform", ("padded", "negative", "padded"), "uniform")
    q = problem_for(prefix, p)
    got, rep = run_gpu(prefix, q, mode="ex", opts=gett.options(family=family))
    assert rep["family_name"] == family
    compare(prefix, q, got, oracle_ref(q))


@pytest.mark.parametrize("config", range(3))
@pytest.mark.parametrize("split_k", (1, 3, 8))
def test_dense_configs_and_split_k(config, split_k):
    p = synth.cfg_small_dgett()
    got, rep = run_gpu("d", p, mode="ex", opts=gett.options(family="dense", config=config, split_k=split_k))
    assert rep["config"] == config
    compare("d", p, got, oracle_ref(p))


def test_small_workload_default_path():
    """The 32x24x16x20 workload (mode a at stride 2) through plain dgett."""
    p = synth.cfg_small_dgett()
    got, _ = run_gpu("d", p)
    rel = compare("d", p, got, oracle.gett_problem(p, "f64", nthreads=4))
    assert rel < 1e-14


def test_small_workload_against_long_double():
    p = synth.cfg_small_dgett()
    got, _ = run_gpu("d", p)
    compare("d", p, got, oracle.gett_problem(p, "ld", nthreads=4))


@pytest.mark.parametrize("variant", ("plain", "perm", "transA", "perm_transA"))
def test_cc_scaled_down(variant):
    """The coupled-cluster-like contraction at extents 24/8 (all outputs)."""
    p = synth.cfg_cc(variant, scale=24, small_ij=8)
    got, _ = run_gpu("d", p)
    compare("d", p, got, oracle.gett_problem(p, "f64", nthreads=8))


def test_accumulates_and_is_deterministic():
    p = synth.thesis_problem("basic", 31, np.float64, "uniform", c_dist="uniform")
    got1, _ = run_gpu("d", p)
    got2, _ = run_gpu("d", p)
    assert np.array_equal(got1, got2)
    q = p.copy()
    q.C = got1
    got3, _ = run_gpu("d", q)
    ref = oracle.gett_problem(p, C=oracle.gett_problem(p))
    compare("d", p, got3, ref)


@pytest.mark.parametrize("seed", range(4))
def test_commutativity_gpu(seed):
    p = synth.thesis_problem("commutativity", 40 + seed, np.float64, "int", c_dist="int")
    a, _ = run_gpu("d", p)
    b, _ = run_gpu("d", synth.swapped(p))
    assert np.array_equal(a, b)


def test_async_on_torch_stream():
    import torch
    p = synth.cfg_small_dgett()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        got, _ = run_gpu("d", p, mode="async", stream=s.cuda_stream)
    compare("d", p, got, oracle_ref(p))


def test_empty_and_degenerate():
    # all extents 1: a single product
    sig = synth.Signature((1, 1), (1, 1), (1,), (0,), (0, 1))
    p = synth.make_problem(sig, np.random.default_rng(0), np.float64, "int", c_dist="int")
    got, _ = run_gpu("d", p)
    compare("d", p, got, oracle_ref(p), exact=True)
    # rank 0 with rank 0
    sig = synth.Signature((), (), (), (), ())
    p = synth.make_problem(sig, np.random.default_rng(1), np.float64, "int", c_dist="int")
    got, _ = run_gpu("d", p)
    compare("d", p, got, oracle_ref(p), exact=True)
    # zero contracted extent: C unchanged
    sig = synth.Signature((3, 0), (0, 4), (1,), (0,), (0, 1))
    p = synth.make_problem(sig, np.random.default_rng(2), np.float64, "int", c_dist="int")
    got, _ = run_gpu("d", p)
    assert np.array_equal(got, p.C)


STREAM_SHAPES = {
    # short sum (K = 3) over a large output: OUTER with a register-held K
    "short_sum": (synth.Signature((300, 3, 40), (3, 25), (1,), (0,), (0, 2, 1)), ("contig", "padded", "contig")),
    # matrix-vector with the long operand contiguous along the row index
    "gemv_rows": (synth.Signature((3000, 45), (45, 3), (1,), (0,), (0, 1)), ("contig", "negative", "padded")),
    # matrix-vector with the long operand contiguous along k (warp per row)
    "gemv_k": (synth.Signature((3000, 45), (45, 1), (1,), (0,), (0, 1)), ("rowmajor", "contig", "contig")),
    # short class on the A side, two contracted modes
    "left_skinny": (synth.Signature((2, 9, 7), (7, 9, 900), (1, 2), (1, 0), (1, 0)), ("padded", "rowmajor", "negative")),
    # long sums: several staged K chunks per slice, K split into slices, ragged tails, S = 5
    "gemv_rows_long": (synth.Signature((700, 5000), (5000, 5), (1,), (0,), (0, 1)), ("padded", "contig", "negative")),
    "gemv_k_long": (synth.Signature((300, 5000), (5000, 3), (1,), (0,), (1, 0)), ("rowmajor", "negative", "padded")),
}


@pytest.mark.parametrize("prefix", ("d", "s", "z", "c", "sb"))
@pytest.mark.parametrize("name", sorted(STREAM_SHAPES))
def test_streaming_short_sums_and_skinny(prefix, name):
    sig, kinds = STREAM_SHAPES[name]
    rng = np.random.default_rng(sum(map(ord, name)))
    dtype = np.complex128 if prefix in ("z", "c") else np.float64
    p = synth.make_problem(sig, rng, dtype, "uniform", kinds, "uniform")
    q = problem_for(prefix, p)
    family = "outer" if name == "short_sum" else "skinny"
    got, rep = run_gpu(prefix, q, mode="ex", opts=gett.options(family=family))
    assert rep["family_name"] == family
    compare(prefix, q, got, oracle_ref(q))
    got2, rep2 = run_gpu(prefix, q)  # the selector's own choice
    compare(prefix, q, got2, oracle_ref(q))


@pytest.mark.parametrize("prefix", ("d", "z"))
def test_most_modes_per_class(prefix):
    """24 unfusable free modes in A (the per-class limit after fusion), one
    contracted mode; C holds them in reverse order.  Integer data: bit-exact."""
    n = 24
    exta = (2,) * n + (3,)
    perm = tuple(range(n - 1, -1, -1)) + (n,)
    sig = synth.Signature(exta, (3, 2), (n,), (0,), perm)
    dtype = np.complex128 if prefix == "z" else np.float64
    p = synth.make_problem(sig, np.random.default_rng(24), dtype, "int", ("contig", "contig", "contig"), "int")
    got, rep = run_gpu(prefix, p, mode="ex")
    assert rep["nm"] == n
    compare(prefix, p, got, oracle_ref(p), exact=True)


@pytest.mark.parametrize("prefix", ("d", "z"))
def test_bilinearity_gpu(prefix):
    """gett(A1 + A2, B) = gett(A1, B) + gett(A2, B) on integer data, bit for
    bit, at a size that spans many tiles (a property that holds at any size)."""
    dtype = np.complex128 if prefix == "z" else np.float64
    sig = synth.Signature((96, 40, 70), (70, 130, 40), (1, 2), (2, 0), (1, 0, 2))
    p1 = synth.make_problem(sig, np.random.default_rng(61), dtype, "int", ("padded", "negative", "padded"), "zeros")
    p2 = p1.copy()
    rng = np.random.default_rng(62)
    v = rng.integers(-8, 9, p1.la.numel).astype(np.float64)
    if prefix == "z":
        v = v + 1j * rng.integers(-8, 9, p1.la.numel)
    p2.A = synth.fill(p1.la, v, dtype, np.nan)
    ps = p1.copy()
    ps.A = p1.A + p2.A
    lhs, _ = run_gpu(prefix, ps)
    r1, _ = run_gpu(prefix, p1)
    r2, _ = run_gpu(prefix, p2)
    lg = synth.gather(ps.lc, lhs)
    assert np.array_equal(lg, synth.gather(p1.lc, r1) + synth.gather(p2.lc, r2))
