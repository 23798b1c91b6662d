"""GPU parity of the tensor-core (tcgen05) forms against the oracle.

* bf16 inputs, tensor cores (sbgett, family tc): integer data bit-exact,
  float data within the fp32 rounding bound.
* SGETT split forms (BF16X3, BF16X6) against the fp64 oracle of the fp32
  inputs, element by element within the form's derived bound: x = hi + mid
  (+ lo) in bf16 represents x within 2^-16 |x| with two pieces (each rounding
  to 8 significant bits leaves at most 2^-8 of what it rounds) and exactly
  with three; BF16X3 drops mid*mid and the representation errors, at most
  3.02 * 2^-16 |a b| a product, BF16X6 drops the products of piece ranks
  summing to 3 or more, at most 2.02 * 2^-24 |a b|.  The fp32 sums of the
  3K (6K) piece products add 2 (3K + 2) 2^-24 (6K) of sum |a||b|.  BF16X6
  also meets the fp32 tolerance 1e-5 normwise; BF16X3 is held to its derived
  bound, and to 1e-5 on the split-precision workload's own inputs.
* Split-precision DGETT (modular form on bf16 tensor cores): integer data
  bit-exact (every scaled input is exact and the modular product is exact);
  float data within the scheme's element bound (tests._gpu_util.ozaki_bound)
  and normwise within 1e-13 of the long-double oracle, including log-uniform
  magnitudes over 1e-8..1e8 with random signs.
"""
import numpy as np
import pytest

import oracle
from paper_2410_06770_gb300 import gett, synth
from tests._gpu_util import check_elementwise, compare, oracle_ref, ozaki_bound, problem_for, run_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2410_06770_gb300 import build
    build.build()
    gett.lib()


def _normwise(p, got, ref):
    g = synth.gather(p.lc, got).astype(np.float64)
    r = synth.gather(p.lc, ref)
    return float(np.linalg.norm(g - r) / np.linalg.norm(r))


# shapes that span several 128x256 tiles with ragged M, N and K tails
SHAPES = [
    synth.Signature((130, 70), (70, 300), (1,), (0,), (0, 1)),                # GEMM, ragged
    synth.Signature((37, 9, 5), (5, 9, 61), (1, 2), (1, 0), (1, 0, 2)),        # 2 K modes, permuted out
    synth.Signature((257, 3, 33), (33, 129), (2,), (0,), (2, 0, 1)),          # M two modes
    synth.Signature((64, 1100), (1100, 40), (1,), (0,), (1, 0)),              # K over one chunk
]


@pytest.mark.parametrize("idx", range(len(SHAPES)))
@pytest.mark.parametrize("kinds", [("contig",) * 3, ("padded", "negative", "padded"), ("rowmajor", "lower_rank", "contig")])
def test_bf16_tensor_core_integer_exact(idx, kinds):
    rng = np.random.default_rng(10 + idx)
    p = synth.make_problem(SHAPES[idx], rng, np.float64, "smallint", kinds, "int")
    q = problem_for("sb", p)
    got, rep = run_gpu("sb", q, mode="ex", opts=gett.options(family="tc"))
    assert rep["family_name"] == "tc"
    compare("sb", q, got, oracle_ref(q), exact=True)


@pytest.mark.parametrize("idx", range(len(SHAPES)))
def test_bf16_tensor_core_float(idx):
    rng = np.random.default_rng(20 + idx)
    p = synth.make_problem(SHAPES[idx], rng, np.float64, "uniform", ("padded", "contig", "negative"), "uniform")
    q = problem_for("sb", p)
    got, rep = run_gpu("sb", q, mode="ex", opts=gett.options(family="tc"))
    compare("sb", q, got, oracle_ref(q))


# per split form: piece products per contracted index and the relative error
# of one product that the form drops (derived in the module docstring)
SPLIT_FORMS = {"bf16x3": (3, 3.02 * 2.0 ** -16), "bf16x6": (6, 2.02 * 2.0 ** -24)}


def _split_derived_normwise(q, terms, extra):
    """The normwise bound implied by the element bound:
    || (2 (terms K + 2) u + extra) (|C0| + sum |A||B|) || / || C_ref ||."""
    from tests._gpu_util import abs_bound
    K = max(1, int(np.prod([q.sig.exta[m] for m in q.sig.conta], dtype=np.int64)))
    b = (2.0 * (terms * K + 2) * 2.0 ** -24 + extra) * abs_bound(q)
    r = synth.gather(q.lc, oracle_ref(q))
    return float(np.linalg.norm(b) / np.linalg.norm(r))


@pytest.mark.parametrize("algo", sorted(SPLIT_FORMS))
@pytest.mark.parametrize("idx", range(len(SHAPES)))
@pytest.mark.parametrize("dist", ["uniform", "normal"])
def test_sgett_split_forms(algo, idx, dist):
    rng = np.random.default_rng(30 + idx)
    p = synth.make_problem(SHAPES[idx], rng, np.float64, dist, ("padded", "negative", "contig"), "zeros")
    q = problem_for("s", p)
    got, rep = run_gpu("s", q, mode="ex", opts=gett.options(algo=algo))
    assert rep["family_name"] == "tc"
    terms, extra = SPLIT_FORMS[algo]
    tol = 1e-5 if algo == "bf16x6" else _split_derived_normwise(q, terms, extra)
    compare("s", q, got, oracle_ref(q), tol=tol, k_terms=terms, extra_rel=extra)


@pytest.mark.parametrize("algo", sorted(SPLIT_FORMS))
def test_sgett_split_on_small_workload_shapes(algo):
    """The split-precision workload's SGETT part: 32x24x16x20 shapes in fp32,
    log-uniform magnitudes over 1e-8..1e8 with random signs; both forms within
    the fp32 tolerance 1e-5 normwise and their element bounds."""
    p = synth.cfg_small_dgett(dist="logu")
    q = problem_for("s", p)
    got, _ = run_gpu("s", q, mode="ex", opts=gett.options(algo=algo))
    terms, extra = SPLIT_FORMS[algo]
    compare("s", q, got, oracle_ref(q), tol=1e-5, k_terms=terms, extra_rel=extra)


@pytest.mark.parametrize("idx", range(len(SHAPES)))
@pytest.mark.parametrize("kinds", [("contig",) * 3, ("padded", "negative", "padded")])
def test_ozaki_integer_exact(idx, kinds):
    rng = np.random.default_rng(40 + idx)
    p = synth.make_problem(SHAPES[idx], rng, np.float64, "int", kinds, "int")
    got, rep = run_gpu("d", p, mode="ex", opts=gett.options(algo="ozaki_bf16"))
    assert rep["family_name"] == "tc" and rep["moduli"] >= 8
    compare("d", p, got, oracle_ref(p), exact=True)


@pytest.mark.parametrize("dist", ["uniform", "normal", "logu"])
@pytest.mark.parametrize("idx", range(len(SHAPES)))
def test_ozaki_float(dist, idx):
    rng = np.random.default_rng(50 + idx)
    p = synth.make_problem(SHAPES[idx], rng, np.float64, dist, ("padded", "negative", "contig"), "uniform")
    got, rep = run_gpu("d", p, mode="ex", opts=gett.options(algo="ozaki_bf16"))
    ref = oracle.gett_problem(p, "ld", nthreads=4)
    rel = _normwise(p, got, ref)
    assert rel <= 1e-13, rel
    gaps = synth.gap_mask(p.lc)
    assert np.array_equal(got[gaps], p.C[gaps])
    _, bits, _ = gett.ozaki_params(rep["K"], rep["moduli"])
    check_elementwise(synth.gather(p.lc, got), synth.gather(p.lc, ref), ozaki_bound(p, bits), f"{dist} {idx}")


@pytest.mark.parametrize("family", synth.THESIS_TESTS)
def test_ozaki_thesis_families(family):
    p = synth.thesis_problem(family, 60, np.float64, "uniform", c_dist="uniform")
    got, rep = run_gpu("d", p, mode="ex", opts=gett.options(algo="ozaki_bf16"))
    ref = oracle.gett_problem(p, "ld")
    g = synth.gather(p.lc, got)
    r = synth.gather(p.lc, ref)
    nr = np.linalg.norm(r)
    assert np.linalg.norm(g - r) <= 1e-13 * (nr if nr else 1.0)
    if rep["family_name"] == "tc":
        _, bits, _ = gett.ozaki_params(rep["K"], rep["moduli"])
        check_elementwise(g, r, ozaki_bound(p, bits), family)


def test_ozaki_small_workload_logu():
    """The split-precision workload: 32x24x16x20 shapes, log-uniform
    magnitudes over 1e-8..1e8 with random signs, vs the long-double oracle."""
    p = synth.cfg_small_dgett(dist="logu")
    got, rep = run_gpu("d", p, mode="ex", opts=gett.options(algo="ozaki_bf16"))
    ref = oracle.gett_problem(p, "ld", nthreads=4)
    rel = _normwise(p, got, ref)
    assert rel <= 1e-13, rel
    _, bits, _ = gett.ozaki_params(rep["K"], rep["moduli"])
    check_elementwise(synth.gather(p.lc, got), synth.gather(p.lc, ref), ozaki_bound(p, bits), "small logu")
    plain, _ = run_gpu("d", p)
    assert _normwise(p, plain, ref) <= 1e-13


@pytest.mark.parametrize("L", [10, 14, 18])
def test_ozaki_moduli_counts(L):
    p = synth.cfg_small_dgett(dist="normal")
    got, rep = run_gpu("d", p, mode="ex", opts=gett.options(algo="ozaki_bf16", moduli=L))
    assert rep["moduli"] == L
    ref = oracle.gett_problem(p, "ld", nthreads=4)
    rel = _normwise(p, got, ref)
    # fewer moduli leave fewer bits per operand: error ~ 2^-bits, with
    # bits = floor((log2(p_1...p_L) - 1 - log2 K) / 2), capped at 52
    moduli = [255, 253, 251, 247, 241, 239, 233, 229, 227, 223, 217, 211, 199, 197, 193, 191, 181, 179]
    lp = sum(np.log2(moduli[:L]))
    bits = min(52, int(np.floor((lp - 1 - np.log2(480) - 1e-6) / 2)))
    assert rel <= 2.0 ** (-bits + 6), (rel, bits)


@pytest.mark.parametrize("idx", range(len(SHAPES)))
@pytest.mark.parametrize("dist", ["int", "uniform", "logu"])
def test_ozaki_complex(idx, dist):
    """zgett with the split-precision form: the real 2x2 block form of the
    complex contraction on bf16 tensor cores.  Integer data bit-exact, float
    data normwise within 1e-13 of the complex-double oracle."""
    rng = np.random.default_rng(70 + idx)
    p = synth.make_problem(SHAPES[idx], rng, np.complex128, dist, ("padded", "negative", "contig"),
                           "int" if dist == "int" else "uniform")
    got, rep = run_gpu("z", p, mode="ex", opts=gett.options(algo="ozaki_bf16"))
    assert rep["family_name"] == "tc"
    ref = oracle_ref(p)
    if dist == "int":
        compare("z", p, got, ref, exact=True)
    else:
        g = synth.gather(p.lc, got)
        r = synth.gather(p.lc, ref)
        assert np.linalg.norm(g - r) <= 1e-13 * np.linalg.norm(r)
        gaps = synth.gap_mask(p.lc)
        assert np.array_equal(got[gaps], p.C[gaps])
        _, bits, _ = gett.ozaki_params(2 * rep["K"], rep["moduli"])
        # the complex reference is the fp64 oracle: add its own rounding
        check_elementwise(g, r, ozaki_bound(p, bits, ref_terms=4 * rep["K"]), f"complex {dist} {idx}")


@pytest.mark.parametrize("family", ["basic", "subtensor_negative", "rank_zero", "scalar", "nothing"])
def test_ozaki_complex_thesis_families(family):
    p = synth.thesis_problem(family, 61, np.complex128, "uniform", c_dist="uniform")
    got, _ = run_gpu("z", p, mode="ex", opts=gett.options(algo="ozaki_bf16"))
    g = synth.gather(p.lc, got)
    r = synth.gather(p.lc, oracle_ref(p))
    nr = np.linalg.norm(r)
    assert np.linalg.norm(g - r) <= 1e-13 * (nr if nr else 1.0)


def _explicit_problem(sig, inca, incb, seed):
    """Integer-valued problem with explicit A / B increments, C contiguous."""
    la = synth.layout_explicit(sig.exta, inca)
    lb = synth.layout_explicit(sig.extb, incb)
    lc = synth.layout_contiguous(sig.extc())
    return synth.make_problem(sig, np.random.default_rng(seed), np.float64, "int", c_dist="int",
                              layouts=(la, lb, lc))


# (signature, INCA, INCB, expected in-place mask: bit 0 A, bit 1 B)
IN_PLACE = [
    # both K-major with 64-element pitches
    (synth.Signature((64, 130), (64, 300), (0,), (0,), (0, 1)), (1, 64), (1, 64), 3),
    # K = 70 (TMA fills k >= 70 with zeros) at pitches 72 and 80
    (synth.Signature((70, 130), (70, 50), (0,), (0,), (1, 0)), (1, 72), (1, 80), 3),
    # A row-major M x K is K-major too; two free modes of A fuse into one row mode
    (synth.Signature((5, 7, 32), (32, 33), (2,), (0,), (1, 0, 2)), (224, 32, 1), (1, 40), 3),
    # A M-major (packed), B K-major (in place)
    (synth.Signature((130, 64), (64, 300), (1,), (0,), (0, 1)), (1, 130), (1, 64), 2),
    # pitch 70 elements is not a whole number of 16-byte units: both packed
    (synth.Signature((70, 30), (70, 20), (0,), (0,), (0, 1)), (1, 70), (1, 70), 0),
    # two row modes that do not fuse (a gap between them): A packed
    (synth.Signature((16, 5, 7), (16, 40), (0,), (0,), (0, 1, 2)), (1, 16, 96), (1, 16), 2),
]


@pytest.mark.parametrize("idx", range(len(IN_PLACE)))
def test_bf16_in_place_staging(idx):
    """bf16 operands read in place by TMA (no packed copy) where the planned
    layout allows it, packed otherwise; integer data bit-exact either way."""
    sig, inca, incb, mask = IN_PLACE[idx]
    p = _explicit_problem(sig, inca, incb, 90 + idx)
    q = problem_for("sb", p)
    got, rep = run_gpu("sb", q, mode="ex", opts=gett.options(family="tc"))
    assert rep["family_name"] == "tc" and rep["config"] == mask
    compare("sb", q, got, oracle_ref(q), exact=True)
