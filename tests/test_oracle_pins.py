"""Pins for the CPU oracle against what the thesis and mathematics fix.

Each test names the passage it checks.  None of them compares the oracle with
itself re-typed: the references are numpy BLAS / einsum on logical tensors,
exact rational arithmetic, the coordinate order printed in Sec. 6 and the
layout figures' increments.
"""
import math
import os
import shutil
import subprocess
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_2410_06770_gb300 import synth
from tests._einsum_ref import einsum_logical, einsum_spec

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden_numbers(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append([int(x) for x in line.split()])
    return rows


def run(p, precision="f64", nthreads=1):
    return synth.logical(p.lc, oracle.gett_problem(p, precision, nthreads))


# --------------------------------------------------------------------------
# Alg. 2 and the Sec. 6 figures
# --------------------------------------------------------------------------
def test_inccoords_prints_paper_sequence():
    """Sec. 6: IncCoords visits [0,0,0], [1,0,0], [2,0,0], [0,1,0], [1,1,0],
    [2,1,0], ... for extents (3,3,3)."""
    want = _golden_numbers("inccoords_rank3.txt")
    c = [0, 0, 0]
    seq = [list(c)]
    for _ in range(len(want) - 1):
        c = oracle.inc_coords(c, [3, 3, 3])
        seq.append(list(c))
    assert seq == want


def test_inccoords_full_cycle_and_rank0():
    """Alg. 2 visits every coordinate once and wraps to zero; it returns at
    once for zero indices."""
    ext = [2, 3, 4]
    c = [0, 0, 0]
    seen = {tuple(c)}
    for _ in range(23):
        c = oracle.inc_coords(c, ext)
        seen.add(tuple(c))
    assert len(seen) == 24
    assert oracle.inc_coords(c, ext) == [0, 0, 0]
    assert oracle.inc_coords([], []) == []


@pytest.mark.parametrize("fixture,parent,inc", [
    ("layout_rank3_inc_1_3_9.txt", 27, (1, 3, 9)),
    ("layout_subtensor_inc_1_5_25.txt", 125, (1, 5, 25)),
])
def test_layout_figures(fixture, parent, inc):
    """Sec. 6 figures: a (3,3,3) tensor with increments [1,3,9] and a (3,3,3)
    sub-tensor with increments [1,5,25].  Contracting with the rank-0 tensor 1
    (CONTS=0) copies A into a contiguous C, so C lists A's memory index of each
    coordinate in IncCoords order."""
    want = np.array(_golden_numbers(fixture)[0], dtype=np.float64)
    A = np.arange(parent, dtype=np.float64)
    B = np.ones(1)
    C = np.zeros(27)
    rc = oracle.gett_raw("f64", 3, (3, 3, 3), inc, A, 0, 0, (), (), B, 0, 0, (), (), (0, 1, 2),
                         (1, 3, 9), C, 0)
    assert rc == 0
    np.testing.assert_array_equal(C, want)


# --------------------------------------------------------------------------
# BLAS reductions (Sec. 2.3 background): GEMM, GEMV, DOT, GER
# --------------------------------------------------------------------------
@pytest.mark.parametrize("conta", [0, 1])
@pytest.mark.parametrize("contb", [0, 1])
@pytest.mark.parametrize("perm", [(0, 1), (1, 0)])
@pytest.mark.parametrize("kind", ["contig", "padded", "negative"])
def test_gemm_reduction(conta, contb, perm, kind):
    """Rank-2 x rank-2 with one contraction is GEMM with A/B transposed by the
    choice of contracted mode; PERM (1,0) gives C transposed.  numpy's BLAS
    matmul sums in another order, so agreement is to rounding (1e-14)."""
    m, k, n = 37, 41, 29
    rng = np.random.default_rng(100 + 8 * conta + 4 * contb + 2 * perm[0])
    exta = (k, m) if conta == 0 else (m, k)
    extb = (k, n) if contb == 0 else (n, k)
    sig = synth.Signature(exta, extb, (conta,), (contb,), perm)
    p = synth.make_problem(sig, rng, np.float64, "uniform", (kind, kind, kind), "uniform")
    Am = synth.logical(p.la, p.A)
    Bm = synth.logical(p.lb, p.B)
    Am = Am.T if conta == 0 else Am
    Bm = Bm if contb == 0 else Bm.T
    ref = Am @ Bm
    if perm == (1, 0):
        ref = ref.T
    ref = ref + synth.logical(p.lc, p.C)
    got = run(p)
    assert np.linalg.norm(got - ref) <= 1e-14 * np.linalg.norm(ref)


@pytest.mark.parametrize("conta", [0, 1])
def test_gemv_reduction(conta):
    m, k = 53, 47
    rng = np.random.default_rng(7 + conta)
    exta = (k, m) if conta == 0 else (m, k)
    sig = synth.Signature(exta, (k,), (conta,), (0,), (0,))
    p = synth.make_problem(sig, rng, np.float64, "uniform", ("padded", "negative", "padded"), "zeros")
    Am = synth.logical(p.la, p.A)
    Am = Am.T if conta == 0 else Am
    ref = Am @ synth.logical(p.lb, p.B)
    got = run(p)
    assert np.linalg.norm(got - ref) <= 1e-14 * np.linalg.norm(ref)


def test_dot_reduction_within_error_bound():
    """Rank-1 x rank-1 fully contracted is DOT; the sequential sum of Alg. 1
    lies within the textbook bound n*u*sum|x_i y_i| of the exact value."""
    rng = np.random.default_rng(3)
    n = 1000
    sig = synth.Signature((n,), (n,), (0,), (0,), ())
    p = synth.make_problem(sig, rng, np.float64, "uniform", ("padded", "negative", "contig"), "zeros")
    x = synth.logical(p.la, p.A)
    y = synth.logical(p.lb, p.B)
    exact = sum(Fraction(float(a)) * Fraction(float(b)) for a, b in zip(x, y))
    got = float(run(p))
    bound = n * 2.0 ** -53 * float(np.sum(np.abs(x * y)))
    assert abs(Fraction(got) - exact) <= Fraction(bound)


@pytest.mark.parametrize("perm", [(0, 1), (1, 0)])
def test_ger_is_bit_exact(perm):
    """CONTS=0 on two vectors is GER: each element is one rounded product added
    to zero, so the result equals numpy.outer bit for bit."""
    rng = np.random.default_rng(11)
    sig = synth.Signature((17,), (13,), (), (), perm)
    p = synth.make_problem(sig, rng, np.float64, "normal", ("negative", "padded", "padded"), "zeros")
    ref = np.outer(synth.logical(p.la, p.A), synth.logical(p.lb, p.B))
    if perm == (1, 0):
        ref = ref.T
    got = run(p)
    assert np.array_equal(got, ref)


# --------------------------------------------------------------------------
# Integer-exact comparison with einsum over all thesis test families (Sec. 7)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("family", synth.THESIS_TESTS)
@pytest.mark.parametrize("seed", range(6))
def test_integer_exact_vs_einsum(family, seed):
    """Integer values in [-8, 8] with nonzero initial C: every partial sum is an
    exact double, so the oracle must equal int64 einsum + C0 exactly.  This pins
    the free-index order, the PERM direction, increments, sub-tensors, negative
    increments and the accumulate-into-C semantics of Alg. 1."""
    p = synth.thesis_problem(family, 1000 + seed, np.float64, "int", c_dist="int")
    ref = einsum_logical(p, np.int64)
    got = run(p)
    assert np.array_equal(got, ref.astype(np.float64)), einsum_spec(p.sig)
    out = oracle.gett_problem(p)
    gaps = synth.gap_mask(p.lc)
    assert np.array_equal(out[gaps], p.C[gaps])


@pytest.mark.parametrize("seed", range(8))
def test_complex_integer_exact_vs_einsum(seed):
    """Complex double, no conjugation (Sec. 5 prefix z)."""
    p = synth.thesis_problem("basic", 2000 + seed, np.complex128, "int", c_dist="int")
    ref = einsum_logical(p, np.complex128)
    got = synth.logical(p.lc, oracle.gett_problem(p, "z"))
    assert np.array_equal(got, ref)


def test_complex_no_conjugation():
    """(1+2i)*(3+4i) = -5+10i; a conjugating implementation gives 11-2i or 11+2i."""
    A = np.array([1 + 2j])
    B = np.array([3 + 4j])
    C = np.zeros(1, dtype=np.complex128)
    assert oracle.gett_raw("z", 1, (1,), (1,), A, 0, 1, (1,), (1,), B, 0, 1, (0,), (0,), (), (), C, 0) == 0
    assert C[0] == -5 + 10j


# --------------------------------------------------------------------------
# Bit-identity invariants of the oracle (Sec. 7 permutation / commutativity /
# sub-tensor tests): the contracted summation order does not depend on PERM,
# operand order or layout.
# --------------------------------------------------------------------------
@pytest.mark.parametrize("seed", range(10))
def test_permutation_rotations_bit_identical(seed):
    rng = np.random.default_rng(seed)
    p = synth.thesis_problem("permutations", 3000 + seed, np.float64, "uniform")
    base = run(p)
    r = p.sig.rank_c
    spec_letters = list(range(r))
    for n in range(1, r):
        q = synth.rotated_output(p, n, rng)
        got = run(q)
        # free index p moved from output position perm[p] to (perm[p]-n) mod r
        axes = [(i + n) % r for i in spec_letters]
        assert np.array_equal(got, np.transpose(base, axes)), (n, p.sig)


@pytest.mark.parametrize("seed", range(10))
def test_commutativity_bit_identical(seed):
    p = synth.thesis_problem("commutativity", 4000 + seed, np.float64, "uniform", c_dist="uniform")
    assert np.array_equal(run(p), run(synth.swapped(p)))


@pytest.mark.parametrize("seed", range(6))
def test_stride_invariance_bit_identical(seed):
    """The same logical tensors stored contiguous, row-major, padded, negative,
    padded-negative and inside a higher-rank parent give identical C bits; the
    NaN-filled input gaps are never read and C's gaps keep their sentinel."""
    rng = np.random.default_rng(5000 + seed)
    sig = synth.random_signature(rng, 1, 5, 1, 5)
    A_log = synth.draw_values(rng, int(np.prod(sig.exta, dtype=np.int64)), "uniform", np.float64)
    B_log = synth.draw_values(rng, int(np.prod(sig.extb, dtype=np.int64)), "uniform", np.float64)
    C_log = synth.draw_values(rng, int(np.prod(sig.extc(), dtype=np.int64)), "uniform", np.float64)
    results = []
    for kind in synth.LAYOUT_KINDS:
        la = synth.make_layout(sig.exta, kind, rng)
        lb = synth.make_layout(sig.extb, kind, rng)
        lc = synth.make_layout(sig.extc(), kind, rng)
        p = synth.Problem(sig, la, lb, lc, synth.fill(la, A_log, np.float64, np.nan),
                          synth.fill(lb, B_log, np.float64, np.nan),
                          synth.fill(lc, C_log, np.float64, synth.C_GAP_SENTINEL))
        out = oracle.gett_problem(p)
        gaps = synth.gap_mask(lc)
        assert np.all(out[gaps] == synth.C_GAP_SENTINEL)
        results.append(synth.gather(lc, out))
    for r in results[1:]:
        assert np.array_equal(r, results[0])


# --------------------------------------------------------------------------
# Brute force on tiny inputs and exact arithmetic
# --------------------------------------------------------------------------
@pytest.mark.parametrize("seed", range(40))
def test_direct_oracle_bit_identical(seed):
    p = synth.thesis_problem(synth.THESIS_TESTS[seed % len(synth.THESIS_TESTS)], 6000 + seed,
                             np.float64, "uniform", c_dist="uniform")
    a = oracle.gett_problem(p, "f64")
    b = oracle.gett_problem(p, "direct")
    assert np.array_equal(a, b)


@pytest.mark.parametrize("seed", range(12))
def test_against_exact_rationals(seed):
    """Tiny random contractions evaluated in exact rational arithmetic: the
    fp64 oracle lies within the sequential-sum error bound (n+1)*u*sum|terms|
    per element; the long-double oracle is at most one fp64 rounding away
    from the exact value when long double carries >= 64 significand bits and
    n is small."""
    rng = np.random.default_rng(7000 + seed)
    sig = synth.random_signature(rng, 1, 4, 1, 4)
    p = synth.make_problem(sig, rng, np.float64, "uniform", ("padded", "negative", "contig"), "uniform")
    A = synth.logical(p.la, p.A)
    B = synth.logical(p.lb, p.B)
    C0 = synth.logical(p.lc, p.C)
    got = run(p)
    got_ld = run(p, "ld")
    # exact via einsum over object arrays of Fractions
    fa = np.vectorize(lambda v: Fraction(float(v)), otypes=[object])(A)
    fb = np.vectorize(lambda v: Fraction(float(v)), otypes=[object])(B)
    terms_abs = np.einsum(einsum_spec(sig), np.abs(A), np.abs(B))
    exact = np.einsum(einsum_spec(sig), fa, fb) + np.vectorize(lambda v: Fraction(float(v)), otypes=[object])(C0)
    n = int(np.prod([sig.exta[m] for m in sig.conta], dtype=np.int64))
    exact = np.asarray(exact, dtype=object)
    terms_abs = np.asarray(terms_abs)
    C0 = np.asarray(C0)
    got = np.asarray(got)
    got_ld = np.asarray(got_ld)
    for idx in np.ndindex(*sig.extc()):
        e = exact[idx]
        bound = (n + 1) * 2.0 ** -53 * (float(terms_abs[idx]) + abs(float(C0[idx])))
        assert abs(Fraction(float(got[idx])) - e) <= Fraction(bound)
        if oracle.long_double_bits() >= 64 and n <= 16:
            ulp = math.ulp(float(e)) if e != 0 else 0.0
            assert abs(Fraction(float(got_ld[idx])) - e) <= Fraction(ulp)


def test_summation_order_first_contracted_index_fastest():
    """Alg. 1 adds products in IncCoords order (first contracted index fastest,
    Alg. 2).  With A = [1e16, 1, -1e16, 1] over contracted extents (2, 2)
    (element (i, j) at position i + 2j) and B = 1, adding in that order from
    C = 0 gives ((1e16 + 1) - 1e16) + 1 = 1 in doubles, while the transposed
    order (second index fastest) gives ((1e16 - 1e16) + 1) + 1 = 2."""
    A = np.array([1e16, 1.0, -1e16, 1.0])
    B = np.ones(4)
    C = np.zeros(1)
    rc = oracle.gett_raw("f64", 2, (2, 2), (1, 2), A, 0, 2, (2, 2), (1, 2), B, 0,
                         2, (0, 1), (0, 1), (), (), C, 0)
    assert rc == 0
    assert C[0] == 1.0


# --------------------------------------------------------------------------
# Special cases
# --------------------------------------------------------------------------
def test_rank_zero_operand_scales_elementwise():
    """Sec. 7 "rank zero tensor": C = C0 + s*B, one rounding per element."""
    rng = np.random.default_rng(9)
    sig = synth.Signature((), (3, 4, 2), (), (), (2, 0, 1))
    p = synth.make_problem(sig, rng, np.float64, "uniform", ("contig", "padded", "padded"), "uniform")
    s = float(p.A[p.la.off])
    B = synth.logical(p.lb, p.B)
    ref = synth.logical(p.lc, p.C) + np.transpose(s * B, (1, 2, 0))
    assert np.array_equal(run(p), ref)


def test_scalar_output_vs_fsum():
    """Sec. 7 "scalar contraction": every mode contracted gives a rank-0 C."""
    rng = np.random.default_rng(10)
    sig = synth.Signature((3, 4, 5), (5, 3, 4), (0, 1, 2), (1, 2, 0), ())
    p = synth.make_problem(sig, rng, np.float64, "uniform")
    A = synth.logical(p.la, p.A)
    B = synth.logical(p.lb, p.B)
    ref = math.fsum((A * np.transpose(B, (1, 2, 0))).ravel())
    got = float(run(p))
    assert abs(got - ref) <= 60 * 2.0 ** -53 * float(np.sum(np.abs(A * np.transpose(B, (1, 2, 0)))))


def test_zero_extents_leave_c_unchanged():
    """A zero free extent writes nothing; a zero contracted extent adds an
    empty sum, so C keeps its value."""
    A = np.ones(1)
    B = np.ones(1)
    C = np.full(4, 7.0)
    assert oracle.gett_raw("f64", 2, (0, 2), (1, 1), A, 0, 1, (2,), (1,), B, 0, 1, (1,), (0,),
                           (0,), (1,), C, 0) == 0
    assert oracle.gett_raw("f64", 2, (4, 0), (1, 4), A, 0, 1, (0,), (1,), B, 0, 1, (1,), (0,),
                           (0,), (1,), C, 0) == 0
    assert np.all(C == 7.0)


def test_accumulates_into_c():
    """Alg. 1 adds to C: calling twice on a zero C gives twice the result."""
    p = synth.thesis_problem("basic", 77, np.float64, "int")
    once = oracle.gett_problem(p)
    twice = oracle.gett_problem(p, C=once.copy())
    assert np.array_equal(synth.gather(p.lc, twice), 2 * synth.gather(p.lc, once))


def test_parallel_oracle_matches_serial():
    p = synth.cfg_small_dgett()
    a = oracle.gett_problem(p, "f64", nthreads=1)
    b = oracle.gett_problem(p, "f64", nthreads=4)
    assert np.array_equal(a, b)


def test_small_workload_matches_einsum():
    p = synth.cfg_small_dgett()
    got = run(p, nthreads=4)
    ref = einsum_logical(p)
    assert np.linalg.norm(got - ref) <= 1e-14 * np.linalg.norm(ref)
    assert np.all(np.isnan(p.A[1::2]))  # mode a at stride 2: odd slots are gaps


# --------------------------------------------------------------------------
# Planted mistakes: each plausible bug in the oracle must fail a pin above.
# --------------------------------------------------------------------------
MUTANTS = {
    # PERM read as "free index at output position q" (the inverse reading)
    "perm_inverse": ("int q = PERM[fp];", "int q = fp; (void)PERM;"),
    # contracted B increments taken from A
    "inc_cont_b_from_a": ("p->inc_cont_b[t] = INCB[mb];", "p->inc_cont_b[t] = INCA[ma];"),
    # C overwritten instead of accumulated
    "overwrite_c": ("#define LOAD_SAME(x) (x)", "#define LOAD_SAME(x) (0.0 * (x))"),
    # B's free modes listed before A's
    "free_b_first": ("for (int tensor = 0; tensor < 2; ++tensor) {\n        int rank = tensor == 0 ? RANKA : RANKB;",
                     "for (int tensor = 0; tensor < 2; ++tensor) {\n        tensor = 1 - tensor; int rank = tensor == 0 ? RANKA : RANKB;"),
}


@pytest.mark.parametrize("mutant", sorted(MUTANTS))
def test_planted_mistakes_are_caught(mutant, tmp_path):
    if shutil.which("gcc") is None:
        pytest.skip("gcc missing")
    src = open(os.path.join(os.path.dirname(oracle.__file__), "gett_oracle.c")).read()
    old, new = MUTANTS[mutant]
    assert old in src
    mutated = src.replace(old, new, 1)
    if mutant == "free_b_first":
        # loop over tensor 1 then 0 (B's free modes first)
        mutated = src.replace("for (int tensor = 0; tensor < 2; ++tensor) {\n        int rank",
                              "for (int tt = 0; tt < 2; ++tt) { int tensor = 1 - tt;\n        int rank", 1)
    c_path = tmp_path / "m.c"
    so_path = tmp_path / "m.so"
    c_path.write_text(mutated)
    subprocess.check_call(["gcc", "-O1", "-std=c11", "-ffp-contract=off", "-fopenmp", "-fPIC",
                           "-shared", "-o", str(so_path), str(c_path)])
    import ctypes
    lib = ctypes.CDLL(str(so_path))
    fn = lib.oracle_dgett
    caught = False
    for fam in ("basic", "permutations", "subtensor_same_rank", "rank_one"):
        for seed in range(4):
            p = synth.thesis_problem(fam, 8000 + seed, np.float64, "int", c_dist="int")
            if p.sig.rank_c < 2 and mutant in ("perm_inverse", "free_b_first"):
                continue
            ref = einsum_logical(p, np.int64).astype(np.float64)
            # a mutant may address C outside its layout: give it a large guard band
            guard = 32 * p.C.size + 4096
            C_big = np.zeros(p.C.size + 2 * guard)
            C_big[guard:guard + p.C.size] = oracle.widen(p.C)
            a = p.args()
            i64 = lambda xs: (ctypes.c_int64 * max(len(xs), 1))(*xs)
            i32 = lambda xs: (ctypes.c_int * max(len(xs), 1))(*xs)
            A = oracle.widen(p.A)
            B = oracle.widen(p.B)
            rc = fn(ctypes.c_int(a["RANKA"]), i64(a["EXTA"]), i64(a["INCA"]),
                    ctypes.c_void_p(A.ctypes.data + 8 * p.la.off),
                    ctypes.c_int(a["RANKB"]), i64(a["EXTB"]), i64(a["INCB"]),
                    ctypes.c_void_p(B.ctypes.data + 8 * p.lb.off),
                    ctypes.c_int(a["CONTS"]), i32(a["CONTA"]), i32(a["CONTB"]), i32(a["PERM"]),
                    i64(a["INCC"]), ctypes.c_void_p(C_big.ctypes.data + 8 * (guard + p.lc.off)),
                    ctypes.c_int(1))
            C = C_big[guard:guard + p.C.size]
            if rc != 0 or not np.array_equal(synth.logical(p.lc, C), ref):
                caught = True
                break
        if caught:
            break
    assert caught, f"mutant {mutant} survived the integer-exact einsum pin"


@pytest.mark.parametrize("seed", range(4))
def test_bilinearity(seed):
    """The contraction is linear in A (and in B): gett(A1 + A2, B) = gett(A1, B)
    + gett(A2, B), exactly on integer data (every partial sum is an exact
    double), within rounding on uniform data."""
    for dist in ("int", "uniform"):
        p1 = synth.thesis_problem("basic", 4000 + seed, np.float64, dist)
        p2 = p1.copy()
        rng = np.random.default_rng(4100 + seed)
        vals = rng.integers(-8, 9, p1.A.shape).astype(np.float64) if dist == "int" else rng.uniform(-1, 1, p1.A.shape)
        p2.A = np.where(np.isnan(p1.A), np.nan, vals)
        ps = p1.copy()
        ps.A = p1.A + p2.A
        lhs = synth.logical(ps.lc, oracle.gett_problem(ps))
        rhs = synth.logical(p1.lc, oracle.gett_problem(p1)) + synth.logical(p2.lc, oracle.gett_problem(p2))
        if dist == "int":
            assert np.array_equal(lhs, rhs)
        else:
            assert np.linalg.norm(lhs - rhs) <= 1e-14 * np.linalg.norm(lhs)
