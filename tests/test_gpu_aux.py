"""GPU parity of the transpose (xGETP) and the reduction (xGETR) through the
C ABI against the oracle's contraction with a unit / ones B (their
definition; Sec. 9 lists both as future work).

A pure transpose (alpha = 1, beta = 0) moves values: bit-exact for every
type.  Scaled forms and reductions: the element bound of the scaled form and
the normwise tolerance of the type; integer data bit-exact."""
import numpy as np
import pytest

from paper_2410_06770_gb300 import gett
from tests._aux_ref import reduction_problem, transpose_problem
from tests._gpu_util import download, problem_for, upload
from tests.test_gpu_scaled import _nan_c, compare_scaled

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2410_06770_gb300 import build
    build.build()
    gett.lib()


def _run_getp(prefix, p, alpha, beta):
    dA, dC = upload(p.A), upload(p.C)
    a = p.args()
    gett.getp(prefix, a["RANKA"], a["EXTA"], a["INCA"], dA, a["PERM"], a["INCC"], dC, alpha=alpha, beta=beta,
              a_off=p.la.off, c_off=p.lc.off)
    return download(dC, p.C.dtype)


def _run_getr(prefix, p, alpha, beta):
    dA, dC = upload(p.A), upload(p.C)
    a = p.args()
    gett.getr(prefix, a["RANKA"], a["EXTA"], a["INCA"], dA, a["CONTS"], a["CONTA"], a["PERM"], a["INCC"], dC,
              alpha=alpha, beta=beta, a_off=p.la.off, c_off=p.lc.off)
    return download(dC, p.C.dtype)


TRANSPOSES = [
    # extents spanning several 32 x 32 tiles with ragged edges
    ((70, 45, 3), (2, 0, 1), ("padded", "negative")),
    ((70, 45, 3), (1, 0, 2), ("contig", "padded")),
    ((33, 2, 65, 5), (3, 2, 1, 0), ("negative", "contig")),
    ((1000, 7), (0, 1), ("padded", "padded")),          # same fastest mode: streaming copy
    ((9, 300), (1, 0), ("rowmajor", "contig")),
    ((4, 5, 6, 7, 2), (4, 0, 3, 1, 2), ("padded", "padded")),
    ((1,), (0,), ("contig", "contig")),
    ((3000, 5, 7), (0, 2, 1), ("contig", "padded")),    # long fastest mode, short next mode: wide blocks
    ((100, 3, 2), (0, 2, 1), ("padded", "negative")),
    ((2000, 40), (0, 1), ("contig", "contig")),         # fuses to one mode
    ((), (), ("contig", "contig")),
]


@pytest.mark.parametrize("prefix", ("d", "s", "z", "c", "sb"))
@pytest.mark.parametrize("case", range(len(TRANSPOSES)))
def test_transpose_bit_exact(prefix, case):
    exta, perm, kinds = TRANSPOSES[case]
    dtype = np.complex128 if prefix in ("z", "c") else np.float64
    p = problem_for(prefix, transpose_problem(exta, perm, np.random.default_rng(case), dtype, kinds=kinds))
    p = _nan_c(p)  # beta = 0: C is never read
    got = _run_getp(prefix, p, 1.0, 0.0)
    compare_scaled(prefix, p, got, 1.0, 0.0, exact=True)


@pytest.mark.parametrize("prefix", ("d", "z", "sb"))
@pytest.mark.parametrize("alpha,beta", [(2.5, -0.75), (1.0, 1.0), (0.0, 2.0), (-1.0, 0.0)])
def test_transpose_scaled(prefix, alpha, beta):
    exta, perm, kinds = TRANSPOSES[0]
    dtype = np.complex128 if prefix == "z" else np.float64
    p = problem_for(prefix, transpose_problem(exta, perm, np.random.default_rng(40), dtype, kinds=kinds))
    if beta == 0:
        p = _nan_c(p)
    got = _run_getp(prefix, p, alpha, beta)
    compare_scaled(prefix, p, got, alpha, beta)


REDUCTIONS = [
    ((37, 3000), (1,), (0,), ("padded", "negative")),            # long sums, 37 rows: SKINNY
    ((3000, 37), (0,), (0,), ("contig", "padded")),              # fast mode reduced
    ((64, 64, 64), (0, 1, 2), (), ("contig", "contig")),         # everything: REDUCE
    ((5, 300, 40), (1,), (1, 0), ("padded", "padded")),          # DENSE with one column
    ((20, 3, 40), (1,), (0, 1), ("rowmajor", "contig")),         # short sum: OUTER
    ((6, 7, 8, 9), (3, 1), (1, 0), ("negative", "padded")),
]


@pytest.mark.parametrize("prefix", ("d", "s", "z", "c", "sb"))
@pytest.mark.parametrize("case", range(len(REDUCTIONS)))
def test_reduction(prefix, case):
    exta, red, perm, kinds = REDUCTIONS[case]
    dtype = np.complex128 if prefix in ("z", "c") else np.float64
    p = problem_for(prefix, reduction_problem(exta, red, perm, np.random.default_rng(100 + case), dtype,
                                              kinds=kinds))
    for alpha, beta in ((1.0, 0.0), (2.5, -0.75)):
        q = _nan_c(p) if beta == 0 else p
        got = _run_getr(prefix, q, alpha, beta)
        compare_scaled(prefix, q, got, alpha, beta)


@pytest.mark.parametrize("prefix", ("d", "s", "z"))
@pytest.mark.parametrize("case", range(len(REDUCTIONS)))
def test_reduction_integer_exact(prefix, case):
    exta, red, perm, kinds = REDUCTIONS[case]
    dtype = np.complex128 if prefix == "z" else np.float64
    p = problem_for(prefix, reduction_problem(exta, red, perm, np.random.default_rng(200 + case), dtype,
                                              dist="int", kinds=kinds, c_dist="int"))
    got = _run_getr(prefix, p, 2.0, -3.0)
    compare_scaled(prefix, p, got, 2.0, -3.0, exact=True)


def test_reduction_of_nothing_is_a_copy():
    """NRED = 0: the transpose path."""
    p = reduction_problem((30, 40), (), (1, 0), np.random.default_rng(7), kinds=("padded", "padded"))
    got = _run_getr("d", p, 1.0, 0.0)
    compare_scaled("d", p, got, 1.0, 0.0, exact=True)
