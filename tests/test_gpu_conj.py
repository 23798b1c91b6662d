"""The conjugation option of the complex forms (gett_options.conj) and the
report's device time.

conj(A) and conj(B) are what an xGEMM-style interface offers next to its
ALPHA and BETA (Sec. 2.3.1); Alg. 1 itself never conjugates.  The oracle is
Alg. 1 run on conjugated copies of the host inputs, so the test pins the
option's meaning independently of how the library realises it (a conjugated
copy of the operand in workspace, which every kernel family then reads).
"""
import numpy as np
import pytest

from paper_2410_06770_gb300 import gett, synth
from tests._gpu_util import check_elementwise, compare, oracle_ref, ozaki_bound, run_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2410_06770_gb300 import build
    build.build()
    gett.lib()


def conj_problem(p: synth.Problem, mask: int) -> synth.Problem:
    q = p.copy()
    if mask & gett.GETT_CONJ_A:
        q.A = np.conj(q.A)
    if mask & gett.GETT_CONJ_B:
        q.B = np.conj(q.B)
    return q


# (signature, forced family or None): the selector's choice plus every
# CUDA-core family the shape allows
CASES = [
    (synth.Signature((37, 9, 5), (5, 9, 61), (1, 2), (1, 0), (1, 0, 2)), None),        # dense
    (synth.Signature((40, 3), (3, 50), (1,), (0,), (1, 0)), "outer"),                    # short sum
    (synth.Signature((300, 4), (300,), (0,), (0,), (0,)), "skinny"),                     # gemv-like
    (synth.Signature((64, 33), (64, 33), (0, 1), (0, 1), ()), "reduce"),                 # full inner product
]


@pytest.mark.parametrize("mask", [1, 2, 3])
@pytest.mark.parametrize("case", range(len(CASES)))
@pytest.mark.parametrize("prefix", ["c", "z"])
def test_conjugated_operands(prefix, case, mask):
    sig, family = CASES[case]
    rng = np.random.default_rng(300 + 7 * case + mask)
    p = synth.make_problem(sig, rng, np.complex128, "uniform", ("padded", "negative", "rowmajor"), "uniform")
    if prefix == "c":
        p.A, p.B, p.C = p.A.astype(np.complex64), p.B.astype(np.complex64), p.C.astype(np.complex64)
    opts = gett.options(family=family or "auto", conj=mask)
    got, rep = run_gpu(prefix, p, mode="ex", opts=opts)
    if family:
        assert rep["family_name"] == family
    compare(prefix, p, got, oracle_ref(conj_problem(p, mask)))


@pytest.mark.parametrize("mask", [1, 2, 3])
def test_conjugated_split_zgett(mask):
    """The split-precision ZGETT reads the conjugated copy like any family."""
    sig = synth.Signature((37, 9, 5), (5, 9, 61), (1, 2), (1, 0), (1, 0, 2))
    p = synth.make_problem(sig, np.random.default_rng(40 + mask), np.complex128, "normal",
                           ("padded", "negative", "contig"), "uniform")
    got, rep = run_gpu("z", p, mode="ex", opts=gett.options(algo="ozaki_bf16", conj=mask))
    assert rep["family_name"] == "tc"
    q = conj_problem(p, mask)
    g, r = synth.gather(p.lc, got), synth.gather(p.lc, oracle_ref(q))
    assert np.linalg.norm(g - r) <= 1e-13 * np.linalg.norm(r)
    _, bits, _ = gett.ozaki_params(2 * rep["K"], rep["moduli"])
    check_elementwise(g, r, ozaki_bound(q, bits, ref_terms=4 * rep["K"]), f"conj {mask}")


def test_conjugation_is_identity_for_real_types():
    sig = synth.Signature((37, 9, 5), (5, 9, 61), (1, 2), (1, 0), (1, 0, 2))
    p = synth.make_problem(sig, np.random.default_rng(9), np.float64, "int", ("contig",) * 3, "int")
    got, _ = run_gpu("d", p, mode="ex", opts=gett.options(conj=3))
    compare("d", p, got, oracle_ref(p), exact=True)


def test_report_time():
    """gett_report.time_ms: the device time of the call's work, positive for a
    call that launched kernels and zero for an empty one."""
    p = synth.cfg_small_dgett()
    _, rep = run_gpu("d", p, mode="ex")
    assert 0.0 < rep["time_ms"] < 1000.0
    e = synth.make_problem(synth.Signature((4, 0), (0, 5), (1,), (0,), (0, 1)), np.random.default_rng(0),
                           np.float64, "uniform", c_dist="uniform")
    _, rep0 = run_gpu("d", e, mode="ex")
    assert rep0["time_ms"] == 0.0
