"""Randomised GPU parity: contractions drawn with the thesis's generator
parameters (Sec. 7: ranks up to 5, random contracted pairs and output
permutation) but larger extents, every layout kind (contiguous, row-major,
sub-tensor, negative increments, lower-rank embedding) and every precision
form, against the oracle.  Integer data must match bit for bit; float data
within the per-element rounding bound and the form's normwise tolerance.
Forced kernel families run the same draws, so every family meets the same
signatures."""
import numpy as np
import pytest

from paper_2410_06770_gb300 import gett, synth
from tests._gpu_util import compare, oracle_ref, problem_for, run_gpu

pytestmark = pytest.mark.gpu

N_DRAWS = 40


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2410_06770_gb300 import build
    build.build()
    gett.lib()


def _draw(i, dtype, dist):
    rng = np.random.default_rng(5000 + i)
    sig = synth.random_signature(rng, min_rank=0, max_rank=5, min_ext=1, max_ext=9, max_conts=3,
                                 max_elems=1 << 16)
    kinds = tuple(synth.LAYOUT_KINDS[int(rng.integers(len(synth.LAYOUT_KINDS)))] for _ in range(3))
    return synth.make_problem(sig, rng, dtype, dist, kinds, dist)


@pytest.mark.parametrize("prefix", ("d", "s", "z", "c", "sb"))
@pytest.mark.parametrize("i", range(N_DRAWS))
def test_fuzz_integer_exact(prefix, i):
    dtype = np.complex128 if prefix in ("z", "c") else np.float64
    q = problem_for(prefix, _draw(i, dtype, "int"))
    got, _ = run_gpu(prefix, q)
    compare(prefix, q, got, oracle_ref(q), exact=True)


@pytest.mark.parametrize("prefix", ("d", "z"))
@pytest.mark.parametrize("family", ("dense", "outer", "reduce", "skinny"))
@pytest.mark.parametrize("i", range(0, N_DRAWS, 3))
def test_fuzz_forced_families(prefix, family, i):
    """Each family on the draws it accepts (OUTER needs K <= 8, SKINNY a free
    class of at most 8, REDUCE at most 4096 outputs); float data."""
    dtype = np.complex128 if prefix == "z" else np.float64
    q = _draw(i, dtype, "uniform")
    st, info = gett.plan_describe(len(q.sig.exta), q.sig.exta, q.la.inc, len(q.sig.extb), q.sig.extb, q.lb.inc,
                                  q.sig.conts, q.sig.conta, q.sig.contb, q.sig.perm, q.lc.inc)
    assert st == gett.GETT_OK
    if info["empty"]:
        pytest.skip("empty problem")
    M, N, K = info["M"], info["N"], info["K"]
    if family == "outer" and K > 8:
        pytest.skip("OUTER takes K <= 8")
    if family == "skinny" and (min(M, N) > 8 or K <= 1):
        pytest.skip("SKINNY takes a free class of at most 8 and K > 1")
    if family == "reduce" and M * N > 4096:
        pytest.skip("REDUCE takes at most 4096 outputs")
    got, rep = run_gpu(prefix, q, mode="ex", opts=gett.options(family=family))
    assert rep["family_name"] == family
    compare(prefix, q, got, oracle_ref(q))
