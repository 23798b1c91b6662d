"""Pins for the transpose and reduction references (the contraction with a
unit / ones B, run by the oracle) against numpy.transpose and numpy.sum on the
logical tensors.  Both operations are listed as future work in Sec. 9."""
import numpy as np
import pytest

import oracle
from paper_2410_06770_gb300 import synth
from tests._aux_ref import reduction_problem, transpose_problem

PERMS = [(0, 1, 2), (2, 1, 0), (1, 0, 2), (0, 2, 1), (2, 0, 1)]


@pytest.mark.parametrize("perm", PERMS)
@pytest.mark.parametrize("kinds", [("contig", "contig"), ("padded", "negative"), ("rowmajor", "padded")])
def test_transpose_is_numpy_transpose(perm, kinds):
    """A's mode p goes to output position PERM[p] (the PERM convention of
    Sec. 5.6): C = transpose(A, argsort(PERM)), bit-exact (products by 1)."""
    rng = np.random.default_rng(sum(perm) * 7 + len(kinds[0]))
    p = transpose_problem((5, 7, 3), perm, rng, kinds=kinds)
    got = synth.logical(p.lc, oracle.gett_scaled(p, 1.0, 0.0))
    ref = np.transpose(synth.logical(p.la, p.A), np.argsort(perm))
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("red,perm", [((0,), (0, 1)), ((1,), (1, 0)), ((2,), (0, 1)), ((0, 2), (0,)),
                                      ((2, 0), (0,)), ((0, 1, 2), ())])
def test_reduction_is_numpy_sum_integer_exact(red, perm):
    """C = sum of A over the RED modes, the remaining modes (ascending) placed
    by PERM; integer data, so exact."""
    rng = np.random.default_rng(11 + len(red))
    p = reduction_problem((6, 5, 4), red, perm, rng, dist="int", kinds=("padded", "negative"), c_dist="int")
    got = synth.logical(p.lc, oracle.gett_scaled(p, 1.0, 0.0))
    s = np.sum(synth.logical(p.la, p.A).astype(np.int64), axis=tuple(red))
    ref = np.transpose(s, np.argsort(perm)) if perm else s
    assert np.array_equal(got, np.asarray(ref, dtype=np.float64))


def test_reduction_float_within_rounding():
    rng = np.random.default_rng(5)
    p = reduction_problem((40, 30, 20), (1,), (1, 0), rng, kinds=("padded", "contig"))
    got = synth.logical(p.lc, oracle.gett_scaled(p, 1.0, 0.0))
    ref = np.transpose(np.sum(synth.logical(p.la, p.A), axis=1), (1, 0))
    assert np.linalg.norm(got - ref) <= 1e-14 * np.linalg.norm(ref)
