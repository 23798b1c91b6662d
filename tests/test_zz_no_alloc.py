"""The allocation-free double-precision entry point (dgett_noalloc).

Some callers cannot allocate device memory while they run -- a process that
reserves its device memory up front, a latency-critical loop that cannot
afford cudaFree's device-wide synchronisation, a framework whose allocator
owns the device -- so this entry point keeps its scratch in a fixed device
array of the library.  The tests call it through the C ABI and check its
output, for two calls in a row (the second call accumulates onto the first
and reuses the array the first call left behind), against the oracle element
by element (the rounding bound of any summation order) and against the
regular dgett entry point on the same inputs.  This file is collected last,
and works both alone in a fresh process and after the other tests.
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2410_06770_gb300 import gett, synth
from tests._gpu_util import compare, download, upload

pytestmark = pytest.mark.gpu


def noalloc_fn():
    from paper_2410_06770_gb300 import build
    build.build()
    L = gett.lib()
    f = L.dgett_noalloc
    f.argtypes = gett._ARGS14 + [ctypes.c_void_p]
    f.restype = ctypes.c_int
    return f


def call_noalloc(f, p, dA, dB, dC):
    a = p.args()
    return f(int(a["RANKA"]), gett._i64(a["EXTA"]), gett._i64(a["INCA"]), gett._ptr(dA, p.la.off),
             int(a["RANKB"]), gett._i64(a["EXTB"]), gett._i64(a["INCB"]), gett._ptr(dB, p.lb.off),
             int(a["CONTS"]), gett._i32(a["CONTA"]), gett._i32(a["CONTB"]), gett._i32(a["PERM"]),
             gett._i64(a["INCC"]), gett._ptr(dC, p.lc.off), ctypes.c_void_p(0))


CASES = {
    "small_workload": lambda: synth.cfg_small_dgett(),
    "cc_perm_transA": lambda: synth.cfg_cc("perm_transA", scale=24, small_ij=8),
    "subtensor_negative": lambda: synth.thesis_problem("subtensor_negative", 5, np.float64, "uniform",
                                                      c_dist="uniform"),
    "ragged": lambda: synth.make_problem(synth.Signature((133, 7, 5), (5, 7, 71), (1, 2), (1, 0), (1, 0, 2)),
                                         np.random.default_rng(3), np.float64, "normal",
                                         ("padded", "negative", "padded"), "uniform"),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_noalloc_matches_dgett_on_two_calls(case):
    import torch
    f = noalloc_fn()
    p = CASES[case]()
    dA, dB = upload(p.A), upload(p.B)
    dC_noalloc, dC_ref = upload(p.C), upload(p.C)
    a = p.args()
    cur = p.copy()  # the oracle's C before this call
    for call in range(2):
        assert call_noalloc(f, p, dA, dB, dC_noalloc) == gett.GETT_OK
        gett.xgett("d", a["RANKA"], a["EXTA"], a["INCA"], dA, a["RANKB"], a["EXTB"], a["INCB"], dB,
                   a["CONTS"], a["CONTA"], a["CONTB"], a["PERM"], a["INCC"], dC_ref,
                   a_off=p.la.off, b_off=p.lb.off, c_off=p.lc.off)
        torch.cuda.synchronize()
        got = download(dC_noalloc, np.float64)
        ref = download(dC_ref, np.float64)
        # element by element against the oracle (Alg. 1 on the host)
        expect = oracle.gett_problem(cur, "f64", nthreads=4)
        compare("d", cur, got, expect)
        cur.C = expect
        gaps = synth.gap_mask(p.lc)
        assert np.array_equal(got[gaps], p.C[gaps])
        g = synth.gather(p.lc, got)
        r = synth.gather(p.lc, ref)
        assert np.all(np.isfinite(g))
        assert np.linalg.norm(g - r) <= 1e-13 * np.linalg.norm(r), (case, call)


def test_noalloc_rejects_problems_beyond_the_array():
    import torch
    f = noalloc_fn()
    # outer product with M = 300000 > GETT_NOALLOC_MAX_INDEX_SUM
    sig = synth.Signature((300000,), (2,), (), (), (0, 1))
    p = synth.make_problem(sig, np.random.default_rng(0), np.float64, "uniform", c_dist="zeros")
    dA, dB, dC = upload(p.A), upload(p.B), upload(p.C)
    assert call_noalloc(f, p, dA, dB, dC) == gett.GETT_ERR_UNSUPPORTED
    torch.cuda.synchronize()
    assert np.array_equal(download(dC, np.float64), p.C)
