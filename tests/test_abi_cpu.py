"""CPU-only checks of the C-ABI library: it loads, exports every symbol the
public header declares, validates arguments (Sec. 5.7 rules) and plans
correctly.  No device work is started: every call here fails validation or is
the host-only planner."""
import os
import re

import numpy as np
import pytest

import oracle
from paper_2410_06770_gb300 import gett, synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_2410_06770_gb300 import build
    build.build()
    return gett.lib()


def declared_functions():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if not h.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", h)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b([a-z_][a-z0-9_]*)\s*\(", src, re.M):
            name = m.group(1)
            if name not in ("if", "while", "for", "sizeof", "return"):
                names.add(name)
    return sorted(names)


def test_exports_every_declared_symbol(L):
    names = declared_functions()
    assert "dgett" in names and "zgett_async" in names and "gett_plan_describe" in names
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing


def _args(**kw):
    base = dict(RANKA=2, EXTA=(3, 4), INCA=(1, 3), RANKB=2, EXTB=(4, 5), INCB=(1, 4), CONTS=1,
                CONTA=(1,), CONTB=(0,), PERM=(0, 1), INCC=(1, 3))
    base.update(kw)
    return base


def _call(L, **kw):
    a = _args(**kw)
    st, _ = gett.xgett("d", a["RANKA"], a["EXTA"], a["INCA"], 0, a["RANKB"], a["EXTB"], a["INCB"], 0,
                       a["CONTS"], a["CONTA"], a["CONTB"], a["PERM"], a["INCC"], 0,
                       raise_on_error=False)
    return st, gett.last_error_arg()


@pytest.mark.parametrize("kw,pos", [
    (dict(RANKA=-1), 1),
    (dict(EXTA=None), 2),
    (dict(EXTA=(3, -4)), 2),
    (dict(INCA=None), 3),
    (dict(RANKB=-2), 5),
    (dict(EXTB=None), 6),
    (dict(INCB=None), 7),
    (dict(CONTS=3), 9),
    (dict(CONTA=(2,)), 10),
    (dict(CONTB=(2,)), 11),
    (dict(CONTB=(1,), PERM=(0, 1)), 11),  # extents 4 vs 5 do not match
    (dict(PERM=(0, 0)), 12),
    (dict(PERM=(0, 2)), 12),
    (dict(PERM=None), 12),
    (dict(INCC=None), 13),
    (dict(CONTS=2, CONTA=(1, 1), CONTB=(0, 1)), 10),
    (dict(CONTS=2, CONTA=(0, 1), CONTB=(0, 0)), 11),
])
def test_invalid_arguments(L, kw, pos):
    st, arg = _call(L, **kw)
    assert st == gett.GETT_ERR_ARG
    assert arg == pos


def test_null_pointers_reported(L):
    st, arg = _call(L)
    assert st == gett.GETT_ERR_ARG and arg == 4


def test_non_injective_c_is_alias(L):
    # two free modes of extent 3 and 4 mapped onto overlapping increments
    st, _ = _call(L, INCC=(1, 2))
    assert st == gett.GETT_ERR_ALIAS
    st, _ = _call(L, INCC=(0, 3))
    assert st == gett.GETT_ERR_ALIAS


def test_empty_problem_is_noop(L):
    # zero free extent: nothing to do, no pointer needed
    st, _ = _call(L, EXTA=(0, 4))
    assert st == gett.GETT_OK
    # zero contracted extent: empty sum, C unchanged
    st, _ = _call(L, EXTA=(3, 0), EXTB=(0, 5), INCC=(1, 3))
    assert st == gett.GETT_OK


def test_status_strings(L):
    for s in (0, -1, -2, -3, -4, -5, -6):
        assert L.gett_status_string(s)


def test_plan_small_config(L):
    p = synth.cfg_small_dgett()
    a = p.args()
    st, info = gett.plan_describe(a["RANKA"], a["EXTA"], a["INCA"], a["RANKB"], a["EXTB"], a["INCB"],
                                  a["CONTS"], a["CONTA"], a["CONTB"], a["PERM"], a["INCC"])
    assert st == 0
    assert (info["M"], info["N"], info["K"]) == (512, 336, 480)
    assert (info["nm"], info["nn"], info["nk"]) == (2, 2, 2)


def test_plan_fuses_colmajor_cc_to_gemm(L):
    p = synth.cfg_cc("plain", scale=8, small_ij=4)
    a = p.args()
    st, info = gett.plan_describe(a["RANKA"], a["EXTA"], a["INCA"], a["RANKB"], a["EXTB"], a["INCB"],
                                  a["CONTS"], a["CONTA"], a["CONTB"], a["PERM"], a["INCC"])
    assert st == 0
    assert (info["nm"], info["nn"], info["nk"]) == (1, 1, 1)
    assert info["m"] == [(64, 1, 1)]
    assert info["k"] == [(64, 64, 1)]
    assert info["n"] == [(16, 64, 64)]


def test_plan_transposed_a_keeps_modes(L):
    p = synth.cfg_cc("perm_transA", scale=8, small_ij=4)
    a = p.args()
    st, info = gett.plan_describe(a["RANKA"], a["EXTA"], a["INCA"], a["RANKB"], a["EXTB"], a["INCB"],
                                  a["CONTS"], a["CONTA"], a["CONTB"], a["PERM"], a["INCC"])
    assert st == 0
    assert (info["nm"], info["nn"], info["nk"]) == (2, 2, 2)


def _planned_problem(p, info):
    """The canonical M/N/K problem the planner describes, as an xGETT call on
    the same buffers: A'(M modes, K modes), B'(K modes, N modes), C'(M, N)."""
    nm, nn, nk = info["nm"], info["nn"], info["nk"]
    exta = [e for e, _, _ in info["m"]] + [e for e, _, _ in info["k"]]
    inca = [s for _, s, _ in info["m"]] + [s for _, s, _ in info["k"]]
    extb = [e for e, _, _ in info["k"]] + [e for e, _, _ in info["n"]]
    incb = [s for _, _, s in info["k"]] + [s for _, s, _ in info["n"]]
    incc = [s for _, _, s in info["m"]] + [s for _, _, s in info["n"]]
    conta = list(range(nm, nm + nk))
    contb = list(range(nk))
    perm = list(range(nm + nn))
    return dict(RANKA=nm + nk, EXTA=exta, INCA=inca, RANKB=nk + nn, EXTB=extb, INCB=incb,
                CONTS=nk, CONTA=conta, CONTB=contb, PERM=perm, INCC=incc)


@pytest.mark.parametrize("family", synth.THESIS_TESTS)
@pytest.mark.parametrize("seed", range(3))
def test_planner_preserves_the_contraction(L, family, seed):
    """Planner property: the canonical problem (after squeeze, flips, fusion,
    ordering) evaluated by the oracle on the same buffers gives exactly the
    original problem's result on integer data."""
    p = synth.thesis_problem(family, 9000 + seed, np.float64, "int", c_dist="int")
    a = p.args()
    st, info = gett.plan_describe(a["RANKA"], a["EXTA"], a["INCA"], a["RANKB"], a["EXTB"], a["INCB"],
                                  a["CONTS"], a["CONTA"], a["CONTB"], a["PERM"], a["INCC"])
    assert st == 0
    ref = oracle.gett_problem(p)
    if info["empty"]:
        assert np.array_equal(ref, p.C)
        return
    q = _planned_problem(p, info)
    Cq = p.C.copy()
    rc = oracle.gett_raw("f64", q["RANKA"], q["EXTA"], q["INCA"], p.A, p.la.off + info["off_a"],
                         q["RANKB"], q["EXTB"], q["INCB"], p.B, p.lb.off + info["off_b"],
                         q["CONTS"], q["CONTA"], q["CONTB"], q["PERM"], q["INCC"], Cq,
                         p.lc.off + info["off_c"])
    assert rc == 0
    assert np.array_equal(Cq, ref)
    # canonical form: positive C increments on free modes, sorted classes
    for _, _, sc in info["m"] + info["n"]:
        assert sc > 0
    for _, sa, sb in info["k"]:
        assert sa > 0 or (sa == 0 and sb >= 0)


def _call_scaled(L, alpha=1.0, beta=1.0, prefix="d", C=0, **kw):
    a = _args(**kw)
    st, _ = gett.xgett(prefix, a["RANKA"], a["EXTA"], a["INCA"], 0, a["RANKB"], a["EXTB"], a["INCB"], 0,
                       a["CONTS"], a["CONTA"], a["CONTB"], a["PERM"], a["INCC"], C, mode="scaled",
                       alpha=alpha, beta=beta, raise_on_error=False)
    return st, gett.last_error_arg()


@pytest.mark.parametrize("prefix", ("s", "d", "c", "z", "sb"))
def test_scaled_null_scalars_reported(L, prefix):
    """alpha and beta are arguments 15 and 16 of the scaled form."""
    assert _call_scaled(L, alpha=None, prefix=prefix) == (gett.GETT_ERR_ARG, 15)
    assert _call_scaled(L, beta=None, prefix=prefix) == (gett.GETT_ERR_ARG, 16)


def test_scaled_validates_like_the_plain_form(L):
    assert _call_scaled(L, alpha=2.0, beta=0.5, PERM=(0, 0)) == (gett.GETT_ERR_ARG, 12)
    st, _ = _call_scaled(L, alpha=2.0, beta=0.5, INCC=(1, 2))
    assert st == gett.GETT_ERR_ALIAS


def test_scaled_empty_sum(L):
    """A contracted extent 0 with beta == 1 changes nothing (no pointer read);
    with another beta C is written, so a NULL C and a non-injective C are
    reported before any device work."""
    kw = dict(EXTA=(3, 0), EXTB=(0, 5), INCC=(1, 3))
    assert _call_scaled(L, alpha=2.0, beta=1.0, **kw)[0] == gett.GETT_OK
    assert _call_scaled(L, alpha=2.0, beta=0.5, **kw) == (gett.GETT_ERR_ARG, 14)
    # a C layout that is not injective (never dereferenced: the check comes first)
    kw_alias = dict(EXTA=(3, 0), EXTB=(0, 5), INCC=(1, 2))
    assert _call_scaled(L, alpha=2.0, beta=0.5, C=4096, **kw_alias)[0] == gett.GETT_ERR_ALIAS
    assert _call_scaled(L, alpha=2.0, beta=1.0, C=4096, **kw_alias)[0] == gett.GETT_OK
    # zero free extent: nothing to write at all
    assert _call_scaled(L, alpha=2.0, beta=0.5, EXTA=(0, 4))[0] == gett.GETT_OK


def _getp(**kw):
    a = dict(RANKA=3, EXTA=(3, 4, 5), INCA=(1, 3, 12), A=0, PERM=(2, 0, 1), INCC=(1, 4, 20), C=0,
             alpha=1.0, beta=0.0)
    a.update(kw)
    st = gett.getp("d", a["RANKA"], a["EXTA"], a["INCA"], a["A"], a["PERM"], a["INCC"], a["C"],
                   alpha=a["alpha"], beta=a["beta"], raise_on_error=False)
    return st, gett.last_error_arg()


def _getr(**kw):
    a = dict(RANKA=3, EXTA=(3, 4, 5), INCA=(1, 3, 12), A=0, NRED=1, RED=(1,), PERM=(1, 0), INCC=(1, 5), C=0,
             alpha=1.0, beta=0.0)
    a.update(kw)
    st = gett.getr("d", a["RANKA"], a["EXTA"], a["INCA"], a["A"], a["NRED"], a["RED"], a["PERM"], a["INCC"],
                   a["C"], alpha=a["alpha"], beta=a["beta"], raise_on_error=False)
    return st, gett.last_error_arg()


@pytest.mark.parametrize("kw,pos", [
    (dict(RANKA=-1), 1), (dict(EXTA=None), 2), (dict(EXTA=(3, -4, 5)), 2), (dict(INCA=None), 3),
    (dict(PERM=(0, 0, 1)), 5), (dict(PERM=(0, 1, 3)), 5), (dict(PERM=None), 5), (dict(INCC=None), 6),
    (dict(alpha=None), 8), (dict(beta=None), 9), (dict(), 4), (dict(A=4096), 7),
])
def test_transpose_argument_positions(L, kw, pos):
    """xGETP positions: 1 RANKA, 2 EXTA, 3 INCA, 4 A, 5 PERM, 6 INCC, 7 C, 8 alpha, 9 beta (A and C
    are only checked for NULL / alignment here, never dereferenced)."""
    assert _getp(**kw) == (gett.GETT_ERR_ARG, pos)


def test_transpose_non_injective_c_is_alias(L):
    assert _getp(INCC=(1, 2, 3))[0] == gett.GETT_ERR_ALIAS


@pytest.mark.parametrize("kw,pos", [
    (dict(NRED=4), 5), (dict(NRED=-1), 5), (dict(RED=None), 6), (dict(RED=(3,)), 6), (dict(RED=(-1,)), 6),
    (dict(NRED=2, RED=(1, 1), PERM=(0,), INCC=(1,)), 6), (dict(PERM=(0, 0)), 7), (dict(PERM=(0,)), 7),
    (dict(INCC=None), 8), (dict(alpha=None), 10), (dict(beta=None), 11),
])
def test_reduction_argument_positions(L, kw, pos):
    """xGETR positions: 5 NRED, 6 RED, 7 PERM, 8 INCC, 10 alpha, 11 beta."""
    assert _getr(**kw) == (gett.GETT_ERR_ARG, pos)


def test_aux_empty_outputs_are_noops(L):
    assert _getp(EXTA=(3, 0, 5))[0] == gett.GETT_OK
    assert _getr(EXTA=(0, 4, 5))[0] == gett.GETT_OK


def _unfusable_free_modes(n):
    """A with n free modes of extent 2 (increments 1, 2, 4, ...) and one
    contracted mode of extent 3, B a vector over that mode; C holds A's free
    modes in reverse order, so no two of them fuse (their C increments fall
    as their A increments rise)."""
    exta = (2,) * n + (3,)
    inca = tuple(2 ** i for i in range(n)) + (2 ** n,)
    perm = tuple(range(n - 1, -1, -1))
    incc = tuple(2 ** i for i in range(n))
    return exta, inca, perm, incc


@pytest.mark.parametrize("n,ok", [(24, True), (25, False)])
def test_modes_per_class_limit(L, n, ok):
    """At most 24 modes of extent > 1 per class after fusion (GETT_MAX_MODES);
    beyond that GETT_ERR_UNSUPPORTED, before any device work."""
    exta, inca, perm, incc = _unfusable_free_modes(n)
    st, info = gett.plan_describe(n + 1, exta, inca, 1, (3,), (1,), 1, (n,), (0,), perm, incc)
    if ok:
        assert st == gett.GETT_OK and info["nm"] == n and info["M"] == 2 ** n
    else:
        assert st == gett.GETT_ERR_UNSUPPORTED


def test_rank_limit_as_passed(L):
    """64 modes per tensor as passed (GETT_MAX_RANK); extent-1 modes squeeze."""
    st, info = gett.plan_describe(64, (1,) * 63 + (5,), (1,) * 64, 1, (5,), (1,), 1, (63,), (0,),
                                  tuple(range(63)), (1,) * 63)
    assert st == gett.GETT_OK and info["K"] == 5 and info["nm"] == 0
    st, _ = _call(L, RANKA=65, EXTA=(1,) * 65, INCA=(1,) * 65)
    assert st == gett.GETT_ERR_ARG and gett.last_error_arg() == 1


@pytest.mark.parametrize("ext,ok", [(1 << 31, True), ((1 << 31) + 1, False), (1 << 40, False)])
def test_broadcast_index_count_limit(L, ext, ok):
    """Contracted modes with increment 0 in both operands (broadcast) occupy
    no memory, so the spans do not bound their index count: two of extent
    `ext` give K = ext^2, accepted up to 2^62 and GETT_ERR_UNSUPPORTED above,
    before any device work and with no overflow in the planner."""
    st, info = gett.plan_describe(2, (ext, ext), (0, 0), 2, (ext, ext), (0, 0), 2, (0, 1), (0, 1), (), ())
    if ok:
        assert st == gett.GETT_OK and info["K"] == ext * ext and info["nk"] == 1
    else:
        assert st == gett.GETT_ERR_UNSUPPORTED


def test_noalloc_bounds_each_class_before_adding(L):
    """dgett_noalloc's fixed array bounds M + N + K.  Broadcast modes let two
    classes count 2^62 indices each (M = K = 2^62, N = 1), whose sum does not
    fit int64: the entry point must still answer GETT_ERR_UNSUPPORTED, before
    any device work (the device pointers here are fake and never used).  C
    spans 2^62 elements above both operands, so nothing overlaps."""
    import ctypes
    f = L.dgett_noalloc
    f.argtypes = gett._ARGS14 + [ctypes.c_void_p]
    f.restype = ctypes.c_int
    e31 = 1 << 31
    st = f(4, gett._i64((e31, e31, e31, e31)), gett._i64((0, 0, 0, 0)), ctypes.c_void_p(4096),
           2, gett._i64((e31, e31)), gett._i64((0, 0)), ctypes.c_void_p(8192),
           2, gett._i32((2, 3)), gett._i32((0, 1)), gett._i32((0, 1)), gett._i64((1, e31)),
           ctypes.c_void_p(1 << 40), ctypes.c_void_p(0))
    assert st == gett.GETT_ERR_UNSUPPORTED
    st, info = gett.plan_describe(4, (e31,) * 4, (0,) * 4, 2, (e31, e31), (0, 0), 2, (2, 3), (0, 1), (0, 1),
                                  (1, e31))
    assert st == gett.GETT_OK and info["M"] == 1 << 62 and info["K"] == 1 << 62 and info["N"] == 1


def test_options_and_report_layout(L):
    """gett_options carries the conjugation mask where three reserved ints
    were (same size); gett_report ends with the call's device time."""
    import ctypes
    assert ctypes.sizeof(gett.Options) == 8 * 4
    assert gett.Report.time_ms.offset == ctypes.sizeof(gett.Report) - 8
    o = gett.options(conj=gett.GETT_CONJ_A | gett.GETT_CONJ_B)
    assert o.conj == 3 and o.algo == 0 and o.config == -1


def test_conj_mask_validated(L):
    """Bits outside GETT_CONJ_A | GETT_CONJ_B are an argument error, before
    any device work."""
    a = _args()
    st, _ = gett.xgett("z", a["RANKA"], a["EXTA"], a["INCA"], 4096, a["RANKB"], a["EXTB"], a["INCB"], 8192,
                       a["CONTS"], a["CONTA"], a["CONTB"], a["PERM"], a["INCC"], 1 << 40, mode="ex",
                       opts=gett.options(conj=4), raise_on_error=False)
    assert st == gett.GETT_ERR_ARG
