"""Host-side validation of gett_batch_create.  Every check runs before the
library touches a device, so these run without a GPU: the rejected problem is
reported by index together with the failing argument's position (the
problem's own xGETT argument list, Sec. 5.7); C regions of different problems
may overlap neither each other nor any operand, while operands may be shared.
Device addresses are fake: validation never dereferences them."""
import pytest

from paper_2410_06770_gb300 import batch as gb
from paper_2410_06770_gb300 import gett

BASE = 1 << 40
SLOT = 4096


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2410_06770_gb300 import build
    build.build()
    gett.lib()


def desc(i, **kw):
    """C[m, n] += sum_k A[m, k] B[k, n], 8 x 6 x 5, column-major fp32, in
    the i-th disjoint slot of fake device memory."""
    d = dict(dtype="f32", EXTA=(8, 5), INCA=(1, 8), EXTB=(5, 6), INCB=(1, 5), CONTA=(1,), CONTB=(0,),
             PERM=(0, 1), INCC=(1, 8), A=BASE + i * SLOT, B=BASE + i * SLOT + 1024, C=BASE + i * SLOT + 2048)
    d.update(kw)
    return d


def rejected(descs, **opts):
    with pytest.raises(gett.GettError) as ei:
        gb.Batch(descs, **opts)
    return ei.value


def _gpu():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:  # pragma: no cover
        return False


def test_valid_batch_needs_the_device():
    """A valid batch passes validation; with no GPU the library reports a CUDA
    error (there is no CPU fallback)."""
    descs = [desc(i) for i in range(4)]
    descs[3] = desc(3, A=descs[0]["A"], B=descs[1]["B"])  # operands may be shared
    if _gpu():
        gb.Batch(descs).close()
    else:
        assert rejected(descs).status == gett.GETT_ERR_CUDA


@pytest.mark.parametrize("field,value,pos", [
    ("PERM", (0, 0), 12),          # not a permutation
    ("CONTA", (2,), 10),           # contracted mode out of range
    ("CONTB", (1,), None),         # B's contracted mode has another extent
    ("EXTB", (4, 6), None),        # paired extents differ
    ("EXTA", (8, -5), 2),          # negative extent
    ("A", 0, 4),                   # NULL operand of a non-empty problem
    ("B", 0, 8),
    ("C", 0, 14),
])
def test_invalid_problem_reported_by_index(field, value, pos):
    descs = [desc(i) for i in range(3)]
    descs[1] = desc(1, **{field: value})
    e = rejected(descs)
    assert e.status == gett.GETT_ERR_ARG
    assert e.bad_index == 1
    if pos is not None:
        assert e.arg == pos


def test_unknown_operand_type():
    """An operand type other than fp32 (0) or bf16 (1), through the C ABI."""
    import ctypes
    L = gb._bind()
    keep = []
    arr = (gb.ProblemDesc * 2)()
    for i in range(2):
        d, pr = arr[i], desc(i)
        d.dtype = 0 if i == 0 else 7
        for name in ("EXTA", "INCA", "EXTB", "INCB", "INCC"):
            x = gett._i64(pr[name])
            keep.append(x)
            setattr(d, name, ctypes.cast(x, gb._i64p))
        for name in ("CONTA", "CONTB", "PERM"):
            x = gett._i32(pr[name])
            keep.append(x)
            setattr(d, name, ctypes.cast(x, gb._ip))
        d.RANKA, d.RANKB, d.CONTS = 2, 2, 1
        d.A, d.B, d.C = pr["A"], pr["B"], pr["C"]
    h = ctypes.c_void_p()
    bad = ctypes.c_int(-5)
    st = L.gett_batch_create(2, arr, None, ctypes.byref(h), ctypes.byref(bad))
    assert st == gett.GETT_ERR_ARG and bad.value == 1 and not h.value


def test_empty_problem_needs_no_pointers():
    """A zero extent: nothing to compute, so NULL buffers are accepted."""
    descs = [desc(0), desc(1, EXTA=(8, 0), EXTB=(0, 6), A=0, B=0, C=0)]
    if _gpu():
        gb.Batch(descs).close()
    else:
        assert rejected(descs).status == gett.GETT_ERR_CUDA


def test_non_injective_c_is_alias():
    descs = [desc(0), desc(1, INCC=(1, 1))]
    e = rejected(descs)
    assert e.status == gett.GETT_ERR_ALIAS and e.bad_index == 1


@pytest.mark.parametrize("what", ["C", "A", "B"])
def test_overlap_with_another_problems_c_is_alias(what):
    """Problem 2's C, A or B starts inside problem 0's C (192 bytes from
    offset 2048 of slot 0)."""
    descs = [desc(i) for i in range(3)]
    descs[2] = desc(2, **{what: descs[0]["C"] + 64})
    e = rejected(descs)
    assert e.status == gett.GETT_ERR_ALIAS
    assert e.bad_index in (0, 2)


def test_adjacent_c_regions_are_not_overlap():
    """C of problem 1 starts at the first byte after problem 0's C."""
    descs = [desc(0), desc(1, C=desc(0)["C"] + 8 * 6 * 4)]
    if _gpu():
        gb.Batch(descs).close()
    else:
        assert rejected(descs).status == gett.GETT_ERR_CUDA


def test_selection_options_validated():
    descs = [desc(0)]
    assert rejected(descs, select="fixed", config=gb.num_configs()).status == gett.GETT_ERR_ARG
    assert rejected(descs, select="fixed", config=-1).status == gett.GETT_ERR_ARG
    assert rejected(descs, select="table", configs=None).status == gett.GETT_ERR_ARG
    assert rejected(descs, serial=2).status == gett.GETT_ERR_ARG


def test_broadcast_class_beyond_the_table_limit():
    """A contracted mode with increment 0 in both operands occupies no memory,
    so its extent is not bounded by the address spans; a class of 2^40
    indices would need terabytes of host offset tables.  The batch rejects it
    with GETT_ERR_UNSUPPORTED and the problem's index, before allocating."""
    big = 1 << 40
    descs = [desc(0), desc(1, EXTA=(8, big), INCA=(1, 0), EXTB=(big, 6), INCB=(0, 5))]
    e = rejected(descs)
    assert e.status == gett.GETT_ERR_UNSUPPORTED and e.bad_index == 1


def test_shipped_planner_model_matches_the_configuration_space():
    """The trained planner weights beside the package predict one score per
    batched configuration the library offers (a stale file from a smaller
    configuration space would be refused by install_model at run time)."""
    import os
    from paper_2410_06770_gb300 import tune
    path = os.path.join(os.path.dirname(gb.__file__), "planner_mlp.npz")
    model = tune.load_model(path)
    assert model["nout"] == gb.num_configs()
    assert model["mean"].shape == model["std"].shape == (24,)
    h, n = model["hidden"], model["nout"]
    assert model["params"].size == (24 * h + h) + (h * h + h) + (h * n + n)

