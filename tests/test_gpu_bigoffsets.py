"""Parity with element offsets above 2^31.  One mode of A, B or C has an
increment of 2^31 elements, so every kernel family's address arithmetic has to
be 64-bit.  The logical values are those of a compact problem with integer data
(every family and precision form is then exact, so the comparison with the
oracle is bit-exact); the rest of each large device buffer holds NaN (inputs)
or a sentinel (C), and C's sentinels are checked untouched on the device.

Each large buffer is about 2^31 elements (17 GB in FP64)."""
import numpy as np
import pytest

import oracle
from paper_2410_06770_gb300 import gett, synth
from tests._aux_ref import reduction_problem, transpose_problem
from tests._gpu_util import download, problem_for, upload

pytestmark = pytest.mark.gpu

BIG = 1 << 31
BF16_NAN = 0x7FC0


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2410_06770_gb300 import build
    build.build()
    gett.lib()
    yield
    import torch
    torch.cuda.empty_cache()


def big_layout(ext, big_mode):
    """First mode fastest and compact, except mode `big_mode`, whose increment
    is 2^31 (more than the compact part spans, so the layout stays injective)."""
    inc, s = [], 1
    for i, e in enumerate(ext):
        if i == big_mode:
            inc.append(BIG)
        else:
            inc.append(s)
            s *= e
    assert s < BIG
    size = 1 + sum((e - 1) * i for e, i in zip(ext, inc))
    return synth.Layout(tuple(ext), tuple(inc), 0, size)


def device_buffer(layout, values, fill):
    """A device buffer of layout.size elements holding `values` (logical
    order, first coordinate fastest) at the layout's positions and `fill`
    everywhere else; returns (buffer, positions on the device).  bfloat16
    values (uint16 bit patterns) travel as int16."""
    import torch
    if values.dtype == np.uint16:
        values, fill, dt = values.view(np.int16), int(np.uint16(fill).view(np.int16)), torch.int16
    else:
        fill, dt = float(fill), {np.dtype(np.float64): torch.float64, np.dtype(np.float32): torch.float32}[values.dtype]
    buf = torch.full((layout.size,), fill, dtype=dt, device="cuda")
    pos = torch.from_numpy(layout.positions()).cuda()
    buf[pos] = torch.from_numpy(np.ascontiguousarray(values)).cuda()
    return buf, pos


def place(q, big, big_modes):
    """Device buffers and increments of q's three tensors, tensor `big` (one
    of "A", "B", "C") laid out with the 2^31 increment on its mode
    big_modes[big]."""
    out = {}
    for name, lay, buf in (("A", q.la, q.A), ("B", q.lb, q.B), ("C", q.lc, q.C)):
        if name == big:
            L = big_layout(lay.ext, big_modes[name])
            fill = synth.C_GAP_SENTINEL if name == "C" else (BF16_NAN if buf.dtype == np.uint16 else np.nan)
            d, pos = device_buffer(L, synth.gather(lay, buf), fill)
            out[name] = (d, L.inc, pos)
        else:
            out[name] = (upload(buf), lay.inc, None)
    return out


def read_c(q, placed, big):
    """C's logical values after the call; for a large C also checks that
    every other element still holds the sentinel."""
    dC, _, pos = placed["C"]
    if big != "C":
        return synth.gather(q.lc, download(dC, q.C.dtype))
    got = dC[pos].cpu().numpy()
    dC[pos] = synth.C_GAP_SENTINEL
    assert bool((dC == synth.C_GAP_SENTINEL).all()), "C outside the tensor was modified"
    return got


# C[m, m2, n1, n2] += sum_k A[m, k, m2] B[k, n1, n2]: M = 80, N = 30, K = 50
GEMM = synth.Signature((40, 50, 2), (50, 15, 2), (1,), (0,), (0, 1, 2, 3))
# N = 2: the skinny family
SKINNY = synth.Signature((40, 50, 2), (50, 2), (1,), (0,), (0, 1, 2))
# K = 4: the outer family's short sums
SHORT = synth.Signature((40, 4, 2), (4, 15, 2), (1,), (0,), (0, 1, 2, 3))
# the mode of extent 2 of each tensor carries the 2^31 increment
MODES = {"GEMM": (GEMM, {"A": 2, "B": 2, "C": 1}), "SKINNY": (SKINNY, {"A": 2, "B": 1, "C": 1}),
         "SHORT": (SHORT, {"A": 2, "B": 2, "C": 1})}

CASES = [
    # (signature, prefix, options)
    ("GEMM", "d", {}),
    ("GEMM", "d", {"family": "dense", "split_k": 2}),
    ("GEMM", "d", {"family": "reduce"}),
    ("GEMM", "d", {"algo": "ozaki_bf16"}),
    ("GEMM", "s", {"algo": "bf16x6"}),
    ("GEMM", "sb", {"family": "tc"}),
    ("SKINNY", "d", {"family": "skinny"}),
    ("SHORT", "d", {"family": "outer"}),
]


@pytest.mark.parametrize("big", ["A", "B", "C"])
@pytest.mark.parametrize("case", range(len(CASES)))
def test_contraction_with_offsets_above_2_31(case, big):
    import torch
    name, prefix, kw = CASES[case]
    sig, modes = MODES[name]
    p = synth.make_problem(sig, np.random.default_rng(500 + case), np.float64, "int",
                           ("contig", "contig", "contig"), c_dist="int")
    q = problem_for(prefix, p)
    placed = place(q, big, modes)
    a = q.args()
    _, rep = gett.xgett(prefix, a["RANKA"], a["EXTA"], placed["A"][1], placed["A"][0], a["RANKB"], a["EXTB"],
                        placed["B"][1], placed["B"][0], a["CONTS"], a["CONTA"], a["CONTB"], a["PERM"],
                        placed["C"][1], placed["C"][0], mode="ex", opts=gett.options(**kw))
    torch.cuda.synchronize()
    if "family" in kw:
        assert rep["family_name"] == kw["family"]
    got = read_c(q, placed, big)
    ref = synth.gather(q.lc, oracle.gett_problem(q, "f64"))
    assert np.array_equal(got.astype(np.float64), ref), f"max |diff| {np.max(np.abs(got - ref))}"
    del placed
    torch.cuda.empty_cache()


@pytest.mark.parametrize("big", ["A", "C"])
@pytest.mark.parametrize("perm", [(2, 0, 1), (0, 2, 1), (0, 1, 2)])
def test_transpose_with_offsets_above_2_31(perm, big):
    """xGETP: the tiled kernel (fastest modes differ) and the rows kernel
    (fastest modes coincide) with A's or C's mode of extent 2 at 2^31."""
    import torch
    p = transpose_problem((40, 2, 50), perm, np.random.default_rng(600), kinds=("contig", "contig"))
    p.C[:] = 0.0
    c_big_mode = perm[1]  # C's mode holding A's mode 1 (extent 2)
    placed = place(p, big, {"A": 1, "C": c_big_mode})
    a = p.args()
    gett.getp("d", a["RANKA"], a["EXTA"], placed["A"][1], placed["A"][0], a["PERM"], placed["C"][1],
              placed["C"][0], alpha=1.0, beta=0.0)
    torch.cuda.synchronize()
    got = read_c(p, placed, big)
    ref = synth.gather(p.lc, oracle.gett_scaled(p, 1.0, 0.0))
    assert np.array_equal(got, ref)
    del placed
    torch.cuda.empty_cache()


@pytest.mark.parametrize("red", [(0,), (2,)])
def test_reduction_with_offsets_above_2_31(red):
    """xGETR over A's fastest or slowest mode, A's mode of extent 2 at 2^31."""
    import torch
    perm = (0, 1)
    p = reduction_problem((40, 2, 50), red, perm, np.random.default_rng(700), dist="int",
                          kinds=("contig", "contig"), c_dist="int")
    placed = place(p, "A", {"A": 1})
    a = p.args()
    gett.getr("d", a["RANKA"], a["EXTA"], placed["A"][1], placed["A"][0], a["CONTS"], a["CONTA"], a["PERM"],
              placed["C"][1], placed["C"][0], alpha=2.0, beta=-3.0)
    torch.cuda.synchronize()
    got = read_c(p, placed, "A")
    ref = synth.gather(p.lc, oracle.gett_scaled(p, 2.0, -3.0))
    assert np.array_equal(got, ref)
    del placed
    torch.cuda.empty_cache()
