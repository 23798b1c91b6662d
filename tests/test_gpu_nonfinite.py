"""Inf and NaN inputs on every precision form, against the oracle.

Alg. 1 (Sec. 6) forms every product in the operand type and adds it to C, so
an Inf or NaN in row m of A (column n of B) reaches C[m, n] through IEEE
arithmetic: +-Inf when it meets nonzero finite values of one sign, NaN when
it meets a zero, an Inf of the other sign or a NaN.  The oracle is that loop.
The plain forms follow it by construction; the split forms (the modular DGETT
and ZGETT, the bf16 piece forms of SGETT, bf16 tensor cores) cannot carry a
non-finite value in their integer or bf16 pieces, so they mark its row or
column and compute the outputs there by the definition.  The test plants
+Inf, -Inf and NaN at a few logical positions of A and B and checks that
every output is NaN, +Inf or -Inf exactly where the oracle's is, that the
other outputs keep their form's accuracy, and that C's gaps stay untouched.
"""
import numpy as np
import pytest

import oracle
from paper_2410_06770_gb300 import gett, synth
from tests._gpu_util import UNIT, abs_bound, oracle_ref, ozaki_bound, problem_for, run_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2410_06770_gb300 import build
    build.build()
    gett.lib()


SHAPES = [
    synth.Signature((130, 70), (70, 300), (1,), (0,), (0, 1)),
    synth.Signature((37, 9, 5), (5, 9, 61), (1, 2), (1, 0), (1, 0, 2)),
    synth.Signature((64, 1100), (1100, 40), (1,), (0,), (1, 0)),
]

# (prefix, options): every precision form, plus the plain forms for reference
FORMS = [
    ("d", dict()),
    ("d", dict(algo="ozaki_bf16")),
    ("z", dict()),
    ("z", dict(algo="ozaki_bf16")),
    ("s", dict()),
    ("s", dict(algo="bf16x3")),
    ("s", dict(algo="bf16x6")),
    ("sb", dict(family="tc")),
]


def plant(p: synth.Problem, rng, n_a=3, n_b=2):
    """+Inf, -Inf and NaN at random logical positions of A and B (in the
    real or the imaginary part for complex data)."""
    vals = [np.inf, -np.inf, np.nan]
    for buf, lay, n in ((p.A, p.la, n_a), (p.B, p.lb, n_b)):
        pos = synth._positions_f(lay.ext, lay.inc, lay.off)
        for j, i in enumerate(rng.choice(len(pos), size=min(n, len(pos)), replace=False)):
            v = vals[j % 3]
            if np.iscomplexobj(buf):
                if j % 2:
                    buf[pos[i]] = complex(buf[pos[i]].real, v)
                else:
                    buf[pos[i]] = complex(v, buf[pos[i]].imag)
            else:
                buf[pos[i]] = v
    return p


def classes(x):
    """Per element: 0 finite, 1 NaN, 2 +Inf, 3 -Inf (each part for complex)."""
    parts = [x.real, x.imag] if np.iscomplexobj(x) else [x]
    out = []
    for v in parts:
        c = np.zeros(v.shape, dtype=np.int8)
        c[np.isnan(v)] = 1
        c[np.isposinf(v)] = 2
        c[np.isneginf(v)] = 3
        out.append(c)
    return np.stack(out)


@pytest.mark.parametrize("idx", range(len(SHAPES)))
@pytest.mark.parametrize("form", range(len(FORMS)))
def test_nonfinite_inputs_propagate(form, idx):
    prefix, kw = FORMS[form]
    rng = np.random.default_rng(900 + 10 * idx + form)
    dtype = np.complex128 if prefix in ("z", "c") else np.float64
    p = synth.make_problem(SHAPES[idx], rng, dtype, "uniform", ("padded", "negative", "contig"), "uniform")
    plant(p, rng)
    q = problem_for(prefix, p) if prefix in ("s", "sb") else p
    got, rep = run_gpu(prefix, q, mode="ex", opts=gett.options(**kw))
    ref = oracle_ref(q)
    gaps = synth.gap_mask(q.lc)
    assert np.array_equal(got[gaps].view(np.uint8), q.C[gaps].view(np.uint8)), "C gaps were modified"
    g = synth.gather(q.lc, got)
    r = synth.gather(q.lc, ref)
    cg, cr = classes(g), classes(r)
    assert np.any(cr != 0), "the planted values reach no output"
    assert np.array_equal(cg, cr), f"{int((cg != cr).sum())} outputs differ in NaN/Inf class"
    # the finite outputs keep their form's accuracy
    fin = np.all(cr == 0, axis=0)
    assert np.any(fin)
    K = max(1, int(np.prod([q.sig.exta[m] for m in q.sig.conta], dtype=np.int64)))
    algo = kw.get("algo", "native")
    if algo == "ozaki_bf16":
        kk = 2 * rep["K"] if prefix == "z" else rep["K"]
        _, bits, _ = gett.ozaki_params(kk, rep["moduli"])
        with np.errstate(invalid="ignore", over="ignore"):
            bound = ozaki_bound(q, bits, ref_terms=4 * K)
    else:
        terms, extra = {"bf16x3": (3, 3.02 * 2.0 ** -16), "bf16x6": (6, 2.02 * 2.0 ** -24)}.get(algo, (1, 0.0))
        cplx = 2.0 if prefix in ("z", "c") else 1.0
        with np.errstate(invalid="ignore", over="ignore"):
            bound = (2.0 * (terms * K + 2) * UNIT[prefix] * cplx + extra) * abs_bound(q)
    d = g[fin] - r[fin]
    err = np.maximum(np.abs(d.real), np.abs(d.imag)) if np.iscomplexobj(d) else np.abs(d)
    assert np.all(err <= bound[fin] + 1e-300), np.max(err - bound[fin])


def test_nonfinite_in_a_column_of_b_only():
    """A NaN in one column of B leaves every other column of the split DGETT
    result exact to its bound and turns exactly that column of C into NaN."""
    sig = synth.Signature((96, 200), (200, 50), (1,), (0,), (0, 1))
    p = synth.make_problem(sig, np.random.default_rng(5), np.float64, "normal", ("contig",) * 3, "zeros")
    col = 17
    p.B[p.lb.off + 3 * p.lb.inc[0] + col * p.lb.inc[1]] = np.nan
    got, rep = run_gpu("d", p, mode="ex", opts=gett.options(algo="ozaki_bf16"))
    g = synth.gather(p.lc, got).reshape(96, 50, order="F")
    assert np.all(np.isnan(g[:, col]))
    others = np.delete(g, col, axis=1)
    assert np.all(np.isfinite(others))
    r = synth.gather(p.lc, oracle.gett_problem(p, "ld")).reshape(96, 50, order="F")
    assert np.linalg.norm(others - np.delete(r, col, axis=1)) <= 1e-13 * np.linalg.norm(np.delete(r, col, axis=1))
