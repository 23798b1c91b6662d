"""Helpers shared by the GPU parity tests: upload a synth.Problem, call the
C ABI through the binding, download, compare with the oracle."""
import numpy as np

import oracle
from paper_2410_06770_gb300 import gett, synth

# tolerances of the precision forms (normwise relative), and the bound factor
# used for the element-by-element check (|err_i| <= FACTOR * K * u *
# (|C0_i| + sum_k |A||B|)_i, the rounding bound of any summation order)
TOL = {"d": 1e-13, "z": 1e-13, "s": 1e-5, "c": 1e-5, "sb": 1e-5}
UNIT = {"d": 2.0 ** -53, "z": 2.0 ** -53, "s": 2.0 ** -24, "c": 2.0 ** -24, "sb": 2.0 ** -24}
NP_DTYPE = {"d": np.float64, "s": np.float32, "z": np.complex128, "c": np.complex64, "sb": np.uint16}
C_DTYPE = {"d": np.float64, "s": np.float32, "z": np.complex128, "c": np.complex64, "sb": np.float32}


def to_bf16_bits(x: np.ndarray) -> np.ndarray:
    """float64 -> bfloat16 bit patterns (round to nearest even); NaN stays NaN."""
    f = x.astype(np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    rounded = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16).astype(np.uint16)
    nan = np.isnan(f)
    rounded[nan] = 0x7FC0
    return rounded


def problem_for(prefix, p: synth.Problem) -> synth.Problem:
    """Cast a float64/complex128 problem to the buffers of the given form."""
    q = p.copy()
    if prefix == "sb":
        q.A = to_bf16_bits(p.A.real)
        q.B = to_bf16_bits(p.B.real)
        q.C = p.C.real.astype(np.float32)
    else:
        q.A = p.A.astype(NP_DTYPE[prefix])
        q.B = p.B.astype(NP_DTYPE[prefix])
        q.C = p.C.astype(C_DTYPE[prefix])
    return q


def upload(buf: np.ndarray):
    import torch
    if buf.dtype == np.uint16:
        t = torch.from_numpy(buf.view(np.int16).copy())
    else:
        t = torch.from_numpy(buf.copy())
    return t.cuda()


def download(t, dtype) -> np.ndarray:
    a = t.cpu().numpy()
    return a.view(dtype) if a.dtype != dtype else a


def run_gpu(prefix, p: synth.Problem, mode="sync", opts=None, stream=None, alpha=1.0, beta=1.0):
    """Run the contraction on the GPU; returns (C buffer after, report).
    alpha and beta are used by mode "scaled"."""
    dA, dB, dC = upload(p.A), upload(p.B), upload(p.C)
    a = p.args()
    st, rep = gett.xgett(prefix, a["RANKA"], a["EXTA"], a["INCA"], dA, a["RANKB"], a["EXTB"], a["INCB"],
                         dB, a["CONTS"], a["CONTA"], a["CONTB"], a["PERM"], a["INCC"], dC,
                         a_off=p.la.off, b_off=p.lb.off, c_off=p.lc.off, mode=mode, opts=opts,
                         stream=stream, alpha=alpha, beta=beta)
    if mode == "async":
        import torch
        torch.cuda.synchronize()
    return download(dC, p.C.dtype), rep


def oracle_ref(p: synth.Problem, precision="f64"):
    """Oracle C buffer (widened to float64/complex128)."""
    return oracle.gett_problem(p, "z" if np.iscomplexobj(p.A) else precision)


def abs_bound(p: synth.Problem):
    """sum_k |A||B| + |C0| per logical output element (oracle on |A|, |B|)."""
    q = p.copy()
    q.A = np.abs(oracle.widen(p.A)).astype(np.float64)
    q.B = np.abs(oracle.widen(p.B)).astype(np.float64)
    q.C = np.abs(oracle.widen(p.C)).astype(np.float64)
    q.A[np.isnan(q.A)] = np.nan
    return synth.gather(p.lc, oracle.gett_problem(q, "f64"))


def _free_cont_matrices(p: synth.Problem):
    """A as an M x K and B as a K x N matrix of the logical values (free modes
    ascending, first fastest; contracted modes in CONTA / CONTB pair order)."""
    s = p.sig
    la, lb = synth.logical(p.la, p.A), synth.logical(p.lb, p.B)
    fa = [m for m in range(len(s.exta)) if m not in s.conta]
    fb = [m for m in range(len(s.extb)) if m not in s.contb]
    M = int(np.prod([s.exta[m] for m in fa], dtype=np.int64))
    N = int(np.prod([s.extb[m] for m in fb], dtype=np.int64))
    K = int(np.prod([s.exta[m] for m in s.conta], dtype=np.int64))
    Am = np.transpose(la, fa + list(s.conta)).reshape((M, K), order="F") if la.ndim else la.reshape(1, 1)
    Bm = np.transpose(lb, list(s.contb) + fb).reshape((K, N), order="F") if lb.ndim else lb.reshape(1, 1)
    return Am, Bm


def _to_output(p: synth.Problem, mat: np.ndarray) -> np.ndarray:
    """An M x N matrix over (A-free, B-free) indices -> the logical C order."""
    s = p.sig
    ext = [(s.exta if t == 0 else s.extb)[m] for t, m in s.free_modes()]
    if not ext:
        return mat.reshape(-1)
    t = mat.reshape(ext, order="F")
    # PERM's first r_C entries (the ABI reads no more)
    return np.transpose(t, np.argsort(s.perm[:len(ext)])).ravel(order="F")


def ozaki_bound(p: synth.Problem, bits: int, ref_terms: int = 0) -> np.ndarray:
    """Element bound of the split-precision (modular) DGETT / ZGETT in the
    logical C order.  Each input is rounded to an integer of `bits` bits
    relative to its row's (column's) largest magnitude, an error of at most
    2^-bits max|A[m,:]| per element (2^-bits max|B[:,n]| for B); the integer
    sum is then recovered exactly.  So
      |err| <= 2^-b (mA sB + sA mB) + K 2^-2b mA mB + 2^-52 (|C0| + sum|A||B|)
    with mA, sA the row maximum and sum of |A[m,:]| (mB, sB of B[:,n]); the
    last term covers the one rounded conversion and the addition into C.  For
    complex data the real form is bounded (|x| taken as |Re| + |Im|, the row
    maximum over both parts, 2K sums); the bound holds for each part.
    ref_terms > 0 adds the rounding error of an fp64 reference summed in
    ref_terms additions, 2 (ref_terms + 2) 2^-53 (|C0| + sum|A||B|)."""
    Am, Bm = _free_cont_matrices(p)
    if np.iscomplexobj(Am):
        aA = np.abs(Am.real) + np.abs(Am.imag)
        aB = np.abs(Bm.real) + np.abs(Bm.imag)
        mxA = np.maximum(np.abs(Am.real), np.abs(Am.imag)).max(axis=1, initial=0.0)
        mxB = np.maximum(np.abs(Bm.real), np.abs(Bm.imag)).max(axis=0, initial=0.0)
        K = 2 * Am.shape[1]
    else:
        aA, aB = np.abs(Am), np.abs(Bm)
        mxA, mxB = aA.max(axis=1, initial=0.0), aB.max(axis=0, initial=0.0)
        K = Am.shape[1]
    sA, sB = aA.sum(axis=1), aB.sum(axis=0)
    u = 2.0 ** -bits
    rnd = 2.0 ** -52 + (2.0 * (ref_terms + 2) * 2.0 ** -53 if ref_terms > 0 else 0.0)
    mat = u * (np.outer(mxA, sB) + np.outer(sA, mxB)) + K * u * u * np.outer(mxA, mxB) + rnd * (aA @ aB)
    c0 = synth.gather(p.lc, p.C)
    c0 = np.abs(c0.real) + np.abs(c0.imag) if np.iscomplexobj(c0) else np.abs(c0)
    return _to_output(p, mat) + rnd * c0


def check_elementwise(g: np.ndarray, r: np.ndarray, bound: np.ndarray, what=""):
    """|g - r| <= bound element by element (each part for complex data)."""
    if np.iscomplexobj(g) or np.iscomplexobj(r):
        err = np.maximum(np.abs((g - r).real), np.abs((g - r).imag))
    else:
        err = np.abs(g - r)
    bad = err > bound + 1e-300
    assert not np.any(bad), f"{what}: {int(bad.sum())} elements above the bound, worst excess {np.max(err - bound)}"


def compare(prefix, p: synth.Problem, got: np.ndarray, ref: np.ndarray, exact=False, tol=None, k_terms=1,
            extra_rel=0.0):
    """Element-by-element comparison of the logical C plus untouched gaps.
    The element bound is (2 (k_terms K + 2) u + extra_rel) (|C0| + sum |A||B|):
    k_terms counts the products summed per contracted index (3 or 6 for the
    bf16 split forms), extra_rel their representation error."""
    gaps = synth.gap_mask(p.lc)
    assert np.array_equal(got[gaps].view(np.uint8), p.C[gaps].view(np.uint8)), "C gaps were modified"
    g = synth.gather(p.lc, got).astype(np.complex128 if np.iscomplexobj(got) else np.float64)
    r = synth.gather(p.lc, ref)
    if exact:
        assert np.array_equal(g, r), f"max |diff| {np.max(np.abs(g - r)) if g.size else 0}"
        return 0.0
    assert np.all(np.isfinite(g)), "non-finite output"
    K = max(1, int(np.prod([p.sig.exta[m] for m in p.sig.conta], dtype=np.int64)))
    bound = abs_bound(p)
    factor = 2.0 * (k_terms * K + 2) * UNIT[prefix] * (2.0 if np.iscomplexobj(got) else 1.0) + extra_rel
    err = np.abs(g - r)
    assert np.all(err <= factor * bound + 1e-300), \
        f"element error {np.max(err - factor * bound)} above the rounding bound"
    nr = np.linalg.norm(r)
    rel = np.linalg.norm(g - r) / nr if nr > 0 else np.linalg.norm(g - r)
    assert rel <= (tol if tol is not None else TOL[prefix]), f"normwise error {rel}"
    return rel
