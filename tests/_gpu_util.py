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


def compare(prefix, p: synth.Problem, got: np.ndarray, ref: np.ndarray, exact=False, tol=None):
    """Element-by-element comparison of the logical C plus untouched gaps."""
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
    factor = 2.0 * (K + 2) * UNIT[prefix] * (2.0 if np.iscomplexobj(got) else 1.0)
    err = np.abs(g - r)
    assert np.all(err <= factor * bound + 1e-300), \
        f"element error {np.max(err - factor * bound)} above the rounding bound"
    nr = np.linalg.norm(r)
    rel = np.linalg.norm(g - r) / nr if nr > 0 else np.linalg.norm(g - r)
    assert rel <= (tol if tol is not None else TOL[prefix]), f"normwise error {rel}"
    return rel
