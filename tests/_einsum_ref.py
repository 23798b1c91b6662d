"""Independent references for the oracle pins: numpy.einsum / BLAS on the
logical tensors, written from the contraction's definition (thesis Sec. 2.2)
and the PERM encoding (Sec. 5.6), not from the oracle's code."""
import string

import numpy as np

from paper_2410_06770_gb300 import synth


def einsum_spec(sig: synth.Signature) -> str:
    letters = iter(string.ascii_letters)
    a = [next(letters) for _ in sig.exta]
    b = [None] * len(sig.extb)
    for ma, mb in zip(sig.conta, sig.contb):
        b[mb] = a[ma]
    for i in range(len(b)):
        if b[i] is None:
            b[i] = next(letters)
    free = [a[m] for m in range(len(sig.exta)) if m not in sig.conta] + \
           [b[m] for m in range(len(sig.extb)) if m not in sig.contb]
    out = [None] * len(free)
    for p, letter in enumerate(free):
        out[sig.perm[p]] = letter
    return "".join(a) + "," + "".join(b) + "->" + "".join(out)


def einsum_logical(p: synth.Problem, dtype=None):
    """Logical C (shape extc, column-major semantics) = C0 + contraction."""
    A = synth.logical(p.la, p.A)
    B = synth.logical(p.lb, p.B)
    C0 = synth.logical(p.lc, p.C)
    if dtype is not None:
        A, B, C0 = A.astype(dtype), B.astype(dtype), C0.astype(dtype)
    return C0 + np.einsum(einsum_spec(p.sig), A, B)
