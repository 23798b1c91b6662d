"""Transpose and reduction problems as contractions (their definition): the
transpose is xGETT with a rank-0 B of value 1, the reduction xGETT with B a
tensor of ones over the reduced modes contracted with them."""
import numpy as np

from paper_2410_06770_gb300 import synth


def transpose_problem(exta, perm, rng, dtype=np.float64, dist="uniform", kinds=("padded", "padded"),
                      c_dist="uniform"):
    sig = synth.Signature(tuple(exta), (), (), (), tuple(perm))
    p = synth.make_problem(sig, rng, dtype, dist, (kinds[0], "contig", kinds[1]), c_dist)
    p.B = np.ones_like(p.B)
    return p


def reduction_problem(exta, red, perm, rng, dtype=np.float64, dist="uniform", kinds=("padded", "padded"),
                      c_dist="uniform"):
    extb = tuple(exta[r] for r in red)
    sig = synth.Signature(tuple(exta), extb, tuple(red), tuple(range(len(red))), tuple(perm))
    p = synth.make_problem(sig, rng, dtype, dist, (kinds[0], "contig", kinds[1]), c_dist)
    p.B = np.ones_like(p.B)
    return p
