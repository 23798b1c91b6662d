"""Parity at the full workload sizes, in the launch configuration bench.py
times, on sampled outputs the oracle computes one by one: each sampled output
element of C is the oracle's contraction of the sub-problem with every free
index fixed (Alg. 1 for one output position)."""
import numpy as np
import pytest

import oracle
from paper_2410_06770_gb300 import gett, synth
from tests._gpu_util import download, upload

pytestmark = pytest.mark.gpu


def sampled_elements(p, C_after, nsamples, seed):
    s = p.sig
    rng = np.random.default_rng(seed)
    fps = s.free_modes()
    out = []
    for _ in range(nsamples):
        o = [int(rng.integers(0, e)) for e in s.extc()]
        offa, offb = p.la.off, p.lb.off
        for pidx, (t, m) in enumerate(fps):
            x = o[s.perm[pidx]]
            if t == 0:
                offa += x * p.la.inc[m]
            else:
                offb += x * p.lb.inc[m]
        r = s.conts
        c = np.zeros(1)
        assert oracle.gett_raw("f64", r, [s.exta[m] for m in s.conta], [p.la.inc[m] for m in s.conta], p.A, offa,
                               r, [s.exta[m] for m in s.conta], [p.lb.inc[m] for m in s.contb], p.B, offb,
                               r, list(range(r)), list(range(r)), [], [], c, 0) == 0
        terms = np.zeros(1)
        assert oracle.gett_raw("f64", r, [s.exta[m] for m in s.conta], [p.la.inc[m] for m in s.conta],
                               np.abs(p.A), offa, r, [s.exta[m] for m in s.conta],
                               [p.lb.inc[m] for m in s.contb], np.abs(p.B), offb,
                               r, list(range(r)), list(range(r)), [], [], terms, 0) == 0
        offc = p.lc.off + sum(x * i for x, i in zip(o, p.lc.inc))
        out.append((C_after[offc], c[0] + p.C[offc], terms[0]))
    return np.array(out)


@pytest.mark.parametrize("algo", ["native", "ozaki_bf16"])
@pytest.mark.parametrize("variant", ["plain", "perm_transA"])
def test_cc_full_size_sampled(algo, variant):
    import torch
    p = synth.cfg_cc(variant)
    dA, dB, dC = upload(p.A), upload(p.B), upload(p.C)
    a = p.args()
    gett.xgett("d", a["RANKA"], a["EXTA"], a["INCA"], dA, a["RANKB"], a["EXTB"], a["INCB"], dB, a["CONTS"],
               a["CONTA"], a["CONTB"], a["PERM"], a["INCC"], dC, mode="ex", opts=gett.options(algo=algo))
    torch.cuda.synchronize()
    res = sampled_elements(p, download(dC, np.float64), 96, 5)
    got, ref, terms = res[:, 0], res[:, 1], res[:, 2]
    K = 128 * 128
    if algo == "native":
        # rounding bound of any summation order
        assert np.all(np.abs(got - ref) <= 2 * (K + 2) * 2.0 ** -53 * terms)
    # normwise over the sample
    assert np.linalg.norm(got - ref) <= 1e-13 * np.linalg.norm(ref)


def test_stream_full_size_sampled():
    import torch
    p = synth.cfg_stream(c_host=False)
    dA, dB = upload(p.A), upload(p.B)
    dC = torch.zeros(p.lc.size, dtype=torch.float64, device="cuda")
    a = p.args()
    _, rep = gett.xgett("d", a["RANKA"], a["EXTA"], a["INCA"], dA, a["RANKB"], a["EXTB"], a["INCB"], dB,
                        a["CONTS"], a["CONTA"], a["CONTB"], a["PERM"], a["INCC"], dC, mode="ex")
    assert rep["family_name"] == "outer"
    torch.cuda.synchronize()
    rng = np.random.default_rng(3)
    idx = rng.integers(0, p.lc.size, 4096)
    got = dC[torch.from_numpy(idx).cuda()].cpu().numpy()
    # C[m, n] = A[m] * B[n] with m fastest (C is (256,256,64,64,8) column-major)
    m, n = idx % p.la.numel, idx // p.la.numel
    ref = p.A[m] * p.B[n]
    assert np.array_equal(got, ref)  # one rounded product added to zero


def test_small_split_precision_logu_full():
    p = synth.cfg_small_dgett(dist="logu")
    from tests._gpu_util import run_gpu
    got, _ = run_gpu("d", p, mode="ex", opts=gett.options(algo="ozaki_bf16"))
    ref = synth.gather(p.lc, oracle.gett_problem(p, "ld", nthreads=8))
    g = synth.gather(p.lc, got)
    assert np.linalg.norm(g - ref) <= 1e-13 * np.linalg.norm(ref)
