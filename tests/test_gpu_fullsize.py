"""Parity at the full workload sizes, in the launch configuration bench.py
times, on sampled outputs the oracle computes one by one: each sampled output
element of C is the oracle's contraction of the sub-problem with every free
index fixed (Alg. 1 for one output position); for the batched workload, whole
sampled problems of the full batch."""
import numpy as np
import pytest

import oracle
from paper_2410_06770_gb300 import gett, synth
from tests._gpu_util import download, upload

pytestmark = pytest.mark.gpu


def sampled_elements(p, C_after, nsamples, seed, precision="f64", extremes=None):
    """Per sampled output: (GPU value, oracle value, sum_k |A||B|).  With
    `extremes` a list, also appends (max_k |A|, sum_k |A|, max_k |B|, sum_k
    |B|) of the output's row of A and column of B for each sample."""
    s = p.sig
    rng = np.random.default_rng(seed)
    fps = s.free_modes()
    kpos_a = synth._positions_f([s.exta[m] for m in s.conta], [p.la.inc[m] for m in s.conta], 0)
    kpos_b = synth._positions_f([s.exta[m] for m in s.conta], [p.lb.inc[m] for m in s.contb], 0)
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
        if extremes is not None:
            ra, cb = np.abs(p.A[offa + kpos_a]), np.abs(p.B[offb + kpos_b])
            extremes.append((ra.max(), ra.sum(), cb.max(), cb.sum()))
        assert oracle.gett_raw(precision, r, [s.exta[m] for m in s.conta], [p.la.inc[m] for m in s.conta], p.A, offa,
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
    ext = []
    res = sampled_elements(p, download(dC, np.float64), 96, 5, precision="ld" if algo == "ozaki_bf16" else "f64",
                           extremes=ext)
    got, ref, terms = res[:, 0], res[:, 1], res[:, 2]
    K = 128 * 128
    if algo == "native":
        # rounding bound of any summation order
        assert np.all(np.abs(got - ref) <= 2 * (K + 2) * 2.0 ** -53 * terms)
    else:
        # the split scheme's element bound against the long-double oracle:
        # 2^-b (mA sB + sA mB) + K 2^-2b mA mB + 2^-52 (|C0| + sum |A||B|)
        # (C0 is zero here), b the bits each operand keeps
        _, bits, _ = gett.ozaki_params(K)
        mA, sA, mB, sB = np.array(ext).T
        u = 2.0 ** -bits
        bound = u * (mA * sB + sA * mB) + K * u * u * mA * mB + 2.0 ** -52 * terms
        assert np.all(np.abs(got - ref) <= bound), np.max(np.abs(got - ref) - bound)
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


def test_batched_full_size_sampled():
    """The batched workload at full size (4096 contractions, seed 7) in the
    launch the bench times (one graph replay, heuristic tile choice, default
    residency): 64 sampled problems -- the 16 with the longest sums and 48
    drawn at random -- against the oracle element by element, within the fp32
    bound 2 (K+2) 2^-24 (|C0| + sum |A||B|), their C gaps untouched."""
    import torch

    from paper_2410_06770_gb300 import batch as gb
    from paper_2410_06770_gb300 import tune
    from tests._gpu_util import abs_bound
    probs = tune.draw_problems(4096, 7, 64)
    bufs = tune.DeviceBuffers(probs, values=True)
    Ks = [int(np.prod([pr["sig"].exta[m] for m in pr["sig"].conta], dtype=np.int64)) for pr in probs]
    rng = np.random.default_rng(8)
    pick = sorted(set(np.argsort(Ks)[-16:].tolist()) | set(rng.choice(len(probs), 48, replace=False).tolist()))

    def host(t, bf16):
        t = t.cpu()
        return t.view(torch.int16).numpy().view(np.uint16).copy() if bf16 else t.numpy().copy()

    before = {i: host(bufs.keep[i][2], False) for i in pick}
    b = gb.Batch(bufs.descs, select="heuristic")
    b.launch(graph=True)
    torch.cuda.synchronize()
    for i in pick:
        pr = probs[i]
        bf16 = pr["dtype"] == "bf16"
        dA, dB, dC = bufs.keep[i]
        q = synth.Problem(pr["sig"], pr["la"], pr["lb"], pr["lc"], host(dA, bf16), host(dB, bf16), before[i])
        ref = oracle.gett_problem(q, "f64", nthreads=8)
        got = host(dC, False)
        gaps = synth.gap_mask(q.lc)
        assert np.array_equal(got[gaps], q.C[gaps]), f"problem {i}: C gaps were modified"
        g = synth.gather(q.lc, got).astype(np.float64)
        r = synth.gather(q.lc, ref)
        bound = 2.0 * (Ks[i] + 2) * 2.0 ** -24 * abs_bound(q)
        assert np.all(np.abs(g - r) <= bound + 1e-30), f"problem {i} ({pr['sig']})"
    b.close()
