"""GPU parity of the batched persistent launch: every problem's C against the
oracle (fp32 arithmetic: element bound 2 (K+2) 2^-24 (|C0| + sum |A||B|)),
plain and graph launches, every configuration (tile shape x GATHER / PACK,
and SKINNY), skinny-heavy batches with K slices, alias rejection."""
import numpy as np
import pytest

import oracle
from paper_2410_06770_gb300 import batch as gb
from paper_2410_06770_gb300 import gett, synth
from tests._gpu_util import abs_bound, download, problem_for, upload

pytestmark = pytest.mark.gpu


def make_batch_problems(n, seed, max_ext=12, pad_frac=0.25):
    rng = np.random.default_rng(seed)
    probs = []
    for i in range(n):
        k = int(rng.integers(0, 4))
        ra = int(rng.integers(max(2, k), 6))
        rb = int(rng.integers(max(2, k), 6))
        sig = synth.capped_signature(rng, ra, rb, k, 2, max_ext, 1 << 16)
        kinds = ("padded",) * 3 if rng.random() < pad_frac else ("contig",) * 3
        p = synth.make_problem(sig, rng, np.float64, "uniform", kinds, "uniform")
        prefix = "sb" if rng.integers(0, 2) else "s"
        probs.append((prefix, problem_for(prefix, p)))
    return probs


def make_skinny_problems(n, seed):
    """Dot products (no free index), GEMV shapes (one free class of at most 8
    indices) and few-output sums (both free classes of at most 4 indices,
    sums long enough for several K slices), in random layouts."""
    rng = np.random.default_rng(seed)
    probs = []
    for i in range(n):
        kind = i % 3
        k1, k2 = int(rng.integers(8, 90)), int(rng.integers(8, 90))
        if kind == 0:
            sig = synth.Signature((k1, k2), (k2, k1), (0, 1), (1, 0), ())
        elif kind == 1:
            m, s_ = int(rng.integers(20, 300)), int(rng.integers(1, 9))
            sig = synth.Signature((k1, m, k2), (k2, s_, k1), (0, 2), (2, 0), (0, 1)) if rng.integers(0, 2) \
                else synth.Signature((k1, s_, k2), (k2, m, k1), (0, 2), (2, 0), (1, 0))
        else:
            m, s_ = int(rng.integers(1, 5)), int(rng.integers(1, 5))
            sig = synth.Signature((m, k1, k2), (k1, k2, s_), (1, 2), (0, 1), (1, 0))
        kinds = tuple(rng.choice(["contig", "padded", "rowmajor", "negative"], 3))
        p = synth.make_problem(sig, rng, np.float64, "uniform", kinds, "uniform")
        prefix = "sb" if rng.integers(0, 2) else "s"
        probs.append((prefix, problem_for(prefix, p)))
    return probs


def upload_all(probs):
    dev = []
    descs = []
    for prefix, q in probs:
        dA, dB, dC = upload(q.A), upload(q.B), upload(q.C)
        dev.append((dA, dB, dC))
        a = q.args()
        descs.append(dict(dtype="bf16" if prefix == "sb" else "f32",
                          EXTA=a["EXTA"], INCA=a["INCA"], EXTB=a["EXTB"], INCB=a["INCB"],
                          CONTA=a["CONTA"], CONTB=a["CONTB"], PERM=a["PERM"], INCC=a["INCC"],
                          A=dA.data_ptr() + q.la.off * dA.element_size(),
                          B=dB.data_ptr() + q.lb.off * dB.element_size(),
                          C=dC.data_ptr() + q.lc.off * dC.element_size()))
    return dev, descs


def check_all(probs, dev, times=1):
    for (prefix, q), (_, _, dC) in zip(probs, dev):
        got = download(dC, np.float32)
        ref = oracle.widen(q.C).copy()
        for _ in range(times):
            ref = oracle.gett_problem(q, C=ref)
        gaps = synth.gap_mask(q.lc)
        assert np.array_equal(got[gaps], q.C[gaps])
        g = synth.gather(q.lc, got).astype(np.float64)
        r = synth.gather(q.lc, ref)
        K = max(1, int(np.prod([q.sig.exta[m] for m in q.sig.conta], dtype=np.int64)))
        bound = abs_bound(q) * times
        assert np.all(np.abs(g - r) <= 2.0 * (K + 2) * times * 2.0 ** -24 * bound + 1e-30)


@pytest.mark.parametrize("select,config", [("heuristic", 0)] + [("fixed", c) for c in range(10)])
def test_batch_matches_oracle(select, config):
    import torch
    probs = make_batch_problems(150, 1 + config)
    dev, descs = upload_all(probs)
    b = gb.Batch(descs, select=select, config=config)
    info = b.info()
    assert info["n"] == 150 and info["tiles"] > 0
    if select == "fixed" and gb.config_method(config) == 1:
        assert info["packed_items"] > 0 and info["pack_items"] > 0
    if select == "fixed" and gb.config_method(config) == 3:
        # the bf16 problems run on the tensor cores, the float ones fall back
        assert info["tc_items"] > 0 and info["tc_pack_items"] > 0 and info["fallbacks"] > 0
    if select == "heuristic":
        assert info["packed_items"] > 0 and info["gather_items"] > 0
    b.launch()
    torch.cuda.synchronize()
    check_all(probs, dev)
    b.close()


@pytest.mark.parametrize("select", ["heuristic", "pack", "gather"])
def test_skinny_heavy_batch(select):
    """Dot, GEMV-like and few-output problems: the skinny warp kernel (lanes
    along the long class, and lanes along the sum with K slices added in
    order by the reduction) under the heuristic, and the same problems as
    packed or gathered tiles through a table."""
    import torch
    probs = make_skinny_problems(90, 31)
    dev, descs = upload_all(probs)
    if select == "heuristic":
        b = gb.Batch(descs)
        info = b.info()
        assert info["skinny_items"] > 0 and info["config_count"][8] == 90
    else:
        cfg = 6 if select == "pack" else 2
        b = gb.Batch(descs, select="table", configs=[cfg] * len(descs))
        assert b.info()["config_count"][cfg] == 90
    b.launch(graph=True)
    torch.cuda.synchronize()
    check_all(probs, dev)
    b.close()


def test_config_descriptions():
    assert gb.num_configs() == 10
    assert [gb.config_method(c) for c in range(10)] == [0] * 4 + [1] * 4 + [2, 3]


def make_tc_problems(n, seed):
    """bf16 problems for the tensor-core method: ragged M, N, K over several
    128 x 128 tiles and 64-wide K tiles (K from 1 to a few hundred), random
    layouts and output permutations."""
    rng = np.random.default_rng(seed)
    probs = []
    for i in range(n):
        m, nn, k1 = int(rng.integers(1, 300)), int(rng.integers(1, 300)), int(rng.integers(1, 40))
        k2 = int(rng.integers(1, 12))
        if i % 2:
            sig = synth.Signature((m, k1, k2), (k2, nn, k1), (1, 2), (2, 0), (1, 0))
        else:
            sig = synth.Signature((k1, m), (nn, k1), (0,), (1,), (0, 1))
        kinds = tuple(rng.choice(["contig", "padded", "rowmajor", "negative"], 3))
        p = synth.make_problem(sig, rng, np.float64, "uniform", kinds, "uniform")
        probs.append(("sb", problem_for("sb", p)))
    return probs


def test_tensor_core_method_matches_oracle():
    """The TC method: bf16 problems packed into swizzled 128 x 64 tiles and
    multiplied by tcgen05 in one grouped launch, graph-replayed twice
    (accumulating), element by element against the oracle."""
    import torch
    probs = make_tc_problems(40, 41)
    dev, descs = upload_all(probs)
    b = gb.Batch(descs, select="fixed", config=9)
    info = b.info()
    assert info["tc_items"] > 0 and info["config_count"][9] == 40 and info["fallbacks"] == 0
    b.launch(graph=True)
    b.launch(graph=True)
    torch.cuda.synchronize()
    check_all(probs, dev, times=2)
    b.close()


@pytest.mark.parametrize("ctas_per_sm", [1, 3, 4, 6])
def test_batch_residency_variants(ctas_per_sm):
    """The kernels compiled for 3 and 4 resident CTAs per SM (and grids of 1
    or 6 CTAs per SM, the last with CTAs that start only when others finish)
    give the same parity; graph launch."""
    import torch
    probs = make_batch_problems(150, 20 + ctas_per_sm)
    dev, descs = upload_all(probs)
    b = gb.Batch(descs, ctas_per_sm=ctas_per_sm)
    b.launch(graph=True)
    torch.cuda.synchronize()
    check_all(probs, dev)
    b.close()


def test_batch_graph_replay_accumulates():
    import torch
    probs = make_batch_problems(100, 7)
    dev, descs = upload_all(probs)
    b = gb.Batch(descs)
    b.launch(graph=True)
    b.launch(graph=True)
    torch.cuda.synchronize()
    check_all(probs, dev, times=2)


def test_batch_deterministic():
    import torch
    probs = make_batch_problems(80, 9)
    outs = []
    for _ in range(2):
        dev, descs = upload_all(probs)
        b = gb.Batch(descs)
        b.launch()
        torch.cuda.synchronize()
        outs.append([download(dC, np.float32).copy() for (_, _, dC) in dev])
    for x, y in zip(*outs):
        assert np.array_equal(x, y)


def test_concurrent_branches_match_serial_launch():
    """A batch that uses every method (gathered, packed, skinny, tensor-core
    tiles, K-slice reduction): its method chains run as concurrent branches
    forked from the launch stream, eagerly and graph-captured, on a side
    stream whose earlier work (zeroing every C) they must wait for; the
    results equal the single-stream launch bit for bit and the oracle."""
    import torch
    probs = (make_batch_problems(60, 71) + make_skinny_problems(30, 72) + make_tc_problems(20, 73))
    outs = {}
    for mode in ("serial", "eager", "graph"):
        dev, descs = upload_all(probs)
        # heuristic choices, and the tensor cores for the bf16 problems
        configs = [-1] * 90 + [9] * 20
        b = gb.Batch(descs, select="table", configs=configs, serial=(mode == "serial"))
        info = b.info()
        assert min(info["gather_items"], info["packed_items"], info["skinny_items"], info["tc_items"]) > 0
        side = torch.cuda.Stream()
        saved = [dC.clone() for (_, _, dC) in dev]
        torch.cuda.synchronize()
        with torch.cuda.stream(side):
            # queued first on the launch stream: C <- 0, then C <- saved C;
            # a branch that ran ahead of these would see the zeros or race them
            for (_, _, dC), c0 in zip(dev, saved):
                dC.zero_()
                torch.cuda._sleep(20000)
                dC.copy_(c0)
            b.launch(stream=side.cuda_stream, graph=(mode == "graph"))
        side.synchronize()
        outs[mode] = [download(dC, np.float32).copy() for (_, _, dC) in dev]
        check_all(probs, dev)
        b.close()
    for x, y, z in zip(outs["serial"], outs["eager"], outs["graph"]):
        assert np.array_equal(x, y) and np.array_equal(x, z)


def test_batch_rejects_overlapping_outputs():
    import torch
    probs = make_batch_problems(2, 11)
    dev, descs = upload_all(probs)
    descs[1]["C"] = descs[0]["C"]
    with pytest.raises(gett.GettError) as ei:
        gb.Batch(descs)
    assert ei.value.status == gett.GETT_ERR_ALIAS


def test_batch_table_selection_and_learned_fallback():
    import torch
    probs = make_batch_problems(60, 13)
    dev, descs = upload_all(probs)
    gb.clear_model()
    b = gb.Batch(descs, select="learned")
    assert b.info()["fallbacks"] == b.info()["nonempty"]  # no model: heuristic everywhere
    cfgs = [i % gb.num_configs() for i in range(60)]
    b2 = gb.Batch(descs, select="table", configs=cfgs)
    b2.launch()
    torch.cuda.synchronize()
    check_all(probs, dev)
