"""Run one contraction of a named workload through the C ABI, for profilers.

    python -m paper_2410_06770_gb300.profile_case WORKLOAD [SCALE] [--calls N] [--algo A] [--tuned]
        [--learned] [--serial]

WORKLOAD: cc, cc_perm_transA (extents a..d = SCALE, i,j = SCALE/4), stream
(A(SCALE, SCALE, 64) x B(64, 8)), small, gemv (A(SCALE, SCALE) x B(SCALE, 2),
the second mode of A contracted), inner (A and B of extents SCALE^4, every
mode contracted), transpose (xGETP of A(SCALE^4) with its modes reversed),
batched (SCALE contractions of the batched workload, one
persistent launch per call).  gemv and inner draw uniform values on the device.  Inputs are generated on the host,
copied once, then the call is made N times (default 2) and synchronised.
--tuned loads the package's tuning database first (the configuration the
bench's calls use).  For batched: --learned selects configurations with the
package's trained planner (the bench's learned launch), --serial launches
every kernel on one stream (a profiler then sees one kernel at a time).
"""
import argparse
import sys


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("workload")
    ap.add_argument("scale", nargs="?", type=int, default=128)
    ap.add_argument("--calls", type=int, default=2)
    ap.add_argument("--algo", default="native")
    ap.add_argument("--prefix", default="d")
    ap.add_argument("--tuned", action="store_true")
    ap.add_argument("--learned", action="store_true")
    ap.add_argument("--serial", action="store_true")
    args = ap.parse_args(argv)
    import os

    import torch

    from . import build, gett, synth
    build.build()
    if args.tuned:
        gett.tune_db_load(os.path.join(os.path.dirname(os.path.abspath(__file__)), "tune_db.txt"))
    if args.workload == "batched":
        from . import batch as gb
        from . import tune
        probs = tune.draw_problems(args.scale, 7, 64)
        bufs = tune.DeviceBuffers(probs)
        if args.learned:
            tune.install(tune.load_model(os.path.join(os.path.dirname(os.path.abspath(__file__)),
                                                      "planner_mlp.npz")))
        b = gb.Batch(bufs.descs, select="learned" if args.learned else "heuristic", serial=args.serial)
        for _ in range(args.calls):
            b.launch()
        torch.cuda.synchronize()
        print(b.info())
        return 0
    if args.workload == "transpose":
        # A(s,s,s,s) -> C with the modes reversed (xGETP), FP64, C not read
        s4 = (args.scale,) * 4
        la = synth.layout_contiguous(s4)
        perm = (3, 2, 1, 0)
        lc = synth.layout_contiguous(s4)
        g = torch.Generator(device="cuda")
        g.manual_seed(9)
        dA = torch.rand(la.size, dtype=torch.float64, device="cuda", generator=g)
        dC = torch.empty(lc.size, dtype=torch.float64, device="cuda")
        for _ in range(args.calls):
            gett.getp("d", 4, s4, la.inc, dA, perm, lc.inc, dC, alpha=1.0, beta=0.0)
        torch.cuda.synchronize()
        print("transpose", s4, perm)
        return 0
    if args.workload in ("gemv", "inner"):
        s = args.scale
        if args.workload == "gemv":
            sig = synth.Signature((s, s), (s, 2), (1,), (0,), (0, 1))
        else:
            sig = synth.Signature((s,) * 4, (s,) * 4, (0, 1, 2, 3), (0, 1, 2, 3), ())
        la, lb, lc = (synth.layout_contiguous(e) for e in (sig.exta, sig.extb, sig.extc()))
        g = torch.Generator(device="cuda")
        g.manual_seed(9)
        dt = torch.float32 if args.prefix == "s" else torch.float64
        dA = torch.rand(la.size, dtype=dt, device="cuda", generator=g)
        dB = torch.rand(lb.size, dtype=dt, device="cuda", generator=g)
        dC = torch.zeros(lc.size, dtype=dt, device="cuda")
        rep = None
        for _ in range(args.calls):
            _, rep = gett.xgett(args.prefix, len(sig.exta), sig.exta, la.inc, dA, len(sig.extb), sig.extb, lb.inc, dB,
                                sig.conts, sig.conta, sig.contb, sig.perm, lc.inc, dC, mode="ex")
        torch.cuda.synchronize()
        print(rep)
        return 0
    if args.workload == "cc":
        p = synth.cfg_cc("plain", scale=args.scale, small_ij=max(1, args.scale // 4))
    elif args.workload == "cc_perm_transA":
        p = synth.cfg_cc("perm_transA", scale=args.scale, small_ij=max(1, args.scale // 4))
    elif args.workload == "stream":
        p = synth.cfg_stream(a_ext=(args.scale, args.scale, 64), b_ext=(64, 8))
    elif args.workload == "small":
        p = synth.cfg_small_dgett()
    else:
        raise SystemExit(f"unknown workload {args.workload}")
    if args.prefix in ("s", "c"):
        # single-precision calls read fp32 (complex64) operands
        import numpy as np
        t = np.float32 if args.prefix == "s" else np.complex64
        p.A, p.B, p.C = p.A.astype(t), p.B.astype(t), p.C.astype(t)
    dA = torch.from_numpy(p.A).cuda()
    dB = torch.from_numpy(p.B).cuda()
    dC = torch.from_numpy(p.C).cuda()
    a = p.args()
    opts = gett.options(algo=args.algo)
    rep = None
    for _ in range(args.calls):
        _, rep = gett.xgett(args.prefix, a["RANKA"], a["EXTA"], a["INCA"], dA, a["RANKB"], a["EXTB"],
                            a["INCB"], dB, a["CONTS"], a["CONTA"], a["CONTB"], a["PERM"], a["INCC"], dC,
                            a_off=p.la.off, b_off=p.lb.off, c_off=p.lc.off, mode="ex", opts=opts)
    torch.cuda.synchronize()
    print(rep)
    return 0


if __name__ == "__main__":
    sys.exit(main())
