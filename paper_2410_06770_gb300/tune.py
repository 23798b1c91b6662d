"""Autotuner and learned-planner training for the batched path.

    python -m paper_2410_06770_gb300.tune --train 20000 --test 2000 \\
        --model OUT.npz --report OUT.json

1. Draws contraction signatures from the batched workload's distribution
   (ranks 2-5, extents up to --max-ext, 0-3 contracted modes, 25 % padded,
   fp32/bf16 operands, <= 2^18 elements per tensor).
2. Autotuner: times every problem with every configuration of the batched
   launch -- tile shape x method: gathered tiles (logical mode fusion only),
   packed tiles (the operands' modes physically fused by a packing copy) or
   the skinny warp kernel where a free class has at most 8 indices
   (gett_batch_profile in throughput mode: the problem's items repeated until
   the GPU is full, CUDA events around back-to-back launches, time per copy)
   -> a table of costs; the exhaustive best configuration is the tuned choice.
3. Learned planner: features of each signature (gett_problem_features) ->
   MLP predicting normalised log times of all configurations, trained on the
   GPU by the library's own kernels (gett_mlp_fit).
4. Held-out evaluation: regret of the network's choice against exhaustive
   tuning (geometric mean of t_pred / t_best - 1, share above 10 %), the same
   for the fixed heuristic, fallback rate, and end-to-end throughput of one
   persistent launch with learned vs heuristic vs tuned configurations.
"""
from __future__ import annotations

import argparse
import json
import sys
import time

import numpy as np

from . import batch as gb
from . import synth


def draw_problems(n, seed, max_ext):
    sigs = synth.batched_signatures(n=n, seed=seed, max_ext=max_ext)
    probs = []
    for d in sigs:
        s = d["sig"]
        pads = d["pads"]
        la = synth.layout_with_pads(s.exta, pads[0] if pads else None)
        lb = synth.layout_with_pads(s.extb, pads[1] if pads else None)
        lc = synth.layout_with_pads(s.extc(), pads[2] if pads else None)
        probs.append(dict(sig=s, la=la, lb=lb, lc=lc, dtype=d["dtype"], seed=d["value_seed"]))
    return probs


def args_of(pr):
    s = pr["sig"]
    return dict(EXTA=s.exta, INCA=pr["la"].inc, EXTB=s.extb, INCB=pr["lb"].inc, CONTA=s.conta,
                CONTB=s.contb, PERM=s.perm, INCC=pr["lc"].inc)


def flops(pr):
    s = pr["sig"]
    K = int(np.prod([s.exta[m] for m in s.conta], dtype=np.int64)) if s.conta else 1
    return 2.0 * int(np.prod(s.extc(), dtype=np.int64)) * K


class DeviceBuffers:
    """Device buffers for a list of problems (values from each problem's seed
    when `values`, zeros otherwise: run times do not depend on values)."""

    def __init__(self, probs, values=False):
        import torch
        self.keep = []
        self.descs = []
        for pr in probs:
            bf = pr["dtype"] == "bf16"
            if values:
                rng = np.random.default_rng(pr["seed"])
                A = synth.fill(pr["la"], rng.uniform(-1, 1, pr["la"].numel), np.float32, 0.0)
                B = synth.fill(pr["lb"], rng.uniform(-1, 1, pr["lb"].numel), np.float32, 0.0)
                C = synth.fill(pr["lc"], rng.uniform(-1, 1, pr["lc"].numel), np.float32, 0.0)
                tA = torch.from_numpy(A)
                tB = torch.from_numpy(B)
                if bf:
                    tA = tA.to(torch.bfloat16)
                    tB = tB.to(torch.bfloat16)
                dA, dB, dC = tA.cuda(), tB.cuda(), torch.from_numpy(C).cuda()
            else:
                dt = torch.bfloat16 if bf else torch.float32
                dA = torch.zeros(pr["la"].size, dtype=dt, device="cuda")
                dB = torch.zeros(pr["lb"].size, dtype=dt, device="cuda")
                dC = torch.zeros(pr["lc"].size, dtype=torch.float32, device="cuda")
            self.keep.append((dA, dB, dC))
            d = args_of(pr)
            d.update(dtype=pr["dtype"], A=dA.data_ptr() + pr["la"].off * dA.element_size(),
                     B=dB.data_ptr() + pr["lb"].off * dB.element_size(),
                     C=dC.data_ptr() + pr["lc"].off * 4)
            self.descs.append(d)


def valid_mask(probs):
    """valid[i][c]: configuration c can run problem i (SKINNY needs a free
    class of at most 8 indices, TC bf16 operands)."""
    nc = gb.num_configs()
    return np.array([[gb.config_valid(args_of(pr), c, pr["dtype"]) for c in range(nc)] for pr in probs], dtype=bool)


def measure(probs, reps=3, chunk=1024, log=None):
    """times[i][c]: mean ms of problem i alone with configuration c (NaN
    where c cannot run problem i)."""
    import torch
    nc = gb.num_configs()
    T = np.zeros((len(probs), nc), dtype=np.float64)
    V = valid_mask(probs)
    for s in range(0, len(probs), chunk):
        part = probs[s:s + chunk]
        bufs = DeviceBuffers(part)
        for c in range(nc):
            b = gb.Batch(bufs.descs, select="fixed", config=c)
            T[s:s + len(part), c] = b.profile(reps)
            b.close()
        T[s:s + len(part)][~V[s:s + len(part)]] = np.nan
        del bufs
        torch.cuda.empty_cache()
        if log:
            log(f"measured {min(s + chunk, len(probs))}/{len(probs)}")
    return T


def featurize(probs):
    return np.stack([gb.features(args_of(pr), pr["dtype"]) for pr in probs]).astype(np.float32)


def train(X, T, hidden=128, epochs=60, batch=256, lr=1e-3, seed=0):
    mean = X.mean(0)
    std = X.std(0)
    std[std == 0] = 1.0
    Xn = (X - mean) / std
    valid = np.isfinite(T)
    Y = np.log(np.maximum(np.where(valid, T, 1.0), 1e-6))
    mu, sd = Y[valid].mean(), Y[valid].std() if Y[valid].std() > 0 else 1.0
    Yn = np.where(valid, (Y - mu) / sd, 0.0).astype(np.float32)
    M = valid.astype(np.float32)  # masked loss: configurations that cannot run a problem teach nothing
    net = gb.MLP(X.shape[1], hidden, T.shape[1], seed=seed)
    loss = net.fit(Xn.astype(np.float32), Yn, M, epochs=epochs, batch=batch, lr=lr, seed=seed + 1)
    return dict(params=net.get_params(), mean=mean.astype(np.float32), std=std.astype(np.float32),
                hidden=hidden, nout=T.shape[1], final_loss=loss, y_mean=mu, y_std=sd)


def predict_configs(model, X, valid=None):
    """The network's choice: argmin of the predicted times over the valid
    configurations; `finite` is False where a prediction is not finite."""
    net = gb.MLP(X.shape[1], model["hidden"], model["nout"], seed=0)
    net.set_params(model["params"])
    Y = net.predict(((X - model["mean"]) / model["std"]).astype(np.float32))
    finite = np.all(np.isfinite(Y), axis=1)
    if valid is not None:
        Y = np.where(valid, Y, np.inf)
    return np.argmin(Y, axis=1), finite


def regret(choice, T):
    best = np.nanmin(T, axis=1)
    r = T[np.arange(len(T)), choice] / best
    return {"geomean_regret": float(np.exp(np.mean(np.log(r))) - 1.0),
            "share_above_10pct": float(np.mean(r > 1.10)),
            "mean_ratio": float(np.mean(r))}


def save_model(path, model):
    np.savez(path, **{k: np.asarray(v) for k, v in model.items()})


def load_model(path):
    z = np.load(path)
    m = {k: z[k] for k in z.files}
    m["hidden"] = int(m["hidden"])
    m["nout"] = int(m["nout"])
    return m


def install(model):
    gb.install_model(model["params"], model["mean"], model["std"], model["hidden"], model["nout"])


def record_batch_db(probs, T):
    """Tuning-database entries (kind GETT_TUNE_BATCH) of the exhaustive best
    configuration of every measured problem."""
    from . import gett
    best = np.nanargmin(T, axis=1)
    for pr, c in zip(probs, best):
        gett.tune_db_put(gett.TUNE_BATCH, pr["dtype"], args_of(pr), int(c))


def single_candidates(plan):
    """Single-call configurations worth timing for a planned problem: every
    dense tile configuration with split-K 1, 2, 4, 8, 16 (bounded by K), and
    the streaming families the shape allows.  (family, config, split_k)."""
    M, N, K = plan["M"], plan["N"], plan["K"]
    out = [("dense", cfg, sk) for cfg in range(3) for sk in (1, 2, 4, 8, 16) if sk == 1 or K // sk >= 64]
    if K <= 8:
        out.append(("outer", 0, 1))
    if min(M, N) <= 8:
        out.append(("skinny", 0, 1))
    if M * N <= 4096:
        out.append(("reduce", 0, 1))
    return out


def tune_single(prefix, p, reps=5, record=True):
    """Times every candidate configuration of one single call (xgett_ex with
    the configuration forced, CUDA events, best of `reps` after a warm-up, C
    accumulating in a scratch copy) and records the fastest in the tuning
    database (kind GETT_TUNE_SINGLE).  Returns {candidate: ms} and the best."""
    import torch
    from . import gett
    a = p.args()
    st, plan = gett.plan_describe(a["RANKA"], a["EXTA"], a["INCA"], a["RANKB"], a["EXTB"], a["INCB"], a["CONTS"],
                                  a["CONTA"], a["CONTB"], a["PERM"], a["INCC"])
    gett.check(st)
    dA, dB = torch.from_numpy(p.A).cuda(), torch.from_numpy(p.B).cuda()
    dC = torch.zeros(p.lc.size, dtype=torch.float64, device="cuda") if p.meta.get("c_zero") \
        else torch.from_numpy(p.C).cuda()
    stream = torch.cuda.current_stream()
    times = {}
    for fam, cfg, sk in single_candidates(plan):
        opts = gett.options(family=fam, config=cfg, split_k=sk)

        def call():
            return gett.xgett(prefix, a["RANKA"], a["EXTA"], a["INCA"], dA, a["RANKB"], a["EXTB"], a["INCB"], dB,
                              a["CONTS"], a["CONTA"], a["CONTB"], a["PERM"], a["INCC"], dC, a_off=p.la.off,
                              b_off=p.lb.off, c_off=p.lc.off, mode="ex", opts=opts, stream=stream.cuda_stream,
                              raise_on_error=False)[0]
        if call() != gett.GETT_OK:
            continue
        best = float("inf")
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            call()
            e1.record(stream)
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1))
        times[(fam, cfg, sk)] = best
    fam, cfg, sk = min(times, key=times.get)
    if record:
        gett.tune_db_put(gett.TUNE_SINGLE, prefix, dict(EXTA=a["EXTA"], INCA=a["INCA"], EXTB=a["EXTB"],
                                                        INCB=a["INCB"], CONTA=a["CONTA"], CONTB=a["CONTB"],
                                                        PERM=a["PERM"], INCC=a["INCC"]),
                         gett.FAMILY[fam], cfg, sk)
    return times, (fam, cfg, sk)


def throughput(probs, select, configs=None, reps=10, serial=False):
    """Contractions/s and TFLOP/s of one batched launch (graph replay; the
    method chains as concurrent branches unless serial)."""
    import torch
    bufs = DeviceBuffers(probs)
    b = gb.Batch(bufs.descs, select=select, configs=configs, serial=serial)
    info = b.info()
    stream = torch.cuda.current_stream()
    for _ in range(3):
        b.launch(stream=stream.cuda_stream, graph=True)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        b.launch(stream=stream.cuda_stream, graph=True)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    b.close()
    del bufs
    return {"ms": ms, "contractions_per_s": len(probs) / (ms * 1e-3),
            "tflops": info["flops"] / (ms * 1e-3) / 1e12, "fallbacks": info["fallbacks"],
            "config_count": info["config_count"][:gb.num_configs()]}


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--train", type=int, default=20000)
    ap.add_argument("--test", type=int, default=2000)
    ap.add_argument("--max-ext", type=int, default=256)
    ap.add_argument("--epochs", type=int, default=60)
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--model", default=None)
    ap.add_argument("--report", default=None)
    ap.add_argument("--db", default=None, help="write the tuning database (exhaustive best of every measured "
                                               "problem, and the single-call workloads with --single)")
    ap.add_argument("--single", action="store_true",
                    help="tune the single-call workloads (CC, its permuted / row-major-A variant, the small "
                         "DGETT, the stream case) into the database and stop")
    args = ap.parse_args(argv)
    if args.single:
        from . import gett
        rep = {}
        for name, p in (("cc", synth.cfg_cc("plain")), ("cc_perm_transA", synth.cfg_cc("perm_transA")),
                        ("small", synth.cfg_small_dgett()), ("stream", synth.cfg_stream(c_host=False))):
            times, best = tune_single("d", p)
            rep[name] = {"best": list(best), "ms": {f"{f}/{c}/{k}": t for (f, c, k), t in times.items()}}
            print(f"{name}: {best} {times[best]:.3f} ms", file=sys.stderr, flush=True)
        if args.db:
            gett.tune_db_save(args.db)
        print(json.dumps(rep))
        return 0
    import torch
    t0 = time.time()
    log = lambda m: print(f"[{time.time() - t0:7.1f}s] {m}", file=sys.stderr, flush=True)
    tr = draw_problems(args.train, 11, args.max_ext)
    te = draw_problems(args.test, 12, args.max_ext)
    log("signatures drawn")
    Ttr = measure(tr, args.reps, log=log)
    Tte = measure(te, args.reps, log=log)
    Xtr, Xte = featurize(tr), featurize(te)
    log("features done")
    model = train(Xtr, Ttr, epochs=args.epochs)
    log(f"trained, final loss {model['final_loss']:.4f}")
    pred, finite = predict_configs(model, Xte, np.isfinite(Tte))
    heur = np.array([gb.heuristic_config(args_of(pr), pr["dtype"]) for pr in te])
    tuned = np.nanargmin(Tte, axis=1)
    pred_used = np.where(finite, pred, heur)
    rep = {
        "train": args.train, "test": args.test, "max_ext": args.max_ext, "epochs": args.epochs,
        "configs": gb.num_configs(), "final_train_loss": model["final_loss"],
        "learned": regret(pred_used, Tte), "heuristic": regret(heur, Tte),
        "fallback_rate": float(np.mean(~finite)),
        "learned_matches_best": float(np.mean(pred_used == tuned)),
    }
    install(model)
    rep["throughput_learned"] = throughput(te, "learned")
    rep["throughput_heuristic"] = throughput(te, "heuristic")
    rep["throughput_tuned"] = throughput(te, "table", configs=list(tuned))
    if args.db:
        from . import gett
        record_batch_db(tr + te, np.concatenate([Ttr, Tte]))
        gett.tune_db_save(args.db)
        rep["db_entries"] = gett.tune_db_size()
    rep["elapsed_s"] = time.time() - t0
    log(json.dumps(rep))
    if args.model:
        save_model(args.model, model)
    if args.report:
        with open(args.report, "w") as f:
            json.dump(rep, f, indent=1)
    print(json.dumps(rep))
    return 0


if __name__ == "__main__":
    sys.exit(main())
