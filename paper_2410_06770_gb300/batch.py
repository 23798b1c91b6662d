"""ctypes binding of the batched launch (gett_batch.h) and of the
learned planner's network (gett_learn.h).  Argument marshalling only."""
from __future__ import annotations

import ctypes
from typing import Sequence

import numpy as np

from . import gett

NFEAT = 24
_i64p = ctypes.POINTER(ctypes.c_int64)
_ip = ctypes.POINTER(ctypes.c_int)
_fp = ctypes.POINTER(ctypes.c_float)

SELECT = {"heuristic": 0, "fixed": 1, "table": 2, "learned": 3, "tuned": 4}


class ProblemDesc(ctypes.Structure):
    _fields_ = [("dtype", ctypes.c_int), ("RANKA", ctypes.c_int), ("EXTA", _i64p), ("INCA", _i64p),
                ("A", ctypes.c_void_p), ("RANKB", ctypes.c_int), ("EXTB", _i64p), ("INCB", _i64p),
                ("B", ctypes.c_void_p), ("CONTS", ctypes.c_int), ("CONTA", _ip), ("CONTB", _ip),
                ("PERM", _ip), ("INCC", _i64p), ("C", ctypes.c_void_p)]


class BatchOptions(ctypes.Structure):
    _fields_ = [("select", ctypes.c_int), ("config", ctypes.c_int), ("configs", _ip),
                ("ctas_per_sm", ctypes.c_int), ("serial", ctypes.c_int)]


MAX_CONFIGS = 16


class BatchInfo(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("nonempty", ctypes.c_int), ("tiles", ctypes.c_int64),
                ("flops", ctypes.c_double), ("config_count", ctypes.c_int * MAX_CONFIGS),
                ("fallbacks", ctypes.c_int), ("gather_items", ctypes.c_int64), ("packed_items", ctypes.c_int64),
                ("pack_items", ctypes.c_int64), ("skinny_items", ctypes.c_int64), ("tuned_hits", ctypes.c_int),
                ("tc_items", ctypes.c_int64), ("tc_pack_items", ctypes.c_int64)]


_bound = False


def _bind():
    global _bound
    L = gett.lib()
    if _bound:
        return L
    L.gett_batch_create.argtypes = [ctypes.c_int, ctypes.POINTER(ProblemDesc), ctypes.POINTER(BatchOptions),
                                    ctypes.POINTER(ctypes.c_void_p), _ip]
    L.gett_batch_create.restype = ctypes.c_int
    for n in ("gett_batch_launch", "gett_batch_launch_graph"):
        getattr(L, n).argtypes = [ctypes.c_void_p, ctypes.c_void_p]
        getattr(L, n).restype = ctypes.c_int
    L.gett_batch_get_info.argtypes = [ctypes.c_void_p, ctypes.POINTER(BatchInfo)]
    L.gett_batch_destroy.argtypes = [ctypes.c_void_p]
    L.gett_batch_profile.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, _fp]
    L.gett_batch_profile.restype = ctypes.c_int
    L.gett_batch_num_configs.restype = ctypes.c_int
    L.gett_batch_heuristic_config.argtypes = [ctypes.c_int, _i64p, _i64p, ctypes.c_int, _i64p, _i64p,
                                              ctypes.c_int, _ip, _ip, _ip, _i64p, ctypes.c_int, _ip]
    L.gett_batch_config_shape.argtypes = [ctypes.c_int, _ip, _ip]
    L.gett_batch_config_method.argtypes = [ctypes.c_int]
    L.gett_batch_config_method.restype = ctypes.c_int
    L.gett_batch_config_valid.argtypes = [ctypes.c_int, _i64p, _i64p, ctypes.c_int, _i64p, _i64p,
                                          ctypes.c_int, _ip, _ip, _ip, _i64p, ctypes.c_int, ctypes.c_int]
    L.gett_batch_config_valid.restype = ctypes.c_int
    L.gett_problem_features.argtypes = [ctypes.c_int, _i64p, _i64p, ctypes.c_int, _i64p, _i64p,
                                        ctypes.c_int, _ip, _ip, _ip, _i64p, ctypes.c_int, _fp]
    L.gett_mlp_create.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_ulonglong,
                                  ctypes.POINTER(ctypes.c_void_p)]
    L.gett_mlp_destroy.argtypes = [ctypes.c_void_p]
    L.gett_mlp_num_params.argtypes = [ctypes.c_void_p]
    L.gett_mlp_get_params.argtypes = [ctypes.c_void_p, _fp]
    L.gett_mlp_set_params.argtypes = [ctypes.c_void_p, _fp]
    L.gett_mlp_loss_grad.argtypes = [ctypes.c_void_p, _fp, _fp, _fp, ctypes.c_int, _fp, _fp]
    L.gett_mlp_fit.argtypes = [ctypes.c_void_p, _fp, _fp, _fp, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                               ctypes.c_float, ctypes.c_ulonglong, _fp]
    L.gett_mlp_predict.argtypes = [ctypes.c_void_p, _fp, ctypes.c_int, _fp]
    L.gett_learn_install.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, _fp, _fp, _fp]
    L.gett_learn_predict.argtypes = [_fp, _fp]
    _bound = True
    return L


def _f(a: np.ndarray):
    return a.ctypes.data_as(_fp)


class Batch:
    """One planned batch of contractions (float C; float or bf16 A/B)."""

    def __init__(self, problems: Sequence[dict], select="heuristic", config=0, configs=None, ctas_per_sm=0,
                 serial=False):
        L = _bind()
        self._keep = []
        n = len(problems)
        arr = (ProblemDesc * max(n, 1))()
        for i, pr in enumerate(problems):
            d = arr[i]
            d.dtype = 1 if pr["dtype"] in ("bf16", 1) else 0
            for name in ("EXTA", "INCA", "EXTB", "INCB", "INCC"):
                x = gett._i64(pr[name])
                self._keep.append(x)
                setattr(d, name, ctypes.cast(x, _i64p) if x is not None else None)
            for name in ("CONTA", "CONTB", "PERM"):
                x = gett._i32(pr[name])
                self._keep.append(x)
                setattr(d, name, ctypes.cast(x, _ip) if x is not None else None)
            d.RANKA = len(pr["EXTA"])
            d.RANKB = len(pr["EXTB"])
            d.CONTS = len(pr["CONTA"])
            d.A = pr["A"]
            d.B = pr["B"]
            d.C = pr["C"]
        o = BatchOptions()
        o.select = SELECT[select]
        o.config = int(config)
        if configs is not None:
            ca = (ctypes.c_int * max(n, 1))(*[int(c) for c in configs])
            self._keep.append(ca)
            o.configs = ctypes.cast(ca, _ip)
        o.ctas_per_sm = int(ctas_per_sm)
        o.serial = int(serial)  # 0/1 (bool); other values are rejected by the library
        h = ctypes.c_void_p()
        bad = ctypes.c_int(-1)
        st = L.gett_batch_create(n, arr, ctypes.byref(o), ctypes.byref(h), ctypes.byref(bad))
        if st != 0:
            err = gett.GettError(st, f"gett_batch_create failed at problem {bad.value}", L.gett_last_error_arg(),
                                 L.gett_last_cuda_error())
            err.bad_index = bad.value
            raise err
        self.h = h
        self.n = n

    def launch(self, stream=0, graph=False):
        L = _bind()
        fn = L.gett_batch_launch_graph if graph else L.gett_batch_launch
        gett.check(fn(self.h, ctypes.c_void_p(int(stream or 0))))

    def profile(self, reps=3, throughput=True) -> np.ndarray:
        """Mean ms of each problem on its own (0 for empty ones): its cost in
        a full GPU (throughput=True) or its latency alone."""
        out = np.zeros(max(self.n, 1), dtype=np.float32)
        gett.check(_bind().gett_batch_profile(self.h, int(reps), 1 if throughput else 0, _f(out)))
        return out[: self.n]

    def info(self) -> dict:
        L = _bind()
        i = BatchInfo()
        L.gett_batch_get_info(self.h, ctypes.byref(i))
        return {"n": i.n, "nonempty": i.nonempty, "tiles": i.tiles, "flops": i.flops,
                "config_count": list(i.config_count), "fallbacks": i.fallbacks,
                "gather_items": i.gather_items, "packed_items": i.packed_items, "pack_items": i.pack_items,
                "skinny_items": i.skinny_items, "tuned_hits": i.tuned_hits, "tc_items": i.tc_items,
                "tc_pack_items": i.tc_pack_items}

    def close(self):
        if getattr(self, "h", None):
            _bind().gett_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def num_configs() -> int:
    return _bind().gett_batch_num_configs()


def _dtype_code(dtype) -> int:
    return 1 if dtype in ("bf16", 1) else 0


def heuristic_config(args: dict, dtype="f32") -> int:
    L = _bind()
    c = ctypes.c_int(0)
    gett.check(L.gett_batch_heuristic_config(len(args["EXTA"]), gett._i64(args["EXTA"]), gett._i64(args["INCA"]),
                                             len(args["EXTB"]), gett._i64(args["EXTB"]), gett._i64(args["INCB"]),
                                             len(args["CONTA"]), gett._i32(args["CONTA"]), gett._i32(args["CONTB"]),
                                             gett._i32(args["PERM"]), gett._i64(args["INCC"]), _dtype_code(dtype),
                                             ctypes.byref(c)))
    return c.value


def config_method(config: int) -> int:
    """0 GATHER, 1 PACK, 2 SKINNY, 3 TC."""
    return _bind().gett_batch_config_method(int(config))


def config_valid(args: dict, config: int, dtype="f32") -> bool:
    L = _bind()
    st = L.gett_batch_config_valid(len(args["EXTA"]), gett._i64(args["EXTA"]), gett._i64(args["INCA"]),
                                   len(args["EXTB"]), gett._i64(args["EXTB"]), gett._i64(args["INCB"]),
                                   len(args["CONTA"]), gett._i32(args["CONTA"]), gett._i32(args["CONTB"]),
                                   gett._i32(args["PERM"]), gett._i64(args["INCC"]), _dtype_code(dtype), int(config))
    if st < 0:
        gett.check(st)
    return st == 1


def features(args: dict, dtype) -> np.ndarray:
    L = _bind()
    f = np.zeros(NFEAT, dtype=np.float32)
    st = L.gett_problem_features(len(args["EXTA"]), gett._i64(args["EXTA"]), gett._i64(args["INCA"]),
                                 len(args["EXTB"]), gett._i64(args["EXTB"]), gett._i64(args["INCB"]),
                                 len(args["CONTA"]), gett._i32(args["CONTA"]), gett._i32(args["CONTB"]),
                                 gett._i32(args["PERM"]), gett._i64(args["INCC"]),
                                 1 if dtype in ("bf16", 1) else 0, _f(f))
    gett.check(st)
    return f


class MLP:
    """The planner network, trained on the GPU by the library's kernels."""

    def __init__(self, nfeat=NFEAT, hidden=128, nout=4, seed=0):
        L = _bind()
        h = ctypes.c_void_p()
        gett.check(L.gett_mlp_create(nfeat, hidden, nout, seed, ctypes.byref(h)))
        self.h, self.nfeat, self.hidden, self.nout = h, nfeat, hidden, nout

    @property
    def nparams(self) -> int:
        return _bind().gett_mlp_num_params(self.h)

    def get_params(self) -> np.ndarray:
        p = np.zeros(self.nparams, dtype=np.float32)
        gett.check(_bind().gett_mlp_get_params(self.h, _f(p)))
        return p

    def set_params(self, p: np.ndarray):
        p = np.ascontiguousarray(p, dtype=np.float32)
        gett.check(_bind().gett_mlp_set_params(self.h, _f(p)))

    def loss_grad(self, X, Y, M):
        X, Y, M = (np.ascontiguousarray(a, dtype=np.float32) for a in (X, Y, M))
        g = np.zeros(self.nparams, dtype=np.float32)
        loss = np.zeros(1, dtype=np.float32)
        gett.check(_bind().gett_mlp_loss_grad(self.h, _f(X), _f(Y), _f(M), X.shape[0], _f(loss), _f(g)))
        return float(loss[0]), g

    def fit(self, X, Y, M, epochs=50, batch=256, lr=1e-3, seed=0) -> float:
        X, Y, M = (np.ascontiguousarray(a, dtype=np.float32) for a in (X, Y, M))
        loss = np.zeros(1, dtype=np.float32)
        gett.check(_bind().gett_mlp_fit(self.h, _f(X), _f(Y), _f(M), X.shape[0], epochs, batch, lr, seed,
                                        _f(loss)))
        return float(loss[0])

    def predict(self, X) -> np.ndarray:
        X = np.ascontiguousarray(X, dtype=np.float32)
        Y = np.zeros((X.shape[0], self.nout), dtype=np.float32)
        gett.check(_bind().gett_mlp_predict(self.h, _f(X), X.shape[0], _f(Y)))
        return Y

    def close(self):
        if getattr(self, "h", None):
            _bind().gett_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def install_model(params: np.ndarray, mean: np.ndarray, std: np.ndarray, hidden=128, nout=4):
    L = _bind()
    params = np.ascontiguousarray(params, dtype=np.float32)
    mean = np.ascontiguousarray(mean, dtype=np.float32)
    std = np.ascontiguousarray(std, dtype=np.float32)
    gett.check(L.gett_learn_install(NFEAT, hidden, nout, _f(params), _f(mean), _f(std)))


def clear_model():
    _bind().gett_learn_clear()
