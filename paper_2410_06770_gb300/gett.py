"""ctypes binding of libgett.so: the xGETT C ABI with the same names.

Argument marshalling only -- every step of a contraction runs inside the CUDA
library.  Pointers are device addresses (ints); torch tensors may be passed
instead, in which case `data_ptr()` of the tensor plus `off` elements is used.
If the library is missing the import-time loader raises: there is no CPU
fallback.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libgett.so")

GETT_OK, GETT_ERR_ARG, GETT_ERR_ALIAS, GETT_ERR_UNSUPPORTED = 0, -1, -2, -3
GETT_ERR_CUDA, GETT_ERR_TIMEOUT, GETT_ERR_NOMEM = -4, -5, -6
GETT_CONJ_A, GETT_CONJ_B = 1, 2
MAX_MODES = 24

ALGO = {"default": 0, "native": 1, "ozaki_bf16": 2, "bf16x3": 3, "bf16x6": 4}
FAMILY = {"auto": 0, "noop": 1, "dense": 2, "outer": 3, "reduce": 4, "skinny": 5, "tc": 6}
FAMILY_NAME = {v: k for k, v in FAMILY.items()}
PREFIXES = ("s", "d", "c", "z", "sb")


class GettError(RuntimeError):
    def __init__(self, status: int, msg: str, arg: int = 0, cuda: int = 0):
        super().__init__(f"{msg} (status {status}, arg {arg}, cudaError {cuda})")
        self.status = status
        self.arg = arg
        self.cuda = cuda


class Options(ctypes.Structure):
    _fields_ = [("algo", ctypes.c_int), ("family", ctypes.c_int), ("config", ctypes.c_int),
                ("split_k", ctypes.c_int), ("moduli", ctypes.c_int), ("conj", ctypes.c_int),
                ("reserved", ctypes.c_int * 2)]


class Report(ctypes.Structure):
    _fields_ = [("family", ctypes.c_int), ("config", ctypes.c_int), ("split_k", ctypes.c_int),
                ("moduli", ctypes.c_int), ("nm", ctypes.c_int), ("nn", ctypes.c_int),
                ("nk", ctypes.c_int), ("selector", ctypes.c_int), ("M", ctypes.c_int64),
                ("N", ctypes.c_int64), ("K", ctypes.c_int64), ("flops", ctypes.c_double),
                ("time_ms", ctypes.c_double)]

    def as_dict(self):
        d = {f: getattr(self, f) for f, _ in self._fields_}
        d["family_name"] = FAMILY_NAME.get(self.family, str(self.family))
        return d


_M = MAX_MODES


class PlanInfo(ctypes.Structure):
    _fields_ = [("nm", ctypes.c_int), ("nn", ctypes.c_int), ("nk", ctypes.c_int),
                ("empty", ctypes.c_int), ("M", ctypes.c_int64), ("N", ctypes.c_int64),
                ("K", ctypes.c_int64),
                ("m_ext", ctypes.c_int64 * _M), ("m_inca", ctypes.c_int64 * _M), ("m_incc", ctypes.c_int64 * _M),
                ("n_ext", ctypes.c_int64 * _M), ("n_incb", ctypes.c_int64 * _M), ("n_incc", ctypes.c_int64 * _M),
                ("k_ext", ctypes.c_int64 * _M), ("k_inca", ctypes.c_int64 * _M), ("k_incb", ctypes.c_int64 * _M),
                ("off_a", ctypes.c_int64), ("off_b", ctypes.c_int64), ("off_c", ctypes.c_int64)]

    def as_dict(self):
        def lst(arr, n):
            return [int(arr[i]) for i in range(n)]
        return dict(nm=self.nm, nn=self.nn, nk=self.nk, empty=bool(self.empty), M=self.M, N=self.N,
                    K=self.K, m=list(zip(lst(self.m_ext, self.nm), lst(self.m_inca, self.nm), lst(self.m_incc, self.nm))),
                    n=list(zip(lst(self.n_ext, self.nn), lst(self.n_incb, self.nn), lst(self.n_incc, self.nn))),
                    k=list(zip(lst(self.k_ext, self.nk), lst(self.k_inca, self.nk), lst(self.k_incb, self.nk))),
                    off_a=self.off_a, off_b=self.off_b, off_c=self.off_c)


_lib = None
_i64p = ctypes.POINTER(ctypes.c_int64)
_ip = ctypes.POINTER(ctypes.c_int)
_vp = ctypes.c_void_p
_ARGS14 = [ctypes.c_int, _i64p, _i64p, _vp, ctypes.c_int, _i64p, _i64p, _vp,
           ctypes.c_int, _ip, _ip, _ip, _i64p, _vp]


def lib():
    """Load libgett.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2410_06770_gb300.build.build() "
                           "(there is no CPU fallback)")
    L = ctypes.CDLL(LIB_PATH)
    for p in PREFIXES:
        getattr(L, p + "gett").argtypes = _ARGS14
        getattr(L, p + "gett").restype = ctypes.c_int
        getattr(L, p + "gett_async").argtypes = _ARGS14 + [_vp]
        getattr(L, p + "gett_async").restype = ctypes.c_int
        getattr(L, p + "gett_ex").argtypes = _ARGS14 + [ctypes.POINTER(Options), ctypes.POINTER(Report), _vp]
        getattr(L, p + "gett_ex").restype = ctypes.c_int
        getattr(L, p + "gett_scaled").argtypes = _ARGS14 + [_vp, _vp, ctypes.POINTER(Options),
                                                            ctypes.POINTER(Report), _vp]
        getattr(L, p + "gett_scaled").restype = ctypes.c_int
        getattr(L, p + "getp").argtypes = [ctypes.c_int, _i64p, _i64p, _vp, _ip, _i64p, _vp, _vp, _vp, _vp]
        getattr(L, p + "getp").restype = ctypes.c_int
        getattr(L, p + "getr").argtypes = [ctypes.c_int, _i64p, _i64p, _vp, ctypes.c_int, _ip, _ip, _i64p, _vp,
                                           _vp, _vp, _vp]
        getattr(L, p + "getr").restype = ctypes.c_int
    L.gett_plan_describe.argtypes = [ctypes.c_int, _i64p, _i64p, ctypes.c_int, _i64p, _i64p,
                                     ctypes.c_int, _ip, _ip, _ip, _i64p, ctypes.POINTER(PlanInfo)]
    L.gett_plan_describe.restype = ctypes.c_int
    L.gett_last_error_arg.restype = ctypes.c_int
    L.gett_last_cuda_error.restype = ctypes.c_int
    L.gett_status_string.argtypes = [ctypes.c_int]
    L.gett_status_string.restype = ctypes.c_char_p
    L.gett_device_status.restype = ctypes.c_int
    L.gett_version.restype = ctypes.c_int
    L.gett_ozaki_params.argtypes = [ctypes.c_int64, ctypes.c_int, _ip, _ip, _ip]
    L.gett_ozaki_params.restype = ctypes.c_int
    L.gett_options_init.argtypes = [ctypes.POINTER(Options)]
    L.gett_options_init.restype = None
    L.gett_tune_db_put.argtypes = [ctypes.c_int, ctypes.c_int] + _ARGS14[:3] + _ARGS14[4:7] + \
        [ctypes.c_int, _ip, _ip, _ip, _i64p, ctypes.c_int, ctypes.c_int, ctypes.c_int]
    L.gett_tune_db_put.restype = ctypes.c_int
    L.gett_tune_db_get.argtypes = [ctypes.c_int, ctypes.c_int] + _ARGS14[:3] + _ARGS14[4:7] + \
        [ctypes.c_int, _ip, _ip, _ip, _i64p, _ip, _ip, _ip]
    L.gett_tune_db_get.restype = ctypes.c_int
    for n in ("gett_tune_db_clear", "gett_tune_db_size"):
        getattr(L, n).restype = ctypes.c_int
    for n in ("gett_tune_db_save", "gett_tune_db_load"):
        getattr(L, n).argtypes = [ctypes.c_char_p]
        getattr(L, n).restype = ctypes.c_int
    _lib = L
    return L


def _i64(xs: Sequence[int]):
    if xs is None or len(xs) == 0:
        return None
    return (ctypes.c_int64 * len(xs))(*[int(x) for x in xs])


def _i32(xs: Sequence[int]):
    if xs is None or len(xs) == 0:
        return None
    return (ctypes.c_int * len(xs))(*[int(x) for x in xs])


def _ptr(x, off: int = 0, itemsize: int = 0):
    if x is None:
        return None
    if isinstance(x, int):
        return ctypes.c_void_p(x + off * itemsize) if x else None
    # torch tensor
    return ctypes.c_void_p(x.data_ptr() + off * x.element_size())


def check(status: int):
    if status != GETT_OK:
        L = lib()
        raise GettError(status, L.gett_status_string(status).decode(), L.gett_last_error_arg(),
                        L.gett_last_cuda_error())
    return status


def options(algo="default", family="auto", config=-1, split_k=0, moduli=0, conj=0) -> Options:
    """gett_options; conj is a GETT_CONJ_A | GETT_CONJ_B mask (complex types)."""
    o = Options()
    lib().gett_options_init(ctypes.byref(o))
    o.algo = ALGO[algo] if isinstance(algo, str) else int(algo)
    o.family = FAMILY[family] if isinstance(family, str) else int(family)
    o.config = int(config)
    o.split_k = int(split_k)
    o.moduli = int(moduli)
    o.conj = int(conj)
    return o


def _scalar(prefix: str, x):
    """A host scalar of C's element type for the scaled entry points (kept
    alive by the caller); None passes NULL."""
    if x is None:
        return None
    if prefix in ("s", "sb"):
        return ctypes.c_float(float(x))
    if prefix == "d":
        return ctypes.c_double(float(x))
    z = complex(x)
    t = ctypes.c_float if prefix == "c" else ctypes.c_double
    return (t * 2)(z.real, z.imag)


def xgett(prefix: str, RANKA, EXTA, INCA, A, RANKB, EXTB, INCB, B, CONTS, CONTA, CONTB, PERM, INCC, C,
          *, a_off=0, b_off=0, c_off=0, stream=None, mode="sync", opts: Optional[Options] = None,
          alpha=1.0, beta=1.0, raise_on_error=True):
    """Call {prefix}gett / _async / _ex / _scaled (mode "scaled": C <- alpha
    A.B + beta C).  Returns (status, report dict or None)."""
    L = lib()
    args = [int(RANKA), _i64(EXTA), _i64(INCA), _ptr(A, a_off), int(RANKB), _i64(EXTB), _i64(INCB),
            _ptr(B, b_off), int(CONTS), _i32(CONTA), _i32(CONTB), _i32(PERM), _i64(INCC), _ptr(C, c_off)]
    rep = None
    if mode == "sync":
        st = getattr(L, prefix + "gett")(*args)
    elif mode == "async":
        st = getattr(L, prefix + "gett_async")(*args, ctypes.c_void_p(int(stream or 0)))
    elif mode == "ex":
        rep = Report()
        o = opts if opts is not None else options()
        st = getattr(L, prefix + "gett_ex")(*args, ctypes.byref(o), ctypes.byref(rep),
                                            ctypes.c_void_p(int(stream or 0)))
    elif mode == "scaled":
        rep = Report()
        o = opts if opts is not None else options()
        al, be = _scalar(prefix, alpha), _scalar(prefix, beta)
        st = getattr(L, prefix + "gett_scaled")(*args, ctypes.byref(al) if al is not None else None,
                                                ctypes.byref(be) if be is not None else None,
                                                ctypes.byref(o), ctypes.byref(rep), ctypes.c_void_p(int(stream or 0)))
    else:
        raise ValueError(mode)
    if raise_on_error:
        check(st)
    return st, (rep.as_dict() if rep is not None else None)


def plan_describe(RANKA, EXTA, INCA, RANKB, EXTB, INCB, CONTS, CONTA, CONTB, PERM, INCC):
    """Host-only planner output (no device work).  Returns (status, dict)."""
    L = lib()
    info = PlanInfo()
    st = L.gett_plan_describe(int(RANKA), _i64(EXTA), _i64(INCA), int(RANKB), _i64(EXTB), _i64(INCB),
                              int(CONTS), _i32(CONTA), _i32(CONTB), _i32(PERM), _i64(INCC),
                              ctypes.byref(info))
    return st, (info.as_dict() if st == GETT_OK else None)


def ozaki_params(K: int, moduli: int = 0):
    """gett_ozaki_params: (count, bits a operand, moduli) of the split form
    for K summed terms.  Host only."""
    L = lib()
    n, bits = ctypes.c_int(0), ctypes.c_int(0)
    mods = (ctypes.c_int * 20)()
    check(L.gett_ozaki_params(int(K), int(moduli), ctypes.byref(n), ctypes.byref(bits), mods))
    return n.value, bits.value, list(mods[: n.value])


# ---------------------------------------------------------------------------
# tuning database (gett_tune.h)
# ---------------------------------------------------------------------------
TUNE_BATCH, TUNE_SINGLE = 0, 1
TUNE_DTYPE = {"s": 0, "d": 1, "c": 2, "z": 3, "sb": 4, "f32": 0, "bf16": 1}


def _idx11(a: dict):
    return [int(len(a["EXTA"])), _i64(a["EXTA"]), _i64(a["INCA"]), int(len(a["EXTB"])), _i64(a["EXTB"]),
            _i64(a["INCB"]), int(len(a["CONTA"])), _i32(a["CONTA"]), _i32(a["CONTB"]), _i32(a["PERM"]),
            _i64(a["INCC"])]


def tune_db_put(kind: int, dtype, args: dict, v0: int, v1: int = 0, v2: int = 0) -> int:
    """Record a tuned configuration for a problem (args: EXTA, INCA, EXTB,
    INCB, CONTA, CONTB, PERM, INCC).  dtype: a TUNE_DTYPE key or its code."""
    dt = TUNE_DTYPE[dtype] if isinstance(dtype, str) else int(dtype)
    return check(lib().gett_tune_db_put(int(kind), dt, *_idx11(args), int(v0), int(v1), int(v2)))


def tune_db_get(kind: int, dtype, args: dict):
    """(v0, v1, v2) of the problem's entry, or None."""
    dt = TUNE_DTYPE[dtype] if isinstance(dtype, str) else int(dtype)
    v = [ctypes.c_int(0) for _ in range(3)]
    st = lib().gett_tune_db_get(int(kind), dt, *_idx11(args), *[ctypes.byref(x) for x in v])
    if st < 0:
        check(st)
    return tuple(x.value for x in v) if st == 1 else None


def tune_db_clear():
    lib().gett_tune_db_clear()


def tune_db_size() -> int:
    return lib().gett_tune_db_size()


def tune_db_save(path: str):
    check(lib().gett_tune_db_save(path.encode()))


def tune_db_load(path: str):
    check(lib().gett_tune_db_load(path.encode()))


def last_error_arg() -> int:
    return lib().gett_last_error_arg()


def device_status() -> int:
    return lib().gett_device_status()


def getp(prefix: str, RANKA, EXTA, INCA, A, PERM, INCC, C, *, alpha=1.0, beta=0.0, a_off=0, c_off=0,
         stream=None, raise_on_error=True) -> int:
    """{prefix}getp: C[o placed by PERM] <- alpha A[o] + beta C (transpose)."""
    L = lib()
    al, be = _scalar(prefix, alpha), _scalar(prefix, beta)
    st = getattr(L, prefix + "getp")(int(RANKA), _i64(EXTA), _i64(INCA), _ptr(A, a_off), _i32(PERM), _i64(INCC),
                                     _ptr(C, c_off), ctypes.byref(al) if al is not None else None,
                                     ctypes.byref(be) if be is not None else None, ctypes.c_void_p(int(stream or 0)))
    if raise_on_error:
        check(st)
    return st


def getr(prefix: str, RANKA, EXTA, INCA, A, NRED, RED, PERM, INCC, C, *, alpha=1.0, beta=0.0, a_off=0, c_off=0,
         stream=None, raise_on_error=True) -> int:
    """{prefix}getr: C[free modes placed by PERM] <- alpha sum_{RED} A + beta C (reduction)."""
    L = lib()
    al, be = _scalar(prefix, alpha), _scalar(prefix, beta)
    st = getattr(L, prefix + "getr")(int(RANKA), _i64(EXTA), _i64(INCA), _ptr(A, a_off), int(NRED), _i32(RED),
                                     _i32(PERM), _i64(INCC), _ptr(C, c_off),
                                     ctypes.byref(al) if al is not None else None,
                                     ctypes.byref(be) if be is not None else None, ctypes.c_void_p(int(stream or 0)))
    if raise_on_error:
        check(st)
    return st
