"""CPU oracle for xGETT -- TEST INFRASTRUCTURE ONLY.

Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline / reference
legs may import this package.  The CUDA library never calls it; the two share
no code.

`gett_raw()` (and `gett_problem()` on a synth.Problem) runs Alg. 1 of the
thesis (Sec. 6) in plain C (gett_oracle.c) on numpy buffers.  Precisions:
  'f64'    -- products and sums in double, each product added to C in turn
              (exactly the loop of Alg. 1);
  'ld'     -- the same loop accumulated in long double, rounded once;
  'z'      -- complex double, no conjugation;
  'direct' -- second, independent implementation (flat-index decode, no
              odometer) in double, for brute-force cross-checks.
`gett_scaled()` is the scaled form C <- alpha * S + beta * C (the ALPHA and
BETA of xGEMM, Sec. 2.3.1): S is Alg. 1 run on a zeroed C, combined with the
original C element by element in double (complex double for c/z).
Float32 and bfloat16 inputs are widened exactly to double before the call, so
the oracle of every precision form is the fp64 (or long double) contraction of
the exact input values.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gett_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile gett_oracle.c with gcc (-O2, no FMA contraction, OpenMP)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
           "-fPIC", "-shared", "-o", tmp, _SRC]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i64p = ctypes.POINTER(ctypes.c_int64)
            ip = ctypes.POINTER(ctypes.c_int)
            vp = ctypes.c_void_p
            sig = [ctypes.c_int, i64p, i64p, vp, ctypes.c_int, i64p, i64p, vp,
                   ctypes.c_int, ip, ip, ip, i64p, vp]
            for name in ("oracle_dgett", "oracle_dgett_ld", "oracle_zgett"):
                fn = getattr(lib, name)
                fn.argtypes = sig + [ctypes.c_int]
                fn.restype = ctypes.c_int
            lib.oracle_dgett_direct.argtypes = sig
            lib.oracle_dgett_direct.restype = ctypes.c_int
            lib.oracle_inc_coords.argtypes = [ctypes.c_int, i64p, i64p]
            lib.oracle_inc_coords.restype = None
            lib.oracle_long_double_mant_dig.restype = ctypes.c_int
            _lib = lib
    return _lib


def _i64(xs):
    arr = (ctypes.c_int64 * max(len(xs), 1))(*[int(x) for x in xs])
    return arr


def _i32(xs):
    return (ctypes.c_int * max(len(xs), 1))(*[int(x) for x in xs])


def _ptr(buf: np.ndarray, off: int, itemsize: int):
    return ctypes.c_void_p(buf.ctypes.data + off * itemsize)


def gett_raw(precision, RANKA, EXTA, INCA, A, a_off, RANKB, EXTB, INCB, B, b_off,
             CONTS, CONTA, CONTB, PERM, INCC, C, c_off, nthreads=1) -> int:
    """Call the oracle on numpy buffers; pointers are buffer base + offset.

    A, B and C must be contiguous 1-D arrays of float64 (precision f64, ld,
    direct) or complex128 (precision z).  C is updated in place."""
    lib = _load()
    want = np.complex128 if precision == "z" else np.float64
    for name, buf in (("A", A), ("B", B), ("C", C)):
        if buf.dtype != want or not buf.flags.c_contiguous:
            raise TypeError(f"{name} must be a contiguous {np.dtype(want).name} array")
    isz = np.dtype(want).itemsize
    args = [int(RANKA), _i64(EXTA), _i64(INCA), _ptr(A, a_off, isz),
            int(RANKB), _i64(EXTB), _i64(INCB), _ptr(B, b_off, isz),
            int(CONTS), _i32(CONTA), _i32(CONTB), _i32(PERM), _i64(INCC), _ptr(C, c_off, isz)]
    if precision == "f64":
        return lib.oracle_dgett(*args, int(nthreads))
    if precision == "ld":
        return lib.oracle_dgett_ld(*args, int(nthreads))
    if precision == "z":
        return lib.oracle_zgett(*args, int(nthreads))
    if precision == "direct":
        return lib.oracle_dgett_direct(*args)
    raise ValueError(precision)


def widen(buf: np.ndarray) -> np.ndarray:
    """Exact widening of any supported input buffer to float64/complex128.
    bfloat16 buffers are given as uint16 bit patterns."""
    if buf.dtype == np.uint16:  # bfloat16 bits -> float32 (exact) -> float64
        return (buf.astype(np.uint32) << 16).view(np.float32).astype(np.float64)
    if buf.dtype.kind == "c":
        return np.ascontiguousarray(buf, dtype=np.complex128)
    return np.ascontiguousarray(buf, dtype=np.float64)


def gett_problem(p, precision="f64", nthreads=1, C=None) -> np.ndarray:
    """Run the oracle on a synth.Problem; returns the updated (widened) C buffer.

    `C` optionally overrides the initial C buffer (already widened)."""
    A = widen(p.A)
    B = widen(p.B)
    Cw = widen(p.C).copy() if C is None else C
    if precision == "f64" and A.dtype.kind == "c":
        precision = "z"
    a = p.args()
    rc = gett_raw(precision, a["RANKA"], a["EXTA"], a["INCA"], A, p.la.off,
                  a["RANKB"], a["EXTB"], a["INCB"], B, p.lb.off,
                  a["CONTS"], a["CONTA"], a["CONTB"], a["PERM"], a["INCC"], Cw, p.lc.off,
                  nthreads=nthreads)
    if rc != 0:
        raise ValueError(f"oracle rejected the problem (code {rc})")
    return Cw


def output_positions(extc, incc, off) -> np.ndarray:
    """Buffer positions of every logical output element (first mode fastest):
    off + sum_q o_q INCC[q]."""
    pos = np.array([int(off)], dtype=np.int64)
    for e, inc in zip(extc, incc):
        # each later mode is slower than the ones already in pos
        pos = (pos[None, :] + np.arange(int(e), dtype=np.int64)[:, None] * int(inc)).reshape(-1)
    return pos


def gett_scaled(p, alpha, beta, precision="f64", nthreads=1) -> np.ndarray:
    """The scaled form C <- alpha * S + beta * C, S the contraction's sum over
    the contracted indices (xGEMM's ALPHA and BETA, Sec. 2.3.1; the sum itself
    is Alg. 1 run on a zeroed C, so it starts from 0).  beta == 0 does not read
    C (NaN there does not propagate); alpha == 0 does not form S.  Returns the
    updated (widened) C buffer; elements outside the output layout keep their
    values."""
    C0 = widen(p.C).copy()
    a = p.args()
    pos = output_positions(p.sig.extc(), a["INCC"], p.lc.off)
    out = C0.copy()
    alpha = complex(alpha) if C0.dtype.kind == "c" else float(np.real(alpha))
    beta = complex(beta) if C0.dtype.kind == "c" else float(np.real(beta))
    if alpha != 0:
        Z = C0.copy()
        Z[pos] = 0
        S = gett_problem(p, precision, nthreads, C=Z)[pos]
        out[pos] = alpha * S if beta == 0 else alpha * S + beta * C0[pos]
    else:
        out[pos] = 0 if beta == 0 else beta * C0[pos]
    return out


def inc_coords(coords, exts):
    """Alg. 2 on a coordinate list; returns the incremented coordinates."""
    lib = _load()
    c = _i64(coords)
    e = _i64(exts)
    lib.oracle_inc_coords(len(coords), c, e)
    return [c[i] for i in range(len(coords))]


def long_double_bits() -> int:
    """Significand bits of the host's long double (64 on x86_64, 113 on aarch64)."""
    return _load().oracle_long_double_mant_dig()
