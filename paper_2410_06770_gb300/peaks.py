"""Binding of the pipe/HBM microbenchmarks (gett_measure_peaks)."""
import ctypes

from . import gett


class _Peaks(ctypes.Structure):
    _fields_ = [("dfma_tflops", ctypes.c_double), ("dmma_m8n8k4_tflops", ctypes.c_double),
                ("dmma_m16n8k4_tflops", ctypes.c_double), ("dmma_m16n8k8_tflops", ctypes.c_double),
                ("ffma_tflops", ctypes.c_double), ("copy_gbs", ctypes.c_double), ("sms", ctypes.c_int),
                ("imma_s8_tops", ctypes.c_double), ("tc_bf16_tflops", ctypes.c_double),
                ("tc_e4m3_tflops", ctypes.c_double), ("fp64_mixed_tflops", ctypes.c_double)]


def measure(copy_bytes: int = 1 << 30) -> dict:
    L = gett.lib()
    L.gett_measure_peaks.argtypes = [ctypes.POINTER(_Peaks), ctypes.c_size_t]
    L.gett_measure_peaks.restype = ctypes.c_int
    out = _Peaks()
    st = L.gett_measure_peaks(ctypes.byref(out), ctypes.c_size_t(copy_bytes))
    if st != 0:
        raise gett.GettError(st, "gett_measure_peaks failed")
    return {f: getattr(out, f) for f, _ in _Peaks._fields_}
