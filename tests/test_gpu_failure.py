"""Device-side failure detection without a GPU fault: a bounded wait on a
barrier that nothing completes gives up after its limit, the host reads
GETT_ERR_TIMEOUT from the device error word, the word is cleared, and the
CUDA context keeps working (a contraction right after still matches the
oracle)."""
import ctypes

import numpy as np
import pytest

from paper_2410_06770_gb300 import gett, synth
from tests._gpu_util import compare, oracle_ref, run_gpu

pytestmark = pytest.mark.gpu


def test_bounded_wait_reports_timeout_and_context_survives():
    from paper_2410_06770_gb300 import build
    build.build()
    L = gett.lib()
    L.gett_check_wait_timeout.argtypes = [ctypes.c_longlong]
    L.gett_check_wait_timeout.restype = ctypes.c_int
    assert L.gett_check_wait_timeout(2_000_000) == gett.GETT_ERR_TIMEOUT  # ~1 ms at 2 GHz
    assert gett.device_status() == gett.GETT_OK  # the word was cleared
    p = synth.cfg_small_dgett()
    got, _ = run_gpu("d", p, mode="ex", opts=gett.options(algo="ozaki_bf16"))
    ref = oracle_ref(p)
    g = synth.gather(p.lc, got)
    r = synth.gather(p.lc, ref)
    assert np.linalg.norm(g - r) <= 1e-13 * np.linalg.norm(r)
    got2, _ = run_gpu("d", p)
    compare("d", p, got2, ref)
