"""Host checks of the split-precision parameters (gett_ozaki_params) against
the conditions that make the modular form exact (Ozaki, Uchino and Imamura
2025; the thesis names no split method: its arithmetic is that of the
operand types, Sec. 6).  Scaled operands are integers of at most `bits` bits, so a sum of K
products has magnitude below K * 2^(2 bits); it is recovered exactly from its
residues when that stays below P / 2, P the product of the moduli.  Every
bound is checked here in exact integer arithmetic, not in the library's
floating-point logarithms."""
import ctypes
import math

import numpy as np
import pytest

from paper_2410_06770_gb300 import gett


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2410_06770_gb300 import build
    build.build()
    gett.lib()


def max_bits(K, P):
    """The largest b with K * 2^(2b) < P / 2 (exact), or -1."""
    b = -1
    while 2 * max(K, 1) * 4 ** (b + 1) < P:
        b += 1
    return b


KS = [0, 1, 2, 3, 64, 440, 441, 480, 1024, 16384, 85043, 85044, 1 << 20, 16248323, 16248324, (1 << 31) - 1]


def test_moduli_are_odd_coprime_and_bf16_exact():
    L, _, mods = gett.ozaki_params(1 << 20, 20)
    assert L == 20 and len(set(mods)) == 20
    for p in mods:
        assert p % 2 == 1 and 3 <= p <= 255
        # symmetric residues lie in [-(p-1)/2, (p-1)/2]: at most 8 significant
        # bits, so the low 16 bits of their fp32 patterns are zero (exact bf16)
        r = np.arange(-(p - 1) // 2, (p - 1) // 2 + 1, dtype=np.float32)
        assert not np.any(r.view(np.uint32) & 0xFFFF)
    for i in range(20):
        for j in range(i):
            assert math.gcd(mods[i], mods[j]) == 1


@pytest.mark.parametrize("K", KS)
def test_automatic_count_is_the_smallest_exact_one(K):
    """bits >= 50 with L moduli, and fewer moduli could not keep 50 bits; the
    sum bound K * 2^(2 bits) < P / 2 holds exactly."""
    L, bits, mods = gett.ozaki_params(K)
    P = math.prod(mods)
    assert bits == min(52, max_bits(K, P))
    assert bits >= 50
    assert 2 * max(K, 1) * 4 ** bits < P
    assert max_bits(K, math.prod(mods[:-1])) < 50


@pytest.mark.parametrize("want", [1, 2, 8, 15, 20])
@pytest.mark.parametrize("K", [1, 480, 16384])
def test_requested_count(K, want):
    """A requested count is used as given (counts below 2 become 2); the bits
    are then the exact maximum for that count, capped at 52."""
    L, bits, mods = gett.ozaki_params(K, want)
    assert L == max(2, want)
    assert bits == max(1, min(52, max_bits(K, math.prod(mods))))


def test_complex_sums_count_twice_the_terms():
    """The complex real form sums 2K products: its parameters are those of 2K."""
    assert gett.ozaki_params(2 * 16384) == gett.ozaki_params(32768)
    assert gett.ozaki_params(2 * 16384)[1] <= gett.ozaki_params(16384)[1]


@pytest.mark.parametrize("K,want", [(-1, 0), (10, -1), (10, 21)])
def test_invalid_arguments(K, want):
    with pytest.raises(gett.GettError) as ei:
        gett.ozaki_params(K, want)
    assert ei.value.status == gett.GETT_ERR_ARG


def test_null_outputs_rejected_and_moduli_optional():
    L = gett.lib()
    n, bits = ctypes.c_int(0), ctypes.c_int(0)
    assert L.gett_ozaki_params(480, 0, None, ctypes.byref(bits), None) == gett.GETT_ERR_ARG
    assert L.gett_ozaki_params(480, 0, ctypes.byref(n), None, None) == gett.GETT_ERR_ARG
    assert L.gett_ozaki_params(480, 0, ctypes.byref(n), ctypes.byref(bits), None) == gett.GETT_OK
    assert (n.value, bits.value) == gett.ozaki_params(480)[:2]
