"""Host-side pins of two facts the map output relies on (no GPU needed).

The quantised coefficients are s_hat = c / Ls and o_hat = e P / Lo (eq 11-12
with the codes of the quantiser); the oracle forms them as FP64 quotients and
the map stores them as FP32.  The CUDA path forms the FP32 quotient directly.
Ls = 2^(s_bits-1) - 1, Lo = 2^(o_bits-1) - 1 and P = 2^B - 1, so the FP64
quotient rounded to FP32 must equal the correctly rounded FP32 quotient for
every code the encoder can emit; these tests check that exhaustively over the
supported widths (s_bits 2..8, o_bits 2..10, bit depth 1..12).
"""
import numpy as np


def test_s_hat_float_quotient_matches_double_rounding():
    for s_bits in range(2, 9):
        Ls = (1 << (s_bits - 1)) - 1
        c = np.arange(-Ls, Ls + 1)
        via_double = (c.astype(np.float64) / np.float64(Ls)).astype(np.float32)
        direct = c.astype(np.float32) / np.float32(Ls)
        assert np.array_equal(via_double, direct), s_bits


def test_o_hat_float_quotient_matches_double_rounding():
    for B in range(1, 13):
        P = (1 << B) - 1
        for o_bits in range(2, 11):
            Lo = (1 << (o_bits - 1)) - 1
            eP = np.arange(-Lo, Lo + 1, dtype=np.int64) * P
            assert np.all(np.abs(eP) < 1 << 24)  # exact in FP32
            via_double = (eP.astype(np.float64) / np.float64(Lo)).astype(np.float32)
            direct = eP.astype(np.float32) / np.float32(Lo)
            assert np.array_equal(via_double, direct), (B, o_bits)


def test_double_rounding_can_differ_for_other_denominators():
    # the property is specific to denominators 2^k - 1: for an arbitrary
    # denominator the two roundings do differ somewhere, which is what the
    # tests above would catch
    x = np.arange(1, 1 << 22, dtype=np.int64)
    den = 3 * 5 * 7 * 11 * 13 * 17 * 19 * 23 + 2
    via_double = (x.astype(np.float64) / np.float64(den)).astype(np.float32)
    direct = x.astype(np.float32) / np.float32(den)
    assert not np.array_equal(via_double, direct)
