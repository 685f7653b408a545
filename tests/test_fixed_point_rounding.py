"""The fixed-point spread (variants 5 and 6) rounds each contribution with
FMAs against 1.5 * 2^23 and reads the integer from the float's bits, and sizes
its unit so that no cell of a subproblem overflows int32.  These CPU checks
pin both claims: the FMA rounding is emulated exactly in float64 (a float32
product is exact in float64, and the sum with the constant spans at most 50
bits here), and the unit follows the formula of the fixed-point spreads."""
import os
import re

import numpy as np

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_1605_05231_gb300", "csrc",
                   "interp_common.cuh")
MAGIC = np.float32(12582912.0)   # 1.5 * 2^23
MAGIC_BITS = 0x4B400000


def _fma32(a, b, c):
    """fmaf(a, b, c): the exact a b + c rounded once to float32."""
    return (np.float64(a) * np.float64(b) + np.float64(c)).astype(np.float32)


def _round_units(a, b, c, d):
    t = _fma32(c, d, np.full_like(c, MAGIC))
    t = _fma32(a, b, t)
    return t.view(np.int32).astype(np.int64) - MAGIC_BITS


def test_source_constants():
    src = open(SRC).read()
    assert re.search(r"kRoundMagic = 12582912\.0f", src)
    assert re.search(r"kRoundMagicBits = 0x4B400000", src)


def test_magic_rounding_matches_nearest_integer():
    rng = np.random.default_rng(0)
    n = 200000
    # products up to the unit budget (2^22 (1 - 2^-10)) in magnitude, of either sign
    lim = 2.0 ** 22 * (1 - 2.0 ** -10)
    a = rng.uniform(-1, 1, n).astype(np.float32)
    c = rng.uniform(-1, 1, n).astype(np.float32)
    b = (rng.uniform(-1, 1, n) * lim / 2).astype(np.float32)
    d = (rng.uniform(-1, 1, n) * lim / 2).astype(np.float32)
    got = _round_units(a, b, c, d)
    exact = np.float64(a) * np.float64(b) + np.float64(c) * np.float64(d)
    # two roundings to integers (after c d, after a b): within one unit of the exact sum
    assert np.max(np.abs(got - exact)) <= 1.0
    # and mostly the nearest integer
    assert np.mean(got == np.rint(exact)) > 0.7
    assert np.max(np.abs(got)) < 2 ** 22


def test_unit_budget_bounds_cells():
    """B = 2^min(22, 30 - ceil(log2 S)) (1 - 2^-10) per contribution: every
    contribution stays inside the magic constant's exact range and no cell of
    S contributions (one per point) reaches 2^31."""
    for S in range(1, 513):
        lg = int(np.ceil(np.log2(S))) if S > 1 else 0
        bits = 22 if lg <= 8 else 30 - lg
        B = 2.0 ** bits * (1 - 2.0 ** -10)
        worst = B * (1 + 4 * 2.0 ** -24) + 2          # FP32 rounding of the products, two integer roundings
        assert worst < 2 ** 22
        assert S * worst < 2 ** 31
    # the CTA-shared variant fixes S <= 256 and B = 2^22 (1 - 2^-10)
    assert 256 * (2.0 ** 22 * (1 - 2.0 ** -10) + 3) < 2 ** 31


def test_single_product_rounding_is_nearest_integer():
    """round_unit1 (the real-weight spread): one FMA of a b with 1.5 * 2^23 puts
    the product in [2^23, 2^24), where floats are spaced by 1, so the result is
    a b rounded to the nearest integer (ties to even) for |a b| < 2^22."""
    rng = np.random.default_rng(1)
    n = 200000
    lim = 2.0 ** 22 * (1 - 2.0 ** -10)
    a = rng.uniform(-1, 1, n).astype(np.float32)
    b = (rng.uniform(-1, 1, n) * lim).astype(np.float32)
    exact = np.float64(a) * np.float64(b)
    # FMA: exact product, one rounding of the sum with the magic constant
    s = (exact + 12582912.0).astype(np.float32)
    got = s.view(np.int32).astype(np.int64) - 0x4B400000
    assert np.array_equal(got, np.rint(exact).astype(np.int64))
