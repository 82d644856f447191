"""Oracle pins of the order of the BFGS dot products (reading: one fused
multiply-add chain in index order up to 32 terms; past that 32 strided
chains added in a fixed tree, so that 32 lanes can form one sum).  Both
orders are exact where the arithmetic is exact, stay within the textbook
error bound of a recursive sum, and agree with each other up to 32 terms."""
import math

import numpy as np
import pytest


@pytest.mark.parametrize("n", [1, 7, 32])
def test_short_dots_are_one_fma_chain(oracle_mod, n):
    # up to 32 terms the order is one chain: exact on integers, and the
    # cancellation case below (which the split order survives) loses the
    # small terms
    rng = np.random.default_rng(n)
    ai, bi = rng.integers(-50, 50, n).astype(float), rng.integers(-50, 50, n).astype(float)
    assert oracle_mod.dot_split(ai, bi) == float(np.dot(ai.astype(np.int64), bi.astype(np.int64)))


@pytest.mark.parametrize("n", [33, 64, 100, 129, 1000])
def test_split_dots_exact_on_integers(oracle_mod, n):
    rng = np.random.default_rng(n)
    a = rng.integers(-1000, 1000, n).astype(float)
    b = rng.integers(-1000, 1000, n).astype(float)
    assert oracle_mod.dot_split(a, b) == float(np.dot(a.astype(np.int64), b.astype(np.int64)))


@pytest.mark.parametrize("n", [5, 33, 64, 100, 257, 4096])
def test_dots_within_the_error_bound(oracle_mod, n):
    # |computed - exact| <= gamma_k * sum |a_i b_i| with k the longest chain
    # of roundings (n for one chain; n/32 + 1 + 5 for the split order)
    rng = np.random.default_rng(100 + n)
    a, b = rng.normal(size=n), rng.normal(size=n)
    # the exact sum of the exact products
    from fractions import Fraction
    exact = float(sum(Fraction(float(x)) * Fraction(float(y)) for x, y in zip(a, b)))
    k = n if n <= 32 else (n + 31) // 32 + 5
    u = 2.0 ** -53
    bound = (k * u / (1 - k * u)) * float(np.sum(np.abs(a * b))) + 2 * u * abs(exact)
    assert abs(oracle_mod.dot_split(a, b) - exact) <= bound


def test_split_order_differs_from_one_chain_only_in_rounding(oracle_mod):
    # with terms whose sequential chain loses the small ones, the strided
    # partials keep them: 1e16 in partial 0 and 32 ones spread over all
    # partials, n = 64
    a = np.ones(64)
    b = np.ones(64)
    b[0] = 1e16
    b[32] = -1e16
    # exact sum: 62; one chain: 1e16 + 1 + ... is rounded at every step
    assert oracle_mod.dot_split(a, b) == 62.0
    # the same terms in one chain (n = 32): 1e16 absorbs every 1 (the
    # spacing of doubles near 1e16 is 2), so the sum is 0 + the ones
    # after the cancellation
    a32, b32 = np.ones(32), np.ones(32)
    b32[0], b32[16] = 1e16, -1e16
    assert oracle_mod.dot_split(a32, b32) == 15.0
