"""Pins of the oracle's plain rounding order (ORDER_PLAIN), the reading that
shares no design choice with any GPU kernel: every product and every sum
rounded on its own, sums left to right, the rank-two update of Alg. 4
formed element by element over the whole matrix.  Checked against what the
arithmetic fixes (exact integer cases, the error bound of a recursive inner
product, a case that tells one rounding per product from a fused
multiply-add) and against the library order, which the paper's exact
arithmetic says it must agree with wherever the trajectory is determined.
"""
from fractions import Fraction

import numpy as np
import pytest

from paper_2603_28770_gb300 import workloads


@pytest.mark.parametrize("n", [1, 7, 32, 33, 100, 1000])
def test_plain_dots_exact_on_integers(oracle_mod, n):
    rng = np.random.default_rng(n)
    a = rng.integers(-1000, 1000, n).astype(float)
    b = rng.integers(-1000, 1000, n).astype(float)
    assert oracle_mod.dot_plain(a, b) == float(np.dot(a.astype(np.int64), b.astype(np.int64)))


@pytest.mark.parametrize("n", [5, 33, 100, 257, 4096])
def test_plain_dots_within_the_error_bound(oracle_mod, n):
    # recursive inner product: |fl - exact| <= gamma_n sum |a_i b_i|
    # (Higham, Accuracy and Stability of Numerical Algorithms, eq. 3.5)
    rng = np.random.default_rng(300 + n)
    a, b = rng.normal(size=n), rng.normal(size=n)
    exact = float(sum(Fraction(float(x)) * Fraction(float(y)) for x, y in zip(a, b)))
    u = 2.0 ** -53
    bound = (n * u / (1 - n * u)) * float(np.sum(np.abs(a * b))) + 2 * u * abs(exact)
    assert abs(oracle_mod.dot_plain(a, b) - exact) <= bound


def test_plain_dot_rounds_each_product(oracle_mod):
    # (1 + 2^-30)^2 = 1 + 2^-29 + 2^-60 is rounded to 1 + 2^-29 before the
    # sum: the plain order gives exactly 0 where one rounding per term (fma)
    # keeps 2^-60
    oracle = oracle_mod
    e = 2.0 ** -30
    a = np.array([1.0, 1.0 + e])
    b = np.array([-(1.0 + 2 * e), 1.0 + e])
    assert oracle.dot_plain(a, b) == 0.0
    assert oracle.dot_split(a, b) == 2.0 ** -60


def test_plain_dot_is_one_left_to_right_chain(oracle_mod):
    # 1e16 absorbs every 1 that follows it (the spacing of doubles near 1e16
    # is 2) until -1e16 cancels it, at any length: one chain
    for n in (32, 64, 100):
        a, b = np.ones(n), np.ones(n)
        b[0], b[n // 2] = 1e16, -1e16
        assert oracle_mod.dot_plain(a, b) == float(n - n // 2 - 1)


@pytest.mark.parametrize("obj", ["rosenbrock", "rastrigin", "quadratic"])
@pytest.mark.parametrize("d", [2, 33, 64, 129])
def test_plain_objectives_exact_on_integer_points(oracle_mod, obj, d):
    # integer points: every term and partial sum is an integer (or a half
    # integer for the quadratic) far below 2^53, so both orders are exact
    rng = np.random.default_rng(d)
    x = rng.integers(-3, 4, d).astype(float)
    xi = x.astype(np.int64)
    if obj == "rosenbrock":
        want = float(np.sum((1 - xi[:-1]) ** 2 + 100 * (xi[1:] - xi[:-1] ** 2) ** 2))
    elif obj == "rastrigin":  # cos(2 pi k) = 1 exactly (exact argument reduction)
        want = float(10 * d + np.sum(xi ** 2 - 10))
    else:
        want = float(Fraction(int(np.sum(np.arange(1, d + 1) * xi ** 2)), 2))
    assert oracle_mod.f(obj, x, order=oracle_mod.ORDER_PLAIN) == want
    assert oracle_mod.f(obj, x, order=oracle_mod.ORDER_LIB) == want


@pytest.mark.parametrize("obj,lo,hi", [("rosenbrock", -2.0, 2.0), ("rastrigin", -5.12, 5.12),
                                       ("ackley", -5.0, 5.0)])
@pytest.mark.parametrize("d", [40, 100])
def test_plain_gradients_match_complex_step(oracle_mod, obj, lo, hi, d):
    # the plain order's dual passes against complex-step derivatives written
    # from Section V-B with numpy complex arithmetic
    from test_oracle_objectives import _cs_grad
    rng = np.random.default_rng(7 * d)
    for _ in range(3):
        x = rng.uniform(lo, hi, d)
        fv, g = oracle_mod.grad_forward(obj, x, order=oracle_mod.ORDER_PLAIN)
        cs = _cs_grad(obj, x)
        assert np.abs(g - cs).max() <= 1e-11 * max(1.0, np.abs(cs).max())
        assert abs(fv - oracle_mod.f(obj, x, order=oracle_mod.ORDER_PLAIN)) == 0.0


def _runs(oracle_mod, obj, d, x0, K, order):
    p = oracle_mod.Problem(objective=obj, dim=d, n_starts=len(x0), bfgs_max_iters=K, order=order,
                           n_threads=4)
    return oracle_mod.bfgs_many(p, x0)


def _rel(a, b):
    r = np.abs(a["x"] - b["x"]).max(axis=1) / np.maximum(1.0, np.abs(b["x"]).max(axis=1))
    r = np.maximum(r, np.abs(a["f"] - b["f"]) / np.maximum(1.0, np.abs(b["f"])))
    r = np.maximum(r, np.abs(a["gnorm"] - b["gnorm"]) / np.maximum(1.0, np.abs(b["gnorm"])))
    r[(a["status"] != b["status"]) | (a["iters"] != b["iters"])] = np.inf
    return r


@pytest.mark.parametrize("obj,d,n,lo,hi", [("rosenbrock", 10, 256, -5.0, 5.0),
                                           ("rosenbrock", 256, 24, -2.0, 2.0),
                                           ("rastrigin", 100, 64, -5.12, 5.12),
                                           ("ackley", 1024, 6, -5.0, 5.0)])
def test_orders_agree_over_twenty_iterations(oracle_mod, obj, d, n, lo, hi):
    # the two rounding orders compute the same exact arithmetic: after 20
    # iterations they agree to 1e-9 per start wherever the run is determined
    # to that accuracy (a one-ulp move of the start moves the plain run by
    # less than 1e-10), and on nearly all starts
    x0 = workloads.start_points(n, d, lo, hi, 23)
    lib = _runs(oracle_mod, obj, d, x0, 20, oracle_mod.ORDER_LIB)
    plain = _runs(oracle_mod, obj, d, x0, 20, oracle_mod.ORDER_PLAIN)
    up = _runs(oracle_mod, obj, d, np.nextafter(x0, np.inf), 20, oracle_mod.ORDER_PLAIN)
    dn = _runs(oracle_mod, obj, d, np.nextafter(x0, -np.inf), 20, oracle_mod.ORDER_PLAIN)
    sens = np.maximum(_rel(up, plain), _rel(dn, plain))
    r = _rel(lib, plain)
    determined = sens <= 1e-10
    assert np.all(r[determined] <= 1e-9)
    assert np.mean(r <= 1e-9) >= 0.9
