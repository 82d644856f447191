"""Pins of the oracle's objectives (Section V-B) and of its forward-mode
dual-number gradient (Alg. 5, dual algebra of Section III-C).

Independent checks:
* closed-form values (tests/golden/objective_closed_forms.txt);
* complex-step differentiation (Squire & Trapp 1998): Im f(x + i h e_k)/h
  with h = 1e-30 is the derivative to rounding for analytic f, computed
  here with numpy complex arithmetic, not with dual numbers;
* a hand-derived Rosenbrock gradient and central differences.
"""
import math
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "objective_closed_forms.txt")


def _golden():
    for line in open(GOLDEN):
        if line.strip() and not line.startswith("#"):
            obj, xs, fv, _why = [t.strip() for t in line.split("|")]
            yield obj, [float(v) for v in xs.split(",")], float(fv)


def test_closed_form_values(oracle_mod):
    for obj, x, want in _golden():
        got = oracle_mod.f(obj, x)
        assert abs(got - want) <= 1e-12 * max(1.0, abs(want)), (obj, x, got, want)


# --- complex-step versions of the objectives, straight from Section V-B ---

def _cs_f(obj, z):
    d = z.size
    if obj == "rosenbrock":
        return np.sum((1 - z[:-1]) ** 2 + 100 * (z[1:] - z[:-1] ** 2) ** 2)
    if obj == "rastrigin":
        return 10 * d + np.sum(z ** 2 - 10 * np.cos(2 * np.pi * z))
    if obj == "ackley":
        return (-20 * np.exp(-0.2 * np.sqrt(np.sum(z ** 2) / d))
                - np.exp(np.sum(np.cos(2 * np.pi * z)) / d) + 20 + np.e)
    if obj == "goldstein_price":
        x1, x2 = z[0], z[1]
        a = 1 + (x1 + x2 + 1) ** 2 * (19 - 14 * x1 + 3 * x1 ** 2 - 14 * x2 + 6 * x1 * x2 + 3 * x2 ** 2)
        b = 30 + (2 * x1 - 3 * x2) ** 2 * (18 - 32 * x1 + 12 * x1 ** 2 + 48 * x2 - 36 * x1 * x2 + 27 * x2 ** 2)
        return a * b
    if obj == "quadratic":
        return np.sum(0.5 * np.arange(1, d + 1) * z ** 2)
    raise ValueError(obj)


def _cs_grad(obj, x, h=1e-30):
    x = np.asarray(x, dtype=np.float64)
    g = np.zeros_like(x)
    for k in range(x.size):
        z = x.astype(np.complex128)
        z[k] += 1j * h
        g[k] = _cs_f(obj, z).imag / h
    return g


CASES = [("rosenbrock", 2, 2.0), ("rosenbrock", 7, 2.0), ("rastrigin", 3, 5.12),
         ("rastrigin", 10, 5.12), ("ackley", 2, 5.0), ("ackley", 9, 5.0),
         ("goldstein_price", 2, 2.0), ("quadratic", 6, 3.0)]


@pytest.mark.parametrize("obj,d,box", CASES)
def test_dual_gradient_vs_complex_step(oracle_mod, obj, d, box):
    rng = np.random.default_rng(d * 31 + len(obj))
    for _ in range(20):
        x = rng.uniform(-box, box, size=d)
        fv, g = oracle_mod.grad_forward(obj, x)
        assert fv == oracle_mod.f(obj, x)  # value part equals the plain f
        gc = _cs_grad(obj, x)
        scale = max(1.0, np.abs(gc).max())
        assert np.abs(g - gc).max() <= 1e-12 * scale, (x, g, gc)


def test_rosenbrock_hand_gradient(oracle_mod):
    # df/dx_i = -2(1-x_i) - 400 x_i (x_{i+1} - x_i^2) + 200 (x_i - x_{i-1}^2)
    rng = np.random.default_rng(1)
    for d in (2, 3, 8):
        x = rng.uniform(-2, 2, size=d)
        want = np.zeros(d)
        for i in range(d - 1):
            want[i] += -2 * (1 - x[i]) - 400 * x[i] * (x[i + 1] - x[i] ** 2)
            want[i + 1] += 200 * (x[i + 1] - x[i] ** 2)
        _, g = oracle_mod.grad_forward("rosenbrock", x)
        np.testing.assert_allclose(g, want, rtol=1e-12, atol=1e-10)


@pytest.mark.parametrize("obj,d,box", CASES)
def test_dual_gradient_vs_central_differences(oracle_mod, obj, d, box):
    rng = np.random.default_rng(5 + d)
    x = rng.uniform(-box, box, size=d)
    _, g = oracle_mod.grad_forward(obj, x)
    h = 1e-6
    for k in range(d):
        e = np.zeros(d); e[k] = h
        fd = (oracle_mod.f(obj, x + e) - oracle_mod.f(obj, x - e)) / (2 * h)
        assert abs(fd - g[k]) <= 1e-5 * max(1.0, abs(g[k]))


def test_minimisers_have_zero_gradient(oracle_mod):
    assert np.all(oracle_mod.grad_forward("rosenbrock", np.ones(6))[1] == 0)
    assert np.abs(oracle_mod.grad_forward("rastrigin", np.zeros(4))[1]).max() == 0
    fv, g = oracle_mod.grad_forward("goldstein_price", [0.0, -1.0])
    assert fv == 3.0 and np.abs(g).max() < 1e-12
    # Ackley: derivative undefined at 0; the reading takes sqrt'(0) = 0
    fv, g = oracle_mod.grad_forward("ackley", np.zeros(3))
    assert fv == 0.0 and np.all(g == 0.0)


@pytest.mark.parametrize("op", ["mul", "div", "sin", "cos", "exp", "sqrt"])
def test_dual_ops_vs_complex_step(oracle_mod, op):
    # a dual number a + b eps behaves like the complex number a + i h b for h -> 0
    rng = np.random.default_rng(11)
    h = 1e-30
    fn = {"mul": lambda x, y: x * y, "div": lambda x, y: x / y, "sin": lambda x, y: np.sin(x),
          "cos": lambda x, y: np.cos(x), "exp": lambda x, y: np.exp(x), "sqrt": lambda x, y: np.sqrt(x)}[op]
    for _ in range(50):
        a1, b1, a2, b2 = rng.uniform(0.1, 3.0), rng.normal(), rng.uniform(0.1, 3.0), rng.normal()
        ra, rb = oracle_mod.dual_op(op, a1, b1, a2, b2)
        z = fn(complex(a1, h * b1), complex(a2, h * b2))
        assert ra == pytest.approx(z.real, rel=1e-15, abs=1e-300)
        assert rb == pytest.approx(z.imag / h, rel=1e-13, abs=1e-13)


def test_dual_add_sub_exact(oracle_mod):
    assert oracle_mod.dual_op("add", 1.5, 2.0, 0.25, -3.0) == (1.75, -1.0)
    assert oracle_mod.dual_op("sub", 1.5, 2.0, 0.25, -3.0) == (1.25, 5.0)
    assert oracle_mod.dual_op("sqrt", 0.0, 1.0) == (0.0, 0.0)


def test_forward_pass_seeds_unit_vectors(oracle_mod):
    # pass i reads df/dx_i: on the separable quadratic 0.5 sum (i+1) x_i^2
    # the gradient is exactly (i+1) x_i
    x = np.array([0.5, -1.25, 3.0, 2.0])
    _, g = oracle_mod.grad_forward("quadratic", x)
    assert np.array_equal(g, np.arange(1, 5) * x)
    assert math.isnan(oracle_mod.f(999, x))


@pytest.mark.parametrize("d", [33, 64, 1000])
def test_split_sums_exact_on_integer_points(oracle_mod, d):
    # past 32 coordinates the sums run as 32 chains and a tree; at integer
    # points every Rastrigin term is the integer x^2 - 10 (cos 2 pi x = 1
    # exactly), so any order gives the exact value sum x^2
    rng = np.random.default_rng(d)
    x = rng.integers(-5, 6, d).astype(float)
    assert oracle_mod.f("rastrigin", x) == float(np.sum(x.astype(np.int64) ** 2))
    fv, g = oracle_mod.grad_forward("rastrigin", x)
    assert fv == oracle_mod.f("rastrigin", x) and np.array_equal(g, 2 * x)


@pytest.mark.parametrize("obj,d", [("quadratic", 100), ("rosenbrock", 64), ("ackley", 200)])
def test_split_sums_within_the_error_bound(oracle_mod, obj, d):
    # the value stays within the rounding bound of its longest chain
    # (d / 32 + 1 additions, then 5 tree levels) of the exact sum of the
    # exactly evaluated terms (fractions)
    from fractions import Fraction
    rng = np.random.default_rng(7 + d)
    x = rng.uniform(-2, 2, d)
    u = 2.0 ** -53
    k = d // 32 + 1 + 5
    if obj == "quadratic":
        terms = [Fraction(0.5 * (i + 1)) * Fraction(float(x[i])) ** 2 for i in range(d)]
        exact = sum(terms)
        mag = float(sum(abs(t) for t in terms))
        # each term itself is rounded at most twice
        bound = (k + 2) * u * mag / (1 - (k + 2) * u)
        assert abs(oracle_mod.f(obj, x) - float(exact)) <= bound
    elif obj == "rosenbrock":
        terms = [(1 - Fraction(float(x[i]))) ** 2
                 + 100 * (Fraction(float(x[i + 1])) - Fraction(float(x[i])) ** 2) ** 2
                 for i in range(d - 1)]
        exact = sum(terms)
        mag = float(sum(abs(t) for t in terms))
        bound = (k + 6) * u * mag / (1 - (k + 6) * u)
        assert abs(oracle_mod.f(obj, x) - float(exact)) <= bound
    else:
        # Ackley: the sums enter exp and sqrt; compare with an mpmath-free
        # double evaluation in fractions of the sums
        s1 = float(sum(Fraction(float(v)) ** 2 for v in x))
        s2 = float(np.sum(np.cos(2 * np.pi * x)))
        ref = -20 * np.exp(-0.2 * np.sqrt(s1 / d)) - np.exp(s2 / d) + 20 + np.e
        assert abs(oracle_mod.f(obj, x) - ref) <= 1e-12 * max(1.0, abs(ref))
