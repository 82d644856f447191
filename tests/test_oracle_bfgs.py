"""Pins of the oracle's line search (Alg. 6), inverse-Hessian update and
BFGS loop (Alg. 4), and of the whole method (Alg. 7) on small cases.
Tests that take `order` run in both rounding orders of the oracle (the
library order and the plain order: every operation rounded on its own,
sums left to right, the update over the whole matrix).
"""
import math

import numpy as np
import pytest


# ---------------------------------------------------------------- line search

@pytest.mark.parametrize("gamma", [0.1, 1.0, 1.9, 2.5, 7.0, 100.0, 3e6, 1e9])
@pytest.mark.parametrize("c", [1e-4, 0.3])
def test_line_search_quadratic_closed_form(oracle_mod, gamma, c):
    # f = 0.5 x^2 (the d = 1 test quadratic), p = -gamma x0, ddir = -gamma x0^2:
    # f(x0 + a p) <= f0 + c a ddir  <=>  a <= 2 (1 - c) / gamma, so the
    # accepted step is the largest 0.5^m (m < L) below that bound, or 0.5^L.
    x0, L, beta = 1.75, 20, 0.5
    f0 = 0.5 * x0 * x0
    alpha, acc, nf = oracle_mod.line_search("quadratic", [x0], [-gamma * x0], f0, -gamma * x0 * x0,
                                            c=c, beta=beta, L=L)
    bound = 2 * (1 - c) / gamma
    ms = [m for m in range(L) if beta**m <= bound]
    if ms:
        assert acc and alpha == beta ** ms[0] and nf == ms[0] + 1
    else:
        assert (not acc) and alpha == beta**L and nf == L


def test_line_search_armijo_property(oracle_mod):
    rng = np.random.default_rng(2)
    for _ in range(50):
        x = rng.uniform(-2, 2, size=4)
        f0, g = oracle_mod.grad_forward("rosenbrock", x)
        p = -g
        ddir = float(g @ p)
        a, acc, _ = oracle_mod.line_search("rosenbrock", x, p, f0, ddir)
        assert acc
        assert oracle_mod.f("rosenbrock", x + a * p) <= f0 + 1e-4 * a * ddir
        if a < 1.0:  # the previous trial (2a) failed the test
            assert oracle_mod.f("rosenbrock", x + 2 * a * p) > f0 + 1e-4 * 2 * a * ddir


# ------------------------------------------------------------- BFGS update

def _spd(rng, d):
    m = rng.normal(size=(d, d))
    return m @ m.T + d * np.eye(d)


@pytest.mark.parametrize("order", [0, 1])
def test_update_secant_symmetry_and_product_form(oracle_mod, order):
    rng = np.random.default_rng(3)
    for d in (1, 2, 5, 8, 40):
        for _ in range(10):
            H = np.linalg.inv(_spd(rng, d))
            H = (H + H.T) / 2  # exactly symmetric, as every H of a run is
            s = rng.normal(size=d)
            y = _spd(rng, d) @ s  # y^T s > 0
            Hn, ok = oracle_mod.bfgs_update(H, s, y, order=order)
            assert ok
            # secant condition H+ y = s
            assert np.abs(Hn @ y - s).max() <= 1e-10 * max(1.0, np.abs(s).max())
            assert np.array_equal(Hn, Hn.T)  # mirrored, or symmetric by its expression
            assert np.linalg.eigvalsh((Hn + Hn.T) / 2).min() > 0
            # the product form printed in Alg. 4
            rho = 1.0 / (y @ s)
            I = np.eye(d)
            P = (I - rho * np.outer(s, y)) @ H @ (I - rho * np.outer(y, s)) + rho * np.outer(s, s)
            assert np.abs(Hn - P).max() <= 1e-11 * max(1.0, np.abs(P).max())


@pytest.mark.parametrize("order", [0, 1])
def test_update_skipped_without_curvature(oracle_mod, order):
    H = np.eye(3)
    s = np.array([1.0, 0.0, 0.0])
    for y in (np.array([-1.0, 0.5, 0.0]), np.zeros(3), np.array([0.0, 1.0, 0.0])):
        Hn, ok = oracle_mod.bfgs_update(H, s, y, order=order)
        assert not ok and np.array_equal(Hn, H)


@pytest.mark.parametrize("order", [0, 1])
@pytest.mark.parametrize("d", [2, 3, 6, 12, 20, 40, 64])  # 40, 64: the split dot order
def test_quadratic_termination_exact_steps(oracle_mod, d, order):
    # with exact line searches BFGS minimises 0.5 x^T A x in at most d steps
    # and ends with H = A^{-1} (quadratic termination of the Broyden class)
    rng = np.random.default_rng(d)
    A = _spd(rng, d)
    x0 = rng.normal(size=d)
    k, x, H = oracle_mod.bfgs_quadratic_exact(A, x0, max_iters=5 * d, tol=1e-9, order=order)
    assert k <= d
    assert np.abs(A @ x).max() < 1e-9
    if k == d:
        Ainv = np.linalg.inv(A)
        assert np.abs(H - Ainv).max() <= 1e-7 * np.abs(Ainv).max()


# --------------------------------------------------------------- BFGS loop

@pytest.mark.parametrize("order", [0, 1])
def test_identity_quadratic_one_step(oracle_mod, order):
    # f = 0.5 x^2 (d = 1): p = -g = -x, alpha = 1 lands on 0 exactly
    p = oracle_mod.Problem("quadratic", dim=1, bfgs_max_iters=50, order=order)
    r = oracle_mod.bfgs(p, [3.5])
    assert r["status"] == 1 and r["iters"] == 1 and r["x"][0] == 0.0 and r["f"] == 0.0


@pytest.mark.parametrize("order", [0, 1])
def test_rosenbrock_classic_start(oracle_mod, order):
    p = oracle_mod.Problem("rosenbrock", dim=2, bfgs_max_iters=100, order=order)
    r = oracle_mod.bfgs(p, [-1.2, 1.0])
    assert r["status"] == 1 and r["gnorm"] < 1e-8
    assert np.linalg.norm(r["x"] - 1.0) < 1e-6  # Euclidean criterion, Section V-A
    assert r["f"] < 1e-12


def test_zero_iteration_cap(oracle_mod):
    p = oracle_mod.Problem("rosenbrock", dim=2, bfgs_max_iters=0)
    r = oracle_mod.bfgs(p, [0.3, -0.2])
    assert r["status"] == 0 and r["iters"] == 0
    assert r["f"] == oracle_mod.f("rosenbrock", [0.3, -0.2]) and np.array_equal(r["x"], [0.3, -0.2])


def test_converged_start_needs_no_iteration(oracle_mod):
    p = oracle_mod.Problem("rastrigin", dim=4, bfgs_max_iters=10)
    r = oracle_mod.bfgs(p, np.zeros(4))
    assert r["status"] == 1 and r["iters"] == 0 and r["f"] == 0.0


def test_non_finite_start(oracle_mod):
    p = oracle_mod.Problem("rosenbrock", dim=2, bfgs_max_iters=10)
    r = oracle_mod.bfgs(p, [1e160, 1e160])
    assert r["status"] == 3 and r["iters"] == 0


def test_ackley_never_meets_gradient_test_near_zero(oracle_mod):
    # Section VI: Ackley's minimum sits on a kink, runs near 0 end at the cap
    p = oracle_mod.Problem("ackley", dim=2, bfgs_max_iters=200)
    r = oracle_mod.bfgs(p, [0.02, -0.03])
    assert r["status"] == 0 and r["f"] < 1e-3


@pytest.mark.parametrize("order,d", [(0, 10), (1, 10), (0, 40), (1, 40)])
def test_iterates_decrease_f(oracle_mod, order, d):
    rng = np.random.default_rng(9)
    x0 = rng.uniform(-5.12, 5.12, size=(32, d))
    for K in (1, 2, 5, 10):
        p = oracle_mod.Problem("rastrigin", dim=d, bfgs_max_iters=K, n_threads=2, order=order)
        r = oracle_mod.bfgs_many(p, x0)
        f0 = np.array([oracle_mod.f("rastrigin", xi, order=order) for xi in x0])
        assert np.all(r["f"] <= f0)


# --------------------------------------------------------------- whole method

def test_rosenbrock_2d_workload(oracle_mod):
    # 2-D Rosenbrock, 128 particles, 5 PSO iterations, 100 BFGS iterations
    r = oracle_mod.solve(oracle_mod.Problem())
    b = r["best"]
    assert r["f"][b] < 1e-6 and np.linalg.norm(r["x"][b] - 1.0) < 1e-6
    assert np.mean(r["status"] == 1) > 0.9


def _grid_min(fn, lo, hi, n):
    t = np.linspace(lo, hi, n)
    X, Y = np.meshgrid(t, t, indexing="ij")
    return fn(X, Y).min()


@pytest.mark.parametrize("obj,lo,hi,fn", [
    ("rastrigin", -5.12, 5.12, lambda X, Y: 20 + X**2 - 10 * np.cos(2 * np.pi * X) + Y**2 - 10 * np.cos(2 * np.pi * Y)),
    ("rosenbrock", -5.0, 5.0, lambda X, Y: (1 - X) ** 2 + 100 * (Y - X**2) ** 2),
    ("goldstein_price", -2.0, 2.0, lambda X, Y: (1 + (X + Y + 1) ** 2 * (19 - 14 * X + 3 * X**2 - 14 * Y + 6 * X * Y + 3 * Y**2))
     * (30 + (2 * X - 3 * Y) ** 2 * (18 - 32 * X + 12 * X**2 + 48 * Y - 36 * X * Y + 27 * Y**2))),
])
@pytest.mark.parametrize("order", [0, 1])
def test_two_dimensional_brute_force(oracle_mod, obj, lo, hi, fn, order):
    # a 2001 x 2001 grid over the box (containing the minimiser) bounds the
    # global minimum from above; the method must do at least as well
    gmin = _grid_min(fn, lo, hi, 2001)
    p = oracle_mod.Problem(obj, dim=2, lower=lo, upper=hi, n_starts=256, pso_iters=5, bfgs_max_iters=200,
                           seed=1, order=order)
    r = oracle_mod.solve(p)
    assert r["f"][r["best"]] <= gmin + 1e-9
