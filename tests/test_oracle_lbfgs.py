"""Oracle pins of the limited-memory direction (L-BFGS, the paper's future
work in Section VI; two-loop recursion of Nocedal & Wright, Alg. 7.4).

The two-loop recursion computes -H g for the matrix H obtained by applying
the BFGS update (the product form printed in Alg. 4) to gamma I once per
stored pair, oldest first; that definition is written out here with numpy
matrices and compared with the oracle."""
import numpy as np
import pytest


def _spd(rng, d):
    m = rng.normal(size=(d, d))
    return m @ m.T + d * np.eye(d)


def _pairs(rng, d, n):
    A = _spd(rng, d)
    S = rng.normal(size=(n, d))
    Y = S @ A.T  # y = A s: every pair has y's > 0
    return S, Y


def _explicit(S, Y, g):
    d = g.shape[0]
    n = S.shape[0]
    gamma = float(S[-1] @ Y[-1]) / float(Y[-1] @ Y[-1]) if n else 1.0
    H = gamma * np.eye(d)
    I = np.eye(d)
    for s, y in zip(S, Y):
        rho = 1.0 / float(y @ s)
        H = (I - rho * np.outer(s, y)) @ H @ (I - rho * np.outer(y, s)) + rho * np.outer(s, s)
    return -H @ g


@pytest.mark.parametrize("order", [0, 1])
@pytest.mark.parametrize("d,n", [(1, 1), (3, 2), (6, 6), (10, 4), (17, 8)])
def test_two_loop_equals_the_explicit_bfgs_matrix(oracle_mod, d, n, order):
    rng = np.random.default_rng(100 * d + n)
    S, Y = _pairs(rng, d, n)
    g = rng.normal(size=d)
    p = oracle_mod.lbfgs_direction(S, Y, g, order=order)
    q = _explicit(S, Y, g)
    assert np.abs(p - q).max() <= 1e-10 * max(1.0, np.abs(q).max())


def test_no_pairs_gives_steepest_descent(oracle_mod):
    g = np.array([1.0, -2.0, 0.5])
    assert np.array_equal(oracle_mod.lbfgs_direction(np.zeros((0, 3)), np.zeros((0, 3)), g), -g)


@pytest.mark.parametrize("order", [0, 1])
def test_secant_condition_of_the_newest_pair(oracle_mod, order):
    # H maps the newest y to its s: the direction for g = -y is s
    rng = np.random.default_rng(7)
    S, Y = _pairs(rng, 8, 5)
    p = oracle_mod.lbfgs_direction(S, Y, -Y[-1], order=order)
    assert np.abs(p - S[-1]).max() <= 1e-10 * np.abs(S[-1]).max()


@pytest.mark.parametrize("obj,d,lo,hi", [("rosenbrock", 20, -2.0, 2.0), ("quadratic", 30, -3.0, 3.0),
                                         ("rastrigin", 6, -0.4, 0.4), ("ackley", 12, -0.3, 0.3)])
@pytest.mark.parametrize("order", [0, 1])
def test_lbfgs_reaches_the_known_minimum(oracle_mod, obj, d, lo, hi, order):
    # the closed-form minima (Rosenbrock chain 0 at 1; the others 0 at 0)
    p = oracle_mod.Problem(objective=obj, dim=d, lower=lo, upper=hi, n_starts=8, pso_iters=2,
                           bfgs_max_iters=2000, lbfgs_m=6, seed=3, order=order)
    r = oracle_mod.solve(p)
    b = r["best"]
    assert r["f"][b] < 1e-10
    xstar = np.ones(d) if obj == "rosenbrock" else np.zeros(d)
    assert np.abs(r["x"][b] - xstar).max() < 1e-5


def test_lbfgs_memory_one_vs_dense_on_a_quadratic(oracle_mod):
    # on f = 0.5 x'x (H* = I) one step of either method reaches the minimum
    for m in (0, 1, 5):
        p = oracle_mod.Problem(objective="quadratic", dim=1, lower=-1, upper=1, n_starts=4,
                               pso_iters=0, bfgs_max_iters=50, lbfgs_m=m)
        r = oracle_mod.solve(p)
        assert (r["status"] == 1).all() and (r["iters"] <= 2).all()
