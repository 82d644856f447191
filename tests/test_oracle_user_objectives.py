"""Oracle pins of the two objectives the library's default plug-in of user
objectives supplies (Section IV-A: Zeus accepts any f written for a generic
scalar type and differentiates it on dual numbers, Alg. 5).

Each pin is fixed by mathematics outside the oracle's own formulas: known
minima, symmetries, one-coordinate reductions, and central differences
(an independent way to differentiate) for the dual-number gradients."""
import numpy as np
import pytest

# Himmelblau's four minima (value 0): (3, 2) exactly, the other three as
# published to six decimals (Himmelblau, Applied Nonlinear Programming, 1972)
HIMMELBLAU_MINIMA = np.array([[3.0, 2.0], [-2.805118, 3.131312],
                              [-3.779310, -3.283186], [3.584428, -1.848126]])


def central_diff(f, x, h=1e-5):
    """Fourth-order central difference of f at x, coordinate by coordinate."""
    x = np.asarray(x, dtype=np.float64)
    g = np.empty_like(x)
    for i in range(x.size):
        e = np.zeros_like(x)
        e[i] = h
        g[i] = (-f(x + 2 * e) + 8 * f(x + e) - 8 * f(x - e) + f(x - 2 * e)) / (12 * h)
    return g


@pytest.mark.parametrize("d", [1, 2, 7, 40])
def test_griewank_is_zero_at_the_origin(oracle_mod, d):
    assert oracle_mod.f("griewank", np.zeros(d)) == 0.0
    fv, g = oracle_mod.grad_forward("griewank", np.zeros(d))
    assert fv == 0.0 and np.all(g == 0.0)


def test_griewank_on_the_cosine_lattice(oracle_mod):
    # x_i = 2 pi k_i sqrt(i) makes every cosine 1: f = sum x_i^2 / 4000
    k = np.array([1, -2, 0, 3, 1])
    x = 2 * np.pi * k * np.sqrt(np.arange(1, 6))
    assert abs(oracle_mod.f("griewank", x) - (x @ x) / 4000) <= 1e-12 * (x @ x) / 4000


def test_griewank_one_coordinate_reduction(oracle_mod):
    # with only x_k non-zero the product keeps one factor cos(x_k / sqrt(k))
    # and the sum one square; the other factors are cos(0) = 1
    for k, v in [(1, 0.7), (3, -2.5), (9, 11.0)]:
        x = np.zeros(12)
        x[k - 1] = v
        ref = 1 + v * v / 4000 - np.cos(v / np.sqrt(k))
        assert abs(oracle_mod.f("griewank", x) - ref) <= 1e-15 * max(1.0, abs(ref))


def test_griewank_is_even_in_every_coordinate(oracle_mod):
    rng = np.random.default_rng(4)
    x = rng.uniform(-20, 20, 9)
    f0 = oracle_mod.f("griewank", x)
    for i in range(9):
        y = x.copy()
        y[i] = -y[i]
        assert oracle_mod.f("griewank", y) == f0


@pytest.mark.parametrize("obj,d,scale", [("griewank", 6, 15.0), ("griewank", 1, 3.0),
                                         ("himmelblau", 2, 5.0)])
def test_dual_gradient_matches_central_differences(oracle_mod, obj, d, scale):
    rng = np.random.default_rng(d)
    for _ in range(5):
        x = rng.uniform(-scale, scale, d)
        fv, g = oracle_mod.grad_forward(obj, x)
        assert fv == oracle_mod.f(obj, x)
        fd = central_diff(lambda y: oracle_mod.f(obj, y), x)
        assert np.abs(g - fd).max() <= 1e-6 * max(1.0, np.abs(fd).max())


def test_himmelblau_minima(oracle_mod):
    assert oracle_mod.f("himmelblau", [3.0, 2.0]) == 0.0
    fv, g = oracle_mod.grad_forward("himmelblau", [3.0, 2.0])
    assert fv == 0.0 and np.all(g == 0.0)
    for m in HIMMELBLAU_MINIMA[1:]:
        assert oracle_mod.f("himmelblau", m) < 1e-9  # six-decimal points


def test_himmelblau_bfgs_finds_exactly_the_four_minima(oracle_mod):
    # BFGS from every PSO start: the converged points with f ~ 0 fall into
    # four groups, one at each published minimum
    p = oracle_mod.Problem(objective="himmelblau", dim=2, lower=-5, upper=5, n_starts=256,
                           pso_iters=0, bfgs_max_iters=200, seed=2)
    r = oracle_mod.solve(p)
    ok = (r["status"] == 1) & (r["f"] < 1e-12)
    assert ok.mean() > 0.9
    pts = r["x"][ok]
    dist = np.linalg.norm(pts[:, None, :] - HIMMELBLAU_MINIMA[None, :, :], axis=2)
    assert (dist.min(axis=1) < 1e-5).all()
    assert set(np.argmin(dist, axis=1).tolist()) == {0, 1, 2, 3}


def test_griewank_bfgs_reaches_the_origin(oracle_mod):
    # inside the central basin (|x_i| < ~pi sqrt(i)) BFGS reaches 0 at 0
    p = oracle_mod.Problem(objective="griewank", dim=10, lower=-1.5, upper=1.5, n_starts=16,
                           pso_iters=2, bfgs_max_iters=500, seed=5)
    r = oracle_mod.solve(p)
    b = r["best"]
    assert r["f"][b] < 1e-14 and np.abs(r["x"][b]).max() < 1e-6
