"""Pins of the oracle's PSO phase (Alg. 2 InitSwarm, Alg. 3 UpdateSwarm,
synchronous global best) and of its argmin (Alg. 7 ParallelReduction).

The random draws are recomputed here with numpy's own Philox4x64-10, so the
counter layout and the [lo, hi) mapping are checked independently.
"""
import numpy as np
import pytest


def _u(seed, phase, i, j, problem=0):
    c = [j // 4, i, problem, phase]
    # numpy increments before use: start one below (no borrow needed for j//4 > 0
    # handled generally)
    k = 0
    c = list(c)
    while True:
        c[k] = (c[k] - 1) % 2**64
        if c[k] != 2**64 - 1 or k == 3:
            break
        k += 1
    bg = np.random.Philox(key=np.array([seed, 0], dtype=np.uint64), counter=np.array(c, dtype=np.uint64))
    return float(int(bg.random_raw(4)[j % 4]) >> 11) * 2.0**-53


def _init(seed, n, d, lo, hi):
    x0 = np.array([[lo + (hi - lo) * _u(seed, 0, i, j) for j in range(d)] for i in range(n)])
    vr = hi - lo
    v0 = np.array([[-vr + (vr - (-vr)) * _u(seed, 1, i, j) for j in range(d)] for i in range(n)])
    return x0, v0


def test_init_positions_and_velocities(oracle_mod):
    p = oracle_mod.Problem("rastrigin", dim=5, lower=-5.12, upper=5.12, n_starts=17, pso_iters=0, seed=99)
    r = oracle_mod.pso(p)
    x0, v0 = _init(99, 17, 5, -5.12, 5.12)
    assert np.array_equal(r["x"], x0) and np.array_equal(r["v"], v0)
    assert np.array_equal(r["px"], x0)
    assert np.all(np.abs(r["v"]) <= 10.24) and np.all((x0 >= -5.12) & (x0 < 5.12))
    assert np.array_equal(r["pf"], [oracle_mod.f("rastrigin", xi) for xi in x0])
    b = int(np.argmin(r["pf"]))
    assert r["gidx"] == b and r["gf"] == r["pf"][b] and np.array_equal(r["gx"], x0[b])


@pytest.mark.parametrize("w,T", [(0.7, 5), (0.5, 3), (0.9, 10)])
def test_no_attraction_closed_form(oracle_mod, w, T):
    # c1 = c2 = 0: v_t = w^t v0 and x_T = x0 + v0 * w (1 - w^T) / (1 - w)
    p = oracle_mod.Problem("rosenbrock", dim=3, n_starts=9, pso_iters=T, w=w, c1=0.0, c2=0.0, seed=4)
    r = oracle_mod.pso(p)
    x0, v0 = _init(4, 9, 3, -5.0, 5.0)
    np.testing.assert_allclose(r["v"], v0 * w**T, rtol=1e-13, atol=1e-14)
    np.testing.assert_allclose(r["x"], x0 + v0 * (w * (1 - w**T) / (1 - w)), rtol=1e-12, atol=1e-12)


def test_social_term_first_iteration(oracle_mod):
    # after init pX = x, so with w = 0 the first update is x1 = x0 + c2 r2 (g - x0)
    seed, n, d = 21, 12, 4
    p = oracle_mod.Problem("rastrigin", dim=d, lower=-5.12, upper=5.12, n_starts=n, pso_iters=1,
                           w=0.0, c1=1.3, c2=1.7, seed=seed)
    r = oracle_mod.pso(p)
    x0, _ = _init(seed, n, d, -5.12, 5.12)
    g = x0[int(np.argmin([oracle_mod.f("rastrigin", xi) for xi in x0]))]
    r2 = np.array([[_u(seed, 3, i, j) for j in range(d)] for i in range(n)])
    np.testing.assert_allclose(r["x"], x0 + 1.7 * r2 * (g - x0), rtol=1e-14, atol=1e-14)


def test_cognitive_term_second_iteration(oracle_mod):
    # w = 1, c2 = 0: x1 = x0 + v0; the personal best p is x1 if f(x1) < f(x0)
    # else x0; then v2 = v0 + c1 r1' (p - x1) with r1' drawn in phase 2 + 2*1
    seed, n, d, c1 = 8, 10, 3, 1.4
    p = oracle_mod.Problem("rosenbrock", dim=d, n_starts=n, pso_iters=2, w=1.0, c1=c1, c2=0.0, seed=seed)
    r = oracle_mod.pso(p)
    x0, v0 = _init(seed, n, d, -5.0, 5.0)
    x1 = x0 + v0
    better = np.array([oracle_mod.f("rosenbrock", a) < oracle_mod.f("rosenbrock", b) for a, b in zip(x1, x0)])
    pb = np.where(better[:, None], x1, x0)
    r1 = np.array([[_u(seed, 4, i, j) for j in range(d)] for i in range(n)])
    v2 = v0 + c1 * r1 * (pb - x1)
    np.testing.assert_allclose(r["v"], v2, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(r["x"], x1 + v2, rtol=1e-12, atol=1e-12)


def test_personal_bests_monotone_and_consistent(oracle_mod):
    prev = None
    for T in range(0, 7):
        p = oracle_mod.Problem("rastrigin", dim=6, lower=-5.12, upper=5.12, n_starts=64, pso_iters=T, seed=3)
        r = oracle_mod.pso(p)
        assert np.array_equal(r["pf"], [oracle_mod.f("rastrigin", xi) for xi in r["px"]])
        assert r["gf"] == r["pf"].min() and np.array_equal(r["gx"], r["px"][r["gidx"]])
        if prev is not None:
            assert np.all(r["pf"] <= prev)
        prev = r["pf"]


def test_single_particle(oracle_mod):
    p = oracle_mod.Problem("ackley", dim=3, n_starts=1, pso_iters=6, seed=5)
    r = oracle_mod.pso(p)
    assert r["gidx"] == 0 and np.array_equal(r["gx"], r["px"][0])


def test_argmin_brute_force(oracle_mod):
    rng = np.random.default_rng(0)
    for n in (1, 2, 31, 33, 1000):
        v = rng.integers(0, 5, size=n).astype(np.float64)  # many ties
        v[rng.random(n) < 0.2] = np.nan
        want = min(range(n), key=lambda i: (np.inf if np.isnan(v[i]) else v[i], i))
        assert oracle_mod.argmin(v) == want
    assert oracle_mod.argmin([np.nan, np.nan]) == 0
    assert oracle_mod.argmin([np.inf, 3.0, -np.inf, -np.inf]) == 2
