"""Pins of the oracle's branches that only change which starts run on:
the shared stop flag of Alg. 10 (required_c converged starts, or a target
value reached), the non-descent restart of the direction step (reading:
H <- I, p = -g when g'p < 0 fails) and the choice of BFGS start points
(the swarm's current positions, or the personal bests).

With one OpenMP thread the oracle runs the starts in index order, so the
flag's effect is fixed: every start after the one that raised it stops at
its first test (status 2, no iteration, x = x0)."""
import numpy as np
import pytest

from paper_2603_28770_gb300 import workloads


def _starts(n, d, lo=-3.0, hi=3.0, seed=5):
    return workloads.start_points(n, d, lo, hi, seed)


@pytest.mark.parametrize("order", [0, 1])
@pytest.mark.parametrize("R", [1, 7, 20])
def test_required_converged_stops_after_exactly_r(oracle_mod, R, order):
    # the quadratic objective: every start converges, so the first R starts
    # converge (status 1) and the flag stops every later one at once
    n, d = 32, 6
    x0 = _starts(n, d)
    p = oracle_mod.Problem("quadratic", dim=d, n_starts=n, bfgs_max_iters=200,
                           required_converged=R, n_threads=1, order=order)
    r = oracle_mod.bfgs_many(p, x0)
    assert np.array_equal(r["status"][:R], np.ones(R, dtype=np.int32))
    assert (r["iters"][:R] > 0).all()
    assert np.array_equal(r["status"][R:], np.full(n - R, 2, dtype=np.int32))
    assert (r["iters"][R:] == 0).all() and np.array_equal(r["x"][R:], x0[R:])


def test_required_converged_off_runs_every_start(oracle_mod):
    n, d = 16, 6
    x0 = _starts(n, d)
    p = oracle_mod.Problem("quadratic", dim=d, n_starts=n, bfgs_max_iters=200,
                           required_converged=0, n_threads=1)
    r = oracle_mod.bfgs_many(p, x0)
    assert (r["status"] == 1).all()


def test_required_converged_counts_only_converged_starts(oracle_mod):
    # starts that reach the iteration cap (status 0) do not count toward R:
    # with a cap of 2 iterations on 2-D Rosenbrock most starts stop at the
    # cap, and the flag is raised only by the R-th start that converges
    n = 64
    x0 = _starts(n, 2, -2.0, 2.0, seed=8)
    free = oracle_mod.bfgs_many(oracle_mod.Problem("rosenbrock", dim=2, n_starts=n,
                                                   bfgs_max_iters=30, n_threads=1), x0)
    conv = np.flatnonzero(free["status"] == 1)
    assert len(conv) >= 3
    R = 2
    r = oracle_mod.bfgs_many(oracle_mod.Problem("rosenbrock", dim=2, n_starts=n, bfgs_max_iters=30,
                                                required_converged=R, n_threads=1), x0)
    last = conv[R - 1]  # the start whose convergence raises the flag
    assert np.array_equal(r["status"][:last + 1], free["status"][:last + 1])
    assert (r["status"][last + 1:] == 2).all() and (r["iters"][last + 1:] == 0).all()


def _f_after(oracle_mod, obj, d, x, K):
    p = oracle_mod.Problem(obj, dim=d, n_starts=1, bfgs_max_iters=K, n_threads=1)
    return oracle_mod.bfgs(p, x)


def test_target_f_stops_at_the_first_iterate_at_or_below_it(oracle_mod):
    # target = f of start 0's iterate 5 exactly: the test is f <= target, so
    # start 0 stops at iteration 5 (status 1), and every later start at once
    n, d = 12, 2
    x0 = _starts(n, d, -2.0, 2.0, seed=3)
    traj = [_f_after(oracle_mod, "rosenbrock", d, x0[0], K) for K in range(7)]
    fk = [t["f"] for t in traj]
    assert all(t["status"] == 0 for t in traj[1:]) and all(np.diff(fk) < 0)
    target = fk[5]
    p = oracle_mod.Problem("rosenbrock", dim=d, n_starts=n, bfgs_max_iters=100, target_f=target,
                           n_threads=1)
    r = oracle_mod.bfgs_many(p, x0)
    assert r["status"][0] == 1 and r["iters"][0] == 5 and r["f"][0] == target
    assert (r["status"][1:] == 2).all() and (r["iters"][1:] == 0).all()
    assert np.array_equal(r["x"][1:], x0[1:])


def test_target_f_nan_is_off(oracle_mod):
    n, d = 8, 2
    x0 = _starts(n, d, -2.0, 2.0, seed=3)
    a = oracle_mod.bfgs_many(oracle_mod.Problem("rosenbrock", dim=d, n_starts=n, bfgs_max_iters=100,
                                                n_threads=1), x0)
    assert not (a["status"] == 2).any()


# ------------------------------------------------------- non-descent restart

@pytest.mark.parametrize("order", [0, 1])
def test_direction_resets_on_a_non_descent_h(oracle_mod, order):
    g = np.array([0.5, -1.25, 2.0, 0.75])
    d = g.size
    for H in (-np.eye(d), np.zeros((d, d)), np.diag([1.0, 1.0, -10.0, 1.0])):
        p, Ha, dd, reset = oracle_mod.direction(H, g, order=order)
        assert reset
        assert np.array_equal(p, -g)
        assert np.array_equal(Ha, np.eye(d))
        assert dd == -float(np.sum(g * g))  # dyadic values: exact in any order


@pytest.mark.parametrize("order", [0, 1])
def test_direction_keeps_a_descent_h(oracle_mod, order):
    g = np.array([0.5, -1.25, 2.0, 0.75])
    H = np.diag([2.0, 0.5, 1.0, 4.0])
    H[0, 1] = H[1, 0] = 0.25
    p, Ha, dd, reset = oracle_mod.direction(H, g, order=order)
    assert not reset and np.array_equal(Ha, H)
    assert np.array_equal(p, -(H @ g))  # dyadic values: exact
    assert dd == float(g @ p) and dd < 0


def test_direction_resets_on_nan(oracle_mod):
    g = np.array([1.0, 2.0])
    H = np.array([[np.nan, 0.0], [0.0, 1.0]])
    p, Ha, dd, reset = oracle_mod.direction(H, g)
    assert reset and np.array_equal(p, -g) and np.array_equal(Ha, np.eye(2)) and dd == -5.0


# ------------------------------------------------------- BFGS start points

@pytest.mark.parametrize("pbest", [0, 1])
def test_start_points_current_or_personal_best(oracle_mod, pbest):
    # with no BFGS iteration the run returns its start point and f there:
    # the personal best (and its value pF, Alg. 3) or the current position
    fields = dict(objective="rastrigin", dim=3, lower=-5.12, upper=5.12, n_starts=64, pso_iters=4,
                  bfgs_max_iters=0, seed=2)
    r = oracle_mod.solve(oracle_mod.Problem(**fields, start_from_pbest=pbest))
    sw = oracle_mod.pso(oracle_mod.Problem(**fields))
    assert not np.array_equal(sw["x"], sw["px"])  # the two choices differ here
    if pbest:
        assert np.array_equal(r["x"], sw["px"]) and np.array_equal(r["f"], sw["pf"])
    else:
        assert np.array_equal(r["x"], sw["x"])
        assert np.array_equal(r["f"], [oracle_mod.f("rastrigin", xi) for xi in sw["x"]])
    assert (r["iters"] == 0).all()
