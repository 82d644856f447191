"""The shared stop flag of Alg. 10 on the GPU against the oracle.

When the flag is raised (required_c converged starts, or a start at the
target value) the starts still running stop at the top of their next
iteration, on whichever SM they run; which ones that is depends on timing,
so it is not compared start by start.  What is unique is compared: a start
that ended converged (status 1) followed the same trajectory as without
the flag, so its outputs equal the oracle's run without the flag bit for
bit; a start the flag stopped (status 2) after k iterations is exactly the
oracle's iterate k of that start (checked on a sample with the oracle's
iteration cap set to k); the counts reach the requested number."""
import numpy as np
import pytest
import torch

from paper_2603_28770_gb300 import workloads
from parity import oracle_problem, to_np, zeus_problem

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def z():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2603_28770_gb300 as z
    z.lib()
    return z


@pytest.fixture(scope="module")
def ora():
    import oracle
    oracle.build()
    return oracle


def _check_stopped_run(z, ora, fields, x0, g):
    free = ora.bfgs_many(oracle_problem(ora, fields), x0)
    st = g["status"]
    assert set(np.unique(st)) <= {0, 1, 2, 3}
    conv = np.flatnonzero(st == 1)
    for k in ("x", "f", "gnorm", "iters", "status"):
        a, b = np.asarray(g[k])[conv], np.asarray(free[k])[conv]
        assert np.array_equal(a, b), k
    stopped = np.flatnonzero(st == 2)
    assert (g["iters"][stopped] <= free["iters"][stopped]).all()
    rng = np.random.default_rng(1)
    for i in rng.choice(stopped, size=min(24, stopped.size), replace=False) if stopped.size else []:
        k = int(g["iters"][i])
        one = ora.bfgs(oracle_problem(ora, fields, bfgs_max_iters=k), x0[i])
        assert np.array_equal(one["x"], g["x"][i]) and one["f"] == g["f"][i], (i, k)
    return free


@pytest.mark.parametrize("layout,R", [(0, 50), (1, 200), (128, 30), (0, 1)])
def test_required_converged_against_oracle(z, ora, layout, R):
    n, d = 3000, 4
    x0 = workloads.start_points(n, d, -5.12, 5.12, seed=44)
    fields = dict(objective="rastrigin", dim=d, lower=-5.12, upper=5.12, n_starts=n,
                  bfgs_max_iters=200, threads_per_start=layout)
    g = to_np(z.solve_from(zeus_problem(z, fields, required_converged=R), torch.from_numpy(x0).cuda()))
    s = g["summary"]
    assert s["stop_flag"] == 1
    assert s["n_converged"] >= R and s["n_converged"] == int((g["status"] == 1).sum())
    free = _check_stopped_run(z, ora, fields, x0, g)
    # without the flag the GPU run equals the oracle's whole
    g0 = to_np(z.solve_from(zeus_problem(z, fields), torch.from_numpy(x0).cuda()))
    for k in ("x", "f", "gnorm", "iters", "status"):
        assert np.array_equal(np.asarray(g0[k]), np.asarray(free[k])), k


def test_target_f_against_oracle(z, ora):
    # 2-D Rosenbrock from uniform starts: most runs pass below the target
    n, d = 2000, 2
    x0 = workloads.start_points(n, d, -5.0, 5.0, seed=45)
    fields = dict(objective="rosenbrock", dim=d, lower=-5.0, upper=5.0, n_starts=n,
                  bfgs_max_iters=300)
    g = to_np(z.solve_from(zeus_problem(z, fields, target_f=1e-6), torch.from_numpy(x0).cuda()))
    s = g["summary"]
    assert s["stop_flag"] == 1 and s["best_f"] <= 1e-6
    # a start ends converged on the gradient test (then it followed its
    # trajectory without the flag) or at f <= target
    free = ora.bfgs_many(oracle_problem(ora, fields), x0)
    conv = np.flatnonzero(g["status"] == 1)
    by_grad = conv[g["f"][conv] > 1e-6]
    assert np.array_equal(g["x"][by_grad], free["x"][by_grad])
    assert np.array_equal(g["iters"][by_grad], free["iters"][by_grad])
    hit = conv[g["f"][conv] <= 1e-6]
    assert hit.size >= 1
    for i in hit[:16]:
        # the oracle's run of the same start with the same target stops at
        # the same iterate (its first f <= 1e-6 or convergence)
        one = ora.bfgs(oracle_problem(ora, fields, target_f=1e-6), x0[i])
        assert one["iters"] == g["iters"][i] and np.array_equal(one["x"], g["x"][i])
    stopped = np.flatnonzero(g["status"] == 2)
    assert (g["iters"][stopped] <= free["iters"][stopped]).all()
