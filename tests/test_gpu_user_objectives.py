"""GPU parity of user objectives (Section IV-A: f written once for any scalar
type, differentiated on dual numbers by Alg. 5): the two objectives of the
default plug-in, Griewank and Himmelblau, through every form that takes
them (lane tiles with hand-over, block per start, the fused cooperative
launch, FP32 with FP64 guards, the batch) against the oracle's own
implementation.

Himmelblau is a polynomial: with every product and sum rounded once in the
same order on both sides its runs are bit-exact.  Griewank goes through
cosines, which CUDA's and the host's math libraries round differently in
the last bit, so it is compared within the parity tolerance (tests/parity.py)."""
import math

import numpy as np
import pytest
import torch

from paper_2603_28770_gb300 import workloads
from parity import assert_bitwise, compare_runs, oracle_problem, to_np, zeus_problem

pytestmark = pytest.mark.gpu

HIMMELBLAU_MINIMA = np.array([[3.0, 2.0], [-2.805118, 3.131312],
                              [-3.779310, -3.283186], [3.584428, -1.848126]])


@pytest.fixture(scope="module")
def z():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2603_28770_gb300 as z
    z.lib()
    assert set(z.user_objectives()) == {"griewank", "himmelblau"}
    return z


@pytest.fixture(scope="module")
def ora():
    import oracle
    oracle.build()
    return oracle


def test_objective_values_and_gradients(z, ora):
    rng = np.random.default_rng(3)
    for obj, d, box in (("himmelblau", 2, 5.0), ("griewank", 1, 50.0), ("griewank", 13, 50.0)):
        x = rng.uniform(-box, box, (257, d))
        f, g = z.objective(obj, torch.from_numpy(x).cuda())
        f, g = f.cpu().numpy(), g.cpu().numpy()
        want = [ora.grad_forward(obj, xi) for xi in x]
        wf = np.array([w[0] for w in want])
        wg = np.array([w[1] for w in want])
        if obj == "himmelblau":
            assert np.array_equal(f, wf) and np.array_equal(g, wg)
        else:
            assert np.abs(f - wf).max() <= 1e-14 * max(1.0, np.abs(wf).max())
            assert np.abs(g - wg).max() <= 1e-13 * max(1.0, np.abs(wg).max())
        f32, g32 = z.objective(obj, torch.from_numpy(x).float().cuda())
        assert np.abs(f32.cpu().numpy() - wf).max() <= 1e-5 * max(1.0, np.abs(wf).max())
        assert np.abs(g32.cpu().numpy() - wg).max() <= 1e-4 * max(1.0, np.abs(wg).max())
    with pytest.raises(z.ZeusError):  # forward mode only
        z.objective("griewank", torch.zeros(4, 3, dtype=torch.float64, device="cuda"),
                    grad_mode="adjoint")


def test_himmelblau_whole_method_bit_exact(z, ora):
    # PSO, BFGS from every particle (lane tiles), argmin: the oracle's bits
    fields = dict(objective="himmelblau", dim=2, lower=-5.0, upper=5.0, n_starts=1000,
                  pso_iters=5, bfgs_max_iters=200, seed=9)
    g = to_np(z.solve(zeus_problem(z, fields)))
    o = ora.solve(oracle_problem(ora, fields))
    assert_bitwise(g, o)
    s = g["summary"]
    assert s["best_index"] == o["best"]
    assert s["gbest_index"] == ora.pso(oracle_problem(ora, fields))["gidx"]
    assert s["total_iters"] == int(o["iters"].sum())
    # the converged starts sit at the four minima, and all four are found
    ok = (g["status"] == 1) & (g["f"] < 1e-12)
    dist = np.linalg.norm(g["x"][ok][:, None, :] - HIMMELBLAU_MINIMA[None], axis=2)
    assert (dist.min(axis=1) < 1e-5).all()
    assert set(np.argmin(dist, axis=1).tolist()) == {0, 1, 2, 3}


def _n_apart(a, b):
    """Starts whose runs differ: status, iteration count, f beyond 1e-9
    relative or a coordinate beyond 1e-9 relative."""
    dx = np.abs(a["x"] - b["x"]).max(axis=1) / np.maximum(1.0, np.abs(b["x"]).max(axis=1))
    df = np.abs(a["f"] - b["f"]) / np.maximum(1.0, np.abs(b["f"]))
    return int(((a["status"] != b["status"]) | (a["iters"] != b["iters"]) | (df > 1e-9)
                | (dx > 1e-9)).sum())


def _ulp_spread(ora, fields, x0):
    """How far the oracle moves from itself when every start coordinate is
    moved by one unit in the last place (up, then down): the scale of the
    disagreement that last-bit differences alone cause along these runs."""
    prob = oracle_problem(ora, fields)
    o = ora.bfgs_many(prob, x0)
    up = ora.bfgs_many(prob, np.nextafter(x0, np.inf))
    down = ora.bfgs_many(prob, np.nextafter(x0, -np.inf))
    return o, max(_n_apart(up, o), _n_apart(down, o))


@pytest.mark.parametrize("d,n,mode", [(8, 700, 0), (8, 300, 1), (8, 96, 128), (40, 48, 0)])
@pytest.mark.parametrize("iters", [5, 20, 60])
def test_griewank_forms_against_oracle(z, ora, d, n, mode, iters):
    # mode 0: the automatic plan (lane tiles for d = 8, one block per start
    # for d = 40); 1: lanes only; 128: one block per start.  The cosines of
    # CUDA's and the host's math libraries differ in the last bit, and
    # BFGS on this flat, coupled function amplifies last-bit differences
    # (the curvature y's is small against |y||s|): the CUDA path may be as
    # far from the oracle as the oracle is from itself after a one-ulp move
    # of the starts, and no farther
    x0 = workloads.start_points(n, d, -20.0, 20.0, seed=d + n)
    fields = dict(objective="griewank", dim=d, n_starts=n, bfgs_max_iters=iters,
                  threads_per_start=mode)
    g = to_np(z.solve_from(zeus_problem(z, fields), torch.from_numpy(x0).cuda()))
    o, spread = _ulp_spread(ora, fields, x0)
    apart = _n_apart(g, o)
    assert apart <= 2 * spread + max(2, n // 100), (apart, spread)
    assert g["summary"]["best_index"] == ora.argmin(g["f"])


def test_griewank_long_runs_through_the_handover(z, ora):
    # whole runs, with starts that pass the lane kernel's budget of 160
    # iterations and line-search evaluations (the fused launch serves them):
    # the same bar, and every start that converged to the same point on
    # both sides has the same f to 1e-12
    d, n = 12, 400
    x0 = workloads.start_points(n, d, -60.0, 60.0, seed=5)
    fields = dict(objective="griewank", dim=d, n_starts=n, bfgs_max_iters=400)
    assert z.zeus_plan_info(zeus_problem(z, fields))["handover"] == 1
    g = to_np(z.solve_from(zeus_problem(z, fields), torch.from_numpy(x0).cuda()))
    o, spread = _ulp_spread(ora, fields, x0)
    assert ((o["iters"] + o["n_feval"]) > 160).sum() >= 40
    apart = _n_apart(g, o)
    assert apart <= 2 * spread + 4, (apart, spread)
    both = (g["status"] == 1) & (o["status"] == 1) & (np.abs(g["x"] - o["x"]).max(axis=1) <= 1e-6)
    assert both.sum() > n // 2
    assert np.all(np.abs(g["f"][both] - o["f"][both]) <= 1e-12)


@pytest.mark.parametrize("obj,d", [("griewank", 10), ("himmelblau", 2)])
def test_fp32_guarded_form(z, ora, obj, d):
    # FP32 objective, gradient and H with FP64 guards: the final f (an FP64
    # evaluation at the FP32 point) is close to the FP64 oracle's for most
    # starts over the first iterations
    x0 = workloads.start_points(256, d, -5.0, 5.0, seed=17)
    fields = dict(objective=obj, dim=d, n_starts=256, bfgs_max_iters=8)
    g = to_np(z.solve_from(zeus_problem(z, fields, precision="fp32_guarded"),
                           torch.from_numpy(x0).cuda()))
    o = ora.bfgs_many(oracle_problem(ora, fields), x0)
    err = np.abs(g["f"] - o["f"]) / np.maximum(1.0, np.abs(o["f"]))
    assert np.isfinite(g["f"]).all() and (err <= 1e-3).mean() >= 0.9, err


@pytest.mark.parametrize("precision", ["fp64", "fp32_guarded"])
def test_batch_with_user_objectives_equals_single_solves(z, ora, precision):
    probs = [z.Problem(objective="griewank", dim=7, lower=-10, upper=10, n_starts=200,
                       pso_iters=2, bfgs_max_iters=300, seed=1, precision=precision),
             z.Problem(objective="rastrigin", dim=4, lower=-5.12, upper=5.12, n_starts=150,
                       pso_iters=3, bfgs_max_iters=100, seed=2, precision=precision),
             z.Problem(objective="himmelblau", dim=2, lower=-5, upper=5, n_starts=129,
                       pso_iters=1, bfgs_max_iters=100, seed=3, precision=precision),
             z.Problem(objective="griewank", dim=48, lower=-5, upper=5, n_starts=10,
                       pso_iters=1, bfgs_max_iters=40, seed=4, precision=precision)]
    b = z.Batch(probs)
    assert b.plan.n_user == 3
    b.solve()
    torch.cuda.synchronize()
    for P, p in enumerate(probs):
        got, want = to_np(b.problem(P)), to_np(z.solve(p))
        assert_bitwise(got, want)
        for k in ("best_index", "total_iters", "total_feval", "gbest_index"):
            assert got["summary"][k] == want["summary"][k], (P, k)
    if precision == "fp64":  # the polynomial problem against the oracle's bits
        o = ora.solve(oracle_problem(ora, {f: getattr(probs[2], f) for f in
                                           ("objective", "dim", "lower", "upper", "n_starts",
                                            "pso_iters", "bfgs_max_iters", "seed")}))
        assert_bitwise(to_np(b.problem(2)), o)


def test_autograd_function_with_a_user_objective(z, ora):
    x = torch.tensor([[0.5, -1.0, 2.0], [3.0, 0.1, -0.2]], dtype=torch.float64, device="cuda",
                     requires_grad=True)
    y = z.ObjectiveFn.apply(x, "griewank", "forward")
    y.sum().backward()
    for i in range(2):
        fv, gv = ora.grad_forward("griewank", x[i].detach().cpu().numpy())
        assert math.isclose(y[i].item(), fv, rel_tol=1e-14, abs_tol=1e-15)
        assert np.allclose(x.grad[i].cpu().numpy(), gv, rtol=1e-13, atol=1e-15)
