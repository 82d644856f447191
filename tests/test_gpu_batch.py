"""GPU tests of the batched form (zeus_batch_*): many problems of mixed
objective, dimension, swarm size and PSO length solved by one fixed
sequence of launches.  Each problem's outputs must equal, bit for bit, those
of its own zeus_solve (which the parity tests pin to the oracle), the
oracle itself within the parity tolerance, and a CUDA-graph replay."""
import math

import numpy as np
import pytest
import torch

from paper_2603_28770_gb300 import workloads
from parity import assert_bitwise, compare_runs, oracle_problem, to_np

pytestmark = pytest.mark.gpu

SUMMARY_KEYS = ("best_f", "best_index", "n_converged", "total_iters", "total_feval", "gbest_f",
                "gbest_index", "error", "stop_flag")

BOX = dict(workloads.BOXES, goldstein_price=(-2.0, 2.0), quadratic=(-3.0, 3.0))

# (objective, d, N, PSO updates, BFGS cap, extra fields): lane tiles with
# and without hand-over, block-per-start problems, ragged N (1, 129, 257),
# no PSO update, start from the personal bests, forced kernel choices
# (one lane, one block or one warp per start)
CASES = [
    ("rosenbrock", 2, 130, 5, 200, {}),
    ("rastrigin", 10, 300, 3, 400, {}),
    ("ackley", 17, 40, 2, 60, {}),
    ("rastrigin", 33, 24, 0, 50, {}),
    ("goldstein_price", 2, 1, 4, 30, {}),
    ("quadratic", 5, 129, 1, 30, {}),
    ("rosenbrock", 64, 9, 2, 40, {}),
    ("ackley", 3, 257, 2, 100, {"start_from_pbest": 1}),
    ("rastrigin", 1, 77, 3, 50, {}),
    ("rosenbrock", 16, 100, 2, 300, {}),
    ("rastrigin", 20, 50, 1, 40, {"threads_per_start": 1}),
    ("ackley", 5, 60, 2, 40, {"threads_per_start": 128}),
    ("rosenbrock", 12, 70, 2, 200, {"threads_per_start": 32}),
    ("ackley", 40, 30, 1, 50, {"threads_per_start": 32}),
    ("rastrigin", 3, 101, 2, 100, {"threads_per_start": 32}),
]


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


def _fields(obj, d, n, t, k, extra, seed):
    lo, hi = BOX[obj]
    f = dict(objective=obj, dim=d, lower=lo, upper=hi, n_starts=n, pso_iters=t, bfgs_max_iters=k,
             seed=seed)
    f.update(extra)
    return f


def _problems(z, **kw):
    return [z.Problem(**_fields(*c, seed=101 + i), **kw) for i, c in enumerate(CASES)]


def _check_against_single(z, batch, probs, P):
    got = batch.problem(P)
    want = z.solve(probs[P])
    assert_bitwise(to_np(got), to_np(want))
    for k in SUMMARY_KEYS:
        a, b = got["summary"][k], want["summary"][k]
        assert a == b or (isinstance(a, float) and math.isnan(a) and math.isnan(b)), (P, k, a, b)


@pytest.mark.parametrize("precision", ["fp64", "fp32_guarded"])
@pytest.mark.parametrize("grad_mode", ["forward", "adjoint"])
def test_batch_equals_single_solves(z, precision, grad_mode):
    probs = _problems(z, precision=precision, grad_mode=grad_mode)
    b = z.Batch(probs)
    assert b.plan.q_cap > 0 and b.plan.n_classes >= 2
    b.solve()
    torch.cuda.synchronize()
    for P in range(len(probs)):
        _check_against_single(z, b, probs, P)


# L-BFGS problems (one 256-thread block per start, classes of their own)
LBFGS_CASES = [
    ("rosenbrock", 12, 70, 2, 100, {"lbfgs_m": 5}),
    ("ackley", 40, 20, 1, 60, {"lbfgs_m": 3}),
    ("rastrigin", 10, 33, 2, 80, {"lbfgs_m": 7}),
    ("quadratic", 200, 5, 0, 40, {"lbfgs_m": 9}),
    ("rosenbrock", 300, 3, 1, 30, {"lbfgs_m": 2, "start_from_pbest": 1}),
]


@pytest.mark.parametrize("precision", ["fp64", "fp32_guarded"])
@pytest.mark.parametrize("grad_mode", ["forward", "adjoint"])
def test_batch_with_lbfgs_problems(z, precision, grad_mode):
    # L-BFGS problems beside dense ones in one batch: each problem equals
    # its own zeus_solve bit for bit (the batch runs the single-problem
    # L-BFGS body per start)
    kw = dict(precision=precision, grad_mode=grad_mode)
    probs = _problems(z, **kw)[:7]
    probs += [z.Problem(**_fields(*c, seed=301 + i), **kw) for i, c in enumerate(LBFGS_CASES)]
    b = z.Batch(probs)
    kinds = list(b.plan.class_kind[: b.plan.n_classes])
    assert kinds[0] == 3 and kinds == sorted(kinds, reverse=True)
    b.solve()
    torch.cuda.synchronize()
    for P in range(len(probs)):
        _check_against_single(z, b, probs, P)


def test_batch_against_oracle(z, ora):
    # the oracle runs the whole method of each small problem of the batch
    probs = _problems(z)
    b = z.Batch(probs)
    b.solve()
    for P, c in enumerate(CASES):
        if c[1] * c[2] > 3000:
            continue
        g = to_np(b.problem(P))
        o = ora.solve(oracle_problem(ora, _fields(*c, seed=101 + P)))
        compare_runs(g, o, rtol=1e-8, max_flip_frac=0.05)
        assert g["summary"]["best_index"] == o["best"]


def test_batch_graph_replay(z):
    probs = _problems(z)
    b = z.Batch(probs)
    b.solve()
    torch.cuda.synchronize()
    ref = {k: getattr(b, k).clone() for k in ("x", "f", "gnorm", "status", "iters", "results")}
    b.capture()
    for _ in range(2):
        for k in ("x", "f", "gnorm", "status", "iters", "results"):
            getattr(b, k).zero_()
        b.replay()
        torch.cuda.synchronize()
        for k, v in ref.items():
            assert torch.equal(getattr(b, k), v), k


def test_batch_stop_flag_is_per_problem(z):
    # a target on one problem (2-D Rosenbrock, reached by many starts) raises
    # only that problem's stop flag; the others are untouched
    probs = _problems(z)
    probs[0] = probs[0].replace(target_f=1e-6)
    b = z.Batch(probs)
    b.solve()
    torch.cuda.synchronize()
    s0 = b.problem(0)
    assert s0["summary"]["stop_flag"] == 1 and s0["summary"]["best_f"] <= 1e-6
    assert (s0["status"] == 2).any().item() or (s0["status"] == 1).all().item()
    for P in range(1, len(probs)):
        _check_against_single(z, b, probs, P)
        assert b.problem(P)["summary"]["stop_flag"] == 0


def test_batch_mixed_workload_sampled(z):
    # the mixed-problem generator of the batched benchmark (d log-uniform in
    # [2, 128], Rosenbrock / Rastrigin / Ackley) at reduced count; a sample
    # of problems checked against their own solves
    mix = workloads.mixed_batch(192, seed=12345)
    probs = [z.Problem(**m, n_starts=64, pso_iters=10, bfgs_max_iters=200, seed=P)
             for P, m in enumerate(mix)]
    b = z.Batch(probs)
    b.solve()
    torch.cuda.synchronize()
    rng = np.random.default_rng(3)
    dims = np.array([p.dim for p in probs])
    sample = set(rng.choice(len(probs), 10, replace=False).tolist())
    sample |= {int(np.argmax(dims)), int(np.argmin(dims))}
    for P in sorted(sample):
        _check_against_single(z, b, probs, P)
    sums = b.summaries()
    assert sum(s["total_iters"] for s in sums) == int(b.iters.sum().item())
    assert all(s["error"] == 0 for s in sums)


def test_autotuned_batch_is_bitwise_the_same(z, tmp_path):
    # the tuner only moves starts between lane and block layouts: the
    # outputs of the tuned batch are those of the automatic one
    from paper_2603_28770_gb300.autotune import Autotuner
    probs = _problems(z)
    ref = z.Batch(probs)
    ref.solve()
    t = Autotuner(str(tmp_path / "tune.json"), probe_problems=2, probe_starts=32, reps=1, probe_total=256)
    b = z.Batch(probs, autotuner=t)
    assert t.table[t.device_name()]
    b.solve()
    torch.cuda.synchronize()
    for k in ("x", "f", "gnorm", "status", "iters", "results"):
        assert torch.equal(getattr(b, k), getattr(ref, k)), k
