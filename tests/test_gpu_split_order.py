"""Bit-exact parity past 32 coordinates.  The oracle's readings fix the
order of the dot products of the BFGS step and of the objectives' sums for
d > 32 (32 strided chains and a fixed pairwise tree), and the kernels form
them that way: one lane (lane kernel, single-thread sweeps), one warp (the
block kernel's dot products and line-search sums), a warp per particle
(PSO, objective evaluation).  So values, gradients, swarms and whole BFGS
runs equal the oracle's bit for bit at these sizes too."""
import numpy as np
import pytest
import torch

from paper_2603_28770_gb300 import workloads
from parity import assert_bitwise, oracle_problem, to_np, zeus_problem

pytestmark = pytest.mark.gpu

BOX = {"rosenbrock": (-2.0, 2.0), "rastrigin": (-5.12, 5.12), "ackley": (-5.0, 5.0),
       "quadratic": (-3.0, 3.0)}


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


@pytest.mark.parametrize("obj", sorted(BOX))
@pytest.mark.parametrize("d", [33, 64, 100, 257])
def test_values_and_forward_gradients_bit_exact(z, ora, obj, d):
    lo, hi = BOX[obj]
    x = workloads.start_points(97, d, lo, hi, seed=d)
    f, g = z.objective(obj, torch.from_numpy(x).cuda(), grad=True, grad_mode="forward")
    fv = z.objective(obj, torch.from_numpy(x).cuda(), grad=False)
    f, g, fv = f.cpu().numpy(), g.cpu().numpy(), fv.cpu().numpy()
    for i in range(x.shape[0]):
        fo, go = ora.grad_forward(obj, x[i])
        assert f[i] == fo and fv[i] == fo, (i, f[i], fv[i], fo)
        assert np.array_equal(g[i], go), (i, np.abs(g[i] - go).max())


@pytest.mark.parametrize("obj,d,n,T", [("rastrigin", 33, 200, 4), ("ackley", 64, 130, 3),
                                       ("rosenbrock", 100, 65, 2), ("quadratic", 48, 77, 5)])
def test_pso_bit_exact(z, ora, obj, d, n, T):
    lo, hi = BOX[obj]
    case = dict(objective=obj, dim=d, lower=lo, upper=hi, n_starts=n, pso_iters=T, seed=d)
    g = z.pso(zeus_problem(z, case))
    o = ora.pso(oracle_problem(ora, case))
    for k in ("x", "v", "px", "pf"):
        assert np.array_equal(g[k].cpu().numpy(), o[k]), k
    assert g["gidx"] == o["gidx"]


@pytest.mark.parametrize("obj,d,mode", [("rastrigin", 40, 128), ("rosenbrock", 64, 128),
                                        ("ackley", 48, 128), ("quadratic", 100, 128),
                                        ("rastrigin", 33, 0), ("rosenbrock", 36, 0)])
def test_bfgs_runs_bit_exact(z, ora, obj, d, mode):
    # one block per start (128) or the automatic plan (block per start at
    # these d; one lane per start does not fit an FP64 start past d = 29):
    # the oracle's bits, start by start
    lo, hi = BOX[obj]
    n = 48
    x0 = workloads.start_points(n, d, lo, hi, seed=3 * d + mode)
    fields = dict(objective=obj, dim=d, n_starts=n, bfgs_max_iters=60, threads_per_start=mode)
    g = to_np(z.solve_from(zeus_problem(z, fields), torch.from_numpy(x0).cuda()))
    o = ora.bfgs_many(oracle_problem(ora, fields), x0)
    assert_bitwise(g, o)
    assert g["summary"]["total_feval"] == int(o["n_feval"].sum())


def test_whole_method_bit_exact_past_32(z, ora):
    # PSO, BFGS from every particle, argmin at d = 40
    fields = dict(objective="rastrigin", dim=40, lower=-5.12, upper=5.12, n_starts=96,
                  pso_iters=3, bfgs_max_iters=40, seed=17)
    g = to_np(z.solve(zeus_problem(z, fields)))
    o = ora.solve(oracle_problem(ora, fields))
    assert_bitwise(g, o)
    assert g["summary"]["best_index"] == o["best"]
