"""The FP32 form with FP64 guards under the problem's own gradient tolerance
(1e-8, out of reach at FP32 resolution): its runs end on the stall test
(status 4, an iteration whose decrease of f FP32 cannot resolve) or on the
gradient test, close to where the FP64 oracle's runs end.  Per start, the
FP64 value at the FP32 run's final point is compared with the oracle's final
value; the success rate (f within 1e-6 of the known minimum) must lie in the
oracle's 95 % Clopper-Pearson interval; and the runs must not carry on to
the iteration cap where the FP64 method stops."""
import numpy as np
import pytest
import torch

from paper_2603_28770_gb300 import workloads
from parity import clopper_pearson, oracle_problem, to_np, zeus_problem

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


# (objective, d, starts, box, cap, layouts, share of starts that must end
# within the tolerance of the FP64 oracle's value).  The FP32 form states
# its error per start rather than bounding it: a start can end in another
# local minimum.  At d = 256 about 86 % of 128 uniform starts end with the
# FP64 method (the same share for the streamed kernel's row and tiled
# layouts of H, measured); 32 starts resolve such a share only to about
# +-10 %, so that case takes 128 starts and a bar of 0.8.
CASES = [("rastrigin", 10, 2000, -5.12, 5.12, 1000, (0, 1, 128), 0.9),
         ("rastrigin", 5, 2000, -5.12, 5.12, 1000, (0,), 0.9),
         ("rosenbrock", 2, 1000, -5.0, 5.0, 1000, (0, 1, 128), 0.9),
         ("ackley", 6, 1000, -5.0, 5.0, 1000, (0,), 0.85),
         ("rosenbrock", 40, 128, -2.0, 2.0, 2000, (0,), 0.9),
         ("rosenbrock", 256, 128, -2.0, 2.0, 3000, (0,), 0.8)]
PARAMS = [(o, d, n, lo, hi, K, lay, need) for (o, d, n, lo, hi, K, lays, need) in CASES
          for lay in lays]


@pytest.mark.parametrize("obj,d,n,lo,hi,K,layout,need", PARAMS)
def test_fp32_runs_end_where_fp64_runs_end(z, ora, obj, d, n, lo, hi, K, layout, need):
    x0 = workloads.start_points(n, d, lo, hi, seed=17 * n + d)
    base = dict(objective=obj, dim=d, lower=lo, upper=hi, n_starts=n, bfgs_max_iters=K)
    g = to_np(z.solve_from(zeus_problem(z, base, precision="fp32_guarded", threads_per_start=layout),
                           torch.from_numpy(x0).cuda()))
    o = ora.bfgs_many(oracle_problem(ora, base), x0)
    st = g["status"]
    assert set(np.unique(st)) <= {0, 1, 4}
    # the stall test ends the runs: far fewer reach the cap than would
    # without it, and no more than the FP64 method's share plus a little
    capped32, capped64 = float(np.mean(st == 0)), float(np.mean(o["status"] == 0))
    assert capped32 <= capped64 + 0.05, (capped32, capped64)
    assert int(g["iters"].sum()) <= 3 * int(o["iters"].sum()) + 10 * n
    # per start: the FP64 value at the FP32 point against the oracle's value
    err = np.abs(g["f"] - o["f"]) / np.maximum(1.0, np.abs(o["f"]))
    tol = 1e-3 if obj == "ackley" else 1e-5
    assert (err <= tol).mean() >= need, f"{int((err > tol).sum())} of {n}; median {np.median(err):.2e}"
    k_o = int((o["f"] <= 1e-6).sum())
    lo_, hi_ = clopper_pearson(k_o, n)
    rate = float((g["f"] <= 1e-6).mean())
    assert lo_ - 1e-12 <= rate <= hi_ + 1e-12, (rate, k_o, lo_, hi_)


def test_fp64_form_never_stalls(z):
    # the stall test belongs to the FP32 form only: the FP64 method keeps
    # the paper's tests (a start ends on ||g|| < tol or the cap)
    x0 = torch.from_numpy(workloads.start_points(2000, 10, -5.12, 5.12, seed=3)).cuda()
    p = zeus_problem(z, dict(objective="rastrigin", dim=10, n_starts=2000, bfgs_max_iters=1000))
    g = to_np(z.solve_from(p, x0))
    assert not (g["status"] == 4).any()


def test_precision_error_per_start(z):
    # the per-start comparison of the two precisions the package reports:
    # FP32 form and FP64 method from the same starts
    p = z.Problem(objective="rosenbrock", dim=2, n_starts=256, bfgs_max_iters=500, seed=1)
    x0 = torch.from_numpy(workloads.start_points(256, 2, -5.0, 5.0, seed=1)).cuda()
    r = z.precision_error(p, x0)
    assert r["abs_f"].shape == (256,) and r["rel_x"].shape == (256,)
    assert np.all(np.isfinite(r["abs_f"]))
    assert np.median(r["abs_f"]) < 1e-6
    s = r["summary"]
    assert s["starts"] == 256 and 0.0 <= s["within_1e-6"] <= 1.0
