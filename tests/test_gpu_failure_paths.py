"""Failure paths, exercised without faulting the GPU.

* Bounded device waits: with zeus_set_wait_limit(1) the servers of the
  fused BFGS launch and the blocks at the clustering kernel's grid barrier
  give up after one or two polls.  The kernel must return with its error
  word set (the host-buffer call reports ZEUS_ETIMEOUT), and the next call
  with the default limit must run normally and give the usual results.
* Non-finite values in mid-run: Rosenbrock starts scaled by 10^3 overflow
  after several iterations (status 3) while the starts beside them in the
  same lane tile run on; statuses, iteration counts and outputs equal the
  oracle's bit for bit (||g|| of a non-finite end compared as non-finite).
"""
import numpy as np
import pytest
import torch

from paper_2603_28770_gb300 import workloads
from parity import assert_bitwise, oracle_problem, to_np, zeus_problem

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def z():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2603_28770_gb300 as z
    z.lib()
    yield z
    z.zeus_set_wait_limit(0)


@pytest.fixture(scope="module")
def ora():
    import oracle
    oracle.build()
    return oracle


def _handover_problem(z):
    # 10-D Rastrigin with the automatic layout: lane tiles plus the
    # hand-over service in one cooperative launch; 4096 starts make fewer
    # tiles than resident blocks, so most blocks start out as servers
    fields = workloads.workload("rastrigin10d_n16384", n_starts=4096, bfgs_max_iters=1000)
    p = zeus_problem(z, fields)
    plan = z.zeus_plan_info(p)
    assert plan["narrow"] == 1 and plan["handover"] == 1
    return p


def test_fused_kernel_wait_runs_out_then_recovers(z):
    p = _handover_problem(z)
    x0 = torch.from_numpy(workloads.start_points(p.n_starts, p.dim, -5.12, 5.12, seed=9)).cuda()
    ref = to_np(z.solve_from(p, x0))
    assert ref["summary"]["error"] == 0
    try:
        z.zeus_set_wait_limit(1)
        out = z.solve_from(p, x0)  # synchronizes: the kernel returned
        assert out["summary"]["error"] == 1
        # the host-buffer entry point reports the expired wait
        ctx = z.Context()
        n, d = p.n_starts, p.dim
        hx = torch.empty(n, d, dtype=torch.float64)
        with pytest.raises(z.ZeusError) as ei:
            ctx.zeus_solve_host(p, hx)
        assert ei.value.code == -4  # ZEUS_ETIMEOUT
        ctx.close()
    finally:
        z.zeus_set_wait_limit(0)
    again = to_np(z.solve_from(p, x0))
    assert again["summary"]["error"] == 0
    assert_bitwise(again, ref)


def test_cluster_barrier_wait_runs_out_then_recovers(z, ora):
    n, d = 1 << 16, 4
    rng = np.random.default_rng(3)
    x = rng.normal(size=(n, d)) * 0.01 + rng.integers(0, 6, size=(n, 1))
    f = np.abs(x).sum(axis=1)
    xt, ft = torch.from_numpy(x).cuda(), torch.from_numpy(f).cuda()
    ref = z.cluster(xt, ft, None, method="x", tol=0.2, max_clusters=16)
    assert ref["summary"]["error"] == 0
    try:
        z.zeus_set_wait_limit(1)
        bad = z.cluster(xt, ft, None, method="x", tol=0.2, max_clusters=16)
        assert bad["summary"]["error"] == 1
    finally:
        z.zeus_set_wait_limit(0)
    again = z.cluster(xt, ft, None, method="x", tol=0.2, max_clusters=16)
    assert again["summary"]["error"] == 0
    assert torch.equal(again["labels"], ref["labels"])
    o = ora.cluster(x, f, None, method="x", tol=0.2, max_clusters=16)
    assert np.array_equal(again["labels"].cpu().numpy(), o["labels"])


@pytest.mark.parametrize("layout", [1, 128, 0])
def test_nonfinite_in_mid_run_matches_oracle(z, ora, layout):
    n, d = 256, 5
    x0 = workloads.start_points(n, d, -5.0, 5.0, seed=21)
    x0[1::3] *= 1e3  # every third start overflows after a few iterations
    fields = dict(objective="rosenbrock", dim=d, n_starts=n, bfgs_max_iters=60,
                  threads_per_start=layout)
    g = to_np(z.solve_from(zeus_problem(z, fields), torch.from_numpy(x0).cuda()))
    o = ora.bfgs_many(oracle_problem(ora, fields), x0)
    mid = (o["status"] == 3) & (o["iters"] >= 3)
    assert mid.sum() >= 40 and ((o["status"] != 3) & (o["iters"] > 0)).sum() >= 100
    # at a non-finite point the oracle's full dual passes carry 0 * inf = NaN
    # from terms without x_i into the gradient, which the kernels' passes
    # leave out (they add exact zeros at finite points): ||g|| is non-finite
    # on both sides, compared as such
    nf = o["status"] == 3
    assert np.array_equal(np.isfinite(g["gnorm"][nf]), np.isfinite(o["gnorm"][nf]))
    g["gnorm"] = np.where(nf, 0.0, g["gnorm"])
    o["gnorm"] = np.where(nf, 0.0, o["gnorm"])
    assert_bitwise(g, o)
    s = g["summary"]
    assert s["total_iters"] == int(o["iters"].sum()) and s["error"] == 0
