"""Parity at the benchmark's full sizes, in the launch configurations the
benchmark times, on outputs the oracle can compute one by one: whole
problems of the 4096-problem batch, and sampled starts of the streamed-H
workloads (d = 256 and d = 1024)."""
import numpy as np
import pytest
import torch

from paper_2603_28770_gb300 import workloads
from parity import compare_runs, oracle_problem, to_np, zeus_problem

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


def test_mixed_batch_full_size_sampled_problems(z, ora):
    # all 4096 problems (2^20 starts) in one batch; the oracle runs the
    # whole method (PSO + BFGS + argmin) of a sample of them
    fields = workloads.batch_problems("mixed4096_n256", None)
    b = z.Batch([z.Problem(**f) for f in fields])
    b.solve()
    torch.cuda.synchronize()
    dims = np.array([f["dim"] for f in fields])
    rng = np.random.default_rng(11)
    sample = {int(np.argmin(dims)), int(np.argmax(dims))}
    sample |= set(rng.choice(len(fields), 4, replace=False).tolist())
    for P in sorted(sample):
        g = to_np(b.problem(P))
        o = ora.solve(oracle_problem(ora, fields[P]))
        compare_runs(g, o, rtol=1e-9, max_flip_frac=0.02)
        assert g["summary"]["best_index"] == o["best"]
        assert g["summary"]["total_iters"] == int(o["iters"].sum())
    sums = b.summaries()
    assert all(s["error"] == 0 for s in sums)
    assert sum(s["total_iters"] for s in sums) == int(b.iters.sum().item())


@pytest.mark.parametrize("name,grad", [("rosenbrock256d_n8192", "forward"),
                                       ("rosenbrock1024d_n2048", "adjoint")])
def test_streamed_full_size_sampled_starts(z, ora, name, grad):
    # the whole workload in the streamed launch configuration (all N
    # particles, PSO then BFGS from every one); the oracle runs BFGS from a
    # sample of the same PSO positions.  First 10 iterations: FP64 within
    # 1e-8 (the lagged update and tree sums reorder the arithmetic), the
    # FP32 form within 1e-3 of the FP64 oracle in f.
    fields = workloads.workload(name, grad_mode=grad, bfgs_max_iters=10)
    op = ora.pso(oracle_problem(ora, fields))
    sample = np.random.default_rng(5).choice(fields["n_starts"], 16, replace=False)
    o = ora.bfgs_many(oracle_problem(ora, fields), op["x"][sample])
    for precision in ("fp64", "fp32_guarded"):
        p = zeus_problem(z, fields, precision=precision, threads_per_start=256)
        assert z.zeus_plan_info(p)["stream"] == 1
        g = z.solve(p)
        s = g["summary"]
        assert s["gbest_index"] == op["gidx"]
        gs = {k: g[k].cpu().numpy()[sample] for k in ("x", "f", "gnorm", "status", "iters")}
        if precision == "fp64":
            compare_runs(gs, o, rtol=1e-8, max_flip_frac=0.1)
        else:
            err = np.abs(gs["f"] - o["f"]) / np.maximum(1.0, np.abs(o["f"]))
            assert (err <= 1e-3).mean() >= 0.8, err
        assert s["h_reads"] + s["h_writes"] > 0 and s["total_iters"] == int(g["iters"].sum().item())


def test_streamed_fp32_benchmark_configuration(z):
    # the streamed FP32 workload exactly as the benchmark times it: every
    # start ends finite, the counters add up, H went through device memory
    fields = workloads.workload("rosenbrock256d_n8192", precision="fp32_guarded")
    g = z.solve(zeus_problem(z, fields))
    s = g["summary"]
    assert np.isfinite(g["f"].cpu().numpy()).all() and s["error"] == 0
    assert s["total_iters"] == int(g["iters"].sum().item())
    assert 0 < s["h_writes"] <= s["total_iters"] and s["h_reads"] <= s["total_iters"]
    assert s["best_f"] < 1e-3
