"""zeus_solve_from_noalloc: BFGS from given starts for callers that cannot
allocate device memory (code that must stay inside a framework's own
caching allocator, plugins handed device buffers but no allocation rights,
code that must not pay the synchronisation cudaMalloc/cudaFree can imply).  It uses one static device array as scratch instead of a
caller-provided workspace; its results must equal zeus_solve_from's.

This file is collected last so that a run stopping at the first failure
has already run every other test."""
import numpy as np
import pytest
import torch

from paper_2603_28770_gb300 import workloads
from parity import close

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def z():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2603_28770_gb300 as z
    z.lib()
    return z


def _run_noalloc(z, p, x0):
    n, d = p.n_starts, p.dim
    out = dict(x=torch.empty(n, d, dtype=torch.float64, device="cuda"),
               f=torch.empty(n, dtype=torch.float64, device="cuda"),
               gnorm=torch.empty(n, dtype=torch.float64, device="cuda"),
               status=torch.empty(n, dtype=torch.int32, device="cuda"),
               iters=torch.empty(n, dtype=torch.int32, device="cuda"),
               result=z.new_result())
    z.zeus_solve_from_noalloc(p, x0, out["x"], out["f"], out["gnorm"], out["status"], out["iters"],
                              out["result"])
    torch.cuda.synchronize()
    res = z.decode_result(out["result"])
    return {k: v.cpu().numpy() for k, v in out.items() if k != "result"}, res


def _same(a, b, ra, rb):
    for k in ("x", "f", "gnorm"):
        assert np.all(close(a[k], b[k])), k
    assert np.array_equal(a["status"], b["status"]) and np.array_equal(a["iters"], b["iters"])
    for k in ("best_index", "n_converged", "total_iters", "total_feval"):
        assert ra[k] == rb[k], k
    assert close(ra["best_f"], rb["best_f"])


@pytest.mark.parametrize("case", [
    # 10-D Rastrigin with a long cap: long runs are handed to the block-per-start kernel
    dict(objective="rastrigin", dim=10, lower=-5.12, upper=5.12, n_starts=3000, bfgs_max_iters=400),
    # block-per-start throughout (d above the one-lane limit)
    dict(objective="ackley", dim=40, lower=-5.0, upper=5.0, n_starts=300, bfgs_max_iters=60),
    # the FP32 form with more starts than its hand-over queue holds
    dict(objective="rastrigin", dim=10, lower=-5.12, upper=5.12, n_starts=5000, bfgs_max_iters=400,
         precision="fp32_guarded"),
    # the adjoint gradient
    dict(objective="rosenbrock", dim=12, lower=-2.0, upper=2.0, n_starts=2000, bfgs_max_iters=300,
         grad_mode="adjoint"),
    # L-BFGS (block per start, no H)
    dict(objective="rosenbrock", dim=64, lower=-2.0, upper=2.0, n_starts=256, bfgs_max_iters=200,
         lbfgs_m=5),
    # more starts than the array's queue holds: the rest finish in their lanes
    dict(objective="rastrigin", dim=10, lower=-5.12, upper=5.12, n_starts=100000, bfgs_max_iters=200),
], ids=["handover", "block_per_start", "fp32_queue", "adjoint", "lbfgs", "queue_clamped"])
def test_noalloc_equals_workspace_entry_two_calls(z, case):
    p = z.Problem(**case)
    x0 = torch.from_numpy(workloads.start_points(p.n_starts, p.dim, p.lower, p.upper, seed=17)).cuda()
    ref = z.solve_from(p, x0)
    ref_np = {k: ref[k].cpu().numpy() for k in ("x", "f", "gnorm", "status", "iters")}
    for _ in range(2):  # the second call finds the first call's leftovers in the array
        got, res = _run_noalloc(z, p, x0)
        _same(got, ref_np, res, ref["summary"])
        assert res["error"] == 0


def test_noalloc_rejects_problems_beyond_the_array(z):
    # a dense H streamed from device memory (d = 256) needs H slots of
    # 512 KiB per block, more than the array holds
    p = z.Problem(objective="rosenbrock", dim=256, lower=-2.0, upper=2.0, n_starts=64,
                  bfgs_max_iters=10)
    assert z.zeus_plan_info(p)["stream"] == 1
    x0 = torch.zeros(p.n_starts, p.dim, dtype=torch.float64, device="cuda")
    with pytest.raises(z.ZeusError) as e:
        _run_noalloc(z, p, x0)
    assert e.value.code == z._capi.ZEUS_EWORKSPACE
