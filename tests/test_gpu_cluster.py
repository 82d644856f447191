"""GPU parity of the solution clustering (Section VI, future work; the
reading and the definition are in include/zeus.h and zeus_oracle.c):
labels, leaders, member counts and the summary are integer results or
decisions taken in FP64 with the same operations on both sides, so they
must equal the oracle's bit for bit on the same inputs."""
import numpy as np
import pytest
import torch

from paper_2603_28770_gb300 import workloads

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


def _same(g, o):
    assert np.array_equal(g["labels"].cpu().numpy(), o["labels"])
    assert np.array_equal(g["leaders"].cpu().numpy(), o["leaders"])
    assert np.array_equal(g["counts"].cpu().numpy(), o["counts"])
    for k, v in o["summary"].items():
        a = g["summary"][k]
        assert a == v or (np.isnan(a) and np.isnan(v)), (k, a, v)


def _points(n, d, seed, n_centres=12, nan_frac=0.02, ties=False):
    rng = np.random.default_rng(seed)
    centres = rng.uniform(-5, 5, size=(n_centres, d))
    x = centres[rng.integers(0, n_centres, n)] + 0.05 * rng.normal(size=(n, d))
    f = np.sum(x * x, axis=1) / 10 + rng.uniform(0, 0.1, n)
    if ties:
        f = np.round(f, 1)
    f[rng.random(n) < nan_frac] = np.nan
    f[rng.random(n) < nan_frac / 2] = np.inf
    st = (rng.random(n) < 0.8).astype(np.int32)
    return x, f, st


@pytest.mark.parametrize("n,d,method,tol,mc,only", [
    (1000, 4, "x", 0.5, 64, False), (1025, 3, "x", 0.2, 7, True), (4096, 10, "f", 0.02, 256, False),
    (3000, 2, "f", 1e-3, 4096, True), (1, 5, "x", 1.0, 1, False), (777, 6, "x", 0.0, 128, False)])
def test_cluster_matches_oracle(z, ora, n, d, method, tol, mc, only):
    x, f, st = _points(n, d, seed=n + d)
    g = z.cluster(torch.from_numpy(x).cuda(), torch.from_numpy(f).cuda(), torch.from_numpy(st).cuda(),
                  method=method, tol=tol, max_clusters=mc, only_converged=only)
    o = ora.cluster(x, f, st, method=method, tol=tol, max_clusters=mc, only_converged=only)
    _same(g, o)


def test_ties_and_empty(z, ora):
    # many equal f values: the lower start index leads
    x, f, st = _points(5000, 3, seed=2, ties=True)
    for method in ("f", "x"):
        g = z.cluster(torch.from_numpy(x).cuda(), torch.from_numpy(f).cuda(), method=method,
                      tol=0.3, max_clusters=512)
        _same(g, ora.cluster(x, f, method=method, tol=0.3, max_clusters=512))
    # no candidate at all, and no start at all
    fn = np.full(100, np.nan)
    g = z.cluster(torch.zeros(100, 2, dtype=torch.float64, device="cuda"),
                  torch.from_numpy(fn).cuda(), method="x", tol=1.0, max_clusters=4)
    _same(g, ora.cluster(np.zeros((100, 2)), fn, method="x", tol=1.0, max_clusters=4))
    g = z.cluster(torch.zeros(0, 2, dtype=torch.float64, device="cuda"),
                  torch.zeros(0, dtype=torch.float64, device="cuda"), max_clusters=4)
    assert g["summary"]["n_candidates"] == 0 and g["summary"]["best_leader"] == -1


def test_large_swarm(z, ora):
    # 2^18 points in 8-D, the first 64 clusters
    x, f, st = _points(1 << 18, 8, seed=9, n_centres=200)
    g = z.cluster(torch.from_numpy(x).cuda(), torch.from_numpy(f).cuda(), method="x", tol=0.5,
                  max_clusters=64)
    _same(g, ora.cluster(x, f, method="x", tol=0.5, max_clusters=64))


@pytest.mark.parametrize("name,method,tol", [("rastrigin5d_n16384", "x", 1e-4),
                                             ("rastrigin10d_n16384", "f", 1e-6)])
def test_cluster_solver_outputs(z, ora, name, method, tol):
    # the final points of a whole run, clustered on the device and by the
    # oracle from the same arrays
    fields = workloads.workload(name, n_starts=4096, bfgs_max_iters=300)
    out = z.solve(z.Problem(**fields))
    g = z.cluster(out["x"], out["f"], out["status"], method=method, tol=tol, max_clusters=1024,
                  only_converged=True)
    o = ora.cluster(out["x"].cpu().numpy(), out["f"].cpu().numpy(), out["status"].cpu().numpy(),
                    method=method, tol=tol, max_clusters=1024, only_converged=True)
    _same(g, o)
    s = g["summary"]
    assert s["best_leader"] >= 0 and s["best_count"] >= 1
    assert s["best_f"] == out["f"][s["best_leader"]].item()


def test_solve_until_confident(z, ora):
    # the iterative process: pooled rounds of 5-D Rastrigin until three
    # starts sit in the region of the lowest f
    p = z.Problem(**workloads.workload("rastrigin5d_n16384", n_starts=1024, bfgs_max_iters=300))
    c = z.solve_until_confident(p, required=3, tol=1e-4, method="x", max_rounds=12)
    x, f, st = (c[k].cpu().numpy() for k in ("x", "f", "status"))
    o = ora.cluster(x, f, st, method="x", tol=1e-4, max_clusters=1, only_converged=True)
    assert c["summary"]["best_count"] == o["summary"]["best_count"] >= 3
    assert c["summary"]["best_leader"] == o["summary"]["best_leader"]
    # it stopped at the first round that reached three
    n = p.n_starts
    for r in range(1, c["rounds"]):
        orr = ora.cluster(x[:r * n], f[:r * n], st[:r * n], method="x", tol=1e-4, max_clusters=1,
                          only_converged=True)
        assert orr["summary"]["best_count"] < 3


@pytest.mark.parametrize("method,tol,mc,only", [("x", 1e-4, 64, True), ("f", 1e-6, 16, False),
                                                ("x", 0.5, 3, False)])
def test_batch_cluster_matches_oracle_per_problem(z, ora, method, tol, mc, only):
    # every problem of a mixed batch (built-in and user objectives, lane and
    # block layouts, ragged swarms) clustered in one launch, each against the
    # oracle on that problem's own outputs
    probs = [z.Problem(**m, n_starts=40 + 37 * i, pso_iters=i % 3, bfgs_max_iters=80, seed=i)
             for i, m in enumerate(workloads.mixed_batch(10, seed=3, dmin=2, dmax=48))]
    probs += [z.Problem(objective="himmelblau", dim=2, lower=-5, upper=5, n_starts=300, seed=1),
              z.Problem(objective="griewank", dim=6, lower=-20, upper=20, n_starts=1, seed=2)]
    b = z.Batch(probs)
    b.solve()
    c = b.cluster(method=method, tol=tol, max_clusters=mc, only_converged=only)
    lab = c["labels"].cpu().numpy()
    for P, p in enumerate(probs):
        v = b.problem(P)
        x, f, st = (v[k].cpu().numpy() for k in ("x", "f", "status"))
        o = ora.cluster(x, f, st, method=method, tol=tol, max_clusters=mc, only_converged=only)
        so = b.soff[P]
        assert np.array_equal(lab[so:so + p.n_starts], o["labels"]), P
        assert np.array_equal(c["leaders"][P].cpu().numpy(), o["leaders"]), P
        assert np.array_equal(c["counts"][P].cpu().numpy(), o["counts"]), P
        for k, val in o["summary"].items():
            a = c["summaries"][P][k]
            assert a == val or (np.isnan(a) and np.isnan(val)), (P, k, a, val)
    # the Himmelblau problem: its four minima are four regions
    if method == "x" and tol == 1e-4:
        assert c["summaries"][10]["n_clusters"] == 4


def test_cluster_replays_from_a_cuda_graph(z):
    # zeus_cluster is one memset and one cooperative launch: a captured call
    # replays to the same labels and summary
    import ctypes as C
    x, f, st = _points(20000, 5, seed=21)
    xt, ft, stt = (torch.from_numpy(a).cuda() for a in (x, f, st))
    cp = z._capi.zeus_cluster_params(1, 128, 1, 0, 0.3)
    lab = torch.empty(20000, dtype=torch.int32, device="cuda")
    lead = torch.empty(128, dtype=torch.int32, device="cuda")
    cnt = torch.empty(128, dtype=torch.int32, device="cuda")
    res = torch.empty(C.sizeof(z._capi.zeus_cluster_result), dtype=torch.uint8, device="cuda")
    ws = torch.empty(z.zeus_cluster_workspace_size(128), dtype=torch.uint8, device="cuda")
    z.zeus_cluster(cp, 20000, 5, xt, ft, stt, lab, lead, cnt, res, ws)
    torch.cuda.synchronize()
    ref = (lab.clone(), lead.clone(), cnt.clone(), res.clone())
    g = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        g.capture_begin()
        z.zeus_cluster(cp, 20000, 5, xt, ft, stt, lab, lead, cnt, res, ws, side)
        g.capture_end()
    torch.cuda.current_stream().wait_stream(side)
    for _ in range(2):
        lab.fill_(7)
        cnt.zero_()
        g.replay()
        torch.cuda.synchronize()
        for a, b in zip((lab, lead, cnt, res), ref):
            assert torch.equal(a, b)
