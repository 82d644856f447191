"""Host logic of solve_until_confident (the iterative process Section VI
proposes): rounds with seeds s, s + 1, ..., pooled points clustered after
each round, stop at the first round whose lowest region holds the required
number of starts, or after max_rounds.  The device solve and clustering are
replaced by CPU stand-ins (the oracle's clustering), so no GPU is needed."""
import numpy as np
import pytest
import torch


@pytest.fixture()
def z(monkeypatch):
    import oracle
    import paper_2603_28770_gb300 as z
    seeds = []

    def fake_solve(p, device="cuda"):
        # round r puts r + 1 starts at the global minimum 0, the rest far
        r = p.seed - 100
        seeds.append(p.seed)
        n, d = p.n_starts, p.dim
        x = torch.full((n, d), 3.0, dtype=torch.float64)
        x[: r + 1] = 0.0
        f = (x * x).sum(dim=1)
        st = torch.ones(n, dtype=torch.int32)
        return {"x": x, "f": f, "status": st}

    def fake_cluster(x, f, status=None, method="x", tol=1e-3, max_clusters=256,
                     only_converged=False, stream=None):
        o = oracle.cluster(x.numpy(), f.numpy(), status.numpy(), method=method, tol=tol,
                           max_clusters=max_clusters, only_converged=only_converged)
        return {"labels": torch.from_numpy(o["labels"]), "summary": o["summary"]}

    monkeypatch.setattr(z, "solve", fake_solve)
    monkeypatch.setattr(z, "cluster", fake_cluster)
    z._seeds = seeds
    return z


def test_stops_at_the_first_round_that_reaches_the_count(z):
    p = z.Problem(objective="rastrigin", dim=3, n_starts=10, seed=100)
    # pooled counts at the minimum after rounds 1, 2, 3: 1, 3, 6
    c = z.solve_until_confident(p, required=3, tol=1e-6, max_rounds=10)
    assert c["rounds"] == 2 and z._seeds == [100, 101]
    assert c["summary"]["best_count"] == 3 and c["summary"]["best_f"] == 0.0
    assert c["x"].shape == (20, 3) and c["f"].shape == (20,)


def test_gives_up_after_max_rounds(z):
    p = z.Problem(objective="rastrigin", dim=2, n_starts=4, seed=100)
    c = z.solve_until_confident(p, required=1000, tol=1e-6, max_rounds=3)
    assert c["rounds"] == 3 and z._seeds == [100, 101, 102]
    assert c["summary"]["best_count"] == 1 + 2 + 3
