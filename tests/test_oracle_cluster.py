"""Oracle pins of the solution clustering (Section VI, future work: group
the candidate solutions of the multistart by function value or by
coordinates; the number of starts in the region of the lowest f is the
confidence in it).  The oracle implements the reading in zeus_oracle.c
(leader clustering in order of increasing f).  The pins are a hand-worked
example, the limiting tolerances, the properties that define a leader
clustering (checked with numpy, not with the oracle's loop), invariance
under relabelling of the starts, and the four minima of Himmelblau's
function."""
import numpy as np
import pytest


def test_hand_worked_example(oracle_mod):
    # five 1-D points; by x with tol 1: visiting in order of f
    # (x=3 f=.5) leader 0; (3.2, .6) joins 0; (0, 1) leader 1; (.5, 2)
    # joins 1; (10, 9) leader 2
    x = np.array([[0.0], [0.5], [3.0], [3.2], [10.0]])
    f = np.array([1.0, 2.0, 0.5, 0.6, 9.0])
    r = oracle_mod.cluster(x, f, method="x", tol=1.0, max_clusters=4)
    assert r["labels"].tolist() == [1, 1, 0, 0, 2]
    assert r["leaders"].tolist() == [2, 0, 4, -1] and r["counts"].tolist() == [2, 2, 1, 0]
    s = r["summary"]
    assert (s["n_clusters"], s["best_count"], s["best_leader"], s["best_f"]) == (3, 2, 2, 0.5)
    assert s["best_spread"] == abs(3.2 - 3.0)
    # two clusters at most: the point at 10 is left out
    r = oracle_mod.cluster(x, f, method="x", tol=1.0, max_clusters=2)
    assert r["labels"].tolist() == [1, 1, 0, 0, -2] and r["summary"]["n_left"] == 1
    # by f with tol 0.2 (relative to max(1, |f_L|)): .5 and .6 together;
    # 1 is 0.5 from .5; 2 is 1.0 from 1 (> 0.2 * 1); 9 alone
    r = oracle_mod.cluster(x, f, method="f", tol=0.2, max_clusters=8)
    assert r["labels"].tolist() == [1, 2, 0, 0, 3]
    assert r["summary"]["best_spread"] == 0.6 - 0.5


def test_tolerance_limits(oracle_mod):
    rng = np.random.default_rng(1)
    x = rng.normal(size=(50, 3))
    x[7] = x[3]  # an exact duplicate point
    f = rng.uniform(0, 1, 50)
    # tol 0: only identical points share a cluster
    r = oracle_mod.cluster(x, f, method="x", tol=0.0, max_clusters=64)
    assert r["summary"]["n_clusters"] == 49 and r["labels"][7] == r["labels"][3]
    # a tolerance past every distance: one cluster led by the lowest f
    r = oracle_mod.cluster(x, f, method="x", tol=1e6, max_clusters=1)
    b = int(np.argmin(f))
    assert r["summary"]["best_count"] == 50 and r["summary"]["best_leader"] == b
    assert np.isclose(r["summary"]["best_spread"], np.linalg.norm(x - x[b], axis=1).max(),
                      rtol=1e-14)
    r = oracle_mod.cluster(x, f, method="f", tol=1e6, max_clusters=1)
    assert r["summary"]["best_count"] == 50 and r["summary"]["best_spread"] == f.max() - f.min()


def test_candidates_and_ties(oracle_mod):
    f = np.array([np.nan, 1.0, np.inf, 1.0, -np.inf, 0.5])
    x = np.arange(6.0).reshape(6, 1) * 10
    st = np.array([1, 1, 1, 0, 1, 1], dtype=np.int32)
    r = oracle_mod.cluster(x, f, st, method="x", tol=1.0, max_clusters=8)
    assert r["labels"].tolist() == [-1, 1, -1, 2, -1, 0]  # equal f: lower index first
    assert r["summary"]["n_candidates"] == 3
    r = oracle_mod.cluster(x, f, st, method="x", tol=1.0, max_clusters=8, only_converged=True)
    assert r["labels"].tolist() == [-1, 1, -1, -1, -1, 0]
    r = oracle_mod.cluster(x, np.full(6, np.nan), method="f", tol=1.0, max_clusters=8)
    s = r["summary"]
    assert s["n_clusters"] == 0 and s["best_leader"] == -1 and np.isnan(s["best_f"])


def _check_leader_clustering(x, f, r, method, tol, max_clusters):
    """The properties that define the result, checked from scratch."""
    lab, lead, cnt = r["labels"], r["leaders"], r["counts"]
    K = r["summary"]["n_clusters"]
    cand = np.isfinite(f)

    def near(i, l):
        if method == "x":
            return np.sum((x[i] - x[l]) ** 2) <= tol * tol * (1 + 1e-12)
        return abs(f[i] - f[l]) <= tol * max(1.0, abs(f[l])) * (1 + 1e-12)

    def far(i, l):
        if method == "x":
            return np.sum((x[i] - x[l]) ** 2) > tol * tol * (1 - 1e-12)
        return abs(f[i] - f[l]) > tol * max(1.0, abs(f[l])) * (1 - 1e-12)

    assert np.all(lab[~cand] == -1) and np.all(lab[cand] >= -2)
    keys = sorted(np.flatnonzero(cand).tolist(), key=lambda i: (f[i], i))
    rank = {i: q for q, i in enumerate(keys)}
    for k in range(K):
        members = np.flatnonzero(lab == k)
        assert len(members) == cnt[k] and lead[k] in members
        # the leader is the first member in the visiting order, all members
        # are within tol of it, and none is within tol of an earlier leader
        assert min(members, key=lambda i: rank[i]) == lead[k]
        assert all(near(i, lead[k]) for i in members)
        assert all(far(i, lead[j]) for i in members for j in range(k))
    # leaders come in the visiting order
    assert all(rank[lead[k]] < rank[lead[k + 1]] for k in range(K - 1))
    # left-out candidates are far from every leader, and exist only when
    # every cluster slot is used
    left = np.flatnonzero(lab == -2)
    assert all(far(i, lead[j]) for i in left for j in range(K))
    assert len(left) == 0 or K == max_clusters
    assert cnt[:K].sum() + len(left) == cand.sum()


@pytest.mark.parametrize("method,tol,mc", [("x", 0.8, 64), ("x", 0.3, 12), ("f", 0.05, 64),
                                           ("f", 0.01, 5)])
def test_leader_clustering_properties(oracle_mod, method, tol, mc):
    rng = np.random.default_rng(11)
    centres = rng.uniform(-5, 5, size=(9, 4))
    x = centres[rng.integers(0, 9, 400)] + 0.2 * rng.normal(size=(400, 4))
    f = np.sum(x * x, axis=1) / 10 + rng.uniform(0, 0.3, 400)
    f[rng.choice(400, 10, replace=False)] = np.nan
    r = oracle_mod.cluster(x, f, method=method, tol=tol, max_clusters=mc)
    _check_leader_clustering(x, f, r, method, tol, mc)


def test_relabelling_the_starts(oracle_mod):
    # the partition does not depend on the order of the starts (distinct f)
    rng = np.random.default_rng(5)
    x = rng.normal(size=(300, 3))
    f = rng.uniform(size=300)
    perm = rng.permutation(300)
    a = oracle_mod.cluster(x, f, method="x", tol=0.7, max_clusters=300)
    b = oracle_mod.cluster(x[perm], f[perm], method="x", tol=0.7, max_clusters=300)
    assert np.array_equal(b["labels"], a["labels"][perm])
    assert np.array_equal(perm[b["leaders"][:b["summary"]["n_clusters"]]],
                          a["leaders"][:a["summary"]["n_clusters"]])


def test_himmelblau_regions(oracle_mod):
    # the converged BFGS points of Himmelblau's function form four regions
    # by coordinates (its four minima) and one by value (all have f = 0)
    minima = np.array([[3.0, 2.0], [-2.805118, 3.131312], [-3.779310, -3.283186],
                       [3.584428, -1.848126]])
    p = oracle_mod.Problem(objective="himmelblau", dim=2, lower=-5, upper=5, n_starts=300,
                           pso_iters=0, bfgs_max_iters=200, seed=4)
    out = oracle_mod.solve(p)
    r = oracle_mod.cluster(out["x"], out["f"], out["status"], method="x", tol=1e-3,
                           max_clusters=16, only_converged=True)
    s = r["summary"]
    assert s["n_clusters"] == 4 and s["n_candidates"] == (out["status"] == 1).sum()
    lead = out["x"][r["leaders"][:4]]
    assert np.all(np.min(np.linalg.norm(lead[:, None] - minima[None], axis=2), axis=1) < 1e-5)
    r = oracle_mod.cluster(out["x"], out["f"], out["status"], method="f", tol=1e-9,
                           max_clusters=16, only_converged=True)
    assert r["summary"]["n_clusters"] == 1 and r["summary"]["best_count"] == s["n_candidates"]
