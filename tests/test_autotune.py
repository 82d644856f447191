"""Host logic of the batched-form autotuner: keys, candidate filtering,
choice of the fastest layout, the JSON cache and how choices are applied.
The GPU timing is replaced by a stand-in measure function."""
import json

import pytest


@pytest.fixture(scope="module")
def z():
    import paper_2603_28770_gb300 as z
    z.lib()
    return z


def test_buckets():
    from paper_2603_28770_gb300.autotune import bucket
    assert [bucket(d) for d in (1, 2, 3, 4, 5, 16, 17, 128, 129, 5000)] == [2, 2, 4, 4, 8, 16, 24, 128, 192, 4096]


def test_tuner_picks_fastest_and_caches(z, tmp_path):
    from paper_2603_28770_gb300.autotune import Autotuner
    cost = {0: 3.0, 1: 2.0, 32: 4.0, 128: 5.0}
    calls = []

    def measure(probe):
        tps = {int(q.threads_per_start) for q in probe}
        assert len(tps) == 1 and all(q.n_starts <= 64 for q in probe) and len(probe) <= 3
        calls.append(tps.pop())
        return cost[calls[-1]]

    path = tmp_path / "tune.json"
    probs = [z.Problem(objective="rastrigin", dim=10, n_starts=500, seed=i) for i in range(5)]
    probs.append(z.Problem(objective="rastrigin", dim=30, n_starts=100))  # lanes do not fit in FP64
    probs.append(z.Problem(objective="ackley", dim=9, n_starts=100, threads_per_start=128))
    t = Autotuner(str(path), probe_problems=3, probe_starts=64, measure=measure, device_name="dev",
                  probe_total=0)
    out = t.apply(probs)
    assert [q.threads_per_start for q in out[:5]] == [1] * 5
    assert out[5].threads_per_start in (0, 128) and out[6].threads_per_start == 128
    k30 = t.key(probs[5].to_c())
    assert set(t.table["dev"][k30]["ms"]) == {"0", "32", "128"}  # lanes were not a candidate
    assert t.key(probs[6].to_c()) not in t.table["dev"]    # explicit choices are not tuned
    saved = json.loads(path.read_text())
    assert saved["dev"][t.key(probs[0].to_c())]["threads_per_start"] == 1
    # a second tuner reads the cache and measures nothing
    n = len(calls)
    t2 = Autotuner(str(path), measure=lambda probe: pytest.fail("measured again"), device_name="dev")
    assert [q.threads_per_start for q in t2.apply(probs[:5])] == [1] * 5
    assert len(calls) == n
    # another device name is tuned separately
    t3 = Autotuner(str(path), probe_problems=3, probe_starts=64, measure=measure, device_name="other",
                   probe_total=0)
    t3.apply(probs[:1])
    assert len(calls) > n and set(json.loads(path.read_text())) == {"dev", "other"}


def test_tuner_ties_go_to_the_smaller_layout(z, tmp_path):
    from paper_2603_28770_gb300.autotune import Autotuner
    t = Autotuner(str(tmp_path / "t.json"), measure=lambda probe: 1.0, device_name="dev")
    assert t.apply([z.Problem(objective="rosenbrock", dim=4)])[0].threads_per_start == 0


def test_candidates_of_user_objectives(z):
    # a user objective takes the lane and block layouts the plan accepts,
    # never the streamed-H one (no user objective streams H)
    from paper_2603_28770_gb300.autotune import Autotuner
    small = z.Problem(objective="griewank", dim=8, n_starts=64).to_c()
    large = z.Problem(objective="griewank", dim=100, n_starts=64).to_c()
    assert Autotuner._valid(small, 0) and Autotuner._valid(small, 1) and Autotuner._valid(small, 128)
    assert not Autotuner._valid(small, 256)
    assert Autotuner._valid(large, 128) and not Autotuner._valid(large, 1)
    assert not Autotuner._valid(large, 256)
    # forward mode only: the adjoint form of the same problem has no layout
    adj = z.Problem(objective="griewank", dim=8, n_starts=64, grad_mode="adjoint").to_c()
    assert not any(Autotuner._valid(adj, t) for t in (0, 1, 128, 256))
