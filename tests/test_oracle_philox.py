"""Pins of the oracle's Philox4x64-10 and of its uniform-draw mapping.

The generator replaces the paper's cuRAND seeding (Section IV-A).  It is
pinned by the published known-answer vectors (tests/golden) and by numpy's
independent Philox4x64-10 implementation.
"""
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x64_10_kat.txt")


def _kat():
    rows = []
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        w = [int(t, 16) for t in line.split()]
        rows.append((w[0:4], w[4:6], w[6:10]))
    return rows


def _numpy_block(ctr, key):
    # numpy's Philox increments the counter before producing a block, so
    # start it one below the wanted counter (with borrow).
    c = list(ctr)
    i = 0
    while True:
        c[i] = (c[i] - 1) % 2**64
        if c[i] != 2**64 - 1 or i == 3:
            break
        i += 1
    bg = np.random.Philox(key=np.array(key, dtype=np.uint64),
                          counter=np.array(c, dtype=np.uint64))
    return [int(v) for v in bg.random_raw(4)]


def test_known_answer_vectors(oracle_mod):
    for ctr, key, out in _kat():
        assert [int(v) for v in oracle_mod.philox4x64_10(ctr, key)] == out


def test_matches_numpy_philox(oracle_mod):
    rng = np.random.default_rng(7)
    for _ in range(200):
        ctr = [int(v) for v in rng.integers(0, 2**64, size=4, dtype=np.uint64)]
        key = [int(v) for v in rng.integers(0, 2**64, size=2, dtype=np.uint64)]
        assert [int(v) for v in oracle_mod.philox4x64_10(ctr, key)] == _numpy_block(ctr, key)


@pytest.mark.parametrize("seed", [0, 1, 12345, 2**63 + 5])
def test_uniform_layout(oracle_mod, seed):
    # draw (phase, particle, j) = word j%4 of block ctr=(j//4, particle, problem, phase),
    # key=(seed, 0), mapped to [0,1) with its top 53 bits
    for (problem, phase, particle, j) in [(0, 0, 0, 0), (0, 1, 3, 5), (2, 7, 1000, 11), (0, 41, 16383, 9)]:
        blk = _numpy_block([j // 4, particle, problem, phase], [seed, 0])
        want = float(blk[j % 4] >> 11) * 2.0**-53
        assert oracle_mod.uniform(seed, problem, phase, particle, j) == want


def test_uniform_moments(oracle_mod):
    u = np.array([oracle_mod.uniform(3, 0, ph, i, j) for ph in range(2) for i in range(200) for j in range(10)])
    assert u.min() >= 0.0 and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 0.02
    assert abs(u.var() - 1.0 / 12.0) < 0.01
