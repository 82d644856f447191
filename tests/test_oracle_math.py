"""Pins of the oracle's own elementary functions (sin/cos of 2 pi x by exact
reduction + Taylor series, e^x by Cody-Waite reduction + Taylor series)
against 60-digit mpmath references and exact special values."""
import math

import numpy as np
import pytest

mp = pytest.importorskip("mpmath")
mp.mp.dps = 60


def _ref_sc(x):
    t = 2 * mp.pi * mp.mpf(x)
    return float(mp.sin(t)), float(mp.cos(t))


def test_sincos2pi_against_mpmath(oracle_mod):
    rng = np.random.default_rng(0)
    xs = np.concatenate([rng.uniform(-10, 10, 3000), rng.uniform(-1e6, 1e6, 300),
                         rng.uniform(-1e-3, 1e-3, 300), np.arange(-40, 41) / 8.0,
                         np.arange(-40, 41) / 8.0 + 1e-9])
    for x in xs:
        s, c = oracle_mod.sincos2pi(x)
        rs, rc = _ref_sc(x)
        # within about one ulp of 1 (absolute), and bounded like sin/cos
        assert abs(s - rs) <= 2.3e-16 and abs(c - rc) <= 2.3e-16, (x, s, rs, c, rc)
        assert abs(s) <= 1.0 and abs(c) <= 1.0


def test_sincos2pi_exact_points(oracle_mod):
    for k in range(-8, 9):
        s, c = oracle_mod.sincos2pi(k)
        assert (s, c) == (0.0, 1.0) or (s == 0.0 and c == 1.0)
        s, c = oracle_mod.sincos2pi(k + 0.5)
        assert s == 0.0 and c == -1.0
        s, c = oracle_mod.sincos2pi(k + 0.25)
        assert s == 1.0 and c == 0.0
        s, c = oracle_mod.sincos2pi(k - 0.25)
        assert s == -1.0 and c == 0.0


def test_exp_against_mpmath(oracle_mod):
    rng = np.random.default_rng(1)
    xs = np.concatenate([rng.uniform(-30, 30, 3000), rng.uniform(-700, 700, 300),
                         rng.uniform(-1e-8, 1e-8, 100), [0.0, 1.0, -1.0, 0.5, -0.2, 709.0, -700.0]])
    for x in xs:
        got = oracle_mod.exp(x)
        ref = float(mp.exp(mp.mpf(x)))
        assert abs(got - ref) <= 2.3e-16 * ref, (x, got, ref)
    assert oracle_mod.exp(0.0) == 1.0
    assert oracle_mod.exp(1000.0) == math.inf and oracle_mod.exp(-1000.0) == 0.0
    assert math.isnan(oracle_mod.exp(float("nan")))


def test_cos2pi_dual_rule(oracle_mod):
    # (cos 2 pi a, -2 pi sin(2 pi a) b) against 60-digit references
    rng = np.random.default_rng(2)
    for _ in range(300):
        a, b = rng.uniform(-6, 6), rng.normal()
        ra, rb = oracle_mod.dual_op("cos2pi", a, b)
        t = 2 * mp.pi * mp.mpf(a)
        assert abs(ra - float(mp.cos(t))) <= 2.3e-16
        want = float(-2 * mp.pi * mp.sin(t) * mp.mpf(b))
        assert abs(rb - want) <= 2e-15 * max(1.0, abs(want))
