"""Helpers shared by the GPU parity tests: build the same problem for the
CUDA path and the oracle, and compare per-start results.

Tolerance (floating point): 1e-9 relative per start over the first 20 BFGS
iterations, |a - b| <= 1e-9 * max(1, |b|) element-wise, with identical
status and iteration counts.  Starts whose oracle trajectory passed a
branch decision (Armijo test, ||g|| < tol) within 1e-12 relative are
flip-prone: a last-bit difference may take the other branch; they are
reported and excluded, and must stay rare.
"""
import numpy as np

RTOL = 1e-9
FLIP_MARGIN = 1e-12


def oracle_problem(oracle, fields: dict, **kw):
    f = dict(fields)
    f.update(kw)
    keep = {k: v for k, v in f.items() if k in oracle.Problem.__dataclass_fields__}
    return oracle.Problem(**keep)


def zeus_problem(z, fields: dict, **kw):
    f = dict(fields)
    f.update(kw)
    keep = {k: v for k, v in f.items() if k in z.Problem.__dataclass_fields__}
    return z.Problem(**keep)


def close(a, b, rtol=RTOL):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    both_nan = np.isnan(a) & np.isnan(b)
    same_inf = np.isinf(a) & np.isinf(b) & (np.sign(a) == np.sign(b))
    ok = np.abs(a - b) <= rtol * np.maximum(1.0, np.abs(b))
    return ok | both_nan | same_inf


def compare_runs(gpu: dict, ora: dict, rtol=RTOL, max_flip_frac=0.02):
    """Per-start comparison of BFGS outputs; returns (n_compared, flagged)."""
    n = len(ora["f"])
    flagged = np.asarray(ora["margin"]) < FLIP_MARGIN
    bad, excused = [], []
    for i in range(n):
        ok = (gpu["status"][i] == ora["status"][i] and gpu["iters"][i] == ora["iters"][i]
              and close(gpu["f"][i], ora["f"][i], rtol) and close(gpu["gnorm"][i], ora["gnorm"][i], rtol)
              and np.all(np.abs(gpu["x"][i] - ora["x"][i]) <= rtol * max(1.0, np.abs(ora["x"][i]).max())))
        if not ok:
            (excused if flagged[i] else bad).append(i)
    assert not bad, (f"{len(bad)} of {n} starts differ, first {bad[:5]}: "
                     + "; ".join(f"i={i} gpu(f={gpu['f'][i]!r}, g={gpu['gnorm'][i]!r}, it={gpu['iters'][i]}, "
                                 f"st={gpu['status'][i]}) ora(f={ora['f'][i]!r}, g={ora['gnorm'][i]!r}, "
                                 f"it={ora['iters'][i]}, st={ora['status'][i]}) "
                                 f"dx={np.abs(gpu['x'][i] - ora['x'][i]).max():.2e}"
                                 for i in bad[:3]))
    assert len(excused) <= max_flip_frac * n, f"{len(excused)} flip-prone starts of {n} differ"
    return n - len(excused), len(excused)


def assert_bitwise(gpu: dict, ora: dict):
    """Identical bits in every output of every start."""
    for k in ("x", "f", "gnorm", "status", "iters"):
        a, b = np.asarray(gpu[k]), np.asarray(ora[k])
        same = (a == b) | (np.isnan(a) & np.isnan(b)) if a.dtype.kind == "f" else (a == b)
        if same.ndim > 1:
            same = same.all(axis=1)
        assert same.all(), f"{k}: {int((~same).sum())} of {len(same)} starts differ, first {np.flatnonzero(~same)[:5]}"


def to_np(out: dict) -> dict:
    return {k: (v.cpu().numpy() if hasattr(v, "cpu") else v) for k, v in out.items()}


def clopper_pearson(k: int, n: int, level: float = 0.95):
    """Exact two-sided binomial confidence interval for k successes in n."""
    from scipy.stats import beta
    a = (1.0 - level) / 2.0
    lo = 0.0 if k == 0 else float(beta.ppf(a, k, n - k + 1))
    hi = 1.0 if k == n else float(beta.ppf(1.0 - a, k + 1, n - k))
    return lo, hi
