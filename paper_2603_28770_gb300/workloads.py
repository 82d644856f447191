"""Workload definitions and seeded synthetic inputs.

This module holds no arithmetic of the method: only problem parameters and
seeded random inputs (start points, batched problem lists).  Both the CUDA
path and the CPU oracle are fed from here.  The workloads mirror the
paper's own test-function experiments (Section V: Rosenbrock, Rastrigin,
Ackley on their usual boxes, swarms of 10^2..10^5 particles); every input is
synthetic, there is no dataset.
"""
from __future__ import annotations

import numpy as np

# name -> problem fields (keys of zeus_problem / oracle Problem)
WORKLOADS = {
    # 2-D Rosenbrock: 128 particles in [-5,5]^2, 5 PSO updates, 100 BFGS iterations
    "rosenbrock2d_n128": dict(objective="rosenbrock", dim=2, lower=-5.0, upper=5.0, n_starts=128,
                              pso_iters=5, bfgs_max_iters=100, ls_max_iters=20, grad_tol=1e-8,
                              w=0.7, c1=1.5, c2=1.5, armijo_c=1e-4, backtrack=0.5, seed=0),
    # 10-D Rastrigin: 16384 particles in [-5.12,5.12]^10, 20 PSO updates, 1000 BFGS iterations
    "rastrigin10d_n16384": dict(objective="rastrigin", dim=10, lower=-5.12, upper=5.12,
                                n_starts=16384, pso_iters=20, bfgs_max_iters=1000, ls_max_iters=20,
                                grad_tol=1e-8, w=0.7, c1=1.5, c2=1.5, armijo_c=1e-4, backtrack=0.5,
                                seed=0),
    # 5-D Rastrigin: 16384 particles in [-5.12,5.12]^5, 20 PSO updates, 1000 BFGS iterations
    "rastrigin5d_n16384": dict(objective="rastrigin", dim=5, lower=-5.12, upper=5.12,
                               n_starts=16384, pso_iters=20, bfgs_max_iters=1000, ls_max_iters=20,
                               grad_tol=1e-8, w=0.7, c1=1.5, c2=1.5, armijo_c=1e-4, backtrack=0.5,
                               seed=0),
    # Rosenbrock chain d=256: 8192 particles in [-2,2]^256, 10 PSO updates, 2000 iterations
    "rosenbrock256d_n8192": dict(objective="rosenbrock", dim=256, lower=-2.0, upper=2.0,
                                 n_starts=8192, pso_iters=10, bfgs_max_iters=2000, ls_max_iters=20,
                                 grad_tol=1e-8, w=0.7, c1=1.5, c2=1.5, armijo_c=1e-4,
                                 backtrack=0.5, seed=0),
    # d=1024 Ackley / Rosenbrock chain: 2048 particles in [-5,5]^1024, 10 PSO, 500 iterations
    "ackley1024d_n2048": dict(objective="ackley", dim=1024, lower=-5.0, upper=5.0, n_starts=2048,
                              pso_iters=10, bfgs_max_iters=500, ls_max_iters=20, grad_tol=1e-8,
                              w=0.7, c1=1.5, c2=1.5, armijo_c=1e-4, backtrack=0.5, seed=0),
    "rosenbrock1024d_n2048": dict(objective="rosenbrock", dim=1024, lower=-5.0, upper=5.0,
                                  n_starts=2048, pso_iters=10, bfgs_max_iters=500, ls_max_iters=20,
                                  grad_tol=1e-8, w=0.7, c1=1.5, c2=1.5, armijo_c=1e-4,
                                  backtrack=0.5, seed=0),
    # a user objective (the default plug-in's Griewank, not built in): 16384
    # particles in its usual box [-600,600]^10, 20 PSO updates, 1000 iterations
    "griewank10d_n16384": dict(objective="griewank", dim=10, lower=-600.0, upper=600.0,
                               n_starts=16384, pso_iters=20, bfgs_max_iters=1000, ls_max_iters=20,
                               grad_tol=1e-8, w=0.7, c1=1.5, c2=1.5, armijo_c=1e-4, backtrack=0.5,
                               seed=0),
}

# batched form: many independent problems, each with its own swarm
BATCH_WORKLOADS = {
    # 4096 problems x 256 starts (2^20 starts), d log-uniform in [2, 128],
    # objective uniform over Rosenbrock chain / Rastrigin / Ackley, 10 PSO
    # updates, BFGS cap 500, FP64
    "mixed4096_n256": dict(n_problems=4096, n_starts=256, pso_iters=10, bfgs_max_iters=500,
                           mix_seed=12345, dmin=2, dmax=128),
}

# sampling box per objective for the mixed batches
BOXES = {"rosenbrock": (-5.0, 5.0), "rastrigin": (-5.12, 5.12), "ackley": (-5.0, 5.0)}


def workload(name: str, **override) -> dict:
    d = dict(WORKLOADS[name])
    d.update(override)
    return d


def start_points(n: int, d: int, lo: float, hi: float, seed: int) -> np.ndarray:
    """n seeded start points, uniform in [lo, hi)^d, row-major [n][d]."""
    rng = np.random.default_rng(seed)
    return rng.uniform(lo, hi, size=(n, d))


def mixed_batch(n_problems: int, seed: int = 12345, dmin: int = 2, dmax: int = 128):
    """Seeded list of problems for the batched form: d log-uniform in
    [dmin, dmax] (rounded), objective uniform over Rosenbrock chain,
    Rastrigin and Ackley, each on its usual box."""
    rng = np.random.default_rng(seed)
    dims = np.rint(np.exp(rng.uniform(np.log(dmin), np.log(dmax), size=n_problems))).astype(int)
    objs = rng.choice(["rosenbrock", "rastrigin", "ackley"], size=n_problems)
    return [dict(objective=str(o), dim=int(d), lower=BOXES[o][0], upper=BOXES[o][1])
            for o, d in zip(objs, dims)]


def batch_problems(name: str, n_problems: int | None = None, **override) -> list[dict]:
    """Problem fields of a batched workload (optionally its first n_problems);
    problem P gets seed P."""
    w = dict(BATCH_WORKLOADS[name])
    mix = mixed_batch(w["n_problems"], seed=w["mix_seed"], dmin=w["dmin"], dmax=w["dmax"])
    if n_problems is not None:
        mix = mix[:n_problems]
    out = []
    for P, m in enumerate(mix):
        f = dict(m, n_starts=w["n_starts"], pso_iters=w["pso_iters"],
                 bfgs_max_iters=w["bfgs_max_iters"], seed=P)
        f.update(override)
        out.append(f)
    return out
