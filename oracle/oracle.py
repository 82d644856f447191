"""ctypes/numpy marshalling for the C oracle (``zeus_oracle.c``).

TEST INFRASTRUCTURE ONLY (see the package docstring).  No arithmetic of the
method lives here: every number is computed by the C file, this module
builds it with gcc, converts arguments and allocates result arrays.
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess
import tempfile
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "zeus_oracle.c")
_BUILD_DIR = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD_DIR, "libzeus_oracle.so")

# rounding orders of zeus_oracle.c (see its ZO_ORDER_* note)
ORDER_LIB = 0
ORDER_PLAIN = 1

# Section V-B test functions; QUADRATIC is a test objective 0.5*sum (i+1) x_i^2.
OBJECTIVES = {"rosenbrock": 0, "rastrigin": 1, "ackley": 2,
              "goldstein_price": 3, "quadratic": 100,
              # objectives a user adds to the library (not built in there)
              "griewank": 200, "himmelblau": 201}


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (FP64, no FMA contraction, OpenMP)."""
    if (not force and os.path.exists(_SO)
            and os.path.getmtime(_SO) >= os.path.getmtime(_SRC)):
        return _SO
    os.makedirs(_BUILD_DIR, exist_ok=True)
    fd, tmp = tempfile.mkstemp(suffix=".so", dir=_BUILD_DIR)
    os.close(fd)
    cmd = ["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fno-fast-math",
           "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


class _Problem(C.Structure):
    _fields_ = [
        ("objective", C.c_int32), ("dim", C.c_int32),
        ("lower", C.c_double), ("upper", C.c_double),
        ("n_starts", C.c_int64),
        ("pso_iters", C.c_int32), ("bfgs_max_iters", C.c_int32),
        ("ls_max_iters", C.c_int32), ("required_converged", C.c_int32),
        ("grad_tol", C.c_double),
        ("w", C.c_double), ("c1", C.c_double), ("c2", C.c_double),
        ("armijo_c", C.c_double), ("backtrack", C.c_double),
        ("target_f", C.c_double),
        ("seed", C.c_uint64),
        ("start_from_pbest", C.c_int32), ("n_threads", C.c_int32),
        ("lbfgs_m", C.c_int32), ("order", C.c_int32),
    ]


class _Result(C.Structure):
    _fields_ = [("f", C.c_double), ("gnorm", C.c_double), ("margin", C.c_double),
                ("iters", C.c_int32), ("status", C.c_int32),
                ("n_feval", C.c_int32), ("pad", C.c_int32)]


@dataclass
class Problem:
    """Arguments of the parallel Zeus procedure (Alg. 7).  Defaults: the
    2-D Rosenbrock workload (128 particles, 5 PSO iterations, w=0.7,
    c1=c2=1.5, Armijo c=1e-4, backtracking 0.5, 20 trials, 100 BFGS
    iterations, ||g|| < 1e-8)."""
    objective: str | int = "rosenbrock"
    dim: int = 2
    lower: float = -5.0
    upper: float = 5.0
    n_starts: int = 128
    pso_iters: int = 5
    bfgs_max_iters: int = 100
    ls_max_iters: int = 20
    required_converged: int = 0
    grad_tol: float = 1e-8
    w: float = 0.7
    c1: float = 1.5
    c2: float = 1.5
    armijo_c: float = 1e-4
    backtrack: float = 0.5
    target_f: float = float("nan")
    seed: int = 0
    start_from_pbest: int = 0
    n_threads: int = 0
    lbfgs_m: int = 0  # 0: dense inverse Hessian (Alg. 4); m > 0: L-BFGS with m pairs
    # rounding order of sums and the update: ORDER_LIB (fma per product term,
    # 32-chain sums past 32 terms, mirrored triangle) or ORDER_PLAIN (every
    # operation rounded on its own, sums left to right, whole-matrix update)
    order: int = 0

    def obj_id(self) -> int:
        o = self.objective
        return OBJECTIVES[o] if isinstance(o, str) else int(o)

    def c(self) -> _Problem:
        return _Problem(self.obj_id(), self.dim, self.lower, self.upper,
                        self.n_starts, self.pso_iters, self.bfgs_max_iters,
                        self.ls_max_iters, self.required_converged,
                        self.grad_tol, self.w, self.c1, self.c2,
                        self.armijo_c, self.backtrack, self.target_f,
                        self.seed & (2**64 - 1), self.start_from_pbest,
                        self.n_threads, self.lbfgs_m, int(self.order))


class _ClusterResult(C.Structure):
    _fields_ = [("n_candidates", C.c_int64), ("n_clusters", C.c_int64), ("n_left", C.c_int64),
                ("best_count", C.c_int64), ("best_leader", C.c_int64), ("best_f", C.c_double),
                ("best_spread", C.c_double), ("error", C.c_int32), ("pad", C.c_int32)]


_lib = None
_D = C.POINTER(C.c_double)
_U64 = C.POINTER(C.c_uint64)
_I64 = C.POINTER(C.c_int64)
_I32 = C.POINTER(C.c_int)


def lib():
    global _lib
    if _lib is not None:
        return _lib
    L = C.CDLL(build())
    L.zo_philox4x64_10.argtypes = [_U64, _U64, _U64]
    L.zo_uniform.argtypes = [C.c_uint64] * 5
    L.zo_uniform.restype = C.c_double
    L.zo_dual_op.argtypes = [C.c_int, C.c_double, C.c_double, C.c_double,
                             C.c_double, _D, _D]
    L.zo_sincos2pi.argtypes = [C.c_double, _D, _D]
    L.zo_exp.argtypes = [C.c_double]
    L.zo_exp.restype = C.c_double
    L.zo_f.argtypes = [C.c_int, C.c_int, _D]
    L.zo_f.restype = C.c_double
    L.zo_f_ord.argtypes = [C.c_int, C.c_int, _D, C.c_int]
    L.zo_f_ord.restype = C.c_double
    L.zo_grad_forward.argtypes = [C.c_int, C.c_int, _D, _D, _D]
    L.zo_grad_forward_ord.argtypes = [C.c_int, C.c_int, _D, _D, _D, C.c_int]
    L.zo_dot_plain.argtypes = [C.c_int, _D, _D]
    L.zo_dot_plain.restype = C.c_double
    L.zo_direction.argtypes = [C.c_int, _D, _D, _D, _D, C.c_int]
    L.zo_direction.restype = C.c_int
    L.zo_bfgs_update_ord.argtypes = [C.c_int, _D, _D, _D, C.c_int]
    L.zo_bfgs_update_ord.restype = C.c_int
    L.zo_lbfgs_direction_ord.argtypes = [C.c_int, C.c_int, _D, _D, _D, _D, _D, C.c_int]
    L.zo_line_search_ord.argtypes = [C.c_int, C.c_int, _D, _D, C.c_double, C.c_double,
                                     C.c_double, C.c_double, C.c_int, _D, _I32, _I32, _D,
                                     C.c_int]
    L.zo_line_search_ord.restype = C.c_double
    L.zo_cluster.argtypes = [C.c_int, C.c_double, C.c_int32, C.c_int, C.c_int64, C.c_int, _D,
                             _D, _I32, _I32, _I32, _I32, C.POINTER(_ClusterResult)]
    L.zo_dot_split.argtypes = [C.c_int, _D, _D]
    L.zo_dot_split.restype = C.c_double
    L.zo_argmin.argtypes = [_D, C.c_int64]
    L.zo_argmin.restype = C.c_int64
    L.zo_pso.argtypes = [C.POINTER(_Problem), _D, _D, _D, _D, _D, _D, _I64]
    L.zo_line_search.argtypes = [C.c_int, C.c_int, _D, _D, C.c_double,
                                 C.c_double, C.c_double, C.c_double, C.c_int,
                                 _D, _I32, _I32, _D]
    L.zo_line_search.restype = C.c_double
    L.zo_bfgs_update.argtypes = [C.c_int, _D, _D, _D]
    L.zo_lbfgs_direction.argtypes = [C.c_int, C.c_int, _D, _D, _D, _D, _D]
    L.zo_bfgs_update.restype = C.c_int
    L.zo_bfgs.argtypes = [C.POINTER(_Problem), _D, _D, C.POINTER(_Result),
                          C.c_void_p, C.c_void_p]
    L.zo_bfgs_many.argtypes = [C.POINTER(_Problem), C.c_int64, _D, _D,
                               C.POINTER(_Result)]
    L.zo_solve.argtypes = [C.POINTER(_Problem), _D, _D, _D, _D, _D, _D,
                           C.POINTER(_Result)]
    L.zo_solve.restype = C.c_int64
    L.zo_bfgs_quadratic_exact.argtypes = [C.c_int, _D, _D, C.c_int,
                                          C.c_double, _D, _D, C.c_int]
    L.zo_bfgs_quadratic_exact.restype = C.c_int
    L.zo_max_threads.restype = C.c_int
    assert L.zo_sizeof_problem() == C.sizeof(_Problem)
    assert L.zo_sizeof_result() == C.sizeof(_Result)
    _lib = L
    return L


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_D)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def max_threads() -> int:
    return int(lib().zo_max_threads())


def philox4x64_10(ctr, key) -> np.ndarray:
    """Philox4x64-10 block function (Salmon et al., SC'11)."""
    c = np.ascontiguousarray(np.asarray(ctr, dtype=np.uint64))
    k = np.ascontiguousarray(np.asarray(key, dtype=np.uint64))
    out = np.zeros(4, dtype=np.uint64)
    lib().zo_philox4x64_10(c.ctypes.data_as(_U64), k.ctypes.data_as(_U64),
                           out.ctypes.data_as(_U64))
    return out


def uniform(seed: int, problem: int, phase: int, particle: int, j: int) -> float:
    """The uniform draw of (phase, particle, dimension j) (Section IV-A reading)."""
    return float(lib().zo_uniform(seed & (2**64 - 1), problem, phase, particle, j))


def sincos2pi(x: float):
    """(sin 2 pi x, cos 2 pi x) by the oracle's own exact-reduction Taylor method."""
    sv, cv = C.c_double(), C.c_double()
    lib().zo_sincos2pi(float(x), C.byref(sv), C.byref(cv))
    return sv.value, cv.value


def exp(x: float) -> float:
    """e^x by the oracle's own Cody-Waite / Taylor method."""
    return float(lib().zo_exp(float(x)))


def dual_op(op: str, a1, b1, a2=0.0, b2=0.0):
    """One dual-number operation (Section III-C): returns (value, tangent)."""
    code = ["add", "sub", "mul", "div", "sin", "cos", "exp", "sqrt", "cos2pi"].index(op)
    ra, rb = C.c_double(), C.c_double()
    lib().zo_dual_op(code, a1, b1, a2, b2, C.byref(ra), C.byref(rb))
    return ra.value, rb.value


def _obj(o) -> int:
    return OBJECTIVES[o] if isinstance(o, str) else int(o)


def f(objective, x, order: int = ORDER_LIB) -> float:
    """Objective value (Section V-B), its sums in the given rounding order."""
    x = _f64(x)
    return float(lib().zo_f_ord(_obj(objective), x.size, _dp(x), int(order)))


def grad_forward(objective, x, order: int = ORDER_LIB):
    """Forward-mode gradient by d dual passes (Alg. 5); returns (f, g)."""
    x = _f64(x)
    g = np.zeros_like(x)
    fv = C.c_double()
    lib().zo_grad_forward_ord(_obj(objective), x.size, _dp(x), C.byref(fv), _dp(g), int(order))
    return fv.value, g


def argmin(fv) -> int:
    """Best-of-swarm reduction (Alg. 7): NaN as +inf, ties to the lowest index."""
    fv = _f64(fv)
    return int(lib().zo_argmin(_dp(fv), fv.size))


def pso(p: Problem) -> dict:
    """PSO phase (Alg. 2 then Alg. 3 pso_iters times, synchronous gbest)."""
    n, d = p.n_starts, p.dim
    x = np.zeros((n, d)); v = np.zeros((n, d)); px = np.zeros((n, d))
    pf = np.zeros(n); gx = np.zeros(d); gf = C.c_double(); gi = C.c_int64()
    pc = p.c()
    lib().zo_pso(C.byref(pc), _dp(x), _dp(v), _dp(px), _dp(pf), _dp(gx),
                 C.byref(gf), C.byref(gi))
    return dict(x=x, v=v, px=px, pf=pf, gx=gx, gf=gf.value, gidx=gi.value)


def line_search(objective, x, p, f0, ddir, c=1e-4, beta=0.5, L=20, order: int = ORDER_LIB):
    """Backtracking Armijo line search (Alg. 6): returns (alpha, accepted, n_feval)."""
    x = _f64(x); p = _f64(p)
    xt = np.zeros_like(x)
    acc = C.c_int(); nf = C.c_int(0); mg = C.c_double(math.inf)
    a = lib().zo_line_search_ord(_obj(objective), x.size, _dp(x), _dp(p), f0, ddir,
                                 c, beta, L, _dp(xt), C.byref(acc), C.byref(nf),
                                 C.byref(mg), int(order))
    return float(a), bool(acc.value), int(nf.value)


def bfgs_update(H, s, y, order: int = ORDER_LIB):
    """Inverse-Hessian rank-two update of Alg. 4; returns (H_new, applied)."""
    H = _f64(H).copy(); s = _f64(s); y = _f64(y)
    ok = lib().zo_bfgs_update_ord(s.size, _dp(H), _dp(s), _dp(y), int(order))
    return H, bool(ok)


def direction(H, g, order: int = ORDER_LIB):
    """Search direction of Alg. 4 with the non-descent reset: returns
    (p, H after the call, g'p, reset taken)."""
    H = _f64(H).copy(); g = _f64(g)
    p = np.zeros_like(g)
    dd = C.c_double()
    r = lib().zo_direction(g.size, _dp(H), _dp(g), _dp(p), C.byref(dd), int(order))
    return p, H, dd.value, bool(r)


def _results(res, n):
    return dict(
        f=np.array([res[i].f for i in range(n)]),
        gnorm=np.array([res[i].gnorm for i in range(n)]),
        margin=np.array([res[i].margin for i in range(n)]),
        iters=np.array([res[i].iters for i in range(n)], dtype=np.int32),
        status=np.array([res[i].status for i in range(n)], dtype=np.int32),
        n_feval=np.array([res[i].n_feval for i in range(n)], dtype=np.int32))


def bfgs(p: Problem, x0):
    """One BFGS run from x0 (Alg. 4); returns dict with x and the result."""
    x0 = _f64(x0)
    xo = np.zeros_like(x0)
    r = _Result()
    pc = p.c()
    lib().zo_bfgs(C.byref(pc), _dp(x0), _dp(xo), C.byref(r), None, None)
    out = _results([r], 1)
    out = {k: v[0] for k, v in out.items()}
    out["x"] = xo
    return out


def bfgs_many(p: Problem, x0):
    """BFGS from each row of x0 ([n, d]); OpenMP over starts."""
    x0 = _f64(x0)
    n = x0.shape[0]
    xo = np.zeros_like(x0)
    res = (_Result * max(n, 1))()
    pc = p.c()
    lib().zo_bfgs_many(C.byref(pc), n, _dp(x0), _dp(xo), res)
    out = _results(res, n)
    out["x"] = xo
    return out


def solve(p: Problem) -> dict:
    """Whole method (Alg. 7): PSO, BFGS from every particle, argmin."""
    n, d = p.n_starts, p.dim
    x = np.zeros((n, d)); v = np.zeros((n, d)); px = np.zeros((n, d))
    pf = np.zeros(n); gx = np.zeros(d); xo = np.zeros((n, d))
    res = (_Result * max(n, 1))()
    pc = p.c()
    b = lib().zo_solve(C.byref(pc), _dp(x), _dp(v), _dp(px), _dp(pf), _dp(gx),
                       _dp(xo), res)
    out = _results(res, n)
    out.update(x=xo, swarm=x, v=v, px=px, pf=pf, gx=gx, best=int(b))
    return out


def bfgs_quadratic_exact(A, x0, max_iters=100, tol=1e-10, order: int = ORDER_LIB):
    """Test-only BFGS with exact steps on 0.5 x^T A x; returns (iters, x, H)."""
    A = _f64(A); x0 = _f64(x0)
    d = x0.size
    xo = np.zeros(d); H = np.zeros((d, d))
    k = lib().zo_bfgs_quadratic_exact(d, _dp(A), _dp(x0), max_iters, tol,
                                      _dp(xo), _dp(H), int(order))
    return int(k), xo, H


def lbfgs_direction(S, Y, g, order: int = ORDER_LIB):
    """Two-loop L-BFGS direction p = -H g over the pairs (rows of S and Y,
    oldest first) with the initial matrix gamma I."""
    S = np.ascontiguousarray(S, dtype=np.float64)
    Y = np.ascontiguousarray(Y, dtype=np.float64)
    g = np.ascontiguousarray(g, dtype=np.float64)
    n, d = (S.shape[0], g.shape[0]) if S.size else (0, g.shape[0])
    rho = np.array([1.0 / float(np.dot(Y[i], S[i])) for i in range(n)], dtype=np.float64)
    p = np.zeros(d)
    lib().zo_lbfgs_direction_ord(d, n, _dp(S if n else np.zeros(1)),
                                 _dp(Y if n else np.zeros(1)), _dp(rho if n else np.zeros(1)),
                                 _dp(g), _dp(p), int(order))
    return p


CLUSTER_METHODS = {"f": 0, "x": 1}


def cluster(x, f, status=None, method="x", tol=1e-3, max_clusters=256, only_converged=False):
    """Leader clustering of final points (the reading of Section VI's
    clustering in zeus_oracle.c): labels [n] (cluster id, -1 not a
    candidate, -2 left), leaders and counts [max_clusters], summary."""
    f = _f64(f)
    n = f.size
    x = _f64(x).reshape(n, -1) if x is not None else np.zeros((n, 1))
    d = x.shape[1]
    st = (np.ascontiguousarray(status, dtype=np.int32) if status is not None
          else np.ones(n, dtype=np.int32))
    lab = np.zeros(max(n, 1), dtype=np.int32)
    lead = np.zeros(max_clusters, dtype=np.int32)
    cnt = np.zeros(max_clusters, dtype=np.int32)
    r = _ClusterResult()
    m = CLUSTER_METHODS[method] if isinstance(method, str) else int(method)
    p32 = C.POINTER(C.c_int)
    lib().zo_cluster(m, float(tol), int(max_clusters), int(only_converged), n, d, _dp(x), _dp(f),
                     st.ctypes.data_as(p32), lab.ctypes.data_as(p32), lead.ctypes.data_as(p32),
                     cnt.ctypes.data_as(p32), C.byref(r))
    summary = {k: getattr(r, k) for k, _ in _ClusterResult._fields_}
    return dict(labels=lab[:n], leaders=lead, counts=cnt, summary=summary)


def dot_plain(a, b) -> float:
    """The BFGS dot product in the plain order: left to right, each
    product and each sum rounded on its own."""
    a, b = _f64(a), _f64(b)
    return float(lib().zo_dot_plain(a.size, _dp(a), _dp(b)))


def dot_split(a, b) -> float:
    """The BFGS dot product as read in zeus_oracle.c (zo_bdot): one fma
    chain for n <= 32, else 32 strided partial chains and a fixed tree."""
    a, b = _f64(a), _f64(b)
    return float(lib().zo_dot_split(a.size, _dp(a), _dp(b)))
