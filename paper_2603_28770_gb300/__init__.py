"""GB300 (sm_103a) implementation of the data-parallel hot path of Zeus
(arXiv 2603.28770): PSO seeding, one BFGS run per start with forward-mode
dual-number (or reverse-mode adjoint) gradients, backtracking Armijo line
search and the dense inverse-Hessian rank-two update, and a best-of-swarm
reduction.

The arithmetic runs in the CUDA kernels of ``libzeus.so`` behind the C ABI
of ``include/zeus.h``.  This module is the thin binding above it: functions
named like the C entry points marshal torch CUDA tensors (device memory) and
the current torch stream; PyTorch is plumbing here, not the compute path.
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass, fields

import torch

from . import _capi
from ._capi import (GRAD_MODES, OBJECTIVES, PRECISIONS, RUN_STATUS, ZeusError, check, lib,
                    objective_code, user_objectives,
                    library_path, strerror, zeus_problem, zeus_result)

__all__ = [
    "Problem", "ZeusError", "zeus_solve", "zeus_solve_from", "zeus_solve_from_noalloc", "zeus_pso", "zeus_objective_eval",
    "zeus_objective_eval_f32", "zeus_argmin", "zeus_argmin_workspace_size", "zeus_uniform",
    "zeus_workspace_size", "zeus_plan_info", "zeus_validate", "zeus_default_problem", "zeus_strerror",
    "zeus_abi_version", "zeus_set_wait_limit", "zeus_math_eval", "Context", "solve", "solve_from", "pso", "objective", "ObjectiveFn",
    "decode_result", "library_path", "lib", "zeus_batch_plan_make", "zeus_batch_prepare",
    "zeus_batch_solve", "Batch", "user_objectives", "zeus_cluster", "zeus_cluster_workspace_size", "cluster", "solve_until_confident",
    "precision_error",
]


@dataclass
class Problem:
    """Arguments of the parallel Zeus procedure (Alg. 7).  Field meanings and
    ranges are those of ``zeus_problem`` in include/zeus.h; the defaults are
    ``zeus_default_problem`` (2-D Rosenbrock, 128 particles, 5 PSO updates)."""
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
    precision: str | int = "fp64"
    grad_mode: str | int = "forward"
    start_from_pbest: int = 0
    threads_per_start: int = 0
    lbfgs_m: int = 0

    def to_c(self) -> zeus_problem:
        def code(v, table):
            return table[v] if isinstance(v, str) else int(v)
        return zeus_problem(
            objective_code(self.objective), self.dim, self.lower, self.upper, self.n_starts,
            self.pso_iters, self.bfgs_max_iters, self.ls_max_iters, self.required_converged,
            self.grad_tol, self.w, self.c1, self.c2, self.armijo_c, self.backtrack,
            self.target_f, self.seed & (2**64 - 1), code(self.precision, PRECISIONS),
            code(self.grad_mode, GRAD_MODES), self.start_from_pbest, self.threads_per_start,
            self.lbfgs_m, 0)

    def replace(self, **kw) -> "Problem":
        d = {f.name: getattr(self, f.name) for f in fields(self)}
        d.update(kw)
        return Problem(**d)


# ------------------------------------------------------------------ helpers

def _ptr(t: torch.Tensor | None, dtype=None, numel=None, name="") -> int | None:
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError(f"{name}: expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name}: expected a contiguous tensor")
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"{name}: expected {dtype}, got {t.dtype}")
    if numel is not None and t.numel() < numel:
        raise ValueError(f"{name}: needs {numel} elements, has {t.numel()}")
    return t.data_ptr()


def _stream(stream) -> int | None:
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


def _prob(p) -> zeus_problem:
    return p.to_c() if isinstance(p, Problem) else p


RESULT_BYTES = C.sizeof(zeus_result)


def new_result(device="cuda") -> torch.Tensor:
    """Device buffer for one zeus_result."""
    return torch.empty(RESULT_BYTES, dtype=torch.uint8, device=device)


def decode_result(t: torch.Tensor) -> dict:
    """zeus_result buffer (device or host) -> dict (synchronizes if on device)."""
    raw = bytes(t.detach().cpu().numpy().tobytes())
    r = zeus_result.from_buffer_copy(raw)
    return {name: getattr(r, name) for name, _ in zeus_result._fields_}


# ------------------------------------------------- same-name entry points

def zeus_strerror(code: int) -> str:
    return strerror(code)


def zeus_abi_version() -> int:
    return lib().zeus_abi_version()


def zeus_set_wait_limit(polls: int) -> None:
    """Polls (about 256 ns each) a bounded device wait makes before it
    gives up and sets the call's error word; 0 restores the default
    (about two seconds).  Process-wide."""
    check(lib().zeus_set_wait_limit(int(polls)), "zeus_set_wait_limit")


def zeus_default_problem() -> zeus_problem:
    p = zeus_problem()
    check(lib().zeus_default_problem(C.byref(p)), "zeus_default_problem")
    return p


def zeus_validate(problem) -> int:
    return lib().zeus_validate(C.byref(_prob(problem)))


def zeus_plan_info(problem) -> dict:
    """Which kernels a solve of this problem runs."""
    pl = _capi.zeus_plan()
    check(lib().zeus_plan_info(C.byref(_prob(problem)), C.byref(pl)), "zeus_plan_info")
    return {name: getattr(pl, name) for name, _ in _capi.zeus_plan._fields_}


def zeus_workspace_size(problem) -> int:
    n = C.c_size_t()
    check(lib().zeus_workspace_size(C.byref(_prob(problem)), C.byref(n)), "zeus_workspace_size")
    return n.value


def new_workspace(problem, device="cuda") -> torch.Tensor:
    return torch.empty(max(zeus_workspace_size(problem), 256), dtype=torch.uint8, device=device)


def zeus_solve(problem, workspace, x_out, f_out=None, gnorm_out=None, status_out=None,
               iters_out=None, result=None, stream=None) -> None:
    pc = _prob(problem)
    n, d = pc.n_starts, pc.dim
    check(lib().zeus_solve(
        C.byref(pc), _ptr(workspace, torch.uint8, name="workspace"), workspace.numel(),
        _ptr(x_out, torch.float64, n * d, "x_out"), _ptr(f_out, torch.float64, n, "f_out"),
        _ptr(gnorm_out, torch.float64, n, "gnorm_out"),
        _ptr(status_out, torch.int32, n, "status_out"), _ptr(iters_out, torch.int32, n, "iters_out"),
        _ptr(result, torch.uint8, RESULT_BYTES, "result"), _stream(stream)), "zeus_solve")


def zeus_solve_from(problem, x0, workspace, x_out, f_out=None, gnorm_out=None, status_out=None,
                    iters_out=None, result=None, stream=None) -> None:
    pc = _prob(problem)
    n, d = pc.n_starts, pc.dim
    check(lib().zeus_solve_from(
        C.byref(pc), _ptr(x0, torch.float64, n * d, "x0"),
        _ptr(workspace, torch.uint8, name="workspace"), workspace.numel(),
        _ptr(x_out, torch.float64, n * d, "x_out"), _ptr(f_out, torch.float64, n, "f_out"),
        _ptr(gnorm_out, torch.float64, n, "gnorm_out"),
        _ptr(status_out, torch.int32, n, "status_out"), _ptr(iters_out, torch.int32, n, "iters_out"),
        _ptr(result, torch.uint8, RESULT_BYTES, "result"), _stream(stream)), "zeus_solve_from")


def zeus_solve_from_noalloc(problem, x0, x_out, f_out, gnorm_out=None, status_out=None,
                            iters_out=None, result=None, stream=None) -> None:
    """zeus_solve_from without a workspace: for callers that cannot allocate
    device memory (the library uses one static device array instead)."""
    pc = _prob(problem)
    n, d = pc.n_starts, pc.dim
    check(lib().zeus_solve_from_noalloc(
        C.byref(pc), _ptr(x0, torch.float64, n * d, "x0"), _ptr(x_out, torch.float64, n * d, "x_out"),
        _ptr(f_out, torch.float64, n, "f_out"), _ptr(gnorm_out, torch.float64, n, "gnorm_out"),
        _ptr(status_out, torch.int32, n, "status_out"), _ptr(iters_out, torch.int32, n, "iters_out"),
        _ptr(result, torch.uint8, RESULT_BYTES, "result"), _stream(stream)), "zeus_solve_from_noalloc")


def zeus_pso(problem, workspace, x_out, v_out, px_out, pf_out, gx_out, result=None,
             stream=None) -> None:
    pc = _prob(problem)
    n, d = pc.n_starts, pc.dim
    check(lib().zeus_pso(
        C.byref(pc), _ptr(workspace, torch.uint8, name="workspace"), workspace.numel(),
        _ptr(x_out, torch.float64, n * d, "x_out"), _ptr(v_out, torch.float64, n * d, "v_out"),
        _ptr(px_out, torch.float64, n * d, "px_out"), _ptr(pf_out, torch.float64, n, "pf_out"),
        _ptr(gx_out, torch.float64, d, "gx_out"), _ptr(result, torch.uint8, RESULT_BYTES, "result"),
        _stream(stream)), "zeus_pso")


def _obj_code(o) -> int:
    return objective_code(o)


def _grad_code(g) -> int:
    return GRAD_MODES[g] if isinstance(g, str) else int(g)


def zeus_objective_eval(objective, dim, x, f_out=None, g_out=None, grad_mode=0, stream=None):
    n = x.numel() // dim
    check(lib().zeus_objective_eval(
        _obj_code(objective), dim, n, _ptr(x, torch.float64, n * dim, "x"),
        _ptr(f_out, torch.float64, n, "f_out"), _ptr(g_out, torch.float64, n * dim, "g_out"),
        _grad_code(grad_mode), _stream(stream)), "zeus_objective_eval")


def zeus_objective_eval_f32(objective, dim, x, f_out=None, g_out=None, grad_mode=0, stream=None):
    n = x.numel() // dim
    check(lib().zeus_objective_eval_f32(
        _obj_code(objective), dim, n, _ptr(x, torch.float32, n * dim, "x"),
        _ptr(f_out, torch.float32, n, "f_out"), _ptr(g_out, torch.float32, n * dim, "g_out"),
        _grad_code(grad_mode), _stream(stream)), "zeus_objective_eval_f32")


def zeus_argmin_workspace_size(n: int) -> int:
    b = C.c_size_t()
    check(lib().zeus_argmin_workspace_size(n, C.byref(b)), "zeus_argmin_workspace_size")
    return b.value


def zeus_argmin(f, workspace, result, stream=None) -> None:
    check(lib().zeus_argmin(_ptr(f, torch.float64, name="f"), f.numel(),
                            _ptr(workspace, torch.uint8, name="workspace"), workspace.numel(),
                            _ptr(result, torch.uint8, RESULT_BYTES, "result"), _stream(stream)),
          "zeus_argmin")


def zeus_uniform(seed, problem_index, phase, n, dim, out, stream=None) -> None:
    check(lib().zeus_uniform(seed & (2**64 - 1), problem_index, phase, n, dim,
                             _ptr(out, torch.float64, n * dim, "out"), _stream(stream)),
          "zeus_uniform")


def zeus_math_eval(fn: int, x, y0, y1=None, stream=None) -> None:
    check(lib().zeus_math_eval(fn, x.numel(), _ptr(x, torch.float64, name="x"),
                               _ptr(y0, torch.float64, x.numel(), "y0"),
                               _ptr(y1, torch.float64, x.numel(), "y1"), _stream(stream)),
          "zeus_math_eval")


class Context:
    """zeus_context: the host-buffer interface (zeus_solve_host)."""

    def __init__(self):
        h = C.c_void_p()
        check(lib().zeus_context_create(C.byref(h)), "zeus_context_create")
        self._h = h

    def close(self):
        if self._h:
            lib().zeus_context_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def zeus_solve_host(self, problem, x_out, f_out=None, gnorm_out=None, status_out=None,
                        iters_out=None, stream=None) -> dict:
        """Host (numpy / pinned CPU tensor) outputs; returns the decoded result."""
        pc = _prob(problem)
        res = zeus_result()

        def hp(a):
            if a is None:
                return None
            if isinstance(a, torch.Tensor):
                assert not a.is_cuda and a.is_contiguous()
                return a.data_ptr()
            assert a.flags.c_contiguous
            return a.ctypes.data

        check(lib().zeus_solve_host(self._h, C.byref(pc), hp(x_out), hp(f_out), hp(gnorm_out),
                                    hp(status_out), hp(iters_out), C.addressof(res),
                                    _stream(stream)), "zeus_solve_host")
        return {name: getattr(res, name) for name, _ in zeus_result._fields_}


# ------------------------------------------------------------ batched form

def _prob_array(problems):
    arr = (zeus_problem * len(problems))()
    for i, p in enumerate(problems):
        arr[i] = _prob(p)
    return arr


def zeus_batch_plan_make(problems) -> _capi.zeus_batch_plan:
    """Host-only plan of a batch (work list classes, workspace size)."""
    arr = _prob_array(problems)
    plan = _capi.zeus_batch_plan()
    check(lib().zeus_batch_plan_make(arr, len(problems), C.byref(plan)), "zeus_batch_plan_make")
    return plan


def zeus_batch_prepare(problems, plan, workspace, stream=None) -> None:
    """Upload the batch's tables into the workspace (synchronizes the stream)."""
    arr = _prob_array(problems)
    check(lib().zeus_batch_prepare(arr, len(problems), C.byref(plan),
                                   _ptr(workspace, torch.uint8, name="workspace"),
                                   workspace.numel(), _stream(stream)), "zeus_batch_prepare")


def zeus_batch_solve(plan, workspace, x_out, f_out, gnorm_out=None, status_out=None,
                     iters_out=None, results=None, stream=None) -> None:
    """Run a prepared batch (kernels only: capturable in a CUDA graph)."""
    ns, nc, npb = plan.total_starts, plan.total_coords, plan.n_problems
    check(lib().zeus_batch_solve(
        C.byref(plan), _ptr(workspace, torch.uint8, name="workspace"), workspace.numel(),
        _ptr(x_out, torch.float64, nc, "x_out"), _ptr(f_out, torch.float64, ns, "f_out"),
        _ptr(gnorm_out, torch.float64, ns, "gnorm_out"),
        _ptr(status_out, torch.int32, ns, "status_out"), _ptr(iters_out, torch.int32, ns, "iters_out"),
        _ptr(results, torch.uint8, npb * RESULT_BYTES, "results"), _stream(stream)),
        "zeus_batch_solve")


class Batch:
    """A prepared batch of problems: owns the workspace and the concatenated
    outputs; ``solve()`` runs it, ``capture()`` records one solve in a CUDA
    graph that ``replay()`` runs again (same tables, same outputs).  With an
    ``autotune.Autotuner`` the per-start layout of each problem is the
    measured fastest (the results do not depend on it)."""

    def __init__(self, problems, device="cuda", stream=None, autotuner=None):
        self.problems = [_prob(p) for p in problems]
        if autotuner is not None:  # per-start layout chosen by measurement
            self.problems = autotuner.apply(self.problems)
        self.plan = zeus_batch_plan_make(self.problems)
        pl = self.plan
        self.workspace = torch.empty(max(int(pl.workspace_bytes), 256), dtype=torch.uint8,
                                     device=device)
        self.x = torch.empty(pl.total_coords, dtype=torch.float64, device=device)
        self.f = torch.empty(pl.total_starts, dtype=torch.float64, device=device)
        self.gnorm = torch.empty(pl.total_starts, dtype=torch.float64, device=device)
        self.status = torch.empty(pl.total_starts, dtype=torch.int32, device=device)
        self.iters = torch.empty(pl.total_starts, dtype=torch.int32, device=device)
        self.results = torch.empty(pl.n_problems * RESULT_BYTES, dtype=torch.uint8, device=device)
        zeus_batch_prepare(self.problems, pl, self.workspace, stream)
        self.graph = None
        # row offsets of each problem in the concatenated outputs
        self.xoff, self.soff = [], []
        xo = so = 0
        for p in self.problems:
            self.xoff.append(xo)
            self.soff.append(so)
            xo += p.n_starts * p.dim
            so += p.n_starts

    @property
    def launches(self) -> int:
        """Kernels one solve launches (plus one memset)."""
        pl = self.plan
        return (pl.pso_iters_max + 1) + pl.n_classes + (1 if pl.q_cap > 0 else 0) + 1

    def solve(self, stream=None) -> None:
        zeus_batch_solve(self.plan, self.workspace, self.x, self.f, self.gnorm, self.status,
                         self.iters, self.results, stream)

    def capture(self) -> "torch.cuda.CUDAGraph":
        """Record one solve in a CUDA graph (on a side stream, as torch requires)."""
        g = torch.cuda.CUDAGraph()
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            g.capture_begin()
            try:
                self.solve(side)
            finally:
                g.capture_end()
        torch.cuda.current_stream().wait_stream(side)
        self.graph = g
        return g

    def replay(self) -> None:
        if self.graph is None:
            self.capture()
        self.graph.replay()

    def problem(self, P: int) -> dict:
        """Views of problem P's outputs and its decoded summary (synchronizes)."""
        p = self.problems[P]
        xo, so, n, d = self.xoff[P], self.soff[P], p.n_starts, p.dim
        raw = self.results[P * RESULT_BYTES:(P + 1) * RESULT_BYTES]
        return dict(x=self.x[xo:xo + n * d].view(n, d), f=self.f[so:so + n],
                    gnorm=self.gnorm[so:so + n], status=self.status[so:so + n],
                    iters=self.iters[so:so + n], summary=decode_result(raw))

    def cluster(self, method="x", tol: float = 1e-3, max_clusters: int = 64,
                only_converged: bool = True, stream=None) -> dict:
        """Clusters every problem's final points on its own (one launch;
        the definition of ``cluster``): labels [total_starts] in the order
        of ``f``, leaders and counts [n_problems, max_clusters] (leaders are
        start indices within their problem), and one summary per problem."""
        pl, dev = self.plan, self.f.device
        cp = _capi.zeus_cluster_params(_capi.CLUSTER_METHODS[method] if isinstance(method, str)
                                       else int(method), int(max_clusters),
                                       int(bool(only_converged)), 0, float(tol))
        n = pl.n_problems
        lab = torch.empty(pl.total_starts, dtype=torch.int32, device=dev)
        lead = torch.empty(n, max_clusters, dtype=torch.int32, device=dev)
        cnt = torch.empty(n, max_clusters, dtype=torch.int32, device=dev)
        rb = C.sizeof(_capi.zeus_cluster_result)
        res = torch.empty(n * rb, dtype=torch.uint8, device=dev)
        check(lib().zeus_batch_cluster(
            C.byref(pl), _ptr(self.workspace, torch.uint8), self.workspace.numel(), C.byref(cp),
            _ptr(self.x, torch.float64), _ptr(self.f, torch.float64),
            _ptr(self.status, torch.int32), _ptr(lab, torch.int32), _ptr(lead, torch.int32),
            _ptr(cnt, torch.int32), _ptr(res, torch.uint8), _stream(stream)), "zeus_batch_cluster")
        raw = res.cpu().numpy().tobytes()
        sums = []
        for P in range(n):
            r = _capi.zeus_cluster_result.from_buffer_copy(raw[P * rb:(P + 1) * rb])
            sums.append({k: getattr(r, k) for k, _ in _capi.zeus_cluster_result._fields_})
        return {"labels": lab, "leaders": lead, "counts": cnt, "summaries": sums}

    def summaries(self) -> list[dict]:
        raw = self.results.cpu().numpy().tobytes()
        out = []
        for P in range(self.plan.n_problems):
            r = zeus_result.from_buffer_copy(raw[P * RESULT_BYTES:(P + 1) * RESULT_BYTES])
            out.append({name: getattr(r, name) for name, _ in zeus_result._fields_})
        return out


# ------------------------------------------------------------ conveniences

def _alloc_outputs(pc: zeus_problem, device):
    n, d = pc.n_starts, pc.dim
    return dict(x=torch.empty(n, d, dtype=torch.float64, device=device),
                f=torch.empty(n, dtype=torch.float64, device=device),
                gnorm=torch.empty(n, dtype=torch.float64, device=device),
                status=torch.empty(n, dtype=torch.int32, device=device),
                iters=torch.empty(n, dtype=torch.int32, device=device),
                result=new_result(device))


def solve(problem: Problem, device="cuda", stream=None) -> dict:
    """The whole method (Alg. 7) on the device; returns the output tensors
    and the decoded summary (synchronizes)."""
    pc = _prob(problem)
    out = _alloc_outputs(pc, device)
    ws = new_workspace(pc, device)
    zeus_solve(pc, ws, out["x"], out["f"], out["gnorm"], out["status"], out["iters"],
               out["result"], stream)
    out["summary"] = decode_result(out["result"])
    return out


def solve_from(problem: Problem, x0: torch.Tensor, device="cuda", stream=None) -> dict:
    """BFGS from given starts, then the best-of-swarm reduction."""
    pc = _prob(problem)
    out = _alloc_outputs(pc, device)
    ws = new_workspace(pc, device)
    zeus_solve_from(pc, x0.contiguous(), ws, out["x"], out["f"], out["gnorm"], out["status"],
                    out["iters"], out["result"], stream)
    out["summary"] = decode_result(out["result"])
    return out


def pso(problem: Problem, device="cuda", stream=None) -> dict:
    """The PSO phase alone (Alg. 2 then Alg. 3 pso_iters times)."""
    pc = _prob(problem)
    n, d = pc.n_starts, pc.dim
    t = {k: torch.empty(n, d, dtype=torch.float64, device=device) for k in ("x", "v", "px")}
    t["pf"] = torch.empty(n, dtype=torch.float64, device=device)
    t["gx"] = torch.empty(d, dtype=torch.float64, device=device)
    res = new_result(device)
    ws = new_workspace(pc, device)
    zeus_pso(pc, ws, t["x"], t["v"], t["px"], t["pf"], t["gx"], res, stream)
    r = decode_result(res)
    t["gf"], t["gidx"] = r["gbest_f"], r["gbest_index"]
    return t


def objective(obj, x: torch.Tensor, grad: bool = True, grad_mode="forward"):
    """f (and g) at the rows of x ([n, d], float64 or float32, CUDA)."""
    n, d = x.shape
    x = x.contiguous()
    f = torch.empty(n, dtype=x.dtype, device=x.device)
    g = torch.empty_like(x) if grad else None
    fn = zeus_objective_eval if x.dtype == torch.float64 else zeus_objective_eval_f32
    fn(obj, d, x, f, g, grad_mode)
    return (f, g) if grad else f


class ObjectiveFn(torch.autograd.Function):
    """f(x) for the rows of x with the gradient from the hand-written
    reverse-mode adjoint kernel (or forward-mode duals) of libzeus."""

    @staticmethod
    def forward(ctx, x, obj="rosenbrock", grad_mode="adjoint"):
        f, g = objective(obj, x.detach(), grad=True, grad_mode=grad_mode)
        ctx.save_for_backward(g)
        return f

    @staticmethod
    def backward(ctx, grad_out):
        (g,) = ctx.saved_tensors
        return grad_out.unsqueeze(1) * g, None, None


# ------------------------------------------------ solution clustering

def zeus_cluster_workspace_size(max_clusters: int) -> int:
    b = C.c_size_t()
    check(lib().zeus_cluster_workspace_size(int(max_clusters), C.byref(b)),
          "zeus_cluster_workspace_size")
    return b.value


def zeus_cluster(params, n, dim, x, f, status, label_out, leader_out, count_out, result,
                 workspace, stream=None) -> None:
    mc = params.max_clusters
    check(lib().zeus_cluster(
        C.byref(params), n, dim, _ptr(x, torch.float64, n * dim, "x"), _ptr(f, torch.float64, n, "f"),
        _ptr(status, torch.int32, n, "status"), _ptr(label_out, torch.int32, n, "label_out"),
        _ptr(leader_out, torch.int32, mc, "leader_out"), _ptr(count_out, torch.int32, mc, "count_out"),
        _ptr(result, torch.uint8, C.sizeof(_capi.zeus_cluster_result), "result"),
        _ptr(workspace, torch.uint8, None, "workspace"),
        workspace.numel() if workspace is not None else 0, _stream(stream)),
        "zeus_cluster")


def cluster(x: torch.Tensor, f: torch.Tensor, status: torch.Tensor | None = None, method="x",
            tol: float = 1e-3, max_clusters: int = 256, only_converged: bool = False,
            stream=None) -> dict:
    """Clusters final points on the device (leader clustering in order of
    increasing f, by f or by coordinates; include/zeus.h): labels [n],
    leaders and member counts [max_clusters], and the summary (synchronizes)."""
    n = f.numel()
    dim = x.shape[1] if x is not None and x.dim() == 2 else 1
    cp = _capi.zeus_cluster_params(_capi.CLUSTER_METHODS[method] if isinstance(method, str) else int(method),
                                   int(max_clusters), int(bool(only_converged)), 0, float(tol))
    dev = f.device
    out = {"labels": torch.empty(n, dtype=torch.int32, device=dev),
           "leaders": torch.empty(max_clusters, dtype=torch.int32, device=dev),
           "counts": torch.empty(max_clusters, dtype=torch.int32, device=dev),
           "result": torch.empty(C.sizeof(_capi.zeus_cluster_result), dtype=torch.uint8, device=dev)}
    ws = torch.empty(zeus_cluster_workspace_size(max_clusters), dtype=torch.uint8, device=dev)
    zeus_cluster(cp, n, dim, x.contiguous() if x is not None else None, f.contiguous(),
                 status.contiguous() if status is not None else None, out["labels"], out["leaders"],
                 out["counts"], out["result"], ws, stream)
    raw = bytes(out["result"].cpu().numpy().tobytes())
    r = _capi.zeus_cluster_result.from_buffer_copy(raw)
    out["summary"] = {k: getattr(r, k) for k, _ in _capi.zeus_cluster_result._fields_}
    return out


def solve_until_confident(problem: Problem, required: int, tol: float = 1e-3, method="x",
                          max_rounds: int = 10, device="cuda") -> dict:
    """The iterative process Section VI proposes: solve the problem again
    with fresh seeds (seed, seed + 1, ...), cluster the converged points of
    all rounds so far, and stop once the region of the lowest f holds at
    least `required` starts (or after max_rounds).  Returns the clustering
    of the pooled points, the pooled outputs and the number of rounds."""
    xs, fs, ss = [], [], []
    for r in range(max_rounds):
        out = solve(problem.replace(seed=problem.seed + r), device=device)
        xs.append(out["x"])
        fs.append(out["f"])
        ss.append(out["status"])
        x, f, st = torch.cat(xs), torch.cat(fs), torch.cat(ss)
        c = cluster(x, f, st, method=method, tol=tol, max_clusters=1, only_converged=True)
        if c["summary"]["best_count"] >= required:
            break
    c.update(x=x, f=f, status=st, rounds=r + 1)
    return c


def status_names(status: torch.Tensor):
    return [RUN_STATUS.get(int(s), str(int(s))) for s in status.cpu().tolist()]



def precision_error(problem: Problem, x0: torch.Tensor, device="cuda", stream=None) -> dict:
    """The FP32 form's error, start by start: BFGS from the same starts x0
    in the FP32 form with FP64 guards and in the FP64 method (the paper's
    precision), then per start |f32 - f64| (both final values are FP64
    evaluations) and max_j |x32_j - x64_j| / max(1, max_j |x64_j|).  Returns
    the per-start arrays (numpy), both runs' statuses and a summary of the
    error distribution (synchronizes)."""
    p = problem if isinstance(problem, Problem) else None
    if p is None:
        raise TypeError("precision_error takes a Problem")
    r64 = solve_from(p.replace(precision="fp64"), x0, device, stream)
    r32 = solve_from(p.replace(precision="fp32_guarded"), x0, device, stream)
    f64, f32 = r64["f"].double(), r32["f"].double()
    x64, x32 = r64["x"], r32["x"]
    abs_f = (f32 - f64).abs()
    both_inf = torch.isinf(f32) & torch.isinf(f64) & (torch.sign(f32) == torch.sign(f64))
    abs_f = torch.where(both_inf, torch.zeros_like(abs_f), abs_f)
    rel_x = (x32 - x64).abs().amax(dim=1) / torch.clamp(x64.abs().amax(dim=1), min=1.0)
    a = abs_f.cpu().numpy()
    q = torch.quantile(abs_f[torch.isfinite(abs_f)].cpu(), torch.tensor([0.5, 0.9, 1.0],
                                                                       dtype=torch.float64))
    return {"abs_f": a, "rel_x": rel_x.cpu().numpy(),
            "status_fp32": r32["status"].cpu().numpy(), "status_fp64": r64["status"].cpu().numpy(),
            "summary": {"starts": int(a.size), "median": float(q[0]), "p90": float(q[1]),
                        "max": float(q[2]), "within_1e-6": float((a <= 1e-6).mean()),
                        "iters_fp32": int(r32["iters"].sum().item()),
                        "iters_fp64": int(r64["iters"].sum().item())}}
