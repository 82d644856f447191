"""The C-ABI library (include/zeus.h) builds, loads without a GPU, exports
every declared symbol, and its host-side logic (defaults, validation,
workspace sizing, error strings) behaves as documented.  No device work."""
import ctypes as C
import math
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "zeus.h")


@pytest.fixture(scope="module")
def z():
    import paper_2603_28770_gb300 as z
    z.lib()
    return z


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(zeus_[a-z0-9_]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(z):
    names = _declared()
    assert "zeus_solve" in names and len(names) >= 15
    L = C.CDLL(z.library_path())
    for n in names:
        assert hasattr(L, n), n
    # and the Python binding declares exactly the header's entry points
    from paper_2603_28770_gb300 import _capi
    assert sorted(_capi.SIGNATURES) == names


def test_struct_layouts_match_header(z, tmp_path):
    # compile the header with the host C compiler and compare every field
    # offset and the struct sizes with the ctypes declarations
    from paper_2603_28770_gb300 import _capi
    import subprocess
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "zeus.h"', 'int main(void){']
    structs = (("zeus_problem", _capi.zeus_problem), ("zeus_result", _capi.zeus_result),
               ("zeus_plan", _capi.zeus_plan), ("zeus_batch_plan", _capi.zeus_batch_plan),
               ("zeus_cluster_params", _capi.zeus_cluster_params),
               ("zeus_cluster_result", _capi.zeus_cluster_result))
    for cname, cls in structs:
        lines.append(f'printf("{cname} %zu\\n", sizeof({cname}));')
        for f, _ in cls._fields_:
            lines.append(f'printf("{cname}.{f} %zu\\n", offsetof({cname}, {f}));')
    lines.append("return 0;}")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = dict(l.split() for l in subprocess.run([str(exe)], capture_output=True, text=True,
                                                  check=True).stdout.splitlines())
    for cname, cls in structs:
        assert int(out[cname]) == C.sizeof(cls)
        for f, _ in cls._fields_:
            assert int(out[f"{cname}.{f}"]) == getattr(cls, f).offset, f


def test_defaults(z):
    p = z.zeus_default_problem()
    assert (p.objective, p.dim, p.n_starts, p.pso_iters, p.bfgs_max_iters, p.ls_max_iters) == (0, 2, 128, 5, 100, 20)
    assert (p.w, p.c1, p.c2, p.armijo_c, p.backtrack, p.grad_tol) == (0.7, 1.5, 1.5, 1e-4, 0.5, 1e-8)
    assert math.isnan(p.target_f) and p.precision == 0 and p.grad_mode == 0
    assert z.zeus_validate(p) == 0
    assert z.zeus_validate(z.Problem()) == 0


@pytest.mark.parametrize("kw", [
    dict(dim=1), dict(objective="goldstein_price", dim=3), dict(objective=7), dict(dim=0), dict(dim=5000),
    dict(lower=1.0, upper=1.0), dict(lower=float("nan")), dict(upper=float("inf")), dict(n_starts=0),
    dict(n_starts=2**31), dict(pso_iters=-1), dict(bfgs_max_iters=-1), dict(ls_max_iters=0),
    dict(required_converged=-2), dict(grad_tol=-1.0), dict(grad_tol=float("nan")), dict(w=float("inf")),
    dict(armijo_c=0.0), dict(armijo_c=1.0), dict(backtrack=1.0), dict(backtrack=0.0), dict(grad_mode=2),
    dict(start_from_pbest=2), dict(threads_per_start=3), dict(threads_per_start=64), dict(threads_per_start=512), dict(precision=5),
    dict(lbfgs_m=-1), dict(lbfgs_m=65),
])
def test_validation_rejects(z, kw):
    assert z.zeus_validate(z.Problem(**kw)) == z._capi.ZEUS_EINVAL


@pytest.mark.parametrize("kw", [
    dict(objective="rastrigin", dim=1), dict(objective="quadratic", dim=1), dict(objective="ackley", dim=4096),
    dict(n_starts=1), dict(pso_iters=0), dict(bfgs_max_iters=0), dict(grad_mode="adjoint"),
    dict(threads_per_start=128), dict(threads_per_start=1), dict(start_from_pbest=1), dict(precision="fp32_guarded"), dict(required_converged=3), dict(target_f=1e-6),
    dict(lbfgs_m=1), dict(lbfgs_m=64, dim=1000),
])
def test_validation_accepts(z, kw):
    assert z.zeus_validate(z.Problem(**kw)) == 0


def test_workspace_sizes(z):
    small = z.zeus_workspace_size(z.Problem())
    assert small % 256 == 0 and small >= 256 + 128 * 8 * 5
    big = z.zeus_workspace_size(z.Problem(objective="rastrigin", dim=10, n_starts=16384))
    assert big > small and big >= 16384 * 10 * 8 * 2
    assert z.zeus_argmin_workspace_size(1) >= 256
    with pytest.raises(z.ZeusError):
        z.zeus_workspace_size(z.Problem(dim=0))


def test_null_and_workspace_errors_before_any_launch(z):
    L = z.lib()
    p = z.Problem().to_c()
    # NULL problem, NULL x_out, missing workspace: rejected on the host
    assert L.zeus_solve(None, None, 0, None, None, None, None, None, None, None) == z._capi.ZEUS_EINVAL
    assert L.zeus_solve(C.byref(p), None, 0, None, None, None, None, None, None, None) == z._capi.ZEUS_EINVAL
    assert L.zeus_solve(C.byref(p), None, 0, C.c_void_p(256), None, None, None, None, None, None) == z._capi.ZEUS_EWORKSPACE
    # misaligned workspace
    assert L.zeus_solve(C.byref(p), C.c_void_p(4096 + 8), 1 << 20, C.c_void_p(256), None, None, None,
                        None, None, None) == z._capi.ZEUS_EWORKSPACE
    assert L.zeus_argmin(None, 10, None, 0, None, None) == z._capi.ZEUS_EINVAL
    assert L.zeus_uniform(0, 0, 0, -1, 2, None, None) == z._capi.ZEUS_EINVAL
    assert L.zeus_context_destroy(None) == z._capi.ZEUS_EINVAL


def test_strerror(z):
    for code in (0, -1, -2, -3, -4, -5, -6):
        assert z.zeus_strerror(code) and "unknown" not in z.zeus_strerror(code)
    assert "unknown" in z.zeus_strerror(-99)


def test_plan_choice(z):
    small = z.zeus_plan_info(z.Problem(objective="rastrigin", dim=10, n_starts=16384))
    assert small["narrow"] == 1 and small["handover"] == 1 and small["stream"] == 0
    mid = z.zeus_plan_info(z.Problem(objective="rastrigin", dim=100, n_starts=100))
    assert mid["block"] == 1 and mid["narrow"] == 0 and mid["stream"] == 0
    big = z.zeus_plan_info(z.Problem(objective="rosenbrock", dim=256, n_starts=8192,
                                     precision="fp32_guarded"))
    # streamed FP32 H: the tiles of the upper triangle (16 x 32 at d = 256)
    tiles = sum(8 - (16 * I) // 32 for I in range(16))
    assert big["stream"] == 1 and big["h_bytes"] == tiles * 16 * 32 * 4 < 0.57 * 256 * 256 * 4
    assert z.zeus_plan_info(z.Problem(objective="rosenbrock", dim=256, n_starts=8))["h_bytes"] == \
        256 * 256 * 8  # FP64 H streams whole
    forced = z.zeus_plan_info(z.Problem(objective="rastrigin", dim=10, threads_per_start=256))
    assert forced["stream"] == 1 and forced["narrow"] == 0
    # the stream slots are part of the workspace
    assert z.zeus_workspace_size(z.Problem(objective="rosenbrock", dim=256, n_starts=8192,
                                           precision="fp32_guarded")) >= 300 * tiles * 16 * 32 * 4


def _tiles_fp32(d):
    # the tiled triangle of streamed FP32 H: d padded to 32, tiles of th
    # rows x 32 columns, th = dp / 16 rounded down to a power of two within
    # [4, 32], tile (I, J) stored when J >= I th / 32
    dp = (d + 31) // 32 * 32
    th = min(32, dp // 16)
    p2 = 1
    while p2 * 2 <= th:
        p2 *= 2
    th = max(p2, 4)
    tiles = sum(dp // 32 - (I * th) // 32 for I in range(dp // th))
    return tiles * th * 32, dp


@pytest.mark.parametrize("d", [2, 10, 33, 64, 100, 200, 256, 300, 1024])
def test_streamed_fp32_slot_is_the_tiled_triangle(z, d):
    p = z.Problem(objective="rosenbrock", dim=d, n_starts=16, precision="fp32_guarded",
                  threads_per_start=256)
    info = z.zeus_plan_info(p)
    elems, dp = _tiles_fp32(d)
    assert info["stream"] == 1 and info["h_bytes"] == elems * 4
    # every element r <= c < d is in some stored tile, and the slot holds at
    # most the padded matrix
    assert d * (d + 1) // 2 <= elems <= dp * dp
    # the workspace holds one slot per block
    assert z.zeus_workspace_size(p) >= info["blocks"] * elems * 4
    # FP64 H streams whole
    info64 = z.zeus_plan_info(p.replace(precision="fp64"))
    assert info64["h_bytes"] == d * d * 8


def test_streamed_fp32_whole_matrix_past_the_tiles(z):
    # past d ~ 3200 the tiled pass's shared memory would not fit a block:
    # FP32 H streams as the full matrix there (up to the largest d)
    p = z.Problem(objective="rosenbrock", dim=4000, n_starts=4, precision="fp32_guarded")
    info = z.zeus_plan_info(p)
    assert info["stream"] == 1 and info["h_bytes"] == 4000 * 4000 * 4


# ---------------------------------------------------------------- batched form

def _mixed(z, n=12, **kw):
    from paper_2603_28770_gb300.workloads import mixed_batch
    return [z.Problem(**m, n_starts=64 + 7 * i, pso_iters=i % 4, bfgs_max_iters=50, seed=i, **kw)
            for i, m in enumerate(mixed_batch(n, seed=7, dmin=2, dmax=64))]


def test_batch_plan(z):
    probs = _mixed(z)
    pl = z.zeus_batch_plan_make(probs)
    assert pl.n_problems == len(probs)
    assert pl.total_starts == sum(p.n_starts for p in probs)
    assert pl.total_coords == sum(p.n_starts * p.dim for p in probs)
    assert pl.total_g == sum(p.dim for p in probs)
    assert pl.pso_iters_max == max(p.pso_iters for p in probs)
    assert pl.workspace_bytes % 256 == 0
    # the classes tile the work list in order, each with some shared memory
    nxt = 0
    for c in range(pl.n_classes):
        assert pl.class_first[c] == nxt and pl.class_count[c] > 0
        assert 0 < pl.class_smem[c] <= 227 * 1024
        nxt += pl.class_count[c]
    assert nxt == pl.items
    # block-per-start classes first, then the lane-tile classes (which run
    # on the library's second stream with the hand-over launch)
    kinds = [pl.class_kind[c] for c in range(pl.n_classes)]
    assert set(kinds) <= {0, 1, 2} and kinds == sorted(kinds, reverse=True)
    # work items: one per block-per-start start, one per lane tile of <= 128 starts
    lane = [p for p in probs if z.zeus_plan_info(p)["narrow"]]
    block = [p for p in probs if not z.zeus_plan_info(p)["narrow"]]
    assert pl.items >= sum(p.n_starts for p in block) + sum(-(-p.n_starts // 128) for p in lane)
    # hand-over queue only when some lane problem hands over
    assert (pl.q_cap > 0) == any(z.zeus_plan_info(p)["handover"] for p in probs)
    # planning is deterministic
    assert bytes(z.zeus_batch_plan_make(probs)) == bytes(pl)


def test_batch_plan_with_lbfgs(z):
    # L-BFGS problems (also at a d whose dense H would stream) join a batch
    # as one 256-thread-block item per start, in classes of kind 3 that come
    # first
    probs = _mixed(z, 6)
    lb = [z.Problem(objective="rosenbrock", dim=300, n_starts=5, lbfgs_m=4, seed=1),
          z.Problem(objective="ackley", dim=20, n_starts=9, lbfgs_m=7, seed=2)]
    pl = z.zeus_batch_plan_make(probs + lb)
    kinds = [pl.class_kind[c] for c in range(pl.n_classes)]
    assert kinds[0] == 3 and set(kinds) <= {0, 1, 2, 3} and kinds == sorted(kinds, reverse=True)
    n3 = sum(pl.class_count[c] for c in range(pl.n_classes) if pl.class_kind[c] == 3)
    assert n3 == sum(p.n_starts for p in lb)
    assert all(pl.class_smem[c] > 0 for c in range(pl.n_classes) if pl.class_kind[c] == 3)
    assert pl.total_starts == sum(p.n_starts for p in probs + lb)


def test_batch_rejects(z):
    L = z.lib()
    EINVAL, EUNS, EWS = z._capi.ZEUS_EINVAL, z._capi.ZEUS_EUNSUPPORTED, z._capi.ZEUS_EWORKSPACE
    probs = _mixed(z, 4)
    arr = (z._capi.zeus_problem * 4)(*[p.to_c() for p in probs])
    pl = z._capi.zeus_batch_plan()
    assert L.zeus_batch_plan_make(arr, 0, C.byref(pl)) == EINVAL
    assert L.zeus_batch_plan_make(None, 4, C.byref(pl)) == EINVAL
    assert L.zeus_batch_plan_make(arr, 4, None) == EINVAL
    # all problems share precision and gradient mode
    mixed = probs[:3] + [probs[3].replace(precision="fp32_guarded")]
    with pytest.raises(z.ZeusError) as e:
        z.zeus_batch_plan_make(mixed)
    assert e.value.code == EINVAL
    mixed = probs[:3] + [probs[3].replace(grad_mode="adjoint")]
    with pytest.raises(z.ZeusError):
        z.zeus_batch_plan_make(mixed)
    # an invalid member problem
    with pytest.raises(z.ZeusError):
        z.zeus_batch_plan_make(probs[:3] + [probs[3].replace(dim=0)])
    # dense H streamed from HBM is not batched, nor L-BFGS on Goldstein-Price
    with pytest.raises(z.ZeusError) as e:
        z.zeus_batch_plan_make(probs[:3] + [z.Problem(objective="rosenbrock", dim=256, n_starts=8)])
    assert e.value.code == EUNS
    with pytest.raises(z.ZeusError) as e:
        z.zeus_batch_plan_make(probs[:3] + [z.Problem(objective="goldstein_price", dim=2,
                                                      n_starts=8, lbfgs_m=3)])
    assert e.value.code == EUNS
    assert L.zeus_batch_plan_make(arr, 4, C.byref(pl)) == 0
    # prepare: missing or small workspace, and a plan of another batch, fail on the host
    assert L.zeus_batch_prepare(arr, 4, C.byref(pl), None, 0, None) == EWS
    assert L.zeus_batch_prepare(arr, 4, C.byref(pl), C.c_void_p(4096), pl.workspace_bytes - 256,
                                None) == EWS
    assert L.zeus_batch_prepare(arr, 4, C.byref(pl), C.c_void_p(4096 + 16), pl.workspace_bytes,
                                None) == EWS
    other = z.zeus_batch_plan_make(probs[:3])
    assert L.zeus_batch_prepare(arr, 4, C.byref(other), C.c_void_p(4096), 1 << 40, None) == EINVAL
    # solve: a damaged plan, a missing output or workspace
    bad = z._capi.zeus_batch_plan.from_buffer_copy(bytes(pl))
    bad.class_count[0] += 1
    assert L.zeus_batch_solve(C.byref(bad), C.c_void_p(4096), 1 << 40, C.c_void_p(256),
                              C.c_void_p(256), None, None, None, None, None) == EINVAL
    assert L.zeus_batch_solve(C.byref(pl), C.c_void_p(4096), 1 << 40, None, C.c_void_p(256), None,
                              None, None, None, None) == EINVAL
    assert L.zeus_batch_solve(C.byref(pl), None, 0, C.c_void_p(256), C.c_void_p(256), None, None,
                              None, None, None) == EWS


def test_lbfgs_plan(z):
    p = z.Problem(objective="rosenbrock", dim=1024, n_starts=2048, lbfgs_m=8, precision="fp32_guarded")
    pl = z.zeus_plan_info(p)
    assert pl["lbfgs"] == 1 and pl["stream"] == 0 and pl["narrow"] == 0 and pl["h_bytes"] == 0
    dense = z.zeus_plan_info(p.replace(lbfgs_m=0))
    assert dense["stream"] == 1 and dense["lbfgs"] == 0
    # no H slots: the workspace is far smaller than the dense streamed one
    assert z.zeus_workspace_size(p) * 25 < z.zeus_workspace_size(p.replace(lbfgs_m=0))
    for bad in (dict(objective="goldstein_price", dim=2), dict(threads_per_start=128),
                dict(threads_per_start=1), dict(dim=4096, precision="fp64", lbfgs_m=64)):
        with pytest.raises(z.ZeusError) as e:
            z.zeus_plan_info(p.replace(**bad))
        assert e.value.code == z._capi.ZEUS_EUNSUPPORTED
    assert z.zeus_plan_info(p.replace(threads_per_start=256))["lbfgs"] == 1
    # batched beside a dense problem: one item per start, a class of kind 3
    pl = z.zeus_batch_plan_make([z.Problem(), p.replace(precision="fp64", dim=20, n_starts=8)])
    assert pl.class_kind[0] == 3 and pl.class_count[0] == 8


def test_user_objectives_of_the_default_plugin(z):
    L = z.lib()
    assert L.zeus_user_objective_count() == 2
    assert z.user_objectives() == {"griewank": (200, 1, 0), "himmelblau": (201, 2, 2)}
    buf = C.create_string_buffer(4)  # truncated to fit, NUL-terminated
    lo, hi = C.c_int32(), C.c_int32()
    assert L.zeus_user_objective_info(0, buf, 4, C.byref(lo), C.byref(hi)) == 0
    assert buf.value == b"gri" and (lo.value, hi.value) == (1, 0)
    assert L.zeus_user_objective_info(1, None, 0, None, None) == 0
    for k in (-1, 2, 4, 200):
        assert L.zeus_user_objective_info(k, buf, 4, None, None) == z._capi.ZEUS_EINVAL
    assert z.Problem(objective="himmelblau").to_c().objective == 201
    with pytest.raises(KeyError):
        z.Problem(objective="no_such_function").to_c()


def test_user_objective_validation_and_plans(z):
    EINVAL, EUNS = z._capi.ZEUS_EINVAL, z._capi.ZEUS_EUNSUPPORTED
    g = z.Problem(objective="griewank", dim=8, n_starts=64)
    assert z.zeus_validate(g) == 0 and z.zeus_validate(g.replace(dim=1)) == 0
    assert z.zeus_validate(g.replace(objective="himmelblau", dim=2)) == 0
    # the plug-in's dimension range; ids past the plug-in's objectives
    assert z.zeus_validate(g.replace(objective="himmelblau", dim=3)) == EINVAL
    assert z.zeus_validate(g.replace(objective=202)) == EINVAL
    assert z.zeus_validate(g.replace(objective=199)) == EINVAL
    # forward mode only
    assert z.zeus_validate(g.replace(grad_mode="adjoint")) == EUNS
    # lane, block and hand-over forms as for a built-in objective
    assert z.zeus_plan_info(g)["narrow"] == 1 and z.zeus_plan_info(g)["handover"] == 1
    assert z.zeus_plan_info(g.replace(dim=64))["block"] == 1
    # no form that streams H, and no L-BFGS
    for bad in (dict(dim=512), dict(threads_per_start=256), dict(lbfgs_m=4)):
        with pytest.raises(z.ZeusError) as e:
            z.zeus_plan_info(g.replace(**bad))
        assert e.value.code == EUNS


def test_user_objectives_in_a_batch_plan(z):
    probs = _mixed(z, 4) + [z.Problem(objective="griewank", dim=6, n_starts=100),
                            z.Problem(objective="himmelblau", dim=2, n_starts=300, seed=3)]
    pl = z.zeus_batch_plan_make(probs)
    assert pl.n_user == 2 and pl.pad == 0
    assert z.zeus_batch_plan_make(probs[:4]).n_user == 0
    with pytest.raises(z.ZeusError) as e:
        z.zeus_batch_plan_make([p.replace(grad_mode="adjoint") for p in probs])
    assert e.value.code == z._capi.ZEUS_EUNSUPPORTED
    # a plan whose user count was altered is refused before any launch
    L = z.lib()
    bad = z._capi.zeus_batch_plan.from_buffer_copy(bytes(pl))
    bad.n_user = len(probs) + 1
    assert L.zeus_batch_solve(C.byref(bad), C.c_void_p(4096), 1 << 40, C.c_void_p(256),
                              C.c_void_p(256), None, None, None, None, None) == z._capi.ZEUS_EINVAL


def test_cluster_argument_errors(z):
    L = z.lib()
    EINVAL = z._capi.ZEUS_EINVAL
    P = z._capi.zeus_cluster_params
    ok = dict(method=1, max_clusters=8, only_converged=1, pad=0, tol=0.1)
    fake = C.c_void_p(4096)

    def call(n=10, dim=2, x=fake, f=fake, st=fake, lab=fake, ws=fake, wsb=1 << 30, **kw):
        cp = P(**dict(ok, **kw))
        return L.zeus_cluster(C.byref(cp), n, dim, x, f, st, lab, None, None, None, ws, wsb, None)

    for bad in (dict(method=2), dict(method=-1), dict(max_clusters=0), dict(max_clusters=4097),
                dict(only_converged=2), dict(pad=1), dict(tol=-1.0), dict(tol=float("nan")),
                dict(tol=float("inf")), dict(n=-1), dict(n=1 << 31), dict(dim=0), dict(f=None),
                dict(lab=None), dict(x=None), dict(st=None)):
        assert call(**bad) == EINVAL, bad
    assert L.zeus_cluster(None, 10, 2, fake, fake, fake, fake, None, None, None, fake, 1 << 30,
                          None) == EINVAL
    # the workspace: present, large enough for max_clusters, 256-byte aligned
    need = z.zeus_cluster_workspace_size(8)
    assert need % 256 == 0 and z.zeus_cluster_workspace_size(4096) > need
    EWS = z._capi.ZEUS_EWORKSPACE
    assert call(ws=None) == EWS and call(wsb=need - 1) == EWS
    assert call(ws=C.c_void_p(4096 + 128), wsb=need) == EWS
    with pytest.raises(z.ZeusError):
        z.zeus_cluster_workspace_size(0)
    assert C.sizeof(z._capi.zeus_cluster_result) == 64 and C.sizeof(P) == 24


def test_batch_cluster_argument_errors(z):
    L = z.lib()
    EINVAL, EWS = z._capi.ZEUS_EINVAL, z._capi.ZEUS_EWORKSPACE
    pl = z.zeus_batch_plan_make(_mixed(z, 4))
    P = z._capi.zeus_cluster_params
    fake = C.c_void_p(4096)

    def call(cp=P(1, 8, 1, 0, 0.1), plan=pl, ws=fake, wsb=1 << 40, x=fake, f=fake, st=fake,
             lab=fake):
        return L.zeus_batch_cluster(C.byref(plan) if plan is not None else None, ws, wsb,
                                    C.byref(cp) if cp is not None else None, x, f, st, lab,
                                    None, None, None, None)

    for bad in (dict(cp=None), dict(plan=None), dict(cp=P(2, 8, 1, 0, 0.1)),
                dict(cp=P(1, 0, 1, 0, 0.1)), dict(cp=P(1, 8, 1, 0, -1.0)), dict(f=None),
                dict(lab=None), dict(x=None), dict(st=None)):
        assert call(**bad) == EINVAL, bad
    bad_plan = z._capi.zeus_batch_plan.from_buffer_copy(bytes(pl))
    bad_plan.n_classes = 0
    assert call(plan=bad_plan) == EINVAL
    assert call(ws=None) == EWS and call(wsb=pl.workspace_bytes - 256) == EWS
