// zeus_capi.cu -- the extern "C" entry points declared in include/zeus.h:
// argument validation, workspace carve-up and kernel dispatch.  Every path
// of the method runs in the kernels of the sibling translation units; this
// file does no arithmetic of the method.
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include <atomic>

#include "zeus.h"
#include "zeus_internal.h"

using namespace zeus;

namespace zeus {
namespace {
std::atomic<unsigned> g_wait_polls{kDefaultWaitPolls};
}
unsigned wait_limit() { return g_wait_polls.load(std::memory_order_relaxed); }
}  // namespace zeus

namespace {

inline cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

bool valid_lanes(int g) { return g == 0 || g == 1 || g == 32 || g == kWideThreads || g == 256; }

int validate(const zeus_problem* p) {
    if (!p) return ZEUS_EINVAL;
    switch (p->objective) {
        case ZEUS_OBJ_ROSENBROCK:
            if (p->dim < 2) return ZEUS_EINVAL;
            break;
        case ZEUS_OBJ_GOLDSTEIN_PRICE:
            if (p->dim != 2) return ZEUS_EINVAL;
            break;
        case ZEUS_OBJ_RASTRIGIN:
        case ZEUS_OBJ_ACKLEY:
        case ZEUS_OBJ_QUADRATIC:
            break;
        default: {  // a user objective of the plug-in, within its dimension range
            const char* name;
            int lo, hi;
            if (p->objective < ZEUS_OBJ_USER ||
                !user_objective_meta(p->objective - ZEUS_OBJ_USER, &name, &lo, &hi))
                return ZEUS_EINVAL;
            if (p->dim < lo || (hi > 0 && p->dim > hi)) return ZEUS_EINVAL;
        }
    }
    if (p->dim < 1 || p->dim > 4096) return ZEUS_EINVAL;
    if (!isfinite(p->lower) || !isfinite(p->upper) || !(p->lower < p->upper)) return ZEUS_EINVAL;
    if (!isfinite(p->upper - p->lower)) return ZEUS_EINVAL;
    if (p->n_starts < 1 || p->n_starts > 0x7fffffffll) return ZEUS_EINVAL;
    if (p->pso_iters < 0 || p->pso_iters > (1 << 24)) return ZEUS_EINVAL;
    if (p->bfgs_max_iters < 0) return ZEUS_EINVAL;
    if (p->ls_max_iters < 1 || p->ls_max_iters > 4096) return ZEUS_EINVAL;
    if (p->required_converged < 0) return ZEUS_EINVAL;
    if (!(p->grad_tol >= 0.0) || !isfinite(p->grad_tol)) return ZEUS_EINVAL;
    if (!isfinite(p->w) || !isfinite(p->c1) || !isfinite(p->c2)) return ZEUS_EINVAL;
    if (!(p->armijo_c > 0.0 && p->armijo_c < 1.0)) return ZEUS_EINVAL;
    if (!(p->backtrack > 0.0 && p->backtrack < 1.0)) return ZEUS_EINVAL;
    if (p->grad_mode != ZEUS_GRAD_FORWARD && p->grad_mode != ZEUS_GRAD_ADJOINT) return ZEUS_EINVAL;
    if (p->start_from_pbest != 0 && p->start_from_pbest != 1) return ZEUS_EINVAL;
    if (!valid_lanes(p->threads_per_start)) return ZEUS_EINVAL;
    if (p->lbfgs_m < 0 || p->lbfgs_m > 64 || p->pad != 0) return ZEUS_EINVAL;
    if (p->precision != ZEUS_FP64 && p->precision != ZEUS_FP32_GUARDED) return ZEUS_EINVAL;
    // a user objective has no hand-written reverse sweep
    if (p->objective >= ZEUS_OBJ_USER && p->grad_mode == ZEUS_GRAD_ADJOINT)
        return ZEUS_EUNSUPPORTED;
    return ZEUS_OK;
}

Layout layout_for(const zeus_problem& p, const BfgsLaunch& L) {
    const size_t n = (size_t)p.n_starts, d = (size_t)p.dim;
    size_t nparts = (size_t)pso_blocks(p, lanes_for_dim(p.dim));
    const size_t na = (size_t)argmin_blocks(p.n_starts);
    if (na > nparts) nparts = na;
    const size_t qc = (size_t)L.q_cap;
    Layout lay;
    size_t off = 0;
    lay.ctrl = off;
    off += align256(sizeof(Ctrl));
    lay.q_ready = off;  // zeroed with the control block, as is the per-SM table
    off += align256(qc * sizeof(int));
    lay.q_smlong = off;
    off += align256(kMaxSMs * sizeof(int));
    lay.partials = off;
    off += align256(nparts * sizeof(ArgPair));
    lay.f_tmp = off;
    off += align256(n * sizeof(double));
    lay.v = off;
    off += align256(n * d * sizeof(double));
    lay.px = off;
    off += align256(n * d * sizeof(double));
    lay.pf = off;
    off += align256(n * sizeof(double));
    lay.gx = off;
    off += align256(d * sizeof(double));
    lay.q_start = off;
    off += align256(qc * sizeof(int));
    lay.q_k = off;
    off += align256(qc * sizeof(int));
    lay.q_feval = off;
    off += align256(qc * sizeof(int));
    lay.q_h = off;
    off += align256(qc * d * d * sizeof(double));
    lay.hslots = off;
    off += align256(L.hslot_bytes);
    lay.total = off;
    return lay;
}

int check_ws(void* ws, size_t have, size_t need) {
    if (need > have) return ZEUS_EWORKSPACE;
    if (!ws) return ZEUS_EWORKSPACE;
    if (((uintptr_t)ws & 255u) != 0) return ZEUS_EWORKSPACE;
    return ZEUS_OK;
}

template <class T>
T* at(void* ws, size_t off) {
    return reinterpret_cast<T*>(reinterpret_cast<char*>(ws) + off);
}

int cuda_status(cudaError_t e) { return e == cudaSuccess ? ZEUS_OK : ZEUS_ECUDA; }

Queue queue_for(void* ws, const Layout& lay, const BfgsLaunch& L) {
    Queue q;
    q.prob = nullptr;
    q.start = reinterpret_cast<int*>(reinterpret_cast<char*>(ws) + lay.q_start);
    q.k = reinterpret_cast<int*>(reinterpret_cast<char*>(ws) + lay.q_k);
    q.feval = reinterpret_cast<int*>(reinterpret_cast<char*>(ws) + lay.q_feval);
    q.H = reinterpret_cast<double*>(reinterpret_cast<char*>(ws) + lay.q_h);
    q.cap = L.q_cap;
    q.hslots = reinterpret_cast<char*>(ws) + lay.hslots;
    q.ready = reinterpret_cast<int*>(reinterpret_cast<char*>(ws) + lay.q_ready);
    q.sm_long = reinterpret_cast<int*>(reinterpret_cast<char*>(ws) + lay.q_smlong);
    return q;
}

// Best-of-swarm reduction over the final f, with the run's counters.
int finish_with_argmin(const zeus_problem& p, void* ws, const Layout& lay, const double* f,
                       zeus_result* res, bool had_pso, cudaStream_t st) {
    Ctrl* ctrl = at<Ctrl>(ws, lay.ctrl);
    ArgPair* parts = at<ArgPair>(ws, lay.partials);
    return cuda_status(launch_argmin(f, p.n_starts, ctrl, parts, res, had_pso ? 1 : 2, st));
}

}  // namespace

extern "C" {

const char* zeus_strerror(int code) {
    switch (code) {
        case ZEUS_OK:
            return "ok";
        case ZEUS_EINVAL:
            return "invalid argument";
        case ZEUS_ENOMEM:
            return "out of device memory";
        case ZEUS_ECUDA:
            return "CUDA error";
        case ZEUS_ETIMEOUT:
            return "bounded device wait expired";
        case ZEUS_EUNSUPPORTED:
            return "unsupported option combination";
        case ZEUS_EWORKSPACE:
            return "workspace missing, too small or not 256-byte aligned";
        default:
            return "unknown zeus status";
    }
}

int zeus_abi_version(void) { return ZEUS_ABI_VERSION; }

int zeus_set_wait_limit(uint32_t polls) {
    g_wait_polls.store(polls ? (unsigned)polls : kDefaultWaitPolls, std::memory_order_relaxed);
    return ZEUS_OK;
}

int zeus_default_problem(zeus_problem* p) {
    if (!p) return ZEUS_EINVAL;
    memset(p, 0, sizeof(*p));
    p->objective = ZEUS_OBJ_ROSENBROCK;
    p->dim = 2;
    p->lower = -5.0;
    p->upper = 5.0;
    p->n_starts = 128;
    p->pso_iters = 5;
    p->bfgs_max_iters = 100;
    p->ls_max_iters = 20;
    p->required_converged = 0;
    p->grad_tol = 1e-8;
    p->w = 0.7;
    p->c1 = 1.5;
    p->c2 = 1.5;
    p->armijo_c = 1e-4;
    p->backtrack = 0.5;
    p->target_f = NAN;
    p->seed = 0;
    p->precision = ZEUS_FP64;
    p->grad_mode = ZEUS_GRAD_FORWARD;
    p->start_from_pbest = 0;
    p->threads_per_start = 0;
    p->lbfgs_m = 0;
    p->pad = 0;
    return ZEUS_OK;
}

int zeus_validate(const zeus_problem* p) { return validate(p); }

int zeus_plan_info(const zeus_problem* p, zeus_plan* plan) {
    if (!plan) return ZEUS_EINVAL;
    const int v = validate(p);
    if (v != ZEUS_OK) return v;
    BfgsLaunch L;
    const int r = plan_bfgs(*p, &L);
    if (r != ZEUS_OK) return r;
    memset(plan, 0, sizeof(*plan));
    plan->narrow = L.narrow ? 1 : 0;
    plan->handover = L.budget > 0 ? 1 : 0;
    plan->lbfgs = L.lbfgs ? 1 : 0;
    plan->stream = (L.stream && !L.lbfgs) ? 1 : 0;
    plan->block = (!L.narrow && !L.stream && !L.warp) ? 1 : 0;
    plan->warp = L.warp ? 1 : 0;
    plan->blocks = L.stream ? L.stream_blocks : L.wide_blocks;
    // H per start: d^2 elements, except streamed FP32 H, held as the tiles
    // of its upper triangle (what one pass moves each way)
    const bool f32 = p->precision == ZEUS_FP32_GUARDED;
    plan->h_bytes = L.lbfgs    ? 0
                    : L.stream ? stream_slot_elems(p->dim, f32 ? 4 : 8) * (f32 ? 4 : 8)
                               : (int64_t)p->dim * p->dim * (f32 ? 4 : 8);
    return ZEUS_OK;
}

int zeus_workspace_size(const zeus_problem* p, size_t* bytes) {
    if (!bytes) return ZEUS_EINVAL;
    const int v = validate(p);
    if (v != ZEUS_OK) return v;
    BfgsLaunch L;
    const int r = plan_bfgs(*p, &L);
    if (r != ZEUS_OK) return r;
    *bytes = layout_for(*p, L).total;
    return ZEUS_OK;
}

int zeus_solve(const zeus_problem* p, void* workspace, size_t workspace_bytes, double* x_out,
               double* f_out, double* gnorm_out, int32_t* status_out, int32_t* iters_out,
               zeus_result* result, void* stream) {
    int v = validate(p);
    if (v != ZEUS_OK) return v;
    if (!x_out) return ZEUS_EINVAL;
    BfgsLaunch L;
    v = plan_bfgs(*p, &L);
    if (v != ZEUS_OK) return v;
    const Layout lay = layout_for(*p, L);
    v = check_ws(workspace, workspace_bytes, lay.total);
    if (v != ZEUS_OK) return v;
    cudaStream_t st = as_stream(stream);
    Ctrl* ctrl = at<Ctrl>(workspace, lay.ctrl);
    ArgPair* parts = at<ArgPair>(workspace, lay.partials);
    double* vv = at<double>(workspace, lay.v);
    double* px = at<double>(workspace, lay.px);
    double* pf = at<double>(workspace, lay.pf);
    double* gx = at<double>(workspace, lay.gx);
    double* f = f_out ? f_out : at<double>(workspace, lay.f_tmp);
    // the control block and the hand-over queue's ready flags start at zero
    cudaError_t e = cudaMemsetAsync(ctrl, 0, lay.partials - lay.ctrl, st);
    if (e != cudaSuccess) return ZEUS_ECUDA;
    e = launch_pso(*p, lanes_for_dim(p->dim), x_out, vv, px, pf, gx, ctrl, parts, result, st);
    if (e != cudaSuccess) return ZEUS_ECUDA;
    const double* x0 = p->start_from_pbest ? px : x_out;
    e = launch_bfgs(*p, L, x0, x_out, f, gnorm_out, status_out, iters_out, ctrl,
                    queue_for(workspace, lay, L), st);
    if (e != cudaSuccess) return ZEUS_ECUDA;
    return finish_with_argmin(*p, workspace, lay, f, result, true, st);
}

int zeus_solve_from(const zeus_problem* p, const double* x0, void* workspace,
                    size_t workspace_bytes, double* x_out, double* f_out, double* gnorm_out,
                    int32_t* status_out, int32_t* iters_out, zeus_result* result, void* stream) {
    int v = validate(p);
    if (v != ZEUS_OK) return v;
    if (!x0 || !x_out) return ZEUS_EINVAL;
    BfgsLaunch L;
    v = plan_bfgs(*p, &L);
    if (v != ZEUS_OK) return v;
    const Layout lay = layout_for(*p, L);
    v = check_ws(workspace, workspace_bytes, lay.total);
    if (v != ZEUS_OK) return v;
    cudaStream_t st = as_stream(stream);
    Ctrl* ctrl = at<Ctrl>(workspace, lay.ctrl);
    double* f = f_out ? f_out : at<double>(workspace, lay.f_tmp);
    cudaError_t e = cudaMemsetAsync(ctrl, 0, lay.partials - lay.ctrl, st);  // control, ready flags
    if (e != cudaSuccess) return ZEUS_ECUDA;
    e = launch_bfgs(*p, L, x0, x_out, f, gnorm_out, status_out, iters_out, ctrl,
                    queue_for(workspace, lay, L), st);
    if (e != cudaSuccess) return ZEUS_ECUDA;
    return finish_with_argmin(*p, workspace, lay, f, result, false, st);
}

int zeus_pso(const zeus_problem* p, void* workspace, size_t workspace_bytes, double* x_out,
             double* v_out, double* px_out, double* pf_out, double* gx_out, zeus_result* result,
             void* stream) {
    int v = validate(p);
    if (v != ZEUS_OK) return v;
    if (!x_out || !v_out || !px_out || !pf_out || !gx_out) return ZEUS_EINVAL;
    BfgsLaunch L;
    v = plan_bfgs(*p, &L);
    if (v != ZEUS_OK) return v;
    const Layout lay = layout_for(*p, L);
    // only the control block and the partials are used
    v = check_ws(workspace, workspace_bytes, lay.f_tmp);
    if (v != ZEUS_OK) return v;
    cudaStream_t st = as_stream(stream);
    Ctrl* ctrl = at<Ctrl>(workspace, lay.ctrl);
    cudaError_t e = cudaMemsetAsync(ctrl, 0, sizeof(Ctrl), st);
    if (e != cudaSuccess) return ZEUS_ECUDA;
    e = launch_pso(*p, lanes_for_dim(p->dim), x_out, v_out, px_out, pf_out, gx_out, ctrl,
                   at<ArgPair>(workspace, lay.partials), result, st);
    return cuda_status(e);
}

int zeus_objective_eval(int32_t objective, int32_t dim, int64_t n, const double* x,
                        double* f_out, double* g_out, int32_t grad_mode, void* stream) {
    zeus_problem p;
    zeus_default_problem(&p);
    p.objective = objective;
    p.dim = dim;
    p.grad_mode = grad_mode;
    const int v = validate(&p);
    if (v != ZEUS_OK) return v;
    if (n < 0 || (n > 0 && !x)) return ZEUS_EINVAL;
    return cuda_status(launch_objective(objective, dim, n, x, f_out, g_out, grad_mode,
                                        as_stream(stream)));
}

int zeus_objective_eval_f32(int32_t objective, int32_t dim, int64_t n, const float* x,
                            float* f_out, float* g_out, int32_t grad_mode, void* stream) {
    zeus_problem p;
    zeus_default_problem(&p);
    p.objective = objective;
    p.dim = dim;
    p.grad_mode = grad_mode;
    const int v = validate(&p);
    if (v != ZEUS_OK) return v;
    if (n < 0 || (n > 0 && !x)) return ZEUS_EINVAL;
    return cuda_status(launch_objective_f32(objective, dim, n, x, f_out, g_out, grad_mode,
                                            as_stream(stream)));
}

int zeus_argmin_workspace_size(int64_t n, size_t* bytes) {
    if (!bytes || n < 1) return ZEUS_EINVAL;
    *bytes = align256(sizeof(Ctrl)) + align256((size_t)argmin_blocks(n) * sizeof(ArgPair));
    return ZEUS_OK;
}

int zeus_argmin(const double* f, int64_t n, void* workspace, size_t workspace_bytes,
                zeus_result* result, void* stream) {
    size_t need = 0;
    int v = zeus_argmin_workspace_size(n, &need);
    if (v != ZEUS_OK) return v;
    if (!f || !result) return ZEUS_EINVAL;
    v = check_ws(workspace, workspace_bytes, need);
    if (v != ZEUS_OK) return v;
    cudaStream_t st = as_stream(stream);
    Ctrl* ctrl = at<Ctrl>(workspace, 0);
    ArgPair* parts = at<ArgPair>(workspace, align256(sizeof(Ctrl)));
    cudaError_t e = cudaMemsetAsync(ctrl, 0, sizeof(Ctrl), st);
    if (e != cudaSuccess) return ZEUS_ECUDA;
    return cuda_status(launch_argmin(f, n, ctrl, parts, result, 0, st));
}

int zeus_uniform(uint64_t seed, uint64_t problem, uint64_t phase, int64_t n, int32_t dim,
                 double* out, void* stream) {
    if (n < 0 || dim < 1 || (n > 0 && !out)) return ZEUS_EINVAL;
    return cuda_status(launch_uniform(seed, problem, phase, n, dim, out, as_stream(stream)));
}

int zeus_cluster_workspace_size(int32_t max_clusters, size_t* bytes) {
    if (!bytes || max_clusters < 1 || max_clusters > ZEUS_CLUSTER_MAX) return ZEUS_EINVAL;
    *bytes = cluster_work_bytes(max_clusters);
    return ZEUS_OK;
}

int zeus_cluster(const zeus_cluster_params* cp, int64_t n, int32_t dim, const double* x,
                 const double* f, const int32_t* status, int32_t* label_out, int32_t* leader_out,
                 int32_t* count_out, zeus_cluster_result* result, void* workspace,
                 size_t workspace_bytes, void* stream) {
    if (!cp) return ZEUS_EINVAL;
    if (cp->method != ZEUS_CLUSTER_BY_F && cp->method != ZEUS_CLUSTER_BY_X) return ZEUS_EINVAL;
    if (cp->max_clusters < 1 || cp->max_clusters > ZEUS_CLUSTER_MAX) return ZEUS_EINVAL;
    if (cp->only_converged != 0 && cp->only_converged != 1) return ZEUS_EINVAL;
    if (cp->pad != 0 || !isfinite(cp->tol) || !(cp->tol >= 0.0)) return ZEUS_EINVAL;
    if (n < 0 || n > 0x7fffffffll || dim < 1 || dim > 4096) return ZEUS_EINVAL;
    if (n > 0 && (!f || !label_out)) return ZEUS_EINVAL;
    if (n > 0 && cp->method == ZEUS_CLUSTER_BY_X && !x) return ZEUS_EINVAL;
    if (n > 0 && cp->only_converged && !status) return ZEUS_EINVAL;
    if (!workspace || workspace_bytes < cluster_work_bytes(cp->max_clusters) ||
        ((uintptr_t)workspace & 255u) != 0)
        return ZEUS_EWORKSPACE;
    return cuda_status(launch_cluster(*cp, (int)n, dim, x, f, status, label_out, leader_out,
                                      count_out, result, workspace, as_stream(stream)));
}

int32_t zeus_user_objective_count(void) { return user_objective_count(); }

int zeus_user_objective_info(int32_t k, char* name, int32_t name_len, int32_t* min_dim,
                             int32_t* max_dim) {
    const char* nm;
    int lo, hi;
    if (!user_objective_meta(k, &nm, &lo, &hi)) return ZEUS_EINVAL;
    if (name && name_len > 0) {
        strncpy(name, nm, (size_t)name_len - 1);
        name[name_len - 1] = '\0';
    }
    if (min_dim) *min_dim = lo;
    if (max_dim) *max_dim = hi;
    return ZEUS_OK;
}

int zeus_math_eval(int32_t fn, int64_t n, const double* x, double* y0, double* y1, void* stream) {
    if (fn < 0 || fn > 4 || n < 0) return ZEUS_EINVAL;
    if (n > 0 && (!x || !y0 || ((fn == 0 || fn == 2) && !y1))) return ZEUS_EINVAL;
    return cuda_status(launch_math(fn, n, x, y0, y1, as_stream(stream)));
}

// ---------------------------------------------------------------------------
// Host-buffer interface
// ---------------------------------------------------------------------------
struct zeus_context {
    int device;
    void* ws;
    size_t ws_bytes;
    double* x;
    double* f;
    double* gn;
    int32_t* st;
    int32_t* it;
    zeus_result* res;
    size_t cap_n, cap_nd;
};

static void ctx_free_buffers(zeus_context* c) {
    cudaFree(c->ws);
    cudaFree(c->x);
    cudaFree(c->f);
    cudaFree(c->gn);
    cudaFree(c->st);
    cudaFree(c->it);
    c->ws = nullptr;
    c->x = c->f = c->gn = nullptr;
    c->st = c->it = nullptr;
    c->ws_bytes = 0;
    c->cap_n = c->cap_nd = 0;
}

int zeus_context_create(zeus_context** ctx) {
    if (!ctx) return ZEUS_EINVAL;
    zeus_context* c = (zeus_context*)calloc(1, sizeof(zeus_context));
    if (!c) return ZEUS_ENOMEM;
    if (cudaGetDevice(&c->device) != cudaSuccess) {
        free(c);
        return ZEUS_ECUDA;
    }
    if (cudaMalloc(&c->res, sizeof(zeus_result)) != cudaSuccess) {
        free(c);
        return ZEUS_ENOMEM;
    }
    *ctx = c;
    return ZEUS_OK;
}

int zeus_context_destroy(zeus_context* ctx) {
    if (!ctx) return ZEUS_EINVAL;
    cudaDeviceSynchronize();
    ctx_free_buffers(ctx);
    cudaFree(ctx->res);
    free(ctx);
    return ZEUS_OK;
}

int zeus_solve_host(zeus_context* ctx, const zeus_problem* p, double* x_out, double* f_out,
                    double* gnorm_out, int32_t* status_out, int32_t* iters_out,
                    zeus_result* result, void* stream) {
    if (!ctx || !x_out) return ZEUS_EINVAL;
    size_t need = 0;
    int v = zeus_workspace_size(p, &need);
    if (v != ZEUS_OK) return v;
    const size_t n = (size_t)p->n_starts, nd = n * (size_t)p->dim;
    if (need > ctx->ws_bytes || n > ctx->cap_n || nd > ctx->cap_nd) {
        cudaStream_t st0 = as_stream(stream);
        cudaStreamSynchronize(st0);
        ctx_free_buffers(ctx);
        if (cudaMalloc(&ctx->ws, need) != cudaSuccess || cudaMalloc(&ctx->x, nd * 8) != cudaSuccess ||
            cudaMalloc(&ctx->f, n * 8) != cudaSuccess || cudaMalloc(&ctx->gn, n * 8) != cudaSuccess ||
            cudaMalloc(&ctx->st, n * 4) != cudaSuccess || cudaMalloc(&ctx->it, n * 4) != cudaSuccess) {
            ctx_free_buffers(ctx);
            cudaGetLastError();
            return ZEUS_ENOMEM;
        }
        ctx->ws_bytes = need;
        ctx->cap_n = n;
        ctx->cap_nd = nd;
    }
    cudaStream_t st = as_stream(stream);
    v = zeus_solve(p, ctx->ws, ctx->ws_bytes, ctx->x, ctx->f, ctx->gn, ctx->st, ctx->it, ctx->res,
                   stream);
    if (v != ZEUS_OK) return v;
    cudaError_t e = cudaMemcpyAsync(x_out, ctx->x, nd * 8, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && f_out) e = cudaMemcpyAsync(f_out, ctx->f, n * 8, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && gnorm_out)
        e = cudaMemcpyAsync(gnorm_out, ctx->gn, n * 8, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && status_out)
        e = cudaMemcpyAsync(status_out, ctx->st, n * 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && iters_out)
        e = cudaMemcpyAsync(iters_out, ctx->it, n * 4, cudaMemcpyDeviceToHost, st);
    // the summary always comes back: its error word says whether a bounded
    // device wait gave up (the outputs are then incomplete)
    zeus_result local;
    zeus_result* r = result ? result : &local;
    if (e == cudaSuccess) e = cudaMemcpyAsync(r, ctx->res, sizeof(zeus_result), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_status(e);
    return r->error ? ZEUS_ETIMEOUT : ZEUS_OK;
}

}  // extern "C"
