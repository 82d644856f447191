// zeus_batch.cu -- the batched form: many independent problems (mixed
// objective, dimension and swarm size) solved by one fixed sequence of
// launches.  PSO: one launch per update over every problem's blocks.
// BFGS: persistent blocks pull items from a device work list, one launch per
// shared-memory class (items that need about the same shared memory, so
// that each launch runs at the occupancy its items allow), then one launch
// over the starts the lane tiles handed over.  Then one reduction block per
// problem.  zeus_batch_solve enqueues kernels and one memset only, so the
// sequence can be recorded in a CUDA graph and replayed; the tables it reads
// are uploaded once by zeus_batch_prepare.
//
// Work items: problems with d <= 16 run one lane per start in tiles of up to
// 128 starts (long runs handed over to one block per start, as in
// zeus_bfgs.cu); larger problems run one block per start.  Every start runs
// the same bodies as in a single-problem solve, so each problem's result
// equals its zeus_solve result bit for bit.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "zeus.h"
#include "zeus_internal.h"

namespace zeus {

cudaError_t launch_batch_bfgs(const BatchDev& bd, int precision, int grad_mode, bool user, int cls,
                              int first, int count, size_t smem, bool warp_items, double* x_out,
                              double* f_out, double* gnorm_out, int32_t* status_out,
                              int32_t* iters_out, cudaStream_t st) {
    const bool f32 = precision == ZEUS_FP32_GUARDED;
    auto go = [&](auto launch) {
        return launch(bd, cls, first, count, smem, warp_items, x_out, f_out, gnorm_out, status_out,
                      iters_out, st);
    };
    if (grad_mode == ZEUS_GRAD_ADJOINT)
        return f32 ? go(batch_launch_gt<ZEUS_GRAD_ADJOINT, float, false>)
                   : go(batch_launch_gt<ZEUS_GRAD_ADJOINT, double, false>);
    if (user)
        return f32 ? go(batch_launch_gt<ZEUS_GRAD_FORWARD, float, true>)
                   : go(batch_launch_gt<ZEUS_GRAD_FORWARD, double, true>);
    return f32 ? go(batch_launch_gt<ZEUS_GRAD_FORWARD, float, false>)
               : go(batch_launch_gt<ZEUS_GRAD_FORWARD, double, false>);
}

}  // namespace zeus

// ===========================================================================
// Host side: plan, upload, solve
// ===========================================================================
using namespace zeus;

namespace {

constexpr size_t kSmemCap = 226 * 1024;   // dynamic shared memory per block (the kernel's
                                          // static shared memory takes the rest of 227 KB)
constexpr size_t kSmemPerSM = 228 * 1024; // shared memory per SM
constexpr int kMaxPerSM = 16;             // 128-thread blocks per SM (2048 threads)

struct BatchLayout {
    size_t probs, xoff, soff, goff, poff, pblk0, pblk, plane, pso_table, items, stride, budget,
        pctrl, gctrl, heads, partials, v, px, pf, gx, q_prob, q_start, q_k, q_feval, q_h, total;
};

struct Sizes {
    long long n = 0, pso_blocks = 0, items = 0, total_starts = 0, total_coords = 0, total_g = 0;
    long long q_cap = 0, d_max_handover = 0;
};

struct BatchHost {
    std::vector<zeus_problem> probs;
    std::vector<long long> xoff, soff, goff, poff;
    std::vector<int> pblk0, pblk, plane, pso_table, stride, budget;
    std::vector<int4> items;
    Sizes sz;
    int pso_iters_max = 0, handover_smem = 0, n_classes = 0, n_user = 0;
    int class_first[ZEUS_BATCH_MAX_CLASSES], class_count[ZEUS_BATCH_MAX_CLASSES],
        class_smem[ZEUS_BATCH_MAX_CLASSES], class_kind[ZEUS_BATCH_MAX_CLASSES];
};

// blocks of the batched BFGS kernel that share an SM at this dynamic shared
// memory (an estimate for grouping; the launch asks the occupancy API)
int per_sm(size_t smem) {
    const size_t per = smem + 1024 + 1024;  // static shared memory + reservation
    const int n = (int)(kSmemPerSM / per);
    return n < 1 ? 1 : (n > kMaxPerSM ? kMaxPerSM : n);
}

struct Work {
    int4 item;
    size_t smem;
    int dim;
};

int build_host(const zeus_problem* probs, int n, BatchHost& B) {
    if (!probs || n < 1) return ZEUS_EINVAL;
    const int prec = probs[0].precision, grad = probs[0].grad_mode;
    const size_t ts = prec == ZEUS_FP32_GUARDED ? 4 : 8;
    B.probs.assign(probs, probs + n);
    std::vector<Work> work;
    long long handover_starts = 0;
    size_t hsmem = 0;
    for (int P = 0; P < n; ++P) {
        const zeus_problem& p = probs[P];
        const int v = zeus_validate(&p);
        if (v != ZEUS_OK) return v;
        if (p.precision != prec || p.grad_mode != grad) return ZEUS_EINVAL;
        if (p.n_starts >= (1ll << 30)) return ZEUS_EINVAL;
        BfgsLaunch L;
        const int r = plan_bfgs(p, &L);
        if (r != ZEUS_OK) return r;
        if (L.stream && !L.lbfgs) return ZEUS_EUNSUPPORTED;  // dense H on chip in a batch
        if (p.objective >= ZEUS_OBJ_USER) ++B.n_user;
        const int d = p.dim;
        const int G = lanes_for_dim(d);
        const int nb = pso_blocks(p, G);
        B.xoff.push_back(B.sz.total_coords);
        B.soff.push_back(B.sz.total_starts);
        B.goff.push_back(B.sz.total_g);
        B.poff.push_back((long long)B.pso_table.size());
        B.pblk0.push_back((int)B.pso_table.size());
        B.pblk.push_back(nb);
        B.plane.push_back(G);
        for (int b = 0; b < nb; ++b) B.pso_table.push_back(P);
        B.sz.total_coords += p.n_starts * d;
        B.sz.total_starts += p.n_starts;
        B.sz.total_g += d;
        B.pso_iters_max = std::max(B.pso_iters_max, (int)p.pso_iters);
        B.stride.push_back(L.stride);
        B.budget.push_back(L.budget);
        if (L.lbfgs) {  // one 256-thread block per start, the pairs in shared memory
            for (long long s = 0; s < p.n_starts; ++s)
                work.push_back({make_int4(P, (int)s, 0, 3), L.stream_smem, d});
        } else if (L.narrow) {
            const size_t row = (size_t)L.stride * ts;
            const int tile = (int)std::min<size_t>(kWideThreads, kSmemCap / row);
            for (long long s = 0; s < p.n_starts; s += tile) {
                const int c = (int)std::min<long long>(tile, p.n_starts - s);
                work.push_back({make_int4(P, (int)s, c, 0), (size_t)c * row, d});
            }
            if (L.budget > 0) {
                handover_starts += p.n_starts;
                B.sz.d_max_handover = std::max<long long>(B.sz.d_max_handover, d);
                hsmem = std::max(hsmem, L.wide_smem);
            }
        } else if (L.warp) {  // one warp per start, four starts to a block
            for (long long s = 0; s < p.n_starts; ++s)
                work.push_back({make_int4(P, (int)s, L.W, 2), 4 * L.warp_slot, d});
        } else {
            for (long long s = 0; s < p.n_starts; ++s)
                work.push_back({make_int4(P, (int)s, L.W, 1), L.wide_smem, d});
        }
    }
    if (work.size() >= (size_t)1 << 31) return ZEUS_EINVAL;
    // classes by kind (L-BFGS, warp-per-start and block-per-start items,
    // then lane tiles, which feed the hand-over queue) and occupancy (fewest
    // blocks per SM first); within a class larger d first (long work starts
    // early)
    std::stable_sort(work.begin(), work.end(), [](const Work& a, const Work& b) {
        if (a.item.w != b.item.w) return a.item.w > b.item.w;
        const int ca = per_sm(a.smem), cb = per_sm(b.smem);
        if (ca != cb) return ca < cb;
        return a.dim > b.dim;
    });
    B.n_classes = 0;
    for (size_t i = 0; i < work.size(); ++i) {
        const int c = per_sm(work[i].smem);
        if (i == 0 || c != per_sm(work[i - 1].smem) || work[i].item.w != work[i - 1].item.w) {
            if (B.n_classes == ZEUS_BATCH_MAX_CLASSES) return ZEUS_EUNSUPPORTED;
            B.class_first[B.n_classes] = (int)i;
            B.class_count[B.n_classes] = 0;
            B.class_smem[B.n_classes] = 0;
            B.class_kind[B.n_classes] = work[i].item.w;
            ++B.n_classes;
        }
        const int k = B.n_classes - 1;
        B.class_count[k] += 1;
        B.class_smem[k] = std::max(B.class_smem[k], (int)work[i].smem);
        B.items.push_back(work[i].item);
    }
    B.sz.n = n;
    B.sz.pso_blocks = (long long)B.pso_table.size();
    B.sz.items = (long long)B.items.size();
    // Hand-over queue.  FP64: room for many long runs, so that lane tiles
    // do not wait on a few of their lanes (lane efficiency); FP32 runs
    // rarely meet the gradient tolerance and would all be handed over, so
    // as in the single-problem plan at most two per block of the hand-over
    // launch.  Within 256 MB of H either way.
    B.sz.q_cap = std::min<long long>(handover_starts,
                                     prec == ZEUS_FP32_GUARDED ? 2ll * 152 * 4 : 65536ll);
    if (B.sz.q_cap > 0) {
        const long long per = B.sz.d_max_handover * B.sz.d_max_handover * 8;
        B.sz.q_cap = std::max<long long>(1, std::min<long long>(B.sz.q_cap, (256ll << 20) / per));
    }
    B.handover_smem = (int)hsmem;
    return ZEUS_OK;
}

BatchLayout batch_layout(const Sizes& z) {
    BatchLayout l;
    size_t off = 0;
    auto put = [&](size_t bytes) {
        const size_t o = off;
        off += align256(bytes);
        return o;
    };
    const size_t n = (size_t)z.n;
    l.probs = put(n * sizeof(zeus_problem));
    l.xoff = put(n * 8);
    l.soff = put(n * 8);
    l.goff = put(n * 8);
    l.poff = put(n * 8);
    l.pblk0 = put(n * 4);
    l.pblk = put(n * 4);
    l.plane = put(n * 4);
    l.pso_table = put((size_t)z.pso_blocks * 4);
    l.items = put((size_t)z.items * sizeof(int4));
    l.stride = put(n * 4);
    l.budget = put(n * 4);
    // from here on: zeroed by every solve (counters), then scratch
    l.pctrl = put(n * sizeof(Ctrl));
    l.gctrl = put(sizeof(Ctrl));
    l.heads = put(ZEUS_BATCH_MAX_CLASSES * sizeof(unsigned));
    l.partials = put((size_t)z.pso_blocks * sizeof(ArgPair));
    l.v = put((size_t)z.total_coords * 8);
    l.px = put((size_t)z.total_coords * 8);
    l.pf = put((size_t)z.total_starts * 8);
    l.gx = put((size_t)z.total_g * 8);
    const size_t qc = (size_t)z.q_cap;
    l.q_prob = put(qc * 4);
    l.q_start = put(qc * 4);
    l.q_k = put(qc * 4);
    l.q_feval = put(qc * 4);
    l.q_h = put(qc * (size_t)z.d_max_handover * (size_t)z.d_max_handover * 8);
    l.total = off;
    return l;
}

BatchDev batch_dev(void* ws, const BatchLayout& l, const Sizes& z) {
    char* b = static_cast<char*>(ws);
    BatchDev d;
    d.probs = reinterpret_cast<const zeus_problem*>(b + l.probs);
    d.xoff = reinterpret_cast<const long long*>(b + l.xoff);
    d.soff = reinterpret_cast<const long long*>(b + l.soff);
    d.goff = reinterpret_cast<const long long*>(b + l.goff);
    d.poff = reinterpret_cast<const long long*>(b + l.poff);
    d.pblk0 = reinterpret_cast<const int*>(b + l.pblk0);
    d.pblk = reinterpret_cast<const int*>(b + l.pblk);
    d.plane = reinterpret_cast<const int*>(b + l.plane);
    d.pso_table = reinterpret_cast<const int*>(b + l.pso_table);
    d.items = reinterpret_cast<const int4*>(b + l.items);
    d.stride = reinterpret_cast<const int*>(b + l.stride);
    d.budget = reinterpret_cast<const int*>(b + l.budget);
    d.pctrl = reinterpret_cast<Ctrl*>(b + l.pctrl);
    d.gctrl = reinterpret_cast<Ctrl*>(b + l.gctrl);
    d.heads = reinterpret_cast<unsigned*>(b + l.heads);
    d.partials = reinterpret_cast<ArgPair*>(b + l.partials);
    d.v = reinterpret_cast<double*>(b + l.v);
    d.px = reinterpret_cast<double*>(b + l.px);
    d.pf = reinterpret_cast<double*>(b + l.pf);
    d.gx = reinterpret_cast<double*>(b + l.gx);
    d.q.prob = reinterpret_cast<int*>(b + l.q_prob);
    d.q.start = reinterpret_cast<int*>(b + l.q_start);
    d.q.k = reinterpret_cast<int*>(b + l.q_k);
    d.q.feval = reinterpret_cast<int*>(b + l.q_feval);
    d.q.H = reinterpret_cast<double*>(b + l.q_h);
    d.q.cap = (int)z.q_cap;
    d.q.hslots = nullptr;
    d.q.hstride = z.d_max_handover * z.d_max_handover;
    d.n = (int)z.n;
    d.n_items = (int)z.items;
    d.pso_blocks = (int)z.pso_blocks;
    return d;
}

Sizes plan_sizes(const zeus_batch_plan& p) {
    Sizes z;
    z.n = p.n_problems;
    z.pso_blocks = p.pso_blocks;
    z.items = p.items;
    z.total_starts = p.total_starts;
    z.total_coords = p.total_coords;
    z.total_g = p.total_g;
    z.q_cap = p.q_cap;
    z.d_max_handover = p.d_max_handover;
    return z;
}

void fill_plan(const BatchHost& B, const BatchLayout& l, zeus_batch_plan* plan) {
    memset(plan, 0, sizeof(*plan));
    plan->n_problems = (int32_t)B.sz.n;
    plan->pso_blocks = (int32_t)B.sz.pso_blocks;
    plan->items = (int32_t)B.sz.items;
    plan->pso_iters_max = B.pso_iters_max;
    plan->q_cap = (int32_t)B.sz.q_cap;
    plan->d_max_handover = (int32_t)B.sz.d_max_handover;
    plan->precision = B.probs[0].precision;
    plan->grad_mode = B.probs[0].grad_mode;
    plan->n_classes = B.n_classes;
    plan->handover_smem = B.handover_smem;
    plan->n_user = B.n_user;
    plan->pad = 0;
    for (int c = 0; c < B.n_classes; ++c) {
        plan->class_first[c] = B.class_first[c];
        plan->class_count[c] = B.class_count[c];
        plan->class_smem[c] = B.class_smem[c];
        plan->class_kind[c] = B.class_kind[c];
    }
    plan->total_starts = B.sz.total_starts;
    plan->total_coords = B.sz.total_coords;
    plan->total_g = B.sz.total_g;
    plan->workspace_bytes = l.total;
    plan->table_bytes = l.pctrl;
}

int check_ws(void* ws, size_t have, size_t need) {
    if (!ws || need > have || ((uintptr_t)ws & 255u) != 0) return ZEUS_EWORKSPACE;
    return ZEUS_OK;
}

// The library's own streams of each device: `stream` carries the lane-tile
// classes and the hand-over launch, `stream2` every other block-, warp- or
// L-BFGS class (the rest run on the caller's stream), so that one class's
// tail (its last long runs, on a few SMs) overlaps the next class's start;
// and the events that fork them from and join them to the caller's stream.
// Created once per device, kept until exit; the mutex also keeps one
// call's fork and join from interleaving with another's.
constexpr int kMaxDevices = 64;
struct Aux {
    cudaStream_t stream = nullptr, stream2 = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr, join2 = nullptr;
};
std::mutex g_aux_mu;
Aux g_aux[kMaxDevices];

// with g_aux_mu held
cudaError_t aux_for_device(Aux** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    Aux& a = g_aux[dev];
    if (!a.stream) {
        e = cudaStreamCreateWithFlags(&a.stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&a.stream2, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&a.fork, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&a.join, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&a.join2, cudaEventDisableTiming);
        if (e != cudaSuccess) {
            a = Aux();
            return e;
        }
    }
    *out = &a;
    return cudaSuccess;
}

bool plan_sane(const zeus_batch_plan& p) {
    if (p.n_problems < 1 || p.pso_blocks < 1 || p.items < 1 || p.pso_iters_max < 0) return false;
    if (p.n_classes < 1 || p.n_classes > ZEUS_BATCH_MAX_CLASSES) return false;
    if (p.q_cap < 0 || p.d_max_handover < 0 || p.handover_smem < 0) return false;
    if (p.q_cap > 0 && (p.d_max_handover < 1 || p.handover_smem < 1)) return false;
    if (p.handover_smem > (int)kSmemCap) return false;
    long long next = 0;
    for (int c = 0; c < p.n_classes; ++c) {
        if (p.class_first[c] != next || p.class_count[c] < 1) return false;
        if (p.class_smem[c] < 0 || p.class_smem[c] > (int)kSmemCap) return false;
        if (p.class_kind[c] < 0 || p.class_kind[c] > 3) return false;
        next += p.class_count[c];
    }
    if (next != p.items) return false;
    if (p.precision != ZEUS_FP64 && p.precision != ZEUS_FP32_GUARDED) return false;
    if (p.grad_mode != ZEUS_GRAD_FORWARD && p.grad_mode != ZEUS_GRAD_ADJOINT) return false;
    if (p.n_user < 0 || p.n_user > p.n_problems || p.pad != 0) return false;
    if (p.n_user > 0 && p.grad_mode != ZEUS_GRAD_FORWARD) return false;
    const BatchLayout l = batch_layout(plan_sizes(p));
    return l.total == p.workspace_bytes && l.pctrl == p.table_bytes;
}

}  // namespace

extern "C" {

int zeus_batch_plan_make(const zeus_problem* probs, int32_t n, zeus_batch_plan* plan) {
    if (!plan) return ZEUS_EINVAL;
    BatchHost B;
    const int v = build_host(probs, n, B);
    if (v != ZEUS_OK) return v;
    fill_plan(B, batch_layout(B.sz), plan);
    return ZEUS_OK;
}

int zeus_batch_prepare(const zeus_problem* probs, int32_t n, const zeus_batch_plan* plan,
                       void* workspace, size_t workspace_bytes, void* stream) {
    if (!plan) return ZEUS_EINVAL;
    BatchHost B;
    int v = build_host(probs, n, B);
    if (v != ZEUS_OK) return v;
    const BatchLayout l = batch_layout(B.sz);
    zeus_batch_plan mine;
    fill_plan(B, l, &mine);
    if (memcmp(&mine, plan, sizeof(mine)) != 0) return ZEUS_EINVAL;  // not this batch's plan
    v = check_ws(workspace, workspace_bytes, l.total);
    if (v != ZEUS_OK) return v;
    // the tables, staged in host memory and copied in one transfer
    std::vector<char> host(l.pctrl, 0);
    auto put = [&](size_t off, const void* src, size_t bytes) {
        if (bytes) memcpy(host.data() + off, src, bytes);
    };
    const size_t nn = B.probs.size();
    put(l.probs, B.probs.data(), nn * sizeof(zeus_problem));
    put(l.xoff, B.xoff.data(), nn * 8);
    put(l.soff, B.soff.data(), nn * 8);
    put(l.goff, B.goff.data(), nn * 8);
    put(l.poff, B.poff.data(), nn * 8);
    put(l.pblk0, B.pblk0.data(), nn * 4);
    put(l.pblk, B.pblk.data(), nn * 4);
    put(l.plane, B.plane.data(), nn * 4);
    put(l.pso_table, B.pso_table.data(), B.pso_table.size() * 4);
    put(l.items, B.items.data(), B.items.size() * sizeof(int4));
    put(l.stride, B.stride.data(), nn * 4);
    put(l.budget, B.budget.data(), nn * 4);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemcpyAsync(workspace, host.data(), host.size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess) {
        std::lock_guard<std::mutex> lock(g_aux_mu);
        Aux* a = nullptr;
        e = aux_for_device(&a);
    }
    return e == cudaSuccess ? ZEUS_OK : ZEUS_ECUDA;
}

int zeus_batch_solve(const zeus_batch_plan* plan, void* workspace, size_t workspace_bytes,
                     double* x_out, double* f_out, double* gnorm_out, int32_t* status_out,
                     int32_t* iters_out, zeus_result* results, void* stream) {
    if (!plan || !x_out || !f_out || !plan_sane(*plan)) return ZEUS_EINVAL;
    const Sizes z = plan_sizes(*plan);
    const BatchLayout l = batch_layout(z);
    int v = check_ws(workspace, workspace_bytes, l.total);
    if (v != ZEUS_OK) return v;
    const BatchDev bd = batch_dev(workspace, l, z);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    // per-problem control blocks, queue counters and class counters start at zero
    cudaError_t e =
        cudaMemsetAsync(static_cast<char*>(workspace) + l.pctrl, 0, l.partials - l.pctrl, st);
    for (int t = -1; t < plan->pso_iters_max && e == cudaSuccess; ++t)
        e = launch_batch_pso(bd, t, x_out, st);
    if (e != cudaSuccess) return ZEUS_ECUDA;
    {
        // fork: lane-tile classes then the hand-over launch on the library's
        // stream, the other classes alternately on `stream` and the
        // library's second stream; join before the reduction.  Classes
        // touch disjoint starts, and the lane-tile set disjoint problems (a
        // problem's starts are all lane tiles or all of one other kind).
        std::lock_guard<std::mutex> lock(g_aux_mu);
        Aux* a = nullptr;
        e = aux_for_device(&a);
        if (e == cudaSuccess) e = cudaEventRecord(a->fork, st);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(a->stream, a->fork, 0);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(a->stream2, a->fork, 0);
        int n_other = 0;
        for (int c = 0; c < plan->n_classes && e == cudaSuccess; ++c) {
            const int kind = plan->class_kind[c];
            const cudaStream_t cs = kind == 0 ? a->stream : ((n_other++ & 1) ? a->stream2 : st);
            if (kind == 3)
                e = launch_batch_lbfgs(bd, plan->precision, plan->grad_mode, c,
                                       plan->class_first[c], plan->class_count[c],
                                       (size_t)plan->class_smem[c], x_out, f_out, gnorm_out,
                                       status_out, iters_out, cs);
            else
                e = launch_batch_bfgs(bd, plan->precision, plan->grad_mode, plan->n_user > 0, c,
                                      plan->class_first[c], plan->class_count[c],
                                      (size_t)plan->class_smem[c], kind == 2, x_out, f_out,
                                      gnorm_out, status_out, iters_out, cs);
        }
        if (e == cudaSuccess && plan->q_cap > 0)
            e = launch_batch_bfgs(bd, plan->precision, plan->grad_mode, plan->n_user > 0, -1, 0, 0,
                                  (size_t)plan->handover_smem, false, x_out, f_out, gnorm_out,
                                  status_out, iters_out, a->stream);
        // join whatever was enqueued, also after a failed launch, so that a
        // capture never ends with the second stream still forked
        if (a) {
            cudaError_t e1 = cudaEventRecord(a->join, a->stream);
            if (e1 == cudaSuccess) e1 = cudaStreamWaitEvent(st, a->join, 0);
            if (e1 == cudaSuccess) e1 = cudaEventRecord(a->join2, a->stream2);
            if (e1 == cudaSuccess) e1 = cudaStreamWaitEvent(st, a->join2, 0);
            if (e == cudaSuccess) e = e1;
        }
    }
    if (e == cudaSuccess) e = launch_batch_argmin(bd, f_out, results, st);
    return e == cudaSuccess ? ZEUS_OK : ZEUS_ECUDA;
}

int zeus_batch_cluster(const zeus_batch_plan* plan, const void* workspace, size_t workspace_bytes,
                       const zeus_cluster_params* cp, const double* x_out, const double* f_out,
                       const int32_t* status_out, int32_t* label_out, int32_t* leader_out,
                       int32_t* count_out, zeus_cluster_result* results, void* stream) {
    if (!plan || !cp || !plan_sane(*plan)) return ZEUS_EINVAL;
    if (cp->method != ZEUS_CLUSTER_BY_F && cp->method != ZEUS_CLUSTER_BY_X) return ZEUS_EINVAL;
    if (cp->max_clusters < 1 || cp->max_clusters > ZEUS_CLUSTER_MAX) return ZEUS_EINVAL;
    if (cp->only_converged != 0 && cp->only_converged != 1) return ZEUS_EINVAL;
    if (cp->pad != 0 || !isfinite(cp->tol) || !(cp->tol >= 0.0)) return ZEUS_EINVAL;
    if (!f_out || !label_out || (cp->method == ZEUS_CLUSTER_BY_X && !x_out)) return ZEUS_EINVAL;
    if (cp->only_converged && !status_out) return ZEUS_EINVAL;
    const Sizes z = plan_sizes(*plan);
    const BatchLayout l = batch_layout(z);
    const int v = check_ws(const_cast<void*>(workspace), workspace_bytes, l.total);
    if (v != ZEUS_OK) return v;
    const BatchDev bd = batch_dev(const_cast<void*>(workspace), l, z);
    const cudaError_t e = launch_batch_cluster(*cp, bd, x_out, f_out, status_out, label_out,
                                               leader_out, count_out, results,
                                               reinterpret_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? ZEUS_OK : ZEUS_ECUDA;
}

}  // extern "C"
