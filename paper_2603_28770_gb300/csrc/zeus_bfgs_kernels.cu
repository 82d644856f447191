// zeus_bfgs_kernels.cu -- the narrow and wide BFGS kernels of zeus_bfgs.cu
// for one (gradient mode, precision) pair, chosen at compile time by
// ZEUS_KGRAD (0 forward, 1 adjoint) and ZEUS_KF32 (0 FP64, 1 FP32 with FP64
// guards): the library compiles this file once per pair, in parallel.
#include "zeus_bfgs.cuh"

#if !defined(ZEUS_KGRAD) || !defined(ZEUS_KF32)
#error "compile with -DZEUS_KGRAD=0|1 -DZEUS_KF32=0|1"
#endif

namespace zeus {

template <int OBJ, int GRAD, class T>
__global__ void __launch_bounds__(kNarrowThreads)
    bfgs_narrow_kernel(const zeus_problem p, const int stride, const int budget,
                       const double* x0, double* x_out,  // may alias (in-place run)
                       double* __restrict__ f_out, double* __restrict__ gnorm_out,
                       int32_t* __restrict__ status_out, int32_t* __restrict__ iters_out,
                       Ctrl* __restrict__ ctrl, const Queue q) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* smem = reinterpret_cast<T*>(smem_raw);
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= p.n_starts) return;
    const RunIO io{x0, x_out, f_out, gnorm_out, status_out, iters_out, ctrl};
    narrow_run<OBJ, GRAD, T>(p, s, smem + (size_t)threadIdx.x * stride, budget, io, ctrl, q, 0);
}

template <int OBJ, int GRAD, class T>
__global__ void __launch_bounds__(kWideThreads)
    bfgs_wide_kernel(const zeus_problem p, const int W, const double* x0, double* x_out,
                     double* __restrict__ f_out, double* __restrict__ gnorm_out,
                     int32_t* __restrict__ status_out, int32_t* __restrict__ iters_out,
                     Ctrl* __restrict__ ctrl, const Queue q, const int all_starts) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ WideShared sh;
    const int tid = wide_role(blockDim.x);
    const RunIO io{x0, x_out, f_out, gnorm_out, status_out, iters_out, ctrl};
    const long long n_items =
        all_starts ? p.n_starts
                   : (long long)min(*((volatile unsigned*)&ctrl->q_count), (unsigned)q.cap);
    for (;;) {
        __syncthreads();
        if (tid == 0) sh.item = (int)atomicAdd(&ctrl->q_head, 1u);
        __syncthreads();
        const long long item = sh.item;
        if (item >= n_items) break;
        if (all_starts) {
            wide_run<OBJ, GRAD, T>(p, W, item, 0, 0, nullptr, nullptr, io, sh, smem_raw, tid);
        } else {
            const long long s = q.start[item];
            const T* Hq = reinterpret_cast<const T*>(q.H) + (size_t)item * p.dim * p.dim;
            const T* xq = reinterpret_cast<const T*>(x_out + s * p.dim);
            wide_run<OBJ, GRAD, T>(p, W, s, q.k[item], q.feval[item], Hq, xq, io, sh, smem_raw,
                                   tid);
        }
    }
}

// One warp per start: four starts to a 128-thread block, each warp pulling
// the next start for itself; the body is the block kernel's on 32 threads.
template <int OBJ, int GRAD, class T>
__global__ void __launch_bounds__(kWideThreads)
    bfgs_warp_kernel(const zeus_problem p, const int W, const int slot, const double* x0,
                     double* x_out, double* __restrict__ f_out, double* __restrict__ gnorm_out,
                     int32_t* __restrict__ status_out, int32_t* __restrict__ iters_out,
                     Ctrl* __restrict__ ctrl) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ WideShared shw[kWideThreads / 32];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const RunIO io{x0, x_out, f_out, gnorm_out, status_out, iters_out, ctrl};
    unsigned char* mine = smem_raw + (size_t)w * slot;
    for (;;) {
        unsigned item = 0;
        if (lane == 0) item = atomicAdd(&ctrl->q_head, 1u);
        item = __shfl_sync(0xffffffffu, item, 0);
        if ((long long)item >= p.n_starts) break;
        wide_run<OBJ, GRAD, T, 32>(p, W, (long long)item, 0, 0, nullptr, nullptr, io, shw[w], mine,
                                   lane);
    }
}

// Narrow and wide in one cooperative launch.  Every block first takes lane
// tiles (tile starts, one lane each, with the hand-over budget); once no
// tile is left it serves the hand-over queue, so the starts handed over
// early run on blocks that have no tile while the tiles are still in
// progress.  Servers poll for entries while a tile may still produce one;
// the launch is cooperative, so every block is resident and the polls
// end.  Each poll loop is bounded by `spin_limit` polls of about 256 ns
// (zeus_set_wait_limit; then the error word is set and the block stops
// serving).

__device__ __forceinline__ int smid_of() {
    unsigned r;
    asm volatile("mov.u32 %0, %%smid;" : "=r"(r));
    return (int)r;
}

// waits (bounded) until entry `slot` is marked written
__device__ __forceinline__ bool wait_ready(const Queue& q, int slot, Ctrl* ctrl,
                                           unsigned spin_limit) {
    volatile int* rd = q.ready + slot;
    for (unsigned spin = 0; !*rd; ++spin) {
        if (spin >= spin_limit) {
            atomicExch(&ctrl->error, 1);
            return false;
        }
        __nanosleep(256);
    }
    return true;
}

// Takes the next entry of the region [base, base + cap_r) counted by
// *count if a producer has claimed it (it is then written shortly: waits
// for its flag); -1 if there is none now.  Never waits for production.
__device__ __forceinline__ int claim_now(unsigned* head, unsigned* count, int base, int cap_r,
                                         const Queue& q, Ctrl* ctrl, unsigned spin_limit) {
    for (;;) {
        const unsigned h = *((volatile unsigned*)head);
        const unsigned c = min(*((volatile unsigned*)count), (unsigned)cap_r);
        if (h >= c) return -1;
        if (atomicCAS(head, h, h + 1) == h)
            return wait_ready(q, base + (int)h, ctrl, spin_limit) ? base + (int)h : -1;
    }
}

// region exhausted: every entry a producer claimed has been taken
__device__ __forceinline__ bool drained(const unsigned* head, const unsigned* count, int cap_r) {
    return *((volatile const unsigned*)head) >= min(*((volatile const unsigned*)count), (unsigned)cap_r);
}

template <int OBJ, int GRAD, class T>
__global__ void __launch_bounds__(kWideThreads)
    bfgs_fused_kernel(const zeus_problem p, const int stride, const int budget, const int tile,
                      const int n_tiles, const int W, const double* x0, double* x_out,
                      double* __restrict__ f_out, double* __restrict__ gnorm_out,
                      int32_t* __restrict__ status_out, int32_t* __restrict__ iters_out,
                      Ctrl* __restrict__ ctrl, const Queue q, const unsigned spin_limit) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ WideShared sh;
    const int tid = wide_role(blockDim.x);
    const RunIO io{x0, x_out, f_out, gnorm_out, status_out, iters_out, ctrl};
    T* smem = reinterpret_cast<T*>(smem_raw);
    for (;;) {  // lane tiles
        __syncthreads();
        if (threadIdx.x == 0) sh.item = (int)atomicAdd(&ctrl->tile_head, 1u);
        __syncthreads();
        const int t = sh.item;
        if (t >= n_tiles) break;
        const long long s = (long long)t * tile + threadIdx.x;
        if ((int)threadIdx.x < tile && s < p.n_starts)
            narrow_run<OBJ, GRAD, T>(p, s, smem + (size_t)threadIdx.x * stride, budget, io, ctrl, q,
                                     0);
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            atomicAdd(&ctrl->tiles_done, 1u);
        }
    }
    // the hand-over queue.  Servers poll both regions and take only
    // entries already claimed by a producer; an SM serves at most one long
    // entry at a time until the tiles are done, so long runs spread over
    // the SMs.  Every poll loop is bounded.
    const int sm = smid_of();
    const int ncap = q.cap - q.long_cap, lbase = q.cap - q.long_cap;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) {
            int item = -1, held = 0;
            for (unsigned spin = 0;; ++spin) {
                if (q.long_cap > 0 && sm < kMaxSMs && atomicCAS(q.sm_long + sm, 0, 1) == 0) {
                    item = claim_now(&ctrl->q_head_long, &ctrl->q_count_long, lbase, q.long_cap, q,
                                     ctrl, spin_limit);
                    if (item >= 0) {
                        held = 1;
                        break;
                    }
                    atomicExch(q.sm_long + sm, 0);
                }
                item = claim_now(&ctrl->q_head, &ctrl->q_count, 0, ncap, q, ctrl, spin_limit);
                if (item >= 0) break;
                if (*((volatile unsigned*)&ctrl->tiles_done) >= (unsigned)n_tiles) {
                    __threadfence();  // the counts are final now
                    if (q.long_cap > 0) {
                        item = claim_now(&ctrl->q_head_long, &ctrl->q_count_long, lbase, q.long_cap,
                                         q, ctrl, spin_limit);
                        if (item >= 0) break;
                    }
                    if (drained(&ctrl->q_head, &ctrl->q_count, ncap) &&
                        (q.long_cap == 0 ||
                         drained(&ctrl->q_head_long, &ctrl->q_count_long, q.long_cap)))
                        break;
                }
                if (spin >= spin_limit) {
                    atomicExch(&ctrl->error, 1);
                    break;
                }
                __nanosleep(256);
            }
            sh.item = item;
            sh.status = held;
        }
        __syncthreads();
        const int item = sh.item;
        if (item < 0) break;
        __threadfence();
        const long long s = __ldcg(q.start + item);
        const T* Hq = reinterpret_cast<const T*>(q.H) + (size_t)item * p.dim * p.dim;
        const T* xq = reinterpret_cast<const T*>(x_out + s * p.dim);
        const int held = sh.status;
        wide_run<OBJ, GRAD, T>(p, W, s, __ldcg(q.k + item), __ldcg(q.feval + item), Hq, xq, io, sh,
                               smem_raw, tid, true);
        if (threadIdx.x == 0 && held) atomicExch(q.sm_long + sm, 0);
    }
}

// Cooperative fused launch of the narrow and wide kernels, if the device
// offers cooperative launches; returns cudaErrorNotSupported otherwise.
template <int OBJ, int GRAD, class T>
static cudaError_t fused_go(const zeus_problem& p, const BfgsLaunch& L, const double* x0,
                            double* x_out, double* f_out, double* gnorm_out, int32_t* status_out,
                            int32_t* iters_out, Ctrl* ctrl, const Queue& q, cudaStream_t st) {
    int dev = 0, coop = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    if (!coop) return cudaErrorNotSupported;
    // tiles of 32..128 lanes: as many as keep a block within 56 KB of shared
    // memory (four blocks per SM), at least one warp
    const size_t row = (size_t)L.stride * sizeof(T);
    int tile = (int)((56u << 10) / row) / 32 * 32;
    if (tile > kWideThreads) tile = kWideThreads;
    if (tile < 32) tile = 32;
    const size_t smem = (size_t)tile * row > L.wide_smem ? (size_t)tile * row : L.wide_smem;
    auto kf = bfgs_fused_kernel<OBJ, GRAD, T>;
    e = allow_smem(kf, smem);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kf, kWideThreads, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorNotSupported;
    zeus_problem pp = p;
    int stride = L.stride, budget = L.budget, W = L.W;
    int n_tiles = (int)((p.n_starts + tile - 1) / tile);
    const double* xin = x0;
    double *xo = x_out, *fo = f_out, *go = gnorm_out;
    int32_t *so = status_out, *io = iters_out;
    Ctrl* c = ctrl;
    Queue qq = q;
    // long entries: half of the queue (and the per-SM table)
    qq.long_cap = (q.sm_long && sms <= kMaxSMs) ? q.cap / 2 : 0;
    unsigned spin_limit = wait_limit();
    void* args[] = {&pp,  &stride, &budget, &tile, &n_tiles, &W, &xin, &xo,
                    &fo,  &go,     &so,     &io,   &c,       &qq, &spin_limit};
    return cudaLaunchCooperativeKernel((const void*)kf, dim3(sms * per_sm), dim3(kWideThreads), args,
                                       smem, st);
}

template <int OBJ, int GRAD, class T>
static cudaError_t bfgs_go(const zeus_problem& p, const BfgsLaunch& L, const double* x0,
                           double* x_out, double* f_out, double* gnorm_out, int32_t* status_out,
                           int32_t* iters_out, Ctrl* ctrl, const Queue& q, cudaStream_t st) {
    cudaError_t e;
    if (L.warp) {
        auto kw = bfgs_warp_kernel<OBJ, GRAD, T>;
        const size_t smem = 4 * L.warp_slot;
        int dev = 0, sms = 0, per_sm = 0;
        e = allow_smem(kw, smem);
        if (e == cudaSuccess) e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kw, kWideThreads, smem);
        if (e != cudaSuccess) return e;
        long long blocks = (long long)sms * (per_sm > 0 ? per_sm : 1);
        const long long need = (p.n_starts + 3) / 4;
        if (blocks > need) blocks = need;
        kw<<<(int)blocks, kWideThreads, smem, st>>>(p, L.W, (int)L.warp_slot, x0, x_out, f_out,
                                                    gnorm_out, status_out, iters_out, ctrl);
        return cudaGetLastError();
    }
    if (L.narrow && L.budget > 0 && q.ready) {
        e = fused_go<OBJ, GRAD, T>(p, L, x0, x_out, f_out, gnorm_out, status_out, iters_out, ctrl,
                                   q, st);
        if (e != cudaErrorNotSupported) return e;
        cudaGetLastError();  // not offered: the two launches below
    }
    if (L.narrow) {
        auto kn = bfgs_narrow_kernel<OBJ, GRAD, T>;
        e = allow_smem(kn, L.narrow_smem);
        if (e != cudaSuccess) return e;
        kn<<<L.narrow_blocks, L.narrow_threads, L.narrow_smem, st>>>(
            p, L.stride, L.budget, x0, x_out, f_out, gnorm_out, status_out, iters_out, ctrl, q);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        if (L.budget == 0) return cudaSuccess;
    }
    auto kw = bfgs_wide_kernel<OBJ, GRAD, T>;
    e = allow_smem(kw, L.wide_smem);
    if (e != cudaSuccess) return e;
    kw<<<L.wide_blocks, kWideThreads, L.wide_smem, st>>>(p, L.W, x0, x_out, f_out, gnorm_out,
                                                         status_out, iters_out, ctrl, q,
                                                         L.narrow ? 0 : 1);
    return cudaGetLastError();
}

template <int GRAD, class T>
cudaError_t bfgs_launch_gt(const zeus_problem& p, const BfgsLaunch& L, const double* x0,
                           double* x_out, double* f_out, double* gnorm_out, int32_t* status_out,
                           int32_t* iters_out, Ctrl* ctrl, const Queue& q, cudaStream_t st) {
    if constexpr (GRAD == ZEUS_GRAD_FORWARD) {  // user objectives: forward mode only
        switch (p.objective) {
#define ZEUS_UCASE(O)                                                                       \
    case O:                                                                                 \
        return bfgs_go<O, GRAD, T>(p, L, x0, x_out, f_out, gnorm_out, status_out, iters_out, \
                                   ctrl, q, st);
            ZEUS_USER_EACH(ZEUS_UCASE)
#undef ZEUS_UCASE
            default:
                break;
        }
    }
    switch (p.objective) {
        case ZEUS_OBJ_ROSENBROCK:
            return bfgs_go<ZEUS_OBJ_ROSENBROCK, GRAD, T>(p, L, x0, x_out, f_out, gnorm_out,
                                                         status_out, iters_out, ctrl, q, st);
        case ZEUS_OBJ_RASTRIGIN:
            return bfgs_go<ZEUS_OBJ_RASTRIGIN, GRAD, T>(p, L, x0, x_out, f_out, gnorm_out,
                                                        status_out, iters_out, ctrl, q, st);
        case ZEUS_OBJ_ACKLEY:
            return bfgs_go<ZEUS_OBJ_ACKLEY, GRAD, T>(p, L, x0, x_out, f_out, gnorm_out,
                                                     status_out, iters_out, ctrl, q, st);
        case ZEUS_OBJ_GOLDSTEIN_PRICE:
            return bfgs_go<ZEUS_OBJ_GOLDSTEIN_PRICE, GRAD, T>(p, L, x0, x_out, f_out, gnorm_out,
                                                              status_out, iters_out, ctrl, q, st);
        default:
            return bfgs_go<ZEUS_OBJ_QUADRATIC, GRAD, T>(p, L, x0, x_out, f_out, gnorm_out,
                                                        status_out, iters_out, ctrl, q, st);
    }
}

#if ZEUS_KF32
template cudaError_t bfgs_launch_gt<ZEUS_KGRAD, float>(const zeus_problem&, const BfgsLaunch&,
                                                       const double*, double*, double*, double*,
                                                       int32_t*, int32_t*, Ctrl*, const Queue&,
                                                       cudaStream_t);
#else
template cudaError_t bfgs_launch_gt<ZEUS_KGRAD, double>(const zeus_problem&, const BfgsLaunch&,
                                                        const double*, double*, double*, double*,
                                                        int32_t*, int32_t*, Ctrl*, const Queue&,
                                                        cudaStream_t);
#endif

}  // namespace zeus
