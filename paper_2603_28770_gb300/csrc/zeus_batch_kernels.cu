// zeus_batch_kernels.cu -- the batched BFGS kernel of zeus_batch.cu for one
// (gradient mode, precision) pair, chosen at compile time by ZEUS_KGRAD
// (0 forward, 1 adjoint) and ZEUS_KF32 (0 FP64, 1 FP32 with FP64 guards):
// the library compiles this file once per pair, in parallel.
#include "zeus_bfgs.cuh"

#if !defined(ZEUS_KGRAD) || !defined(ZEUS_KF32)
#error "compile with -DZEUS_KGRAD=0|1 -DZEUS_KF32=0|1"
#endif
// ZEUS_KUSER=1: the variant whose objective switch also holds the user
// objectives (forward mode only).  It is compiled apart so that the kernel
// of the built-in objectives keeps its own registers and compile time.
#ifndef ZEUS_KUSER
#define ZEUS_KUSER 0
#endif
#if ZEUS_KUSER && ZEUS_KGRAD
#error "user objectives have forward-mode gradients only"
#endif

namespace zeus {

template <int GRAD, class T, bool U>
__device__ __forceinline__ void batch_narrow(const zeus_problem& p, int P, long long s, T* slot,
                                             const BatchDev& bd, const RunIO& io) {
    const int b = bd.budget[P];
    Ctrl* qc = bd.gctrl;
    if constexpr (U && GRAD == ZEUS_GRAD_FORWARD) {  // user objectives: forward mode only
        switch (p.objective) {
#define ZEUS_UCASE(O)                                                \
    case O:                                                          \
        narrow_run<O, GRAD, T>(p, s, slot, b, io, qc, bd.q, P);      \
        return;
            ZEUS_USER_EACH(ZEUS_UCASE)
#undef ZEUS_UCASE
            default:
                break;
        }
    }
    switch (p.objective) {
        case ZEUS_OBJ_ROSENBROCK:
            narrow_run<ZEUS_OBJ_ROSENBROCK, GRAD, T>(p, s, slot, b, io, qc, bd.q, P);
            break;
        case ZEUS_OBJ_RASTRIGIN:
            narrow_run<ZEUS_OBJ_RASTRIGIN, GRAD, T>(p, s, slot, b, io, qc, bd.q, P);
            break;
        case ZEUS_OBJ_ACKLEY:
            narrow_run<ZEUS_OBJ_ACKLEY, GRAD, T>(p, s, slot, b, io, qc, bd.q, P);
            break;
        case ZEUS_OBJ_GOLDSTEIN_PRICE:
            narrow_run<ZEUS_OBJ_GOLDSTEIN_PRICE, GRAD, T>(p, s, slot, b, io, qc, bd.q, P);
            break;
        default:
            narrow_run<ZEUS_OBJ_QUADRATIC, GRAD, T>(p, s, slot, b, io, qc, bd.q, P);
            break;
    }
}

template <int GRAD, class T, bool U, int NTW = kWideThreads>
__device__ __forceinline__ void batch_wide(const zeus_problem& p, int W, long long s, int k,
                                           int fe, const T* Hq, const T* xq, const RunIO& io,
                                           WideShared& sh, unsigned char* smem_raw, int tid) {
    if constexpr (U && GRAD == ZEUS_GRAD_FORWARD) {  // user objectives: forward mode only
        switch (p.objective) {
#define ZEUS_UCASE(O)                                                                  \
    case O:                                                                            \
        wide_run<O, GRAD, T, NTW>(p, W, s, k, fe, Hq, xq, io, sh, smem_raw, tid);      \
        return;
            ZEUS_USER_EACH(ZEUS_UCASE)
#undef ZEUS_UCASE
            default:
                break;
        }
    }
    switch (p.objective) {
        case ZEUS_OBJ_ROSENBROCK:
            wide_run<ZEUS_OBJ_ROSENBROCK, GRAD, T, NTW>(p, W, s, k, fe, Hq, xq, io, sh, smem_raw,
                                                        tid);
            break;
        case ZEUS_OBJ_RASTRIGIN:
            wide_run<ZEUS_OBJ_RASTRIGIN, GRAD, T, NTW>(p, W, s, k, fe, Hq, xq, io, sh, smem_raw,
                                                       tid);
            break;
        case ZEUS_OBJ_ACKLEY:
            wide_run<ZEUS_OBJ_ACKLEY, GRAD, T, NTW>(p, W, s, k, fe, Hq, xq, io, sh, smem_raw, tid);
            break;
        case ZEUS_OBJ_GOLDSTEIN_PRICE:
            wide_run<ZEUS_OBJ_GOLDSTEIN_PRICE, GRAD, T, NTW>(p, W, s, k, fe, Hq, xq, io, sh,
                                                             smem_raw, tid);
            break;
        default:
            wide_run<ZEUS_OBJ_QUADRATIC, GRAD, T, NTW>(p, W, s, k, fe, Hq, xq, io, sh, smem_raw,
                                                       tid);
            break;
    }
}

__device__ __forceinline__ RunIO batch_io(const BatchDev& bd, const zeus_problem& p, int P,
                                          double* x_out, double* f_out, double* gnorm_out,
                                          int32_t* status_out, int32_t* iters_out) {
    const long long xo = bd.xoff[P], so = bd.soff[P];
    const double* x0 = p.start_from_pbest ? bd.px + xo : x_out + xo;
    return RunIO{x0,
                 x_out + xo,
                 f_out + so,
                 gnorm_out ? gnorm_out + so : nullptr,
                 status_out ? status_out + so : nullptr,
                 iters_out ? iters_out + so : nullptr,
                 bd.pctrl + P};
}

// Persistent blocks over work items [first, first + count) (cls >= 0) or
// over the hand-over queue (cls < 0).  Item (P, s, c, 0): a tile of c
// starts s.. of problem P, one lane each; item (P, s, W, 1): start s on the
// whole block with W line-search trials at once; item (P, s, W, 2): start s
// on one warp (a class holds one kind of item; in a class of warp items
// each warp of a block pulls items for itself, its start's shared memory
// the warp's quarter of the block's).
// at least six blocks per SM: the lane-tile classes keep their residency
template <int GRAD, class T, bool U>
__global__ void __launch_bounds__(kWideThreads, 6)
    batch_bfgs_kernel(const BatchDev bd, const int cls, const int first, const int count,
                      const int smem_bytes, double* x_out, double* __restrict__ f_out,
                      double* __restrict__ gnorm_out, int32_t* __restrict__ status_out,
                      int32_t* __restrict__ iters_out) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ WideShared sh;
    (void)smem_bytes;
    const int tid = wide_role(blockDim.x);
    unsigned* head = cls >= 0 ? bd.heads + cls : &bd.gctrl->q_head;
    const int n_items =
        cls >= 0 ? count
                 : (int)min(*((volatile unsigned*)&bd.gctrl->q_count), (unsigned)bd.q.cap);
    for (;;) {
        __syncthreads();
        if (tid == 0) sh.item = (int)atomicAdd(head, 1u);
        __syncthreads();
        const int item = sh.item;
        if (item >= n_items) break;
        if (cls >= 0) {
            const int4 w = bd.items[first + item];
            const int P = w.x;
            const zeus_problem p = bd.probs[P];
            const RunIO io = batch_io(bd, p, P, x_out, f_out, gnorm_out, status_out, iters_out);
            if (w.w == 0) {
                if ((int)threadIdx.x < w.z) {
                    T* slot = reinterpret_cast<T*>(smem_raw) + (size_t)threadIdx.x * bd.stride[P];
                    batch_narrow<GRAD, T, U>(p, P, (long long)w.y + threadIdx.x, slot, bd, io);
                }
            } else {
                batch_wide<GRAD, T, U>(p, w.z, w.y, 0, 0, nullptr, nullptr, io, sh, smem_raw, tid);
            }
        } else {
            const int P = bd.q.prob[item];
            const zeus_problem p = bd.probs[P];
            const RunIO io = batch_io(bd, p, P, x_out, f_out, gnorm_out, status_out, iters_out);
            const long long s = bd.q.start[item];
            const T* Hq = reinterpret_cast<const T*>(bd.q.H) + (size_t)item * bd.q.hstride;
            const T* xq = reinterpret_cast<const T*>(io.x_out + s * p.dim);
            batch_wide<GRAD, T, U>(p, wide_trials(p.dim, p.ls_max_iters), s, bd.q.k[item],
                                bd.q.feval[item], Hq, xq, io, sh, smem_raw, tid);
        }
    }
}

// A class of warp items (P, s, W, 2): each warp of a block pulls items for
// itself; its start's shared memory is the warp's quarter of the block's.
template <int GRAD, class T, bool U>
__global__ void __launch_bounds__(kWideThreads, 5)
    batch_warp_kernel(const BatchDev bd, const int cls, const int first, const int count,
                      const int smem_bytes, double* x_out, double* __restrict__ f_out,
                      double* __restrict__ gnorm_out, int32_t* __restrict__ status_out,
                      int32_t* __restrict__ iters_out) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ WideShared shw[kWideThreads / 32];
    unsigned* head = bd.heads + cls;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const size_t slot = ((size_t)smem_bytes / 4) & ~size_t(15);
    unsigned char* mine = smem_raw + (size_t)w * slot;
    for (;;) {
        unsigned it = 0;
        if (lane == 0) it = atomicAdd(head, 1u);
        it = __shfl_sync(0xffffffffu, it, 0);
        if ((int)it >= count) break;
        const int4 wi = bd.items[first + (int)it];
        const int P = wi.x;
        const zeus_problem p = bd.probs[P];
        const RunIO io = batch_io(bd, p, P, x_out, f_out, gnorm_out, status_out, iters_out);
        batch_wide<GRAD, T, U, 32>(p, wi.z, wi.y, 0, 0, nullptr, nullptr, io, shw[w], mine, lane);
    }
}

template <int GRAD, class T, bool U>
cudaError_t batch_launch_gt(const BatchDev& bd, int cls, int first, int count, size_t smem,
                            bool warp_items, double* x_out, double* f_out, double* gnorm_out,
                            int32_t* status_out, int32_t* iters_out, cudaStream_t st) {
    auto k = warp_items ? batch_warp_kernel<GRAD, T, U> : batch_bfgs_kernel<GRAD, T, U>;
    // The launches of one solve use different shared memory sizes, and a
    // captured graph launches its kernel nodes later: allow the largest
    // size the device offers once, rather than the size of the launch at
    // hand (which a later launch would lower again).
    int dev = 0, sms = 0, per_sm = 0, optin = 0;
    cudaFuncAttributes fa;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, k);
    if (e != cudaSuccess) return e;
    const int maxdyn = optin - (int)fa.sharedSizeBytes;
    if ((long long)smem > (long long)maxdyn) return cudaErrorInvalidValue;
    e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, maxdyn);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kWideThreads, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    long long blocks = (long long)sms * per_sm;
    const long long holders = (cls >= 0 && warp_items) ? (count + 3) / 4 : count;
    if (cls >= 0 && blocks > holders) blocks = holders;  // no block without an item
    if (cls < 0 && blocks > bd.q.cap) blocks = bd.q.cap;
    if (blocks < 1) return cudaSuccess;
    k<<<(int)blocks, kWideThreads, smem, st>>>(bd, cls, first, count, (int)smem, x_out, f_out,
                                                gnorm_out, status_out, iters_out);
    return cudaGetLastError();
}

#if ZEUS_KF32
template cudaError_t batch_launch_gt<ZEUS_KGRAD, float, ZEUS_KUSER != 0>(
    const BatchDev&, int, int, int, size_t, bool, double*, double*, double*, int32_t*, int32_t*,
    cudaStream_t);
#else
template cudaError_t batch_launch_gt<ZEUS_KGRAD, double, ZEUS_KUSER != 0>(
    const BatchDev&, int, int, int, size_t, bool, double*, double*, double*, int32_t*, int32_t*,
    cudaStream_t);
#endif

}  // namespace zeus
