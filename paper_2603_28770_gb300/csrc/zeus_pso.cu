// zeus_pso.cu -- PSO phase (Alg. 2 / Alg. 8 initialisation, Alg. 3 / Alg. 9
// update) with a synchronous, deterministic global best, the best-of-swarm
// argmin of Alg. 7, and the Philox draw kernel used by the RNG parity tests.
//
// One group of G lanes per particle; lanes split the dimensions in Philox
// blocks of four (one block = four draws).  Each PSO launch ends with a
// fused grid argmin over the personal bests (threadfence reduction): the
// last block to finish writes gbest and copies gX, so the next update reads
// the global best of the previous iteration (synchronous PSO) and no
// floating-point atomics are needed.
#include "zeus_device.cuh"
#include "zeus_internal.h"
#include "zeus_reduce.cuh"

namespace zeus {

constexpr int kPsoThreads = 128;

template <int OBJ>
__device__ __forceinline__ double group_value(const double* x, int d, const Group& grp) {
    Part<double> p = value_partial<OBJ, double, double>(x, d, grp.lane, grp.G);
    p.s0 = grp.sum(p.s0);
    if (OBJ == ZEUS_OBJ_ACKLEY) p.s1 = grp.sum(p.s1);
    return value_finish<OBJ, double>(p, d);
}

// One block of PSO particles (Alg. 2 for t < 0, Alg. 3 update number t
// otherwise): `block` of `nblocks` blocks of this problem; the last block of
// the problem to finish reduces the personal bests to the global best.
template <int OBJ>
__device__ __forceinline__ void pso_block(const zeus_problem& p, const int t, const int G,
                                          const int block, const int nblocks, double* x,
                                          double* v, double* px, double* pf, double* gx,
                                          Ctrl* ctrl, ArgPair* partials, zeus_result* res) {
    __shared__ ArgPair scratch[32];
    __shared__ int s_last;
    const Group grp(G);
    const int d = p.dim;
    const int S = kPsoThreads / G;
    const long long i = (long long)block * S + threadIdx.x / G;
    double fbest = CUDART_INF;
    long long ibest = 0x7fffffffffffffffll;
    if (i < p.n_starts) {
        double* xi = x + i * d;
        double* vi = v + i * d;
        double* pi = px + i * d;
        const int nblk = (d + 3) >> 2;
        if (t < 0) {
            const double lo = p.lower, hi = p.upper;
            const double vhi = hi - lo, vlo = -vhi;  // Alg. 2: velocities in [-range, range)
            for (int b = grp.lane; b < nblk; b += G) {
                const U64x4 rx = philox4x64_10(b, i, 0, 0, p.seed, 0);
                const U64x4 rv = philox4x64_10(b, i, 0, 1, p.seed, 0);
#pragma unroll
                for (int w = 0; w < 4; ++w) {
                    const int j = 4 * b + w;
                    if (j < d) {
                        const double xj = lo + (hi - lo) * u01(rx.v[w]);
                        xi[j] = xj;
                        pi[j] = xj;
                        vi[j] = vlo + (vhi - vlo) * u01(rv.v[w]);
                    }
                }
            }
        } else {
            const double w_ = p.w, c1 = p.c1, c2 = p.c2;
            for (int b = grp.lane; b < nblk; b += G) {
                const U64x4 r1 = philox4x64_10(b, i, 0, 2 + 2 * (uint64_t)t, p.seed, 0);
                const U64x4 r2 = philox4x64_10(b, i, 0, 3 + 2 * (uint64_t)t, p.seed, 0);
#pragma unroll
                for (int w = 0; w < 4; ++w) {
                    const int j = 4 * b + w;
                    if (j < d) {
                        const double xj = xi[j];
                        const double vn = w_ * vi[j] + (c1 * u01(r1.v[w])) * (pi[j] - xj) +
                                          (c2 * u01(r2.v[w])) * (gx[j] - xj);
                        vi[j] = vn;
                        xi[j] = xj + vn;
                    }
                }
            }
        }
        grp.sync();
        const double f = group_value<OBJ>(xi, d, grp);
        if (t < 0) {
            if (grp.lane == 0) pf[i] = f;
            fbest = f;
        } else {
            const double old = pf[i];
            grp.sync();
            if (f < old) {  // strict: Alg. 3 personal-best test
                if (grp.lane == 0) pf[i] = f;
                for (int j = grp.lane; j < d; j += G) pi[j] = xi[j];
                fbest = f;
            } else {
                fbest = old;
            }
        }
        fbest = nan_to_inf(fbest);
        ibest = i;
    }
    block_argmin(fbest, ibest, scratch);
    if (publish_and_check_last(fbest, ibest, partials, ctrl, &s_last, block, nblocks)) {
        double bf;
        long long bi;
        reduce_partials(partials, bf, bi, scratch, nblocks);
        if (threadIdx.x == 0) {
            scratch[0].f = bf;
            scratch[0].idx = bi;
            ctrl->gbest_f = bf;
            ctrl->gbest_idx = bi;
            if (res) {
                res->gbest_f = bf;
                res->gbest_index = bi;
            }
            ctrl->blocks_done = 0;
        }
        __syncthreads();
        const long long b = scratch[0].idx;
        for (int j = threadIdx.x; j < d; j += blockDim.x) gx[j] = __ldcg(px + b * d + j);
    }
}

// t < 0: initialisation (Alg. 2); t >= 0: PSO update number t (Alg. 3).
template <int OBJ>
__global__ void __launch_bounds__(kPsoThreads)
    pso_kernel(const zeus_problem p, const int t, const int G, double* __restrict__ x,
               double* __restrict__ v, double* __restrict__ px, double* __restrict__ pf,
               double* __restrict__ gx, Ctrl* __restrict__ ctrl, ArgPair* __restrict__ partials,
               zeus_result* __restrict__ res) {
    pso_block<OBJ>(p, t, G, blockIdx.x, gridDim.x, x, v, px, pf, gx, ctrl, partials, res);
}

// Batched PSO: each block belongs to one problem of the batch.
__global__ void __launch_bounds__(kPsoThreads)
    batch_pso_kernel(const BatchDev bd, const int t, double* __restrict__ x_out) {
    const int P = bd.pso_table[blockIdx.x];
    const zeus_problem p = bd.probs[P];
    if (t >= p.pso_iters) return;  // this problem has made all its updates
    const int lb = blockIdx.x - bd.pblk0[P];
    double* x = x_out + bd.xoff[P];
    double* v = bd.v + bd.xoff[P];
    double* px = bd.px + bd.xoff[P];
    double* pf = bd.pf + bd.soff[P];
    double* gx = bd.gx + bd.goff[P];
    ArgPair* parts = bd.partials + bd.poff[P];
    Ctrl* ctrl = bd.pctrl + P;
    const int G = bd.plane[P], nb = bd.pblk[P];
    switch (p.objective) {
#define ZEUS_UCASE(O)                                                                 \
    case O:                                                                           \
        pso_block<O>(p, t, G, lb, nb, x, v, px, pf, gx, ctrl, parts, nullptr);        \
        break;
        ZEUS_USER_EACH(ZEUS_UCASE)
#undef ZEUS_UCASE
        case ZEUS_OBJ_ROSENBROCK:
            pso_block<ZEUS_OBJ_ROSENBROCK>(p, t, G, lb, nb, x, v, px, pf, gx, ctrl, parts, nullptr);
            break;
        case ZEUS_OBJ_RASTRIGIN:
            pso_block<ZEUS_OBJ_RASTRIGIN>(p, t, G, lb, nb, x, v, px, pf, gx, ctrl, parts, nullptr);
            break;
        case ZEUS_OBJ_ACKLEY:
            pso_block<ZEUS_OBJ_ACKLEY>(p, t, G, lb, nb, x, v, px, pf, gx, ctrl, parts, nullptr);
            break;
        case ZEUS_OBJ_GOLDSTEIN_PRICE:
            pso_block<ZEUS_OBJ_GOLDSTEIN_PRICE>(p, t, G, lb, nb, x, v, px, pf, gx, ctrl, parts,
                                                nullptr);
            break;
        default:
            pso_block<ZEUS_OBJ_QUADRATIC>(p, t, G, lb, nb, x, v, px, pf, gx, ctrl, parts, nullptr);
            break;
    }
}

cudaError_t launch_batch_pso(const BatchDev& bd, int t, double* x_out, cudaStream_t st) {
    batch_pso_kernel<<<bd.pso_blocks, kPsoThreads, 0, st>>>(bd, t, x_out);
    return cudaGetLastError();
}

int pso_blocks(const zeus_problem& p, int G) {
    const long long S = kPsoThreads / G;
    return (int)((p.n_starts + S - 1) / S);
}

template <int OBJ>
static cudaError_t pso_run(const zeus_problem& p, int G, double* x, double* v, double* px,
                           double* pf, double* gx, Ctrl* ctrl, ArgPair* partials,
                           zeus_result* res, cudaStream_t st) {
    const int blocks = pso_blocks(p, G);
    for (int t = -1; t < p.pso_iters; ++t) {
        pso_kernel<OBJ><<<blocks, kPsoThreads, 0, st>>>(p, t, G, x, v, px, pf, gx, ctrl, partials,
                                                        res);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_pso(const zeus_problem& p, int G, double* x, double* v, double* px, double* pf,
                       double* gx, Ctrl* ctrl, ArgPair* partials, zeus_result* res,
                       cudaStream_t st) {
    switch (p.objective) {
#define ZEUS_UCASE(O) \
    case O:           \
        return pso_run<O>(p, G, x, v, px, pf, gx, ctrl, partials, res, st);
        ZEUS_USER_EACH(ZEUS_UCASE)
#undef ZEUS_UCASE
        case ZEUS_OBJ_ROSENBROCK:
            return pso_run<ZEUS_OBJ_ROSENBROCK>(p, G, x, v, px, pf, gx, ctrl, partials, res, st);
        case ZEUS_OBJ_RASTRIGIN:
            return pso_run<ZEUS_OBJ_RASTRIGIN>(p, G, x, v, px, pf, gx, ctrl, partials, res, st);
        case ZEUS_OBJ_ACKLEY:
            return pso_run<ZEUS_OBJ_ACKLEY>(p, G, x, v, px, pf, gx, ctrl, partials, res, st);
        case ZEUS_OBJ_GOLDSTEIN_PRICE:
            return pso_run<ZEUS_OBJ_GOLDSTEIN_PRICE>(p, G, x, v, px, pf, gx, ctrl, partials, res,
                                                     st);
        default:
            return pso_run<ZEUS_OBJ_QUADRATIC>(p, G, x, v, px, pf, gx, ctrl, partials, res, st);
    }
}

// ---------------------------------------------------------------------------
// Best-of-swarm argmin over f[n] (Alg. 7), grid-stride, fused grid finish.
// mode 0: argmin only (counters zeroed, gbest NaN / -1); 1: also copy the
// BFGS counters of the control block and keep the PSO gbest already in res;
// 2: counters, gbest NaN / -1 (BFGS from given starts).
// ---------------------------------------------------------------------------
constexpr int kArgminThreads = 256;

__global__ void __launch_bounds__(kArgminThreads)
    argmin_kernel(const double* __restrict__ f, const long long n, Ctrl* __restrict__ ctrl,
                  ArgPair* __restrict__ partials, zeus_result* __restrict__ res,
                  const int mode) {
    __shared__ ArgPair scratch[32];
    __shared__ int s_last;
    double bf = CUDART_INF;
    long long bi = 0x7fffffffffffffffll;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const double v = nan_to_inf(f[i]);
        if (better(v, i, bf, bi)) {
            bf = v;
            bi = i;
        }
    }
    block_argmin(bf, bi, scratch);
    if (publish_and_check_last(bf, bi, partials, ctrl, &s_last)) {
        reduce_partials(partials, bf, bi, scratch);
        if (threadIdx.x == 0) {
            if (res) {
                res->best_f = bf;
                res->best_index = bi;
                if (mode != 0) {
                    volatile Ctrl* c = ctrl;
                    res->n_converged = (int64_t)c->n_conv;
                    res->total_iters = (int64_t)c->total_iters;
                    res->total_feval = (int64_t)c->total_feval;
                    res->error = c->error;
                    res->stop_flag = c->stop;
                    res->h_reads = (int64_t)c->h_reads;
                    res->h_writes = (int64_t)c->h_writes;
                } else {
                    res->n_converged = 0;
                    res->total_iters = 0;
                    res->total_feval = 0;
                    res->error = 0;
                    res->stop_flag = 0;
                    res->h_reads = 0;
                    res->h_writes = 0;
                }
                if (mode != 1) {  // no PSO phase in this call
                    res->gbest_f = CUDART_NAN;
                    res->gbest_index = -1;
                }
            }
            ctrl->blocks_done = 0;
        }
    }
}

int argmin_blocks(long long n) {
    long long b = (n + kArgminThreads - 1) / kArgminThreads;
    if (b > 1216) b = 1216;  // 8 blocks per SM on 152 SMs
    if (b < 1) b = 1;
    return (int)b;
}

cudaError_t launch_argmin(const double* f, long long n, Ctrl* ctrl, ArgPair* partials,
                          zeus_result* res, int mode, cudaStream_t st) {
    argmin_kernel<<<argmin_blocks(n), kArgminThreads, 0, st>>>(f, n, ctrl, partials, res, mode);
    return cudaGetLastError();
}

// Batched best-of-swarm reduction: one block per problem.
__global__ void __launch_bounds__(kArgminThreads)
    batch_argmin_kernel(const BatchDev bd, const double* __restrict__ f, zeus_result* res) {
    __shared__ ArgPair scratch[32];
    const int P = blockIdx.x;
    const long long n = bd.probs[P].n_starts;
    const double* fp = f + bd.soff[P];
    double bf = CUDART_INF;
    long long bi = 0x7fffffffffffffffll;
    for (long long i = threadIdx.x; i < n; i += blockDim.x) {
        const double v = nan_to_inf(fp[i]);
        if (better(v, i, bf, bi)) {
            bf = v;
            bi = i;
        }
    }
    block_argmin(bf, bi, scratch);
    if (threadIdx.x == 0 && res) {
        volatile Ctrl* c = bd.pctrl + P;
        zeus_result* r = res + P;
        r->best_f = bf;
        r->best_index = bi;
        r->n_converged = (int64_t)c->n_conv;
        r->total_iters = (int64_t)c->total_iters;
        r->total_feval = (int64_t)c->total_feval;
        r->gbest_f = c->gbest_f;
        r->gbest_index = c->gbest_idx;
        r->error = c->error;
        r->stop_flag = c->stop;
        r->h_reads = (int64_t)c->h_reads;
        r->h_writes = (int64_t)c->h_writes;
    }
}

cudaError_t launch_batch_argmin(const BatchDev& bd, const double* f_out, zeus_result* res,
                                cudaStream_t st) {
    batch_argmin_kernel<<<bd.n, kArgminThreads, 0, st>>>(bd, f_out, res);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Philox draws for the RNG parity tests: out[i*d + j] = draw(phase, i, j).
// ---------------------------------------------------------------------------
__global__ void uniform_kernel(const uint64_t seed, const uint64_t problem, const uint64_t phase,
                               const long long n, const int d, double* __restrict__ out) {
    const int nblk = (d + 3) >> 2;
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (tid >= n * nblk) return;
    const long long i = tid / nblk;
    const int b = (int)(tid % nblk);
    const U64x4 r = philox4x64_10(b, i, problem, phase, seed, 0);
#pragma unroll
    for (int w = 0; w < 4; ++w) {
        const int j = 4 * b + w;
        if (j < d) out[i * d + j] = u01(r.v[w]);
    }
}

cudaError_t launch_uniform(uint64_t seed, uint64_t problem, uint64_t phase, long long n, int d,
                           double* out, cudaStream_t st) {
    const long long work = n * ((d + 3) / 4);
    if (work == 0) return cudaSuccess;
    const int threads = 256;
    const long long blocks = (work + threads - 1) / threads;
    uniform_kernel<<<(unsigned)blocks, threads, 0, st>>>(seed, problem, phase, n, d, out);
    return cudaGetLastError();
}

}  // namespace zeus
