// zeus_cluster.cu -- clustering of the final points of a multistart run
// (Section VI proposes it: group the candidate solutions by function value
// or by coordinates, and weigh the region of the lowest f by how many
// starts reached it).
//
// Leader clustering in the order of increasing (f, start index), done in
// rounds over the whole grid: round k takes the lowest open candidate as
// leader k and closes every open candidate within tol of it.  A candidate
// that a round does not close is farther than tol from that round's
// leader, so it joins the first leader (in creation order) it is within
// tol of, and the leaders are exactly those of the sequential definition
// in zeus.h.
//
// Layout of the work: start i belongs to one thread for the whole kernel
// (i = global thread id + m * grid threads), so its label is only read and
// written by that thread.  A round is: block argmins of the open
// candidates into this round's half of a double buffer, one grid barrier,
// every block reduces the partials to the same leader, then closes its
// candidates.  The next round writes the other half, and its barrier is
// reached only after every block has read this round's half, so one
// barrier per round suffices.  The launch is cooperative (every block
// resident); each barrier wait is bounded.
#include <math.h>
#include <math_constants.h>
#include <stdint.h>

#include "zeus.h"
#include "zeus_internal.h"

namespace zeus {

constexpr int kClusterThreads = 256;
constexpr int kClusterMaxBlocks = 1024;
constexpr int kOpen = -3;                      // a candidate not yet in a cluster


struct ClusterPart {
    double f;
    int i;
    int pad;
};

// device workspace (zeroed before the launch)
struct ClusterWork {
    unsigned bar_count, bar_gen;
    int error, pad;
    unsigned long long n_cand, n_left, spread0_bits;
    ClusterPart part[2][kClusterMaxBlocks];
    // then int leader[max_clusters], int count[max_clusters]
};

size_t cluster_work_bytes(int max_clusters) {
    return align256(sizeof(ClusterWork) + 2 * sizeof(int) * (size_t)max_clusters);
}

struct ClusterShared {
    double wf[32];
    int wi[32];
    long long wn[32];
    double wd[32];
    int L;
};

__device__ __forceinline__ bool key_less(double fa, int ia, double fb, int ib) {
    return ia >= 0 && (ib < 0 || fa < fb || (fa == fb && ia < ib));
}

// lowest (f, i) over the block, into every thread; (inf, -1) if none
__device__ __forceinline__ void block_argmin(double& f, int& i, ClusterShared& sh) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int o = 16; o > 0; o >>= 1) {
        const double of = __shfl_down_sync(0xffffffffu, f, o);
        const int oi = __shfl_down_sync(0xffffffffu, i, o);
        if (key_less(of, oi, f, i)) {
            f = of;
            i = oi;
        }
    }
    if (lane == 0) {
        sh.wf[warp] = f;
        sh.wi[warp] = i;
    }
    __syncthreads();
    if (warp == 0) {
        const int nw = blockDim.x >> 5;
        f = lane < nw ? sh.wf[lane] : INFINITY;
        i = lane < nw ? sh.wi[lane] : -1;
        for (int o = 16; o > 0; o >>= 1) {
            const double of = __shfl_down_sync(0xffffffffu, f, o);
            const int oi = __shfl_down_sync(0xffffffffu, i, o);
            if (key_less(of, oi, f, i)) {
                f = of;
                i = oi;
            }
        }
        if (lane == 0) {
            sh.wf[0] = f;
            sh.L = i;
        }
    }
    __syncthreads();
    f = sh.wf[0];
    i = sh.L;
    __syncthreads();  // wf, wi are reused by the next reduction
}

// block sum of a count and block maximum of a distance (both exact), into
// every thread
__device__ __forceinline__ void block_count_max(long long& c, double& m, ClusterShared& sh) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int o = 16; o > 0; o >>= 1) {
        c += __shfl_down_sync(0xffffffffu, c, o);
        m = fmax(m, __shfl_down_sync(0xffffffffu, m, o));
    }
    if (lane == 0) {
        sh.wn[warp] = c;
        sh.wd[warp] = m;
    }
    __syncthreads();
    if (warp == 0) {
        const int nw = blockDim.x >> 5;
        c = lane < nw ? sh.wn[lane] : 0;
        m = lane < nw ? sh.wd[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) {
            c += __shfl_down_sync(0xffffffffu, c, o);
            m = fmax(m, __shfl_down_sync(0xffffffffu, m, o));
        }
        if (lane == 0) {
            sh.wn[0] = c;
            sh.wd[0] = m;
        }
    }
    __syncthreads();
    c = sh.wn[0];
    m = sh.wd[0];
    __syncthreads();
}

// Grid barrier over the resident blocks of a cooperative launch: the last
// block to arrive resets the count and advances the generation; the others
// poll the generation (bounded: on timeout the error word is set).  Returns
// false once the error word is set.
__device__ __forceinline__ bool grid_barrier(ClusterWork* w, unsigned nblocks, unsigned spin_limit) {
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned* gen = &w->bar_gen;
        const unsigned g = *gen;  // read before arriving: it cannot advance before that
        __threadfence();
        if (atomicAdd(&w->bar_count, 1u) == nblocks - 1) {
            atomicExch(&w->bar_count, 0u);
            __threadfence();
            atomicAdd(&w->bar_gen, 1u);
        } else {
            for (unsigned spin = 0; *gen == g; ++spin) {
                if (spin >= spin_limit || *((volatile int*)&w->error)) {
                    atomicExch(&w->error, 1);
                    break;
                }
                __nanosleep(256);
            }
        }
        __threadfence();
    }
    __syncthreads();
    return *((volatile int*)&w->error) == 0;
}

__global__ void __launch_bounds__(kClusterThreads)
    cluster_kernel(const zeus_cluster_params cp, const int n, const int d,
                   const double* __restrict__ x, const double* __restrict__ f,
                   const int32_t* __restrict__ status, int32_t* __restrict__ label,
                   int32_t* __restrict__ leader_out, int32_t* __restrict__ count_out,
                   zeus_cluster_result* __restrict__ res, ClusterWork* __restrict__ w,
                   const unsigned spin_limit) {
    __shared__ ClusterShared sh;
    int* leader = reinterpret_cast<int*>(w + 1);
    int* count = leader + cp.max_clusters;
    const unsigned G = gridDim.x;
    const int NT = blockDim.x;
    const long long stride = (long long)G * NT;
    const long long gtid = (long long)blockIdx.x * NT + threadIdx.x;
    const bool by_x = cp.method == ZEUS_CLUSTER_BY_X;
    const double tol = cp.tol, tol2 = cp.tol * cp.tol;

    long long nc = 0;
    for (long long i = gtid; i < n; i += stride) {
        const bool c = isfinite(f[i]) && (!cp.only_converged || status[i] == ZEUS_RUN_CONVERGED);
        label[i] = c ? kOpen : ZEUS_LABEL_NONE;
        nc += c ? 1 : 0;
    }
    double unused = 0.0;
    block_count_max(nc, unused, sh);
    if (threadIdx.x == 0 && nc) atomicAdd(&w->n_cand, (unsigned long long)nc);

    int K = 0;
    bool ok = true;
    for (int k = 0; k < cp.max_clusters; ++k) {
        double bf = INFINITY;
        int bi = -1;
        for (long long i = gtid; i < n; i += stride) {
            if (label[i] != kOpen) continue;
            const double fi = f[i];
            if (bi < 0 || fi < bf) {  // i grows: ties keep the lower index
                bf = fi;
                bi = (int)i;
            }
        }
        block_argmin(bf, bi, sh);
        ClusterPart* part = w->part[k & 1];
        if (threadIdx.x == 0) {
            part[blockIdx.x].f = bf;
            part[blockIdx.x].i = bi;
        }
        ok = grid_barrier(w, G, spin_limit);
        if (!ok) break;
        bf = INFINITY;
        bi = -1;
        for (unsigned b = threadIdx.x; b < G; b += NT) {
            const double pf = __ldcg(&part[b].f);
            const int pi = __ldcg(&part[b].i);
            if (key_less(pf, pi, bf, bi)) {
                bf = pf;
                bi = pi;
            }
        }
        block_argmin(bf, bi, sh);
        const int L = bi;
        if (L < 0) break;  // every block sees the same partials
        const double fL = f[L];
        const double* xL = by_x ? x + (size_t)L * d : nullptr;
        long long cnt = 0;
        double sp = 0.0;
        for (long long i = gtid; i < n; i += stride) {
            if (label[i] != kOpen) continue;
            double dist;
            bool in;
            if (by_x) {
                // the partial sums only grow (each term is a square added
                // with one rounding), so a sum past tol^2 settles the test
                const double* xi = x + (size_t)i * d;
                double acc = 0.0;
                in = true;
                for (int j = 0; j < d; ++j) {
                    const double del = xi[j] - xL[j];
                    acc = fma(del, del, acc);
                    if (acc > tol2) {
                        in = false;
                        break;
                    }
                }
                dist = in ? sqrt(acc) : 0.0;
            } else {
                dist = fabs(f[i] - fL);
                in = dist <= tol * fmax(1.0, fabs(fL));
            }
            if (in) {
                label[i] = k;
                ++cnt;
                sp = fmax(sp, dist);
            }
        }
        block_count_max(cnt, sp, sh);
        if (threadIdx.x == 0) {
            if (cnt) atomicAdd(&count[k], (int)cnt);
            if (k == 0 && cnt) atomicMax(&w->spread0_bits, (unsigned long long)__double_as_longlong(sp));
            if (blockIdx.x == 0) leader[k] = L;
        }
        K = k + 1;
    }
    long long left = 0;
    for (long long i = gtid; i < n; i += stride) {
        if (label[i] == kOpen) {
            label[i] = ZEUS_LABEL_LEFT;
            ++left;
        }
    }
    block_count_max(left, unused, sh);
    if (threadIdx.x == 0 && left) atomicAdd(&w->n_left, (unsigned long long)left);
    if (ok) ok = grid_barrier(w, G, spin_limit);
    if (blockIdx.x != 0) return;
    // block 0 formed every leader entry; the counts are complete after the
    // barrier (read past L1)
    for (int k = threadIdx.x; k < cp.max_clusters; k += NT) {
        const bool formed = k < K;
        if (leader_out) leader_out[k] = formed ? leader[k] : -1;
        if (count_out) count_out[k] = formed ? __ldcg(&count[k]) : 0;
    }
    if (threadIdx.x == 0 && res) {
        zeus_cluster_result r;
        r.n_candidates = (long long)__ldcg(&w->n_cand);
        r.n_clusters = K;
        r.n_left = (long long)__ldcg(&w->n_left);
        r.best_count = K > 0 ? __ldcg(&count[0]) : 0;
        r.best_leader = K > 0 ? leader[0] : -1;
        r.best_f = K > 0 ? f[leader[0]] : CUDART_NAN;
        r.best_spread = K > 0 ? __longlong_as_double((long long)__ldcg(&w->spread0_bits)) : CUDART_NAN;
        r.error = ok ? 0 : 1;
        r.pad = 0;
        *res = r;
    }
}

// Every problem of a batch: block P (grid-stride over the problems) runs
// the rounds of problem P's starts with block barriers only; start i of the
// problem belongs to thread i mod blockDim for the whole problem.
constexpr int kBatchClusterThreads = 256;

__global__ void __launch_bounds__(kBatchClusterThreads)
    batch_cluster_kernel(const zeus_cluster_params cp, const BatchDev bd,
                         const double* __restrict__ x_all, const double* __restrict__ f_all,
                         const int32_t* __restrict__ st_all, int32_t* __restrict__ lab_all,
                         int32_t* __restrict__ leader_all, int32_t* __restrict__ count_all,
                         zeus_cluster_result* __restrict__ res_all) {
    __shared__ ClusterShared sh;
    const int tid = threadIdx.x, NT = blockDim.x;
    const bool by_x = cp.method == ZEUS_CLUSTER_BY_X;
    const double tol = cp.tol, tol2 = cp.tol * cp.tol;
    const int mc = cp.max_clusters;
    for (int P = blockIdx.x; P < bd.n; P += gridDim.x) {
        const zeus_problem& pr = bd.probs[P];
        const int n = (int)pr.n_starts, d = pr.dim;
        const double* x = x_all + bd.xoff[P];
        const double* f = f_all + bd.soff[P];
        const int32_t* status = st_all ? st_all + bd.soff[P] : nullptr;
        int32_t* label = lab_all + bd.soff[P];
        int32_t* leader = leader_all ? leader_all + (size_t)P * mc : nullptr;
        int32_t* count = count_all ? count_all + (size_t)P * mc : nullptr;

        long long nc = 0;
        for (int i = tid; i < n; i += NT) {
            const bool c =
                isfinite(f[i]) && (!cp.only_converged || status[i] == ZEUS_RUN_CONVERGED);
            label[i] = c ? kOpen : ZEUS_LABEL_NONE;
            nc += c ? 1 : 0;
        }
        double unused = 0.0;
        block_count_max(nc, unused, sh);
        int K = 0, L0 = -1;
        long long c0 = 0;
        double spread0 = 0.0;
        for (int k = 0; k < mc; ++k) {
            double bf = INFINITY;
            int bi = -1;
            for (int i = tid; i < n; i += NT) {
                if (label[i] != kOpen) continue;
                const double fi = f[i];
                if (bi < 0 || fi < bf) {  // i grows: ties keep the lower index
                    bf = fi;
                    bi = i;
                }
            }
            block_argmin(bf, bi, sh);
            const int L = bi;
            if (L < 0) break;
            const double fL = f[L];
            const double* xL = by_x ? x + (size_t)L * d : nullptr;
            long long cnt = 0;
            double sp = 0.0;
            for (int i = tid; i < n; i += NT) {
                if (label[i] != kOpen) continue;
                double dist;
                bool in;
                if (by_x) {  // partial sums only grow: past tol^2 settles the test
                    const double* xi = x + (size_t)i * d;
                    double acc = 0.0;
                    in = true;
                    for (int j = 0; j < d; ++j) {
                        const double del = xi[j] - xL[j];
                        acc = fma(del, del, acc);
                        if (acc > tol2) {
                            in = false;
                            break;
                        }
                    }
                    dist = in ? sqrt(acc) : 0.0;
                } else {
                    dist = fabs(f[i] - fL);
                    in = dist <= tol * fmax(1.0, fabs(fL));
                }
                if (in) {
                    label[i] = k;
                    ++cnt;
                    sp = fmax(sp, dist);
                }
            }
            block_count_max(cnt, sp, sh);
            if (tid == 0) {
                if (leader) leader[k] = L;
                if (count) count[k] = (int)cnt;
            }
            if (k == 0) {
                L0 = L;
                c0 = cnt;
                spread0 = sp;
            }
            K = k + 1;
        }
        long long left = 0;
        for (int i = tid; i < n; i += NT) {
            if (label[i] == kOpen) {
                label[i] = ZEUS_LABEL_LEFT;
                ++left;
            }
        }
        block_count_max(left, unused, sh);
        for (int k = K + tid; k < mc; k += NT) {
            if (leader) leader[k] = -1;
            if (count) count[k] = 0;
        }
        if (tid == 0 && res_all) {
            zeus_cluster_result r;
            r.n_candidates = nc;
            r.n_clusters = K;
            r.n_left = left;
            r.best_count = K > 0 ? c0 : 0;
            r.best_leader = K > 0 ? L0 : -1;
            r.best_f = K > 0 ? f[L0] : CUDART_NAN;
            r.best_spread = K > 0 ? spread0 : CUDART_NAN;
            r.error = 0;
            r.pad = 0;
            res_all[P] = r;
        }
        __syncthreads();  // the next problem reuses the shared scratch
    }
}

cudaError_t launch_batch_cluster(const zeus_cluster_params& cp, const BatchDev& bd,
                                 const double* x, const double* f, const int32_t* status,
                                 int32_t* label, int32_t* leader_out, int32_t* count_out,
                                 zeus_cluster_result* res, cudaStream_t st) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_cluster_kernel,
                                                          kBatchClusterThreads, 0);
    if (e != cudaSuccess) return e;
    long long blocks = (long long)sms * (per_sm > 0 ? per_sm : 1);
    if (blocks > bd.n) blocks = bd.n;
    if (blocks < 1) return cudaSuccess;
    batch_cluster_kernel<<<(unsigned)blocks, kBatchClusterThreads, 0, st>>>(
        cp, bd, x, f, status, label, leader_out, count_out, res);
    return cudaGetLastError();
}

cudaError_t launch_cluster(const zeus_cluster_params& cp, int n, int d, const double* x,
                           const double* f, const int32_t* status, int32_t* label,
                           int32_t* leader_out, int32_t* count_out, zeus_cluster_result* res,
                           void* workspace, cudaStream_t st) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, cluster_kernel, kClusterThreads, 0);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    long long blocks = (long long)sms * per_sm;
    const long long need = ((long long)n + kClusterThreads - 1) / kClusterThreads;
    if (blocks > need) blocks = need;
    if (blocks > kClusterMaxBlocks) blocks = kClusterMaxBlocks;
    if (blocks < 1) blocks = 1;
    ClusterWork* w = static_cast<ClusterWork*>(workspace);
    e = cudaMemsetAsync(w, 0, cluster_work_bytes(cp.max_clusters), st);
    if (e != cudaSuccess) return e;
    zeus_cluster_params pp = cp;
    int nn = n, dd = d;
    unsigned spin_limit = wait_limit();
    void* args[] = {&pp, &nn, &dd, &x, &f, &status, &label, &leader_out, &count_out, &res, &w,
                    &spin_limit};
    return cudaLaunchCooperativeKernel((const void*)cluster_kernel, dim3((unsigned)blocks),
                                       dim3(kClusterThreads), args, 0, st);
}

}  // namespace zeus
