// zeus_cluster.cu -- clustering of the final points of a multistart run
// (Section VI proposes it: group the candidate solutions by function value
// or by coordinates, and judge the region of the lowest f by how many
// starts reached it).
//
// Leader clustering in the order of increasing (f, start index), done in
// rounds by one block: round k takes the lowest open candidate as leader k
// and closes every open candidate within tol of it.  A candidate that some
// round does not close is at least tol away from that round's leader, so
// it joins the first leader (in creation order) it is within tol of, and
// the leaders are exactly those of the sequential definition in zeus.h.
// Every start index belongs to one thread for the whole kernel (i = tid +
// m * blockDim), so its label is only read and written by that thread.
#include <math.h>
#include <math_constants.h>
#include <stdint.h>

#include "zeus.h"
#include "zeus_internal.h"

namespace zeus {

constexpr int kClusterThreads = 1024;
constexpr int kOpen = -3;  // a candidate not yet in a cluster

struct ClusterShared {
    int leader[ZEUS_CLUSTER_MAX];
    int count[ZEUS_CLUSTER_MAX];
    double wf[32];
    int wi[32];
    double wd[32];
    long long wn[32];
    int L;
};

// lowest (f, i) over the block; (inf, -1) if no thread has one
__device__ __forceinline__ void block_argmin(double& f, int& i, ClusterShared& sh) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int o = 16; o > 0; o >>= 1) {
        const double of = __shfl_down_sync(0xffffffffu, f, o);
        const int oi = __shfl_down_sync(0xffffffffu, i, o);
        if (oi >= 0 && (i < 0 || of < f || (of == f && oi < i))) {
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
            if (oi >= 0 && (i < 0 || of < f || (of == f && oi < i))) {
                f = of;
                i = oi;
            }
        }
        if (lane == 0) sh.L = i;
    }
    __syncthreads();
    i = sh.L;
}

// block sum of a count and block maximum of a distance (both exact)
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
    __syncthreads();  // wn, wd are reused by the next reduction
}

__global__ void __launch_bounds__(kClusterThreads)
    cluster_kernel(const zeus_cluster_params cp, const int n, const int d,
                   const double* __restrict__ x, const double* __restrict__ f,
                   const int32_t* __restrict__ status, int32_t* __restrict__ label,
                   int32_t* __restrict__ leader_out, int32_t* __restrict__ count_out,
                   zeus_cluster_result* __restrict__ res) {
    __shared__ ClusterShared sh;
    const int tid = threadIdx.x, NT = blockDim.x;
    const bool by_x = cp.method == ZEUS_CLUSTER_BY_X;
    const double tol = cp.tol, tol2 = cp.tol * cp.tol;

    long long nc = 0;
    for (int i = tid; i < n; i += NT) {
        const bool c = isfinite(f[i]) && (!cp.only_converged || status[i] == ZEUS_RUN_CONVERGED);
        label[i] = c ? kOpen : ZEUS_LABEL_NONE;
        nc += c ? 1 : 0;
    }
    for (int k = tid; k < cp.max_clusters; k += NT) {
        sh.leader[k] = -1;
        sh.count[k] = 0;
    }
    double unused = 0.0;
    block_count_max(nc, unused, sh);

    int K = 0;
    double spread0 = 0.0;
    for (int k = 0; k < cp.max_clusters; ++k) {
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
            if (by_x) {
                const double* xi = x + (size_t)i * d;
                double acc = 0.0;
                for (int j = 0; j < d; ++j) {
                    const double del = xi[j] - xL[j];
                    acc = fma(del, del, acc);
                }
                in = acc <= tol2;
                dist = sqrt(acc);
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
            sh.leader[k] = L;
            sh.count[k] = (int)cnt;
        }
        if (k == 0) spread0 = sp;
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
    for (int k = tid; k < cp.max_clusters; k += NT) {
        if (leader_out) leader_out[k] = sh.leader[k];
        if (count_out) count_out[k] = sh.count[k];
    }
    if (tid == 0 && res) {
        zeus_cluster_result r;
        r.n_candidates = nc;
        r.n_clusters = K;
        r.n_left = left;
        r.best_count = K > 0 ? sh.count[0] : 0;
        r.best_leader = K > 0 ? sh.leader[0] : -1;
        r.best_f = K > 0 ? f[sh.leader[0]] : CUDART_NAN;
        r.best_spread = K > 0 ? spread0 : CUDART_NAN;
        r.error = 0;
        r.pad = 0;
        *res = r;
    }
}

cudaError_t launch_cluster(const zeus_cluster_params& cp, int n, int d, const double* x,
                           const double* f, const int32_t* status, int32_t* label,
                           int32_t* leader_out, int32_t* count_out, zeus_cluster_result* res,
                           cudaStream_t st) {
    cluster_kernel<<<1, kClusterThreads, 0, st>>>(cp, n, d, x, f, status, label, leader_out,
                                                  count_out, res);
    return cudaGetLastError();
}

}  // namespace zeus
