// zeus_bfgs.cu -- one BFGS run per start (Alg. 4, per-thread body of
// Alg. 10), FP64.
//
// A group of G lanes (G = 1..32, one warp at most) owns one start.  The
// start's state lives in shared memory, one contiguous slot per start:
//     H [d*d] (row-major, symmetric) | x [d] | g [d] | p [d] | xn [d] | gn [d]
// (for large d, H instead lives in the workspace, one d*d block per start).
// Lane l owns vector elements and H rows j = l, l+G, ...; it runs the
// forward-mode passes i = l, l+G, ... (Alg. 5), so every vector step reads
// and writes its own elements and the group synchronises only where a lane
// reads all of a vector (objective, matrix-vector product, rank-two update).
//
// Per iteration (readings of the paper are listed in the design notes):
//   ||g|| < tol -> converged; p = -H g (reset H = I, p = -g if not a descent
//   direction); backtracking Armijo line search (Alg. 6); x_new = x + a p;
//   (f, g) at x_new; y = g_new - g, s = x_new - x; if y's > 1e-12 |s||y|:
//   H <- H - rho (Hy s' + s Hy') + (rho^2 y'Hy + rho) s s'  (the expanded form
//   of the product update printed in Alg. 4).
#include "zeus_device.cuh"
#include "zeus_internal.h"

namespace zeus {

constexpr int kBfgsMaxThreads = 256;

template <int OBJ>
__device__ __forceinline__ double grp_value(const double* x, int d, const Group& grp) {
    Part<double> q = value_partial<OBJ, double, double>(x, d, grp.lane, grp.G);
    q.s0 = grp.sum(q.s0);
    if (OBJ == ZEUS_OBJ_ACKLEY) q.s1 = grp.sum(q.s1);
    return value_finish<OBJ, double>(q, d);
}

// f and g at x; g[j] written for the lane's own j (except Goldstein-Price's
// adjoint, written by lane 0).  Returns f on every lane.
template <int OBJ, int GRAD>
__device__ __forceinline__ double grp_gradient(const double* x, double* g, int d,
                                               const Group& grp) {
    if (GRAD == ZEUS_GRAD_FORWARD) {
        double f = 0.0;
        for (int i = grp.lane; i < d; i += grp.G) {
            const Dual<double> r = forward_pass<OBJ, double>(x, d, i);
            g[i] = r.b;
            if (i == 0) f = r.a;  // value part of the first pass
        }
        return grp.bcast(f);
    } else {
        return adjoint<OBJ, double>(x, d, g, grp);
    }
}

template <int OBJ, int GRAD, bool HG>
__global__ void __launch_bounds__(kBfgsMaxThreads)
    bfgs_kernel(const zeus_problem p, const int G, const int S, const int stride,
                const double* x0, double* x_out,  // may alias (in-place run)
                double* __restrict__ f_out, double* __restrict__ gnorm_out,
                int32_t* __restrict__ status_out, int32_t* __restrict__ iters_out,
                double* __restrict__ h_ws, Ctrl* __restrict__ ctrl) {
    extern __shared__ double smem[];
    const Group grp(G);
    const int lane = grp.lane;
    const int slot = threadIdx.x / G;
    const long long s = (long long)blockIdx.x * S + slot;
    if (s >= p.n_starts) return;  // whole groups leave together
    const int d = p.dim;
    double* base = smem + (size_t)slot * stride;
    double* H = HG ? h_ws + (size_t)s * d * d : base;
    double* x = HG ? base : base + (size_t)d * d;
    double* g = x + d;
    double* pv = g + d;
    double* xn = pv + d;
    double* gn = xn + d;

    const bool use_target = !isnan(p.target_f);
    const bool use_stop = use_target || p.required_converged > 0;
    const double tol = p.grad_tol, cA = p.armijo_c, beta = p.backtrack;
    const int K = p.bfgs_max_iters, L = p.ls_max_iters;

    for (int j = lane; j < d; j += G) x[j] = x0[s * d + j];
    for (int r = lane; r < d; r += G) {
        double* Hr = H + (size_t)r * d;
        for (int c = 0; c < d; ++c) Hr[c] = (c == r) ? 1.0 : 0.0;
    }
    grp.sync();
    double f0 = grp_gradient<OBJ, GRAD>(x, g, d, grp);
    grp.sync();

    int k = 0, status = ZEUS_RUN_MAX_ITER, feval = 0;
    double gnorm;
    for (;;) {
        double gg = 0.0;
        int bad = 0;
        for (int j = lane; j < d; j += G) {
            const double gj = g[j];
            gg += gj * gj;
            bad |= !isfinite(gj);
        }
        gg = grp.sum(gg);
        bad = grp.sum(bad);
        gnorm = sqrt(gg);
        if (k >= K) {
            status = ZEUS_RUN_MAX_ITER;
            break;
        }
        if (use_stop) {
            int stop = 0;
            if (lane == 0) stop = *((volatile int*)&ctrl->stop);
            if (grp.bcast(stop)) {
                status = ZEUS_RUN_STOPPED;
                break;
            }
        }
        if (!isfinite(f0) || bad) {
            status = ZEUS_RUN_NONFINITE;
            break;
        }
        if (gnorm < tol) {
            status = ZEUS_RUN_CONVERGED;
            if (use_stop && lane == 0) {
                const unsigned long long c = atomicAdd(&ctrl->n_conv, 1ull) + 1ull;
                if (p.required_converged > 0 && c >= (unsigned long long)p.required_converged)
                    atomicExch(&ctrl->stop, 1);
            }
            break;
        }
        if (use_target && f0 <= p.target_f) {
            status = ZEUS_RUN_CONVERGED;
            if (lane == 0) {
                atomicAdd(&ctrl->n_conv, 1ull);
                atomicExch(&ctrl->stop, 1);
            }
            break;
        }
        // direction p = -H g and ddir = g'p
        double ddir = 0.0;
        for (int r = lane; r < d; r += G) {
            const double* Hr = H + (size_t)r * d;
            double a = 0.0;
            for (int c = 0; c < d; ++c) a += Hr[c] * g[c];
            pv[r] = -a;
            ddir += g[r] * (-a);
        }
        ddir = grp.sum(ddir);
        if (!(ddir < 0.0)) {  // not a descent direction: restart from H = I
            double dd = 0.0;
            for (int r = lane; r < d; r += G) {
                double* Hr = H + (size_t)r * d;
                for (int c = 0; c < d; ++c) Hr[c] = (c == r) ? 1.0 : 0.0;
                pv[r] = -g[r];
                dd += g[r] * pv[r];
            }
            ddir = grp.sum(dd);
        }
        // backtracking Armijo line search (Alg. 6)
        double alpha = 1.0;
        bool accepted = false;
        for (int m = 0; m < L; ++m) {
            for (int j = lane; j < d; j += G) xn[j] = x[j] + alpha * pv[j];
            grp.sync();
            const double ft = grp_value<OBJ>(xn, d, grp);
            ++feval;
            if (ft <= f0 + cA * alpha * ddir) {
                accepted = true;
                break;
            }
            alpha = beta * alpha;
            grp.sync();
        }
        if (!accepted)
            for (int j = lane; j < d; j += G) xn[j] = x[j] + alpha * pv[j];
        grp.sync();
        const double fn = grp_gradient<OBJ, GRAD>(xn, gn, d, grp);
        grp.sync();
        // curvature pair
        double sy = 0.0, ss = 0.0, yy = 0.0;
        for (int j = lane; j < d; j += G) {
            const double sj = xn[j] - x[j], yj = gn[j] - g[j];
            sy += yj * sj;
            ss += sj * sj;
            yy += yj * yj;
        }
        sy = grp.sum(sy);
        ss = grp.sum(ss);
        yy = grp.sum(yy);
        if (sy > 1e-12 * sqrt(ss) * sqrt(yy)) {
            const double rho = 1.0 / sy;
            double yhy = 0.0;
            for (int r = lane; r < d; r += G) {  // Hy into pv (the direction is spent)
                const double* Hr = H + (size_t)r * d;
                double a = 0.0;
                for (int c = 0; c < d; ++c) a += Hr[c] * (gn[c] - g[c]);
                pv[r] = a;
                yhy += (gn[r] - g[r]) * a;
            }
            yhy = grp.sum(yhy);
            grp.sync();
            const double b2 = rho * rho * yhy + rho;
            for (int r = lane; r < d; r += G) {
                double* Hr = H + (size_t)r * d;
                const double sr = xn[r] - x[r], hr = pv[r];
                for (int c = 0; c < d; ++c) {
                    const double sc = xn[c] - x[c];
                    Hr[c] = Hr[c] - rho * (hr * sc + sr * pv[c]) + b2 * (sr * sc);
                }
            }
        }
        grp.sync();
        for (int j = lane; j < d; j += G) {
            x[j] = xn[j];
            g[j] = gn[j];
        }
        f0 = fn;
        ++k;
        grp.sync();
    }

    for (int j = lane; j < d; j += G) x_out[s * d + j] = x[j];
    if (lane == 0) {
        if (f_out) f_out[s] = f0;
        if (gnorm_out) gnorm_out[s] = gnorm;
        if (status_out) status_out[s] = status;
        if (iters_out) iters_out[s] = k;
        atomicAdd(&ctrl->total_iters, (unsigned long long)k);
        atomicAdd(&ctrl->total_feval, (unsigned long long)feval);
        if (!use_stop && status == ZEUS_RUN_CONVERGED) atomicAdd(&ctrl->n_conv, 1ull);
    }
}

// ---------------------------------------------------------------------------
// Launch planning
// ---------------------------------------------------------------------------
int lanes_for_dim(int d, int requested) {
    if (requested > 0) return requested;
    if (d <= 8) return 1;
    if (d <= 16) return 2;
    if (d <= 32) return 4;
    if (d <= 64) return 8;
    if (d <= 128) return 16;
    return 32;
}

int plan_bfgs(const zeus_problem& p, BfgsLaunch* L) {
    const int d = p.dim;
    L->G = lanes_for_dim(d, p.threads_per_start);
    const size_t smem_cap = 227 * 1024;
    // words per start, odd so that lane-per-start slots fall in distinct banks
    int stride = d * d + 5 * d;
    if ((stride & 1) == 0) stride += 1;
    L->h_global = false;
    if ((size_t)stride * sizeof(double) > smem_cap / 2) {
        L->h_global = true;
        stride = 5 * d;
        if ((stride & 1) == 0) stride += 1;
    }
    int S = kBfgsMaxThreads / L->G;
    const int fit = (int)(smem_cap / ((size_t)stride * sizeof(double)));
    if (fit < S) S = fit;
    if (S < 1) return ZEUS_EUNSUPPORTED;
    L->S = S;
    L->stride = stride;
    L->smem = (size_t)S * stride * sizeof(double);
    L->blocks = (int)((p.n_starts + S - 1) / S);
    return ZEUS_OK;
}

template <int OBJ, int GRAD, bool HG>
static cudaError_t bfgs_go(const zeus_problem& p, const BfgsLaunch& L, const double* x0,
                           double* x_out, double* f_out, double* gnorm_out, int32_t* status_out,
                           int32_t* iters_out, double* h_ws, Ctrl* ctrl, cudaStream_t st) {
    auto kern = bfgs_kernel<OBJ, GRAD, HG>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)L.smem);
    if (e != cudaSuccess) return e;
    kern<<<L.blocks, L.S * L.G, L.smem, st>>>(p, L.G, L.S, L.stride, x0, x_out, f_out, gnorm_out,
                                              status_out, iters_out, h_ws, ctrl);
    return cudaGetLastError();
}

template <int OBJ>
static cudaError_t bfgs_obj(const zeus_problem& p, const BfgsLaunch& L, const double* x0,
                            double* x_out, double* f_out, double* gnorm_out, int32_t* status_out,
                            int32_t* iters_out, double* h_ws, Ctrl* ctrl, cudaStream_t st) {
    if (p.grad_mode == ZEUS_GRAD_ADJOINT) {
        return L.h_global ? bfgs_go<OBJ, ZEUS_GRAD_ADJOINT, true>(p, L, x0, x_out, f_out, gnorm_out,
                                                                  status_out, iters_out, h_ws,
                                                                  ctrl, st)
                          : bfgs_go<OBJ, ZEUS_GRAD_ADJOINT, false>(
                                p, L, x0, x_out, f_out, gnorm_out, status_out, iters_out, h_ws,
                                ctrl, st);
    }
    return L.h_global ? bfgs_go<OBJ, ZEUS_GRAD_FORWARD, true>(p, L, x0, x_out, f_out, gnorm_out,
                                                              status_out, iters_out, h_ws, ctrl,
                                                              st)
                      : bfgs_go<OBJ, ZEUS_GRAD_FORWARD, false>(p, L, x0, x_out, f_out, gnorm_out,
                                                               status_out, iters_out, h_ws, ctrl,
                                                               st);
}

cudaError_t launch_bfgs(const zeus_problem& p, const BfgsLaunch& L, const double* x0,
                        double* x_out, double* f_out, double* gnorm_out, int32_t* status_out,
                        int32_t* iters_out, double* h_ws, Ctrl* ctrl, cudaStream_t st) {
    switch (p.objective) {
        case ZEUS_OBJ_ROSENBROCK:
            return bfgs_obj<ZEUS_OBJ_ROSENBROCK>(p, L, x0, x_out, f_out, gnorm_out, status_out,
                                                 iters_out, h_ws, ctrl, st);
        case ZEUS_OBJ_RASTRIGIN:
            return bfgs_obj<ZEUS_OBJ_RASTRIGIN>(p, L, x0, x_out, f_out, gnorm_out, status_out,
                                                iters_out, h_ws, ctrl, st);
        case ZEUS_OBJ_ACKLEY:
            return bfgs_obj<ZEUS_OBJ_ACKLEY>(p, L, x0, x_out, f_out, gnorm_out, status_out,
                                             iters_out, h_ws, ctrl, st);
        case ZEUS_OBJ_GOLDSTEIN_PRICE:
            return bfgs_obj<ZEUS_OBJ_GOLDSTEIN_PRICE>(p, L, x0, x_out, f_out, gnorm_out,
                                                      status_out, iters_out, h_ws, ctrl, st);
        default:
            return bfgs_obj<ZEUS_OBJ_QUADRATIC>(p, L, x0, x_out, f_out, gnorm_out, status_out,
                                                iters_out, h_ws, ctrl, st);
    }
}

}  // namespace zeus
