// zeus_bfgs.cu -- one BFGS run per start (Alg. 4, per-thread body of
// Alg. 10), FP64, in two kernels.
//
// GB300 runs FP64 at one warp instruction per 64 cycles per SM
// sub-partition whatever the number of active lanes, so FP64 throughput
// needs every lane busy, and the latency of one start is its FP64
// instruction count times 64 cycles.  Hence:
//
//  narrow kernel  one lane per start (the paper's thread-per-start layout),
//                 state in shared memory, the 32 lanes of a warp doing the
//                 same step of 32 different starts.  It carries most starts
//                 to the end.  With a work budget, a start that exceeds it
//                 (iterations + line-search evaluations) is handed over: its
//                 x, H, k and evaluation count go to a queue.
//  wide kernel    one CTA per start, persistent over a queue.  The d
//                 gradient components run on d threads, the line-search
//                 trials are evaluated speculatively in parallel (the first
//                 accepted trial is the one the sequential search accepts),
//                 the matrix work is split over the threads.  It finishes
//                 the long-running starts with low latency, and runs every
//                 start when d is too large for one lane per start.
//
// Both kernels perform exactly the oracle's operations in the oracle's
// order: sums run left to right (the wide kernel gathers the terms in
// shared memory and one thread adds them), no FMA contraction, the same
// elementary functions.  A run is therefore bitwise independent of which
// kernel carried it and of the hand-over point.
//
// Per iteration (readings of the paper are listed in the design notes):
//   ||g|| < tol -> converged; p = -H g (reset H = I, p = -g if not a descent
//   direction); backtracking Armijo line search (Alg. 6); x_new = x + a p;
//   g at x_new; y = g_new - g, s = x_new - x; if y's > 1e-12 |s||y|:
//   H <- H - rho (Hy s' + s Hy') + (rho^2 y'Hy + rho) s s'  (the expanded form
//   of the product update printed in Alg. 4).  The expanded form keeps H
//   exactly symmetric (IEEE products and sums commute), so the narrow
//   kernel computes the upper triangle and mirrors it.
#include "zeus_device.cuh"
#include "zeus_internal.h"

namespace zeus {

// ---------------------------------------------------------------------------
// Objective value sweep in index order: init, term j, finish.  Coordinates
// come through an accessor so the wide kernel can form a trial point
// x + a p on the fly (the same bits as the materialised point).
// ---------------------------------------------------------------------------
struct AtPoint {
    const double* x;
    __device__ __forceinline__ double operator()(int j) const { return x[j]; }
};
struct AtTrial {
    const double* x;
    const double* p;
    double a;
    __device__ __forceinline__ double operator()(int j) const { return x[j] + a * p[j]; }
};

template <int OBJ>
__device__ __forceinline__ Part<double> val_init(int d) {
    Part<double> a;
    a.s0 = (OBJ == ZEUS_OBJ_RASTRIGIN) ? 10.0 * (double)d : 0.0;
    a.s1 = 0.0;
    return a;
}

template <int OBJ>
__device__ __forceinline__ int val_nterms(int d) {
    if (OBJ == ZEUS_OBJ_ROSENBROCK) return d - 1;
    if (OBJ == ZEUS_OBJ_GOLDSTEIN_PRICE) return 1;
    return d;
}

template <int OBJ, class X>
__device__ __forceinline__ void val_term(const X& xa, int j, double& t0, double& t1) {
    t1 = 0.0;
    if (OBJ == ZEUS_OBJ_ROSENBROCK) {
        const double xj = xa(j);
        const double a = 1.0 - xj;
        const double b = xa(j + 1) - xj * xj;
        t0 = a * a + 100.0 * (b * b);
    } else if (OBJ == ZEUS_OBJ_RASTRIGIN) {
        const double xj = xa(j);
        t0 = xj * xj - 10.0 * c_2pi(xj);
    } else if (OBJ == ZEUS_OBJ_ACKLEY) {
        const double xj = xa(j);
        t0 = xj * xj;
        t1 = c_2pi(xj);
    } else if (OBJ == ZEUS_OBJ_GOLDSTEIN_PRICE) {
        const double x1 = xa(0), x2 = xa(1);
        const double t = (x1 + x2) + 1.0;
        const double pa =
            19.0 - 14.0 * x1 + 3.0 * (x1 * x1) - 14.0 * x2 + 6.0 * (x1 * x2) + 3.0 * (x2 * x2);
        const double a = 1.0 + (t * t) * pa;
        const double u = 2.0 * x1 - 3.0 * x2;
        const double pb =
            18.0 - 32.0 * x1 + 12.0 * (x1 * x1) + 48.0 * x2 - 36.0 * (x1 * x2) + 27.0 * (x2 * x2);
        const double b = 30.0 + (u * u) * pb;
        t0 = a * b;
    } else {
        const double xj = xa(j);
        t0 = (0.5 * (double)(j + 1)) * (xj * xj);
    }
}

template <int OBJ>
__device__ __forceinline__ void val_add(Part<double>& acc, double t0, double t1) {
    if (OBJ == ZEUS_OBJ_GOLDSTEIN_PRICE) {
        acc.s0 = t0;
    } else {
        acc.s0 = acc.s0 + t0;
        if (OBJ == ZEUS_OBJ_ACKLEY) acc.s1 = acc.s1 + t1;
    }
}

// f at a point on one thread, index order (equals the oracle's sweep)
template <int OBJ, class X>
__device__ __forceinline__ double seq_value(const X& xa, int d) {
    Part<double> acc = val_init<OBJ>(d);
    const int nt = val_nterms<OBJ>(d);
    for (int j = 0; j < nt; ++j) {
        double t0, t1;
        val_term<OBJ>(xa, j, t0, t1);
        val_add<OBJ>(acc, t0, t1);
    }
    return value_finish<OBJ, double>(acc, d);
}

// Gradient: forward pass i (Alg. 5) or adjoint component i.  The adjoint
// first forms the quantities shared by all components (Ackley's two sums,
// in index order) on one thread.
template <int OBJ, int GRAD>
__device__ __forceinline__ AdjShared grad_prep(const double* x, int d) {
    AdjShared a;
    a.c1 = a.c2 = 0.0;
    if (GRAD == ZEUS_GRAD_ADJOINT) a = adjoint_prep<OBJ>(x, d);
    return a;
}
template <int OBJ, int GRAD>
__device__ __forceinline__ double grad_component(const double* x, int d, int i,
                                                 const AdjShared& a) {
    if (GRAD == ZEUS_GRAD_FORWARD) return forward_pass<OBJ, double>(x, d, i).b;
    return adjoint_component<OBJ>(x, d, i, a);
}

// ---------------------------------------------------------------------------
// Narrow kernel: one lane per start.
// Shared memory per start (doubles): H [d*d] | x | g | p | xn | gn | s
// ---------------------------------------------------------------------------
template <int OBJ, int GRAD>
__global__ void __launch_bounds__(kNarrowThreads)
    bfgs_narrow_kernel(const zeus_problem p, const int stride, const int budget,
                       const double* x0, double* x_out,  // may alias (in-place run)
                       double* __restrict__ f_out, double* __restrict__ gnorm_out,
                       int32_t* __restrict__ status_out, int32_t* __restrict__ iters_out,
                       Ctrl* __restrict__ ctrl, const Queue q) {
    extern __shared__ double smem[];
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= p.n_starts) return;
    const int d = p.dim;
    double* H = smem + (size_t)threadIdx.x * stride;
    double* x = H + (size_t)d * d;
    double* g = x + d;
    double* pv = g + d;
    double* xn = pv + d;
    double* gn = xn + d;
    double* sv = gn + d;

    const bool use_target = !isnan(p.target_f);
    const bool use_stop = use_target || p.required_converged > 0;
    const double tol = p.grad_tol, cA = p.armijo_c, beta = p.backtrack;
    const int K = p.bfgs_max_iters, L = p.ls_max_iters;

    for (int j = 0; j < d; ++j) x[j] = x0[s * d + j];
    for (int r = 0; r < d; ++r)
        for (int c = 0; c < d; ++c) H[r * d + c] = (c == r) ? 1.0 : 0.0;
    {
        const AdjShared a = grad_prep<OBJ, GRAD>(x, d);
        for (int i = 0; i < d; ++i) g[i] = grad_component<OBJ, GRAD>(x, d, i, a);
    }
    double f0 = seq_value<OBJ>(AtPoint{x}, d);

    int k = 0, status = ZEUS_RUN_MAX_ITER, feval = 0;
    double gnorm;
    for (;;) {
        double gg = 0.0;
        bool bad = false;
        for (int j = 0; j < d; ++j) {
            gg = gg + g[j] * g[j];
            bad |= !isfinite(g[j]);
        }
        gnorm = sqrt(gg);
        if (k >= K) {
            status = ZEUS_RUN_MAX_ITER;
            break;
        }
        if (use_stop && *((volatile int*)&ctrl->stop)) {
            status = ZEUS_RUN_STOPPED;
            break;
        }
        if (!isfinite(f0) || bad) {
            status = ZEUS_RUN_NONFINITE;
            break;
        }
        if (gnorm < tol) {
            status = ZEUS_RUN_CONVERGED;
            if (use_stop) {
                const unsigned long long c = atomicAdd(&ctrl->n_conv, 1ull) + 1ull;
                if (p.required_converged > 0 && c >= (unsigned long long)p.required_converged)
                    atomicExch(&ctrl->stop, 1);
            }
            break;
        }
        if (use_target && f0 <= p.target_f) {
            status = ZEUS_RUN_CONVERGED;
            atomicAdd(&ctrl->n_conv, 1ull);
            atomicExch(&ctrl->stop, 1);
            break;
        }
        if (budget > 0 && k + feval >= budget) {
            // hand the start over to the wide kernel at the top of iteration k
            const unsigned slot = atomicAdd(&ctrl->q_count, 1u);
            if (slot < (unsigned)q.cap) {
                q.start[slot] = (int)s;
                q.k[slot] = k;
                q.feval[slot] = feval;
                double* Hq = q.H + (size_t)slot * d * d;
                for (int e = 0; e < d * d; ++e) Hq[e] = H[e];
                for (int j = 0; j < d; ++j) x_out[s * d + j] = x[j];
                return;
            }
        }
        // direction p = -H g and ddir = g'p
        for (int r = 0; r < d; ++r) {
            const double* Hr = H + r * d;
            double a = 0.0;
            for (int c = 0; c < d; ++c) a = a + Hr[c] * g[c];
            pv[r] = -a;
        }
        double ddir = 0.0;
        for (int r = 0; r < d; ++r) ddir = ddir + g[r] * pv[r];
        if (!(ddir < 0.0)) {  // not a descent direction: restart from H = I
            for (int r = 0; r < d; ++r)
                for (int c = 0; c < d; ++c) H[r * d + c] = (c == r) ? 1.0 : 0.0;
            for (int r = 0; r < d; ++r) pv[r] = -g[r];
            ddir = 0.0;
            for (int r = 0; r < d; ++r) ddir = ddir + g[r] * pv[r];
        }
        // backtracking Armijo line search (Alg. 6)
        double alpha = 1.0, fn = 0.0;
        bool accepted = false;
        for (int m = 0; m < L; ++m) {
            for (int j = 0; j < d; ++j) xn[j] = x[j] + alpha * pv[j];
            fn = seq_value<OBJ>(AtPoint{xn}, d);
            ++feval;
            if (fn <= f0 + cA * alpha * ddir) {
                accepted = true;
                break;
            }
            alpha = beta * alpha;
        }
        if (!accepted) {  // Alg. 6 returns the step after the last halving
            for (int j = 0; j < d; ++j) xn[j] = x[j] + alpha * pv[j];
            fn = seq_value<OBJ>(AtPoint{xn}, d);
        }
        {
            const AdjShared a = grad_prep<OBJ, GRAD>(xn, d);
            for (int i = 0; i < d; ++i) gn[i] = grad_component<OBJ, GRAD>(xn, d, i, a);
        }
        // curvature pair
        double sy = 0.0, ss = 0.0, yy = 0.0;
        for (int j = 0; j < d; ++j) {  // s into sv, y over g (g is not needed again)
            const double sj = xn[j] - x[j], yj = gn[j] - g[j];
            sv[j] = sj;
            g[j] = yj;
            sy = sy + yj * sj;
            ss = ss + sj * sj;
            yy = yy + yj * yj;
        }
        if (sy > 1e-12 * sqrt(ss) * sqrt(yy)) {
            const double rho = 1.0 / sy;
            for (int r = 0; r < d; ++r) {  // Hy into p (the direction is spent)
                const double* Hr = H + r * d;
                double a = 0.0;
                for (int c = 0; c < d; ++c) a = a + Hr[c] * g[c];
                pv[r] = a;
            }
            double yhy = 0.0;
            for (int r = 0; r < d; ++r) yhy = yhy + g[r] * pv[r];
            const double b2 = rho * rho * yhy + rho;
            for (int r = 0; r < d; ++r) {
                const double sr = sv[r], hr = pv[r];
                for (int c = r; c < d; ++c) {
                    const double sc = sv[c];
                    const double h = H[r * d + c] - rho * (hr * sc + sr * pv[c]) + b2 * (sr * sc);
                    H[r * d + c] = h;
                    H[c * d + r] = h;
                }
            }
        }
        for (int j = 0; j < d; ++j) {
            x[j] = xn[j];
            g[j] = gn[j];
        }
        f0 = fn;
        ++k;
    }

    for (int j = 0; j < d; ++j) x_out[s * d + j] = x[j];
    if (f_out) f_out[s] = f0;
    if (gnorm_out) gnorm_out[s] = gnorm;
    if (status_out) status_out[s] = status;
    if (iters_out) iters_out[s] = k;
    atomicAdd(&ctrl->total_iters, (unsigned long long)k);
    atomicAdd(&ctrl->total_feval, (unsigned long long)feval);
    if (!use_stop && status == ZEUS_RUN_CONVERGED) atomicAdd(&ctrl->n_conv, 1ull);
}

// ---------------------------------------------------------------------------
// Wide kernel: one CTA per start, persistent over a queue of starts.
// Shared memory (doubles): H [d*d] | x | g | p | xn | gn | s | scratch [3 d]
//   | trial terms [W][d] x 2 | trial f [W] | alpha [L+1]
// ---------------------------------------------------------------------------
struct WideShared {
    int item;
    int status;
    int accepted_m;
    int pad;
    double red[4];
    AdjShared adj;
    int ok[64];
};

// left-to-right sum of v[0..n) starting from init, on the calling thread
__device__ __forceinline__ double ordered_sum(const double* v, int n, double init) {
    double s = init;
    for (int j = 0; j < n; ++j) s = s + v[j];
    return s;
}

template <int OBJ, int GRAD>
__device__ __forceinline__ void wide_gradient(const double* x, double* g, int d, WideShared& sh) {
    const int tid = threadIdx.x, T = blockDim.x;
    if (GRAD == ZEUS_GRAD_ADJOINT) {
        if (tid == 0) sh.adj = adjoint_prep<OBJ>(x, d);
        __syncthreads();
    }
    const AdjShared a = sh.adj;
    for (int i = tid; i < d; i += T) g[i] = grad_component<OBJ, GRAD>(x, d, i, a);
}

template <int OBJ, int GRAD>
__global__ void __launch_bounds__(kWideThreads)
    bfgs_wide_kernel(const zeus_problem p, const int W, const double* x0, double* x_out,
                     double* __restrict__ f_out, double* __restrict__ gnorm_out,
                     int32_t* __restrict__ status_out, int32_t* __restrict__ iters_out,
                     Ctrl* __restrict__ ctrl, const Queue q, const int all_starts) {
    extern __shared__ double smem[];
    __shared__ WideShared sh;
    const int T = blockDim.x;
    // Roles rotate with the block index so that the thread doing the serial
    // work (ordered sums, tests) sits in a different warp, hence on a
    // different SM sub-partition, in each of the blocks sharing an SM.
    const int lead = (32 * (int)blockIdx.x) % T;
    const int tid = (threadIdx.x + T - lead) % T;
    const int d = p.dim;
    double* H = smem;
    double* x = H + (size_t)d * d;
    double* g = x + d;
    double* pv = g + d;
    double* xn = pv + d;
    double* gn = xn + d;
    double* sv = gn + d;
    double* sc0 = sv + d;  // three scratch vectors
    double* sc1 = sc0 + d;
    double* sc2 = sc1 + d;
    double* tb0 = sc2 + d;              // [W][d]
    double* tb1 = tb0 + (size_t)W * d;  // [W][d] (second sum of Ackley)
    double* fb = tb1 + (size_t)W * d;   // [W]
    double* al = fb + W;                // [L + 1]

    const bool use_target = !isnan(p.target_f);
    const bool use_stop = use_target || p.required_converged > 0;
    const double tol = p.grad_tol, cA = p.armijo_c, beta = p.backtrack;
    const int K = p.bfgs_max_iters, L = p.ls_max_iters;
    const int nt = val_nterms<OBJ>(d);

    if (tid == 0) {  // alpha_m = beta^m by repeated multiplication, as the sequential search
        double a = 1.0;
        for (int m = 0; m <= L; ++m) {
            al[m] = a;
            a = beta * a;
        }
        sh.adj.c1 = sh.adj.c2 = 0.0;
    }

    const long long n_items =
        all_starts ? p.n_starts
                   : (long long)min(*((volatile unsigned*)&ctrl->q_count), (unsigned)q.cap);
    for (;;) {
        __syncthreads();
        if (tid == 0) sh.item = (int)atomicAdd(&ctrl->q_head, 1u);
        __syncthreads();
        const long long item = sh.item;
        if (item >= n_items) break;
        const long long s = all_starts ? item : q.start[item];
        int k = all_starts ? 0 : q.k[item];
        int feval = all_starts ? 0 : q.feval[item];
        const double* xs = all_starts ? x0 + s * d : x_out + s * d;
        for (int j = tid; j < d; j += T) x[j] = xs[j];
        if (all_starts) {
            for (int e = tid; e < d * d; e += T) H[e] = (e / d == e % d) ? 1.0 : 0.0;
        } else {
            const double* Hq = q.H + (size_t)item * d * d;
            for (int e = tid; e < d * d; e += T) H[e] = Hq[e];
        }
        __syncthreads();
        wide_gradient<OBJ, GRAD>(x, g, d, sh);
        if (tid == 0) sh.red[0] = seq_value<OBJ>(AtPoint{x}, d);
        __syncthreads();
        double f0 = sh.red[0];
        int status = ZEUS_RUN_MAX_ITER;
        double gnorm = 0.0;
        for (;;) {
            // ---- tests at the top of iteration k
            int b = 0;
            for (int j = tid; j < d; j += T) {
                sc0[j] = g[j] * g[j];
                b |= !isfinite(g[j]);
            }
            const int bad = __syncthreads_or(b);
            if (tid == 0) {
                gnorm = sqrt(ordered_sum(sc0, d, 0.0));
                sh.red[1] = gnorm;
                int st = -1;
                if (k >= K) {
                    st = ZEUS_RUN_MAX_ITER;
                } else if (use_stop && *((volatile int*)&ctrl->stop)) {
                    st = ZEUS_RUN_STOPPED;
                } else if (!isfinite(f0) || bad) {
                    st = ZEUS_RUN_NONFINITE;
                } else if (gnorm < tol) {
                    st = ZEUS_RUN_CONVERGED;
                    if (use_stop) {
                        const unsigned long long c = atomicAdd(&ctrl->n_conv, 1ull) + 1ull;
                        if (p.required_converged > 0 &&
                            c >= (unsigned long long)p.required_converged)
                            atomicExch(&ctrl->stop, 1);
                    }
                } else if (use_target && f0 <= p.target_f) {
                    st = ZEUS_RUN_CONVERGED;
                    atomicAdd(&ctrl->n_conv, 1ull);
                    atomicExch(&ctrl->stop, 1);
                }
                sh.status = st;
            }
            __syncthreads();
            gnorm = sh.red[1];
            if (sh.status >= 0) {
                status = sh.status;
                break;
            }
            // ---- direction p = -H g (one row per thread, columns in order)
            for (int r = tid; r < d; r += T) {
                const double* Hr = H + r * d;
                double a = 0.0;
                for (int c = 0; c < d; ++c) a = a + Hr[c] * g[c];
                pv[r] = -a;
                sc0[r] = g[r] * (-a);
            }
            __syncthreads();
            if (tid == 0) sh.red[0] = ordered_sum(sc0, d, 0.0);
            __syncthreads();
            double ddir = sh.red[0];
            if (!(ddir < 0.0)) {  // not a descent direction: restart from H = I
                __syncthreads();
                for (int e = tid; e < d * d; e += T) H[e] = (e / d == e % d) ? 1.0 : 0.0;
                for (int r = tid; r < d; r += T) {
                    pv[r] = -g[r];
                    sc0[r] = g[r] * (-g[r]);
                }
                __syncthreads();
                if (tid == 0) sh.red[0] = ordered_sum(sc0, d, 0.0);
                __syncthreads();
                ddir = sh.red[0];
            }
            // ---- line search: W trials at a time, the first accepted wins
            int acc_m = -1;
            double fn = 0.0;
            for (int m0 = 0; m0 < L && acc_m < 0; m0 += W) {
                const int nw = min(W, L - m0);
                for (int e = tid; e < nw * nt; e += T) {
                    const int mm = e / nt, j = e - mm * nt;
                    double t0, t1;
                    val_term<OBJ>(AtTrial{x, pv, al[m0 + mm]}, j, t0, t1);
                    tb0[mm * d + j] = t0;
                    tb1[mm * d + j] = t1;
                }
                __syncthreads();
                if (tid < nw) {  // one thread per trial: its terms in order, then the test
                    Part<double> acc = val_init<OBJ>(d);
                    for (int j = 0; j < nt; ++j)
                        val_add<OBJ>(acc, tb0[tid * d + j], tb1[tid * d + j]);
                    const double ft = value_finish<OBJ, double>(acc, d);
                    fb[tid] = ft;
                    sh.ok[tid] = (ft <= f0 + cA * al[m0 + tid] * ddir) ? 1 : 0;
                }
                __syncthreads();
                if (tid == 0) {
                    int am = -1;
                    for (int mm = 0; mm < nw; ++mm)
                        if (sh.ok[mm]) {
                            am = m0 + mm;
                            break;
                        }
                    sh.accepted_m = am;
                    if (am >= 0) sh.red[2] = fb[am - m0];
                }
                __syncthreads();
                acc_m = sh.accepted_m;
                feval += (acc_m >= 0) ? (acc_m - m0 + 1) : nw;
            }
            const double alpha = (acc_m >= 0) ? al[acc_m] : al[L];
            for (int j = tid; j < d; j += T) xn[j] = x[j] + alpha * pv[j];
            __syncthreads();
            if (acc_m < 0 && tid == 0) sh.red[2] = seq_value<OBJ>(AtPoint{xn}, d);
            // ---- gradient at x_new
            wide_gradient<OBJ, GRAD>(xn, gn, d, sh);
            __syncthreads();
            fn = sh.red[2];
            // ---- curvature pair
            for (int j = tid; j < d; j += T) {  // s into sv, y over g
                const double sj = xn[j] - x[j], yj = gn[j] - g[j];
                sv[j] = sj;
                g[j] = yj;
                sc0[j] = yj * sj;
                sc1[j] = sj * sj;
                sc2[j] = yj * yj;
            }
            __syncthreads();
            if (tid < 3) sh.red[tid] = ordered_sum(tid == 0 ? sc0 : (tid == 1 ? sc1 : sc2), d, 0.0);
            __syncthreads();
            const double sy = sh.red[0], ss = sh.red[1], yy = sh.red[2];
            if (sy > 1e-12 * sqrt(ss) * sqrt(yy)) {
                const double rho = 1.0 / sy;
                __syncthreads();
                for (int r = tid; r < d; r += T) {  // Hy into p (the direction is spent)
                    const double* Hr = H + r * d;
                    double a = 0.0;
                    for (int c = 0; c < d; ++c) a = a + Hr[c] * g[c];
                    pv[r] = a;
                    sc0[r] = g[r] * a;
                }
                __syncthreads();
                if (tid == 0) sh.red[3] = ordered_sum(sc0, d, 0.0);
                __syncthreads();
                const double b2 = rho * rho * sh.red[3] + rho;
                for (int e = tid; e < d * d; e += T) {
                    const int r = e / d, c = e - r * d;
                    const double sr = sv[r], sc = sv[c];
                    H[e] = H[e] - rho * (pv[r] * sc + sr * pv[c]) + b2 * (sr * sc);
                }
            }
            __syncthreads();
            for (int j = tid; j < d; j += T) {
                x[j] = xn[j];
                g[j] = gn[j];
            }
            f0 = fn;
            ++k;
            __syncthreads();
        }
        for (int j = tid; j < d; j += T) x_out[s * d + j] = x[j];
        if (tid == 0) {
            if (f_out) f_out[s] = f0;
            if (gnorm_out) gnorm_out[s] = gnorm;
            if (status_out) status_out[s] = status;
            if (iters_out) iters_out[s] = k;
            atomicAdd(&ctrl->total_iters, (unsigned long long)k);
            atomicAdd(&ctrl->total_feval, (unsigned long long)feval);
            if (!use_stop && status == ZEUS_RUN_CONVERGED) atomicAdd(&ctrl->n_conv, 1ull);
        }
    }
}

// ---------------------------------------------------------------------------
// Launch planning
// ---------------------------------------------------------------------------
static size_t narrow_stride(int d) {
    size_t st = (size_t)d * d + 6 * (size_t)d;
    if ((st & 1) == 0) st += 1;  // odd: the 32 starts of a warp fall in distinct banks
    return st;
}

static int wide_trials(int d, int L) {
    int W = (2 * kWideThreads) / (d > 0 ? d : 1);
    if (W < 1) W = 1;
    if (W > 64) W = 64;
    if (W > L) W = L;
    return W;
}

static size_t wide_smem(int d, int W, int L) {
    return sizeof(double) * ((size_t)d * d + 9 * (size_t)d + 2 * (size_t)W * d + W + L + 1);
}

int plan_bfgs(const zeus_problem& p, BfgsLaunch* L) {
    const int d = p.dim;
    const size_t cap = 227 * 1024;
    const int req = p.threads_per_start;
    const size_t row = narrow_stride(d) * sizeof(double);
    const bool narrow_fits = row * 32 <= cap;
    L->narrow = (req == 1) || (req == 0 && narrow_fits && d <= 16);
    if (L->narrow && !narrow_fits) return ZEUS_EUNSUPPORTED;
    L->stride = (int)narrow_stride(d);
    int nthreads = kNarrowThreads;
    while (nthreads > 32 && (size_t)nthreads * row > cap) nthreads -= 32;
    L->narrow_threads = nthreads;
    L->narrow_smem = (size_t)nthreads * row;
    L->narrow_blocks = (int)((p.n_starts + nthreads - 1) / nthreads);
    L->W = wide_trials(d, p.ls_max_iters);
    L->wide_smem = wide_smem(d, L->W, p.ls_max_iters);
    if (!L->narrow && L->wide_smem > cap) return ZEUS_EUNSUPPORTED;
    L->wide_blocks = 152 * 4;
    // hand-over budget (iterations + line-search evaluations) of the narrow
    // kernel; 0 = every start runs to its end in the narrow kernel.  Only
    // used when the wide kernel can hold the start (its shared memory fits).
    L->budget = (L->narrow && L->wide_smem <= cap && req != 1) ? 160 : 0;
    L->q_cap = 0;
    if (L->budget > 0) {
        long long capn = p.n_starts;
        const long long max_bytes = 256ll << 20;
        const long long per = (long long)d * d * 8;
        if (capn * per > max_bytes) capn = max_bytes / per;
        if (capn < 1) capn = 1;
        L->q_cap = (int)capn;
    }
    return ZEUS_OK;
}

template <int OBJ, int GRAD>
static cudaError_t bfgs_go(const zeus_problem& p, const BfgsLaunch& L, const double* x0,
                           double* x_out, double* f_out, double* gnorm_out, int32_t* status_out,
                           int32_t* iters_out, Ctrl* ctrl, const Queue& q, cudaStream_t st) {
    cudaError_t e;
    if (L.narrow) {
        auto kn = bfgs_narrow_kernel<OBJ, GRAD>;
        e = cudaFuncSetAttribute(kn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)L.narrow_smem);
        if (e != cudaSuccess) return e;
        kn<<<L.narrow_blocks, L.narrow_threads, L.narrow_smem, st>>>(
            p, L.stride, L.budget, x0, x_out, f_out, gnorm_out, status_out, iters_out, ctrl, q);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        if (L.budget == 0) return cudaSuccess;
    }
    auto kw = bfgs_wide_kernel<OBJ, GRAD>;
    e = cudaFuncSetAttribute(kw, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.wide_smem);
    if (e != cudaSuccess) return e;
    kw<<<L.wide_blocks, kWideThreads, L.wide_smem, st>>>(p, L.W, x0, x_out, f_out, gnorm_out,
                                                         status_out, iters_out, ctrl, q,
                                                         L.narrow ? 0 : 1);
    return cudaGetLastError();
}

template <int OBJ>
static cudaError_t bfgs_obj(const zeus_problem& p, const BfgsLaunch& L, const double* x0,
                            double* x_out, double* f_out, double* gnorm_out, int32_t* status_out,
                            int32_t* iters_out, Ctrl* ctrl, const Queue& q, cudaStream_t st) {
    if (p.grad_mode == ZEUS_GRAD_ADJOINT)
        return bfgs_go<OBJ, ZEUS_GRAD_ADJOINT>(p, L, x0, x_out, f_out, gnorm_out, status_out,
                                               iters_out, ctrl, q, st);
    return bfgs_go<OBJ, ZEUS_GRAD_FORWARD>(p, L, x0, x_out, f_out, gnorm_out, status_out,
                                           iters_out, ctrl, q, st);
}

cudaError_t launch_bfgs(const zeus_problem& p, const BfgsLaunch& L, const double* x0,
                        double* x_out, double* f_out, double* gnorm_out, int32_t* status_out,
                        int32_t* iters_out, Ctrl* ctrl, const Queue& q, cudaStream_t st) {
    switch (p.objective) {
        case ZEUS_OBJ_ROSENBROCK:
            return bfgs_obj<ZEUS_OBJ_ROSENBROCK>(p, L, x0, x_out, f_out, gnorm_out, status_out,
                                                 iters_out, ctrl, q, st);
        case ZEUS_OBJ_RASTRIGIN:
            return bfgs_obj<ZEUS_OBJ_RASTRIGIN>(p, L, x0, x_out, f_out, gnorm_out, status_out,
                                                iters_out, ctrl, q, st);
        case ZEUS_OBJ_ACKLEY:
            return bfgs_obj<ZEUS_OBJ_ACKLEY>(p, L, x0, x_out, f_out, gnorm_out, status_out,
                                             iters_out, ctrl, q, st);
        case ZEUS_OBJ_GOLDSTEIN_PRICE:
            return bfgs_obj<ZEUS_OBJ_GOLDSTEIN_PRICE>(p, L, x0, x_out, f_out, gnorm_out,
                                                      status_out, iters_out, ctrl, q, st);
        default:
            return bfgs_obj<ZEUS_OBJ_QUADRATIC>(p, L, x0, x_out, f_out, gnorm_out, status_out,
                                                iters_out, ctrl, q, st);
    }
}

}  // namespace zeus
