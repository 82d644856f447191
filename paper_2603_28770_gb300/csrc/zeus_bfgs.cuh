// zeus_bfgs.cuh -- the BFGS bodies shared by the single-problem kernels
// (zeus_bfgs.cu) and the batched kernels (zeus_batch.cu): one start on one
// lane (narrow_run) or on one block (wide_run).  See zeus_bfgs.cu for the
// design.
#pragma once

#include "zeus_device.cuh"
#include "zeus_internal.h"

namespace zeus {

// ---------------------------------------------------------------------------
// Objective value sweep in index order: init, term j, finish.  Coordinates
// come through an accessor so the wide kernel can form a trial point
// x + a p on the fly (the same bits as the materialised point).
// ---------------------------------------------------------------------------
template <class T>
struct AtPoint {
    const T* x;
    __device__ __forceinline__ T operator()(int j) const { return x[j]; }
};
template <class T>
struct AtTrial {
    const T* x;
    const T* p;
    T a;
    __device__ __forceinline__ T operator()(int j) const { return x[j] + a * p[j]; }
};
// FP32 coordinates read as FP64 (the final value of an FP32 run is an FP64
// evaluation at its point)
struct AtPromoted {
    const float* x;
    __device__ __forceinline__ double operator()(int j) const { return (double)x[j]; }
};

// Dot and matrix-vector products accumulate every term with one rounding
// (fused multiply-add), in index order.  dot_fma: an FP64 sum (the FP32
// form promotes its operands first; their product is exact in FP64, so its
// FP64 guard sums also round once per term).  mv_fma: the working precision.
__device__ __forceinline__ double dot_fma(double a, double b, double acc) { return fma(a, b, acc); }
__device__ __forceinline__ double dot_fma(float a, float b, double acc) {
    return fma((double)a, (double)b, acc);
}
__device__ __forceinline__ double mv_fma(double a, double b, double acc) { return fma(a, b, acc); }
__device__ __forceinline__ float mv_fma(float a, float b, float acc) { return fmaf(a, b, acc); }

// The dot products of the BFGS step (||g||^2, g'p, y's, s's, y'y, y'Hy):
// up to kDotSplit terms one chain in index order; past that 32 strided
// chains (chain l over the indices l, l + 32, ...) added in a fixed tree,
// l with l + 16, then l + 8, l + 4, l + 2, l + 1, so that one warp forms
// the sum (a one-lane chain of d FP64 instructions holds its sub-partition's
// FP64 pipe as long as d full-warp instructions would).
constexpr int kDotSplit = 32;

// the split order by one warp (lane = role mod 32); every lane gets the sum
template <class T>
__device__ __forceinline__ double warp_split_dot(const T* a, const T* b, int n, int lane) {
    double acc = 0.0;
#pragma unroll 1
    for (int j = lane; j < n; j += 32) acc = dot_fma(a[j], b[j], acc);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc = acc + __shfl_down_sync(0xffffffffu, acc, o);
    return __shfl_sync(0xffffffffu, acc, 0);
}

// the split order on one thread (the lane kernel meets d > kDotSplit only
// when one lane per start is asked for).  The tree's leaves, left to right,
// are the chains in bit-reversed order (0, 16, 8, 24, 4, ...); they are
// formed one at a time and merged as a binary counter does, so that no
// more than five partial sums are held.
template <class T>
__device__ __forceinline__ double lane_split_dot(const T* a, const T* b, int n) {
    double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0, s4 = 0.0, v = 0.0;
#pragma unroll 1
    for (int k = 0; k < 32; ++k) {
        const int l = (int)(__brev((unsigned)k) >> 27);
        v = 0.0;
#pragma unroll 1
        for (int j = l; j < n; j += 32) v = dot_fma(a[j], b[j], v);
        if (!(k & 1)) { s0 = v; continue; }
        v = s0 + v;
        if (!(k & 2)) { s1 = v; continue; }
        v = s1 + v;
        if (!(k & 4)) { s2 = v; continue; }
        v = s2 + v;
        if (!(k & 8)) { s3 = v; continue; }
        v = s3 + v;
        if (!(k & 16)) { s4 = v; continue; }
        v = s4 + v;
    }
    return v;
}

// ||g|| < tol from g'g: away from the boundary without the square root
// (sqrt is monotone and correctly rounded, and the margins of 1e-12 exceed
// the rounding of tol^2 by far), at it by the square root itself; the same
// decision as sqrt(gg) < tol in every case.  With tol^2 outside the normal
// range every decision takes the square root (lo = -1, hi = inf).
struct GradTest {
    double lo, hi;
    __device__ explicit GradTest(double tol) {
        const double t2 = tol * tol;
        const bool fast = t2 > 1e-280 && t2 < 1e280;
        lo = fast ? t2 * (1.0 - 1e-12) : -1.0;
        hi = fast ? t2 * (1.0 + 1e-12) : CUDART_INF;
    }
    __device__ __forceinline__ bool below(double gg, double tol) const {
        if (gg < lo) return true;
        if (gg >= hi) return false;
        return sqrt(gg) < tol;
    }
};

// one thread's BFGS dot product in the order above
template <class T>
__device__ __forceinline__ double lane_dot(const T* a, const T* b, int n) {
    if (n > kDotSplit) return lane_split_dot(a, b, n);
    double acc = 0.0;
    for (int j = 0; j < n; ++j) acc = dot_fma(a[j], b[j], acc);
    return acc;
}

// The FP32 form evaluates Rastrigin as sum (x^2 + 20 sin^2(pi x)) and the
// cosine mean of Ackley through 1 - (2/d) sum sin^2(pi x): the same
// functions in exact arithmetic, without the cancellation that the literal
// 10 d + sum(x^2 - 10 cos 2 pi x) suffers in FP32 near every integer point.
template <class V>
struct F32Terms {
    static constexpr bool on = sizeof(V) == 4;
};

template <int OBJ, class T = double>
__device__ __forceinline__ Part<double> val_init(int d) {
    Part<double> a;
    a.s0 = (OBJ == ZEUS_OBJ_RASTRIGIN && !F32Terms<T>::on) ? 10.0 * (double)d : 0.0;
    a.s1 = 0.0;
    return a;
}

template <int OBJ, class T = double>
__device__ __forceinline__ double val_finish(const Part<double>& acc, int d) {
    if (OBJ == ZEUS_OBJ_ACKLEY && F32Terms<T>::on) {
        const double dd = (double)d;
        const double t1 = -20.0 * exp_cw(-0.2 * sqrt(acc.s0 / dd));
        const double t2 = exp_cw(1.0 - 2.0 * (acc.s1 / dd));
        return (t1 - t2) + (20.0 + 2.718281828459045235360287471352);
    }
    return value_finish<OBJ, double>(acc, d);
}

// a user objective is a single term (f at the whole point)
template <int OBJ>
__device__ __forceinline__ int val_nterms(int d) {
    if (OBJ == ZEUS_OBJ_ROSENBROCK) return d - 1;
    if (OBJ == ZEUS_OBJ_GOLDSTEIN_PRICE || OBJ >= ZEUS_OBJ_USER) return 1;
    return d;
}

// term j of the sweep in the accessor's type V, returned as FP64 (the sums
// of the FP32 form are FP64 sums of FP32 terms)
template <int OBJ, class X>
__device__ __forceinline__ void val_term(const X& xa, int j, int d, double& t0, double& t1) {
    using V = decltype(xa(0));
    t1 = 0.0;
    if constexpr (OBJ >= ZEUS_OBJ_USER) {
        (void)j;
        t0 = (double)UserObjective<OBJ>::template eval<V>(xa, d);
        return;
    }
    (void)d;
    if (OBJ == ZEUS_OBJ_ROSENBROCK) {
        const V xj = xa(j);
        const V a = V(1) - xj;
        const V b = xa(j + 1) - xj * xj;
        t0 = (double)(a * a + V(100) * (b * b));
    } else if (OBJ == ZEUS_OBJ_RASTRIGIN) {
        const V xj = xa(j);
        if (F32Terms<V>::on) {
            const V sp = (V)sinpif((float)xj);
            t0 = (double)(xj * xj + V(20) * (sp * sp));
        } else {
            t0 = (double)(xj * xj - V(10) * c_2pi(xj));
        }
    } else if (OBJ == ZEUS_OBJ_ACKLEY) {
        const V xj = xa(j);
        t0 = (double)(xj * xj);
        if (F32Terms<V>::on) {
            const V sp = (V)sinpif((float)xj);
            t1 = (double)(sp * sp);
        } else {
            t1 = (double)c_2pi(xj);
        }
    } else if (OBJ == ZEUS_OBJ_GOLDSTEIN_PRICE) {
        const V x1 = xa(0), x2 = xa(1);
        const V t = (x1 + x2) + V(1);
        const V pa = V(19) - V(14) * x1 + V(3) * (x1 * x1) - V(14) * x2 + V(6) * (x1 * x2) +
                     V(3) * (x2 * x2);
        const V a = V(1) + (t * t) * pa;
        const V u = V(2) * x1 - V(3) * x2;
        const V pb = V(18) - V(32) * x1 + V(12) * (x1 * x1) + V(48) * x2 - V(36) * (x1 * x2) +
                     V(27) * (x2 * x2);
        const V b = V(30) + (u * u) * pb;
        t0 = (double)(a * b);
    } else {
        const V xj = xa(j);
        t0 = (double)((V(0.5) * V(j + 1)) * (xj * xj));
    }
}

template <int OBJ>
__device__ __forceinline__ void val_add(Part<double>& acc, double t0, double t1) {
    if (OBJ == ZEUS_OBJ_GOLDSTEIN_PRICE || OBJ >= ZEUS_OBJ_USER) {
        acc.s0 = t0;
    } else {
        acc.s0 = acc.s0 + t0;
        if (OBJ == ZEUS_OBJ_ACKLEY) acc.s1 = acc.s1 + t1;
    }
}

// f at a point on one thread, in the order of the oracle's sweep (the
// objective sums of obj_sum; one term for Goldstein-Price and the user
// objectives)
template <int OBJ, class X>
__device__ __forceinline__ double seq_value(const X& xa, int d) {
    using V = decltype(xa(0));
    const int nt = val_nterms<OBJ>(d);
    if constexpr (OBJ == ZEUS_OBJ_GOLDSTEIN_PRICE || OBJ >= ZEUS_OBJ_USER) {
        Part<double> acc = val_init<OBJ, V>(d);
        for (int j = 0; j < nt; ++j) {
            double t0, t1;
            val_term<OBJ>(xa, j, d, t0, t1);
            val_add<OBJ>(acc, t0, t1);
        }
        return val_finish<OBJ, V>(acc, d);
    } else {
        const Part<double> acc =
            obj_sum<double>(d, nt, val_init<OBJ, V>(d), OBJ == ZEUS_OBJ_ACKLEY, [&](int j) {
                Part<double> t;
                val_term<OBJ>(xa, j, d, t.s0, t.s1);
                return t;
            });
        return val_finish<OBJ, V>(acc, d);
    }
}

// Gradient: forward pass i (Alg. 5) or adjoint component i.  The adjoint
// first forms the quantities shared by all components (Ackley's two sums,
// in index order) on one thread.
template <int OBJ, int GRAD, class T>
__device__ __forceinline__ AdjShared grad_prep(const T* x, int d) {
    AdjShared a;
    a.c1 = a.c2 = 0.0;
    if (GRAD == ZEUS_GRAD_ADJOINT) a = adjoint_prep<OBJ>(x, d);
    return a;
}
template <int OBJ, int GRAD, class T>
__device__ __forceinline__ T grad_component(const T* x, int d, int i, const AdjShared& a) {
    if (GRAD == ZEUS_GRAD_FORWARD) return forward_tangent<OBJ, T>(x, d, i);
    return adjoint_component<OBJ>(x, d, i, a);
}

// The whole gradient on one thread (the lane kernel): component by
// component, or a user objective's chunked passes
template <int OBJ, int GRAD, class T>
__device__ __forceinline__ void grad_all(const T* x, int d, T* g) {
    if constexpr (OBJ >= ZEUS_OBJ_USER && GRAD == ZEUS_GRAD_FORWARD) {
        user_gradient<OBJ, T>(x, d, g);
    } else {
        const AdjShared a = grad_prep<OBJ, GRAD>(x, d);
        for (int i = 0; i < d; ++i) g[i] = grad_component<OBJ, GRAD>(x, d, i, a);
    }
}

// final f and its output: FP64 value at the point (FP32 points promoted)
template <int OBJ>
__device__ __forceinline__ double final_value(const double* x, int d, double f0) {
    (void)x;
    (void)d;
    return f0;
}
template <int OBJ>
__device__ __forceinline__ double final_value(const float* x, int d, double) {
    return seq_value<OBJ>(AtPromoted{x}, d);
}

// ---------------------------------------------------------------------------
// Narrow kernel: one lane per start.  T = double (the paper's FP64 method)
// or float (the FP32 form: objective, gradient, H and the vectors in FP32;
// y's, |s|^2, |y|^2, g'p, y'Hy, rho, the Armijo sums and the final f in
// FP64).  With T = double every FP64 guard below is the plain FP64 operation.
// Shared memory per start (T): H [d*d] | x | g | p | xn | gn | s
// ---------------------------------------------------------------------------
template <int OBJ, int GRAD, class T>
__device__ __forceinline__ void narrow_run(const zeus_problem& p, const long long s, T* H,
                                           const int budget, const RunIO& io, Ctrl* qc,
                                           const Queue& q, const int prob) {
    const int d = p.dim;
    T* x = H + (size_t)d * d;
    T* g = x + d;
    T* pv = g + d;
    T* xn = pv + d;
    T* gn = xn + d;
    T* sv = gn + d;
    Ctrl* ctrl = io.pc;
    const double* x0 = io.x0;
    double* x_out = io.x_out;

    const bool use_target = !isnan(p.target_f);
    const bool use_stop = use_target || p.required_converged > 0;
    const double tol = p.grad_tol, cA = p.armijo_c, beta = p.backtrack;
    const int K = p.bfgs_max_iters, L = p.ls_max_iters;

    for (int j = 0; j < d; ++j) x[j] = T(x0[s * d + j]);
    for (int r = 0; r < d; ++r)
        for (int c = 0; c < d; ++c) H[r * d + c] = (c == r) ? T(1) : T(0);
    {
        grad_all<OBJ, GRAD>(x, d, g);
    }
    double f0 = seq_value<OBJ>(AtPoint<T>{x}, d);

    int k = 0, status = ZEUS_RUN_MAX_ITER, feval = 0;
    bool ls_failed = false;  // the previous iteration's search accepted no trial
    bool stalled = false;    // FP32 form: the previous iteration's decrease was unresolved
    double gnorm;
    for (;;) {
        double gg = 0.0;
        bool bad = false;
        for (int j = 0; j < d; ++j) {
            gg = dot_fma(g[j], g[j], gg);
            bad |= !isfinite(g[j]);
        }
        if (d > kDotSplit) gg = lane_split_dot(g, g, d);
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
        if (stalled) {
            status = ZEUS_RUN_STALLED;
            break;
        }
        if (budget > 0 && (k + feval >= budget || ls_failed)) {
            // hand the start over to the wide kernel at the top of iteration k
            // (work budget spent, or the last line search exhausted its
            // trials: such a start usually keeps failing, and each failing
            // search costs L sweeps on one lane)
            // a start whose searches take many trials (the last one failed,
            // or more than two evaluations per iteration so far) likely
            // keeps failing: it goes to the long entries when the consumer
            // keeps them apart (fused kernel)
            unsigned slot = ~0u;
            if (q.long_cap > 0 && (ls_failed || feval > 2 * k)) {
                const unsigned h = atomicAdd(&qc->q_count_long, 1u);
                if (h < (unsigned)q.long_cap) slot = (unsigned)(q.cap - q.long_cap) + h;
            }
            if (slot == ~0u) {  // the other entries (also when the long ones are full)
                const unsigned h = atomicAdd(&qc->q_count, 1u);
                if (h < (unsigned)(q.cap - q.long_cap)) slot = h;
            }
            if (slot != ~0u) {
                q.start[slot] = (int)s;
                if (q.prob) q.prob[slot] = prob;
                q.k[slot] = k;
                q.feval[slot] = feval;
                const size_t hs = q.hstride ? (size_t)q.hstride : (size_t)d * d;
                T* Hq = reinterpret_cast<T*>(q.H) + (size_t)slot * hs;
                for (int e = 0; e < d * d; ++e) Hq[e] = H[e];
                T* xq = reinterpret_cast<T*>(x_out + s * d);  // the row holds x until the end
                for (int j = 0; j < d; ++j) xq[j] = x[j];
                if (q.ready) {  // a consumer running alongside may take the entry now
                    __threadfence();
                    atomicExch(q.ready + slot, 1);
                }
                return;
            }
        }
        // direction p = -H g and ddir = g'p
        for (int r = 0; r < d; ++r) {
            const T* Hr = H + r * d;
            T a = T(0);
            for (int c = 0; c < d; ++c) a = mv_fma(Hr[c], g[c], a);
            pv[r] = -a;
        }
        double ddir = lane_dot(g, pv, d);
        if (!(ddir < 0.0)) {  // not a descent direction: restart from H = I
            for (int r = 0; r < d; ++r)
                for (int c = 0; c < d; ++c) H[r * d + c] = (c == r) ? T(1) : T(0);
            for (int r = 0; r < d; ++r) pv[r] = -g[r];
            ddir = lane_dot(g, pv, d);
        }
        // backtracking Armijo line search (Alg. 6)
        double alpha = 1.0, fn = 0.0;
        bool accepted = false;
        for (int m = 0; m < L; ++m) {
            const T a = T(alpha);
            for (int j = 0; j < d; ++j) xn[j] = x[j] + a * pv[j];
            fn = seq_value<OBJ>(AtPoint<T>{xn}, d);
            ++feval;
            if (fn <= f0 + cA * alpha * ddir) {
                accepted = true;
                break;
            }
            alpha = beta * alpha;
        }
        if (!accepted) {  // Alg. 6 returns the step after the last halving
            const T a = T(alpha);
            for (int j = 0; j < d; ++j) xn[j] = x[j] + a * pv[j];
            fn = seq_value<OBJ>(AtPoint<T>{xn}, d);
        }
        ls_failed = !accepted;
        {
            grad_all<OBJ, GRAD>(xn, d, gn);
        }
        // curvature pair
        double sy = 0.0, ss = 0.0, yy = 0.0;
        for (int j = 0; j < d; ++j) {  // s into sv, y over g (g is not needed again)
            const T sj = xn[j] - x[j], yj = gn[j] - g[j];
            sv[j] = sj;
            g[j] = yj;
            sy = dot_fma(yj, sj, sy);
            ss = dot_fma(sj, sj, ss);
            yy = dot_fma(yj, yj, yy);
        }
        if (d > kDotSplit) {
            sy = lane_split_dot(g, sv, d);
            ss = lane_split_dot(sv, sv, d);
            yy = lane_split_dot(g, g, d);
        }
        const bool upd = sy > 1e-12 * sqrt(ss) * sqrt(yy);
        T rt = T(0), bt = T(0);
        if (upd) {
            const double rho = 1.0 / sy;
            for (int r = 0; r < d; ++r) {  // Hy into p (the direction is spent)
                const T* Hr = H + r * d;
                T a = T(0);
                for (int c = 0; c < d; ++c) a = mv_fma(Hr[c], g[c], a);
                pv[r] = a;
            }
            const double yhy = lane_dot(g, pv, d);
            const double b2 = rho * rho * yhy + rho;
            rt = T(rho);
            bt = T(b2);
        }
        for (int j = 0; j < d; ++j) {
            x[j] = xn[j];
            g[j] = gn[j];
        }
        if (upd) {
            // H_rc <- fma(s_c, A_r, fma(Hy_c, B_r, H_rc)), A = b2 s - rho Hy
            // and B = -rho s in the spent x_new and g_new rows
            for (int r = 0; r < d; ++r) {
                xn[r] = mv_fma(bt, sv[r], -(rt * pv[r]));
                gn[r] = -(rt * sv[r]);
            }
            for (int r = 0; r < d; ++r) {  // r <= c, mirrored (H stays symmetric)
                const T ar = xn[r], br = gn[r];
                T* Hr = H + r * d;
                for (int c = r; c < d; ++c) {
                    const T v = mv_fma(sv[c], ar, mv_fma(pv[c], br, Hr[c]));
                    Hr[c] = v;
                    H[c * d + r] = v;
                }
            }
        }
        stalled = stalled_step<T>(f0, fn);
        f0 = fn;
        ++k;
    }

    const double ffin = final_value<OBJ>(x, d, f0);
    for (int j = 0; j < d; ++j) x_out[s * d + j] = (double)x[j];
    if (io.f_out) io.f_out[s] = ffin;
    if (io.gnorm_out) io.gnorm_out[s] = gnorm;
    if (io.status_out) io.status_out[s] = status;
    if (io.iters_out) io.iters_out[s] = k;
    atomicAdd(&ctrl->total_iters, (unsigned long long)k);
    atomicAdd(&ctrl->total_feval, (unsigned long long)feval);
    if (!use_stop && status == ZEUS_RUN_CONVERGED) atomicAdd(&ctrl->n_conv, 1ull);
}

// ---------------------------------------------------------------------------
// Wide kernel: one CTA per start, persistent over a queue of starts.
// Shared memory: T region H [d*d] | x | g | p | xn | gn | s, then an FP64
// region scratch [2 d] | trial terms [W][d] x 2 | trial f [W] | alpha [L+1]
// ---------------------------------------------------------------------------
struct WideShared {
    int item;
    int status;
    int accepted_m;
    int pad;
    double red[8];
    AdjShared adj;
    int ok[64];
};

// a'b over [0, n) in index order, one rounding per term (dot_fma), on the
// calling thread
template <class T>
__device__ __forceinline__ double ordered_dot(const T* a, const T* b, int n) {
    double s = 0.0;
    for (int j = 0; j < n; ++j) s = dot_fma(a[j], b[j], s);
    return s;
}

// Synchronisation of the threads that carry one start: the whole block
// (NTW = kWideThreads) or one warp (NTW = 32, several starts per block).
template <int NTW>
__device__ __forceinline__ void group_sync() {
    if constexpr (NTW == 32) __syncwarp();
    else __syncthreads();
}
template <int NTW>
__device__ __forceinline__ int group_sync_or(int b) {
    if constexpr (NTW == 32) {
        __syncwarp();
        return __any_sync(0xffffffffu, b);
    } else {
        return __syncthreads_or(b);
    }
}

template <int OBJ, int GRAD, class T, int NTW = kWideThreads>
__device__ __forceinline__ void wide_gradient(const T* x, T* g, int d, int tid, WideShared& sh) {
    const int NT = NTW == 32 ? 32 : (int)blockDim.x;
    if (GRAD == ZEUS_GRAD_ADJOINT) {
        if (tid == 0) sh.adj = adjoint_prep<OBJ>(x, d);
        group_sync<NTW>();
    }
    const AdjShared a = sh.adj;
    for (int i = tid; i < d; i += NT) g[i] = grad_component<OBJ, GRAD>(x, d, i, a);
}

// The block- and warp-per-start forms hold the symmetric H as its upper
// triangle, packed by rows: (r, c), r <= c, at tri_off(r) + c - r.  Every
// element is the one the full matrix holds (the update keeps H exactly
// symmetric), so rows read through tri_row_dot carry the same values in the
// same column order; the packed form halves the shared memory of H.
__host__ __device__ __forceinline__ int tri_off(int r, int d) { return r * d - (r * (r - 1)) / 2; }

// Element t of the triangle in an order that balances threads: rows p and
// d - 1 - p together hold d + 1 elements, so t = p (d + 1) + q numbers them
// without gaps.
__device__ __forceinline__ void tri_pair(int t, int d, int& r, int& c) {
    const int pr = t / (d + 1), q = t - pr * (d + 1);
    if (q < d - pr) {
        r = pr;
        c = pr + q;
    } else {
        r = d - 1 - pr;
        c = r + (q - (d - pr));
    }
}

// (H v)_r over the packed triangle, columns in order, one fused
// multiply-add per term: (c, r) for c < r, then (r, c).  The element index
// is selected per column, so the lanes of a warp never diverge.
template <class T>
__device__ __forceinline__ T tri_row_dot(const T* H, int d, int r, const T* v) {
    int lo = r;                          // (c, r) while c < r
    const int hi = tri_off(r, d) - r;    // (r, c) = hi + c for c >= r
    T a = T(0);
    for (int c = 0; c < d; ++c) {
        const int e = c < r ? lo : hi + c;
        a = mv_fma(H[e], v[c], a);
        lo += d - c - 1;
    }
    return a;
}

__host__ __device__ __forceinline__ size_t wide_t_bytes(int d, size_t tsize) {
    const size_t nu = (size_t)d * (d + 1) / 2;
    return ((nu + 6 * (size_t)d) * tsize + 7) & ~size_t(7);
}

// Row r of a matrix-vector product goes to the thread of role
// (r + NT - 32) mod NT: the rows start on the last warp, away from the
// threads of roles 0 and 32 that form the ordered sums of the same phase.
__device__ __forceinline__ int row_of(int tid, int NT) { return (tid + 32) % NT; }

// One start on one block (NTW = kWideThreads) or on one warp (NTW = 32),
// from iteration k with `feval` evaluations done: H from Hq (nullptr:
// identity), x from xq (nullptr: row s of io.x0).  The warp form performs
// the same operations in the same order; sums that the block forms on
// different warps at once, it forms one after the other.
template <int OBJ, int GRAD, class T, int NTW = kWideThreads>
__device__ __forceinline__ void wide_run(const zeus_problem& p, const int W, const long long s,
                                         int k, int feval, const T* Hq, const T* xq,
                                         const RunIO& io, WideShared& sh,
                                         unsigned char* smem_raw, const int tid,
                                         const bool peer = false) {
    static_assert(NTW == 32 || NTW >= 96, "a warp, or a block of at least three warps");
    const int NT = NTW == 32 ? 32 : (int)blockDim.x;
    const int d = p.dim;
    T* H = reinterpret_cast<T*>(smem_raw);  // packed upper triangle
    const int nu = d * (d + 1) / 2;
    T* x = H + nu;
    T* g = x + d;
    T* pv = g + d;
    T* xn = pv + d;
    T* gn = xn + d;
    T* sv = gn + d;
    double* sc0 = reinterpret_cast<double*>(smem_raw + wide_t_bytes(d, sizeof(T)));
    double* sc1 = sc0 + d;  // two FP64 scratch vectors
    double* tb0 = sc1 + d;              // [W][d]
    double* tb1 = tb0 + (size_t)W * d;  // [W][d] (second sum of Ackley)
    double* fb = tb1 + (size_t)W * d;   // [W]
    double* al = fb + W;                // [L + 1]
    Ctrl* ctrl = io.pc;

    const bool use_target = !isnan(p.target_f);
    const bool use_stop = use_target || p.required_converged > 0;
    const double tol = p.grad_tol, cA = p.armijo_c, beta = p.backtrack;
    const GradTest gtest(tol);
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
    if (xq) {  // peer: written by another block of this launch, read past L1
        for (int j = tid; j < d; j += NT) x[j] = peer ? __ldcg(xq + j) : xq[j];
    } else {
        for (int j = tid; j < d; j += NT) x[j] = T(io.x0[s * d + j]);
    }
    for (int t = tid; t < nu; t += NT) {  // Hq holds the full matrix, row-major
        int r, c;
        tri_pair(t, d, r, c);
        const int e = tri_off(r, d) + c - r;
        if (Hq) H[e] = peer ? __ldcg(Hq + (size_t)r * d + c) : Hq[(size_t)r * d + c];
        else H[e] = r == c ? T(1) : T(0);
    }
    group_sync<NTW>();
    wide_gradient<OBJ, GRAD, T, NTW>(x, g, d, tid, sh);
    if (tid == 0) sh.red[0] = seq_value<OBJ>(AtPoint<T>{x}, d);
    group_sync<NTW>();
    double f0 = sh.red[0];
    int status = ZEUS_RUN_MAX_ITER;
    double gnorm = 0.0;
    int hint = W;  // trials the previous search needed
    bool stalled = false;  // FP32 form: the previous iteration's decrease was unresolved
    for (;;) {
        // ---- tests at the top of iteration k, with the direction p = -H g
        // formed alongside (one row per thread, columns in order; used only
        // if the start goes on)
        int b = 0;
        for (int j = tid; j < d; j += NT) b |= !isfinite(g[j]);
        for (int r = row_of(tid, NT); r < d; r += NT) pv[r] = -tri_row_dot(H, d, r, g);
        const int bad = group_sync_or<NTW>(b);
        // g'g and g'p on roles 0 and 1 (one warp, one instruction stream:
        // an FP64 warp instruction costs the same for one lane or two)
        double dot01 = 0.0;
        if (d > kDotSplit) {  // g'g on the warp of roles 0-31, g'p on the next
            if constexpr (NTW == 32) {
                const double gp = warp_split_dot(g, pv, d, tid);
                dot01 = warp_split_dot(g, g, d, tid);
                if (tid == 0) sh.red[0] = gp;
            } else {
                if (tid < 64) dot01 = warp_split_dot(g, tid < 32 ? g : pv, d, tid & 31);
                if (tid == 32) sh.red[0] = dot01;
            }
        } else {
            if (tid < 2) dot01 = ordered_dot(g, tid == 0 ? g : pv, d);
            if (tid == 1) sh.red[0] = dot01;
        }
        if (tid == 0) {
            int st = -1;
            if (k >= K) {
                st = ZEUS_RUN_MAX_ITER;
            } else if (use_stop && *((volatile int*)&ctrl->stop)) {
                st = ZEUS_RUN_STOPPED;
            } else if (!isfinite(f0) || bad) {
                st = ZEUS_RUN_NONFINITE;
            } else if (gtest.below(dot01, tol)) {
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
            } else if (stalled) {
                st = ZEUS_RUN_STALLED;
            }
            if (st >= 0) sh.red[1] = sqrt(dot01);  // ||g|| of the final point
            sh.status = st;
        }
        group_sync<NTW>();
        if (sh.status >= 0) {
            gnorm = sh.red[1];
            status = sh.status;
            break;
        }
        double ddir = sh.red[0];
        if (!(ddir < 0.0)) {  // not a descent direction: restart from H = I
            group_sync<NTW>();
            for (int t = tid; t < nu; t += NT) {
                int r, c;
                tri_pair(t, d, r, c);
                H[tri_off(r, d) + c - r] = r == c ? T(1) : T(0);
            }
            for (int r = tid; r < d; r += NT) pv[r] = -g[r];
            group_sync<NTW>();
            if (d > kDotSplit) {
                if (tid < 32) {
                    const double v = warp_split_dot(g, pv, d, tid);
                    if (tid == 0) sh.red[0] = v;
                }
            } else if (tid == 0) {
                sh.red[0] = ordered_dot(g, pv, d);
            }
            group_sync<NTW>();
            ddir = sh.red[0];
        }
        // ---- line search: trials in chunks, the first accepted wins.
        // Index L is the point after the last halving (taken when every
        // trial fails, reading 4); a chunk may include it so that a search
        // that fails costs no separate sweep.  The first chunk has as many
        // trials as the previous iteration's search needed (all of them
        // for a start that keeps failing), the later ones W.
        int acc_m = -1;
        double fn = 0.0;
        int m0 = 0;
        while (acc_m < 0 && m0 <= L) {
            const int nw = min(m0 == 0 ? min(W, hint) : W, L + 1 - m0);
            for (int e = tid; e < nw * nt; e += NT) {
                const int mm = e / nt, j = e - mm * nt;
                double t0, t1;
                val_term<OBJ>(AtTrial<T>{x, pv, T(al[m0 + mm])}, j, d, t0, t1);
                tb0[mm * d + j] = t0;
                tb1[mm * d + j] = t1;
            }
            group_sync<NTW>();
            if (d > kSumSplit && nt > 1) {
                // a warp per trial: lane l forms chain l of the sums, the
                // warp adds the chains in the fixed tree (obj_sum's order)
                const int lane = tid & 31;
                for (int mm = tid >> 5; mm < nw; mm += NT >> 5) {
                    Part<double> acc;
                    acc.s0 = acc.s1 = 0.0;
                    if (lane == 0) acc = val_init<OBJ, T>(d);
                    for (int j = lane; j < nt; j += 32)
                        val_add<OBJ>(acc, tb0[mm * d + j], tb1[mm * d + j]);
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) {
                        acc.s0 = acc.s0 + __shfl_down_sync(0xffffffffu, acc.s0, o);
                        if (OBJ == ZEUS_OBJ_ACKLEY)
                            acc.s1 = acc.s1 + __shfl_down_sync(0xffffffffu, acc.s1, o);
                    }
                    if (lane == 0) {
                        const double ft = val_finish<OBJ, T>(acc, d);
                        fb[mm] = ft;
                        sh.ok[mm] = (m0 + mm < L && ft <= f0 + cA * al[m0 + mm] * ddir) ? 1 : 0;
                    }
                }
            } else if (tid < nw) {  // one thread per trial: its terms in order, then the test
                Part<double> acc = val_init<OBJ, T>(d);
                for (int j = 0; j < nt; ++j)
                    val_add<OBJ>(acc, tb0[tid * d + j], tb1[tid * d + j]);
                const double ft = val_finish<OBJ, T>(acc, d);
                fb[tid] = ft;
                sh.ok[tid] = (m0 + tid < L && ft <= f0 + cA * al[m0 + tid] * ddir) ? 1 : 0;
            }
            group_sync<NTW>();
            // every warp finds the first accepted trial itself with one
            // ballot over the flags (no further barrier: the next chunk
            // writes ok and fb only after its terms)
            {
                const int lane = tid & 31;
                const unsigned b0 = __ballot_sync(0xffffffffu, lane < nw && sh.ok[lane]);
                if (b0) {
                    acc_m = m0 + __ffs(b0) - 1;
                } else if (nw > 32) {  // trials 32-63 of a chunk
                    const unsigned b1 =
                        __ballot_sync(0xffffffffu, lane + 32 < nw && sh.ok[lane + 32]);
                    if (b1) acc_m = m0 + 32 + __ffs(b1) - 1;
                }
            }
            if (acc_m >= 0) fn = fb[acc_m - m0];
            else if (m0 + nw == L + 1) fn = fb[L - m0];  // every trial failed
            feval += (acc_m >= 0) ? (acc_m - m0 + 1) : min(nw, L - m0);
            m0 += nw;
        }
        hint = (acc_m >= 0) ? acc_m + 1 : L + 1;
        const T alpha = T((acc_m >= 0) ? al[acc_m] : al[L]);
        for (int j = tid; j < d; j += NT) xn[j] = x[j] + alpha * pv[j];
        group_sync<NTW>();
        // ---- gradient at x_new
        wide_gradient<OBJ, GRAD, T, NTW>(xn, gn, d, tid, sh);
        group_sync<NTW>();
        // ---- curvature pair; H y formed alongside its sums (used only if
        // the pair passes the curvature test)
        for (int j = tid; j < d; j += NT) {  // s into sv, y over g
            sv[j] = xn[j] - x[j];
            g[j] = gn[j] - g[j];
        }
        group_sync<NTW>();
        if (d > kDotSplit) {  // y's, s's, y'y on the warps of roles 0-95
            if constexpr (NTW == 32) {
                for (int w = 0; w < 3; ++w) {
                    const double v = warp_split_dot(w == 1 ? sv : g, w == 2 ? g : sv, d, tid);
                    if (tid == 0) sh.red[w] = v;
                }
            } else if (tid < 96) {
                const int w = tid >> 5;
                const double v = warp_split_dot(w == 1 ? sv : g, w == 2 ? g : sv, d, tid & 31);
                if ((tid & 31) == 0) sh.red[w] = v;
            }
        } else if (tid < 3) {  // on roles 0-2 (one warp, one instruction stream)
            sh.red[tid] = ordered_dot(tid == 1 ? sv : g, tid == 2 ? g : sv, d);
        }
        for (int r = row_of(tid, NT); r < d; r += NT)  // Hy into p (the direction is spent)
            pv[r] = tri_row_dot(H, d, r, g);
        group_sync<NTW>();
        const double sy = sh.red[0];
        bool pass;
        double rho;
        if constexpr (NTW == 32) {
            pass = sy > 1e-12 * sqrt(sh.red[1]) * sqrt(sh.red[2]);
            rho = 1.0 / sy;
            if (pass) {
                const double v = d > kDotSplit ? warp_split_dot(g, pv, d, tid)
                                               : (tid == 0 ? ordered_dot(g, pv, d) : 0.0);
                if (tid == 0) sh.red[3] = v;
                group_sync<NTW>();
            }
        } else {
            // the scalars of the test and the update on four sub-partitions
            // at once, each formed by one thread: y'Hy on the warp of role 0
            // (whether or not the pair passes), |s|, |y| and 1/y's on the
            // warps of roles 32, 64 and NT - 32
            if (d > kDotSplit) {
                if (tid < 32) {
                    const double v = warp_split_dot(g, pv, d, tid);
                    if (tid == 0) sh.red[3] = v;
                }
            } else if (tid == 0) {
                sh.red[3] = ordered_dot(g, pv, d);
            }
            if (tid == 32) sh.red[4] = sqrt(sh.red[1]);
            if (tid == 64) sh.red[5] = sqrt(sh.red[2]);
            if (tid == NT - 32) sh.red[6] = 1.0 / sy;
            group_sync<NTW>();
            pass = sy > 1e-12 * sh.red[4] * sh.red[5];
            rho = sh.red[6];
        }
        if (pass) {
            const double b2 = rho * rho * sh.red[3] + rho;
            const T rt = T(rho), bt = T(b2);
            // A = b2 s - rho Hy and B = -rho s (in the spent scratch rows)
            for (int r = tid; r < d; r += NT) {
                sc0[r] = (double)mv_fma(bt, sv[r], -(rt * pv[r]));
                sc1[r] = (double)(-(rt * sv[r]));
            }
            group_sync<NTW>();
            // the elements r <= c (H stays symmetric)
            for (int t = tid; t < nu; t += NT) {
                int r, c;
                tri_pair(t, d, r, c);
                const int e = tri_off(r, d) + c - r;
                H[e] = mv_fma(sv[c], T(sc0[r]), mv_fma(pv[c], T(sc1[r]), H[e]));
            }
        }
        // x, g <- x_new, g_new in the same phase (the update reads neither;
        // y, kept in g, was last read by y'Hy before the previous barrier)
        for (int j = tid; j < d; j += NT) {
            x[j] = xn[j];
            g[j] = gn[j];
        }
        stalled = stalled_step<T>(f0, fn);
        f0 = fn;
        ++k;
        group_sync<NTW>();
    }
    if (tid == 0) sh.red[0] = final_value<OBJ>(x, d, f0);
    group_sync<NTW>();
    for (int j = tid; j < d; j += NT) io.x_out[s * d + j] = (double)x[j];
    if (tid == 0) {
        if (io.f_out) io.f_out[s] = sh.red[0];
        if (io.gnorm_out) io.gnorm_out[s] = gnorm;
        if (io.status_out) io.status_out[s] = status;
        if (io.iters_out) io.iters_out[s] = k;
        atomicAdd(&ctrl->total_iters, (unsigned long long)k);
        atomicAdd(&ctrl->total_feval, (unsigned long long)feval);
        if (!use_stop && status == ZEUS_RUN_CONVERGED) atomicAdd(&ctrl->n_conv, 1ull);
    }
    group_sync<NTW>();
}

// Roles rotate with the block index so that the thread doing the serial
// work (ordered sums, tests) sits in a different warp, hence on a different
// SM sub-partition, in each of the blocks sharing an SM.
__device__ __forceinline__ int wide_role(int nt) {
    const int lead = (32 * (int)blockIdx.x) % nt;
    return ((int)threadIdx.x + nt - lead) % nt;
}

// ---- launch-planning helpers (host)
inline size_t narrow_stride(int d) {
    size_t st = (size_t)d * d + 6 * (size_t)d;
    if ((st & 1) == 0) st += 1;  // odd: the 32 starts of a warp fall in distinct banks
    return st;
}

// trials a chunk of the block-per-start line search evaluates at once (up
// to L + 1: the trials and the point after the last halving); nt threads
// carry the start
__host__ __device__ inline int wide_trials(int d, int L, int nt = kWideThreads) {
    int W = (4 * nt) / (d > 0 ? d : 1);
    if (W < 1) W = 1;
    if (W > 64) W = 64;
    if (W > L + 1) W = L + 1;
    return W;
}

inline size_t wide_smem(int d, int W, int L, size_t tsize) {
    return wide_t_bytes(d, tsize) +
           sizeof(double) * (2 * (size_t)d + 2 * (size_t)W * d + W + L + 1);
}

}  // namespace zeus
