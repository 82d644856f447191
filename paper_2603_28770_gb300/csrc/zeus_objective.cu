// zeus_objective.cu -- f and its gradient at n points (Section V-B
// objectives), by forward-mode dual passes (Alg. 5) or the reverse-mode
// adjoint, in FP64 or FP32.  One group of G lanes per point.
#include "zeus_device.cuh"
#include "zeus_internal.h"

namespace zeus {

constexpr int kObjThreads = 128;

template <int OBJ, int GRAD, class T>
__global__ void __launch_bounds__(kObjThreads)
    objective_kernel(const int d, const long long n, const int G, const T* __restrict__ x,
                     T* __restrict__ f, T* __restrict__ g) {
    const Group grp(G);
    const long long i = ((long long)blockIdx.x * blockDim.x + threadIdx.x) / G;
    if (i >= n) return;
    const T* xi = x + i * d;
    T fv;
    if (g) {
        T* gi = g + i * d;
        if (GRAD == ZEUS_GRAD_FORWARD) {
            T f0 = T(0);
            for (int k = grp.lane; k < d; k += G) {
                const Dual<T> r = forward_pass<OBJ, T>(xi, d, k);
                gi[k] = r.b;
                if (k == 0) f0 = r.a;
            }
            fv = grp.bcast(f0);
        } else {
            AdjShared a;
            if (grp.lane == 0) a = adjoint_prep<OBJ, T>(xi, d);
            a.c1 = grp.bcast(a.c1);
            a.c2 = grp.bcast(a.c2);
            for (int k = grp.lane; k < d; k += G) gi[k] = adjoint_component<OBJ, T>(xi, d, k, a);
            Part<double> q = value_partial<OBJ, T, double>(xi, d, grp.lane, G);
            q.s0 = grp.sum(q.s0);
            if (OBJ == ZEUS_OBJ_ACKLEY) q.s1 = grp.sum(q.s1);
            fv = T(value_finish<OBJ, double>(q, d));
        }
    } else {
        Part<double> q = value_partial<OBJ, T, double>(xi, d, grp.lane, G);
        q.s0 = grp.sum(q.s0);
        if (OBJ == ZEUS_OBJ_ACKLEY) q.s1 = grp.sum(q.s1);
        fv = T(value_finish<OBJ, double>(q, d));
    }
    if (grp.lane == 0 && f) f[i] = fv;
}

template <class T>
static cudaError_t objective_go(int obj, int d, long long n, const T* x, T* f, T* g, int grad,
                                cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    const int G = lanes_for_dim(d);
    const long long threads = n * G;
    const unsigned blocks = (unsigned)((threads + kObjThreads - 1) / kObjThreads);
#define ZEUS_OBJ_CASE(O)                                                                    \
    case O:                                                                                 \
        if (grad == ZEUS_GRAD_ADJOINT)                                                      \
            objective_kernel<O, ZEUS_GRAD_ADJOINT, T><<<blocks, kObjThreads, 0, st>>>(d, n, G, x, \
                                                                                   f, g);   \
        else                                                                                \
            objective_kernel<O, ZEUS_GRAD_FORWARD, T><<<blocks, kObjThreads, 0, st>>>(d, n, G, x, \
                                                                                   f, g);   \
        break;
    // user objectives: forward mode only (the entry points reject the adjoint)
#define ZEUS_UCASE(O)                                                                          \
    case O:                                                                                    \
        objective_kernel<O, ZEUS_GRAD_FORWARD, T><<<blocks, kObjThreads, 0, st>>>(d, n, G, x, f, \
                                                                                 g);           \
        break;
    switch (obj) {
        ZEUS_USER_EACH(ZEUS_UCASE)
        ZEUS_OBJ_CASE(ZEUS_OBJ_ROSENBROCK)
        ZEUS_OBJ_CASE(ZEUS_OBJ_RASTRIGIN)
        ZEUS_OBJ_CASE(ZEUS_OBJ_ACKLEY)
        ZEUS_OBJ_CASE(ZEUS_OBJ_GOLDSTEIN_PRICE)
        default:
            ZEUS_OBJ_CASE(ZEUS_OBJ_QUADRATIC)
    }
#undef ZEUS_OBJ_CASE
#undef ZEUS_UCASE
    return cudaGetLastError();
}

__global__ void math_kernel(const int fn, const long long n, const double* __restrict__ x,
                            double* __restrict__ y0, double* __restrict__ y1) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double v = x[i];
    double a = 0.0, b = 0.0;
    if (fn == 0) {
        sincos2pi(v, &a, &b);
    } else if (fn == 1) {
        a = exp_cw(v);
    } else if (fn == 2) {
        sincospi(2.0 * v, &a, &b);
    } else if (fn == 3) {
        a = exp(v);
    } else {
        a = cos2pi(v);
    }
    y0[i] = a;
    if (y1 && (fn == 0 || fn == 2)) y1[i] = b;
}

cudaError_t launch_math(int fn, long long n, const double* x, double* y0, double* y1,
                        cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    math_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(fn, n, x, y0, y1);
    return cudaGetLastError();
}

template <int K>
static void user_meta_of(const char** name, int* min_dim, int* max_dim) {
    *name = zeus_user::objective<K>::name;
    *min_dim = zeus_user::objective<K>::min_dim;
    *max_dim = zeus_user::objective<K>::max_dim;
}

int user_objective_meta(int k, const char** name, int* min_dim, int* max_dim) {
    switch (ZEUS_OBJ_USER + k) {
#define ZEUS_UCASE(O)                                                \
    case O:                                                          \
        user_meta_of<O - ZEUS_OBJ_USER>(name, min_dim, max_dim);     \
        return 1;
        ZEUS_USER_EACH(ZEUS_UCASE)
#undef ZEUS_UCASE
        default:
            return 0;
    }
}

int user_objective_count() { return ZEUS_USER_COUNT; }

cudaError_t launch_objective(int obj, int d, long long n, const double* x, double* f, double* g,
                             int grad_mode, cudaStream_t st) {
    return objective_go<double>(obj, d, n, x, f, g, grad_mode, st);
}

cudaError_t launch_objective_f32(int obj, int d, long long n, const float* x, float* f, float* g,
                                 int grad_mode, cudaStream_t st) {
    return objective_go<float>(obj, d, n, x, f, g, grad_mode, st);
}

}  // namespace zeus
