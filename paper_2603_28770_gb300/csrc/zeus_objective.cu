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
            fv = adjoint<OBJ, T>(xi, d, gi, grp);
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
    const int G = lanes_for_dim(d, 0);
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
    switch (obj) {
        ZEUS_OBJ_CASE(ZEUS_OBJ_ROSENBROCK)
        ZEUS_OBJ_CASE(ZEUS_OBJ_RASTRIGIN)
        ZEUS_OBJ_CASE(ZEUS_OBJ_ACKLEY)
        ZEUS_OBJ_CASE(ZEUS_OBJ_GOLDSTEIN_PRICE)
        default:
            ZEUS_OBJ_CASE(ZEUS_OBJ_QUADRATIC)
    }
#undef ZEUS_OBJ_CASE
    return cudaGetLastError();
}

cudaError_t launch_objective(int obj, int d, long long n, const double* x, double* f, double* g,
                             int grad_mode, cudaStream_t st) {
    return objective_go<double>(obj, d, n, x, f, g, grad_mode, st);
}

cudaError_t launch_objective_f32(int obj, int d, long long n, const float* x, float* f, float* g,
                                 int grad_mode, cudaStream_t st) {
    return objective_go<float>(obj, d, n, x, f, g, grad_mode, st);
}

}  // namespace zeus
