/*
 * zeus_user.cuh -- objectives defined by the user of libzeus (CUDA C++;
 * this header is not part of the C ABI of zeus.h).
 *
 * Zeus takes the objective f as one function written for any scalar type
 * and differentiates it by evaluating it on dual numbers: forward mode,
 * pass i seeds the tangent of x_i with 1 and reads df/dx_i off the result
 * (Section IV-A, Alg. 5).  libzeus keeps that contract for objectives beyond
 * its built-in test functions.  A plug-in header, compiled into the library
 * by its build (the default plug-in is csrc/zeus_user_objectives.cuh of the
 * package; another one is chosen at build time), defines ZEUS_USER_COUNT
 * (0..ZEUS_USER_MAX) and, for K = 0 .. ZEUS_USER_COUNT - 1,
 *
 *     template <> struct zeus_user::objective<K> {
 *         static constexpr const char* name = "...";  // zeus_user_objective_info
 *         static constexpr int min_dim = 1;           // smallest d accepted
 *         static constexpr int max_dim = 0;           // largest d; 0 = no limit
 *         template <class S, class X>
 *         __device__ static S eval(const X& x, int d);
 *     };
 *
 * Every entry point of zeus.h then takes objective ZEUS_OBJ_USER + K.
 *
 * In eval, x(j) returns coordinate j (0 <= j < d) as S, where S is
 *   float or double            for values (the FP32 and FP64 forms), and
 *   zeus_user::dual<T>, zeus_user::duals<T, N>  for derivatives (T float
 *                              or double; duals carries N tangents, so
 *                              that one evaluation gives N components of
 *                              the gradient: each tangent goes through the
 *                              same operations as in its own pass of
 *                              Alg. 5, and the results are the same bits).
 * Write f with + - * / between two S or an S and its scalar type
 * (scalar_t<S>), S(c) for constants, and the functions below, which are
 * defined for all of these types.  Branch on value(s) only.  eval is called by
 * one thread for the whole point: its loops run in index order.
 *
 * Limits: gradients are forward-mode only (ZEUS_GRAD_ADJOINT needs a
 * hand-written reverse sweep and returns ZEUS_EUNSUPPORTED for a user
 * objective), and d is limited to the forms that hold a start's inverse
 * Hessian in shared memory (a plan that would stream H through device
 * memory, or use L-BFGS, returns ZEUS_EUNSUPPORTED).  Values and
 * derivatives use CUDA's double and single precision math functions.
 */
#pragma once

#include <cuda_runtime.h>
#include <math.h>

namespace zeus_user {

template <int K>
struct objective;  // specialised by the plug-in header

// value and tangent (derivative along the seeded direction)
template <class T>
struct dual {
    T v;
    T t;

    dual() = default;
    __host__ __device__ constexpr dual(T value, T tangent = T(0)) : v(value), t(tangent) {}

    friend __host__ __device__ dual operator+(dual a, dual b) { return dual(a.v + b.v, a.t + b.t); }
    friend __host__ __device__ dual operator-(dual a, dual b) { return dual(a.v - b.v, a.t - b.t); }
    friend __host__ __device__ dual operator*(dual a, dual b) {
        return dual(a.v * b.v, a.t * b.v + a.v * b.t);
    }
    friend __host__ __device__ dual operator/(dual a, dual b) {
        return dual(a.v / b.v, (a.t * b.v - a.v * b.t) / (b.v * b.v));
    }
    friend __host__ __device__ dual operator-(dual a) { return dual(-a.v, -a.t); }

    // with a scalar (a constant: its tangent is zero)
    friend __host__ __device__ dual operator+(dual a, T s) { return dual(a.v + s, a.t); }
    friend __host__ __device__ dual operator+(T s, dual a) { return dual(s + a.v, a.t); }
    friend __host__ __device__ dual operator-(dual a, T s) { return dual(a.v - s, a.t); }
    friend __host__ __device__ dual operator-(T s, dual a) { return dual(s - a.v, -a.t); }
    friend __host__ __device__ dual operator*(dual a, T s) { return dual(a.v * s, a.t * s); }
    friend __host__ __device__ dual operator*(T s, dual a) { return dual(s * a.v, s * a.t); }
    friend __host__ __device__ dual operator/(dual a, T s) { return dual(a.v / s, a.t / s); }
    friend __host__ __device__ dual operator/(T s, dual a) {
        return dual(s / a.v, -(s * a.t) / (a.v * a.v));
    }

    __host__ __device__ dual& operator+=(dual b) { return *this = *this + b; }
    __host__ __device__ dual& operator-=(dual b) { return *this = *this - b; }
    __host__ __device__ dual& operator*=(dual b) { return *this = *this * b; }
    __host__ __device__ dual& operator/=(dual b) { return *this = *this / b; }
};

// value and N tangents (N seeded directions in one evaluation)
template <class T, int N>
struct duals {
    T v;
    T t[N];

    duals() = default;
    __host__ __device__ duals(T value) : v(value) {
#pragma unroll
        for (int q = 0; q < N; ++q) t[q] = T(0);
    }

    friend __host__ __device__ duals operator+(duals a, duals b) {
        a.v = a.v + b.v;
#pragma unroll
        for (int q = 0; q < N; ++q) a.t[q] = a.t[q] + b.t[q];
        return a;
    }
    friend __host__ __device__ duals operator-(duals a, duals b) {
        a.v = a.v - b.v;
#pragma unroll
        for (int q = 0; q < N; ++q) a.t[q] = a.t[q] - b.t[q];
        return a;
    }
    friend __host__ __device__ duals operator*(duals a, duals b) {
        duals r;
        r.v = a.v * b.v;
#pragma unroll
        for (int q = 0; q < N; ++q) r.t[q] = a.t[q] * b.v + a.v * b.t[q];
        return r;
    }
    friend __host__ __device__ duals operator/(duals a, duals b) {
        duals r;
        r.v = a.v / b.v;
        const T bb = b.v * b.v;
#pragma unroll
        for (int q = 0; q < N; ++q) r.t[q] = (a.t[q] * b.v - a.v * b.t[q]) / bb;
        return r;
    }
    friend __host__ __device__ duals operator-(duals a) {
        a.v = -a.v;
#pragma unroll
        for (int q = 0; q < N; ++q) a.t[q] = -a.t[q];
        return a;
    }
    friend __host__ __device__ duals operator+(duals a, T s) {
        a.v = a.v + s;
        return a;
    }
    friend __host__ __device__ duals operator+(T s, duals a) {
        a.v = s + a.v;
        return a;
    }
    friend __host__ __device__ duals operator-(duals a, T s) {
        a.v = a.v - s;
        return a;
    }
    friend __host__ __device__ duals operator-(T s, duals a) {
        a.v = s - a.v;
#pragma unroll
        for (int q = 0; q < N; ++q) a.t[q] = -a.t[q];
        return a;
    }
    friend __host__ __device__ duals operator*(duals a, T s) {
        a.v = a.v * s;
#pragma unroll
        for (int q = 0; q < N; ++q) a.t[q] = a.t[q] * s;
        return a;
    }
    friend __host__ __device__ duals operator*(T s, duals a) {
        a.v = s * a.v;
#pragma unroll
        for (int q = 0; q < N; ++q) a.t[q] = s * a.t[q];
        return a;
    }
    friend __host__ __device__ duals operator/(duals a, T s) {
        a.v = a.v / s;
#pragma unroll
        for (int q = 0; q < N; ++q) a.t[q] = a.t[q] / s;
        return a;
    }
    friend __host__ __device__ duals operator/(T s, duals a) {
        duals r;
        r.v = s / a.v;
        const T aa = a.v * a.v;
#pragma unroll
        for (int q = 0; q < N; ++q) r.t[q] = -(s * a.t[q]) / aa;
        return r;
    }

    __host__ __device__ duals& operator+=(duals b) { return *this = *this + b; }
    __host__ __device__ duals& operator-=(duals b) { return *this = *this - b; }
    __host__ __device__ duals& operator*=(duals b) { return *this = *this * b; }
    __host__ __device__ duals& operator/=(duals b) { return *this = *this / b; }
};

// the scalar type under S
template <class S>
struct scalar_of {
    using type = S;
};
template <class T>
struct scalar_of<dual<T>> {
    using type = T;
};
template <class T, int N>
struct scalar_of<duals<T, N>> {
    using type = T;
};
template <class S>
using scalar_t = typename scalar_of<S>::type;

__host__ __device__ inline float value(float a) { return a; }
__host__ __device__ inline double value(double a) { return a; }
template <class T>
__host__ __device__ inline T value(dual<T> a) {
    return a.v;
}
template <class T, int N>
__host__ __device__ inline T value(const duals<T, N>& a) {
    return a.v;
}

// elementary functions on the scalar types (CUDA's math library)
__device__ inline float sin(float a) { return ::sinf(a); }
__device__ inline double sin(double a) { return ::sin(a); }
__device__ inline float cos(float a) { return ::cosf(a); }
__device__ inline double cos(double a) { return ::cos(a); }
__device__ inline float exp(float a) { return ::expf(a); }
__device__ inline double exp(double a) { return ::exp(a); }
__device__ inline float log(float a) { return ::logf(a); }
__device__ inline double log(double a) { return ::log(a); }
__device__ inline float sqrt(float a) { return ::sqrtf(a); }
__device__ inline double sqrt(double a) { return ::sqrt(a); }
__device__ inline float tanh(float a) { return ::tanhf(a); }
__device__ inline double tanh(double a) { return ::tanh(a); }
__device__ inline void sincos(float a, float* s, float* c) { ::sincosf(a, s, c); }
__device__ inline void sincos(double a, double* s, double* c) { ::sincos(a, s, c); }

// ... and on duals, by the chain rule: (f(v), f'(v) t)
template <class T>
__device__ inline dual<T> sin(dual<T> a) {
    T s, c;
    sincos(a.v, &s, &c);
    return dual<T>(s, c * a.t);
}
template <class T>
__device__ inline dual<T> cos(dual<T> a) {
    T s, c;
    sincos(a.v, &s, &c);
    return dual<T>(c, -s * a.t);
}
template <class T>
__device__ inline dual<T> exp(dual<T> a) {
    const T e = exp(a.v);
    return dual<T>(e, e * a.t);
}
template <class T>
__device__ inline dual<T> log(dual<T> a) {
    return dual<T>(log(a.v), a.t / a.v);
}
// sqrt: tangent 0 at 0 (the one-sided derivative is infinite there)
template <class T>
__device__ inline dual<T> sqrt(dual<T> a) {
    const T r = sqrt(a.v);
    return dual<T>(r, r > T(0) ? a.t / (T(2) * r) : T(0));
}
template <class T>
__device__ inline dual<T> tanh(dual<T> a) {
    const T h = tanh(a.v);
    return dual<T>(h, (T(1) - h * h) * a.t);
}

// ... and on N tangents at once, each as in its own pass
template <class T, int N>
__device__ inline duals<T, N> sin(duals<T, N> a) {
    T s, c;
    sincos(a.v, &s, &c);
    a.v = s;
#pragma unroll
    for (int q = 0; q < N; ++q) a.t[q] = c * a.t[q];
    return a;
}
template <class T, int N>
__device__ inline duals<T, N> cos(duals<T, N> a) {
    T s, c;
    sincos(a.v, &s, &c);
    a.v = c;
#pragma unroll
    for (int q = 0; q < N; ++q) a.t[q] = -s * a.t[q];
    return a;
}
template <class T, int N>
__device__ inline duals<T, N> exp(duals<T, N> a) {
    const T e = exp(a.v);
    a.v = e;
#pragma unroll
    for (int q = 0; q < N; ++q) a.t[q] = e * a.t[q];
    return a;
}
template <class T, int N>
__device__ inline duals<T, N> log(duals<T, N> a) {
    const T v = a.v;
    a.v = log(v);
#pragma unroll
    for (int q = 0; q < N; ++q) a.t[q] = a.t[q] / v;
    return a;
}
template <class T, int N>
__device__ inline duals<T, N> sqrt(duals<T, N> a) {
    const T r = sqrt(a.v);
    a.v = r;
#pragma unroll
    for (int q = 0; q < N; ++q) a.t[q] = r > T(0) ? a.t[q] / (T(2) * r) : T(0);
    return a;
}
template <class T, int N>
__device__ inline duals<T, N> tanh(duals<T, N> a) {
    const T h = tanh(a.v);
    a.v = h;
#pragma unroll
    for (int q = 0; q < N; ++q) a.t[q] = (T(1) - h * h) * a.t[q];
    return a;
}

// a^n for n >= 0 by repeated multiplication (any S)
template <class S>
__device__ inline S ipow(S a, int n) {
    S r = S(1);
    for (int i = 0; i < n; ++i) r = r * a;
    return r;
}

}  // namespace zeus_user
