// zeus_device.cuh -- device building blocks shared by the Zeus kernels:
// Philox4x64-10, lane groups, dual numbers and the Section V-B objectives
// (value sweep, forward-mode dual passes of Alg. 5, reverse-mode adjoint).
#pragma once

#include <cuda_runtime.h>
#include <math_constants.h>
#include <stdint.h>

#include "zeus.h"

namespace zeus {

// ---------------------------------------------------------------------------
// Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC'11).  Counter-based: the
// draw of (phase, particle, dimension j) is word j%4 of the block with
// counter (j/4, particle, problem, phase) under key (seed, 0), so no RNG
// state is stored (this replaces the cuRAND states of Section IV-A).
// ---------------------------------------------------------------------------
struct U64x4 {
    uint64_t v[4];
};

__device__ __forceinline__ U64x4 philox4x64_10(uint64_t c0, uint64_t c1, uint64_t c2,
                                               uint64_t c3, uint64_t k0, uint64_t k1) {
    const uint64_t M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
    const uint64_t W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) {
            k0 += W0;
            k1 += W1;
        }
        const uint64_t lo0 = M0 * c0, hi0 = __umul64hi(M0, c0);
        const uint64_t lo1 = M1 * c2, hi1 = __umul64hi(M1, c2);
        const uint64_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
    }
    U64x4 o;
    o.v[0] = c0;
    o.v[1] = c1;
    o.v[2] = c2;
    o.v[3] = c3;
    return o;
}

// top 53 bits -> [0, 1)
__device__ __forceinline__ double u01(uint64_t w) { return (double)(w >> 11) * 0x1.0p-53; }

// ---------------------------------------------------------------------------
// A group of G consecutive lanes (G = 1, 2, 4, 8, 16, 32) of one warp works
// on one start.  Reductions are xor-butterflies, so every lane of the group
// ends with the bitwise-identical total and takes the same branches.
// ---------------------------------------------------------------------------
struct Group {
    int lane;       // 0 .. G-1
    int G;
    unsigned mask;  // the group's lanes within the warp
    __device__ __forceinline__ explicit Group(int G_) {
        const int wl = threadIdx.x & 31;
        G = G_;
        lane = wl & (G_ - 1);
        mask = (G_ == 32) ? 0xffffffffu : (((1u << G_) - 1u) << (wl & ~(G_ - 1)));
    }
    __device__ __forceinline__ void sync() const {
        if (G > 1) __syncwarp(mask);
    }
    template <class T>
    __device__ __forceinline__ T sum(T v) const {
        for (int o = G >> 1; o > 0; o >>= 1) v += __shfl_xor_sync(mask, v, o, G);
        return v;
    }
    template <class T>
    __device__ __forceinline__ T bcast(T v) const {
        return G > 1 ? __shfl_sync(mask, v, 0, G) : v;
    }
};

// ---------------------------------------------------------------------------
// Dual numbers a + b eps, eps^2 = 0 (Section III-C).
// ---------------------------------------------------------------------------
template <class T>
struct Dual {
    T a, b;
};
template <class T>
__device__ __forceinline__ Dual<T> dmk(T a, T b) {
    Dual<T> r;
    r.a = a;
    r.b = b;
    return r;
}
template <class T>
__device__ __forceinline__ Dual<T> operator+(Dual<T> x, Dual<T> y) { return dmk(x.a + y.a, x.b + y.b); }
template <class T>
__device__ __forceinline__ Dual<T> operator-(Dual<T> x, Dual<T> y) { return dmk(x.a - y.a, x.b - y.b); }
template <class T>
__device__ __forceinline__ Dual<T> operator*(Dual<T> x, Dual<T> y) {
    return dmk(x.a * y.a, x.a * y.b + x.b * y.a);
}
template <class T>
__device__ __forceinline__ Dual<T> operator*(T s, Dual<T> x) { return dmk(s * x.a, s * x.b); }

// sin(pi x), cos(pi x) in the working precision
__device__ __forceinline__ void sc_pi(double x, double* s, double* c) { sincospi(x, s, c); }
__device__ __forceinline__ void sc_pi(float x, float* s, float* c) { sincospif(x, s, c); }
__device__ __forceinline__ double c_pi(double x) { return cospi(x); }
__device__ __forceinline__ float c_pi(float x) { return cospif(x); }
__device__ __forceinline__ double xexp(double x) { return exp(x); }
__device__ __forceinline__ float xexp(float x) { return expf(x); }
__device__ __forceinline__ double xsqrt(double x) { return sqrt(x); }
__device__ __forceinline__ float xsqrt(float x) { return sqrtf(x); }

template <class T>
struct Consts;
template <>
struct Consts<double> {
    static __device__ __forceinline__ double two_pi() { return 6.283185307179586476925286766559; }
    static __device__ __forceinline__ double e() { return 2.718281828459045235360287471352; }
};
template <>
struct Consts<float> {
    static __device__ __forceinline__ float two_pi() { return 6.283185307179586476925286766559f; }
    static __device__ __forceinline__ float e() { return 2.718281828459045235360287471352f; }
};

// ---------------------------------------------------------------------------
// Objectives (Section V-B).  Three evaluation forms:
//  value_partial : lanes of a group split the terms; the partial sums are
//                  accumulated in A (double, also in the FP32 form, so the
//                  Armijo test sees an FP64 sum of FP32 terms) and combined
//                  by value_finish after the group reduction.
//  forward_pass  : Alg. 5 pass i -- the objective evaluated on dual numbers
//                  with the tangent of x_i seeded to 1; returns (f, df/dx_i).
//                  The value sweep is repeated in every pass as in Alg. 5;
//                  tangent arithmetic on terms whose inputs all carry a zero
//                  tangent is skipped (it would only add exact zeros).
//  adjoint       : value and full gradient from one forward sweep and one
//                  reverse sweep; lanes split the coordinates.
// x points to the start's coordinates (unit stride).
// ---------------------------------------------------------------------------
template <class A>
struct Part {
    A s0, s1;
};

template <int OBJ, class T, class A>
__device__ __forceinline__ Part<A> value_partial(const T* x, int d, int lane, int G) {
    Part<A> p;
    p.s0 = A(0);
    p.s1 = A(0);
    if (OBJ == ZEUS_OBJ_ROSENBROCK) {
        for (int i = lane; i < d - 1; i += G) {
            const T xi = x[i];
            const T a = T(1) - xi;
            const T b = x[i + 1] - xi * xi;
            p.s0 += A(a * a + T(100) * (b * b));
        }
    } else if (OBJ == ZEUS_OBJ_RASTRIGIN) {
        if (lane == 0) p.s0 = A(10) * A(d);
        for (int i = lane; i < d; i += G) {
            const T xi = x[i];
            p.s0 += A(xi * xi - T(10) * c_pi(T(2) * xi));
        }
    } else if (OBJ == ZEUS_OBJ_ACKLEY) {
        for (int i = lane; i < d; i += G) {
            const T xi = x[i];
            p.s0 += A(xi * xi);
            p.s1 += A(c_pi(T(2) * xi));
        }
    } else if (OBJ == ZEUS_OBJ_GOLDSTEIN_PRICE) {
        if (lane == 0) {
            const T x1 = x[0], x2 = x[1];
            const T t = (x1 + x2) + T(1);
            const T pa = T(19) - T(14) * x1 + T(3) * (x1 * x1) - T(14) * x2 + T(6) * (x1 * x2) +
                         T(3) * (x2 * x2);
            const T a = T(1) + (t * t) * pa;
            const T u = T(2) * x1 - T(3) * x2;
            const T pb = T(18) - T(32) * x1 + T(12) * (x1 * x1) + T(48) * x2 - T(36) * (x1 * x2) +
                         T(27) * (x2 * x2);
            const T b = T(30) + (u * u) * pb;
            p.s0 = A(a * b);
        }
    } else {  // ZEUS_OBJ_QUADRATIC
        for (int i = lane; i < d; i += G) {
            const T xi = x[i];
            p.s0 += A(T(0.5) * T(i + 1) * (xi * xi));
        }
    }
    return p;
}

template <int OBJ, class A>
__device__ __forceinline__ A value_finish(Part<A> p, int d) {
    if (OBJ == ZEUS_OBJ_ACKLEY) {
        const A t1 = A(-20) * xexp(A(-0.2) * xsqrt(p.s0 / A(d)));
        const A t2 = xexp(p.s1 / A(d));
        return (t1 - t2) + (A(20) + Consts<A>::e());
    }
    return p.s0;
}

// Alg. 5, one pass: f on duals with seed e_i.  Returns (value, df/dx_i).
template <int OBJ, class T>
__device__ __forceinline__ Dual<T> forward_pass(const T* x, int d, int i) {
    if (OBJ == ZEUS_OBJ_ROSENBROCK) {
        T val = T(0), tan = T(0);
        for (int j = 0; j < d - 1; ++j) {
            const T xj = x[j], xk = x[j + 1];
            if (j == i || j + 1 == i) {
                const Dual<T> u = dmk(xj, T(j == i ? 1 : 0));
                const Dual<T> v = dmk(xk, T(j + 1 == i ? 1 : 0));
                const Dual<T> a = dmk(T(1), T(0)) - u;
                const Dual<T> b = v - u * u;
                const Dual<T> t = a * a + T(100) * (b * b);
                val += t.a;
                tan += t.b;
            } else {
                const T a = T(1) - xj;
                const T b = xk - xj * xj;
                val += a * a + T(100) * (b * b);
            }
        }
        return dmk(val, tan);
    } else if (OBJ == ZEUS_OBJ_RASTRIGIN) {
        T val = T(10) * T(d), tan = T(0);
        for (int j = 0; j < d; ++j) {
            const T xj = x[j];
            if (j == i) {
                T s, c;
                sc_pi(T(2) * xj, &s, &c);
                // x^2 - 10 cos(2 pi x) on duals with tangent 1
                const T tx2 = xj + xj;
                const T tcos = -s * Consts<T>::two_pi();
                val += xj * xj - T(10) * c;
                tan += tx2 - T(10) * tcos;
            } else {
                val += xj * xj - T(10) * c_pi(T(2) * xj);
            }
        }
        return dmk(val, tan);
    } else if (OBJ == ZEUS_OBJ_ACKLEY) {
        T s1 = T(0), s2 = T(0), t1 = T(0), t2 = T(0);
        for (int j = 0; j < d; ++j) {
            const T xj = x[j];
            if (j == i) {
                T s, c;
                sc_pi(T(2) * xj, &s, &c);
                s1 += xj * xj;
                t1 += xj + xj;
                s2 += c;
                t2 += -s * Consts<T>::two_pi();
            } else {
                s1 += xj * xj;
                s2 += c_pi(T(2) * xj);
            }
        }
        const T invd = T(1) / T(d);
        // u = s1/d, r = sqrt(u) (tangent 0 at u = 0), e1 = exp(-0.2 r)
        const T u = s1 * invd, ut = t1 * invd;
        const T r = xsqrt(u);
        const T rt = r > T(0) ? ut / (T(2) * r) : T(0);
        const T e1 = xexp(T(-0.2) * r);
        const T e1t = e1 * (T(-0.2) * rt);
        const T e2 = xexp(s2 * invd);
        const T e2t = e2 * (t2 * invd);
        const T val = (T(-20) * e1 - e2) + (T(20) + Consts<T>::e());
        const T tan = T(-20) * e1t - e2t;
        return dmk(val, tan);
    } else if (OBJ == ZEUS_OBJ_GOLDSTEIN_PRICE) {
        const Dual<T> x1 = dmk(x[0], T(i == 0 ? 1 : 0));
        const Dual<T> x2 = dmk(x[1], T(i == 1 ? 1 : 0));
        const Dual<T> one = dmk(T(1), T(0));
        const Dual<T> t = (x1 + x2) + one;
        const Dual<T> pa = dmk(T(19), T(0)) - T(14) * x1 + T(3) * (x1 * x1) - T(14) * x2 +
                           T(6) * (x1 * x2) + T(3) * (x2 * x2);
        const Dual<T> a = one + (t * t) * pa;
        const Dual<T> u = T(2) * x1 - T(3) * x2;
        const Dual<T> pb = dmk(T(18), T(0)) - T(32) * x1 + T(12) * (x1 * x1) + T(48) * x2 -
                           T(36) * (x1 * x2) + T(27) * (x2 * x2);
        const Dual<T> b = dmk(T(30), T(0)) + (u * u) * pb;
        return a * b;
    } else {  // quadratic
        T val = T(0), tan = T(0);
        for (int j = 0; j < d; ++j) {
            const T xj = x[j];
            const T c = T(0.5) * T(j + 1);
            val += c * (xj * xj);
            if (j == i) tan += c * (xj + xj);
        }
        return dmk(val, tan);
    }
}

// Reverse-mode adjoint: lanes split coordinates, partial sums reduced over
// the group.  Writes g[j] for the lane's own j (j = lane, lane+G, ...) and
// returns f (identical on every lane of the group).
template <int OBJ, class T, class GRP>
__device__ __forceinline__ T adjoint(const T* x, int d, T* g, const GRP& grp) {
    const int lane = grp.lane, G = grp.G;
    if (OBJ == ZEUS_OBJ_ROSENBROCK) {
        T s = T(0);
        for (int j = lane; j < d; j += G) {
            const T xj = x[j];
            T gj = T(0);
            if (j + 1 < d) {  // term j: (1 - x_j)^2 + 100 (x_{j+1} - x_j^2)^2
                const T a = T(1) - xj;
                const T b = x[j + 1] - xj * xj;
                s += a * a + T(100) * (b * b);
                gj += T(-2) * a - T(400) * xj * b;
            }
            if (j > 0) {  // term j-1 through x_j
                const T xp = x[j - 1];
                const T b = xj - xp * xp;
                gj += T(200) * b;
            }
            g[j] = gj;
        }
        return grp.sum(s);
    } else if (OBJ == ZEUS_OBJ_RASTRIGIN) {
        T s = lane == 0 ? T(10) * T(d) : T(0);
        for (int j = lane; j < d; j += G) {
            const T xj = x[j];
            T sn, c;
            sc_pi(T(2) * xj, &sn, &c);
            s += xj * xj - T(10) * c;
            g[j] = (xj + xj) + T(10) * Consts<T>::two_pi() * sn;
        }
        return grp.sum(s);
    } else if (OBJ == ZEUS_OBJ_ACKLEY) {
        T s1 = T(0), s2 = T(0);
        for (int j = lane; j < d; j += G) {
            const T xj = x[j];
            s1 += xj * xj;
            s2 += c_pi(T(2) * xj);
        }
        s1 = grp.sum(s1);
        s2 = grp.sum(s2);
        const T invd = T(1) / T(d);
        const T r = xsqrt(s1 * invd);
        const T e1 = xexp(T(-0.2) * r);
        const T e2 = xexp(s2 * invd);
        // adjoints of s1 and s2
        const T a1 = r > T(0) ? (T(-20) * e1) * (T(-0.2) / (T(2) * r)) * invd : T(0);
        const T a2 = -e2 * invd;
        for (int j = lane; j < d; j += G) {
            const T xj = x[j];
            T sn, c;
            sc_pi(T(2) * xj, &sn, &c);
            g[j] = a1 * (xj + xj) - a2 * Consts<T>::two_pi() * sn;
        }
        return (T(-20) * e1 - e2) + (T(20) + Consts<T>::e());
    } else if (OBJ == ZEUS_OBJ_GOLDSTEIN_PRICE) {
        T f = T(0);
        if (lane == 0) {
            const T x1 = x[0], x2 = x[1];
            const T t = (x1 + x2) + T(1);
            const T pa = T(19) - T(14) * x1 + T(3) * (x1 * x1) - T(14) * x2 + T(6) * (x1 * x2) +
                         T(3) * (x2 * x2);
            const T a = T(1) + (t * t) * pa;
            const T u = T(2) * x1 - T(3) * x2;
            const T pb = T(18) - T(32) * x1 + T(12) * (x1 * x1) + T(48) * x2 - T(36) * (x1 * x2) +
                         T(27) * (x2 * x2);
            const T b = T(30) + (u * u) * pb;
            f = a * b;
            // reverse sweep: f = a b
            const T da = b, db = a;
            const T dt = da * (T(2) * t * pa), dpa = da * (t * t);
            const T du = db * (T(2) * u * pb), dpb = db * (u * u);
            const T g1 = dt + dpa * (T(-14) + T(6) * x1 + T(6) * x2) + du * T(2) +
                         dpb * (T(-32) + T(24) * x1 - T(36) * x2);
            const T g2 = dt + dpa * (T(-14) + T(6) * x1 + T(6) * x2) + du * T(-3) +
                         dpb * (T(48) - T(36) * x1 + T(54) * x2);
            // lane 0 writes both coordinates; callers sync the group
            // before reading g
            g[0] = g1;
            g[1] = g2;
        }
        return grp.bcast(f);
    } else {
        T s = T(0);
        for (int j = lane; j < d; j += G) {
            const T xj = x[j];
            const T c = T(0.5) * T(j + 1);
            s += c * (xj * xj);
            g[j] = c * (xj + xj);
        }
        return grp.sum(s);
    }
}

}  // namespace zeus
