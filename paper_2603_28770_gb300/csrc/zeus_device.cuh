// zeus_device.cuh -- device building blocks shared by the Zeus kernels:
// Philox4x64-10, lane groups, dual numbers and the Section V-B objectives
// (value sweep, forward-mode dual passes of Alg. 5, reverse-mode adjoint).
#pragma once

#include <cuda_runtime.h>
#include <math_constants.h>
#include <stdint.h>

#include "zeus.h"

// User objectives: the plug-in header named at build time, else the
// default one of the package (contract in zeus_user.cuh).
#ifndef ZEUS_USER_PLUGIN
#define ZEUS_USER_PLUGIN "zeus_user_objectives.cuh"
#endif
#include ZEUS_USER_PLUGIN
#if !defined(ZEUS_USER_COUNT) || ZEUS_USER_COUNT < 0 || ZEUS_USER_COUNT > ZEUS_USER_MAX
#error "the user-objective plug-in must define ZEUS_USER_COUNT in 0..ZEUS_USER_MAX"
#endif

// M(id) once for each user objective id of the plug-in (case labels and
// template arguments at the objective switches)
#define ZEUS_USER_EACH(M) ZEUS_USER_E0(M) ZEUS_USER_E1(M) ZEUS_USER_E2(M) ZEUS_USER_E3(M)
#if ZEUS_USER_COUNT > 0
#define ZEUS_USER_E0(M) M(ZEUS_OBJ_USER + 0)
#else
#define ZEUS_USER_E0(M)
#endif
#if ZEUS_USER_COUNT > 1
#define ZEUS_USER_E1(M) M(ZEUS_OBJ_USER + 1)
#else
#define ZEUS_USER_E1(M)
#endif
#if ZEUS_USER_COUNT > 2
#define ZEUS_USER_E2(M) M(ZEUS_OBJ_USER + 2)
#else
#define ZEUS_USER_E2(M)
#endif
#if ZEUS_USER_COUNT > 3
#define ZEUS_USER_E3(M) M(ZEUS_OBJ_USER + 3)
#else
#define ZEUS_USER_E3(M)
#endif

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

// FP32 form: an iteration whose decrease of f is below what FP32 resolves
// relative to f ends the start (status ZEUS_RUN_STALLED): f_k - f_{k+1} <=
// eps32 max(|f_k|, |f_{k+1}|), eps32 = 2^-23 (a relative-decrease test at
// the working precision; no absolute floor, so runs that still creep
// towards a minimum at f = 0 go on).  Decided at the end of an iteration,
// acted on at the top of the next (after the gradient and target tests), so
// the hand-over point does not change it.
constexpr double kEps32 = 1.1920928955078125e-07;
template <class T>
__device__ __forceinline__ bool stalled_step(double f0, double fn) {
    if (sizeof(T) != 4) return false;
    return !(f0 - fn > kEps32 * fmax(fabs(f0), fabs(fn)));
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

// ---------------------------------------------------------------------------
// FP64 elementary functions of the objectives, written from published
// methods (explicit fused multiply-adds, so the result does not depend on
// compiler contraction):
//  sin/cos(2 pi x): exact argument reduction r = x - rint(x),
//    q = rint(4 r), s = r - q/4 (|s| <= 1/8, every step exact), Taylor
//    series of sin(2 pi s) through s^17 and cos(2 pi s) through s^16 in
//    Horner form in s^2, quarter-turn identities for q.  Coefficients:
//    S_k = (-1)^k (2 pi)^(2k+1)/(2k+1)!, C_k = (-1)^k (2 pi)^(2k)/(2k)!.
//  e^x: Cody & Waite reduction x = k ln2 + r, k = rint(x / ln2),
//    ln2 = L1 + L2 with a 32-bit head L1 (k L1 exact), Taylor series of e^r
//    through r^13 in Horner form, exact scaling by 2^k.
// Cost: sincos 2 rint + 2 add/mul + 17 FMA + 2 mul; e^x 1 rint + 3 +
// 14 FMA (the products by q/4 and by k L1 are exact, so each joins its
// subtraction in one FMA without changing a bit).  FP32 uses CUDA's sincospif / expf.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void sincos2pi(double x, double* sp, double* cp) {
    const double n = rint(x);
    const double r = x - n;
    const double qf = rint(4.0 * r);
    const double s = fma(-0.25, qf, r);  // 0.25 qf is exact: r - qf/4 rounded once, as written
    const int q = ((int)qf) & 3;
    const double z = s * s;
    double ps = 0x1.aaec32af93359p-4, pc = 0x1.20c62c2f2d7f5p-2;
    ps = fma(ps, z, -0x1.6fadb9f155744p-1);
    pc = fma(pc, z, -0x1.b6e24f44b128fp+0);
    ps = fma(ps, z, 0x1.e8f434d018d63p+1);
    pc = fma(pc, z, 0x1.f9d38a3763cc3p+2);
    ps = fma(ps, z, -0x1.e3074fde8871fp+3);
    pc = fma(pc, z, -0x1.a6d1f2a204a8cp+4);
    ps = fma(ps, z, 0x1.50783487ee782p+5);
    pc = fma(pc, z, 0x1.e1f506891babbp+5);
    ps = fma(ps, z, -0x1.32d2cce62bd86p+6);
    pc = fma(pc, z, -0x1.55d3c7e3cbffap+6);
    ps = fma(ps, z, 0x1.466bc6775aae2p+6);
    pc = fma(pc, z, 0x1.03c1f081b5ac4p+6);
    ps = fma(ps, z, -0x1.4abbce625be53p+5);
    pc = fma(pc, z, -0x1.3bd3cc9be45dep+4);
    ps = fma(ps, z, 0x1.921fb54442d18p+2);
    pc = fma(pc, z, 1.0);
    ps = ps * s;
    double so, co;
    if (q == 0) {
        so = ps;
        co = pc;
    } else if (q == 1) {
        so = pc;
        co = -ps;
    } else if (q == 2) {
        so = -ps;
        co = -pc;
    } else {
        so = -pc;
        co = ps;
    }
    *sp = so;
    *cp = co;
}

__device__ __forceinline__ double exp_cw(double x) {
    if (isnan(x)) return x;
    if (x > 709.78) return CUDART_INF;
    if (x < -745.2) return 0.0;
    const double k = rint(x * 0x1.71547652b82fep+0);
    // k L1 is exact (a 32-bit head times |k| < 2^11), so x - k L1 is one rounding
    const double r = fma(-k, 0x1.62e42fee00000p-1, x) - k * 0x1.a39ef35793c76p-33;
    double p = 0x1.6124613a86d09p-33;  // 1/13!
    p = fma(p, r, 0x1.1eed8eff8d898p-29);
    p = fma(p, r, 0x1.ae64567f544e4p-26);
    p = fma(p, r, 0x1.27e4fb7789f5cp-22);
    p = fma(p, r, 0x1.71de3a556c734p-19);
    p = fma(p, r, 0x1.a01a01a01a01ap-16);
    p = fma(p, r, 0x1.a01a01a01a01ap-13);
    p = fma(p, r, 0x1.6c16c16c16c17p-10);
    p = fma(p, r, 0x1.1111111111111p-7);
    p = fma(p, r, 0x1.5555555555555p-5);
    p = fma(p, r, 0x1.5555555555555p-3);
    p = fma(p, r, 0x1.0000000000000p-1);
    p = fma(p, r, 1.0);
    p = fma(p, r, 1.0);
    return ldexp(p, (int)k);
}

// cos(2 pi x) alone, bit for bit the cosine of sincos2pi: the quadrant
// picks per lane which of the two series (sin for odd quarter turns, cos for
// even) the single Horner chain evaluates, so SIMT lanes with different
// quadrants still run one chain (9 FMA instead of 16).
__device__ __forceinline__ double cos2pi(double x) {
    const double n = rint(x);
    const double r = x - n;
    const double qf = rint(4.0 * r);
    const double s = fma(-0.25, qf, r);  // 0.25 qf is exact: r - qf/4 rounded once, as written
    const int q = ((int)qf) & 3;
    const bool odd = (q & 1) != 0;
    const double z = s * s;
    double v = odd ? 0x1.aaec32af93359p-4 : 0x1.20c62c2f2d7f5p-2;
    v = fma(v, z, odd ? -0x1.6fadb9f155744p-1 : -0x1.b6e24f44b128fp+0);
    v = fma(v, z, odd ? 0x1.e8f434d018d63p+1 : 0x1.f9d38a3763cc3p+2);
    v = fma(v, z, odd ? -0x1.e3074fde8871fp+3 : -0x1.a6d1f2a204a8cp+4);
    v = fma(v, z, odd ? 0x1.50783487ee782p+5 : 0x1.e1f506891babbp+5);
    v = fma(v, z, odd ? -0x1.32d2cce62bd86p+6 : -0x1.55d3c7e3cbffap+6);
    v = fma(v, z, odd ? 0x1.466bc6775aae2p+6 : 0x1.03c1f081b5ac4p+6);
    v = fma(v, z, odd ? -0x1.4abbce625be53p+5 : -0x1.3bd3cc9be45dep+4);
    v = fma(v, z, odd ? 0x1.921fb54442d18p+2 : 1.0);
    const double ps = v * s;
    const double w = odd ? ps : v;  // q even: cos series; q odd: sin series times s
    return (q == 0 || q == 3) ? w : -w;
}

// sin(2 pi x), cos(2 pi x) in the working precision
__device__ __forceinline__ void sc_2pi(double x, double* s, double* c) { sincos2pi(x, s, c); }
__device__ __forceinline__ void sc_2pi(float x, float* s, float* c) { sincospif(2.0f * x, s, c); }
__device__ __forceinline__ double c_2pi(double x) { return cos2pi(x); }
__device__ __forceinline__ float c_2pi(float x) { return cospif(2.0f * x); }
__device__ __forceinline__ double xexp(double x) { return exp_cw(x); }
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

// The sums of an objective over its coordinates: left to right for
// d <= kSumSplit; past that 32 chains, chain l over the terms j = l (mod
// 32) left to right with chain 0 starting from the sum's constant, added
// pairwise in a fixed tree (l with l + 16, then l + 8, l + 4, l + 2, l + 1).
// One thread forms them here: the chains in bit-reversed order (0, 16, 8,
// 24, ...), merged as a binary counter does, hold at most five partial sums.
// term(j) returns the two components of term j (s1 is summed if `two`).
constexpr int kSumSplit = 32;

// the split order, out of line so that its partial sums do not weigh on
// the registers of the kernels that mostly take the short path
template <class A, class F>
__device__ __noinline__ Part<A> obj_sum_split(int nt, Part<A> init, bool two, F term) {
    Part<A> q0, q1, q2, q3, q4, v;
    q0.s0 = q0.s1 = q1.s0 = q1.s1 = q2.s0 = q2.s1 = q3.s0 = q3.s1 = q4.s0 = q4.s1 = A(0);
    auto add = [two](Part<A> a, Part<A> b) {
        a.s0 = a.s0 + b.s0;
        if (two) a.s1 = a.s1 + b.s1;
        return a;
    };
#pragma unroll 1
    for (int k = 0; k < 32; ++k) {
        const int l = (int)(__brev((unsigned)k) >> 27);
        if (l == 0) {
            v = init;
        } else {
            v.s0 = A(0);
            v.s1 = A(0);
        }
#pragma unroll 1
        for (int j = l; j < nt; j += 32) {
            const Part<A> t = term(j);
            v.s0 = v.s0 + t.s0;
            if (two) v.s1 = v.s1 + t.s1;
        }
        if (!(k & 1)) { q0 = v; continue; }
        v = add(q0, v);
        if (!(k & 2)) { q1 = v; continue; }
        v = add(q1, v);
        if (!(k & 4)) { q2 = v; continue; }
        v = add(q2, v);
        if (!(k & 8)) { q3 = v; continue; }
        v = add(q3, v);
        if (!(k & 16)) { q4 = v; continue; }
        v = add(q4, v);
    }
    return v;
}

template <class A, class F>
__device__ __forceinline__ Part<A> obj_sum(int d, int nt, Part<A> init, bool two, F term) {
    if (d > kSumSplit) return obj_sum_split<A>(nt, init, two, term);
    Part<A> acc = init;
    for (int j = 0; j < nt; ++j) {
        const Part<A> t = term(j);
        acc.s0 = acc.s0 + t.s0;
        if (two) acc.s1 = acc.s1 + t.s1;
    }
    return acc;
}

// A user objective is one term: f at the whole point, evaluated by one
// thread in the plug-in's own order.  Coordinates reach it through an
// accessor, x(j); duals carry the tangent seeded on coordinate i.
template <int OBJ>
using UserObjective = zeus_user::objective<OBJ - ZEUS_OBJ_USER>;

template <class T>
struct UserAt {
    const T* x;
    __device__ __forceinline__ T operator()(int j) const { return x[j]; }
};
template <class T>
struct UserSeed {
    const T* x;
    int i;
    __device__ __forceinline__ zeus_user::dual<T> operator()(int j) const {
        return zeus_user::dual<T>(x[j], j == i ? T(1) : T(0));
    }
};

// N tangents per evaluation: seeds e_{i0} .. e_{i0+N-1} (those past d
// match no coordinate and stay zero)
template <class T, int N>
struct UserSeeds {
    const T* x;
    int i0;
    __device__ __forceinline__ zeus_user::duals<T, N> operator()(int j) const {
        zeus_user::duals<T, N> r(x[j]);
#pragma unroll
        for (int q = 0; q < N; ++q) r.t[q] = (j - i0 == q) ? T(1) : T(0);
        return r;
    }
};

// The whole gradient of a user objective on one thread: the d passes of
// Alg. 5 taken kUserChunk at a time (vector forward mode).  Each tangent
// goes through the operations of its own pass, so g is the same bits as d
// single passes, while the value part (and its elementary functions) is
// evaluated once per chunk instead of once per pass.
constexpr int kUserChunk = 4;
template <int OBJ, class T>
__device__ __forceinline__ void user_gradient(const T* x, int d, T* g) {
    using V = zeus_user::duals<T, kUserChunk>;
    for (int i0 = 0; i0 < d; i0 += kUserChunk) {
        const V r = UserObjective<OBJ>::template eval<V>(UserSeeds<T, kUserChunk>{x, i0}, d);
#pragma unroll
        for (int q = 0; q < kUserChunk; ++q)
            if (i0 + q < d) g[i0 + q] = r.t[q];
    }
}

template <int OBJ, class T, class A>
__device__ __forceinline__ Part<A> builtin_value_partial(const T* x, int d, int lane, int G) {
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
            p.s0 += A(xi * xi - T(10) * c_2pi(xi));
        }
    } else if (OBJ == ZEUS_OBJ_ACKLEY) {
        for (int i = lane; i < d; i += G) {
            const T xi = x[i];
            p.s0 += A(xi * xi);
            p.s1 += A(c_2pi(xi));
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

template <int OBJ, class T, class A>
__device__ __forceinline__ Part<A> value_partial(const T* x, int d, int lane, int G) {
    if constexpr (OBJ >= ZEUS_OBJ_USER) {
        Part<A> p;
        p.s0 = A(0);
        p.s1 = A(0);
        if (lane == 0) p.s0 = A(UserObjective<OBJ>::template eval<T>(UserAt<T>{x}, d));
        return p;
    } else {
        return builtin_value_partial<OBJ, T, A>(x, d, lane, G);
    }
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
__device__ __forceinline__ Dual<T> builtin_forward_pass(const T* x, int d, int i) {
    // value sums in the order of obj_sum; the tangent sums have at most
    // two non-zero terms, so their order does not change them
    Part<T> zero;
    zero.s0 = zero.s1 = T(0);
    if (OBJ == ZEUS_OBJ_ROSENBROCK) {
        T tan = T(0);
        const Part<T> acc = obj_sum<T>(d, d - 1, zero, false, [&](int j) {
            const T xj = x[j], xk = x[j + 1];
            Part<T> r;
            r.s1 = T(0);
            if (j == i || j + 1 == i) {
                const Dual<T> u = dmk(xj, T(j == i ? 1 : 0));
                const Dual<T> v = dmk(xk, T(j + 1 == i ? 1 : 0));
                const Dual<T> a = dmk(T(1), T(0)) - u;
                const Dual<T> b = v - u * u;
                const Dual<T> t = a * a + T(100) * (b * b);
                r.s0 = t.a;
                tan += t.b;
            } else {
                const T a = T(1) - xj;
                const T b = xk - xj * xj;
                r.s0 = a * a + T(100) * (b * b);
            }
            return r;
        });
        return dmk(acc.s0, tan);
    } else if (OBJ == ZEUS_OBJ_RASTRIGIN) {
        T tan = T(0);
        Part<T> init = zero;
        init.s0 = T(10) * T(d);
        const Part<T> acc = obj_sum<T>(d, d, init, false, [&](int j) {
            const T xj = x[j];
            Part<T> r;
            r.s1 = T(0);
            if (j == i) {
                T s, c;
                sc_2pi(xj, &s, &c);
                // x^2 - 10 cos(2 pi x) on duals with tangent 1
                const T tx2 = xj + xj;
                const T tcos = -s * Consts<T>::two_pi();
                r.s0 = xj * xj - T(10) * c;
                tan += tx2 - T(10) * tcos;
            } else {
                r.s0 = xj * xj - T(10) * c_2pi(xj);
            }
            return r;
        });
        return dmk(acc.s0, tan);
    } else if (OBJ == ZEUS_OBJ_ACKLEY) {
        // the sine of x_i (tangent of the cosine) is taken before the sweep
        // so that the sweep itself is the same for every i (no divergence
        // when passes run on the lanes of one warp); c_2pi is bit for bit
        // the cosine of sc_2pi
        T sn, cn;
        sc_2pi(x[i], &sn, &cn);
        const Part<T> sums = obj_sum<T>(d, d, zero, true, [&](int j) {
            const T xj = x[j];
            Part<T> r;
            r.s0 = xj * xj;
            r.s1 = c_2pi(xj);
            return r;
        });
        const T s1 = sums.s0, s2 = sums.s1;
        // the only non-zero tangents of the two sums are those of term i
        T t1 = T(0), t2 = T(0);
        t1 += x[i] + x[i];
        t2 += -sn * Consts<T>::two_pi();
        // dual division by the constant d: (a/d, (b d - a 0)/(d d))
        const T dd = T(d);
        // u = s1/d, r = sqrt(u) (tangent 0 at u = 0), e1 = exp(-0.2 r)
        const T u = s1 / dd, ut = (t1 * dd) / (dd * dd);
        const T r = xsqrt(u);
        const T rt = r > T(0) ? ut / (T(2) * r) : T(0);
        const T e1 = xexp(T(-0.2) * r);
        const T e1t = e1 * (T(-0.2) * rt);
        const T e2 = xexp(s2 / dd);
        const T e2t = e2 * ((t2 * dd) / (dd * dd));
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
        T tan = T(0);
        const Part<T> acc = obj_sum<T>(d, d, zero, false, [&](int j) {
            const T xj = x[j];
            const T c = T(0.5) * T(j + 1);
            Part<T> r;
            r.s0 = c * (xj * xj);
            r.s1 = T(0);
            if (j == i) tan += c * (xj + xj);
            return r;
        });
        return dmk(acc.s0, tan);
    }
}

template <int OBJ, class T>
__device__ __forceinline__ Dual<T> forward_pass(const T* x, int d, int i) {
    if constexpr (OBJ >= ZEUS_OBJ_USER) {
        const zeus_user::dual<T> r =
            UserObjective<OBJ>::template eval<zeus_user::dual<T>>(UserSeed<T>{x, i}, d);
        return dmk(r.v, r.t);
    } else {
        return builtin_forward_pass<OBJ, T>(x, d, i);
    }
}

// Tangent of pass i alone (Alg. 5): the gradient needs only df/dx_i, so
// the terms whose inputs all carry a zero tangent are left out (they add
// exact zeros) and so is the value sweep wherever the tangent does not
// depend on it; the tangent arithmetic of the remaining terms is that of
// forward_pass, in the same order.  Ackley's tangent depends on its two
// sums, so its pass still sweeps all d terms, as Alg. 5 does.
template <int OBJ, class T>
__device__ __forceinline__ T forward_tangent(const T* x, int d, int i) {
    if (OBJ == ZEUS_OBJ_ROSENBROCK) {
        T tan = T(0);
        for (int j = i - 1; j <= i; ++j) {  // the terms (x_j, x_{j+1}) that contain x_i
            if (j < 0 || j >= d - 1) continue;
            const Dual<T> u = dmk(x[j], T(j == i ? 1 : 0));
            const Dual<T> v = dmk(x[j + 1], T(j + 1 == i ? 1 : 0));
            const Dual<T> a = dmk(T(1), T(0)) - u;
            const Dual<T> b = v - u * u;
            const Dual<T> t = a * a + T(100) * (b * b);
            tan += t.b;
        }
        return tan;
    } else if (OBJ == ZEUS_OBJ_RASTRIGIN) {
        const T xi = x[i];
        T s, c;
        sc_2pi(xi, &s, &c);
        const T tx2 = xi + xi;
        const T tcos = -s * Consts<T>::two_pi();
        T tan = T(0);
        tan += tx2 - T(10) * tcos;
        return tan;
    } else if (OBJ == ZEUS_OBJ_QUADRATIC) {
        const T xi = x[i];
        const T c = T(0.5) * T(i + 1);
        T tan = T(0);
        tan += c * (xi + xi);
        return tan;
    } else {
        return forward_pass<OBJ, T>(x, d, i).b;
    }
}

// Reverse-mode adjoint in two stages: adjoint_prep forms, on one thread,
// the quantities every component shares (for Ackley the adjoints of its two
// sums, which are formed in index order); adjoint_component then gives
// df/dx_i from x_i (and its neighbours) alone, so components can run on
// separate threads.  One forward and one reverse sweep in total, O(d).
struct AdjShared {
    double c1, c2;
};

template <int OBJ, class T>
__device__ __forceinline__ AdjShared adjoint_prep(const T* x, int d) {
    AdjShared a;
    a.c1 = 0.0;
    a.c2 = 0.0;
    if (OBJ == ZEUS_OBJ_ACKLEY) {
        Part<T> zero;
        zero.s0 = zero.s1 = T(0);
        const Part<T> sums = obj_sum<T>(d, d, zero, true, [&](int j) {
            const T xj = x[j];
            Part<T> r;
            r.s0 = xj * xj;
            r.s1 = c_2pi(xj);
            return r;
        });
        const T s1 = sums.s0, s2 = sums.s1;
        const T dd = T(d);
        const T r = xsqrt(s1 / dd);
        const T e1 = xexp(T(-0.2) * r);
        const T e2 = xexp(s2 / dd);
        // f = -20 e1 - e2 + 20 + e; adjoints of s1 and s2
        a.c1 = r > T(0) ? (double)(((T(-20) * e1) * (T(-0.2) / (T(2) * r))) / dd) : 0.0;
        a.c2 = (double)(-e2 / dd);
    }
    return a;
}

template <int OBJ, class T>
__device__ __forceinline__ T adjoint_component(const T* x, int d, int i, const AdjShared& sh) {
    if (OBJ == ZEUS_OBJ_ROSENBROCK) {
        const T xi = x[i];
        T gi = T(0);
        if (i + 1 < d) {  // term i: (1 - x_i)^2 + 100 (x_{i+1} - x_i^2)^2
            const T a = T(1) - xi;
            const T b = x[i + 1] - xi * xi;
            gi = gi + (T(-2) * a - T(400) * xi * b);
        }
        if (i > 0) {  // term i-1 through x_i
            const T xp = x[i - 1];
            gi = gi + T(200) * (xi - xp * xp);
        }
        return gi;
    } else if (OBJ == ZEUS_OBJ_RASTRIGIN) {
        const T xi = x[i];
        T sn, c;
        sc_2pi(xi, &sn, &c);
        return (xi + xi) + T(10) * Consts<T>::two_pi() * sn;
    } else if (OBJ == ZEUS_OBJ_ACKLEY) {
        const T xi = x[i];
        T sn, c;
        sc_2pi(xi, &sn, &c);
        return T(sh.c1) * (xi + xi) - T(sh.c2) * Consts<T>::two_pi() * sn;
    } else if (OBJ == ZEUS_OBJ_GOLDSTEIN_PRICE) {
        const T x1 = x[0], x2 = x[1];
        const T t = (x1 + x2) + T(1);
        const T pa = T(19) - T(14) * x1 + T(3) * (x1 * x1) - T(14) * x2 + T(6) * (x1 * x2) +
                     T(3) * (x2 * x2);
        const T a = T(1) + (t * t) * pa;
        const T u = T(2) * x1 - T(3) * x2;
        const T pb = T(18) - T(32) * x1 + T(12) * (x1 * x1) + T(48) * x2 - T(36) * (x1 * x2) +
                     T(27) * (x2 * x2);
        const T b = T(30) + (u * u) * pb;
        // reverse sweep of f = a b
        const T dt = b * (T(2) * t * pa), dpa = b * (t * t);
        const T du = a * (T(2) * u * pb), dpb = a * (u * u);
        if (i == 0)
            return dt + dpa * (T(-14) + T(6) * x1 + T(6) * x2) + du * T(2) +
                   dpb * (T(-32) + T(24) * x1 - T(36) * x2);
        return dt + dpa * (T(-14) + T(6) * x1 + T(6) * x2) + du * T(-3) +
               dpb * (T(48) - T(36) * x1 + T(54) * x2);
    } else {
        const T xi = x[i];
        return (T(0.5) * T(i + 1)) * (xi + xi);
    }
}

}  // namespace zeus
