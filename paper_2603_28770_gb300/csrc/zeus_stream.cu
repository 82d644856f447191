// zeus_stream.cu -- BFGS for large d: the inverse-Hessian approximation
// streams from HBM (Alg. 4 / Alg. 10, one CTA per start, persistent over
// the starts).
//
// H does not fit in shared memory once d*d*sizeof(T) passes ~200 KB (d >
// ~160 in FP64, > ~230 in FP32).  Each block owns one H slot in the
// workspace and keeps it lagged by one update: the slot holds H_{k-1} and
// the block keeps the pending rank-two correction
//     C_{k-1} = -rho (Hy s' + s Hy') + (rho^2 y'Hy + rho) s s'
//             = s_c A_r + Hy_c B_r,  A = b2 s - rho Hy,  B = -rho s,
// as vectors.  After the line search and the new gradient, ONE pass over
// the slot reads H_{k-1}, writes H_k = H_{k-1} + C_{k-1} and forms
// u = H_k g_{k+1}.  Then H_k y_k = u + p_k (since p_k = -H_k g_k), which
// gives C_k, and the next direction is p_{k+1} = -(u + C_k g_{k+1}) =
// -(u + A (s'g) + B (Hy'g)): no second pass.  Algorithmic traffic per
// start-iteration: d*d*sizeof(T) read + d*d*sizeof(T) written.
//
// The arithmetic is the method's in exact arithmetic; the order of
// operations differs from the oracle (lagged update, tree sums), so this
// path is compared with the oracle within tolerance, not bit for bit.
// T = float is the FP32 form (FP64 for y's, |s|, |y|, g'p, y'Hy, rho, the
// Armijo sums and the final value); T = double is the FP64 method.
#include <type_traits>

#include "zeus_device.cuh"
#include "zeus_internal.h"
#include "zeus_tma.cuh"

namespace zeus {

constexpr int kStreamThreads = 256;
constexpr int kStreamWarps = kStreamThreads / 32;
constexpr int kStreamTrials = 4;  // line-search trials evaluated at once

template <class T>
__device__ __forceinline__ T warp_sum_t(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

struct NoPost {
    __device__ void operator()(const double*) const {}
};

// Sum N doubles over the block; every thread gets the totals.  Warp
// shuffles first, then warp 0 adds the per-warp partials of each value over
// groups of kStreamWarps lanes (three shuffle levels instead of one thread
// adding eight partials per value).  `post`, if given, runs on thread 0
// with the N totals before the barrier that publishes them: scalars that
// every thread needs and one thread can form (square roots, quotients)
// are written there once instead of on every warp.
template <int N, class Post = NoPost>
__device__ __forceinline__ void block_sum(double (&v)[N], double* red, Post post = Post()) {
    static_assert(kStreamWarps == 8, "second stage assumes 8 warps");
    static_assert(N >= 1 && N <= 8, "up to eight sums");
    constexpr int P = N <= 1 ? 1 : (N <= 2 ? 2 : (N <= 4 ? 4 : 8));  // N rounded up
    constexpr int LP = P == 1 ? 0 : (P == 2 ? 1 : (P == 4 ? 2 : 3));
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    // Warp stage, transposed: at each of the first LP levels a lane keeps
    // half of its values and adds its partner's copy of that half (P - 1
    // FP64 adds in all instead of 5 N), then the single value left is
    // summed over the remaining levels.  Lane l ends with the warp total
    // of sum number (l >> (5 - LP)).
    double u[P];
#pragma unroll
    for (int i = 0; i < P; ++i) u[i] = i < N ? v[i] : 0.0;
#pragma unroll
    for (int lev = 0, c = P; lev < LP; ++lev, c >>= 1) {
        const int o = 16 >> lev, half = c >> 1;
        const bool up = (lane & o) != 0;
#pragma unroll
        for (int k = 0; k < half; ++k) {
            const double keep = up ? u[half + k] : u[k];
            const double give = up ? u[k] : u[half + k];
            u[k] = keep + __shfl_xor_sync(0xffffffffu, give, o);
        }
    }
    double a = u[0];
#pragma unroll
    for (int o = 16 >> LP; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    const int which = LP == 0 ? 0 : (lane >> (5 - LP));  // bits of the halving levels
    if ((lane & ((32 >> LP) - 1)) == 0 && which < N) red[which * kStreamWarps + w] = a;
    __syncthreads();
    if (w == 0) {
#pragma unroll
        for (int i0 = 0; i0 < N; i0 += 4) {
            const int i = i0 + (lane >> 3);
            double b = (i < N) ? red[i * kStreamWarps + (lane & 7)] : 0.0;
            b += __shfl_xor_sync(0xffffffffu, b, 4);
            b += __shfl_xor_sync(0xffffffffu, b, 2);
            b += __shfl_xor_sync(0xffffffffu, b, 1);
            if ((lane & 7) == 0 && i < N) red[8 * N + i] = b;
        }
        if constexpr (!std::is_same<Post, NoPost>::value) {
            __syncwarp();
            if (lane == 0) post(red + 8 * N);
        }
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < N; ++i) v[i] = red[8 * N + i];
    __syncthreads();
}

// value of the objective at x + a p (a = 0: at x), FP64 sum of T terms
template <int OBJ, class T>
__device__ __forceinline__ void term_parts(const T* x, const T* p, T a, int d, int j, double& t0,
                                           double& t1) {
    t1 = 0.0;
    const bool at_x = a == T(0);  // value at x itself: p is not read
    const T xj = at_x ? x[j] : x[j] + a * p[j];
    if (OBJ == ZEUS_OBJ_ROSENBROCK) {
        t0 = 0.0;
        if (j + 1 < d) {
            const T xk = at_x ? x[j + 1] : x[j + 1] + a * p[j + 1];
            const T u = T(1) - xj;
            const T v = xk - xj * xj;
            t0 = (double)(u * u + T(100) * (v * v));
        }
    } else if (OBJ == ZEUS_OBJ_RASTRIGIN) {
        if (sizeof(T) == 4) {  // cancellation-free FP32 form of x^2 - 10 cos 2 pi x + 10
            const float sp = sinpif((float)xj);
            t0 = (double)(xj * xj + T(20) * T(sp * sp));
        } else {
            t0 = (double)(xj * xj - T(10) * c_2pi(xj)) + 10.0;
        }
    } else if (OBJ == ZEUS_OBJ_ACKLEY) {
        t0 = (double)(xj * xj);
        if (sizeof(T) == 4) {
            const float sp = sinpif((float)xj);
            t1 = (double)(sp * sp);
        } else {
            t1 = (double)c_2pi(xj);
        }
    } else {  // quadratic (Goldstein-Price is 2-D and never streams)
        t0 = (double)((T(0.5) * T(j + 1)) * (xj * xj));
    }
}

template <int OBJ, class T>
__device__ __forceinline__ double finish_parts(double s0, double s1, int d) {
    if (OBJ == ZEUS_OBJ_ACKLEY) {
        const double dd = (double)d;
        const double t1 = -20.0 * exp_cw(-0.2 * sqrt(s0 / dd));
        const double t2 = sizeof(T) == 4 ? exp_cw(1.0 - 2.0 * (s1 / dd)) : exp_cw(s1 / dd);
        return (t1 - t2) + (20.0 + 2.718281828459045235360287471352);
    }
    return s0;
}

// f(x + a p) into *out, formed by thread 0 and visible to all threads on
// return (one sum, two for Ackley)
template <int OBJ, class T>
__device__ __forceinline__ void block_value(const T* x, const T* p, const double a, int d,
                                            double* out, double* red) {
    constexpr int NP = OBJ == ZEUS_OBJ_ACKLEY ? 2 : 1;
    double s[NP];
#pragma unroll
    for (int m = 0; m < NP; ++m) s[m] = 0.0;
    for (int j = threadIdx.x; j < d; j += blockDim.x) {
        double t0, t1;
        term_parts<OBJ>(x, p, T(a), d, j, t0, t1);
        s[0] += t0;
        if (NP == 2) s[NP - 1] += t1;
    }
    block_sum<NP>(s, red, [=](const double* t) {
        *out = finish_parts<OBJ, T>(t[0], NP == 2 ? t[NP - 1] : 0.0, d);
    });
}

// The trial values f(x + a_m p), m < n <= kStreamTrials, into out and, on
// the thread that forms them (thread 0), the Armijo
// test of each in order: *accepted = the first trial m with
// f(x + a_m p) <= f0 + cA a_m ddir, or -1; visible to all threads on return.
template <int OBJ, class T>
__device__ __forceinline__ void block_trials(const T* x, const T* p, const double (&alpha)[kStreamTrials],
                                             int n, int d, double f0, double cA, double ddir,
                                             double* out, int* accepted, double* red) {
    // one sum per trial (two for Ackley); a chunk of one trial (the first
    // of each search) reduces only its own: the block sum's butterfly is the
    // same for any number of values, so the totals are the same bits
    constexpr int NP = OBJ == ZEUS_OBJ_ACKLEY ? 2 : 1;
    double s[NP * kStreamTrials];
#pragma unroll
    for (int m = 0; m < NP * kStreamTrials; ++m) s[m] = 0.0;
    for (int j = threadIdx.x; j < d; j += blockDim.x) {
#pragma unroll
        for (int m = 0; m < kStreamTrials; ++m) {
            if (m < n) {
                double t0, t1;
                term_parts<OBJ>(x, p, T(alpha[m]), d, j, t0, t1);
                s[NP * m] += t0;
                if (NP == 2) s[NP * m + 1] += t1;
            }
        }
    }
    auto post = [=](const double* t) {
        int acc = -1;
        for (int m = 0; m < n; ++m) {
            const double fm = finish_parts<OBJ, T>(t[NP * m], NP == 2 ? t[NP * m + 1] : 0.0, d);
            out[m] = fm;
            if (acc < 0 && fm <= f0 + cA * alpha[m] * ddir) acc = m;
        }
        *accepted = acc;
    };
    if (n == 1) {
        double s1[NP];
#pragma unroll
        for (int m = 0; m < NP; ++m) s1[m] = s[m];
        block_sum<NP>(s1, red, post);
    } else {
        block_sum<NP * kStreamTrials>(s, red, post);
    }
}

template <int OBJ, int GRAD, class T>
__device__ __forceinline__ void block_gradient(const T* x, T* g, int d, double* red) {
    AdjShared a;
    a.c1 = a.c2 = 0.0;
    if (GRAD == ZEUS_GRAD_ADJOINT && OBJ == ZEUS_OBJ_ACKLEY) {
        // the two shared sums of the adjoint, over the block
        double v[2] = {0.0, 0.0};
        for (int j = threadIdx.x; j < d; j += blockDim.x) {
            v[0] += (double)(x[j] * x[j]);
            v[1] += (double)c_2pi(x[j]);
        }
        block_sum<2>(v, red);
        const T dd = T(d);
        const T r = xsqrt(T(v[0]) / dd);
        const T e1 = xexp(T(-0.2) * r);
        const T e2 = xexp(T(v[1]) / dd);
        a.c1 = r > T(0) ? (double)(((T(-20) * e1) * (T(-0.2) / (T(2) * r))) / dd) : 0.0;
        a.c2 = (double)(-e2 / dd);
    }
    for (int i = threadIdx.x; i < d; i += blockDim.x)
        g[i] = GRAD == ZEUS_GRAD_FORWARD ? forward_tangent<OBJ, T>(x, d, i)
                                         : adjoint_component<OBJ>(x, d, i, a);
    __syncthreads();
}

// 16-byte vector of T
template <class T>
struct Vec16;
template <>
struct Vec16<float> {
    using V = float4;
    static constexpr int n = 4;
    __device__ static float get(const float4& v, int i) {
        return i == 0 ? v.x : (i == 1 ? v.y : (i == 2 ? v.z : v.w));
    }
    __device__ static void set(float4& v, int i, float a) {
        if (i == 0) v.x = a;
        else if (i == 1) v.y = a;
        else if (i == 2) v.z = a;
        else v.w = a;
    }
};
template <>
struct Vec16<double> {
    using V = double2;
    static constexpr int n = 2;
    __device__ static double get(const double2& v, int i) { return i == 0 ? v.x : v.y; }
    __device__ static void set(double2& v, int i, double a) {
        if (i == 0) v.x = a;
        else v.y = a;
    }
};

// The pass over the tiled triangle: H_k = H_{k-1} + (s_c A_r + hy_c B_r) for
// the stored elements r <= c (if corr), and u = H_k g.  A warp takes tile
// rows in pairs (I, TR - 1 - I); in a tile lane l holds column c = 32 J + l
// and reads th rows of it n at a time (16-byte loads, 512 bytes a warp).
// u_c gathers two parts: the row part, c' >= r, H_rc' g_c' summed over the
// lanes of each tile row by row (a warp sum per row, held by the lane of
// that row within the tile row across its tiles), and the column part,
// r < c, H_rc g_r, which lane l of a tile adds up itself over the tile's
// rows and then into its warp's column partials cp[w][c]; after the pass
// the partials join u in warp order.  Elements outside r <= c < d (the
// lower part of the tiles on the diagonal, the padding past d) are carried
// along but never used.
template <class T>
__device__ __forceinline__ void h_pass_tiles(T* __restrict__ Hs, const int d, const bool ident,
                                       const bool corr, const T* s, const T* hy, const T* A,
                                       const T* B, const T* g, T* u, T* cp) {
    using VT = Vec16<T>;
    using V = typename VT::V;
    constexpr int n = VT::n;
    static_assert(n == 4, "the tiled pass holds FP32 H");
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const TileGeo tg = tile_geo(d, n);
    const int th = tg.th, nq = th / n;
    T* cpw = cp + (size_t)w * tg.dp;
    for (int c = lane; c < tg.dp; c += 32) cpw[c] = T(0);  // the lane's own columns
    const bool store = corr || ident;
    for (int q = w; q < (tg.tr + 1) / 2; q += kStreamWarps) {
#pragma unroll 1
        for (int side = 0; side < 2; ++side) {
            const int I = side == 0 ? q : tg.tr - 1 - q;
            if (side == 1 && I == q) break;  // the middle tile row of an odd count
            T rowacc = T(0);
            V* tile = reinterpret_cast<V*>(Hs + tile_row_first(tg, I) * th * 32);
            for (int J = tile_jmin(tg, I); J < tg.tc; ++J, tile += nq * 32) {
                const int c = 32 * J + lane;
                const T sc = s[c], hc = hy[c], gc = g[c];
                T colacc = T(0);
                auto load = [&](int gq) {
                    V h;
                    if (ident) {
#pragma unroll
                        for (int k = 0; k < n; ++k) VT::set(h, k, (I * th + gq * n + k == c) ? T(1) : T(0));
                    } else {
                        h = __ldcs(tile + gq * 32 + lane);
                    }
                    return h;
                };
                V hn = load(0);
                for (int gq = 0; gq < nq; ++gq) {
                    V h = hn;
                    if (gq + 1 < nq) hn = load(gq + 1);  // the next rows in flight
                    const int i0 = I * th + gq * n;
                    const V aq = *reinterpret_cast<const V*>(A + i0);
                    const V bq = *reinterpret_cast<const V*>(B + i0);
                    const V gi = *reinterpret_cast<const V*>(g + i0);
                    T pr[n];
#pragma unroll
                    for (int k = 0; k < n; ++k) {
                        const int i = i0 + k;
                        T e = VT::get(h, k);
                        if (corr) e = fma(sc, VT::get(aq, k), fma(hc, VT::get(bq, k), e));
                        VT::set(h, k, e);
                        const bool ok = c < d && i < d;
                        if (ok && i < c) colacc = fma(e, VT::get(gi, k), colacc);
                        pr[k] = (ok && i <= c) ? e * gc : T(0);
                    }
                    // the four row sums over the lanes at once: two halving
                    // levels leave lane l one value (row (l >> 3)), three
                    // more sum it; the row's lane in the tile row takes it
                    const bool up16 = (lane & 16) != 0, up8 = (lane & 8) != 0;
                    const T k0 = up16 ? pr[2] : pr[0], g0 = up16 ? pr[0] : pr[2];
                    const T k1 = up16 ? pr[3] : pr[1], g1 = up16 ? pr[1] : pr[3];
                    const T a0 = k0 + __shfl_xor_sync(0xffffffffu, g0, 16);
                    const T a1 = k1 + __shfl_xor_sync(0xffffffffu, g1, 16);
                    T rs = (up8 ? a1 : a0) + __shfl_xor_sync(0xffffffffu, up8 ? a0 : a1, 8);
                    rs += __shfl_xor_sync(0xffffffffu, rs, 4);
                    rs += __shfl_xor_sync(0xffffffffu, rs, 2);
                    rs += __shfl_xor_sync(0xffffffffu, rs, 1);
                    const int kr = lane - gq * n;
                    const T mine = __shfl_sync(0xffffffffu, rs, (kr & 3) * 8);
                    if (kr >= 0 && kr < n) rowacc += mine;
                    if (store) __stcs(tile + gq * 32 + lane, h);
                }
                if (c < d) cpw[c] += colacc;
            }
            if (lane < th && I * th + lane < d) u[I * th + lane] = rowacc;
        }
    }
    __syncthreads();
    for (int c = threadIdx.x; c < d; c += blockDim.x) {
        T t = u[c];
#pragma unroll
        for (int w2 = 0; w2 < kStreamWarps; ++w2) t = t + cp[(size_t)w2 * tg.dp + c];
        u[c] = t;
    }
    __syncthreads();
}

// FP64 H, full d x d slot: H_k = H_{k-1} + (s_c A_r + hy_c B_r) (if corr),
// u = H_k g.  One warp per row, 16-byte loads and stores along the row.  (The
// tiled triangle would halve the bytes, but its row sums across lanes cost
// FP64 adds per element, and the FP64 pipe bounds this pass.)
template <class T>
__device__ __forceinline__ void h_pass_rows(T* __restrict__ Hs, int d, bool ident, bool corr,
                                       const T* s, const T* hy, const T* A, const T* B,
                                       const T* g, T* u) {
    using VT = Vec16<T>;
    using V = typename VT::V;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const bool vec = (d % VT::n) == 0;
    for (int r = w; r < d; r += kStreamWarps) {
        T* row = Hs + (size_t)r * d;
        const T ar = corr ? A[r] : T(0), br = corr ? B[r] : T(0);
        T acc = T(0);
        if (vec) {
            const int nv = d / VT::n;
            V* rv = reinterpret_cast<V*>(row);
            // s, Hy and g as 16-byte vectors too (one shared load each per
            // vector of H instead of one per element)
            const V* sv4 = reinterpret_cast<const V*>(s);
            const V* hv4 = reinterpret_cast<const V*>(hy);
            const V* gv4 = reinterpret_cast<const V*>(g);
#pragma unroll 2
            for (int c4 = lane; c4 < nv; c4 += 32) {
                V h;
                if (ident) {
#pragma unroll
                    for (int i = 0; i < VT::n; ++i) VT::set(h, i, (c4 * VT::n + i == r) ? T(1) : T(0));
                } else {
                    h = __ldcs(rv + c4);
                }
                const V gq = gv4[c4];
                V sq, hq;
                if (corr) {
                    sq = sv4[c4];
                    hq = hv4[c4];
                }
#pragma unroll
                for (int i = 0; i < VT::n; ++i) {
                    T e = VT::get(h, i);
                    if (corr) e = fma(VT::get(sq, i), ar, fma(VT::get(hq, i), br, e));
                    VT::set(h, i, e);
                    acc = fma(e, VT::get(gq, i), acc);
                }
                if (corr || ident) __stcs(rv + c4, h);
            }
        } else {
            for (int c = lane; c < d; c += 32) {
                T e = ident ? ((c == r) ? T(1) : T(0)) : row[c];
                if (corr) e = fma(s[c], ar, fma(hy[c], br, e));
                if (corr || ident) row[c] = e;
                acc = fma(e, g[c], acc);
            }
        }
        acc = warp_sum_t(acc);
        if (lane == 0) u[r] = acc;
    }
    __syncthreads();
}

// Staged pass: where a row of H is a multiple of 16 bytes and at most 2 KB
// (d = 256 in FP32 or FP64, the d of the benchmark's streamed workload),
// the rows reach shared memory by bulk copies of one chunk of
// kStreamWarps rows each (one row per warp), `ns` chunks in flight per
// block, so that a block keeps its share of HBM busy whatever its number of
// warps.  The arithmetic and its order are those of h_pass (lane l of a
// row's warp takes the 16-byte vectors l, l + 32, ...); the updated rows go
// back to device memory with streaming stores.
struct StagePlan {
    int ns;                 // chunks in flight (0: the pass reads H directly)
    unsigned chunk_bytes;   // kStreamWarps rows
};

__host__ __device__ inline StagePlan stage_plan(int d, int tsize) {
    StagePlan sp{0, 0};
    const long long row = (long long)d * tsize;
    if (row % 16 != 0 || row > 2048) return sp;
    sp.ns = tsize == 4 ? 3 : 2;
    sp.chunk_bytes = (unsigned)(row * kStreamWarps);
    return sp;
}

__host__ __device__ inline size_t stage_offset(int d, size_t tsize) {
    return (10 * (size_t)d * tsize + 127) & ~size_t(127);
}

// Returns false if a chunk did not arrive within `spin_limit` polls: the
// error word is set, the copies still in flight are waited for (bounded)
// and the caller ends the kernel.  ctr counts the chunks the block has
// waited for (it fixes each chunk's stage and mbarrier parity).
template <class T>
__device__ bool h_pass_staged(T* __restrict__ Hs, int d, bool corr, const T* s, const T* hy,
                              const T* A, const T* B, const T* g, T* u, unsigned char* stage,
                              uint64_t* bar, const StagePlan sp, unsigned& ctr,
                              const unsigned spin_limit, Ctrl* ctrl) {
    using VT = Vec16<T>;
    using V = typename VT::V;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int nc = (d + kStreamWarps - 1) / kStreamWarps;
    const size_t rowb = (size_t)d * sizeof(T);
    const int nv = d / VT::n;
    // the previous pass's stores to H come before the copies that read them
    fence_async_global();
    __syncthreads();
    auto issue = [&](int c) {
        const unsigned k = ctr + (unsigned)c;
        const int st = (int)(k % (unsigned)sp.ns);
        const int r0 = c * kStreamWarps;
        const int nr = min(kStreamWarps, d - r0);
        const unsigned bytes = (unsigned)(nr * rowb);
        mbar_arrive_expect_tx(bar + st, bytes);
        bulk_copy_g2s(stage + (size_t)st * sp.chunk_bytes,
                      reinterpret_cast<const char*>(Hs) + (size_t)r0 * rowb, bytes, bar + st);
    };
    if (threadIdx.x == 0)
        for (int c = 0; c < min(sp.ns, nc); ++c) issue(c);
    bool ok = true;
    int c = 0;
    for (; c < nc; ++c) {
        const unsigned k = ctr + (unsigned)c;
        const int st = (int)(k % (unsigned)sp.ns);
        const bool arrived = mbar_wait_bounded(bar + st, (k / (unsigned)sp.ns) & 1u, spin_limit);
        const int r = c * kStreamWarps + w;
        if (arrived && r < d) {
            const V* rv = reinterpret_cast<const V*>(stage + (size_t)st * sp.chunk_bytes + (size_t)w * rowb);
            V* gvout = reinterpret_cast<V*>(Hs + (size_t)r * d);
            const V* sv4 = reinterpret_cast<const V*>(s);
            const V* hv4 = reinterpret_cast<const V*>(hy);
            const V* gv4 = reinterpret_cast<const V*>(g);
            const T ar = corr ? A[r] : T(0), br = corr ? B[r] : T(0);
            T acc = T(0);
#pragma unroll 2
            for (int c4 = lane; c4 < nv; c4 += 32) {
                V h = rv[c4];
                const V gq = gv4[c4];
                V sq, hq;
                if (corr) {
                    sq = sv4[c4];
                    hq = hv4[c4];
                }
#pragma unroll
                for (int i = 0; i < VT::n; ++i) {
                    T e = VT::get(h, i);
                    if (corr) e = fma(VT::get(sq, i), ar, fma(VT::get(hq, i), br, e));
                    VT::set(h, i, e);
                    acc = fma(e, VT::get(gq, i), acc);
                }
                if (corr) __stcs(gvout + c4, h);
            }
            acc = warp_sum_t(acc);
            if (lane == 0) u[r] = acc;
        }
        // every thread is done with the stage; then it is refilled
        if (__syncthreads_or(arrived ? 0 : 1)) {
            ok = false;
            break;
        }
        if (threadIdx.x == 0 && c + sp.ns < nc) {
            fence_async_shared();
            issue(c + sp.ns);
        }
    }
    if (!ok) {
        if (threadIdx.x == 0) {
            atomicExch(&ctrl->error, 1);
            // the chunks issued and not waited for: c .. min(c + ns, nc) - 1
            for (int cc = c; cc < min(c + sp.ns, nc); ++cc) {
                const unsigned k = ctr + (unsigned)cc;
                mbar_wait_bounded(bar + (k % (unsigned)sp.ns), (k / (unsigned)sp.ns) & 1u, spin_limit);
            }
        }
        __syncthreads();
        return false;
    }
    ctr += (unsigned)nc;
    return true;
}

// One L-BFGS step after the gradient at x_new: the pair (s, y) joins the
// history if it passes the curvature test (as in Alg. 4's update), then
// p = -H g_new by the two-loop recursion (Nocedal & Wright, Alg. 7.4) with
// the initial matrix gamma I, gamma = s'y / y'y of the newest pair.  Dot
// products are FP64 block sums of T products (the FP32 form's guards);
// q and r live in u.
template <class T>
__device__ __forceinline__ void lbfgs_step(const T* x, const T* xn, const T* g, const T* gn,
                                           T* pv, T* u, T* Sm, T* Ym, double* rho_m,
                                           double* gam_m, double* al_m, int m, int& npair,
                                           int& head, int d, double* red) {
    const int tid = threadIdx.x, NT = blockDim.x;
    double v3[3] = {0.0, 0.0, 0.0};
    for (int j = tid; j < d; j += NT) {
        const T sj = xn[j] - x[j], yj = gn[j] - g[j];
        v3[0] += (double)(yj * sj);
        v3[1] += (double)(sj * sj);
        v3[2] += (double)(yj * yj);
    }
    block_sum<3>(v3, red);
    if (v3[0] > 1e-12 * sqrt(v3[1]) * sqrt(v3[2])) {
        int slot;
        if (npair < m) {
            slot = (head + npair) % m;
            ++npair;
        } else {  // drop the oldest
            slot = head;
            head = (head + 1) % m;
        }
        T* sr = Sm + (size_t)slot * d;
        T* yr = Ym + (size_t)slot * d;
        for (int j = tid; j < d; j += NT) {
            sr[j] = xn[j] - x[j];
            yr[j] = gn[j] - g[j];
        }
        if (tid == 0) {
            rho_m[slot] = 1.0 / v3[0];
            gam_m[slot] = v3[0] / v3[2];
        }
    }
    for (int j = tid; j < d; j += NT) u[j] = gn[j];  // q = g_new
    for (int i = npair - 1; i >= 0; --i) {            // newest to oldest
        const int sl = (head + i) % m;
        const T* sr = Sm + (size_t)sl * d;
        const T* yr = Ym + (size_t)sl * d;
        double v1[1] = {0.0};
        for (int j = tid; j < d; j += NT) v1[0] += (double)(sr[j] * u[j]);
        block_sum<1>(v1, red);  // its barriers also publish rho_m of a new pair
        const double a = rho_m[sl] * v1[0];
        if (tid == 0) al_m[i] = a;
        const T at = T(a);
        for (int j = tid; j < d; j += NT) u[j] = fma(-at, yr[j], u[j]);
    }
    if (npair > 0) {
        const T gt = T(gam_m[(head + npair - 1) % m]);
        for (int j = tid; j < d; j += NT) u[j] = gt * u[j];  // r = gamma q
    }
    for (int i = 0; i < npair; ++i) {  // oldest to newest
        const int sl = (head + i) % m;
        const T* sr = Sm + (size_t)sl * d;
        const T* yr = Ym + (size_t)sl * d;
        double v1[1] = {0.0};
        for (int j = tid; j < d; j += NT) v1[0] += (double)(yr[j] * u[j]);
        block_sum<1>(v1, red);
        const T c = T(al_m[i] - rho_m[sl] * v1[0]);
        for (int j = tid; j < d; j += NT) u[j] = fma(c, sr[j], u[j]);
    }
    for (int j = tid; j < d; j += NT) pv[j] = -u[j];
    __syncthreads();
}

struct StreamShared {
    int item;
    int status;
    int accepted;
    int pad;
    double vals[kStreamTrials];
    double red[(kStreamWarps + 1) * 2 * kStreamTrials];
};

// One start on the block: x from row s of x0, the results to row s of the
// outputs, the counters to *ctrl.  LB = false: dense H streamed from the
// block's HBM slot Hs (the pass above; STG: rows staged by bulk copies,
// compiled apart so that the direct pass keeps its own registers).  LB =
// true: L-BFGS (the paper's future work, Section VI) with the m most recent
// pairs in shared memory and the two-loop recursion for p; no H.  Returns
// false if a staged chunk never arrived (the error word is set).
template <int OBJ, int GRAD, class T, bool LB, bool STG>
__device__ __forceinline__ bool stream_start(const zeus_problem& p, const long long s,
                                             const double* x0, double* x_out, double* f_out,
                                             double* gnorm_out, int32_t* status_out,
                                             int32_t* iters_out, Ctrl* ctrl, T* Hs,
                                             const unsigned spin_limit, StreamShared& sh,
                                             unsigned char* smem_raw, uint64_t* stage_bar,
                                             unsigned& chunk_ctr) {
    const int tid = threadIdx.x, NT = blockDim.x;
    const int d = p.dim;
    // vectors of dp elements (the dense pass reads them 16 bytes at a time
    // up to d rounded up to 32; the elements past d are never used); L-BFGS
    // keeps d
    const bool tiled = !LB && stream_tiled(d, sizeof(T));
    const int dp = tiled ? (int)tile_geo(d, Vec16<T>::n).dp : d;
    T* x = reinterpret_cast<T*>(smem_raw);
    T* g = x + dp;
    T* pv = g + dp;
    T* xn = pv + dp;
    T* gn = xn + dp;
    T* sv = gn + dp;  // s of the pending correction
    T* hy = sv + dp;  // Hy of the pending correction
    T* Av = hy + dp;
    T* Bv = Av + dp;
    T* u = Bv + dp;
    T* cp = u + dp;  // tiled pass: kStreamWarps column partials of dp elements
    // L-BFGS history: m pairs (ring, slot of the i-th oldest = (head + i) % m)
    const int lm = LB ? p.lbfgs_m : 0;
    T* Sm = u + dp;
    T* Ym = Sm + (size_t)lm * d;
    double* rho_m = reinterpret_cast<double*>(
        smem_raw + ((((size_t)10 * d + 2 * (size_t)lm * d) * sizeof(T) + 7) & ~size_t(7)));
    double* gam_m = rho_m + lm;  // s'y / y'y of each pair (the initial scaling)
    double* al_m = gam_m + lm;   // alpha of the first loop
    // staged pass (dense H only): chunks of rows in shared memory
    const StagePlan sp = (LB || !STG) ? StagePlan{0, 0} : stage_plan(d, (int)sizeof(T));
    unsigned char* stage = smem_raw + stage_offset(d, sizeof(T));

    const bool use_target = !isnan(p.target_f);
    const bool use_stop = use_target || p.required_converged > 0;
    const double tol = p.grad_tol, cA = p.armijo_c, beta = p.backtrack;
    const int K = p.bfgs_max_iters, L = p.ls_max_iters;

    for (int j = tid; j < d; j += NT) x[j] = T(x0[s * d + j]);
    __syncthreads();
    block_gradient<OBJ, GRAD>(x, g, d, sh.red);
    double a0 = 0.0;
    block_value<OBJ, T>(x, pv, a0, d, sh.vals, sh.red);  // p unused at a = 0
    double f0 = sh.vals[0];
    for (int j = tid; j < d; j += NT) pv[j] = -g[j];  // H_0 = I
    bool ident = true, corr = false;
    int npair = 0, head = 0;  // L-BFGS pairs stored, oldest slot
    int k = 0, feval = 0, status = ZEUS_RUN_MAX_ITER;
    bool stalled = false;  // FP32 form: the previous decrease was below FP32 resolution
    unsigned long long n_read = 0, n_write = 0;  // H passes through HBM
    double gnorm = 0.0;
    __syncthreads();
    for (;;) {
        // ---- tests at the top of iteration k, and g'p, in one reduction
        double v3[3] = {0.0, 0.0, 0.0};
        for (int j = tid; j < d; j += NT) {
            v3[0] += (double)(g[j] * g[j]);
            v3[1] += isfinite(g[j]) ? 0.0 : 1.0;
            v3[2] += (double)(g[j] * pv[j]);
        }
        block_sum<3>(v3, sh.red);
        if (tid == 0) {  // the tests on one thread; |g| is its output alone
            gnorm = sqrt(v3[0]);
            int t = -1;
            if (k >= K) t = ZEUS_RUN_MAX_ITER;
            else if (use_stop && *((volatile int*)&ctrl->stop)) t = ZEUS_RUN_STOPPED;
            else if (!isfinite(f0) || v3[1] != 0.0) t = ZEUS_RUN_NONFINITE;
            else if (gnorm < tol) t = ZEUS_RUN_CONVERGED;
            else if (use_target && f0 <= p.target_f) t = ZEUS_RUN_CONVERGED;
            else if (stalled) t = ZEUS_RUN_STALLED;
            sh.status = t;
        }
        __syncthreads();
        const int st = sh.status;
        if (st >= 0) {
            if (tid == 0 && st == ZEUS_RUN_CONVERGED && use_stop) {
                const unsigned long long c = atomicAdd(&ctrl->n_conv, 1ull) + 1ull;
                if ((use_target && f0 <= p.target_f) ||
                    (p.required_converged > 0 && c >= (unsigned long long)p.required_converged))
                    atomicExch(&ctrl->stop, 1);
            }
            status = st;
            break;
        }
        // ---- descent check
        double ddir = v3[2];
        if (!(ddir < 0.0)) {  // restart from H = I
            ident = true;
            corr = false;
            npair = 0;
            head = 0;
            double v1[1] = {0.0};
            for (int j = tid; j < d; j += NT) {
                pv[j] = -g[j];
                v1[0] += (double)(g[j] * -g[j]);
            }
            block_sum<1>(v1, sh.red);
            ddir = v1[0];
        }
        // ---- backtracking Armijo line search, kStreamTrials trials at once
        double alpha_acc = 0.0, fn = 0.0;
        int acc = -1;
        double a_m = 1.0;
        for (int m0 = 0; m0 < L && acc < 0;) {
            // the first trial alone (usually accepted), then several at once
            const int nw = min(m0 == 0 ? 1 : kStreamTrials, L - m0);
            double al[kStreamTrials];
            double a = a_m;
#pragma unroll
            for (int i = 0; i < kStreamTrials; ++i) {
                al[i] = a;
                if (i + 1 < nw) a = beta * a;
            }
            // values and tests on thread 0 (the first accepted trial wins)
            block_trials<OBJ, T>(x, pv, al, nw, d, f0, cA, ddir, sh.vals, &sh.accepted, sh.red);
            const int ia = sh.accepted;
            if (ia >= 0) {
                acc = m0 + ia;
                alpha_acc = al[ia];
                fn = sh.vals[ia];
            }
            feval += acc >= 0 ? acc - m0 + 1 : nw;
            a_m = al[nw - 1] * beta;
            m0 += nw;
            __syncthreads();
        }
        if (acc < 0) alpha_acc = a_m;  // the step after the last halving
        const T at = T(alpha_acc);
        for (int j = tid; j < d; j += NT) xn[j] = x[j] + at * pv[j];
        __syncthreads();
        if (acc < 0) {
            double z = 0.0;
            block_value<OBJ, T>(xn, pv, z, d, sh.vals, sh.red);
            fn = sh.vals[0];
        }
        block_gradient<OBJ, GRAD>(xn, gn, d, sh.red);
        if (LB) {
            lbfgs_step<T>(x, xn, g, gn, pv, u, Sm, Ym, rho_m, gam_m, al_m, lm, npair, head, d,
                          sh.red);
            for (int j = tid; j < d; j += NT) {
                x[j] = xn[j];
                g[j] = gn[j];
            }
            if (tid == 0) stalled = stalled_step<T>(f0, fn);  // read by the tests alone
            f0 = fn;
            ++k;
            __syncthreads();
            continue;
        }
        // ---- the pass: H_k = H_{k-1} + C_{k-1}, u = H_k g_{k+1}
        if (ident && !corr) {
            for (int j = tid; j < d; j += NT) u[j] = gn[j];
            __syncthreads();
        } else {
            bool done = false;
            if constexpr (sizeof(T) == 4) {
                if (tiled) {
                    h_pass_tiles<T>(Hs, d, ident, corr, sv, hy, Av, Bv, gn, u, cp);
                    done = true;
                }
            }
            if (!done) {
                bool staged = false;
                if constexpr (STG) {
                    if (sp.ns > 0 && !ident) {
                        if (!h_pass_staged<T>(Hs, d, corr, sv, hy, Av, Bv, gn, u, stage,
                                              stage_bar, sp, chunk_ctr, spin_limit, ctrl))
                            return false;  // a chunk never arrived: the error word is set
                        staged = true;
                    }
                }
                if (!staged) h_pass_rows<T>(Hs, d, ident, corr, sv, hy, Av, Bv, gn, u);
            }
            n_read += ident ? 0 : 1;             // H_{k-1} read unless still I
            n_write += (corr || ident) ? 1 : 0;  // H_k stored when it changed
            ident = false;
        }
        // ---- curvature pair and the correction C_k: one reduction for
        //      y's, |s|^2, |y|^2, y'Hy, s'g_new, Hy'g_new
        double v6[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
        for (int j = tid; j < d; j += NT) {
            const T sj = xn[j] - x[j], yj = gn[j] - g[j];
            const T hyj = u[j] + pv[j];  // H_k y_k = H_k g_{k+1} + p_k
            v6[0] += (double)(yj * sj);
            v6[1] += (double)(sj * sj);
            v6[2] += (double)(yj * yj);
            v6[3] += (double)(yj * hyj);
            v6[4] += (double)(sj * gn[j]);
            v6[5] += (double)(hyj * gn[j]);
        }
        // the curvature test, rho and b2 formed once, on thread 0
        block_sum<6>(v6, sh.red, [](double* t) {
            const double sy = t[0];
            t[6] = sy > 1e-12 * sqrt(t[1]) * sqrt(t[2]) ? 1.0 : 0.0;
            const double rho = 1.0 / sy;
            t[7] = rho;
            t[8] = rho * rho * t[3] + rho;
        });
        const double* cs = sh.red + 8 * 6 + 6;  // pass, rho, b2 (until the next sum)
        if (cs[0] != 0.0) {
            const double rho = cs[1];
            const double b2 = cs[2];
            const T sg = T(v6[4]), hg = T(v6[5]), rt = T(rho), bt = T(b2);
            for (int j = tid; j < d; j += NT) {
                const T sj = xn[j] - x[j];
                const T hyj = u[j] + pv[j];
                sv[j] = sj;
                hy[j] = hyj;
                const T a = bt * sj - rt * hyj, b = -rt * sj;
                Av[j] = a;
                Bv[j] = b;
                pv[j] = -(u[j] + a * sg + b * hg);
            }
            corr = true;
        } else {
            for (int j = tid; j < d; j += NT) pv[j] = -u[j];
            corr = false;
        }
        for (int j = tid; j < d; j += NT) {
            x[j] = xn[j];
            g[j] = gn[j];
        }
        if (tid == 0) stalled = stalled_step<T>(f0, fn);  // read by the tests alone
        f0 = fn;
        ++k;
        __syncthreads();
    }
    // final value in FP64 at the final point
    double vf[2] = {0.0, 0.0};
    for (int j = tid; j < d; j += NT) {
        double t0, t1;
        const double xj = (double)x[j];
        if (OBJ == ZEUS_OBJ_ROSENBROCK) {
            t1 = 0.0;
            t0 = 0.0;
            if (j + 1 < d) {
                const double xk = (double)x[j + 1];
                const double a = 1.0 - xj, b = xk - xj * xj;
                t0 = a * a + 100.0 * (b * b);
            }
        } else if (OBJ == ZEUS_OBJ_RASTRIGIN) {
            t0 = (xj * xj - 10.0 * c_2pi(xj)) + 10.0;
            t1 = 0.0;
        } else if (OBJ == ZEUS_OBJ_ACKLEY) {
            t0 = xj * xj;
            t1 = c_2pi(xj);
        } else {
            t0 = (0.5 * (double)(j + 1)) * (xj * xj);
            t1 = 0.0;
        }
        vf[0] += t0;
        vf[1] += t1;
    }
    block_sum<2>(vf, sh.red);
    const double ffin = finish_parts<OBJ, double>(vf[0], vf[1], d);
    for (int j = tid; j < d; j += NT) x_out[s * d + j] = (double)x[j];
    if (tid == 0) {
        if (f_out) f_out[s] = ffin;
        if (gnorm_out) gnorm_out[s] = gnorm;
        if (status_out) status_out[s] = status;
        if (iters_out) iters_out[s] = k;
        atomicAdd(&ctrl->total_iters, (unsigned long long)k);
        atomicAdd(&ctrl->total_feval, (unsigned long long)feval);
        atomicAdd(&ctrl->h_reads, n_read);
        atomicAdd(&ctrl->h_writes, n_write);
        if (!use_stop && status == ZEUS_RUN_CONVERGED) atomicAdd(&ctrl->n_conv, 1ull);
    }
    return true;
}

// Persistent blocks over the starts of one problem (a start per block at a
// time, taken from ctrl->q_head).
template <int OBJ, int GRAD, class T, bool LB, bool STG = false>
__global__ void __launch_bounds__(kStreamThreads, 4)
    bfgs_stream_kernel(const zeus_problem p, const double* x0, double* x_out,
                       double* __restrict__ f_out, double* __restrict__ gnorm_out,
                       int32_t* __restrict__ status_out, int32_t* __restrict__ iters_out,
                       Ctrl* __restrict__ ctrl, T* __restrict__ hslots, const unsigned spin_limit) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ StreamShared sh;
    __shared__ __align__(8) uint64_t stage_bar[4];
    const int d = p.dim;
    T* Hs = LB ? nullptr : hslots + (size_t)blockIdx.x * stream_slot_elems(d, sizeof(T));
    const StagePlan sp = (LB || !STG) ? StagePlan{0, 0} : stage_plan(d, (int)sizeof(T));
    if (sp.ns > 0) {
        if (threadIdx.x == 0) {
            for (int i = 0; i < sp.ns; ++i) mbar_init(stage_bar + i, 1);
            fence_async_shared();
        }
        __syncthreads();
    }
    unsigned chunk_ctr = 0;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) sh.item = (int)atomicAdd(&ctrl->q_head, 1u);
        __syncthreads();
        const long long s = sh.item;
        if (s >= p.n_starts) break;
        if (!stream_start<OBJ, GRAD, T, LB, STG>(p, s, x0, x_out, f_out, gnorm_out, status_out,
                                                 iters_out, ctrl, Hs, spin_limit, sh, smem_raw,
                                                 stage_bar, chunk_ctr))
            return;
    }
}

// L-BFGS items (P, s, 0, 3) of a batch class: persistent blocks over the
// class's items, each start run by the body of the single-problem L-BFGS
// kernel, so that its results are those of zeus_solve bit for bit.
template <int GRAD, class T>
__global__ void __launch_bounds__(kStreamThreads, 4)
    batch_lbfgs_kernel(const BatchDev bd, const int cls, const int first, const int count,
                       double* x_out, double* __restrict__ f_out, double* __restrict__ gnorm_out,
                       int32_t* __restrict__ status_out, int32_t* __restrict__ iters_out,
                       const unsigned spin_limit) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ StreamShared sh;
    unsigned chunk_ctr = 0;
    unsigned* head = bd.heads + cls;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) sh.item = (int)atomicAdd(head, 1u);
        __syncthreads();
        const int item = sh.item;
        if (item >= count) break;
        const int4 w = bd.items[first + item];
        const int P = w.x;
        const zeus_problem p = bd.probs[P];
        const long long xo = bd.xoff[P], so = bd.soff[P];
        const double* x0 = p.start_from_pbest ? bd.px + xo : x_out + xo;
        double* go = gnorm_out ? gnorm_out + so : nullptr;
        int32_t* sto = status_out ? status_out + so : nullptr;
        int32_t* ito = iters_out ? iters_out + so : nullptr;
#define ZEUS_LBCASE(O)                                                                        \
    stream_start<O, GRAD, T, true, false>(p, (long long)w.y, x0, x_out + xo, f_out + so, go, \
                                          sto, ito, bd.pctrl + P, nullptr, spin_limit, sh,   \
                                          smem_raw, nullptr, chunk_ctr)
        switch (p.objective) {
            case ZEUS_OBJ_ROSENBROCK:
                ZEUS_LBCASE(ZEUS_OBJ_ROSENBROCK);
                break;
            case ZEUS_OBJ_RASTRIGIN:
                ZEUS_LBCASE(ZEUS_OBJ_RASTRIGIN);
                break;
            case ZEUS_OBJ_ACKLEY:
                ZEUS_LBCASE(ZEUS_OBJ_ACKLEY);
                break;
            default:
                ZEUS_LBCASE(ZEUS_OBJ_QUADRATIC);
                break;
        }
#undef ZEUS_LBCASE
    }
}

template <int GRAD, class T>
static cudaError_t batch_lbfgs_go(const BatchDev& bd, int cls, int first, int count, size_t smem,
                                  double* x_out, double* f_out, double* gnorm_out,
                                  int32_t* status_out, int32_t* iters_out, cudaStream_t st) {
    auto k = batch_lbfgs_kernel<GRAD, T>;
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = allow_smem(k, smem);
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kStreamThreads, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    long long blocks = (long long)sms * per_sm;
    if (blocks > count) blocks = count;  // no block without an item
    if (blocks < 1) return cudaSuccess;
    k<<<(int)blocks, kStreamThreads, smem, st>>>(bd, cls, first, count, x_out, f_out, gnorm_out,
                                                 status_out, iters_out, wait_limit());
    return cudaGetLastError();
}

cudaError_t launch_batch_lbfgs(const BatchDev& bd, int precision, int grad_mode, int cls,
                               int first, int count, size_t smem, double* x_out, double* f_out,
                               double* gnorm_out, int32_t* status_out, int32_t* iters_out,
                               cudaStream_t st) {
    const bool f32 = precision == ZEUS_FP32_GUARDED;
    if (grad_mode == ZEUS_GRAD_ADJOINT)
        return f32 ? batch_lbfgs_go<ZEUS_GRAD_ADJOINT, float>(bd, cls, first, count, smem, x_out,
                                                               f_out, gnorm_out, status_out,
                                                               iters_out, st)
                   : batch_lbfgs_go<ZEUS_GRAD_ADJOINT, double>(bd, cls, first, count, smem, x_out,
                                                                f_out, gnorm_out, status_out,
                                                                iters_out, st);
    return f32 ? batch_lbfgs_go<ZEUS_GRAD_FORWARD, float>(bd, cls, first, count, smem, x_out, f_out,
                                                           gnorm_out, status_out, iters_out, st)
               : batch_lbfgs_go<ZEUS_GRAD_FORWARD, double>(bd, cls, first, count, smem, x_out,
                                                            f_out, gnorm_out, status_out, iters_out,
                                                            st);
}

size_t stream_smem(int d, size_t tsize) {
    if (stream_tiled(d, tsize)) return 18 * (size_t)tile_geo(d, 4).dp * tsize;  // vectors, partials
    const StagePlan sp = stage_plan(d, (int)tsize);
    if (sp.ns == 0) return 10 * (size_t)d * tsize;
    return stage_offset(d, tsize) + (size_t)sp.ns * sp.chunk_bytes;
}

size_t lbfgs_smem(int d, int m, size_t tsize) {
    return ((((size_t)10 * d + 2 * (size_t)m * d) * tsize + 7) & ~size_t(7)) +
           3 * (size_t)m * sizeof(double);
}

// As many blocks as fit the SMs at once (at most four per SM: the kernel's
// registers; fewer when its shared memory, `smem` bytes, allows fewer), and
// the starts spread evenly over the rounds (each block takes a start, runs
// it to the end, takes the next).  A block beyond those resident would
// start only when a resident one had run out of starts.
int stream_blocks(const zeus_problem& p, size_t smem) {
    long long per_sm = (long long)(233472 / (smem + 2048));  // 228 KB per SM, reserve + static
    if (per_sm > 4) per_sm = 4;
    if (per_sm < 1) per_sm = 1;
    const long long full = 152ll * per_sm;
    const long long rounds = (p.n_starts + full - 1) / full;
    long long b = (p.n_starts + rounds - 1) / rounds;
    if (b < 1) b = 1;
    return (int)b;
}

template <int OBJ, int GRAD, class T>
static cudaError_t stream_go(const zeus_problem& p, const double* x0, double* x_out, double* f_out,
                             double* gnorm_out, int32_t* status_out, int32_t* iters_out,
                             Ctrl* ctrl, void* hslots, cudaStream_t st) {
    if (p.lbfgs_m > 0) {
        auto kl = bfgs_stream_kernel<OBJ, GRAD, T, true>;
        const size_t sl = lbfgs_smem(p.dim, p.lbfgs_m, sizeof(T));
        cudaError_t e = allow_smem(kl, sl);
        if (e != cudaSuccess) return e;
        kl<<<stream_blocks(p, sl), kStreamThreads, sl, st>>>(p, x0, x_out, f_out, gnorm_out,
                                                             status_out,
                                                         iters_out, ctrl, nullptr, wait_limit());
        return cudaGetLastError();
    }
    const bool stg = !stream_tiled(p.dim, sizeof(T)) && stage_plan(p.dim, (int)sizeof(T)).ns > 0;
    auto kern = stg ? bfgs_stream_kernel<OBJ, GRAD, T, false, true>
                    : bfgs_stream_kernel<OBJ, GRAD, T, false, false>;
    const size_t sm = stream_smem(p.dim, sizeof(T));
    cudaError_t e = allow_smem(kern, sm);
    if (e != cudaSuccess) return e;
    kern<<<stream_blocks(p, sm), kStreamThreads, sm, st>>>(p, x0, x_out, f_out, gnorm_out, status_out,
                                                       iters_out, ctrl, static_cast<T*>(hslots),
                                                       wait_limit());
    return cudaGetLastError();
}

template <int OBJ>
static cudaError_t stream_obj(const zeus_problem& p, const double* x0, double* x_out, double* f_out,
                              double* gnorm_out, int32_t* status_out, int32_t* iters_out,
                              Ctrl* ctrl, void* hslots, cudaStream_t st) {
    const bool f32 = p.precision == ZEUS_FP32_GUARDED;
    if (p.grad_mode == ZEUS_GRAD_ADJOINT)
        return f32 ? stream_go<OBJ, ZEUS_GRAD_ADJOINT, float>(p, x0, x_out, f_out, gnorm_out,
                                                              status_out, iters_out, ctrl, hslots, st)
                   : stream_go<OBJ, ZEUS_GRAD_ADJOINT, double>(p, x0, x_out, f_out, gnorm_out,
                                                               status_out, iters_out, ctrl, hslots, st);
    return f32 ? stream_go<OBJ, ZEUS_GRAD_FORWARD, float>(p, x0, x_out, f_out, gnorm_out,
                                                          status_out, iters_out, ctrl, hslots, st)
               : stream_go<OBJ, ZEUS_GRAD_FORWARD, double>(p, x0, x_out, f_out, gnorm_out,
                                                           status_out, iters_out, ctrl, hslots, st);
}

cudaError_t launch_bfgs_stream(const zeus_problem& p, const double* x0, double* x_out,
                               double* f_out, double* gnorm_out, int32_t* status_out,
                               int32_t* iters_out, Ctrl* ctrl, void* hslots, cudaStream_t st) {
    switch (p.objective) {
        case ZEUS_OBJ_ROSENBROCK:
            return stream_obj<ZEUS_OBJ_ROSENBROCK>(p, x0, x_out, f_out, gnorm_out, status_out,
                                                   iters_out, ctrl, hslots, st);
        case ZEUS_OBJ_RASTRIGIN:
            return stream_obj<ZEUS_OBJ_RASTRIGIN>(p, x0, x_out, f_out, gnorm_out, status_out,
                                                  iters_out, ctrl, hslots, st);
        case ZEUS_OBJ_ACKLEY:
            return stream_obj<ZEUS_OBJ_ACKLEY>(p, x0, x_out, f_out, gnorm_out, status_out,
                                               iters_out, ctrl, hslots, st);
        default:
            return stream_obj<ZEUS_OBJ_QUADRATIC>(p, x0, x_out, f_out, gnorm_out, status_out,
                                                  iters_out, ctrl, hslots, st);
    }
}

}  // namespace zeus
