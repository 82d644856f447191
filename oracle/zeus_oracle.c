/*
 * zeus_oracle.c -- plain, slow, obviously-correct FP64 CPU reference of the
 * Zeus method (PSO seeding, then one BFGS run per start with forward-mode
 * dual-number gradients, backtracking Armijo line search and the dense
 * inverse-Hessian rank-two update, then a best-of-swarm argmin).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the oracle that the CUDA path is
 * checked against.  Only tests/, __graft_entry__.smoke() and bench.py's CPU
 * baseline leg may load it.  It shares no code, header, table or constant
 * generator with the CUDA library; it has its own Philox, its own dual
 * numbers and its own objectives.
 *
 * Build: gcc -O2 -std=c11 -ffp-contract=off -fopenmp -fPIC -shared -lm
 * (no FMA contraction, so every product and sum below is rounded exactly
 * once in the order written).
 *
 * Two rounding orders (zo_problem.order): the plain order rounds every
 * operation on its own and sums left to right; the library order is a
 * second fixed order that 32 lanes can form (fma per product term, 32
 * strided chains past 32 terms, the update over one triangle).  The paper
 * states the arithmetic exactly, so both are readings of it; the pins in
 * tests/test_oracle_*.py hold for both.
 *
 * Each function names the part of the paper it follows (Zeus, arXiv
 * 2603.28770).  Readings of points the paper leaves open are marked
 * "Reading:".
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------ */
/* Problem description (the oracle's own copy; not shared with the library) */
/* ------------------------------------------------------------------------ */

enum {
    ZO_ROSENBROCK = 0,      /* Section V-B, Rosenbrock */
    ZO_RASTRIGIN = 1,       /* Section V-B, Rastrigin (A = 10) */
    ZO_ACKLEY = 2,          /* Section V-B, Ackley (a=20, b=0.2, c=2*pi) */
    ZO_GOLDSTEIN_PRICE = 3, /* Section V-B, Goldstein-Price (d = 2) */
    ZO_QUADRATIC = 100,     /* test objective: 0.5 * sum (i+1) x_i^2 */
    /* Objectives supplied by a user of the library rather than built in
     * (Section IV-A: any f written for a generic scalar type): the two of
     * the library's default plug-in, written here on their own. */
    ZO_GRIEWANK = 200,      /* 1 + sum x_i^2 / 4000 - prod cos(x_i / sqrt(i)) */
    ZO_HIMMELBLAU = 201     /* (x^2 + y - 11)^2 + (x + y^2 - 7)^2, d = 2 */
};

typedef struct {
    int32_t objective;
    int32_t dim;
    double lower, upper;
    int64_t n_starts;
    int32_t pso_iters;
    int32_t bfgs_max_iters;
    int32_t ls_max_iters;
    int32_t required_converged; /* 0 = off */
    double grad_tol;
    double w, c1, c2;
    double armijo_c, backtrack;
    double target_f;            /* NaN = off */
    uint64_t seed;
    int32_t start_from_pbest;   /* 0 = current swarm positions (Alg. 10) */
    int32_t n_threads;          /* OpenMP threads for the per-start loops */
    int32_t lbfgs_m;            /* 0 = dense inverse Hessian (Alg. 4); m > 0 = L-BFGS, m pairs */
    int32_t order;              /* rounding order of the sums and the update: ZO_ORDER_LIB or
                                   ZO_ORDER_PLAIN (below) */
} zo_problem;

/* Rounding order.  The paper states every sum and product of the method in
 * exact arithmetic; the oracle offers two readings of the order in which
 * they are rounded.
 *  ZO_ORDER_PLAIN  the textbook order: every sum left to right, every product
 *                  and every sum rounded on its own (no fused multiply-add
 *                  outside the elementary functions), the rank-two update
 *                  formed element by element over the whole matrix from its
 *                  expanded form.  Independent of how any GPU forms a sum.
 *  ZO_ORDER_LIB    a second, fixed order that a warp can form: products
 *                  accumulated with one rounding (fma), sums past 32 terms in
 *                  32 strided chains added by a fixed pairwise tree, the
 *                  update over the upper triangle, mirrored.
 * The two agree to rounding; the GPU path is compared with the plain order
 * within a tolerance and with the library order bit for bit. */
enum { ZO_ORDER_LIB = 0, ZO_ORDER_PLAIN = 1 };

/* per-start result of one BFGS run (Alg. 4) */
typedef struct {
    double f;          /* f at the final x */
    double gnorm;      /* ||g|| at the final x */
    double margin;     /* smallest relative margin of any branch decision */
    int32_t iters;     /* completed iterations k */
    int32_t status;    /* 0 max-iter, 1 converged, 2 stopped, 3 non-finite */
    int32_t n_feval;   /* line-search objective evaluations */
    int32_t pad;
} zo_result;

/* ------------------------------------------------------------------------ */
/* Philox4x64-10 (Salmon, Moraes, Dror, Shaw, "Parallel Random Numbers: As  */
/* Easy as 1, 2, 3", SC'11), written from its published definition.         */
/* Replaces the paper's cuRAND seeding of Section IV-A.                      */
/* ------------------------------------------------------------------------ */

static void mulhilo64(uint64_t a, uint64_t b, uint64_t *hi, uint64_t *lo)
{
    unsigned __int128 p = (unsigned __int128)a * (unsigned __int128)b;
    *hi = (uint64_t)(p >> 64);
    *lo = (uint64_t)p;
}

void zo_philox4x64_10(const uint64_t ctr_in[4], const uint64_t key_in[2],
                      uint64_t out[4])
{
    const uint64_t M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
    const uint64_t W0 = 0x9E3779B97F4A7C15ULL, W1 = 0xBB67AE8584CAA73BULL;
    uint64_t c[4] = {ctr_in[0], ctr_in[1], ctr_in[2], ctr_in[3]};
    uint64_t k[2] = {key_in[0], key_in[1]};
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k[0] += W0; k[1] += W1; }
        uint64_t hi0, lo0, hi1, lo1;
        mulhilo64(M0, c[0], &hi0, &lo0);
        mulhilo64(M1, c[2], &hi1, &lo1);
        uint64_t n0 = hi1 ^ c[1] ^ k[0];
        uint64_t n2 = hi0 ^ c[3] ^ k[1];
        c[0] = n0; c[1] = lo1; c[2] = n2; c[3] = lo0;
    }
    out[0] = c[0]; out[1] = c[1]; out[2] = c[2]; out[3] = c[3];
}

/* Reading of Section IV-A: one uniform double per (phase, particle, dim).
 * Counter = (j / 4, particle i, problem, phase), key = (seed, 0); the
 * draw is word j % 4 of the block, mapped to [0,1) with 53 bits.
 * Phases: 0 = initial position, 1 = initial velocity, 2+2t = r1 and
 * 3+2t = r2 of PSO iteration t. */
double zo_uniform(uint64_t seed, uint64_t problem, uint64_t phase,
                  uint64_t particle, uint64_t j)
{
    uint64_t ctr[4] = {j / 4, particle, problem, phase};
    uint64_t key[2] = {seed, 0};
    uint64_t out[4];
    zo_philox4x64_10(ctr, key, out);
    return (double)(out[j % 4] >> 11) * 0x1.0p-53;
}

/* ------------------------------------------------------------------------ */
/* Elementary functions of the objectives, FP64, written from published      */
/* methods so that the reference fixes every bit (the CUDA library          */
/* implements the same methods independently).                              */
/* ------------------------------------------------------------------------ */

/* Taylor coefficients of sin(2 pi s) = sum_k S_k s^(2k+1) and
 * cos(2 pi s) = sum_k C_k s^(2k): S_k = (-1)^k (2 pi)^(2k+1) / (2k+1)!,
 * C_k = (-1)^k (2 pi)^(2k) / (2k)!, rounded to double. */
static const double ZO_S2PI[9] = {
    0x1.921fb54442d18p+2, -0x1.4abbce625be53p+5, 0x1.466bc6775aae2p+6,
    -0x1.32d2cce62bd86p+6, 0x1.50783487ee782p+5, -0x1.e3074fde8871fp+3,
    0x1.e8f434d018d63p+1, -0x1.6fadb9f155744p-1, 0x1.aaec32af93359p-4};
static const double ZO_C2PI[9] = {
    0x1.0000000000000p+0, -0x1.3bd3cc9be45dep+4, 0x1.03c1f081b5ac4p+6,
    -0x1.55d3c7e3cbffap+6, 0x1.e1f506891babbp+5, -0x1.a6d1f2a204a8cp+4,
    0x1.f9d38a3763cc3p+2, -0x1.b6e24f44b128fp+0, 0x1.20c62c2f2d7f5p-2};

/* sin(2 pi x) and cos(2 pi x).  Exact argument reduction: r = x - rint(x)
 * (|r| <= 1/2), q = rint(4 r), s = r - q/4 (|s| <= 1/8), each step exact in
 * binary floating point; then the Taylor series above through s^17 and s^16
 * (truncation below 3e-18 on |s| <= 1/8) in Horner form with fused
 * multiply-adds in s^2, and the quarter-turn identities for q. */
void zo_sincos2pi(double x, double *sp, double *cp)
{
    double n = rint(x);
    double r = x - n;
    double qf = rint(4.0 * r);
    double s = r - 0.25 * qf;
    int q = ((int)qf) & 3;
    double z = s * s;
    double ps = ZO_S2PI[8], pc = ZO_C2PI[8];
    for (int k = 7; k >= 0; --k) {
        ps = fma(ps, z, ZO_S2PI[k]);
        pc = fma(pc, z, ZO_C2PI[k]);
    }
    ps = ps * s;
    switch (q) {
    case 0: *sp = ps; *cp = pc; break;
    case 1: *sp = pc; *cp = -ps; break;
    case 2: *sp = -ps; *cp = -pc; break;
    default: *sp = -pc; *cp = ps; break;
    }
}

static double zo_cos2pi(double x)
{
    double s, c;
    zo_sincos2pi(x, &s, &c);
    return c;
}

/* e^x.  Cody & Waite reduction x = k ln2 + r with k = rint(x / ln2) and
 * ln2 = L1 + L2, L1 holding 32 significant bits so that k L1 is exact;
 * e^r by its Taylor series through r^13 (|r| <= 0.35, truncation below
 * 5e-18) in Horner form with fused multiply-adds; exact scaling by 2^k. */
static const double ZO_EXPC[14] = {
    0x1.0000000000000p+0, 0x1.0000000000000p+0, 0x1.0000000000000p-1,
    0x1.5555555555555p-3, 0x1.5555555555555p-5, 0x1.1111111111111p-7,
    0x1.6c16c16c16c17p-10, 0x1.a01a01a01a01ap-13, 0x1.a01a01a01a01ap-16,
    0x1.71de3a556c734p-19, 0x1.27e4fb7789f5cp-22, 0x1.ae64567f544e4p-26,
    0x1.1eed8eff8d898p-29, 0x1.6124613a86d09p-33};  /* 1/k! */

double zo_exp(double x)
{
    const double INV_LN2 = 0x1.71547652b82fep+0;
    const double L1 = 0x1.62e42fee00000p-1, L2 = 0x1.a39ef35793c76p-33;
    if (isnan(x)) return x;
    if (x > 709.78) return INFINITY;
    if (x < -745.2) return 0.0;
    double k = rint(x * INV_LN2);
    double r = (x - k * L1) - k * L2;
    double p = ZO_EXPC[13];
    for (int i = 12; i >= 0; --i) p = fma(p, r, ZO_EXPC[i]);
    return ldexp(p, (int)k);
}

/* ------------------------------------------------------------------------ */
/* Dual numbers a + b*eps with eps^2 = 0 (Section III-C).                    */
/* ------------------------------------------------------------------------ */

typedef struct { double a, b; } zo_dual;

static const double ZO_PI_ = 3.14159265358979323846;

static zo_dual dconst(double a) { zo_dual r = {a, 0.0}; return r; }
static zo_dual dadd(zo_dual x, zo_dual y) { zo_dual r = {x.a + y.a, x.b + y.b}; return r; }
static zo_dual dsub(zo_dual x, zo_dual y) { zo_dual r = {x.a - y.a, x.b - y.b}; return r; }
/* (a1 + b1 e)(a2 + b2 e) = a1 a2 + (a1 b2 + b1 a2) e */
static zo_dual dmul(zo_dual x, zo_dual y)
{
    zo_dual r = {x.a * y.a, x.a * y.b + x.b * y.a};
    return r;
}
/* (a1 + b1 e)/(a2 + b2 e) = a1/a2 + (b1 a2 - a1 b2)/a2^2 e */
static zo_dual ddiv(zo_dual x, zo_dual y)
{
    zo_dual r = {x.a / y.a, (x.b * y.a - x.a * y.b) / (y.a * y.a)};
    return r;
}
static zo_dual dscale(double s, zo_dual x) { zo_dual r = {s * x.a, s * x.b}; return r; }
/* g(a + b e) = g(a) + g'(a) b e */
static zo_dual dsin(zo_dual x) { zo_dual r = {sin(x.a), cos(x.a) * x.b}; return r; }
static zo_dual dcos(zo_dual x) { zo_dual r = {cos(x.a), -sin(x.a) * x.b}; return r; }
static zo_dual dexp(zo_dual x) { double e = zo_exp(x.a); zo_dual r = {e, e * x.b}; return r; }
/* cos(2 pi x) as one primitive: (cos 2 pi a, -sin(2 pi a) (2 pi b)) */
static zo_dual dcos2pi(zo_dual x)
{
    double s, c;
    zo_sincos2pi(x.a, &s, &c);
    zo_dual r = {c, -s * (2.0 * ZO_PI_ * x.b)};
    return r;
}
/* Reading: d/du sqrt(u) at u = 0 is taken as 0 (Ackley's kink at the
 * origin, Section V-B, where the derivative is undefined). */
static zo_dual dsqrt(zo_dual x)
{
    double s = sqrt(x.a);
    zo_dual r = {s, s > 0.0 ? x.b / (2.0 * s) : 0.0};
    return r;
}

/* exported for the dual-algebra pins */
void zo_dual_op(int op, double a1, double b1, double a2, double b2,
                double *ra, double *rb)
{
    zo_dual x = {a1, b1}, y = {a2, b2}, r;
    switch (op) {
    case 0: r = dadd(x, y); break;
    case 1: r = dsub(x, y); break;
    case 2: r = dmul(x, y); break;
    case 3: r = ddiv(x, y); break;
    case 4: r = dsin(x); break;
    case 5: r = dcos(x); break;
    case 6: r = dexp(x); break;
    case 7: r = dsqrt(x); break;
    case 8: r = dcos2pi(x); break;
    default: r = dconst(NAN); break;
    }
    *ra = r.a;
    *rb = r.b;
}

/* ------------------------------------------------------------------------ */
/* Objectives (Section V-B), on doubles and on duals.                        */
/* ------------------------------------------------------------------------ */

static const double ZO_E = 2.71828182845904523536;

/* The sums over the coordinates of the built-in objectives (Rosenbrock's
 * d-1 chain terms, the terms of Rastrigin and of the quadratic, Ackley's
 * two sums).  Reading: for d <= 32 left to right from the sum's constant
 * (Rastrigin's 10 d, else 0); for d > 32, 32 chains, chain l over the terms
 * j = l (mod 32) left to right with chain 0 starting from the constant,
 * added pairwise in the tree of zo_bdot (l with l + 16, then l + 8, ...).
 * The paper writes these sums in exact terms.  A sum is accumulated into
 * the chains term by term (zo_sum_add) and closed by zo_sum_end.  In the
 * plain order (ZO_ORDER_PLAIN) every sum is one chain, left to right. */
typedef struct {
    double p[32];
    int split;
} zo_sum;

static void zo_sum_start(zo_sum *a, int d, double c0, int ord)
{
    a->split = ord == ZO_ORDER_LIB && d > 32;
    for (int l = 0; l < 32; ++l) a->p[l] = 0.0;
    a->p[0] = c0;
}
static void zo_sum_add(zo_sum *a, int j, double t)
{
    const int l = a->split ? (j & 31) : 0;
    a->p[l] = a->p[l] + t;
}
static double zo_sum_end(zo_sum *a)
{
    if (a->split)
        for (int w = 16; w >= 1; w >>= 1)
            for (int l = 0; l < w; ++l) a->p[l] = a->p[l] + a->p[l + w];
    return a->p[0];
}

double zo_f_ord(int obj, int d, const double *x, int ord)
{
    double s = 0.0;
    zo_sum a0, a1;
    switch (obj) {
    case ZO_ROSENBROCK:
        /* Reading: the chain sum runs over i = 1..d-1 (the printed upper
         * limit n would need x_{n+1}). */
        zo_sum_start(&a0, d, 0.0, ord);
        for (int i = 0; i + 1 < d; ++i) {
            double a = 1.0 - x[i];
            double b = x[i + 1] - x[i] * x[i];
            zo_sum_add(&a0, i, a * a + 100.0 * (b * b));
        }
        return zo_sum_end(&a0);
    case ZO_RASTRIGIN:
        zo_sum_start(&a0, d, 10.0 * (double)d, ord);
        for (int i = 0; i < d; ++i)
            zo_sum_add(&a0, i, x[i] * x[i] - 10.0 * zo_cos2pi(x[i]));
        return zo_sum_end(&a0);
    case ZO_ACKLEY: {
        zo_sum_start(&a0, d, 0.0, ord);
        zo_sum_start(&a1, d, 0.0, ord);
        for (int i = 0; i < d; ++i) {
            zo_sum_add(&a0, i, x[i] * x[i]);
            zo_sum_add(&a1, i, zo_cos2pi(x[i]));
        }
        double s1 = zo_sum_end(&a0), s2 = zo_sum_end(&a1);
        double t1 = -20.0 * zo_exp(-0.2 * sqrt(s1 / (double)d));
        double t2 = zo_exp(s2 / (double)d);
        return (t1 - t2) + (20.0 + ZO_E);
    }
    case ZO_GOLDSTEIN_PRICE: {
        double x1 = x[0], x2 = x[1];
        double t = (x1 + x2) + 1.0;
        double pa = 19.0 - 14.0 * x1 + 3.0 * (x1 * x1) - 14.0 * x2
                    + 6.0 * (x1 * x2) + 3.0 * (x2 * x2);
        double a = 1.0 + (t * t) * pa;
        double u = 2.0 * x1 - 3.0 * x2;
        double pb = 18.0 - 32.0 * x1 + 12.0 * (x1 * x1) + 48.0 * x2
                    - 36.0 * (x1 * x2) + 27.0 * (x2 * x2);
        double b = 30.0 + (u * u) * pb;
        return a * b;
    }
    case ZO_QUADRATIC:
        zo_sum_start(&a0, d, 0.0, ord);
        for (int i = 0; i < d; ++i)
            zo_sum_add(&a0, i, 0.5 * (double)(i + 1) * (x[i] * x[i]));
        return zo_sum_end(&a0);
    case ZO_GRIEWANK: {
        double prod = 1.0;
        for (int i = 0; i < d; ++i) {
            s = s + x[i] * x[i];
            prod = prod * cos(x[i] / sqrt((double)(i + 1)));
        }
        return (1.0 + s / 4000.0) - prod;
    }
    case ZO_HIMMELBLAU: {
        double a = (x[0] * x[0] + x[1]) - 11.0;
        double b = (x[0] + x[1] * x[1]) - 7.0;
        return a * a + b * b;
    }
    default:
        return NAN;
    }
}

double zo_f(int obj, int d, const double *x) { return zo_f_ord(obj, d, x, ZO_ORDER_LIB); }

/* The same objectives written over dual numbers (Alg. 5 evaluates f on
 * xDual).  Operation order mirrors zo_f, so the value part equals zo_f. */
/* zo_sum on duals (the value part sums exactly as zo_f) */
typedef struct {
    zo_dual p[32];
    int split;
} zo_dsum;

static void zo_dsum_start(zo_dsum *a, int d, zo_dual c0, int ord)
{
    a->split = ord == ZO_ORDER_LIB && d > 32;
    for (int l = 0; l < 32; ++l) a->p[l] = dconst(0.0);
    a->p[0] = c0;
}
static void zo_dsum_add(zo_dsum *a, int j, zo_dual t)
{
    const int l = a->split ? (j & 31) : 0;
    a->p[l] = dadd(a->p[l], t);
}
static zo_dual zo_dsum_end(zo_dsum *a)
{
    if (a->split)
        for (int w = 16; w >= 1; w >>= 1)
            for (int l = 0; l < w; ++l) a->p[l] = dadd(a->p[l], a->p[l + w]);
    return a->p[0];
}

static zo_dual zo_f_dual(int obj, int d, const zo_dual *x, int ord)
{
    zo_dual s = dconst(0.0);
    zo_dsum a0, a1;
    switch (obj) {
    case ZO_ROSENBROCK:
        zo_dsum_start(&a0, d, dconst(0.0), ord);
        for (int i = 0; i + 1 < d; ++i) {
            zo_dual a = dsub(dconst(1.0), x[i]);
            zo_dual b = dsub(x[i + 1], dmul(x[i], x[i]));
            zo_dsum_add(&a0, i, dadd(dmul(a, a), dscale(100.0, dmul(b, b))));
        }
        return zo_dsum_end(&a0);
    case ZO_RASTRIGIN:
        zo_dsum_start(&a0, d, dconst(10.0 * (double)d), ord);
        for (int i = 0; i < d; ++i)
            zo_dsum_add(&a0, i, dsub(dmul(x[i], x[i]), dscale(10.0, dcos2pi(x[i]))));
        return zo_dsum_end(&a0);
    case ZO_ACKLEY: {
        zo_dsum_start(&a0, d, dconst(0.0), ord);
        zo_dsum_start(&a1, d, dconst(0.0), ord);
        for (int i = 0; i < d; ++i) {
            zo_dsum_add(&a0, i, dmul(x[i], x[i]));
            zo_dsum_add(&a1, i, dcos2pi(x[i]));
        }
        zo_dual s1 = zo_dsum_end(&a0), s2 = zo_dsum_end(&a1);
        zo_dual t1 = dscale(-20.0, dexp(dscale(-0.2, dsqrt(ddiv(s1, dconst((double)d))))));
        zo_dual t2 = dexp(ddiv(s2, dconst((double)d)));
        return dadd(dsub(t1, t2), dconst(20.0 + ZO_E));
    }
    case ZO_GOLDSTEIN_PRICE: {
        /* same left-to-right order as zo_f */
        zo_dual x1 = x[0], x2 = x[1];
        zo_dual t = dadd(dadd(x1, x2), dconst(1.0));
        zo_dual pa = dconst(19.0);
        pa = dsub(pa, dscale(14.0, x1));
        pa = dadd(pa, dscale(3.0, dmul(x1, x1)));
        pa = dsub(pa, dscale(14.0, x2));
        pa = dadd(pa, dscale(6.0, dmul(x1, x2)));
        pa = dadd(pa, dscale(3.0, dmul(x2, x2)));
        zo_dual a = dadd(dconst(1.0), dmul(dmul(t, t), pa));
        zo_dual u = dsub(dscale(2.0, x1), dscale(3.0, x2));
        zo_dual pb = dconst(18.0);
        pb = dsub(pb, dscale(32.0, x1));
        pb = dadd(pb, dscale(12.0, dmul(x1, x1)));
        pb = dadd(pb, dscale(48.0, x2));
        pb = dsub(pb, dscale(36.0, dmul(x1, x2)));
        pb = dadd(pb, dscale(27.0, dmul(x2, x2)));
        zo_dual b = dadd(dconst(30.0), dmul(dmul(u, u), pb));
        return dmul(a, b);
    }
    case ZO_QUADRATIC:
        zo_dsum_start(&a0, d, dconst(0.0), ord);
        for (int i = 0; i < d; ++i)
            zo_dsum_add(&a0, i, dscale(0.5 * (double)(i + 1), dmul(x[i], x[i])));
        return zo_dsum_end(&a0);
    case ZO_GRIEWANK: {
        zo_dual prod = dconst(1.0);
        for (int i = 0; i < d; ++i) {
            s = dadd(s, dmul(x[i], x[i]));
            prod = dmul(prod, dcos(ddiv(x[i], dconst(sqrt((double)(i + 1))))));
        }
        return dsub(dadd(dconst(1.0), ddiv(s, dconst(4000.0))), prod);
    }
    case ZO_HIMMELBLAU: {
        zo_dual a = dsub(dadd(dmul(x[0], x[0]), x[1]), dconst(11.0));
        zo_dual b = dsub(dadd(x[0], dmul(x[1], x[1])), dconst(7.0));
        return dadd(dmul(a, a), dmul(b, b));
    }
    default:
        return dconst(NAN);
    }
}

/* Alg. 5 (forwardAD): d passes; pass i seeds the tangent of x_i with 1,
 * evaluates f on duals and reads the tangent as df/dx_i.  The value part
 * of the first pass is returned as f(x) (reading: the line search's f0 is
 * this value). */
void zo_grad_forward_ord(int obj, int d, const double *x, double *f, double *g, int ord)
{
    zo_dual *xd = (zo_dual *)malloc(sizeof(zo_dual) * (size_t)(d > 0 ? d : 1));
    for (int i = 0; i < d; ++i) { xd[i].a = x[i]; xd[i].b = 0.0; }
    double fval = NAN;
    for (int i = 0; i < d; ++i) {
        xd[i].b = 1.0;
        zo_dual r = zo_f_dual(obj, d, xd, ord);
        g[i] = r.b;
        if (i == 0) fval = r.a;
        xd[i].b = 0.0;
    }
    if (d == 0) fval = zo_f_ord(obj, d, x, ord);
    *f = fval;
    free(xd);
}

void zo_grad_forward(int obj, int d, const double *x, double *f, double *g)
{
    zo_grad_forward_ord(obj, d, x, f, g, ZO_ORDER_LIB);
}

/* ------------------------------------------------------------------------ */
/* Argmin (Alg. 7 ParallelReduction).  Reading: NaN counts as +inf, ties go  */
/* to the lowest index.                                                      */
/* ------------------------------------------------------------------------ */

int64_t zo_argmin(const double *f, int64_t n)
{
    int64_t best = -1;
    double bf = INFINITY;
    for (int64_t i = 0; i < n; ++i) {
        double v = isnan(f[i]) ? INFINITY : f[i];
        if (best < 0 || v < bf) { best = i; bf = v; }
    }
    return best;
}

/* ------------------------------------------------------------------------ */
/* PSO (Alg. 2 InitSwarm, Alg. 3 UpdateSwarm).                               */
/* Reading: the global best is refreshed once per iteration from the         */
/* personal bests (synchronous), r1 and r2 are drawn per dimension, no       */
/* clamping is applied, and exactly pso_iters updates are made.              */
/* ------------------------------------------------------------------------ */

static double fmin_nan(double v) { return isnan(v) ? INFINITY : v; }

void zo_pso(const zo_problem *pr, double *x, double *v, double *px,
            double *pf, double *gx, double *gf, int64_t *gidx)
{
    const int d = pr->dim;
    const int64_t n = pr->n_starts;
    const double lo = pr->lower, hi = pr->upper;
    const double vr = hi - lo;          /* Alg. 2: vel_range = upper - lower */
    const double vlo = -vr, vhi = vr;
#ifdef _OPENMP
    if (pr->n_threads > 0) omp_set_num_threads(pr->n_threads);
#endif
    /* Alg. 2 */
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        for (int j = 0; j < d; ++j) {
            double ux = zo_uniform(pr->seed, 0, 0, (uint64_t)i, (uint64_t)j);
            double uv = zo_uniform(pr->seed, 0, 1, (uint64_t)i, (uint64_t)j);
            x[i * d + j] = lo + (hi - lo) * ux;
            v[i * d + j] = vlo + (vhi - vlo) * uv;
            px[i * d + j] = x[i * d + j];
        }
        pf[i] = zo_f_ord(pr->objective, d, x + i * d, pr->order);
    }
    int64_t b = zo_argmin(pf, n);
    *gidx = b;
    *gf = fmin_nan(pf[b]);
    for (int j = 0; j < d; ++j) gx[j] = px[b * d + j];

    /* Alg. 3, pso_iters times */
    for (int t = 0; t < pr->pso_iters; ++t) {
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < n; ++i) {
            double *xi = x + i * d, *vi = v + i * d, *pi = px + i * d;
            for (int j = 0; j < d; ++j) {
                double r1 = zo_uniform(pr->seed, 0, 2 + 2 * (uint64_t)t, (uint64_t)i, (uint64_t)j);
                double r2 = zo_uniform(pr->seed, 0, 3 + 2 * (uint64_t)t, (uint64_t)i, (uint64_t)j);
                double vn = pr->w * vi[j] + (pr->c1 * r1) * (pi[j] - xi[j])
                            + (pr->c2 * r2) * (gx[j] - xi[j]);
                vi[j] = vn;
                xi[j] = xi[j] + vn;
            }
            double fv = zo_f_ord(pr->objective, d, xi, pr->order);
            if (fv < pf[i]) {
                pf[i] = fv;
                for (int j = 0; j < d; ++j) pi[j] = xi[j];
            }
        }
        b = zo_argmin(pf, n);
        *gidx = b;
        *gf = fmin_nan(pf[b]);
        for (int j = 0; j < d; ++j) gx[j] = px[b * d + j];
    }
}

/* ------------------------------------------------------------------------ */
/* Backtracking Armijo line search (Alg. 6).                                 */
/* Returns alpha; *accepted = 1 if the Armijo test held for some trial.      */
/* Reading: trials m = 0..L-1; if none is accepted the returned alpha is     */
/* the value after the last halving (beta^L), as in the printed loop.        */
/* ------------------------------------------------------------------------ */

/* Relative margin of the comparison lhs <= rhs (or lhs < rhs), scaled by
 * the magnitudes compared: below ~1e-12 a last-bit difference in either
 * side could take the other branch. */
static double track_margin(double margin, double lhs, double rhs)
{
    double s = fabs(lhs) > fabs(rhs) ? fabs(lhs) : fabs(rhs);
    double m = fabs(lhs - rhs) / (s > 1e-300 ? s : 1e-300);
    return m < margin ? m : margin;
}

double zo_line_search_ord(int obj, int d, const double *x, const double *p,
                          double f0, double ddir, double c, double beta, int L,
                          double *xt, int *accepted, int *n_feval, double *margin, int ord)
{
    double alpha = 1.0;
    *accepted = 0;
    for (int m = 0; m < L; ++m) {
        for (int j = 0; j < d; ++j) xt[j] = x[j] + alpha * p[j];
        double ft = zo_f_ord(obj, d, xt, ord);
        (*n_feval)++;
        double rhs = f0 + c * alpha * ddir;
        if (margin) *margin = track_margin(*margin, ft, rhs);
        if (ft <= rhs) { *accepted = 1; break; }
        alpha = beta * alpha;
    }
    return alpha;
}

double zo_line_search(int obj, int d, const double *x, const double *p,
                      double f0, double ddir, double c, double beta, int L,
                      double *xt, int *accepted, int *n_feval, double *margin)
{
    return zo_line_search_ord(obj, d, x, p, f0, ddir, c, beta, L, xt, accepted, n_feval,
                              margin, ZO_ORDER_LIB);
}

/* ------------------------------------------------------------------------ */
/* Dot products and matrix-vector products (Alg. 4: H g, g^T p, y^T s,      */
/* H y, y^T H y).  The paper fixes them only in exact terms.                */
/* Plain order: acc = acc + a_i b_i in index order, the product and the sum */
/* each rounded.  Library order: every product term accumulated with one    */
/* rounding, acc = fma(a_i, b_i, acc), in index order.                      */
/* ------------------------------------------------------------------------ */

static double zo_dot(int n, const double *a, const double *b)
{
    double acc = 0.0;
    for (int i = 0; i < n; ++i) acc = fma(a[i], b[i], acc);
    return acc;
}

static double zo_pdot(int n, const double *a, const double *b)
{
    double acc = 0.0;
    for (int i = 0; i < n; ++i) acc = acc + a[i] * b[i];
    return acc;
}

/* The dot products of the BFGS step (||g||^2, g^T p, y^T s, s^T s, y^T y,
 * y^T H y) in the library order: for n <= 32 as zo_dot; for n > 32, 32
 * partial sums, partial l over the indices j = l (mod 32) in increasing
 * order, each term with one rounding (fma), then added pairwise in a fixed
 * tree: partial l with partial l + 16 (l < 16), then l with l + 8 (l < 8),
 * l + 4, l + 2, l + 1.  This order lets 32 lanes form one sum. */
static double zo_bdot(int n, const double *a, const double *b)
{
    if (n <= 32) return zo_dot(n, a, b);
    double p[32];
    for (int l = 0; l < 32; ++l) {
        double acc = 0.0;
        for (int j = l; j < n; j += 32) acc = fma(a[j], b[j], acc);
        p[l] = acc;
    }
    for (int w = 16; w >= 1; w >>= 1)
        for (int l = 0; l < w; ++l) p[l] = p[l] + p[l + w];
    return p[0];
}

/* a step dot product in the given order */
static double zo_sdot(int n, const double *a, const double *b, int ord)
{
    return ord == ZO_ORDER_PLAIN ? zo_pdot(n, a, b) : zo_bdot(n, a, b);
}

/* zo_bdot and zo_pdot for the tests */
double zo_dot_split(int n, const double *a, const double *b) { return zo_bdot(n, a, b); }
double zo_dot_plain(int n, const double *a, const double *b) { return zo_pdot(n, a, b); }

/* out = M v for row-major M [d][d], each row one chain in index order
 * (fma per term in the library order, plain otherwise) */
static void zo_matvec(int d, const double *M, const double *v, double *out, int ord)
{
    for (int r = 0; r < d; ++r)
        out[r] = ord == ZO_ORDER_PLAIN ? zo_pdot(d, M + (size_t)r * d, v)
                                       : zo_dot(d, M + (size_t)r * d, v);
}

/* ------------------------------------------------------------------------ */
/* Inverse-Hessian rank-two update (the update formula of Alg. 4).           */
/* The printed product form (I - rho s y^T) H (I - rho y s^T) + rho s s^T    */
/* expands, for symmetric H, to                                              */
/*   H - rho (Hy s^T + s (Hy)^T) + (rho^2 y^T H y + rho) s s^T.              */
/* Plain order: every element (r, c) of the whole matrix from that           */
/* expression as written, each operation rounded on its own:                 */
/*   H_rc <- (H_rc - rho ((Hy)_r s_c + s_r (Hy)_c)) + beta (s_r s_c),        */
/* beta = rho^2 y^T H y + rho (H stays symmetric: the expression is).        */
/* Library order: the element regrouped as H_rc + s_c A_r + (Hy)_c B_r with  */
/*   A_r = beta s_r - rho (Hy)_r,  B_r = -rho s_r,                           */
/* two fused multiply-adds, H_rc <- fma(s_c, A_r, fma((Hy)_c, B_r, H_rc)),   */
/* A_r = fma(beta, s_r, -(rho (Hy)_r)), over the elements r <= c, mirrored.  */
/* Reading: skipped when y^T s <= 1e-12 |s| |y|.  Returns 1 if applied.      */
/* ------------------------------------------------------------------------ */

int zo_bfgs_update_ord(int d, double *H, const double *s, const double *y, int ord)
{
    const double sy = zo_sdot(d, y, s, ord), ss = zo_sdot(d, s, s, ord),
                 yy = zo_sdot(d, y, y, ord);
    if (!(sy > 1e-12 * sqrt(ss) * sqrt(yy))) return 0;
    double rho = 1.0 / sy;
    double *Hy = (double *)malloc(sizeof(double) * (size_t)d * 3);
    double *A = Hy + d, *B = Hy + 2 * d;
    zo_matvec(d, H, y, Hy, ord);
    const double yHy = zo_sdot(d, y, Hy, ord);
    const double beta = rho * rho * yHy + rho;
    if (ord == ZO_ORDER_PLAIN) {
        for (int r = 0; r < d; ++r)
            for (int c = 0; c < d; ++c)
                H[r * d + c] = H[r * d + c] - rho * (Hy[r] * s[c] + s[r] * Hy[c])
                               + beta * (s[r] * s[c]);
        free(Hy);
        return 1;
    }
    for (int r = 0; r < d; ++r) {
        A[r] = fma(beta, s[r], -(rho * Hy[r]));
        B[r] = -(rho * s[r]);
    }
    for (int r = 0; r < d; ++r)
        for (int c = r; c < d; ++c) {
            const double v = fma(s[c], A[r], fma(Hy[c], B[r], H[r * d + c]));
            H[r * d + c] = v;
            H[c * d + r] = v;
        }
    free(Hy);
    return 1;
}

int zo_bfgs_update(int d, double *H, const double *s, const double *y)
{
    return zo_bfgs_update_ord(d, H, s, y, ZO_ORDER_LIB);
}

/* ------------------------------------------------------------------------ */
/* Limited-memory direction (L-BFGS, the paper's future work, Section VI):   */
/* the two-loop recursion of Nocedal & Wright, Numerical Optimization,       */
/* Alg. 7.4, over the n stored pairs (s_i, y_i), oldest first, with         */
/* rho_i = 1 / y_i's_i and the initial matrix gamma I, gamma = s'y / y'y of  */
/* the newest pair (their eq. 7.20; 1 when no pair is stored).  Returns      */
/* p = -H g in p.  Library order: dot products as zo_dot, each update of q   */
/* and r one fused multiply-add per element; plain order: plain dot          */
/* products, each product and sum of an update rounded on its own.           */
/* ------------------------------------------------------------------------ */

void zo_lbfgs_direction_ord(int d, int n, const double *S, const double *Y, const double *rho,
                            const double *g, double *p, int ord)
{
    const int plain = ord == ZO_ORDER_PLAIN;
    double *q = (double *)malloc(sizeof(double) * (size_t)(d > 0 ? d : 1));
    double *al = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    for (int j = 0; j < d; ++j) q[j] = g[j];
    for (int i = n - 1; i >= 0; --i) {
        const double *si = S + (size_t)i * d, *yi = Y + (size_t)i * d;
        al[i] = rho[i] * (plain ? zo_pdot(d, si, q) : zo_dot(d, si, q));
        for (int j = 0; j < d; ++j)
            q[j] = plain ? q[j] - al[i] * yi[j] : fma(-al[i], yi[j], q[j]);
    }
    double gamma = 1.0;
    if (n > 0) {
        const double *sn = S + (size_t)(n - 1) * d, *yn = Y + (size_t)(n - 1) * d;
        gamma = plain ? zo_pdot(d, sn, yn) / zo_pdot(d, yn, yn)
                      : zo_dot(d, sn, yn) / zo_dot(d, yn, yn);
    }
    for (int j = 0; j < d; ++j) q[j] = gamma * q[j];  /* r = gamma q, in place */
    for (int i = 0; i < n; ++i) {
        const double *si = S + (size_t)i * d, *yi = Y + (size_t)i * d;
        const double b = rho[i] * (plain ? zo_pdot(d, yi, q) : zo_dot(d, yi, q));
        for (int j = 0; j < d; ++j)
            q[j] = plain ? q[j] + (al[i] - b) * si[j] : fma(al[i] - b, si[j], q[j]);
    }
    for (int j = 0; j < d; ++j) p[j] = -q[j];
    free(q);
    free(al);
}

void zo_lbfgs_direction(int d, int n, const double *S, const double *Y, const double *rho,
                        const double *g, double *p)
{
    zo_lbfgs_direction_ord(d, n, S, Y, rho, g, p, ZO_ORDER_LIB);
}

/* Stores the pair (s, y) as the newest of at most m (the oldest is dropped)
 * if it passes the curvature test of zo_bfgs_update; returns 1 if stored. */
static int zo_lbfgs_push(int d, int m, int *n, double *S, double *Y, double *rho,
                         const double *s, const double *y, int ord)
{
    const int plain = ord == ZO_ORDER_PLAIN;
    const double sy = plain ? zo_pdot(d, y, s) : zo_dot(d, y, s);
    const double ss = plain ? zo_pdot(d, s, s) : zo_dot(d, s, s);
    const double yy = plain ? zo_pdot(d, y, y) : zo_dot(d, y, y);
    if (!(sy > 1e-12 * sqrt(ss) * sqrt(yy))) return 0;
    if (*n == m) {  /* drop the oldest */
        memmove(S, S + d, sizeof(double) * (size_t)(m - 1) * d);
        memmove(Y, Y + d, sizeof(double) * (size_t)(m - 1) * d);
        memmove(rho, rho + 1, sizeof(double) * (size_t)(m - 1));
        *n = m - 1;
    }
    memcpy(S + (size_t)(*n) * d, s, sizeof(double) * (size_t)d);
    memcpy(Y + (size_t)(*n) * d, y, sizeof(double) * (size_t)d);
    rho[*n] = 1.0 / sy;
    *n += 1;
    return 1;
}

/* ------------------------------------------------------------------------ */
/* Search direction of Alg. 4: p = -H g and ddir = g^T p.  Reading: when p   */
/* is not a descent direction (ddir < 0 fails, which also catches NaN), H is  */
/* reset to the identity and p = -g, ddir = g^T p recomputed.  Returns 1 if   */
/* the reset was taken.                                                      */
/* ------------------------------------------------------------------------ */

int zo_direction(int d, double *H, const double *g, double *p, double *ddir, int ord)
{
    zo_matvec(d, H, g, p, ord);
    for (int r = 0; r < d; ++r) p[r] = -p[r];
    double dd = zo_sdot(d, g, p, ord);
    int reset = 0;
    if (!(dd < 0.0)) {
        for (int i = 0; i < d * d; ++i) H[i] = 0.0;
        for (int i = 0; i < d; ++i) H[i * d + i] = 1.0;
        for (int r = 0; r < d; ++r) p[r] = -g[r];
        dd = zo_sdot(d, g, p, ord);
        reset = 1;
    }
    *ddir = dd;
    return reset;
}

/* ------------------------------------------------------------------------ */
/* One BFGS run (Alg. 4, with the per-thread body of Alg. 10).               */
/* Readings: the gradient at x_new is reused as the next iteration's         */
/* gradient; a non-descent direction resets H to I and uses p = -g; the      */
/* convergence test ||g|| < tol is made at the top of each iteration only;   */
/* status 3 marks a non-finite f or g.  stop (may be NULL) is the shared     */
/* stop flag of Alg. 10.                                                     */
/* ------------------------------------------------------------------------ */

static int finite_vec(int d, const double *v)
{
    for (int i = 0; i < d; ++i)
        if (!isfinite(v[i])) return 0;
    return 1;
}

void zo_bfgs(const zo_problem *pr, const double *x0, double *x_out,
             zo_result *res, volatile int *stop, volatile int64_t *n_conv)
{
    const int d = pr->dim, obj = pr->objective;
    size_t nb = sizeof(double) * (size_t)(d > 0 ? d : 1);
    /* L-BFGS history (m > 0): pairs oldest first; the dense H otherwise */
    const int m = pr->lbfgs_m;
    int n_pairs = 0;
    double *H = NULL, *S = NULL, *Y = NULL, *rho = NULL;
    if (m > 0) {
        S = (double *)malloc(nb * (size_t)m);
        Y = (double *)malloc(nb * (size_t)m);
        rho = (double *)malloc(sizeof(double) * (size_t)m);
    } else {
        H = (double *)malloc(nb * (size_t)(d > 0 ? d : 1));
        for (int i = 0; i < d * d; ++i) H[i] = 0.0;
        for (int i = 0; i < d; ++i) H[i * d + i] = 1.0;
    }
    double *x = (double *)malloc(nb), *g = (double *)malloc(nb);
    double *p = (double *)malloc(nb), *xn = (double *)malloc(nb);
    double *gn = (double *)malloc(nb), *s = (double *)malloc(nb);
    double *y = (double *)malloc(nb);
    const int ord = pr->order;
    for (int i = 0; i < d; ++i) x[i] = x0[i];
    double f0;
    zo_grad_forward_ord(obj, d, x, &f0, g, ord);
    double margin = INFINITY;
    int k = 0, status = 0, n_feval = 0;
    double gnorm = NAN;
    for (;;) {
        gnorm = sqrt(zo_sdot(d, g, g, ord));
        if (k >= pr->bfgs_max_iters) { status = 0; break; }
        if (stop && *stop) { status = 2; break; }
        if (!isfinite(f0) || !finite_vec(d, g)) { status = 3; break; }
        margin = track_margin(margin, gnorm, pr->grad_tol);
        if (gnorm < pr->grad_tol) {
            status = 1;
            if (n_conv) {
                int64_t c;
#pragma omp atomic capture
                c = ++(*n_conv);
                if (stop && pr->required_converged > 0 && c >= pr->required_converged)
                    *stop = 1;
            }
            break;
        }
        if (!isnan(pr->target_f) && f0 <= pr->target_f) {
            status = 1;
            if (stop) *stop = 1;
            break;
        }
        /* p = -H g, ddir = g^T p (reading: a non-descent direction restarts
         * from H = I, p = -g; L-BFGS forgets its stored pairs) */
        double ddir;
        if (m > 0) {
            zo_lbfgs_direction_ord(d, n_pairs, S, Y, rho, g, p, ord);
            ddir = zo_sdot(d, g, p, ord);
            if (!(ddir < 0.0)) {
                n_pairs = 0;
                for (int r = 0; r < d; ++r) p[r] = -g[r];
                ddir = zo_sdot(d, g, p, ord);
            }
        } else {
            zo_direction(d, H, g, p, &ddir, ord);
        }
        int accepted = 0;
        double alpha = zo_line_search_ord(obj, d, x, p, f0, ddir, pr->armijo_c,
                                          pr->backtrack, pr->ls_max_iters, xn,
                                          &accepted, &n_feval, &margin, ord);
        for (int j = 0; j < d; ++j) xn[j] = x[j] + alpha * p[j];
        double fn;
        zo_grad_forward_ord(obj, d, xn, &fn, gn, ord);
        for (int j = 0; j < d; ++j) {
            s[j] = xn[j] - x[j];
            y[j] = gn[j] - g[j];
        }
        if (m > 0)
            zo_lbfgs_push(d, m, &n_pairs, S, Y, rho, s, y, ord);
        else
            zo_bfgs_update_ord(d, H, s, y, ord);
        for (int j = 0; j < d; ++j) { x[j] = xn[j]; g[j] = gn[j]; }
        f0 = fn;
        ++k;
    }
    for (int j = 0; j < d; ++j) x_out[j] = x[j];
    res->f = f0;
    res->gnorm = gnorm;
    res->margin = margin;
    res->iters = k;
    res->status = status;
    res->n_feval = n_feval;
    res->pad = 0;
    free(H); free(x); free(g); free(p); free(xn); free(gn); free(s); free(y);
    free(S); free(Y); free(rho);
}

/* BFGS from n given starts (x0 row-major [n][d]); OpenMP over starts. */
void zo_bfgs_many(const zo_problem *pr, int64_t n, const double *x0,
                  double *x_out, zo_result *res)
{
    volatile int stop = 0;
    volatile int64_t n_conv = 0;
    const int use_stop = pr->required_converged > 0 || !isnan(pr->target_f);
#ifdef _OPENMP
    if (pr->n_threads > 0) omp_set_num_threads(pr->n_threads);
#endif
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t i = 0; i < n; ++i)
        zo_bfgs(pr, x0 + i * pr->dim, x_out + i * pr->dim, res + i,
                use_stop ? &stop : NULL, use_stop ? &n_conv : NULL);
}

/* Whole method (Alg. 7): PSO, then BFGS from every particle's current
 * position (or personal best), then argmin of the BFGS final values. */
int64_t zo_solve(const zo_problem *pr, double *x, double *v, double *px,
                 double *pf, double *gx, double *x_out, zo_result *res)
{
    double gf;
    int64_t gi;
    zo_pso(pr, x, v, px, pf, gx, &gf, &gi);
    const double *starts = pr->start_from_pbest ? px : x;
    zo_bfgs_many(pr, pr->n_starts, starts, x_out, res);
    double *fo = (double *)malloc(sizeof(double) * (size_t)pr->n_starts);
    for (int64_t i = 0; i < pr->n_starts; ++i) fo[i] = res[i].f;
    int64_t b = zo_argmin(fo, pr->n_starts);
    free(fo);
    return b;
}

/* ------------------------------------------------------------------------ */
/* Test-only: BFGS on f = 0.5 x^T A x (A dense SPD, row-major) with the      */
/* exact line search alpha = -g^T p / (p^T A p).  Used to pin the update:    */
/* with exact steps BFGS terminates on a quadratic in at most d iterations   */
/* and H_d = A^{-1} (Nocedal & Wright, Numerical Optimization, Thm. 6.4 /    */
/* the quadratic-termination property of the Broyden class).  Uses the same  */
/* zo_bfgs_update_ord as the main path, in the order asked for.  Returns the  */
/* iterations taken; H is                                                    */
/* left in H_out.                                                            */
/* ------------------------------------------------------------------------ */

int zo_bfgs_quadratic_exact(int d, const double *A, const double *x0,
                            int max_iters, double tol, double *x_out,
                            double *H_out, int ord)
{
    size_t nb = sizeof(double) * (size_t)d;
    double *x = (double *)malloc(nb), *g = (double *)malloc(nb);
    double *p = (double *)malloc(nb), *Ap = (double *)malloc(nb);
    double *s = (double *)malloc(nb), *y = (double *)malloc(nb);
    double *H = H_out;
    for (int i = 0; i < d; ++i) x[i] = x0[i];
    for (int i = 0; i < d * d; ++i) H[i] = 0.0;
    for (int i = 0; i < d; ++i) H[i * d + i] = 1.0;
    int k = 0;
    for (;;) {
        double gg = 0.0;
        for (int r = 0; r < d; ++r) {
            double a = 0.0;
            for (int c = 0; c < d; ++c) a = a + A[r * d + c] * x[c];
            g[r] = a;
            gg = gg + a * a;
        }
        if (sqrt(gg) < tol || k >= max_iters) break;
        double gp = 0.0, pAp = 0.0;
        for (int r = 0; r < d; ++r) {
            double a = 0.0;
            for (int c = 0; c < d; ++c) a = a + H[r * d + c] * g[c];
            p[r] = -a;
        }
        for (int r = 0; r < d; ++r) {
            double a = 0.0;
            for (int c = 0; c < d; ++c) a = a + A[r * d + c] * p[c];
            Ap[r] = a;
            gp = gp + g[r] * p[r];
        }
        for (int r = 0; r < d; ++r) pAp = pAp + p[r] * Ap[r];
        double alpha = -gp / pAp;
        for (int r = 0; r < d; ++r) {
            s[r] = alpha * p[r];
            x[r] = x[r] + s[r];
            y[r] = alpha * Ap[r];     /* y = A s */
        }
        zo_bfgs_update_ord(d, H, s, y, ord);
        ++k;
    }
    for (int i = 0; i < d; ++i) x_out[i] = x[i];
    free(x); free(g); free(p); free(Ap); free(s); free(y);
    return k;
}

/* ------------------------------------------------------------------------ */
/* Solution clustering (Section VI, future work: group the candidate         */
/* solutions by function value or by coordinates; the number of starts in   */
/* the region of the lowest f measures the confidence in it).               */
/* Reading: leader clustering.  The candidates (finite f; with               */
/* only_converged, status 1 only) are visited in order of increasing         */
/* (f, start index).  A candidate joins the first leader, in the order the  */
/* leaders were made, that it is within tol of; if there is none it becomes */
/* a new leader, unless max_clusters leaders exist already, in which case  */
/* it is left out (label -2).  Non-candidates get label -1.                 */
/* "Within tol" of leader L: method 0 (by f) |f_i - f_L| <= tol max(1,|f_L|);*/
/* method 1 (by x) sum_j (x_ij - x_Lj)^2 <= tol^2, summed in index order    */
/* with one rounding per term (fma), the FMA reading of the dot products.  */
/* ------------------------------------------------------------------------ */

typedef struct {
    int64_t n_candidates, n_clusters, n_left, best_count, best_leader;
    double best_f, best_spread;
    int32_t error, pad;
} zo_cluster_result;

typedef struct {
    double f;
    int64_t i;
} zo_key;

static int zo_key_cmp(const void *a, const void *b)
{
    const zo_key *p = (const zo_key *)a, *q = (const zo_key *)b;
    if (p->f < q->f) return -1;
    if (p->f > q->f) return 1;
    return (p->i > q->i) - (p->i < q->i);
}

/* distance of start i to leader l (by x: the Euclidean norm of the sum
 * above; by f: |f_i - f_l|) and whether it is within tol */
static int zo_within(int method, double tol, int d, const double *x, const double *f,
                     int64_t i, int64_t l, double *dist)
{
    if (method == 1) {
        double acc = 0.0;
        for (int j = 0; j < d; ++j) {
            double del = x[i * d + j] - x[l * d + j];
            acc = fma(del, del, acc);
        }
        *dist = sqrt(acc);
        return acc <= tol * tol;
    }
    *dist = fabs(f[i] - f[l]);
    return *dist <= tol * fmax(1.0, fabs(f[l]));
}

int zo_cluster(int method, double tol, int32_t max_clusters, int only_converged, int64_t n,
               int d, const double *x, const double *f, const int32_t *status, int32_t *label,
               int32_t *leader, int32_t *count, zo_cluster_result *res)
{
    zo_key *keys = (zo_key *)malloc(sizeof(zo_key) * (size_t)(n > 0 ? n : 1));
    int64_t m = 0, left = 0;
    for (int64_t i = 0; i < n; ++i) {
        label[i] = -1;
        if (isfinite(f[i]) && (!only_converged || status[i] == 1)) {
            keys[m].f = f[i];
            keys[m].i = i;
            ++m;
        }
    }
    qsort(keys, (size_t)m, sizeof(zo_key), zo_key_cmp);
    for (int k = 0; k < max_clusters; ++k) { leader[k] = -1; count[k] = 0; }
    int K = 0;
    double spread0 = 0.0;
    for (int64_t q = 0; q < m; ++q) {
        const int64_t i = keys[q].i;
        int joined = 0;
        for (int k = 0; k < K && !joined; ++k) {
            double dist;
            if (zo_within(method, tol, d, x, f, i, leader[k], &dist)) {
                label[i] = k;
                count[k] += 1;
                if (k == 0 && dist > spread0) spread0 = dist;
                joined = 1;
            }
        }
        if (joined) continue;
        if (K < max_clusters) {
            leader[K] = (int32_t)i;
            count[K] = 1;
            label[i] = K;
            ++K;
        } else {
            label[i] = -2;
            ++left;
        }
    }
    res->n_candidates = m;
    res->n_clusters = K;
    res->n_left = left;
    res->best_count = K > 0 ? count[0] : 0;
    res->best_leader = K > 0 ? leader[0] : -1;
    res->best_f = K > 0 ? f[leader[0]] : NAN;
    res->best_spread = K > 0 ? spread0 : NAN;
    res->error = 0;
    res->pad = 0;
    free(keys);
    return 0;
}

int zo_sizeof_problem(void) { return (int)sizeof(zo_problem); }
int zo_sizeof_result(void) { return (int)sizeof(zo_result); }
int zo_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
