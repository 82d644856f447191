// zeus_bfgs.cu -- one BFGS run per start (Alg. 4, per-thread body of
// Alg. 10) in two kernels: launch planning here, the kernels in
// zeus_bfgs_kernels.cu, the per-start bodies in zeus_bfgs.cuh.
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
// shared memory and one thread adds them), dot and matrix-vector products
// take one fused multiply-add per term, no other FMA contraction, the same
// elementary functions.  A run is therefore bitwise independent of which
// kernel carried it and of the hand-over point.
//
// Per iteration (readings of the paper are listed in the design notes):
//   ||g|| < tol -> converged; p = -H g (reset H = I, p = -g if not a descent
//   direction); backtracking Armijo line search (Alg. 6); x_new = x + a p;
//   g at x_new; y = g_new - g, s = x_new - x; if y's > 1e-12 |s||y|: the
//   product update printed in Alg. 4, expanded for symmetric H and grouped
//   by rows, H_rc <- H_rc + s_c A_r + (Hy)_c B_r with A = b2 s - rho Hy,
//   B = -rho s, b2 = rho^2 y'Hy + rho: two fused multiply-adds per element.
#include "zeus_bfgs.cuh"

namespace zeus {

// ---------------------------------------------------------------------------
// Launch planning
// ---------------------------------------------------------------------------
int plan_bfgs(const zeus_problem& p, BfgsLaunch* L) {
    const int d = p.dim;
    const size_t cap = 226 * 1024;  // 227 KB per block, less the kernels' static shared memory
    const size_t ts = p.precision == ZEUS_FP32_GUARDED ? sizeof(float) : sizeof(double);
    const int req = p.threads_per_start;
    // user objectives run in the forms that hold H in shared memory
    const bool user = p.objective >= ZEUS_OBJ_USER;
    L->lbfgs = p.lbfgs_m > 0;
    if (L->lbfgs) {  // one 256-thread block per start, the pairs in shared memory
        if (p.objective == ZEUS_OBJ_GOLDSTEIN_PRICE || user || (req != 0 && req != 256))
            return ZEUS_EUNSUPPORTED;
        L->narrow = false;
        L->stride = 0;
        L->narrow_threads = 0;
        L->narrow_smem = 0;
        L->narrow_blocks = 0;
        L->W = 0;
        L->wide_smem = 0;
        L->wide_blocks = 0;
        L->budget = 0;
        L->q_cap = 0;
        L->stream = true;
        L->stream_smem = lbfgs_smem(d, p.lbfgs_m, ts);
        L->stream_blocks = stream_blocks(p, L->stream_smem);
        L->hslot_bytes = 0;
        return L->stream_smem <= cap ? ZEUS_OK : ZEUS_EUNSUPPORTED;
    }
    L->warp = false;
    L->warp_slot = 0;
    if (req == 32) {  // one warp per start, four starts to a block, H in shared memory
        L->narrow = false;
        L->stride = 0;
        L->narrow_threads = 0;
        L->narrow_smem = 0;
        L->narrow_blocks = 0;
        L->W = wide_trials(d, p.ls_max_iters, 32);
        L->wide_smem = wide_smem(d, L->W, p.ls_max_iters, ts);
        L->warp_slot = (L->wide_smem + 15) & ~size_t(15);
        L->wide_blocks = 152 * 4;
        L->budget = 0;
        L->q_cap = 0;
        L->stream = false;
        L->stream_blocks = 0;
        L->stream_smem = 0;
        L->hslot_bytes = 0;
        L->warp = true;
        // four slots of dynamic and four WideShared of static shared memory
        return 4 * L->warp_slot + 4 * sizeof(WideShared) <= 227 * 1024 ? ZEUS_OK
                                                                        : ZEUS_EUNSUPPORTED;
    }
    const size_t row = narrow_stride(d) * ts;
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
    L->wide_smem = wide_smem(d, L->W, p.ls_max_iters, ts);
    // H streamed from HBM when the block-per-start kernel could not hold the
    // full d x d matrix.  The packed triangle would fit up to about 1.4 times
    // that d, but only one such block fits an SM, and the streamed kernel
    // (four 256-thread blocks per SM) is faster there: 0.66 s against 2.48 s
    // for the d = 256 chain in FP32.
    const size_t full = wide_smem(d, L->W, p.ls_max_iters, ts) +
                        ((size_t)d * d - (size_t)d * (d + 1) / 2) * ts;
    L->stream = (req == 256) || (!L->narrow && full > cap);
    L->stream_smem = stream_smem(d, ts);
    L->stream_blocks = stream_blocks(p, L->stream_smem);
    // FP32 H streams as the tiled upper triangle, FP64 H as the full matrix
    L->hslot_bytes = !L->stream ? 0 : (size_t)L->stream_blocks * stream_slot_elems(d, ts) * ts;
    if (L->stream && (user || L->stream_smem > cap)) return ZEUS_EUNSUPPORTED;
    L->wide_blocks = 152 * 4;
    // hand-over budget (iterations + line-search evaluations) of the narrow
    // kernel; 0 = every start runs to its end in the narrow kernel.  Only
    // used when the wide kernel can hold the start (its shared memory fits).
    L->budget = (L->narrow && !L->stream && L->wide_smem <= cap && req != 1) ? 160 : 0;
    L->q_cap = 0;
    if (L->budget > 0) {
        // FP64: room for every start (a start that finds the queue full
        // runs on in its lane, at one lane's FP64 latency per iteration).
        // FP32 runs rarely meet the gradient tolerance and would all be
        // handed over: at most two per wide block, the long runs being the
        // bulk that stays in the throughput kernel.
        const long long lim = p.precision == ZEUS_FP32_GUARDED ? 2ll * L->wide_blocks : p.n_starts;
        long long capn = p.n_starts < lim ? p.n_starts : lim;
        const long long max_bytes = 256ll << 20;
        const long long per = (long long)d * d * 8;
        if (capn * per > max_bytes) capn = max_bytes / per;
        if (capn < 1) capn = 1;
        L->q_cap = (int)capn;
    }
    return ZEUS_OK;
}

cudaError_t launch_bfgs(const zeus_problem& p, const BfgsLaunch& L, const double* x0,
                        double* x_out, double* f_out, double* gnorm_out, int32_t* status_out,
                        int32_t* iters_out, Ctrl* ctrl, const Queue& q, cudaStream_t st) {
    if (L.stream)
        return launch_bfgs_stream(p, x0, x_out, f_out, gnorm_out, status_out, iters_out, ctrl,
                                  q.hslots, st);
    const bool f32 = p.precision == ZEUS_FP32_GUARDED;
    if (p.grad_mode == ZEUS_GRAD_ADJOINT)
        return f32 ? bfgs_launch_gt<ZEUS_GRAD_ADJOINT, float>(p, L, x0, x_out, f_out, gnorm_out,
                                                              status_out, iters_out, ctrl, q, st)
                   : bfgs_launch_gt<ZEUS_GRAD_ADJOINT, double>(p, L, x0, x_out, f_out, gnorm_out,
                                                               status_out, iters_out, ctrl, q, st);
    return f32 ? bfgs_launch_gt<ZEUS_GRAD_FORWARD, float>(p, L, x0, x_out, f_out, gnorm_out,
                                                          status_out, iters_out, ctrl, q, st)
               : bfgs_launch_gt<ZEUS_GRAD_FORWARD, double>(p, L, x0, x_out, f_out, gnorm_out,
                                                           status_out, iters_out, ctrl, q, st);
}

}  // namespace zeus
