// zeus_internal.h -- host/device contract between the C-ABI layer
// (zeus_capi.cu) and the kernel translation units.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "zeus.h"

namespace zeus {

// Control block at offset 0 of every workspace.  Zeroed (cudaMemsetAsync)
// at the start of each call; the kernels that use `blocks_done` reset it to
// zero when they finish, so kernels of one call can share it in turn.
struct Ctrl {
    unsigned int blocks_done;        // last-block counter of the fused grid reductions
    int stop;                        // shared stop flag (Alg. 10)
    int error;                       // device error word
    unsigned int q_count;            // starts handed from the narrow to the wide kernel
    unsigned int q_head;             // next queue item the wide kernel takes
    unsigned int tile_head;          // next lane tile of the fused kernel
    unsigned long long n_conv;       // starts that converged
    unsigned long long total_iters;  // sum of completed BFGS iterations
    unsigned long long total_feval;  // sum of line-search evaluations
    double gbest_f;                  // PSO global best value
    long long gbest_idx;             // and its particle
    unsigned long long h_reads;      // H passes that read a start's H from HBM (streamed H)
    unsigned long long h_writes;     // H passes that wrote it back
    unsigned int tiles_done;         // lane tiles the fused kernel has finished
    unsigned int q_count_long;       // entries handed over after a failed line search
    unsigned int q_head_long;        // next such entry a server takes
    unsigned int pad2;
    unsigned long long pad1[20];
};
static_assert(sizeof(Ctrl) == 256, "control block is one 256-byte segment");

// (value, index) pair of the argmin reductions
struct ArgPair {
    double f;
    long long idx;
};

constexpr int kMaxReduceBlocks = 4096;  // argmin partials kept in the workspace

// polls (of about 256 ns each) a bounded device wait makes before it gives
// up; zeus_set_wait_limit sets it, 2^23 (about 2 s) by default
constexpr unsigned kDefaultWaitPolls = 1u << 23;
unsigned wait_limit();

inline size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

// Streamed H (zeus_stream.cu) is held as the upper triangle of the
// symmetric matrix in tiles of th rows x 32 columns: tile (I, J) covers rows
// [I th, I th + th) and columns [32 J, 32 J + 32) of the matrix padded to
// dp (d rounded up to 32), and is stored when it holds an element r <= c,
// i.e. for J >= I th / 32; tiles follow one another by tile rows, J
// ascending.  Inside a tile, element (r, c) sits at ((r % th) / n) 32 n +
// (c % 32) n + r % n, n = 16 / sizeof(T): lane c % 32 of a warp reads n
// consecutive rows of its column as one 16-byte vector, and the warp reads
// 512 contiguous bytes.  th = dp / 16 (at least n, at most 32, a power of
// two), so that a matrix has at least 16 tile rows: eight warps take them
// in pairs (I, TR - 1 - I), which hold the same number of tiles.
struct TileGeo {
    int th;  // rows per tile
    int tr;  // tile rows, dp / th
    int tc;  // tile columns, dp / 32
    int dp;  // d rounded up to 32
};
__host__ __device__ inline TileGeo tile_geo(int d, int n) {
    TileGeo t;
    t.dp = (d + 31) / 32 * 32;
    int th = t.dp / 16;
    if (th > 32) th = 32;
    int p2 = 1;
    while (p2 * 2 <= th) p2 *= 2;
    t.th = p2 < n ? n : p2;
    t.tr = t.dp / t.th;
    t.tc = t.dp / 32;
    return t;
}
__host__ __device__ inline int tile_jmin(const TileGeo& t, int I) { return (I * t.th) / 32; }
// tiles before tile row I
__host__ __device__ inline long long tile_row_first(const TileGeo& t, int I) {
    long long s = 0;
    for (int i = 0; i < I; ++i) s += t.tc - tile_jmin(t, i);
    return s;
}
__host__ __device__ inline long long tile_slot_elems(int d, int n) {
    const TileGeo t = tile_geo(d, n);
    return tile_row_first(t, t.tr) * t.th * 32;
}
inline size_t tile_slot_bytes(int d, size_t tsize) {
    return (size_t)tile_slot_elems(d, (int)(16 / tsize)) * tsize;
}
// FP32 H streams as the tiled triangle where the pass's shared memory (ten
// vectors and eight warps' column partials of dp elements) fits a block;
// FP64 H, and FP32 H beyond that d (about 3200), stream as the full matrix
__host__ __device__ inline bool stream_tiled(int d, size_t tsize) {
    return tsize == 4 && (size_t)18 * tile_geo(d, 4).dp * 4 <= (size_t)226 * 1024;
}
// elements of one block's H slot
__host__ __device__ inline long long stream_slot_elems(int d, size_t tsize) {
    return stream_tiled(d, tsize) ? tile_slot_elems(d, 4) : (long long)d * d;
}

// Raises a kernel's dynamic shared-memory limit to the most the device
// allows beside the kernel's static shared memory: the same value on every
// call, so that calls from several host threads never lower it under one
// another's launch.  Fails (cudaErrorInvalidValue) if `need` does not fit.
template <class K>
inline cudaError_t allow_smem(K* kernel, size_t need) {
    int dev = 0, optin = 0;
    cudaFuncAttributes fa;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, kernel);
    if (e != cudaSuccess) return e;
    const int maxdyn = optin - (int)fa.sharedSizeBytes;
    if ((long long)need > (long long)maxdyn) return cudaErrorInvalidValue;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, maxdyn);
}

// Workspace carve-up (offsets in bytes from the workspace base).
constexpr int kMaxSMs = 1024;  // size of the per-SM table of the fused kernel

struct Layout {
    size_t ctrl, q_ready, q_smlong, partials, f_tmp, v, px, pf, gx, q_start, q_k, q_feval, q_h, hslots, total;
};

// Per-problem inputs and outputs of a BFGS run (pointers already offset to
// the problem's rows) and its counters.
struct RunIO {
    const double* x0;
    double* x_out;
    double* f_out;
    double* gnorm_out;
    int32_t* status_out;
    int32_t* iters_out;
    Ctrl* pc;
};

// Hand-over queue from the narrow to the wide BFGS kernel (workspace).
struct Queue {
    int* prob;    // [cap] problem index (batched runs; nullptr otherwise)
    int* start;   // [cap] start index
    int* k;       // [cap] iteration at hand-over
    int* feval;   // [cap] line-search evaluations so far
    double* H;    // [cap][d*d] inverse-Hessian approximation
    int cap;
    void* hslots; // H slots of the streaming kernel
    long long hstride = 0;  // elements per H entry (0: d*d of the run's problem)
    int* ready = nullptr;   // [cap] 1 once entry i is written (fused kernel); zeroed per call
    int long_cap = 0;       // fused kernel: entries [cap - long_cap, cap) take the starts
                            // whose last line search failed (likely long runs)
    int* sm_long = nullptr; // [kMaxSMs] long entries in service per SM (fused kernel)
};

constexpr int kNarrowThreads = 128;
constexpr int kWideThreads = 128;

// Kernel-side configuration of a BFGS launch.
struct BfgsLaunch {
    bool narrow;          // run the narrow (one lane per start) kernel first
    int stride;           // doubles of shared memory per start in the narrow kernel
    int narrow_threads;   // its block size
    size_t narrow_smem;   // its dynamic shared memory
    int narrow_blocks;
    int W;                // line-search trials evaluated at once by the wide kernel
    size_t wide_smem;     // its dynamic shared memory
    int wide_blocks;      // persistent grid of the wide kernel
    int budget;           // narrow-kernel work budget (iterations + evaluations), 0 = none
    int q_cap;            // hand-over queue capacity
    bool stream;          // large d: H streamed from an HBM slot per block
    int stream_blocks;    // blocks (= H slots) of the streaming kernel
    size_t stream_smem;   // its dynamic shared memory
    size_t hslot_bytes;   // bytes of all H slots
    bool lbfgs;           // L-BFGS: the streaming kernel's limited-memory variant (no H)
    bool warp = false;    // one warp per start (threads_per_start 32), four per block
    size_t warp_slot = 0; // dynamic shared memory of one warp's start
};

// Device tables of a batch (zeus_batch_*): per-problem parameters and
// offsets into the concatenated outputs, the PSO block table and the BFGS
// work list.  All pointers address the workspace.
struct BatchDev {
    const zeus_problem* probs;
    const long long* xoff;   // first coordinate of problem P in x_out
    const long long* soff;   // first start of problem P in f_out / status / iters
    const long long* goff;   // its global best position in gx
    const long long* poff;   // its PSO partials
    const int* pblk0;        // its first PSO block
    const int* pblk;         // its number of PSO blocks
    const int* plane;        // PSO lanes per particle
    const int* pso_table;    // problem of each PSO block
    const int4* items;       // BFGS work: (problem, first start, count or W, kind: 0 lane
                             // tile, 1 block, 2 warp, 3 L-BFGS block per start)
    const int* stride;       // one-lane layout stride per problem
    const int* budget;       // hand-over budget per problem (0 = none)
    Ctrl* pctrl;             // [n] per-problem counters, stop flag, global best
    Ctrl* gctrl;             // [1] hand-over queue counters
    unsigned* heads;         // [ZEUS_BATCH_MAX_CLASSES] next work item of each class launch
    ArgPair* partials;
    double* v;
    double* px;
    double* pf;
    double* gx;
    Queue q;
    int n, n_items, pso_blocks;
};

// ---- launchers (defined in the kernel translation units) ----
// lanes per particle of the PSO and objective kernels: one lane (sums in
// index order) up to d = 32, a warp above (lane l forms chain l of the
// objective's sums, the warp adds the chains in the fixed tree)
inline int lanes_for_dim(int d) { return d <= 32 ? 1 : 32; }

cudaError_t launch_pso(const zeus_problem& p, int G, double* x, double* v, double* px, double* pf,
                       double* gx, Ctrl* ctrl, ArgPair* partials, zeus_result* res,
                       cudaStream_t st);
int pso_blocks(const zeus_problem& p, int G);

int plan_bfgs(const zeus_problem& p, BfgsLaunch* L);
cudaError_t launch_bfgs(const zeus_problem& p, const BfgsLaunch& L, const double* x0,
                        double* x_out, double* f_out, double* gnorm_out, int32_t* status_out,
                        int32_t* iters_out, Ctrl* ctrl, const Queue& q, cudaStream_t st);

size_t stream_smem(int d, size_t tsize);
size_t lbfgs_smem(int d, int m, size_t tsize);
int stream_blocks(const zeus_problem& p, size_t smem);
cudaError_t launch_bfgs_stream(const zeus_problem& p, const double* x0, double* x_out,
                               double* f_out, double* gnorm_out, int32_t* status_out,
                               int32_t* iters_out, Ctrl* ctrl, void* hslots, cudaStream_t st);

cudaError_t launch_batch_pso(const BatchDev& bd, int t, double* x_out, cudaStream_t st);
cudaError_t launch_batch_argmin(const BatchDev& bd, const double* f_out, zeus_result* res,
                                cudaStream_t st);
// one persistent launch over work items [first, first + count) with class
// counter `cls`; cls < 0: the hand-over queue
// user: the batch holds user objectives (the kernel variant that has them)
cudaError_t launch_batch_bfgs(const BatchDev& bd, int precision, int grad_mode, bool user, int cls,
                              int first, int count, size_t smem, bool warp_items, double* x_out,
                              double* f_out, double* gnorm_out, int32_t* status_out,
                              int32_t* iters_out, cudaStream_t st);
// one persistent launch over the L-BFGS items [first, first + count) of
// class `cls` (zeus_stream.cu: the body of the single-problem L-BFGS kernel)
cudaError_t launch_batch_lbfgs(const BatchDev& bd, int precision, int grad_mode, int cls,
                               int first, int count, size_t smem, double* x_out, double* f_out,
                               double* gnorm_out, int32_t* status_out, int32_t* iters_out,
                               cudaStream_t st);

// the kernels of one (gradient mode, precision) pair, compiled in a
// translation unit of their own (zeus_bfgs_kernels.cu, zeus_batch_kernels.cu)
template <int GRAD, class T>
cudaError_t bfgs_launch_gt(const zeus_problem& p, const BfgsLaunch& L, const double* x0,
                           double* x_out, double* f_out, double* gnorm_out, int32_t* status_out,
                           int32_t* iters_out, Ctrl* ctrl, const Queue& q, cudaStream_t st);
template <int GRAD, class T, bool U>
cudaError_t batch_launch_gt(const BatchDev& bd, int cls, int first, int count, size_t smem,
                            bool warp_items, double* x_out, double* f_out, double* gnorm_out,
                            int32_t* status_out, int32_t* iters_out, cudaStream_t st);

cudaError_t launch_argmin(const double* f, long long n, Ctrl* ctrl, ArgPair* partials,
                          zeus_result* res, int mode, cudaStream_t st);
int argmin_blocks(long long n);

cudaError_t launch_objective(int obj, int d, long long n, const double* x, double* f, double* g,
                             int grad_mode, cudaStream_t st);
cudaError_t launch_objective_f32(int obj, int d, long long n, const float* x, float* f, float* g,
                                 int grad_mode, cudaStream_t st);

cudaError_t launch_cluster(const zeus_cluster_params& cp, int n, int d, const double* x,
                           const double* f, const int32_t* status, int32_t* label,
                           int32_t* leader_out, int32_t* count_out, zeus_cluster_result* res,
                           void* workspace, cudaStream_t st);
size_t cluster_work_bytes(int max_clusters);
cudaError_t launch_batch_cluster(const zeus_cluster_params& cp, const BatchDev& bd,
                                 const double* x, const double* f, const int32_t* status,
                                 int32_t* label, int32_t* leader_out, int32_t* count_out,
                                 zeus_cluster_result* res, cudaStream_t st);

// plug-in metadata of user objective k (zeus_user.cuh): 0 if k is not one
int user_objective_meta(int k, const char** name, int* min_dim, int* max_dim);
int user_objective_count();

cudaError_t launch_math(int fn, long long n, const double* x, double* y0, double* y1,
                        cudaStream_t st);

cudaError_t launch_uniform(uint64_t seed, uint64_t problem, uint64_t phase, long long n, int d,
                           double* out, cudaStream_t st);

}  // namespace zeus
