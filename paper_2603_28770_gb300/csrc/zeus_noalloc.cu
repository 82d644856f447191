// zeus_noalloc.cu -- zeus_solve_from_noalloc: BFGS from given starts plus
// the best-of-swarm reduction, for callers that cannot allocate device
// memory.  Its scratch (control block, reduction partials, hand-over queue)
// is one file-scope __device__ array that every GPU loading the library
// holds until the process exits.
#include <mutex>

#include "zeus.h"
#include "zeus_internal.h"

using namespace zeus;

namespace {

constexpr size_t kScratchBytes = ZEUS_NOALLOC_SCRATCH_BYTES;
constexpr int kMaxDevices = 64;

// In host code this name is a host-side stand-in, not a device address:
// kernels get the address from cudaGetSymbolAddress below.
__device__ __align__(256) unsigned char g_scratch[kScratchBytes];

std::mutex g_mu;
void* g_ptr[kMaxDevices];

// Device address of g_scratch on the current device, looked up once per
// device (the first call on a device does this set-up) and kept for the
// life of the process: after cudaDeviceReset, or anything else that
// destroys the device's primary context, the kept address is stale.
int scratch_address(void** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return ZEUS_ECUDA;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_ptr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return ZEUS_ECUDA;
        }
        g_ptr[dev] = p;
    }
    *out = g_ptr[dev];
    return ZEUS_OK;
}

}  // namespace

extern "C" int zeus_solve_from_noalloc(const zeus_problem* p, const double* x0, double* x_out,
                                       double* f_out, double* gnorm_out, int32_t* status_out,
                                       int32_t* iters_out, zeus_result* result, void* stream) {
    int v = zeus_validate(p);
    if (v != ZEUS_OK) return v;
    if (!x0 || !x_out || !f_out) return ZEUS_EINVAL;
    BfgsLaunch L;
    v = plan_bfgs(*p, &L);
    if (v != ZEUS_OK) return v;
    if (L.stream && L.hslot_bytes > 0) return ZEUS_EWORKSPACE;  // H slots do not fit the array
    // carve the static scratch as the workspace of zeus_solve_from is
    // carved: control block | ready flags | per-SM table | argmin partials |
    // hand-over queue (start, k, evaluations, H)
    const size_t d = (size_t)p->dim;
    const size_t parts_bytes = align256((size_t)argmin_blocks(p->n_starts) * sizeof(ArgPair));
    const size_t smlong_bytes = align256(kMaxSMs * sizeof(int));
    size_t qc = 0;
    if (L.budget > 0) {
        // the planner's queue, clamped to what the array holds; a start that
        // finds the queue full runs on in its lane, so a shorter queue only
        // changes which kernel finishes a start, not its result
        const size_t per = 4 * sizeof(int) + d * d * sizeof(double);
        const size_t fixed = align256(sizeof(Ctrl)) + smlong_bytes + parts_bytes + 5 * 256;
        const size_t fit = kScratchBytes > fixed ? (kScratchBytes - fixed) / per : 0;
        if (fit < 1) return ZEUS_EWORKSPACE;
        qc = (size_t)L.q_cap < fit ? (size_t)L.q_cap : fit;
        L.q_cap = (int)qc;
    } else {
        L.q_cap = 0;
    }
    const size_t off_ready = align256(sizeof(Ctrl));
    const size_t off_smlong = off_ready + align256(qc * sizeof(int));
    const size_t off_parts = off_smlong + smlong_bytes;
    const size_t off_queue = off_parts + parts_bytes;
    const size_t off_k = off_queue + align256(qc * sizeof(int));
    const size_t off_feval = off_k + align256(qc * sizeof(int));
    const size_t off_h = off_feval + align256(qc * sizeof(int));
    if (off_h + qc * d * d * sizeof(double) > kScratchBytes) return ZEUS_EWORKSPACE;
    void* base = nullptr;
    v = scratch_address(&base);
    if (v != ZEUS_OK) return v;
    char* b = static_cast<char*>(base);
    Queue q;
    q.prob = nullptr;
    q.start = reinterpret_cast<int*>(b + off_queue);
    q.k = reinterpret_cast<int*>(b + off_k);
    q.feval = reinterpret_cast<int*>(b + off_feval);
    q.H = reinterpret_cast<double*>(b + off_h);
    q.cap = L.q_cap;
    q.hslots = nullptr;
    q.ready = reinterpret_cast<int*>(b + off_ready);
    q.sm_long = reinterpret_cast<int*>(b + off_smlong);
    Ctrl* ctrl = reinterpret_cast<Ctrl*>(b);
    ArgPair* parts = reinterpret_cast<ArgPair*>(b + off_parts);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    // the control block, the ready flags and the per-SM table must start at
    // zero; the rest is written before it is read
    if (cudaMemsetAsync(ctrl, 0, off_parts, st) != cudaSuccess) return ZEUS_ECUDA;
    if (launch_bfgs(*p, L, x0, x_out, f_out, gnorm_out, status_out, iters_out, ctrl, q, st) !=
        cudaSuccess)
        return ZEUS_ECUDA;
    if (launch_argmin(f_out, p->n_starts, ctrl, parts, result, 2, st) != cudaSuccess)
        return ZEUS_ECUDA;
    return ZEUS_OK;
}
