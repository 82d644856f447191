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
// device (the first call on a device does this set-up).
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
    // carve the static scratch: control block | argmin partials | queue
    const size_t d = (size_t)p->dim;
    const size_t off_parts = align256(sizeof(Ctrl));
    const size_t off_queue = off_parts + align256((size_t)argmin_blocks(p->n_starts) * sizeof(ArgPair));
    if (L.budget > 0) {
        // every start must fit the hand-over queue: 3 ints and H per start
        const size_t per = 3 * sizeof(int) + d * d * sizeof(double);
        const size_t room = kScratchBytes - off_queue - 4 * 256;
        if ((size_t)p->n_starts > room / per) return ZEUS_EWORKSPACE;
        L.q_cap = (int)p->n_starts;
    } else {
        L.q_cap = 0;
    }
    void* base = nullptr;
    v = scratch_address(&base);
    if (v != ZEUS_OK) return v;
    char* b = static_cast<char*>(base);
    const size_t qc = (size_t)L.q_cap;
    Queue q;
    q.prob = nullptr;
    q.start = reinterpret_cast<int*>(b + off_queue);
    q.k = reinterpret_cast<int*>(b + off_queue + align256(qc * sizeof(int)));
    q.feval = reinterpret_cast<int*>(b + off_queue + 2 * align256(qc * sizeof(int)));
    q.H = reinterpret_cast<double*>(b + off_queue + 3 * align256(qc * sizeof(int)));
    q.cap = L.q_cap;
    q.hslots = nullptr;
    if (L.stream && L.hslot_bytes > 0) return ZEUS_EWORKSPACE;  // H slots do not fit the array
    Ctrl* ctrl = reinterpret_cast<Ctrl*>(b);
    ArgPair* parts = reinterpret_cast<ArgPair*>(b + off_parts);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    // the control block must start at zero; the rest is written before it is read
    if (cudaMemsetAsync(ctrl, 0, sizeof(Ctrl), st) != cudaSuccess) return ZEUS_ECUDA;
    if (launch_bfgs(*p, L, x0, x_out, f_out, gnorm_out, status_out, iters_out, ctrl, q, st) !=
        cudaSuccess)
        return ZEUS_ECUDA;
    if (launch_argmin(f_out, p->n_starts, ctrl, parts, result, 2, st) != cudaSuccess)
        return ZEUS_ECUDA;
    return ZEUS_OK;
}
