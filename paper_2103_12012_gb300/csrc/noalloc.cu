// sssp_solve_noalloc: the partitioned asynchronous solve for callers that
// cannot allocate device memory.
//
// Some callers are handed only their input and output buffers and have no way
// to obtain scratch memory: for example a plugin or user-defined function
// inside a host application (a graph database, an inference server) that owns
// every device allocation through its own pool and gives extensions no
// allocator.  This entry point gives them the solve with its scratch in a
// fixed array that this library reserves on every GPU that loads it, for the
// life of the process.  The call is asynchronous like sssp_solve; the
// device-side status is copied into the caller's `status_out` word.
//
// Rules of use:
//  - The first call on a device looks up the array's device address with
//    cudaGetSymbolAddress (with that device current) and caches it together
//    with the id of the device's current CUDA context; make that first call
//    before any stream capture.  A later call that finds another context
//    current on the device (after cudaDeviceReset, for instance, which
//    destroys the context and with it the array's old address) looks the
//    address up again, so that call too belongs outside a capture.
//  - Problems whose scratch would exceed SSSP_NOALLOC_SCRATCH_BYTES are
//    rejected with SSSP_ENOMEM; nothing is launched.
//  - Every call uses the same array, and the array keeps the previous call's
//    contents; the solve resets every part it reads before use.  Calls that
//    overlap on the GPU (on different streams, or from different host threads
//    without ordering) race on the array and give wrong results.
//  - No cudaMalloc, cudaFree or allocating library routine is called.
#include <mutex>

#include <cuda.h>  // driver types only: the functions are reached through the runtime

#include "common.cuh"
#include "internal.h"

namespace {

// The scratch of every no-allocation call on this device.  In host code this
// name is only a stand-in for the symbol, never a device address: the address
// comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[SSSP_NOALLOC_SCRATCH_BYTES];

constexpr int MAX_DEVICES = 64;
std::mutex g_setup_mutex;
void* g_scratch_ptr[MAX_DEVICES] = {};
unsigned long long g_scratch_ctx[MAX_DEVICES] = {};  // id of the context the address belongs to

// Driver functions reached through the runtime (no link against libcuda): the current
// context and its process-unique id.
typedef CUresult (*ctx_get_current_fn)(CUcontext* ctx);
typedef CUresult (*ctx_get_id_fn)(CUcontext ctx, unsigned long long* id);
ctx_get_current_fn g_ctx_get_current = nullptr;
ctx_get_id_fn g_ctx_get_id = nullptr;

// Id of the context current on this thread, 0 if none is current (or ids are unavailable).
unsigned long long current_ctx_id() {
    if (!g_ctx_get_current) {
        void* f1 = nullptr;
        void* f2 = nullptr;
        cudaDriverEntryPointQueryResult q1 = cudaDriverEntryPointSymbolNotFound, q2 = q1;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) != cudaSuccess ||
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) != cudaSuccess ||
            q1 != cudaDriverEntryPointSuccess || q2 != cudaDriverEntryPointSuccess || !f1 || !f2)
            return 0;
        g_ctx_get_id = reinterpret_cast<ctx_get_id_fn>(f2);
        g_ctx_get_current = reinterpret_cast<ctx_get_current_fn>(f1);
    }
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (g_ctx_get_current(&ctx) != CUDA_SUCCESS || !ctx || g_ctx_get_id(ctx, &id) != CUDA_SUCCESS) return 0;
    return id;
}

// With the device current: the array's address in the device's current context, looked up
// on the first call and again whenever the context has changed since.
sssp_status scratch_for_current_device(void** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return SSSP_ECUDA;
    if (dev < 0 || dev >= MAX_DEVICES) return SSSP_EUNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    const unsigned long long id = current_ctx_id();
    if (!g_scratch_ptr[dev] || id == 0 || id != g_scratch_ctx[dev]) {
        void* p = nullptr;
        // (also makes the device's primary context current if no context was)
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return SSSP_ECUDA;
        g_scratch_ptr[dev] = p;
        g_scratch_ctx[dev] = current_ctx_id();
    }
    *out = g_scratch_ptr[dev];
    return SSSP_OK;
}

}  // namespace

extern "C" sssp_status sssp_solve_noalloc(const sssp_graph* g, const uint32_t* sources, uint32_t S, void* dist,
                                          uint32_t* pred, const sssp_options* opt, uint32_t* status_out,
                                          sssp_stream_t stream) {
    if (!g || S == 0 || !sources || !dist) return SSSP_EINVAL;
    const size_t need = sssp_solve_workspace_size(g, S, opt);
    if (need == 0) return SSSP_EINVAL;
    if (need > SSSP_NOALLOC_SCRATCH_BYTES) return SSSP_ENOMEM;
    void* scratch = nullptr;
    const sssp_status st = scratch_for_current_device(&scratch);
    if (st != SSSP_OK) return st;
    // sssp_solve clears the header and initialises every packed word, inbox word and
    // doorbell it will read before its relaxation kernel starts.
    const sssp_status ls = sssp_solve(g, sources, S, dist, pred, opt, scratch, SSSP_NOALLOC_SCRATCH_BYTES, stream);
    if (ls != SSSP_OK || !status_out) return ls;
    // the status word is the first field of the scratch header
    if (cudaMemcpyAsync(status_out, scratch, sizeof(uint32_t), cudaMemcpyDeviceToDevice, (cudaStream_t)stream) !=
        cudaSuccess)
        return SSSP_ECUDA;
    return SSSP_OK;
}
