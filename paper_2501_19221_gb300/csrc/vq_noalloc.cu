// vq_noalloc.cu -- an energy entry point that never allocates device memory.
//
// veloxq_energy_dev needs scratch for its per-group partial sums and grows a
// buffer owned by the context when a batch is larger than any before, which
// can call cudaMalloc. Some callers cannot allow that: code running inside a
// custom or pooling allocator (an allocation callback, an out-of-memory
// handler) that must not re-enter the driver's allocator; processes that
// reserve their whole device-memory budget up front and refuse any later
// allocation; and latency-critical loops that cannot absorb the implicit
// device synchronisation cudaMalloc may cause. veloxq_energy_dev_noalloc
// computes the same energies with the same kernels, but its scratch is the
// file-scope array below, which the module loader places in device memory.
#include <cudaTypedefs.h>

#include <mutex>

#include "vq_internal.cuh"

namespace {

// Partial sums of the energy kernels: 2^19 int64 (4 MiB). Every GPU that loads
// the library holds this array until the process exits.
constexpr int64_t kNoAllocParts = (int64_t)1 << 19;
static __device__ __align__(256) int64_t g_noalloc_parts[kNoAllocParts];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
// Device address of g_noalloc_parts per device, with the ID of the CUDA
// context it was looked up in: a device reset creates a new context (with a
// new ID) in which the array may sit elsewhere, and the address is looked up
// again there.
struct ScratchSlot {
    unsigned long long ctx_id = 0;
    int64_t* addr = nullptr;
};
ScratchSlot g_slot[kMaxDevices];

// ID of the CUDA context current on this thread (false when none is current
// or the driver does not provide the calls).
bool current_context_id(unsigned long long* id) {
    static PFN_cuCtxGetCurrent_v4000 get_current = nullptr;
    static PFN_cuCtxGetId_v12000 get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        cudaDriverEntryPointQueryResult q;
        void* p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 4000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<PFN_cuCtxGetCurrent_v4000>(p);
        p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<PFN_cuCtxGetId_v12000>(p);
        cudaGetLastError();
    });
    CUcontext c = nullptr;
    if (!get_current || !get_id || get_current(&c) != CUDA_SUCCESS || !c) return false;
    return get_id(c, id) == CUDA_SUCCESS;
}

// Device address of the scratch array on the current device. Host code cannot
// use the array's name as a device address (it names a host-side stand-in), so
// the address is looked up with cudaGetSymbolAddress: once per device and
// context, with that device current; the first call on a device does this
// set-up, which may load the module's device code.
int scratch_on_current_device(int dev, int64_t** out) {
    if (dev < 0 || dev >= kMaxDevices) return vq::fail(VELOXQ_EUNSUPPORTED, "device index out of range");
    std::lock_guard<std::mutex> lock(g_mu);
    unsigned long long id = 0;
    const bool known = current_context_id(&id);
    ScratchSlot& sl = g_slot[dev];
    if (!sl.addr || !known || sl.ctx_id != id) {
        void* p = nullptr;
        VQ_CUDA(cudaGetSymbolAddress(&p, g_noalloc_parts));
        sl.addr = static_cast<int64_t*>(p);
        // the lookup made the device's context current if none was
        sl.ctx_id = current_context_id(&id) ? id : 0;
    }
    *out = sl.addr;
    return VELOXQ_OK;
}

}  // namespace

extern "C" int veloxq_energy_dev_noalloc(veloxq_ctx* ctx, int64_t batch, const uint8_t* X, double* E,
                                         int64_t* E_int) {
    using namespace vq;
    if (!ctx) return fail(VELOXQ_EINVAL, "ctx must not be NULL");
    if (batch < 0) return fail(VELOXQ_EINVAL, "batch must be >= 0");
    if (batch > 0 && !X) return fail(VELOXQ_EINVAL, "X must not be NULL");
    if (E_int && !ctx->integer) return fail(VELOXQ_EINVAL, "E_int requires an integer-valued context");
    int dev = -1;
    VQ_CUDA(cudaGetDevice(&dev));
    if (dev != ctx->device) return fail(VELOXQ_EINVAL, "the context's device must be the current device");
    const int64_t groups = ctx->dense ? div_up(ctx->n, 64) : 64;   // partial sums per vector
    if (batch > 65535 || batch * groups > kNoAllocParts)
        return fail(VELOXQ_EINVAL, "batch too large for the fixed scratch of veloxq_energy_dev_noalloc: need batch <= " +
                                       std::to_string(std::min<int64_t>(65535, kNoAllocParts / groups)) +
                                       " for this context");
    if (batch == 0) return VELOXQ_OK;
    int64_t* parts = nullptr;
    VQ_TRY(scratch_on_current_device(dev, &parts));
    int np = 0;
    // every partial sum is written before it is read: nothing in the scratch needs clearing
    if (ctx->dense) VQ_TRY(dense_energy_x(ctx, batch, X, parts, &np, false));
    else VQ_TRY(sparse_energy_x(ctx, batch, X, parts, &np));
    return launch_sum_parts(ctx, batch, np, parts, E, E_int);
}
