// vq_noalloc.cu -- an energy entry point that never allocates device memory.
//
// veloxq_energy_dev needs scratch for its per-group partial sums and grows a
// buffer owned by the context when a batch is larger than any before, which
// can call cudaMalloc. Some callers cannot allow that: code that runs while a
// CUDA graph is being captured (allocation is not a capturable operation),
// code inside a custom or pooled allocator that must not re-enter the driver's
// allocator, and latency-critical loops that forbid the implicit device
// synchronisation cudaMalloc may cause. veloxq_energy_dev_noalloc computes the
// same energies with the same kernels, but its scratch is the file-scope
// array below, which the module loader places in device memory once.
#include <mutex>

#include "vq_internal.cuh"

namespace {

// Partial sums of the energy kernels: 2^19 int64 (4 MiB). Every GPU that loads
// the library holds this array until the process exits.
constexpr int64_t kNoAllocParts = (int64_t)1 << 19;
static __device__ __align__(256) int64_t g_noalloc_parts[kNoAllocParts];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
int64_t* g_parts_addr[kMaxDevices] = {};   // device address of g_noalloc_parts, per device

// Device address of the scratch array on the current device (looked up once
// per device; the host-side symbol is a stand-in, not a device address).
int scratch_on_current_device(int64_t** out) {
    int dev = 0;
    VQ_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return vq::fail(VELOXQ_EUNSUPPORTED, "device index out of range");
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_parts_addr[dev]) {
        void* p = nullptr;
        VQ_CUDA(cudaGetSymbolAddress(&p, g_noalloc_parts));
        g_parts_addr[dev] = static_cast<int64_t*>(p);
    }
    *out = g_parts_addr[dev];
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
    VQ_TRY(scratch_on_current_device(&parts));
    int np = 0;
    // every partial sum is written before it is read: nothing in the scratch needs clearing
    if (ctx->dense) VQ_TRY(dense_energy_x(ctx, batch, X, parts, &np, false));
    else VQ_TRY(sparse_energy_x(ctx, batch, X, parts, &np));
    return launch_sum_parts(ctx, batch, np, parts, E, E_int);
}
