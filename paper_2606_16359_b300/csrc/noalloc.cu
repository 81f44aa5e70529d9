// Rescale that allocates no device memory.
//
// fe_rescale obtains its scratch (the inverse-transformed last limb and its
// lift to the other limbs) from the stream-ordered allocator.  Some callers
// cannot allow that: a serving process that must keep a fixed device-memory
// footprint after start-up, a host framework that owns all device memory
// through its own pool and forbids other libraries from calling cudaMalloc, or
// latency-critical code that cannot afford an allocation (cudaMalloc may
// synchronise the device).  fe_rescale_noalloc serves them: its scratch is one
// file-scope device array of a fixed size, kNoAllocScratchBytes.
//
// Host code cannot use the array's name as a device address (on the host it is
// only a stand-in symbol); the device address is looked up once per device with
// cudaGetSymbolAddress, on the first call for a context of that device (which
// must be the current device).  Under lazy module loading (the CUDA default) the
// array is only reserved on a device when this file's module first loads there,
// which is that first call.
#include <mutex>

#include "ops.h"

namespace fe {
namespace {

constexpr size_t kNoAllocScratchBytes = 32ull << 20;  // 32 MiB per device, from the module's first load there
constexpr size_t kNoAllocScratchWords = kNoAllocScratchBytes / sizeof(u64);
constexpr int kMaxDevices = 64;

static __device__ __align__(256) u64 g_noalloc_scratch[kNoAllocScratchWords];

std::mutex g_scratch_mu;
u64* g_scratch_addr[kMaxDevices] = {};

// device address of g_noalloc_scratch on the context's device (looked up once per
// device).  The context's tables, the caller's buffers and the stream belong to the
// device the context was created on, so that device must be the current one: the
// symbol's address is per device, and another device's array must never reach
// these kernels.
int scratch_address(const fe_ctx* c, u64** out) {
    int dev = 0;
    FE_CUDA_TRY(cudaGetDevice(&dev));
    if (dev != c->device)
        return fail(FE_EINVAL, "fe_rescale_noalloc: the current device (" + std::to_string(dev) +
                                   ") is not the context's device (" + std::to_string(c->device) + ")");
    if (dev < 0 || dev >= kMaxDevices) return fail(FE_EINVAL, "device index above the supported maximum");
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return fail(FE_ECUDA, std::string("cudaGetSymbolAddress of the static scratch: ") + cudaGetErrorString(e));
        g_scratch_addr[dev] = (u64*)p;
    }
    *out = g_scratch_addr[dev];
    return FE_OK;
}

}  // namespace
}  // namespace fe

using namespace fe;

extern "C" int fe_rescale_noalloc(fe_ctx* c, const void* ct_dev, uint32_t n_ct, uint32_t level, void* out_dev,
                                  void* stream) {
    if (!c || !ct_dev || !out_dev) return fail(FE_EINVAL, "null argument");
    FE_ALIGNED(ct_dev);
    FE_ALIGNED(out_dev);
    if (level == 0) return fail(FE_ELEVEL, "rescale at level 0");
    if ((int)level > c->L) return fail(FE_ELEVEL, "level above L");
    if (n_ct == 0) return FE_OK;
    const size_t need = rescale_tmp_words(c, n_ct, level) * sizeof(u64);
    if (need > kNoAllocScratchBytes)
        return fail(FE_ENOMEM, "fe_rescale_noalloc: " + std::to_string(n_ct) + " ciphertexts at level " +
                                   std::to_string(level) + " need " + std::to_string(need) +
                                   " bytes of scratch, above the fixed " + std::to_string(kNoAllocScratchBytes) +
                                   "-byte static buffer; split the batch or use fe_rescale");
    u64* scratch = nullptr;
    FE_TRY(scratch_address(c, &scratch));
    // profiling would create CUDA events; keep this path free of allocations
    const int saved_kind = c->prof.kind;
    c->prof.kind = -1;
    rescale_batch(c, (const u64*)ct_dev, (int)n_ct, (int)level, (u64*)out_dev, scratch,
                  scratch + 2 * (size_t)n_ct * c->N, (cudaStream_t)stream);
    c->prof.kind = saved_kind;
    FE_CUDA_TRY(cudaGetLastError());
    return FE_OK;
}
