// hea_noalloc.cu -- hea_search_coop_noalloc: the cooperative search for callers that cannot
// allocate device memory.
//
// Some callers of this library have no way to obtain device memory of their own: a host program
// whose device memory is entirely owned by another runtime's allocator, a plugin loaded into a
// process that forbids it from calling cudaMalloc, or a deployment with a fixed device-memory
// budget that must not grow after start-up.  hea_search_coop needs a caller-provided exchange
// area; this entry point instead uses a fixed array that lives in the library's own device image
// (every GPU that loads the library holds it until the process exits).  It allocates nothing.
//
// Properties a caller must know:
//   * The array holds HEA_NOALLOC_SCRATCH_BYTES bytes, enough for up to 512 cooperating CTAs;
//     larger requests are rejected with HEA_EINVAL before anything is launched.
//   * There is one array per device, shared by every call on that device.  It keeps the last
//     call's contents; each call clears the part that must start at zero (the barrier header)
//     on its stream before launching.  Calls whose work overlaps on the GPU (other streams, or
//     other host threads) race on the array and corrupt each other's results: serialise them.
//   * The first call on a device, with that device current, looks up the array's device address
//     (cudaGetSymbolAddress) and caches it; make that first call before any stream capture.
#include <mutex>

#include <cuda_runtime.h>

#include "hea_internal.h"

namespace {

constexpr size_t kScratchBytes = HEA_NOALLOC_SCRATCH_BYTES;
constexpr int kMaxDevices = 64;

// The exchange area.  In host code `g_scratch` names a host-side stand-in, not device memory,
// so host code must pass the address obtained from cudaGetSymbolAddress, never the name.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

std::mutex g_lock;
void* g_address[kMaxDevices] = {};

}  // namespace

extern "C" hea_status hea_search_coop_noalloc(const hea_lattice* lat, const hea_objective* obj,
                                              const hea_search_params* params, int ctas, uint8_t* types,
                                              int32_t* counts, hea_search_result* result, void* stream) {
    if (ctas < 1) return hea::set_last_error(HEA_EINVAL, "ctas must be >= 1");
    if (hea_search_coop_workspace_bytes(ctas) > kScratchBytes)
        return hea::set_last_error(HEA_EINVAL,
                                   "ctas exceeds the fixed exchange area of hea_search_coop_noalloc (at most 512 CTAs)");
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        (void)cudaGetLastError();
        return hea::set_last_error(HEA_ECUDA, "no current CUDA device");
    }
    if (dev < 0 || dev >= kMaxDevices) return hea::set_last_error(HEA_ECUDA, "device index beyond 63");
    void* ptr = nullptr;
    {
        std::lock_guard<std::mutex> guard(g_lock);
        if (g_address[dev] == nullptr) {
            void* p = nullptr;
            const cudaError_t err = cudaGetSymbolAddress(&p, g_scratch);
            if (err != cudaSuccess || p == nullptr) {
                (void)cudaGetLastError();
                return hea::set_last_error(HEA_ECUDA, "cudaGetSymbolAddress of the exchange area failed");
            }
            g_address[dev] = p;
        }
        ptr = g_address[dev];
    }
    return hea_search_coop(lat, obj, params, ctas, types, counts, result, ptr, kScratchBytes, stream);
}
