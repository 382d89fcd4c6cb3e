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
//   * The array holds HEA_NOALLOC_SCRATCH_BYTES bytes, enough for up to HEA_NOALLOC_MAX_CTAS (512)
//     cooperating CTAs; larger requests are rejected with HEA_EINVAL before anything is launched.
//   * There is one array per device, shared by every call on that device.  It keeps the last
//     call's contents; each call clears the part that must start at zero (the header and the tag
//     words) on its stream before launching.  Calls whose work overlaps on the GPU (other streams,
//     or other host threads) race on the array and corrupt each other's results: serialise them.
//   * The first call on a device, with that device current, looks up the array's device address
//     (cudaGetSymbolAddress) and caches it with the identity of the current CUDA context; make that
//     first call before any stream capture.  A call made in another context (after a device reset,
//     say) looks the address up again.
#include <cstdint>
#include <mutex>

#include <cuda_runtime.h>

#include "hea_internal.h"

namespace {

constexpr size_t kScratchBytes = HEA_NOALLOC_SCRATCH_BYTES;
constexpr int kMaxDevices = 64;

// The exchange area.  In host code `g_scratch` names a host-side stand-in, not device memory,
// so host code must pass the address obtained from cudaGetSymbolAddress, never the name.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

struct Cached {
    unsigned long long context;   // identity of the context the address belongs to (0 = none)
    void* address;
};

std::mutex g_lock;
Cached g_cache[kMaxDevices] = {};

// Identity of the calling thread's current CUDA context (its driver id + 1), or 0 when none is
// current or the driver entry points are unavailable.  Driver calls are reached through the
// runtime's entry-point query, so the library does not link the driver library directly.
using CtxGetCurrent = int (*)(void**);
using CtxGetId = int (*)(void*, unsigned long long*);

unsigned long long current_context() {
    static CtxGetCurrent get_current = nullptr;
    static CtxGetId get_id = nullptr;
    static bool looked_up = false;
    if (!looked_up) {
        looked_up = true;
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<CtxGetCurrent>(f);
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<CtxGetId>(f);
        (void)cudaGetLastError();
    }
    void* ctx = nullptr;
    if (!get_current || get_current(&ctx) != 0 || !ctx) return 0ull;
    unsigned long long id = 0ull;
    if (!get_id || get_id(ctx, &id) != 0) return 0ull;
    return id + 1ull;
}

}  // namespace

extern "C" hea_status hea_search_coop_noalloc(const hea_lattice* lat, const hea_objective* obj,
                                              const hea_search_params* params, int ctas, uint8_t* types,
                                              int32_t* counts, hea_search_result* result, void* stream) {
    if (ctas < 1) return hea::set_last_error(HEA_EINVAL, "ctas must be >= 1");
    if (ctas > HEA_NOALLOC_MAX_CTAS || hea_search_coop_workspace_bytes(ctas) > kScratchBytes)
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
        const unsigned long long ctx = current_context();
        if (ctx == 0ull || g_cache[dev].context != ctx || g_cache[dev].address == nullptr) {
            void* p = nullptr;
            const cudaError_t err = cudaGetSymbolAddress(&p, g_scratch);
            if (err != cudaSuccess || p == nullptr) {
                (void)cudaGetLastError();
                return hea::set_last_error(HEA_ECUDA, "cudaGetSymbolAddress of the exchange area failed");
            }
            g_cache[dev].address = p;
            g_cache[dev].context = current_context();   // the lookup made the device's context current
        }
        ptr = g_cache[dev].address;
    }
    return hea_search_coop(lat, obj, params, ctas, types, counts, result, ptr, kScratchBytes, stream);
}
