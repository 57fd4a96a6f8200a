// filter_noalloc.cu -- pgm_filter_noalloc: the final filter with its scratch
// in a fixed device array owned by the library, for callers that cannot
// allocate device memory (see include/pgm.h).
#include <mutex>

#include "pgm_device.cuh"

namespace pgm {
namespace {

constexpr size_t kMaxSeeds = PGM_NOALLOC_MAX_SEEDS;
constexpr size_t kBsumInts = kMaxSeeds / 256 + 1;
// label[kMaxSeeds] | size[kMaxSeeds] | bsum[kBsumInts]
constexpr size_t kScratchBytes = (2 * kMaxSeeds + kBsumInts) * sizeof(int);

// One copy per device, placed by the CUDA runtime when the library's module
// is loaded there; it lives until the process exits.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {};   // device address of g_scratch, per device

// The symbol's name is only a host-side handle: its device address has to be
// asked for with the device current.  It is asked for again on every call
// made outside a stream capture (the array moves if the device was reset);
// during a capture the address cached by an earlier call is used.
pgm_status scratch_address(cudaStream_t st, void** out) {
    int dev = -1;
    PGM_TRY(cudaGetDevice(&dev), "noalloc: cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) return cuda_fail("noalloc: device index", cudaErrorInvalidDevice);
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    PGM_TRY(cudaStreamIsCapturing(st, &cap), "noalloc: capture status");
    std::lock_guard<std::mutex> lock(g_mu);
    if (cap == cudaStreamCaptureStatusNone || !g_addr[dev]) {
        void* ptr = nullptr;
        PGM_TRY(cudaGetSymbolAddress(&ptr, g_scratch), "noalloc: scratch address");
        if (!ptr) return cuda_fail("noalloc: scratch address", cudaErrorInvalidSymbol);
        g_addr[dev] = ptr;
    }
    *out = g_addr[dev];
    return PGM_OK;
}

}  // namespace
}  // namespace pgm

using namespace pgm;

extern "C" pgm_status pgm_filter_noalloc(const pgm_params* p, int nx, int ny, const int32_t* d_u,
                                         const uint8_t* d_flags, int32_t* d_matches,
                                         int64_t max_matches, int32_t* d_count, void* stream) {
    pgm_status r = check_params(p);
    if (r != PGM_OK) return r;
    if (nx < 0 || ny < 0 || !d_count || max_matches < 0 || (max_matches > 0 && !d_matches))
        return PGM_ERR_ARG;
    if ((long long)nx * ny > 0 && (!d_u || !d_flags)) return PGM_ERR_ARG;
    if ((((uintptr_t)d_matches) & 15u) || (((uintptr_t)d_u) & 3u) || (((uintptr_t)d_count) & 3u))
        return PGM_ERR_ARG;
    if ((long long)nx * ny > (long long)kMaxSeeds) return PGM_ERR_UNSUPPORTED;
    void* base = nullptr;
    r = scratch_address(static_cast<cudaStream_t>(stream), &base);
    if (r != PGM_OK) return r;
    int* label = static_cast<int*>(base);
    int* size = label + kMaxSeeds;
    int* bsum = size + kMaxSeeds;
    return launch_filter_ptrs(p, nx, ny, d_u, d_flags, label, size, bsum, d_matches, max_matches,
                              d_count, static_cast<cudaStream_t>(stream));
}
