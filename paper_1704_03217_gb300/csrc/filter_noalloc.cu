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
// asked for, once per device, with that device current.
pgm_status scratch_address(void** out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return PGM_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
        void* ptr = nullptr;
        if (cudaGetSymbolAddress(&ptr, g_scratch) != cudaSuccess || !ptr) return PGM_ERR_CUDA;
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
    if (((uintptr_t)d_matches) & 15u) return PGM_ERR_ARG;
    if ((long long)nx * ny > (long long)kMaxSeeds) return PGM_ERR_UNSUPPORTED;
    void* base = nullptr;
    r = scratch_address(&base);
    if (r != PGM_OK) return r;
    int* label = static_cast<int*>(base);
    int* size = label + kMaxSeeds;
    int* bsum = size + kMaxSeeds;
    return launch_filter_ptrs(p, nx, ny, d_u, d_flags, label, size, bsum, d_matches, max_matches,
                              d_count, static_cast<cudaStream_t>(stream));
}
