// filter.cu -- small-region removal (Sec. III-E) and grid export
// (Sec. III-G) on the level-0 forward field.
//
// Regions are the connected components of inlier seeds under lattice
// 4-adjacency, two neighbours joining iff |u_s - u_t|^2 < region_dmax2.  They
// are found with a lock-free union-find whose links always point to the
// smaller index, so after path compression every seed carries the smallest
// index of its component whatever the thread order.  Components are then
// sized with atomics; survivors (size >= min_region) are compacted in lattice
// raster order by a three-pass scan.
#include "pgm_device.cuh"

namespace pgm {
namespace {

__device__ __forceinline__ int lo16(uint32_t v) { return (int)(int16_t)(v & 0xffffu); }
__device__ __forceinline__ int hi16(uint32_t v) { return ((int)v) >> 16; }

__device__ __forceinline__ bool inlier(uint8_t f) { return (f & F_VALID) && !(f & F_OUTL); }

__device__ __forceinline__ int find_root(const int* L, int a) {
    int p = L[a];
    while (p != a) { a = p; p = L[a]; }
    return a;
}

// find with path halving: each visited node is re-pointed to its
// grandparent.  Labels only ever decrease towards a root of the same
// component, so the plain stores are safe under concurrent unions.
__device__ __forceinline__ int find_halve(int* L, int a) {
    int p = L[a];
    while (p != a) {
        const int g = L[p];
        if (g != p) L[a] = g;
        a = p;
        p = g;
    }
    return a;
}

__global__ void k_cc_init(const uint8_t* __restrict__ flags, int n, int* __restrict__ label,
                          int* __restrict__ size) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    label[s] = inlier(flags[s]) ? s : -1;
    size[s] = 0;
}

__device__ void unite(int* L, int a, int b) {
    // link the larger root below the smaller one; retry if another thread
    // re-linked the root in between
    for (;;) {
        a = find_halve(L, a);
        b = find_halve(L, b);
        if (a == b) return;
        if (a < b) { int t = a; a = b; b = t; }      // a > b: link a -> b
        int old = atomicMin(&L[a], b);
        if (old == a) return;
        a = old;
    }
}

__global__ void k_cc_link(const uint8_t* __restrict__ flags, const int32_t* __restrict__ u,
                          int nx, int ny, int dmax2, int* label) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nx * ny || !inlier(flags[s])) return;
    int i = s % nx, j = s / nx;
    int32_t us = u[s];
    if (i + 1 < nx && inlier(flags[s + 1])) {
        int32_t ut = u[s + 1];
        long long dx = lo16(us) - lo16(ut), dy = hi16(us) - hi16(ut);
        if (dx * dx + dy * dy < dmax2) unite(label, s, s + 1);
    }
    if (j + 1 < ny && inlier(flags[s + nx])) {
        int32_t ut = u[s + nx];
        long long dx = lo16(us) - lo16(ut), dy = hi16(us) - hi16(ut);
        if (dx * dx + dy * dy < dmax2) unite(label, s, s + nx);
    }
}

__global__ void k_cc_flatten(int n, int* label, int* size) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n || label[s] < 0) return;
    // read-only find: a halving store by another thread could otherwise
    // overwrite the root just written to label[s] with a non-root ancestor
    int r = find_root(label, s);
    label[s] = r;
    atomicAdd(&size[r], 1);
}

// pass 1: survivors per block of 256 seeds
__global__ void k_keep_count(int n, const int* __restrict__ label, const int* __restrict__ size,
                             int min_region, int* __restrict__ bsum, uint8_t* keep_out) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    int keep = 0;
    if (s < n) {
        int r = label[s];
        keep = r >= 0 && size[r] >= min_region;
        if (keep_out) keep_out[s] = (uint8_t)keep;
    }
    int c = __syncthreads_count(keep);
    if (threadIdx.x == 0) bsum[blockIdx.x] = c;
}

// pass 2: exclusive scan of the block counts (one block, any count)
__global__ void k_scan_blocks(int nb, int* bsum, int32_t* d_count) {
    __shared__ int part[1024];
    __shared__ int carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < nb; base += 1024) {
        int idx = base + threadIdx.x;
        int v = idx < nb ? bsum[idx] : 0;
        part[threadIdx.x] = v;
        __syncthreads();
        for (int off = 1; off < 1024; off <<= 1) {      // Hillis-Steele inclusive scan
            int t = threadIdx.x >= off ? part[threadIdx.x - off] : 0;
            __syncthreads();
            part[threadIdx.x] += t;
            __syncthreads();
        }
        if (idx < nb) bsum[idx] = carry + part[threadIdx.x] - v;
        __syncthreads();
        if (threadIdx.x == 0) carry += part[1023];
        __syncthreads();
    }
    if (threadIdx.x == 0) *d_count = carry;
}

// pass 3: write survivors in raster order
__global__ void k_keep_write(int n, int nx, int sigma, int c, const int* __restrict__ label,
                             const int* __restrict__ size, int min_region,
                             const int32_t* __restrict__ u, const int* __restrict__ bsum,
                             int32_t* __restrict__ rows, long long max_rows) {
    __shared__ int warp_tot[8];
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    int keep = 0;
    if (s < n) {
        int r = label[s];
        keep = r >= 0 && size[r] >= min_region;
    }
    unsigned m = __ballot_sync(0xffffffffu, keep);
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) warp_tot[w] = __popc(m);
    __syncthreads();
    int off = bsum[blockIdx.x];
    for (int k = 0; k < w; ++k) off += warp_tot[k];
    off += __popc(m & ((1u << lane) - 1u));
    if (keep && off < max_rows) {
        int i = s % nx, j = s / nx;
        int x = c + sigma * i, y = c + sigma * j;
        int32_t uu = u[s];
        int4 row = make_int4(x, y, x + lo16(uu), y + hi16(uu));
        reinterpret_cast<int4*>(rows)[off] = row;
    }
}

}  // namespace

pgm_status launch_filter(const pgm_params* p, const WsPlan& wp, uint8_t* d_ws,
                         int32_t* d_matches, int64_t max_matches, int32_t* d_count,
                         uint8_t* d_keep, cudaStream_t st) {
    const int nx = wp.nx[0][0], ny = wp.ny[0][0], n = nx * ny;
    const uint8_t* flags = d_ws + wp.off_flags[0][0];
    const int32_t* u = reinterpret_cast<const int32_t*>(d_ws + wp.off_u[0][0]);
    int* label = reinterpret_cast<int*>(d_ws + wp.off_label);
    int* size = reinterpret_cast<int*>(d_ws + wp.off_size);
    int* bsum = reinterpret_cast<int*>(d_ws + wp.off_bsum);
    const int nb = (n + 255) / 256;
    if (n == 0) {
        cudaMemsetAsync(d_count, 0, sizeof(int32_t), st);
        return cudaGetLastError() == cudaSuccess ? PGM_OK : PGM_ERR_CUDA;
    }
    KScope ks(PGM_K_FILTER, st, 6);
    k_cc_init<<<nb, 256, 0, st>>>(flags, n, label, size);
    k_cc_link<<<nb, 256, 0, st>>>(flags, u, nx, ny, p->region_dmax2, label);
    k_cc_flatten<<<nb, 256, 0, st>>>(n, label, size);
    k_keep_count<<<nb, 256, 0, st>>>(n, label, size, p->min_region, bsum, d_keep);
    k_scan_blocks<<<1, 1024, 0, st>>>(nb, bsum, d_count);
    k_keep_write<<<nb, 256, 0, st>>>(n, nx, p->seed_stride, p->seed_stride / 2, label, size,
                                     p->min_region, u, bsum, d_matches, max_matches);
    return cudaGetLastError() == cudaSuccess ? PGM_OK : PGM_ERR_CUDA;
}

// The same sequence on explicit pointers: the field (u, flags) and the
// scratch (label, size: nx*ny ints each; bsum: one int per 256 seeds + 1)
// may live anywhere in device memory.
pgm_status launch_filter_ptrs(const pgm_params* p, int nx, int ny, const int32_t* u,
                              const uint8_t* flags, int* label, int* size, int* bsum,
                              int32_t* d_matches, int64_t max_matches, int32_t* d_count,
                              cudaStream_t st) {
    const int n = nx * ny;
    const int nb = (n + 255) / 256;
    if (n == 0) {
        cudaMemsetAsync(d_count, 0, sizeof(int32_t), st);
        return cudaGetLastError() == cudaSuccess ? PGM_OK : PGM_ERR_CUDA;
    }
    KScope ks(PGM_K_FILTER, st, 6);
    k_cc_init<<<nb, 256, 0, st>>>(flags, n, label, size);
    k_cc_link<<<nb, 256, 0, st>>>(flags, u, nx, ny, p->region_dmax2, label);
    k_cc_flatten<<<nb, 256, 0, st>>>(n, label, size);
    k_keep_count<<<nb, 256, 0, st>>>(n, label, size, p->min_region, bsum, nullptr);
    k_scan_blocks<<<1, 1024, 0, st>>>(nb, bsum, d_count);
    k_keep_write<<<nb, 256, 0, st>>>(n, nx, p->seed_stride, p->seed_stride / 2, label, size,
                                     p->min_region, u, bsum, d_matches, max_matches);
    return cudaGetLastError() == cudaSuccess ? PGM_OK : PGM_ERR_CUDA;
}

}  // namespace pgm
