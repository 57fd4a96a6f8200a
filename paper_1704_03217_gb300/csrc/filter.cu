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

// All kernels take a batch of fields: blockIdx.y (blockIdx.x for the scan)
// selects the pair; blocks past a pair's seed count return.
__global__ void k_cc_init(const __grid_constant__ FiltBatch F) {
    const FiltItem& it = F.it[blockIdx.y];
    const int n = it.nx * it.ny;
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    it.label[s] = inlier(it.flags[s]) ? s : -1;
    it.size[s] = 0;
}

__global__ void k_cc_link(const __grid_constant__ FiltBatch F) {
    const FiltItem& it = F.it[blockIdx.y];
    const int nx = it.nx, ny = it.ny;
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nx * ny || !inlier(it.flags[s])) return;
    const int i = s % nx, j = s / nx;
    const int32_t us = it.u[s];
    if (i + 1 < nx && inlier(it.flags[s + 1])) {
        const int32_t ut = it.u[s + 1];
        const long long dx = lo16(us) - lo16(ut), dy = hi16(us) - hi16(ut);
        if (dx * dx + dy * dy < F.dmax2) unite(it.label, s, s + 1);
    }
    if (j + 1 < ny && inlier(it.flags[s + nx])) {
        const int32_t ut = it.u[s + nx];
        const long long dx = lo16(us) - lo16(ut), dy = hi16(us) - hi16(ut);
        if (dx * dx + dy * dy < F.dmax2) unite(it.label, s, s + nx);
    }
}

__global__ void k_cc_flatten(const __grid_constant__ FiltBatch F) {
    const FiltItem& it = F.it[blockIdx.y];
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= it.nx * it.ny || it.label[s] < 0) return;
    // read-only find: a halving store by another thread could otherwise
    // overwrite the root just written to label[s] with a non-root ancestor
    const int r = find_root(it.label, s);
    it.label[s] = r;
    atomicAdd(&it.size[r], 1);
}

// pass 1: survivors per block of 256 seeds
__global__ void k_keep_count(const __grid_constant__ FiltBatch F) {
    const FiltItem& it = F.it[blockIdx.y];
    const int n = it.nx * it.ny;
    if ((int)blockIdx.x * (int)blockDim.x >= n) return;          // whole block
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    int keep = 0;
    if (s < n) {
        const int r = it.label[s];
        keep = r >= 0 && it.size[r] >= F.min_region;
        if (it.keep) it.keep[s] = (uint8_t)keep;
    }
    const int c = __syncthreads_count(keep);
    if (threadIdx.x == 0) it.bsum[blockIdx.x] = c;
}

// pass 2: exclusive scan of the block counts, one block per pair
__global__ void k_scan_blocks(const __grid_constant__ FiltBatch F) {
    const FiltItem& it = F.it[blockIdx.x];
    const int nb = (it.nx * it.ny + 255) / 256;
    __shared__ int part[1024];
    __shared__ int carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < nb; base += 1024) {
        const int idx = base + threadIdx.x;
        const int v = idx < nb ? it.bsum[idx] : 0;
        part[threadIdx.x] = v;
        __syncthreads();
        for (int off = 1; off < 1024; off <<= 1) {      // Hillis-Steele inclusive scan
            const int t = threadIdx.x >= off ? part[threadIdx.x - off] : 0;
            __syncthreads();
            part[threadIdx.x] += t;
            __syncthreads();
        }
        if (idx < nb) it.bsum[idx] = carry + part[threadIdx.x] - v;
        __syncthreads();
        if (threadIdx.x == 0) carry += part[1023];
        __syncthreads();
    }
    if (threadIdx.x == 0) *it.count = carry;
}

// pass 3: write survivors in raster order
__global__ void k_keep_write(const __grid_constant__ FiltBatch F) {
    const FiltItem& it = F.it[blockIdx.y];
    const int n = it.nx * it.ny;
    if ((int)blockIdx.x * (int)blockDim.x >= n) return;          // whole block
    __shared__ int warp_tot[8];
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    int keep = 0;
    if (s < n) {
        const int r = it.label[s];
        keep = r >= 0 && it.size[r] >= F.min_region;
    }
    const unsigned m = __ballot_sync(0xffffffffu, keep);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) warp_tot[w] = __popc(m);
    __syncthreads();
    int off = it.bsum[blockIdx.x];
    for (int k = 0; k < w; ++k) off += warp_tot[k];
    off += __popc(m & ((1u << lane) - 1u));
    if (keep && off < it.max_rows) {
        const int i = s % it.nx, j = s / it.nx;
        const int x = F.c + F.sigma * i, y = F.c + F.sigma * j;
        const int32_t uu = it.u[s];
        reinterpret_cast<int4*>(it.rows)[off] = make_int4(x, y, x + lo16(uu), y + hi16(uu));
    }
}

}  // namespace

// The whole filter for a batch of fields: six launches in all.
pgm_status launch_filter_batch(const pgm_params* p, const FiltBatch& F, int max_seeds,
                               cudaStream_t st) {
    if (F.n == 0) return PGM_OK;
    KScope ks(PGM_K_FILTER, st, 6);
    const int nb = (max_seeds + 255) / 256;
    const dim3 g(nb > 0 ? nb : 1, F.n);
    k_cc_init<<<g, 256, 0, st>>>(F);
    k_cc_link<<<g, 256, 0, st>>>(F);
    k_cc_flatten<<<g, 256, 0, st>>>(F);
    k_keep_count<<<g, 256, 0, st>>>(F);
    k_scan_blocks<<<F.n, 1024, 0, st>>>(F);
    k_keep_write<<<g, 256, 0, st>>>(F);
    (void)p;
    return launch_status("filter: launch");
}

void filter_item(const WsPlan& wp, uint8_t* d_ws, int32_t* d_matches, int64_t max_matches,
                 int32_t* d_count, uint8_t* d_keep, FiltItem* it) {
    it->flags = d_ws + wp.off_flags[0][0];
    it->u = reinterpret_cast<const int32_t*>(d_ws + wp.off_u[0][0]);
    it->label = reinterpret_cast<int*>(d_ws + wp.off_label);
    it->size = reinterpret_cast<int*>(d_ws + wp.off_size);
    it->bsum = reinterpret_cast<int*>(d_ws + wp.off_bsum);
    it->nx = wp.nx[0][0];
    it->ny = wp.ny[0][0];
    it->rows = d_matches;
    it->max_rows = max_matches;
    it->count = d_count;
    it->keep = d_keep;
}

void filter_consts(const pgm_params* p, FiltBatch* F) {
    F->sigma = p->seed_stride;
    F->c = p->seed_stride / 2;
    F->dmax2 = p->region_dmax2;
    F->min_region = p->min_region;
}

pgm_status launch_filter(const pgm_params* p, const WsPlan& wp, uint8_t* d_ws,
                         int32_t* d_matches, int64_t max_matches, int32_t* d_count,
                         uint8_t* d_keep, cudaStream_t st) {
    static thread_local FiltBatch F;
    F.n = 1;
    filter_consts(p, &F);
    filter_item(wp, d_ws, d_matches, max_matches, d_count, d_keep, &F.it[0]);
    return launch_filter_batch(p, F, F.it[0].nx * F.it[0].ny, st);
}

// The same sequence on explicit pointers: the field (u, flags) and the
// scratch (label, size: nx*ny ints each; bsum: one int per 256 seeds + 1)
// may live anywhere in device memory.
pgm_status launch_filter_ptrs(const pgm_params* p, int nx, int ny, const int32_t* u,
                              const uint8_t* flags, int* label, int* size, int* bsum,
                              int32_t* d_matches, int64_t max_matches, int32_t* d_count,
                              cudaStream_t st) {
    static thread_local FiltBatch F;
    F.n = 1;
    filter_consts(p, &F);
    FiltItem& it = F.it[0];
    it.flags = flags; it.u = u; it.label = label; it.size = size; it.bsum = bsum;
    it.nx = nx; it.ny = ny; it.rows = d_matches; it.max_rows = max_matches;
    it.count = d_count; it.keep = nullptr;
    return launch_filter_batch(p, F, nx * ny, st);
}

}  // namespace pgm
