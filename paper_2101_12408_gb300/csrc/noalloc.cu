// Closest-particle search without any allocation (mpm_nearest_parent_noalloc).
//
// For callers that cannot allocate device memory: allocators that forbid
// cudaMalloc after start-up, or host programs that hand the library a fixed
// memory budget, and so cannot create a context. It computes what mpm_resample
// computes for the balance particles' parents -- for every surface sample the
// closest interior particle (smallest squared distance formed as
// (dx^2 + dy^2) + dz^2 in float64, ties to the smaller particle index), searched
// over the 27 cells around the sample and, when none of those holds a particle
// within dx, over the 125 cells around it (every particle within 2 dx) -- but it
// needs no context. Its working memory (cell counts, cell starts, particles
// sorted by cell, scan partials, an error word) is one file-scope device array of
// fixed size, so every GPU that loads the library holds those bytes until the
// process exits.
#include <mutex>

#include "ctx.h"

namespace {

constexpr long long NA_MAX_PARTICLES = 1LL << 19;   // 524 288 interior particles
constexpr long long NA_MAX_CELLS = 1LL << 20;       // 1 048 576 grid cells
constexpr int NA_TILE = 4096;                       // scan tile (1024 threads x 4)
constexpr long long NA_MAX_TILES = (NA_MAX_CELLS + 1 + NA_TILE - 1) / NA_TILE;
// layout in ints: counts (cells + 1) | starts (cells + 1) | sorted ids (particles) |
// ranks (particles) | scan partials (tiles) | error word
constexpr long long NA_OFF_COUNT = 0;
constexpr long long NA_OFF_START = NA_OFF_COUNT + NA_MAX_CELLS + 1;
constexpr long long NA_OFF_SORTED = NA_OFF_START + NA_MAX_CELLS + 1;
constexpr long long NA_OFF_RANK = NA_OFF_SORTED + NA_MAX_PARTICLES;
constexpr long long NA_OFF_PART = NA_OFF_RANK + NA_MAX_PARTICLES;
constexpr long long NA_OFF_ERR = NA_OFF_PART + NA_MAX_TILES;
constexpr long long NA_INTS = NA_OFF_ERR + 64;

// The scratch. Host code must not take its address directly: the name is a host
// stand-in for the symbol; the device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) int g_noalloc_scratch[NA_INTS];

constexpr int NA_MAX_DEVICES = 64;
std::mutex g_setup_mutex;
int* g_scratch_ptr[NA_MAX_DEVICES] = {};

enum : int { NA_ERR_DOMAIN = 1, NA_ERR_FAR = 2 };

struct Grid {
    int n[3];
    double inv_dx, dx, origin[3];
};

__device__ __forceinline__ bool na_cell(const Grid& g, double x, double y, double z, int c[3]) {
    double p[3] = {x, y, z};
    bool ok = true;
    for (int a = 0; a < 3; ++a) {
        double fl = floor((p[a] - g.origin[a]) * g.inv_dx);
        int ci = (fl >= -1e9 && fl <= 1e9) ? (int)fl : -1;
        if (!(ci >= 1 && ci <= g.n[a] - 2)) {
            ok = false;
            ci = ci < 1 ? 1 : g.n[a] - 2;
        }
        c[a] = ci;
    }
    return ok;
}

__device__ __forceinline__ long long na_key(const Grid& g, int cx, int cy, int cz) {
    return cx + (long long)g.n[0] * (cy + (long long)g.n[1] * cz);
}

__global__ void na_count(Grid g, int n, const double* __restrict__ x, int* __restrict__ scratch) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int c[3];
    if (!na_cell(g, x[3 * i], x[3 * i + 1], x[3 * i + 2], c)) atomicOr(scratch + NA_OFF_ERR, NA_ERR_DOMAIN);
    long long k = na_key(g, c[0], c[1], c[2]);
    scratch[NA_OFF_RANK + i] = atomicAdd(scratch + NA_OFF_COUNT + k, 1);
}

__device__ __forceinline__ int na_block_scan(int v, int* sh, int& total) {
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int incl = v;
    for (int o = 1; o < 32; o <<= 1) {
        int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) sh[w] = incl;
    __syncthreads();
    if (w == 0) {
        int t = sh[lane], ti = t;
        for (int o = 1; o < 32; o <<= 1) {
            int u = __shfl_up_sync(0xffffffffu, ti, o);
            if (lane >= o) ti += u;
        }
        sh[lane] = ti - t;
        if (lane == 31) sh[32] = ti;
    }
    __syncthreads();
    int res = incl - v + sh[w];
    total = sh[32];
    __syncthreads();
    return res;
}

// exclusive scan of counts[0..ncell) into starts[0..ncell], three passes
__global__ void na_scan_tiles(long long ncell, int* __restrict__ scratch) {
    __shared__ int sh[33];
    long long base = (long long)blockIdx.x * NA_TILE + threadIdx.x * 4;
    int s = 0;
    for (int k = 0; k < 4; ++k) s += (base + k < ncell) ? scratch[NA_OFF_COUNT + base + k] : 0;
    int total;
    na_block_scan(s, sh, total);
    if (threadIdx.x == 0) scratch[NA_OFF_PART + blockIdx.x] = total;
}

__global__ void na_scan_partials(int ntiles, int* __restrict__ scratch) {
    __shared__ int sh[33];
    int running = 0;
    for (int base = 0; base < ntiles; base += 1024) {
        int i = base + threadIdx.x;
        int v = i < ntiles ? scratch[NA_OFF_PART + i] : 0;
        int total;
        int ex = na_block_scan(v, sh, total);
        if (i < ntiles) scratch[NA_OFF_PART + i] = running + ex;
        running += total;
    }
}

__global__ void na_scan_final(long long ncell, int* __restrict__ scratch) {
    __shared__ int sh[33];
    long long base = (long long)blockIdx.x * NA_TILE + threadIdx.x * 4;
    int vals[4], s = 0;
    for (int k = 0; k < 4; ++k) {
        vals[k] = (base + k < ncell) ? scratch[NA_OFF_COUNT + base + k] : 0;
        s += vals[k];
    }
    int total;
    int ex = na_block_scan(s, sh, total) + scratch[NA_OFF_PART + blockIdx.x];
    for (int k = 0; k < 4; ++k) {
        if (base + k <= ncell) scratch[NA_OFF_START + base + k] = ex;
        ex += vals[k];
    }
}

__global__ void na_place(Grid g, int n, const double* __restrict__ x, int* __restrict__ scratch) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int c[3];
    na_cell(g, x[3 * i], x[3 * i + 1], x[3 * i + 2], c);
    long long k = na_key(g, c[0], c[1], c[2]);
    scratch[NA_OFF_SORTED + scratch[NA_OFF_START + k] + scratch[NA_OFF_RANK + i]] = i;
}

__global__ void na_search(Grid g, int ns, const double* __restrict__ s, const double* __restrict__ x,
                          const int* __restrict__ scratch, int* __restrict__ err, int32_t* __restrict__ parent) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= ns) return;
    double q[3] = {s[3 * j], s[3 * j + 1], s[3 * j + 2]};
    int c[3];
    na_cell(g, q[0], q[1], q[2], c);
    double best = 1e300;
    int bid = 0x7fffffff;
    // the 27 cells around the sample hold every particle within dx; when the
    // nearest is farther (samples generated on the union-of-spheres surface reach
    // ~1.1 dx), the shell of the 125 cells around it holds the rest within 2 dx
    for (int reach = 1; reach <= 2; ++reach) {
        if (reach == 2 && best <= g.dx * g.dx) break;
        for (int dz = -reach; dz <= reach; ++dz)
            for (int dy = -reach; dy <= reach; ++dy)
                for (int dxx = -reach; dxx <= reach; ++dxx) {
                    if (reach == 2 && dz > -2 && dz < 2 && dy > -2 && dy < 2 && dxx > -2 && dxx < 2) continue;
                    const int cx = c[0] + dxx, cy = c[1] + dy, cz = c[2] + dz;
                    if (cx < 0 || cy < 0 || cz < 0 || cx >= g.n[0] || cy >= g.n[1] || cz >= g.n[2]) continue;
                    long long k = na_key(g, cx, cy, cz);
                    int e = scratch[NA_OFF_START + k + 1];
                    for (int t = scratch[NA_OFF_START + k]; t < e; ++t) {
                        int i = scratch[NA_OFF_SORTED + t];
                        double d0 = __dsub_rn(q[0], x[3 * i]);
                        double d1 = __dsub_rn(q[1], x[3 * i + 1]);
                        double d2 = __dsub_rn(q[2], x[3 * i + 2]);
                        double dist = __dadd_rn(__dadd_rn(__dmul_rn(d0, d0), __dmul_rn(d1, d1)), __dmul_rn(d2, d2));
                        if (dist < best || (dist == best && i < bid)) {
                            best = dist;
                            bid = i;
                        }
                    }
                }
    }
    if (bid == 0x7fffffff || best > 4.0 * g.dx * g.dx) {
        atomicOr(err, NA_ERR_FAR);
        parent[j] = -1;
        return;
    }
    parent[j] = bid;
}

// One-time set-up per device, with that device current: the device address of
// the scratch array, kept for the life of the process (a device reset that
// invalidates it is not detected). Returns null on failure.
int* scratch_for_current_device() {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NA_MAX_DEVICES) return nullptr;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[dev]) {
        int* ptr = nullptr;
        if (cudaGetSymbolAddress((void**)&ptr, g_noalloc_scratch) != cudaSuccess) return nullptr;
        g_scratch_ptr[dev] = ptr;
    }
    return g_scratch_ptr[dev];
}

inline unsigned na_blocks(long long n, int nt) { return (unsigned)((n + nt - 1) / nt); }

}  // namespace

extern "C" mpm_status mpm_nearest_parent_noalloc(const mpm_grid_desc* grid, int64_t n_particles, const double* x,
                                                 int64_t n_samples, const double* s, int32_t* parent, void* stream) {
    if (!grid || n_particles < 0 || n_samples < 0) return MPM_ERR_INVALID_ARG;
    if ((n_particles > 0 && !x) || (n_samples > 0 && (!s || !parent))) return MPM_ERR_INVALID_ARG;
    if (grid->n[0] < 4 || grid->n[1] < 4 || grid->n[2] < 4 || !(grid->dx > 0)) return MPM_ERR_INVALID_ARG;
    long long ncell = (long long)grid->n[0] * grid->n[1] * grid->n[2];
    if (ncell > NA_MAX_CELLS || n_particles > NA_MAX_PARTICLES) return MPM_ERR_CAPACITY;
    if (n_samples > 0x7fffffffLL) return MPM_ERR_CAPACITY;
    int* scratch = scratch_for_current_device();
    if (!scratch) return MPM_ERR_CUDA;
    cudaStream_t st = (cudaStream_t)stream;
    Grid g;
    for (int a = 0; a < 3; ++a) {
        g.n[a] = grid->n[a];
        g.origin[a] = grid->origin[a];
    }
    g.dx = grid->dx;
    g.inv_dx = 1.0 / grid->dx;
    int n = (int)n_particles;
    // the counts and the error word must start at zero; everything else is overwritten
    if (cudaMemsetAsync(scratch + NA_OFF_COUNT, 0, sizeof(int) * (size_t)(ncell + 1), st) != cudaSuccess ||
        cudaMemsetAsync(scratch + NA_OFF_ERR, 0, sizeof(int), st) != cudaSuccess)
        return MPM_ERR_CUDA;
    if (n > 0) na_count<<<na_blocks(n, 256), 256, 0, st>>>(g, n, x, scratch);
    long long tiles = (ncell + 1 + NA_TILE - 1) / NA_TILE;
    na_scan_tiles<<<(unsigned)tiles, 1024, 0, st>>>(ncell, scratch);
    na_scan_partials<<<1, 1024, 0, st>>>((int)tiles, scratch);
    na_scan_final<<<(unsigned)tiles, 1024, 0, st>>>(ncell, scratch);
    if (n > 0) na_place<<<na_blocks(n, 256), 256, 0, st>>>(g, n, x, scratch);
    if (n_samples > 0) na_search<<<na_blocks(n_samples, 128), 128, 0, st>>>(g, (int)n_samples, s, x, scratch,
                                                                            scratch + NA_OFF_ERR, parent);
    if (cudaGetLastError() != cudaSuccess) return MPM_ERR_CUDA;
    int err = 0;
    if (cudaMemcpyAsync(&err, scratch + NA_OFF_ERR, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return MPM_ERR_CUDA;
    if (err) return MPM_ERR_DOMAIN;
    return MPM_OK;
}
