// Counting sort of particles and samples by cell, active-block discovery and
// the block neighbour table.
//
// Cells are keyed block-major (global block id * 64 + cell inside the block), so
// after the sort the particles of one 4x4x4 block are one contiguous range and
// every kernel that walks a block reads them with unit stride.
#include "ctx.h"

namespace mpm {

namespace {

constexpr int SCAN_NT = 1024;
constexpr int SCAN_PER = 4;
constexpr int SCAN_TILE = SCAN_NT * SCAN_PER;

__global__ void k_scan_partials(const int* __restrict__ in, long long n, int* __restrict__ part) {
    __shared__ int sh[32];
    long long base = (long long)blockIdx.x * SCAN_TILE + threadIdx.x * SCAN_PER;
    int s = 0;
#pragma unroll
    for (int k = 0; k < SCAN_PER; ++k) s += (base + k < n) ? in[base + k] : 0;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        int t = sh[threadIdx.x];
        for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
        if (threadIdx.x == 0) part[blockIdx.x] = t;
    }
}

__device__ __forceinline__ int block_exclusive_scan(int v, int* sh, int& total) {
    // exclusive scan of one int per thread over SCAN_NT threads
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int incl = v;
    for (int o = 1; o < 32; o <<= 1) {
        int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) sh[w] = incl;
    __syncthreads();
    if (w == 0) {
        int t = sh[lane];
        int ti = t;
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

__global__ void k_scan_top(int* __restrict__ part, int nparts) {
    __shared__ int sh[33];
    int running = 0;
    for (int base = 0; base < nparts; base += SCAN_NT) {
        int i = base + threadIdx.x;
        int v = i < nparts ? part[i] : 0;
        int total;
        int ex = block_exclusive_scan(v, sh, total);
        if (i < nparts) part[i] = running + ex;
        running += total;
    }
}

__global__ void k_scan_final(const int* __restrict__ in, long long n, const int* __restrict__ part, int* __restrict__ out) {
    __shared__ int sh[33];
    long long base = (long long)blockIdx.x * SCAN_TILE + threadIdx.x * SCAN_PER;
    int vals[SCAN_PER];
    int s = 0;
#pragma unroll
    for (int k = 0; k < SCAN_PER; ++k) {
        vals[k] = (base + k < n) ? in[base + k] : 0;
        s += vals[k];
    }
    int total;
    int ex = block_exclusive_scan(s, sh, total) + part[blockIdx.x];
#pragma unroll
    for (int k = 0; k < SCAN_PER; ++k) {
        if (base + k <= n) out[base + k] = ex;   // out has n + 1 entries
        ex += vals[k];
    }
}

__device__ __forceinline__ bool cell_of(const SceneDev& S, const double* p, int c[3]) {
    bool ok = true;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        double u = (p[a] - S.origin[a]) * S.inv_dx;
        double fl = floor(u);
        int ci = (fl >= -1e9 && fl <= 1e9) ? (int)fl : -1;
        if (!(ci >= 1 && ci <= S.n[a] - 2)) {
            ok = false;
            ci = ci < 1 ? 1 : S.n[a] - 2;
        }
        c[a] = ci;
    }
    return ok;
}

__global__ void k_keys(int n, const double* __restrict__ x0, const double* __restrict__ x1, const double* __restrict__ x2,
                       const int* __restrict__ scn, const SceneDev* __restrict__ sc, long long* __restrict__ key,
                       int* __restrict__ rank, int* __restrict__ count, int* err) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (scn[i] < 0) {   // removed by a later set of its scene
        key[i] = -1;
        return;
    }
    const SceneDev& S = sc[scn[i]];
    double p[3] = {x0[i], x1[i], x2[i]};
    int c[3];
    if (!cell_of(S, p, c)) atomicOr(err, ERR_DOMAIN);
    long long k = cell_key(S, c[0], c[1], c[2]);
    key[i] = k;
    rank[i] = atomicAdd(&count[k], 1);
}

__global__ void k_perm(int n, const long long* __restrict__ key, const int* __restrict__ rank,
                       const int* __restrict__ start, int* __restrict__ perm) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || key[i] < 0) return;
    perm[start[key[i]] + rank[i]] = i;
}

template <typename T>
__global__ void k_gather(int n, const int* __restrict__ perm, const T* __restrict__ src, T* __restrict__ dst) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    dst[j] = src[perm[j]];
}

__device__ __forceinline__ void mark_stencil_blocks(const SceneDev& S, const int c[3], int* bflag) {
    int b0[3], b1[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        b0[a] = (c[a] - 1) >> 2;
        b1[a] = (c[a] + 1) >> 2;
    }
    for (int bz = b0[2]; bz <= b1[2]; ++bz)
        for (int by = b0[1]; by <= b1[1]; ++by)
            for (int bx = b0[0]; bx <= b1[0]; ++bx)
                bflag[S.block_base + bx + (long long)S.nb[0] * (by + (long long)S.nb[1] * bz)] = 1;
}

__global__ void k_mark(int n, const double* __restrict__ x0, const double* __restrict__ x1, const double* __restrict__ x2,
                       const int* __restrict__ scn, const int* __restrict__ parent, const SceneDev* __restrict__ sc,
                       int* __restrict__ bflag, int* __restrict__ bwork, int* err) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const SceneDev& S = sc[scn[i]];
    double p[3] = {x0[i], x1[i], x2[i]};
    int c[3];
    if (!cell_of(S, p, c)) atomicOr(err, ERR_DOMAIN);
    mark_stencil_blocks(S, c, bflag);
    if (bwork) bwork[S.block_base + (c[0] >> 2) + (long long)S.nb[0] * ((c[1] >> 2) + (long long)S.nb[1] * (c[2] >> 2))] = 1;
}

__device__ __forceinline__ int scene_of_block(const SceneDev* sc, int nsc, long long gb) {
    int lo = 0, hi = nsc - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (sc[mid].block_base <= gb) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__global__ void k_slots(long long nblk, const int* __restrict__ bflag, const int* __restrict__ bscan,
                        const SceneDev* __restrict__ sc, int nsc, int* __restrict__ bslot, int4* __restrict__ coord,
                        int* __restrict__ counts, long long cap, int* err) {
    long long gb = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (gb >= nblk) return;
    if (gb == nblk - 1) counts[0] = bscan[nblk];
    if (!bflag[gb]) {
        bslot[gb] = -1;
        return;
    }
    int slot = bscan[gb];
    if (slot >= cap) {   // more active blocks than the context was created for
        atomicOr(err, ERR_CAPACITY);
        bslot[gb] = -1;
        return;
    }
    bslot[gb] = slot;
    int s = scene_of_block(sc, nsc, gb);
    long long r = gb - sc[s].block_base;
    int bx = (int)(r % sc[s].nb[0]);
    int by = (int)((r / sc[s].nb[0]) % sc[s].nb[1]);
    int bz = (int)(r / ((long long)sc[s].nb[0] * sc[s].nb[1]));
    coord[slot] = make_int4(bx, by, bz, s);
}

__global__ void k_work(long long nblk, const int* __restrict__ bwork, const int* __restrict__ wscan,
                       const int* __restrict__ bslot, int* __restrict__ work, int* __restrict__ work_gb,
                       int* __restrict__ bw, int* __restrict__ counts, long long cap) {
    long long gb = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (gb >= nblk) return;
    if (gb == nblk - 1) counts[1] = wscan[nblk];
    if (!bwork[gb]) return;
    int w = wscan[gb];
    if (w >= cap) return;
    bw[gb] = w;
    work[w] = bslot[gb];
    work_gb[w] = (int)gb;
}

__global__ void k_nbr(int nb, const int4* __restrict__ coord, const SceneDev* __restrict__ sc,
                      const int* __restrict__ bslot, int* __restrict__ nbr) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nb * 27) return;
    int slot = t / 27, k = t % 27;
    int4 c = coord[slot];
    const SceneDev& S = sc[c.w];
    int bx = c.x + (k % 3) - 1, by = c.y + (k / 3) % 3 - 1, bz = c.z + k / 9 - 1;
    int out = -1;
    if (bx >= 0 && by >= 0 && bz >= 0 && bx < S.nb[0] && by < S.nb[1] && bz < S.nb[2])
        out = bslot[S.block_base + bx + (long long)S.nb[0] * (by + (long long)S.nb[1] * bz)];
    nbr[t] = out;
}

inline int nblocks(long long n, int nt) { return (int)((n + nt - 1) / nt); }

}  // namespace

cudaError_t launch_exclusive_scan(mpm_ctx* c, const int* in, int* out, long long n, int* tmp, cudaStream_t st) {
    // out[0..n] = exclusive scan of in[0..n-1]; out[n] = total
    long long tiles = (n + 1 + SCAN_TILE - 1) / SCAN_TILE;
    MPM_LAUNCH k_scan_partials<<<(unsigned)tiles, SCAN_NT, 0, st>>>(in, n, tmp);
    MPM_LAUNCH k_scan_top<<<1, SCAN_NT, 0, st>>>(tmp, (int)tiles);
    MPM_LAUNCH k_scan_final<<<(unsigned)tiles, SCAN_NT, 0, st>>>(in, n, tmp, out);
    return cudaGetLastError();
}

// Reorder a float64 field by `perm`: gather into the scratch array of the same
// capacity and swap the two (no copy back).
void permute(mpm_ctx* c, int n, const int* perm, double*& a, double*& scratch) {
    MPM_LAUNCH k_gather<double><<<nblocks(n, 256), 256, 0, c->st>>>(n, perm, a, scratch);
    double* old = a;
    a = scratch;
    scratch = old;
}

// Smaller element types keep their own buffer: gather into scratch, copy back.
template <typename T>
void permute(mpm_ctx* c, int n, const int* perm, T* a, double* scratch) {
    MPM_LAUNCH k_gather<T><<<nblocks(n, 256), 256, 0, c->st>>>(n, perm, a, (T*)scratch);
    cudaMemcpyAsync(a, scratch, sizeof(T) * (size_t)n, cudaMemcpyDeviceToDevice, c->st);
}

cudaError_t launch_sort_particles(mpm_ctx* c) {
    Dev& d = c->d;
    cudaStream_t st = c->st;
    int n = (int)c->np;
    cudaMemsetAsync(d.cell_count, 0, sizeof(int) * c->total_cells, st);
    if (n > 0) {
        MPM_LAUNCH k_keys<<<nblocks(n, 256), 256, 0, st>>>(n, d.x[0], d.x[1], d.x[2], d.psc, d.sc, d.key, d.rank, d.cell_count, d.err);
    }
    launch_exclusive_scan(c, d.cell_count, d.cell_start, c->total_cells, d.scan_tmp, st);
    if (n == 0) return cudaGetLastError();
    MPM_LAUNCH k_perm<<<nblocks(n, 256), 256, 0, st>>>(n, d.key, d.rank, d.cell_start, d.perm);
    cudaMemcpyAsync(c->hcounts + 2, d.cell_start + c->total_cells, sizeof(int), cudaMemcpyDeviceToHost, st);
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return e;
    n = c->hcounts[2];   // live particles
    c->np = n;
    if (n == 0) return cudaGetLastError();
    for (int a = 0; a < 3; ++a) {
        permute(c, n, d.perm, d.x[a], d.scratch_p);
        permute(c, n, d.perm, d.v[a], d.scratch_p);
        permute(c, n, d.perm, d.gT[a], d.scratch_p);
    }
    for (int a = 0; a < 9; ++a) {
        permute(c, n, d.perm, d.A[a], d.scratch_p);
        permute(c, n, d.perm, d.F[a], d.scratch_p);
    }
    permute(c, n, d.perm, d.m, d.scratch_p);
    permute(c, n, d.perm, d.V0, d.scratch_p);
    permute(c, n, d.perm, d.J, d.scratch_p);
    permute(c, n, d.perm, d.T, d.scratch_p);
    permute(c, n, d.perm, d.phase, d.scratch_p);
    permute(c, n, d.perm, d.pid, d.scratch_p);
    permute(c, n, d.perm, d.psc, d.scratch_p);
    return cudaGetLastError();
}

cudaError_t launch_sort_surface(mpm_ctx* c) {
    Dev& d = c->d;
    cudaStream_t st = c->st;
    int n = (int)c->ns;
    cudaMemsetAsync(d.scell_count, 0, sizeof(int) * c->total_cells, st);
    if (n > 0) {
        MPM_LAUNCH k_keys<<<nblocks(n, 256), 256, 0, st>>>(n, d.s[0], d.s[1], d.s[2], d.ssc, d.sc, d.skey, d.srank, d.scell_count, d.err);
    }
    launch_exclusive_scan(c, d.scell_count, d.scell_start, c->total_cells, d.scan_tmp, st);
    if (n == 0) return cudaGetLastError();
    MPM_LAUNCH k_perm<<<nblocks(n, 256), 256, 0, st>>>(n, d.skey, d.srank, d.scell_start, d.sperm);
    cudaMemcpyAsync(c->hcounts + 3, d.scell_start + c->total_cells, sizeof(int), cudaMemcpyDeviceToHost, st);
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return e;
    n = c->hcounts[3];   // live samples
    c->ns = n;
    if (n == 0) return cudaGetLastError();
    for (int a = 0; a < 3; ++a) {
        permute(c, n, d.sperm, d.s[a], d.scratch_s);
        permute(c, n, d.sperm, d.dA[a], d.scratch_s);
    }
    permute(c, n, d.sperm, d.bheat, d.scratch_s);
    permute(c, n, d.sperm, d.Tbar, d.scratch_s);
    permute(c, n, d.sperm, d.kind, d.scratch_s);
    permute(c, n, d.sperm, d.sid, d.scratch_s);
    permute(c, n, d.sperm, d.ssc, d.scratch_s);
    return cudaGetLastError();
}

cudaError_t launch_build_blocks(mpm_ctx* c) {
    Dev& d = c->d;
    cudaStream_t st = c->st;
    long long nblk = c->total_blocks;
    cudaMemsetAsync(d.bflag, 0, sizeof(int) * nblk, st);
    cudaMemsetAsync(d.bwork, 0, sizeof(int) * nblk, st);
    if (c->np > 0)
        MPM_LAUNCH k_mark<<<nblocks(c->np, 256), 256, 0, st>>>((int)c->np, d.x[0], d.x[1], d.x[2], d.psc, nullptr, d.sc, d.bflag, d.bwork, d.err);
    if (c->ns > 0) {
        MPM_LAUNCH k_mark<<<nblocks(c->ns, 256), 256, 0, st>>>((int)c->ns, d.s[0], d.s[1], d.s[2], d.ssc, nullptr, d.sc, d.bflag, d.bwork, d.err);
        MPM_LAUNCH k_mark<<<nblocks(c->ns, 256), 256, 0, st>>>((int)c->ns, d.bpos[0], d.bpos[1], d.bpos[2], d.ssc, nullptr, d.sc, d.bflag, nullptr, d.err);
    }
    launch_exclusive_scan(c, d.bflag, d.bscan, nblk, d.scan_tmp, st);
    MPM_LAUNCH k_slots<<<nblocks(nblk, 256), 256, 0, st>>>(nblk, d.bflag, d.bscan, d.sc, c->nsc, d.bslot, d.slot_coord, d.counts, c->block_cap, d.err);
    launch_exclusive_scan(c, d.bwork, d.bscan, nblk, d.scan_tmp, st);
    MPM_LAUNCH k_work<<<nblocks(nblk, 256), 256, 0, st>>>(nblk, d.bwork, d.bscan, d.bslot, d.work, d.work_gb, d.bw, d.counts, c->block_cap);
    cudaMemcpyAsync(c->hcounts, d.counts, 2 * sizeof(int), cudaMemcpyDeviceToHost, st);
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return e;
    c->NB = c->hcounts[0] < c->block_cap ? c->hcounts[0] : (int)c->block_cap;
    c->NW = c->hcounts[1] < c->block_cap ? c->hcounts[1] : (int)c->block_cap;
    if (c->NB > 0) MPM_LAUNCH k_nbr<<<nblocks((long long)c->NB * 27, 256), 256, 0, st>>>(c->NB, d.slot_coord, d.sc, d.bslot, d.nbr);
    return cudaGetLastError();
}

}  // namespace mpm
