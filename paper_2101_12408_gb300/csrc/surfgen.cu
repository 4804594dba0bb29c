// Surface-sample generation on the device: the union-of-spheres level set of the
// interior particles on the grid nodes, its zero isocontour by marching
// tetrahedra, and per-triangle Poisson / Osada sampling with SplitMix64
// counters. Paper section "Surface Particle Sampling"; the readings (node
// lattice, clamp at 1.5 dx, tetrahedral cut, enumeration order, counters, sample
// weight 1 / density) are stated with mpm_generate_surface in include/mpm.h.
//
// Every product and sum of the geometry is written with explicit round-to-
// nearest intrinsics (no fused multiply-add), so the samples are the float64
// values a plain sequential evaluation of the same formulas gives.
#include <cmath>

#include "ctx.h"
#include "mcubes.cuh"

namespace mpm {

namespace {

constexpr double R0_FACTOR = 0.867;
constexpr double CLAMP_FACTOR = 1.5;
constexpr int KMAX = 31;
constexpr unsigned long long GOLDEN = 0x9E3779B97F4A7C15ull;

__device__ __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double sub(double a, double b) { return __dsub_rn(a, b); }

// (k+1)-th output of SplitMix64 started from `seed`
__device__ __forceinline__ unsigned long long splitmix64(unsigned long long seed, unsigned long long k) {
    unsigned long long z = seed + (k + 1ull) * GOLDEN;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ double uniform01(unsigned long long seed, unsigned long long k) {
    return (double)(splitmix64(seed, k) >> 11) * (1.0 / 9007199254740992.0);
}

// phi = min(distance to the nearest particle, 1.5 dx) - 0.867 dx on every node of
// the active blocks (any particle closer than 1.5 dx lies in the 27 cells around)
__global__ void k_phi(int nb, const int4* __restrict__ coord, const SceneDev* __restrict__ sc,
                      const int* __restrict__ cell_start, const double* __restrict__ x0, const double* __restrict__ x1,
                      const double* __restrict__ x2, double* __restrict__ phi) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)nb * 64) return;
    const int slot = (int)(t >> 6), l = (int)(t & 63);
    const int4 bc = coord[slot];
    const SceneDev& S = sc[bc.w];
    const int g[3] = {bc.x * BS + (l & 3), bc.y * BS + ((l >> 2) & 3), bc.z * BS + (l >> 4)};
    double pos[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) pos[a] = add(S.origin[a], mul((double)g[a] + 0.5, S.dx));
    double best = 1e300;
    for (int dz = -1; dz <= 1; ++dz)
        for (int dy = -1; dy <= 1; ++dy)
            for (int dxx = -1; dxx <= 1; ++dxx) {
                const int cx = g[0] + dxx, cy = g[1] + dy, cz = g[2] + dz;
                if (cx < 0 || cy < 0 || cz < 0 || cx >= S.n[0] || cy >= S.n[1] || cz >= S.n[2]) continue;
                const long long k = cell_key(S, cx, cy, cz);
                const int e = cell_start[k + 1];
                for (int i = cell_start[k]; i < e; ++i) {
                    const double d0 = sub(pos[0], x0[i]), d1 = sub(pos[1], x1[i]), d2 = sub(pos[2], x2[i]);
                    const double d = add(add(mul(d0, d0), mul(d1, d1)), mul(d2, d2));
                    best = d < best ? d : best;
                }
            }
    const double dist = best < 1e299 ? sqrt(best) : 1e300;
    const double cl = mul(CLAMP_FACTOR, S.dx);
    phi[t] = sub(dist < cl ? dist : cl, mul(R0_FACTOR, S.dx));
}

// blocks whose nodes can be the lowest corner of a cube with a negative corner:
// the active blocks and their lower neighbours
__global__ void k_cube_flags(int nb, const int4* __restrict__ coord, const SceneDev* __restrict__ sc,
                             int* __restrict__ flag) {
    const int slot = blockIdx.x * blockDim.x + threadIdx.x;
    if (slot >= nb) return;
    const int4 bc = coord[slot];
    const SceneDev& S = sc[bc.w];
    for (int c = 0; c < 8; ++c) {
        const int bx = bc.x - (c & 1), by = bc.y - ((c >> 1) & 1), bz = bc.z - (c >> 2);
        if (bx < 0 || by < 0 || bz < 0) continue;
        flag[S.block_base + bx + (long long)S.nb[0] * (by + (long long)S.nb[1] * bz)] = 1;
    }
}

__global__ void k_cube_list(long long nblk, const int* __restrict__ flag, const int* __restrict__ pos,
                            int* __restrict__ list) {
    const long long gb = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (gb >= nblk || !flag[gb]) return;
    list[pos[gb]] = (int)gb;
}

struct CubeCtx {
    const SceneDev* sc;
    int nsc;
    const int* bslot;
    const double* phi;
};

__device__ __forceinline__ int scene_of(const SceneDev* sc, int nsc, long long gb) {
    int lo = 0, hi = nsc - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (sc[mid].block_base <= gb) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ double node_phi(const CubeCtx& cc, const SceneDev& S, int gx, int gy, int gz) {
    const long long gb = S.block_base + (gx >> 2) + (long long)S.nb[0] * ((gy >> 2) + (long long)S.nb[1] * (gz >> 2));
    const int slot = cc.bslot[gb];
    if (slot < 0) return sub(mul(CLAMP_FACTOR, S.dx), mul(R0_FACTOR, S.dx));
    return cc.phi[(long long)slot * 64 + (gx & 3) + 4 * (gy & 3) + 16 * (gz & 3)];
}

// tetrahedron e of a cube: corners 000, e_a, e_a + e_b, 111 for axis order (a, b, c)
__device__ __forceinline__ void tet_corner(int e, int v, int* o) {
    const int ord[6][2] = {{0, 1}, {0, 2}, {1, 0}, {1, 2}, {2, 0}, {2, 1}};
    o[0] = o[1] = o[2] = 0;
    if (v == 3) {
        o[0] = o[1] = o[2] = 1;
    } else {
        if (v >= 1) o[ord[e][0]] = 1;
        if (v >= 2) o[ord[e][1]] = 1;
    }
}

// the triangles of one tetrahedron; writes up to 2 triangles (9 doubles each) when out != nullptr
__device__ int tet_tris(const SceneDev& S, const int* q, int e, const double* cphi, double* out) {
    int qv[4][3];
    double pv[4];
    for (int v = 0; v < 4; ++v) {
        int o[3];
        tet_corner(e, v, o);
        for (int a = 0; a < 3; ++a) qv[v][a] = q[a] + o[a];
        pv[v] = cphi[o[0] + 2 * o[1] + 4 * o[2]];
    }
    int ins[4], outs[4], ni = 0, no = 0;
    for (int v = 0; v < 4; ++v) {
        if (pv[v] < 0.0) ins[ni++] = v;
        else outs[no++] = v;
    }
    if (ni == 0 || ni == 4) return 0;
    const int nt = ni == 2 ? 2 : 1;
    if (!out) return nt;
    auto edge = [&](int i, int j, double* p) {
        const double t = pv[i] / sub(pv[i], pv[j]);
        for (int a = 0; a < 3; ++a) {
            const double xa = add(S.origin[a], mul((double)qv[i][a] + 0.5, S.dx));
            const double xb = add(S.origin[a], mul((double)qv[j][a] + 0.5, S.dx));
            p[a] = add(xa, mul(t, sub(xb, xa)));
        }
    };
    double* T0 = out;
    double* T1 = out + 9;
    if (ni == 1) {
        edge(ins[0], outs[0], T0);
        edge(ins[0], outs[1], T0 + 3);
        edge(ins[0], outs[2], T0 + 6);
    } else if (ni == 3) {
        edge(ins[0], outs[0], T0);
        edge(ins[1], outs[0], T0 + 3);
        edge(ins[2], outs[0], T0 + 6);
    } else {
        const int i = ins[0], j = ins[1], k = outs[0], l = outs[1];
        edge(i, k, T0);
        edge(i, l, T0 + 3);
        edge(j, l, T0 + 6);
        edge(i, k, T1);
        edge(j, l, T1 + 3);
        edge(j, k, T1 + 6);
    }
    // outward: along (centroid of the outside corners) - (centroid of the inside corners)
    double g[3];
    for (int a = 0; a < 3; ++a) {
        double so = 0.0, si = 0.0;
        for (int v = 0; v < no; ++v) so = add(so, (double)qv[outs[v]][a]);
        for (int v = 0; v < ni; ++v) si = add(si, (double)qv[ins[v]][a]);
        g[a] = sub(so / (double)no, si / (double)ni);
    }
    for (int tt = 0; tt < nt; ++tt) {
        double* T = out + 9 * tt;
        const double u[3] = {sub(T[3], T[0]), sub(T[4], T[1]), sub(T[5], T[2])};
        const double w[3] = {sub(T[6], T[0]), sub(T[7], T[1]), sub(T[8], T[2])};
        const double n0 = sub(mul(u[1], w[2]), mul(u[2], w[1]));
        const double n1 = sub(mul(u[2], w[0]), mul(u[0], w[2]));
        const double n2 = sub(mul(u[0], w[1]), mul(u[1], w[0]));
        if (add(add(mul(n0, g[0]), mul(n1, g[1])), mul(n2, g[2])) < 0.0) {
            for (int a = 0; a < 3; ++a) {
                const double tmp = T[3 + a];
                T[3 + a] = T[6 + a];
                T[6 + a] = tmp;
            }
        }
    }
    return nt;
}

// one thread per cube (lowest corner = local node of a listed block): corner phi
__device__ __forceinline__ bool cube_setup(const CubeCtx& cc, const int* list, long long t, const SceneDev*& Sp,
                                           int& scene, int* q, double* cphi, long long& key) {
    const long long gb = list[t >> 6];
    const int l = (int)(t & 63);
    scene = scene_of(cc.sc, cc.nsc, gb);
    const SceneDev& S = cc.sc[scene];
    Sp = &S;
    const long long r = gb - S.block_base;
    const int bx = (int)(r % S.nb[0]), by = (int)((r / S.nb[0]) % S.nb[1]), bz = (int)(r / ((long long)S.nb[0] * S.nb[1]));
    q[0] = bx * BS + (l & 3);
    q[1] = by * BS + ((l >> 2) & 3);
    q[2] = bz * BS + (l >> 4);
    if (q[0] >= S.n[0] - 1 || q[1] >= S.n[1] - 1 || q[2] >= S.n[2] - 1) return false;
    for (int c = 0; c < 8; ++c)
        cphi[c] = node_phi(cc, S, q[0] + (c & 1), q[1] + ((c >> 1) & 1), q[2] + (c >> 2));
    key = r * 64 + l;   // block-major key of the lowest corner within its scene
    return true;
}

__global__ void k_cube_count(long long ncube, const int* __restrict__ list, CubeCtx cc, int* __restrict__ cnt) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ncube) return;
    const SceneDev* S;
    int scene, q[3];
    double cphi[8];
    long long key;
    int n = 0;
    if (cube_setup(cc, list, t, S, scene, q, cphi, key))
        for (int e = 0; e < 6; ++e) n += tet_tris(*S, q, e, cphi, nullptr);
    cnt[t] = n;
}

// triangle records: 9 vertex coordinates, counter key, scene
__global__ void k_cube_emit(long long ncube, const int* __restrict__ list, CubeCtx cc, const int* __restrict__ off,
                            double* __restrict__ tv, long long* __restrict__ tkey, int* __restrict__ tscene) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ncube) return;
    const SceneDev* S;
    int scene, q[3];
    double cphi[8];
    long long key;
    if (!cube_setup(cc, list, t, S, scene, q, cphi, key)) return;
    long long o = off[t];
    for (int e = 0; e < 6; ++e) {
        double T[18];
        const int nt = tet_tris(*S, q, e, cphi, T);
        if (nt > 0) {   // constant indices keep T out of local memory
#pragma unroll
            for (int a = 0; a < 9; ++a) tv[o * 9 + a] = T[a];
            tkey[o] = (6 * key + e) * 2;
            tscene[o] = scene;
            ++o;
        }
        if (nt > 1) {
#pragma unroll
            for (int a = 0; a < 9; ++a) tv[o * 9 + a] = T[9 + a];
            tkey[o] = (6 * key + e) * 2 + 1;
            tscene[o] = scene;
            ++o;
        }
    }
}

// marching cubes (mcubes.cuh): triangles per cube, then the triangle records,
// triangle t of the cube with key q taking counter slot 12 q + t
__global__ void k_mc_count(long long ncube, const int* __restrict__ list, CubeCtx cc, int* __restrict__ cnt) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ncube) return;
    const SceneDev* S;
    int scene, q[3];
    double cphi[8];
    long long key;
    int n = 0;
    if (cube_setup(cc, list, t, S, scene, q, cphi, key)) {
        mc::Loops L;
        mc::cube_loops(cphi, L);
        n = L.ntri;
    }
    cnt[t] = n;
}

__global__ void k_mc_emit(long long ncube, const int* __restrict__ list, CubeCtx cc, const int* __restrict__ off,
                          double* __restrict__ tv, long long* __restrict__ tkey, int* __restrict__ tscene) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ncube) return;
    const SceneDev* S;
    int scene, q[3];
    double cphi[8];
    long long key;
    if (!cube_setup(cc, list, t, S, scene, q, cphi, key)) return;
    const long long o = off[t];
    const int room = off[t + 1] - off[t];   // the count pass walked the same loops
    mc::cube_triangles(cphi, q, S->dx, S->origin, [&](int k, const double* p0, const double* p1, const double* p2) {
        if (k >= room) return;
        const long long r = o + k;
        for (int a = 0; a < 3; ++a) {
            tv[r * 9 + a] = p0[a];
            tv[r * 9 + 3 + a] = p1[a];
            tv[r * 9 + 6 + a] = p2[a];
        }
        tkey[r] = 12 * key + k;
        tscene[r] = scene;
    });
}

struct TriGeom {
    double n[3], nn;
};

__device__ __forceinline__ TriGeom tri_geom(const double* T) {
    TriGeom g;
    const double u[3] = {sub(T[3], T[0]), sub(T[4], T[1]), sub(T[5], T[2])};
    const double w[3] = {sub(T[6], T[0]), sub(T[7], T[1]), sub(T[8], T[2])};
    g.n[0] = sub(mul(u[1], w[2]), mul(u[2], w[1]));
    g.n[1] = sub(mul(u[2], w[0]), mul(u[0], w[2]));
    g.n[2] = sub(mul(u[0], w[1]), mul(u[1], w[0]));
    g.nn = sqrt(add(add(mul(g.n[0], g.n[0]), mul(g.n[1], g.n[1])), mul(g.n[2], g.n[2])));
    return g;
}

__device__ __forceinline__ unsigned long long scene_seed(unsigned long long seed, int scene) {
    return seed ^ ((unsigned long long)scene * GOLDEN);
}

__device__ __forceinline__ int poisson_count(double lam, unsigned long long seed, unsigned long long base) {
    const double u = uniform01(seed, base);
    int k = 0;
    double p = exp(-lam);
    double F = p;
    while (u >= F && k < KMAX) {
        ++k;
        p = mul(p, lam) / (double)k;
        F = add(F, p);
    }
    return k;
}

__global__ void k_tri_count(long long ntri, const double* __restrict__ tv, const long long* __restrict__ tkey,
                            const int* __restrict__ tscene, const SceneDev* __restrict__ sc, unsigned long long seed,
                            double per_cell_area, int* __restrict__ kcnt, unsigned long long* __restrict__ scene_cnt) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ntri) return;
    const SceneDev& S = sc[tscene[t]];
    const TriGeom g = tri_geom(tv + t * 9);
    const double density = per_cell_area / mul(S.dx, S.dx);
    const double lam = mul(density, mul(0.5, g.nn));
    const int k = poisson_count(lam, scene_seed(seed, tscene[t]), (unsigned long long)tkey[t] * 64ull);
    kcnt[t] = k;
    if (k) atomicAdd(&scene_cnt[tscene[t]], (unsigned long long)k);
}

__global__ void k_tri_emit(long long ntri, const double* __restrict__ tv, const long long* __restrict__ tkey,
                           const int* __restrict__ tscene, const SceneDev* __restrict__ sc, unsigned long long seed,
                           double per_cell_area, const int* __restrict__ koff, const long long* __restrict__ scene_first,
                           Dev d) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ntri) return;
    const int scene = tscene[t];
    const SceneDev& S = sc[scene];
    const double* T = tv + t * 9;
    const TriGeom g = tri_geom(T);
    const double density = per_cell_area / mul(S.dx, S.dx);
    const unsigned long long sd = scene_seed(seed, scene);
    const unsigned long long base = (unsigned long long)tkey[t] * 64ull;
    const int k0 = koff[t], k = koff[t + 1] - k0;
    const double w = 1.0 / mul(g.nn, density);
    for (int i = 0; i < k; ++i) {
        const double r1 = uniform01(sd, base + 2 * i + 1), r2 = uniform01(sd, base + 2 * i + 2);
        const double a = sqrt(r1);
        const double b0 = sub(1.0, a), b1 = mul(a, sub(1.0, r2)), b2 = mul(a, r2);
        const long long j = (long long)k0 + i;
        double p[3];
        for (int c = 0; c < 3; ++c) {
            p[c] = add(add(mul(b0, T[c]), mul(b1, T[3 + c])), mul(b2, T[6 + c]));
            d.s[c][j] = p[c];
            d.dA[c][j] = mul(g.n[c], w);
        }
        uint8_t kind = 0;
        if (S.plane_mode) {
            const double ph = S.plane_n[0] * p[0] + S.plane_n[1] * p[1] + S.plane_n[2] * p[2] - S.plane_d;
            kind = ph < S.dx ? 1 : 0;
        }
        d.kind[j] = kind;
        d.bheat[j] = 0.0;
        d.Tbar[j] = S.T0;
        d.sid[j] = (int)(j - scene_first[scene]);
        d.ssc[j] = scene;
        d.parent[j] = -1;   // no parent until mpm_resample
    }
}

inline unsigned nblk(long long n, int nt) { return (unsigned)((n + nt - 1) / nt); }

}  // namespace

cudaError_t launch_generate_surface(mpm_ctx* c, unsigned long long seed, double per_cell_area, int method,
                                    long long* counts, int* capacity_error) {
    Dev& d = c->d;
    cudaStream_t st = c->st;
    *capacity_error = 0;
    // particles sorted by cell and the blocks of their stencils (no samples yet)
    cudaError_t e = launch_sort_particles(c);
    if (e != cudaSuccess) return e;
    const long long ns_keep = c->ns;
    c->ns = 0;
    e = launch_build_blocks(c);
    c->ns = ns_keep;
    if (e != cudaSuccess) return e;
    const int nb = c->NB;
    long long total = 0;
    for (int s = 0; s < c->nsc; ++s) counts[s] = 0;
    if (nb > 0 && c->np > 0) {
        double* phi = d.gmT;   // grid scratch until the next P2G
        MPM_LAUNCH k_phi<<<nblk((long long)nb * 64, 128), 128, 0, st>>>(nb, d.slot_coord, d.sc, d.cell_start, d.x[0],
                                                                       d.x[1], d.x[2], phi);
        // cube blocks: active blocks and their lower neighbours, in global block order
        const long long nblkg = c->total_blocks;
        cudaMemsetAsync(d.bflag, 0, sizeof(int) * nblkg, st);
        MPM_LAUNCH k_cube_flags<<<nblk(nb, 128), 128, 0, st>>>(nb, d.slot_coord, d.sc, d.bflag);
        launch_exclusive_scan(c, d.bflag, d.bscan, nblkg, d.scan_tmp, st);
        MPM_LAUNCH k_cube_list<<<nblk(nblkg, 256), 256, 0, st>>>(nblkg, d.bflag, d.bscan, d.bwork);
        cudaMemcpyAsync(c->hcounts + 5, d.bscan + nblkg, sizeof(int), cudaMemcpyDeviceToHost, st);
        e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return e;
        const long long ncube = (long long)c->hcounts[5] * 64;
        CubeCtx cc{d.sc, c->nsc, d.bslot, phi};
        // triangles per cube, then the triangle records
        int* tcnt = d.cell_count;     // sort scratch until the next resample
        int* toff = d.scell_count;
        if (method == MPM_ISO_CUBES) {
            MPM_LAUNCH k_mc_count<<<nblk(ncube, 128), 128, 0, st>>>(ncube, d.bwork, cc, tcnt);
        } else {
            MPM_LAUNCH k_cube_count<<<nblk(ncube, 128), 128, 0, st>>>(ncube, d.bwork, cc, tcnt);
        }
        launch_exclusive_scan(c, tcnt, toff, ncube, d.scan_tmp, st);
        cudaMemcpyAsync(c->hcounts + 5, toff + ncube, sizeof(int), cudaMemcpyDeviceToHost, st);
        e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return e;
        const long long ntri = c->hcounts[5];
        if (ntri >= c->total_cells) {   // the scan scratch covers total_cells entries
            *capacity_error = 1;
            return cudaSuccess;
        }
        if (ntri > 0) {
            const size_t need = (size_t)ntri * (9 * sizeof(double) + sizeof(long long) + 3 * sizeof(int)) + 64;
            if (need > c->tri_bytes) {
                if (c->tri_buf) cudaFree(c->tri_buf);
                c->tri_buf = nullptr;
                c->tri_bytes = 0;
                e = cudaMalloc(&c->tri_buf, need + need / 4);
                if (e != cudaSuccess) return e;
                c->tri_bytes = need + need / 4;
            }
            double* tv = (double*)c->tri_buf;
            long long* tkey = (long long*)(tv + 9 * ntri);
            int* tscene = (int*)(tkey + ntri);
            int* kcnt = tscene + ntri;
            int* koff = kcnt + ntri + 1;
            if (method == MPM_ISO_CUBES) {
                MPM_LAUNCH k_mc_emit<<<nblk(ncube, 128), 128, 0, st>>>(ncube, d.bwork, cc, toff, tv, tkey, tscene);
            } else {
                MPM_LAUNCH k_cube_emit<<<nblk(ncube, 128), 128, 0, st>>>(ncube, d.bwork, cc, toff, tv, tkey, tscene);
            }
            cudaMemsetAsync(d.scene_cnt, 0, sizeof(unsigned long long) * c->nsc, st);
            MPM_LAUNCH k_tri_count<<<nblk(ntri, 128), 128, 0, st>>>(ntri, tv, tkey, tscene, d.sc, seed, per_cell_area,
                                                                    kcnt, d.scene_cnt);
            launch_exclusive_scan(c, kcnt, koff, ntri, d.scan_tmp, st);
            cudaMemcpyAsync(c->hscene_cnt.data(), d.scene_cnt, sizeof(unsigned long long) * c->nsc, cudaMemcpyDeviceToHost, st);
            e = cudaStreamSynchronize(st);
            if (e != cudaSuccess) return e;
            long long first = 0;
            for (int s = 0; s < c->nsc; ++s) {
                counts[s] = (long long)c->hscene_cnt[s];
                if (counts[s] > c->hsc[s].s_end - c->hsc[s].s_begin) *capacity_error = 1;
                c->hscene_first[s] = first;
                first += counts[s];
            }
            total = first;
            if (total > c->Scap) *capacity_error = 1;
            if (*capacity_error) return cudaSuccess;
            cudaMemcpyAsync(d.scene_first, c->hscene_first.data(), sizeof(long long) * c->nsc, cudaMemcpyHostToDevice, st);
            MPM_LAUNCH k_tri_emit<<<nblk(ntri, 128), 128, 0, st>>>(ntri, tv, tkey, tscene, d.sc, seed, per_cell_area,
                                                                   koff, d.scene_first, d);
        }
    }
    c->ns = total;
    c->resampled = false;
    return cudaGetLastError();
}

}  // namespace mpm
