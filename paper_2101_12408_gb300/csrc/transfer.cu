// Resampling (closest parent, balance particles, split), P2G, grid finalisation,
// gamma(T), and G2P with the conservative merge. All float64: these run once per
// step and carry the momentum bookkeeping that must close to round-off.
//
// Paper sections: "Conservative Surface Particle Resampling" (Eq. pbal,
// Eq. cons_mom), "Transfer: P2G", "Transfer: G2P", "Thermomechanical Material
// Dependence and Phase Change", "Contact Angle".
#include "ctx.h"

namespace mpm {

namespace {

__device__ __forceinline__ int node_slot_index(const SceneDev& S, const int* __restrict__ bslot, int gx, int gy, int gz) {
    long long gb = S.block_base + (gx >> 2) + (long long)S.nb[0] * ((gy >> 2) + (long long)S.nb[1] * (gz >> 2));
    int slot = bslot[gb];
    return slot < 0 ? -1 : slot * 64 + ((gx & 3) + 4 * (gy & 3) + 16 * (gz & 3));
}

struct P3 { const double* a[3]; };
struct P9 { const double* a[9]; };
struct W3 { double* a[3]; };
struct W9 { double* a[9]; };
struct W12 { double* a[12]; };

// ---------------------------------------------------------------- resample

__global__ void k_nearest(int ns, P3 s, const int* __restrict__ ssc, P3 x, const int* __restrict__ pid,
                          const int* __restrict__ cell_start, const SceneDev* __restrict__ sc, int* __restrict__ parent,
                          W3 bpos, int* __restrict__ gcount, uint8_t* __restrict__ kind, int* err) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= ns) return;
    const SceneDev& S = sc[ssc[j]];
    double q[3] = {s.a[0][j], s.a[1][j], s.a[2][j]};
    int c[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        int ci = (int)floor((q[a] - S.origin[a]) * S.inv_dx);
        c[a] = ci < 1 ? 1 : (ci > S.n[a] - 2 ? S.n[a] - 2 : ci);
    }
    double best = 1e300;
    int bi = -1, bid = 0x7fffffff;
    // the 27 cells around the sample hold every particle within dx; when the
    // nearest is farther (samples generated on the union-of-spheres surface reach
    // ~1.1 dx), the 125 cells around it hold every particle within 2 dx
    for (int reach = 1; reach <= 2; ++reach) {
        if (reach == 2 && best <= S.dx * S.dx) break;
        for (int dz = -reach; dz <= reach; ++dz)
            for (int dy = -reach; dy <= reach; ++dy)
                for (int dxx = -reach; dxx <= reach; ++dxx) {
                    if (reach == 2 && dz > -2 && dz < 2 && dy > -2 && dy < 2 && dxx > -2 && dxx < 2) continue;
                    const int cx = c[0] + dxx, cy = c[1] + dy, cz = c[2] + dz;
                    if (cx < 0 || cy < 0 || cz < 0 || cx >= S.n[0] || cy >= S.n[1] || cz >= S.n[2]) continue;
                    long long k = cell_key(S, cx, cy, cz);
                    int e = cell_start[k + 1];
                    for (int i = cell_start[k]; i < e; ++i) {
                        double d0 = __dsub_rn(q[0], x.a[0][i]);
                        double d1 = __dsub_rn(q[1], x.a[1][i]);
                        double d2 = __dsub_rn(q[2], x.a[2][i]);
                        double dist = __dadd_rn(__dadd_rn(__dmul_rn(d0, d0), __dmul_rn(d1, d1)), __dmul_rn(d2, d2));
                        int id = pid[i];
                        if (dist < best || (dist == best && id < bid)) {
                            best = dist;
                            bi = i;
                            bid = id;
                        }
                    }
                }
    }
    if (bi < 0 || best > 4.0 * S.dx * S.dx) {
        atomicOr(err, ERR_FAR_SURFACE);
        parent[j] = -1;
        for (int a = 0; a < 3; ++a) bpos.a[a][j] = q[a];
        return;
    }
    parent[j] = bi;
    atomicAdd(&gcount[bi], 1);
#pragma unroll
    for (int a = 0; a < 3; ++a) bpos.a[a][j] = __dadd_rn(q[a], 2.0 * __dsub_rn(x.a[a][bi], q[a]));
    // solid-liquid: closer than dx to the plane or to the sphere
    if (S.plane_mode || S.sphere_mode) {
        bool near = false;
        if (S.plane_mode) near = S.plane_n[0] * q[0] + S.plane_n[1] * q[1] + S.plane_n[2] * q[2] - S.plane_d < S.dx;
        if (S.sphere_mode) {
            double nrm[3];
            near = near || sphere_phi_normal(S, q, nrm) < S.dx;
        }
        kind[j] = near ? 1 : 0;
    }
}

__global__ void k_split(int np, const double* __restrict__ m, const int* __restrict__ gcount, const int* __restrict__ psc,
                        const SceneDev* __restrict__ sc, double* __restrict__ mt) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= np) return;
    // the massless-sample variant keeps the parent's whole mass
    mt[i] = sc[psc[i]].massless ? m[i] : m[i] / (2.0 * gcount[i] + 1.0);
}

// ---------------------------------------------------------------- P2G

struct P2GArgs {
    P3 x, v;
    P9 A;
    const double *mt, *m, *T;
    P3 gT;
    const int* cell_start;
    const int* work;
    const int* work_gb;
    const int4* coord;
    const int* nbr;
    const SceneDev* sc;
    double *gm, *gmv, *gmT, *gmTT;
};

// One CTA per work block, one thread per cell, two warps. The cells' particles
// are taken in rows: pass r takes the r-th particle of every cell, so within a
// warp the 32 particles of a pass lie in 32 distinct cells and, for one stencil
// offset, add to 32 distinct nodes. Each warp accumulates into its own z-range of
// the halo (the two-warp layout of common.cuh), and offsets whose z differs by 2
// never meet within a warp, so a pass's 27 offsets go out in 18 phases of plain
// read-add-write ordered by __syncwarp; no shared-memory atomics (float64 atomics
// on shared memory are compare-and-swap loops on this GPU).
__global__ void __launch_bounds__(64) k_p2g_volume(P2GArgs a) {
    __shared__ __align__(16) double acc[6][UN];
    const int w = blockIdx.x;
    const int slot = a.work[w];
    const long long gb = a.work_gb[w];
    const int4 bc = a.coord[slot];
    const SceneDev& S = a.sc[bc.w];
    const int nf = S.thermal ? 6 : 4;
    for (int t = threadIdx.x; t < (int)(6 * UN * sizeof(double) / 16); t += blockDim.x)
        reinterpret_cast<int4*>(&acc[0][0])[t] = make_int4(0, 0, 0, 0);
    __syncthreads();
    const int cell = threadIdx.x, wid = threadIdx.x >> 5;
    const int lx = cell & 3, ly = (cell >> 2) & 3, lz = cell >> 4;
    const int zb = lz + 2 * wid;
    const int cbeg = a.cell_start[gb * 64 + cell], cend = a.cell_start[gb * 64 + cell + 1];
    const int rows = __reduce_max_sync(0xffffffffu, cend - cbeg);
    const double dx = S.dx;
    for (int r = 0; r < rows; ++r) {
        const int i = cbeg + r;
        const bool act = i < cend;
        double wx[3] = {0, 0, 0}, wy[3] = {0, 0, 0}, wz[3] = {0, 0, 0};
        double mt = 0.0, B[3] = {0, 0, 0}, E[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
        double mp = 0.0, TB = 0.0, TE[3] = {0, 0, 0};
        if (act) {
            double u[3];
            for (int q = 0; q < 3; ++q) u[q] = (a.x.a[q][i] - S.origin[q]) * S.inv_dx;
            Stencil<double> st;
            make_stencil<double>(u, S.inv_dx, st);
            double f[3];
            for (int q = 0; q < 3; ++q) f[q] = u[q] - 0.5 - (st.c[q] - 1);
            for (int k = 0; k < 3; ++k) {
                wx[k] = st.w[0][k];
                wy[k] = st.w[1][k];
                wz[k] = st.w[2][k];
            }
            mt = a.mt[i];
            // node (cx, cy, cz) receives mt N (v + A (x_i - x_p)) with x_i - x_p = (c - f) dx,
            // i.e. N (B + E c): B = mt (v - dx A f), E = mt dx A
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                double Aq[3] = {a.A.a[3 * q][i], a.A.a[3 * q + 1][i], a.A.a[3 * q + 2][i]};
                B[q] = mt * (a.v.a[q][i] - dx * (Aq[0] * f[0] + Aq[1] * f[1] + Aq[2] * f[2]));
#pragma unroll
                for (int e = 0; e < 3; ++e) E[3 * q + e] = mt * dx * Aq[e];
            }
            if (S.thermal) {
                mp = a.m[i];
                double g[3] = {a.gT.a[0][i], a.gT.a[1][i], a.gT.a[2][i]};
                TB = mp * (a.T[i] - dx * (g[0] * f[0] + g[1] * f[1] + g[2] * f[2]));
                for (int e = 0; e < 3; ++e) TE[e] = mp * dx * g[e];
            }
        }
        // phases: (cx, cy) with cz in {0, 2}, then (cx, cy) with cz = 1
#pragma unroll
        for (int ph = 0; ph < 2; ++ph)
#pragma unroll
            for (int cy = 0; cy < 3; ++cy)
#pragma unroll
                for (int cx = 0; cx < 3; ++cx) {
                    __syncwarp();
                    if (act) {
#pragma unroll
                        for (int h = 0; h < 2; ++h) {
                            const int cz = ph == 0 ? 2 * h : 1;
                            const double N = wx[cx] * (wy[cy] * wz[cz]);
                            const int k = pidx(lx + cx, ly + cy, zb + cz);
                            acc[0][k] += mt * N;
#pragma unroll
                            for (int q = 0; q < 3; ++q)
                                acc[1 + q][k] += N * (B[q] + E[3 * q] * cx + E[3 * q + 1] * cy + E[3 * q + 2] * cz);
                            if (nf == 6) {
                                acc[4][k] += mp * N;
                                acc[5][k] += N * (TB + TE[0] * cx + TE[1] * cy + TE[2] * cz);
                            }
                            if (ph == 1) break;
                        }
                    }
                }
        __syncwarp();
    }
    __syncthreads();
    // the two warps' levels summed per halo node, then added to the grid
    for (int h = threadIdx.x; h < HN; h += blockDim.x) {
        const int hx = h % HE, hy = (h / HE) % HE, hz = h / (HE * HE);
        double v[6];
#pragma unroll
        for (int f = 0; f < 6; ++f) {
            v[f] = 0.0;
            if (hz <= 3) v[f] += acc[f][pidx(hx, hy, hz)];
            if (hz >= 2) v[f] += acc[f][pidx(hx, hy, hz + 2)];
        }
        if (v[0] == 0.0 && v[4] == 0.0) continue;
        int ns, loc;
        halo_source(a.nbr, slot, h, ns, loc);
        if (ns < 0) continue;
        atomicAdd(&a.gm[ns * 64 + loc], v[0]);
        for (int q = 0; q < 3; ++q) atomicAdd(&a.gmv[ns * 192 + q * 64 + loc], v[1 + q]);
        if (nf == 6) {
            atomicAdd(&a.gmT[ns * 64 + loc], v[4]);
            atomicAdd(&a.gmTT[ns * 64 + loc], v[5]);
        }
    }
}

__global__ void k_p2g_surface(int ns, P3 s, P3 bpos, const int* __restrict__ ssc, const int* __restrict__ parent,
                              P3 x, P3 v, P9 A, const double* __restrict__ mt, const int* __restrict__ bslot,
                              const SceneDev* __restrict__ sc, double* __restrict__ gm, double* __restrict__ gmv) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= ns) return;
    int p = parent[j];
    if (p < 0) return;
    const SceneDev& S = sc[ssc[j]];
    if (S.massless) return;   // massless samples and no balance particles
    double mp = mt[p];
    double vp[3] = {v.a[0][p], v.a[1][p], v.a[2][p]};
    double Ap[9];
    for (int q = 0; q < 9; ++q) Ap[q] = A.a[q][p];
    for (int which = 0; which < 2; ++which) {
        const P3& P = which ? bpos : s;
        double u[3];
        for (int q = 0; q < 3; ++q) u[q] = (P.a[q][j] - S.origin[q]) * S.inv_dx;
        Stencil<double> st;
        make_stencil<double>(u, S.inv_dx, st);
        double f[3];
        for (int q = 0; q < 3; ++q) f[q] = u[q] - 0.5 - (st.c[q] - 1);
        for (int cz = 0; cz < 3; ++cz)
            for (int cy = 0; cy < 3; ++cy)
                for (int cx = 0; cx < 3; ++cx) {
                    int idx = node_slot_index(S, bslot, st.c[0] - 1 + cx, st.c[1] - 1 + cy, st.c[2] - 1 + cz);
                    if (idx < 0) continue;
                    double N = st.w[0][cx] * st.w[1][cy] * st.w[2][cz];
                    double r[3] = {(cx - f[0]) * S.dx, (cy - f[1]) * S.dx, (cz - f[2]) * S.dx};
                    double wm = mp * N;
                    int slot = idx >> 6, loc = idx & 63;
                    atomicAdd(&gm[idx], wm);
                    for (int q = 0; q < 3; ++q)
                        atomicAdd(&gmv[slot * 192 + q * 64 + loc],
                                  wm * (vp[q] + Ap[3 * q] * r[0] + Ap[3 * q + 1] * r[1] + Ap[3 * q + 2] * r[2]));
                }
    }
}

// Node finalisation: v^n, T^n, projection codes, inverse masses.
template <typename R>
__global__ void k_grid_final(int nb, const int4* __restrict__ coord, const SceneDev* __restrict__ sc,
                             const double* __restrict__ gm, const double* __restrict__ gmv, const double* __restrict__ gmT,
                             const double* __restrict__ gmTT, double* __restrict__ gvn, double* __restrict__ gTn,
                             uint8_t* __restrict__ pcode, R* __restrict__ invm, R* __restrict__ hinvd) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nb * 64) return;
    int slot = t >> 6, l = t & 63;
    int4 bc = coord[slot];
    const SceneDev& S = sc[bc.w];
    int g[3] = {bc.x * 4 + (l & 3), bc.y * 4 + ((l >> 2) & 3), bc.z * 4 + (l >> 4)};
    double m = gm[t];
    for (int q = 0; q < 3; ++q) gvn[slot * 192 + q * 64 + l] = m > 0.0 ? gmv[slot * 192 + q * 64 + l] / m : 0.0;
    double mT = S.thermal ? gmT[t] : 0.0;
    gTn[t] = mT > 0.0 ? gmTT[t] / mT : 0.0;
    hinvd[t] = mT > 0.0 ? (R)(S.dt / (S.cp * mT)) : R(0);
    // Dirichlet reading: outer two node layers per face, plus the solid plane
    bool sticky = false, on_plane = false;
    int slip = 0;
    for (int f = 0; f < 6; ++f) {
        int ax = f >> 1, side = f & 1, mode = S.walls[f];
        if (mode == 0) continue;
        bool on = side == 0 ? (g[ax] <= 1) : (g[ax] >= S.n[ax] - 2);
        if (!on) continue;
        if (mode == 2) sticky = true; else slip |= 1 << ax;
    }
    if (S.plane_mode) {
        double xn = 0.0;
        for (int q = 0; q < 3; ++q) xn += S.plane_n[q] * ((g[q] + 0.5) * S.dx + S.origin[q]);
        on_plane = xn - S.plane_d < 0.0;
        if (on_plane && S.plane_mode == 2) sticky = true;
    }
    bool on_sphere = false;
    if (S.sphere_mode) {
        double xi[3], nrm[3];
        for (int q = 0; q < 3; ++q) xi[q] = (g[q] + 0.5) * S.dx + S.origin[q];
        on_sphere = sphere_phi_normal(S, xi, nrm) < 0.0;
        if (on_sphere && S.sphere_mode == 2) sticky = true;
    }
    int nslip = __popc(slip);
    uint8_t code = 0;
    // two independent solid normals at one node fix it (plane and sphere, or a
    // solid and a wall)
    if (sticky || (on_plane && nslip > 0) || (on_sphere && nslip > 0) || (on_plane && on_sphere) || nslip == 3 ||
        !(m > 0.0))
        code = PC_FIXED;
    else {
        if (slip & 1) code |= PC_SLIPX;
        if (slip & 2) code |= PC_SLIPY;
        if (slip & 4) code |= PC_SLIPZ;
        if (on_plane) code |= PC_PLANE;
        if (on_sphere) code |= PC_SPHERE;
    }
    pcode[t] = code;
    invm[t] = (m > 0.0 && code != PC_FIXED) ? (R)(1.0 / m) : R(0);
}

// gamma_r from the grid temperature (normalised over nodes with thermal mass)
template <typename R>
__global__ void k_gamma(int ns, P3 s, const int* __restrict__ ssc, const uint8_t* __restrict__ kind,
                        const int* __restrict__ bslot, const SceneDev* __restrict__ sc, const double* __restrict__ gmT,
                        const double* __restrict__ gTn, double* __restrict__ gamma, double* __restrict__ Tr,
                        R* __restrict__ swn) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= ns) return;
    const SceneDev& S = sc[ssc[j]];
    double T = S.T0, wsum = 0.0;
    if (S.thermal) {
        double u[3];
        for (int q = 0; q < 3; ++q) u[q] = (s.a[q][j] - S.origin[q]) * S.inv_dx;
        Stencil<double> st;
        make_stencil<double>(u, S.inv_dx, st);
        double tw = 0.0;
        for (int cz = 0; cz < 3; ++cz)
            for (int cy = 0; cy < 3; ++cy)
                for (int cx = 0; cx < 3; ++cx) {
                    int idx = node_slot_index(S, bslot, st.c[0] - 1 + cx, st.c[1] - 1 + cy, st.c[2] - 1 + cz);
                    if (idx < 0 || !(gmT[idx] > 0.0)) continue;
                    double N = st.w[0][cx] * st.w[1][cy] * st.w[2][cz];
                    wsum += N;
                    tw += N * gTn[idx];
                }
        if (wsum > 0.0) T = tw / wsum;
    }
    Tr[j] = T;
    swn[j] = wsum > 0.0 ? (R)(1.0 / wsum) : R(0);
    double g;
    if (kind[j] == 1) g = S.gamma_sl;
    else if (S.gamma_law == 0) g = S.gamma_lg;
    else {
        g = S.gamma_p[0] + S.gamma_p[1] * (T - S.T0);
        g = fmin(fmax(g, S.gamma_p[2]), S.gamma_p[3]);
    }
    gamma[j] = g;
}

// ---------------------------------------------------------------- G2P

struct G2PArgs {
    int np;
    P3 x;
    const double *mt;
    const int* psc;
    const uint8_t* phase;
    const int* bslot;
    const SceneDev* sc;
    const double *gvhat, *gThat;
    W12 acc;
    double *J, *T;
    W9 F;
    W3 gT;
    const float *vhi, *vlo;   // float-float copy of gvhat (k_g2p_volume_mixed)
};

// hi = fl32(v), lo = fl32(v - hi): v to about 48 bits in two float32 arrays
__global__ void k_split_ff(long long n, const double* __restrict__ v, float* __restrict__ hi, float* __restrict__ lo) {
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    double x = v[t];
    float h = (float)x;
    hi[t] = h;
    lo[t] = (float)(x - (double)h);
}

// G2P of the float32 operator form. The particle velocity keeps float64
// weights and node values, so sum_p m_p v_p = sum_i m_i v_i still holds to
// float64 round-off; the affine moment, the velocity gradient and the
// temperature gradient are formed in float32 from the node values minus the
// stencil's centre node (exact in exact arithmetic: the B-spline weights have
// zero first moment and their gradients sum to zero). Differences come from the
// float-float copy, so float32 rounds the variation over the stencil, not the
// velocity itself.
__global__ void __launch_bounds__(128) k_g2p_volume_mixed(G2PArgs a) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.np) return;
    const SceneDev& S = a.sc[a.psc[i]];
    double u[3];
    for (int q = 0; q < 3; ++q) u[q] = (a.x.a[q][i] - S.origin[q]) * S.inv_dx;
    Stencil<double> st;
    make_stencil<double>(u, S.inv_dx, st);
    float wf[3][3], dwf[3][3], ff[3];
    const float inv_dxf = (float)S.inv_dx, dxf = (float)S.dx;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        ff[q] = (float)(u[q] - 0.5 - (double)(st.c[q] - 1));
        bspline<float>(ff[q], wf[q], dwf[q]);
#pragma unroll
        for (int k = 0; k < 3; ++k) dwf[q][k] *= inv_dxf;
    }
    const int ic = node_slot_index(S, a.bslot, st.c[0], st.c[1], st.c[2]);
    float rhi[3] = {0.f, 0.f, 0.f}, rlo[3] = {0.f, 0.f, 0.f};
    double Tc = 0.0;
    if (ic >= 0) {
        const int k0 = (ic >> 6) * 192 + (ic & 63);
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            rhi[q] = a.vhi[k0 + q * 64];
            rlo[q] = a.vlo[k0 + q * 64];
        }
        if (S.thermal) Tc = a.gThat[ic];
    }
    double wyz[3][3];
#pragma unroll
    for (int cy = 0; cy < 3; ++cy)
#pragma unroll
        for (int cz = 0; cz < 3; ++cz) wyz[cy][cz] = st.w[1][cy] * st.w[2][cz];
    double pv[3] = {0, 0, 0}, T = 0.0;
    float tv[9] = {0}, L[9] = {0}, gT[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int cz = 0; cz < 3; ++cz)
#pragma unroll
        for (int cy = 0; cy < 3; ++cy)
#pragma unroll
            for (int cx = 0; cx < 3; ++cx) {
                int idx = node_slot_index(S, a.bslot, st.c[0] - 1 + cx, st.c[1] - 1 + cy, st.c[2] - 1 + cz);
                if (idx < 0) continue;
                const int k0 = (idx >> 6) * 192 + (idx & 63);
                const double N = st.w[0][cx] * wyz[cy][cz];
                const float Nf = wf[0][cx] * wf[1][cy] * wf[2][cz];
                const float dN[3] = {dwf[0][cx] * wf[1][cy] * wf[2][cz], wf[0][cx] * dwf[1][cy] * wf[2][cz],
                                     wf[0][cx] * wf[1][cy] * dwf[2][cz]};
                const float r[3] = {((float)cx - ff[0]) * dxf, ((float)cy - ff[1]) * dxf, ((float)cz - ff[2]) * dxf};
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    pv[q] += N * a.gvhat[k0 + q * 64];
                    const float dq = (a.vhi[k0 + q * 64] - rhi[q]) + (a.vlo[k0 + q * 64] - rlo[q]);
                    const float Nd = Nf * dq;
#pragma unroll
                    for (int e = 0; e < 3; ++e) {
                        tv[3 * q + e] += Nd * r[e];
                        L[3 * q + e] += dq * dN[e];
                    }
                }
                if (S.thermal) {
                    double Th = a.gThat[idx];
                    T += N * Th;
                    float dT = (float)(Th - Tc);
#pragma unroll
                    for (int e = 0; e < 3; ++e) gT[e] += dT * dN[e];
                }
            }
    double mt = a.mt[i];
    for (int q = 0; q < 3; ++q) a.acc.a[q][i] = mt * pv[q];
    for (int q = 0; q < 9; ++q) a.acc.a[3 + q][i] = mt * (double)tv[q];
    double dt = S.dt;
    if (a.phase[i] == 0) {
        a.J[i] = (1.0 + dt * (double)(L[0] + L[4] + L[8])) * a.J[i];
    } else {
        double Fo[9], M[9], Fnew[9];
        for (int q = 0; q < 9; ++q) Fo[q] = a.F.a[q][i];
        for (int q = 0; q < 9; ++q) M[q] = dt * (double)L[q] + ((q % 4 == 0) ? 1.0 : 0.0);
        matmul3<double>(M, Fo, Fnew);
        for (int q = 0; q < 9; ++q) a.F.a[q][i] = Fnew[q];
    }
    if (S.thermal) {
        a.T[i] = T;
        for (int e = 0; e < 3; ++e) a.gT.a[e][i] = (double)gT[e];
    }
}

__global__ void k_g2p_volume(G2PArgs a) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.np) return;
    const SceneDev& S = a.sc[a.psc[i]];
    double u[3];
    for (int q = 0; q < 3; ++q) u[q] = (a.x.a[q][i] - S.origin[q]) * S.inv_dx;
    Stencil<double> st;
    make_stencil<double>(u, S.inv_dx, st);
    double f[3];
    for (int q = 0; q < 3; ++q) f[q] = u[q] - 0.5 - (st.c[q] - 1);
    double pv[3] = {0, 0, 0}, tv[9] = {0}, L[9] = {0}, T = 0.0, gT[3] = {0, 0, 0};
    for (int cz = 0; cz < 3; ++cz)
        for (int cy = 0; cy < 3; ++cy)
            for (int cx = 0; cx < 3; ++cx) {
                int idx = node_slot_index(S, a.bslot, st.c[0] - 1 + cx, st.c[1] - 1 + cy, st.c[2] - 1 + cz);
                if (idx < 0) continue;
                int slot = idx >> 6, loc = idx & 63;
                double N = st.w[0][cx] * st.w[1][cy] * st.w[2][cz];
                double dN[3] = {st.dw[0][cx] * st.w[1][cy] * st.w[2][cz], st.w[0][cx] * st.dw[1][cy] * st.w[2][cz],
                                st.w[0][cx] * st.w[1][cy] * st.dw[2][cz]};
                double r[3] = {(cx - f[0]) * S.dx, (cy - f[1]) * S.dx, (cz - f[2]) * S.dx};
                double vh[3];
                for (int q = 0; q < 3; ++q) vh[q] = a.gvhat[slot * 192 + q * 64 + loc];
                for (int q = 0; q < 3; ++q) {
                    pv[q] += N * vh[q];
                    for (int e = 0; e < 3; ++e) {
                        tv[3 * q + e] += N * vh[q] * r[e];
                        L[3 * q + e] += vh[q] * dN[e];
                    }
                }
                if (S.thermal) {
                    double Th = a.gThat[idx];
                    T += N * Th;
                    for (int e = 0; e < 3; ++e) gT[e] += Th * dN[e];
                }
            }
    double mt = a.mt[i];
    for (int q = 0; q < 3; ++q) a.acc.a[q][i] = mt * pv[q];
    for (int q = 0; q < 9; ++q) a.acc.a[3 + q][i] = mt * tv[q];
    double dt = S.dt;
    if (a.phase[i] == 0) {
        a.J[i] = (1.0 + dt * (L[0] + L[4] + L[8])) * a.J[i];
    } else {
        double Fo[9], M[9], Fnew[9];
        for (int q = 0; q < 9; ++q) Fo[q] = a.F.a[q][i];
        for (int q = 0; q < 9; ++q) M[q] = dt * L[q] + ((q % 4 == 0) ? 1.0 : 0.0);
        matmul3<double>(M, Fo, Fnew);
        for (int q = 0; q < 9; ++q) a.F.a[q][i] = Fnew[q];
    }
    if (S.thermal) {
        a.T[i] = T;
        for (int e = 0; e < 3; ++e) a.gT.a[e][i] = gT[e];
    }
}

__global__ void k_g2p_surface(int ns, W3 s, W3 dA, P3 bpos, const int* __restrict__ ssc, const int* __restrict__ parent,
                              P3 x, const double* __restrict__ mt, const int* __restrict__ bslot,
                              const SceneDev* __restrict__ sc, const double* __restrict__ gvhat, W12 acc) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= ns) return;
    int p = parent[j];
    const SceneDev& S = sc[ssc[j]];
    double xp[3] = {x.a[0][p < 0 ? 0 : p], x.a[1][p < 0 ? 0 : p], x.a[2][p < 0 ? 0 : p]};
    double mp = p < 0 ? 0.0 : mt[p];
    double sv[3] = {0, 0, 0}, Ls[9] = {0};
    for (int which = 0; which < 2; ++which) {
        const double* P[3] = {which ? bpos.a[0] : s.a[0], which ? bpos.a[1] : s.a[1], which ? bpos.a[2] : s.a[2]};
        double pos[3] = {P[0][j], P[1][j], P[2][j]};
        double u[3];
        for (int q = 0; q < 3; ++q) u[q] = (pos[q] - S.origin[q]) * S.inv_dx;
        Stencil<double> st;
        make_stencil<double>(u, S.inv_dx, st);
        double f[3];
        for (int q = 0; q < 3; ++q) f[q] = u[q] - 0.5 - (st.c[q] - 1);
        double pv[3] = {0, 0, 0}, tv[9] = {0};
        for (int cz = 0; cz < 3; ++cz)
            for (int cy = 0; cy < 3; ++cy)
                for (int cx = 0; cx < 3; ++cx) {
                    int idx = node_slot_index(S, bslot, st.c[0] - 1 + cx, st.c[1] - 1 + cy, st.c[2] - 1 + cz);
                    if (idx < 0) continue;
                    int slot = idx >> 6, loc = idx & 63;
                    double N = st.w[0][cx] * st.w[1][cy] * st.w[2][cz];
                    // r = x_i - x_p (relative to the parent, the centre of mass of the group)
                    double r[3] = {(cx - f[0]) * S.dx + pos[0] - xp[0], (cy - f[1]) * S.dx + pos[1] - xp[1],
                                   (cz - f[2]) * S.dx + pos[2] - xp[2]};
                    double vh[3];
                    for (int q = 0; q < 3; ++q) vh[q] = gvhat[slot * 192 + q * 64 + loc];
                    for (int q = 0; q < 3; ++q) {
                        pv[q] += N * vh[q];
                        for (int e = 0; e < 3; ++e) tv[3 * q + e] += N * vh[q] * r[e];
                    }
                    if (which == 0) {
                        double dN[3] = {st.dw[0][cx] * st.w[1][cy] * st.w[2][cz], st.w[0][cx] * st.dw[1][cy] * st.w[2][cz],
                                        st.w[0][cx] * st.w[1][cy] * st.dw[2][cz]};
                        for (int q = 0; q < 3; ++q) {
                            sv[q] += N * vh[q];
                            for (int e = 0; e < 3; ++e) Ls[3 * q + e] += vh[q] * dN[e];
                        }
                    }
                }
        if (p >= 0 && !S.massless) {
            for (int q = 0; q < 3; ++q) atomicAdd(&acc.a[q][p], mp * pv[q]);
            for (int q = 0; q < 9; ++q) atomicAdd(&acc.a[3 + q][p], mp * tv[q]);
        }
    }
    // carry the sample: s += dt v(s), dA <- cof(I + dt grad v(s)) dA
    double dt = S.dt;
    double M[9], C[9];
    for (int q = 0; q < 9; ++q) M[q] = dt * Ls[q] + ((q % 4 == 0) ? 1.0 : 0.0);
    cofactor<double>(M, C);
    double a0[3] = {dA.a[0][j], dA.a[1][j], dA.a[2][j]};
    for (int q = 0; q < 3; ++q) dA.a[q][j] = C[3 * q] * a0[0] + C[3 * q + 1] * a0[1] + C[3 * q + 2] * a0[2];
    for (int q = 0; q < 3; ++q) s.a[q][j] = s.a[q][j] + dt * sv[q];
}

__global__ void k_g2p_final(int np, W3 x, W3 v, W9 A, const double* __restrict__ m, const int* __restrict__ psc,
                            const SceneDev* __restrict__ sc, W12 acc, uint8_t* __restrict__ phase,
                            double* __restrict__ J, W9 F, const double* __restrict__ T) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= np) return;
    const SceneDev& S = sc[psc[i]];
    double mp = m[i];
    double vp[3];
    for (int q = 0; q < 3; ++q) vp[q] = acc.a[q][i] / mp;
    double sA = 4.0 / (mp * S.dx * S.dx);
    for (int q = 0; q < 9; ++q) A.a[q][i] = acc.a[3 + q][i] * sA;
    for (int q = 0; q < 3; ++q) {
        v.a[q][i] = vp[q];
        x.a[q][i] = x.a[q][i] + S.dt * vp[q];
    }
    if (S.phase_change) {
        uint8_t ph = phase[i];
        double Tp = T[i];
        bool melt = ph == 1 && Tp > S.T_melt;
        bool freeze = ph == 0 && Tp < S.T_melt;
        if (melt || freeze) {
            phase[i] = melt ? 0 : 1;
            J[i] = 1.0;
            for (int q = 0; q < 9; ++q) F.a[q][i] = (q % 4 == 0) ? 1.0 : 0.0;
        }
    }
}

inline unsigned nblk(long long n, int nt) { return (unsigned)((n + nt - 1) / nt); }

}  // namespace

cudaError_t launch_nearest_parent(mpm_ctx* c) {
    Dev& d = c->d;
    cudaStream_t st = c->st;
    cudaMemsetAsync(d.gcount, 0, sizeof(int) * (c->np > 0 ? c->np : 1), st);
    if (c->ns > 0) {
        MPM_LAUNCH k_nearest<<<nblk(c->ns, 128), 128, 0, st>>>((int)c->ns, P3{{d.s[0], d.s[1], d.s[2]}}, d.ssc,
                                                    P3{{d.x[0], d.x[1], d.x[2]}}, d.pid, d.cell_start, d.sc, d.parent,
                                                    W3{{d.bpos[0], d.bpos[1], d.bpos[2]}}, d.gcount, d.kind, d.err);
    }
    if (c->np > 0) MPM_LAUNCH k_split<<<nblk(c->np, 256), 256, 0, st>>>((int)c->np, d.m, d.gcount, d.psc, d.sc, d.mt);
    return cudaGetLastError();
}

cudaError_t launch_p2g(mpm_ctx* c) {
    Dev& d = c->d;
    cudaStream_t st = c->st;
    size_t nn = (size_t)c->NB * 64;
    cudaMemsetAsync(d.gm, 0, sizeof(double) * nn, st);
    cudaMemsetAsync(d.gmv, 0, sizeof(double) * nn * 3, st);
    cudaMemsetAsync(d.gmT, 0, sizeof(double) * nn, st);
    cudaMemsetAsync(d.gmTT, 0, sizeof(double) * nn, st);
    if (c->NW > 0) {
        P2GArgs a;
        a.x = P3{{d.x[0], d.x[1], d.x[2]}};
        a.v = P3{{d.v[0], d.v[1], d.v[2]}};
        for (int q = 0; q < 9; ++q) a.A.a[q] = d.A[q];
        a.mt = d.mt;
        a.m = d.m;
        a.T = d.T;
        a.gT = P3{{d.gT[0], d.gT[1], d.gT[2]}};
        a.cell_start = d.cell_start;
        a.work = d.work;
        a.work_gb = d.work_gb;
        a.coord = d.slot_coord;
        a.nbr = d.nbr;
        a.sc = d.sc;
        a.gm = d.gm;
        a.gmv = d.gmv;
        a.gmT = d.gmT;
        a.gmTT = d.gmTT;
        MPM_LAUNCH k_p2g_volume<<<c->NW, 64, 0, st>>>(a);
    }
    if (c->ns > 0) {
        P9 A;
        for (int q = 0; q < 9; ++q) A.a[q] = d.A[q];
        MPM_LAUNCH k_p2g_surface<<<nblk(c->ns, 128), 128, 0, st>>>((int)c->ns, P3{{d.s[0], d.s[1], d.s[2]}},
                                                        P3{{d.bpos[0], d.bpos[1], d.bpos[2]}}, d.ssc, d.parent,
                                                        P3{{d.x[0], d.x[1], d.x[2]}}, P3{{d.v[0], d.v[1], d.v[2]}}, A,
                                                        d.mt, d.bslot, d.sc, d.gm, d.gmv);
    }
    if (c->NB > 0) {
        if (c->rsize == 4)
            MPM_LAUNCH k_grid_final<float><<<nblk(nn, 256), 256, 0, st>>>(c->NB, d.slot_coord, d.sc, d.gm, d.gmv, d.gmT, d.gmTT,
                                                              d.gvn, d.gTn, d.pcode, (float*)d.invm, (float*)d.hinvd);
        else
            MPM_LAUNCH k_grid_final<double><<<nblk(nn, 256), 256, 0, st>>>(c->NB, d.slot_coord, d.sc, d.gm, d.gmv, d.gmT, d.gmTT,
                                                               d.gvn, d.gTn, d.pcode, (double*)d.invm, (double*)d.hinvd);
    }
    if (c->ns > 0) {
        if (c->rsize == 4)
            MPM_LAUNCH k_gamma<float><<<nblk(c->ns, 128), 128, 0, st>>>((int)c->ns, P3{{d.s[0], d.s[1], d.s[2]}}, d.ssc, d.kind,
                                                             d.bslot, d.sc, d.gmT, d.gTn, d.gamma, d.Tr, (float*)d.swn);
        else
            MPM_LAUNCH k_gamma<double><<<nblk(c->ns, 128), 128, 0, st>>>((int)c->ns, P3{{d.s[0], d.s[1], d.s[2]}}, d.ssc, d.kind,
                                                              d.bslot, d.sc, d.gmT, d.gTn, d.gamma, d.Tr, (double*)d.swn);
    }
    return cudaGetLastError();
}

cudaError_t launch_g2p(mpm_ctx* c) {
    Dev& d = c->d;
    cudaStream_t st = c->st;
    if (c->np > 0) {
        G2PArgs a;
        a.np = (int)c->np;
        a.x = P3{{d.x[0], d.x[1], d.x[2]}};
        a.mt = d.mt;
        a.psc = d.psc;
        a.phase = d.phase;
        a.bslot = d.bslot;
        a.sc = d.sc;
        a.gvhat = d.gvhat;
        a.gThat = d.gThat;
        for (int q = 0; q < 12; ++q) a.acc.a[q] = d.acc[q];
        a.J = d.J;
        a.T = d.T;
        for (int q = 0; q < 9; ++q) a.F.a[q] = d.F[q];
        for (int q = 0; q < 3; ++q) a.gT.a[q] = d.gT[q];
        if (c->rsize == 4 && c->NB > 0) {
            // the momentum CG vectors are free after the solve: hold the float-float copy
            long long n3 = (long long)c->NB * 192;
            a.vhi = (const float*)d.cr;
            a.vlo = (const float*)d.cp;
            MPM_LAUNCH k_split_ff<<<nblk(n3, 256), 256, 0, st>>>(n3, d.gvhat, (float*)d.cr, (float*)d.cp);
            MPM_LAUNCH k_g2p_volume_mixed<<<nblk(c->np, 128), 128, 0, st>>>(a);
        } else {
            a.vhi = a.vlo = nullptr;
            MPM_LAUNCH k_g2p_volume<<<nblk(c->np, 128), 128, 0, st>>>(a);
        }
    }
    W12 acc;
    for (int q = 0; q < 12; ++q) acc.a[q] = d.acc[q];
    if (c->ns > 0) {
        MPM_LAUNCH k_g2p_surface<<<nblk(c->ns, 128), 128, 0, st>>>((int)c->ns, W3{{d.s[0], d.s[1], d.s[2]}},
                                                        W3{{d.dA[0], d.dA[1], d.dA[2]}},
                                                        P3{{d.bpos[0], d.bpos[1], d.bpos[2]}}, d.ssc, d.parent,
                                                        P3{{d.x[0], d.x[1], d.x[2]}}, d.mt, d.bslot, d.sc, d.gvhat, acc);
    }
    if (c->np > 0) {
        W9 A, F;
        for (int q = 0; q < 9; ++q) {
            A.a[q] = d.A[q];
            F.a[q] = d.F[q];
        }
        MPM_LAUNCH k_g2p_final<<<nblk(c->np, 256), 256, 0, st>>>((int)c->np, W3{{d.x[0], d.x[1], d.x[2]}},
                                                      W3{{d.v[0], d.v[1], d.v[2]}}, A, d.m, d.psc, d.sc, acc, d.phase,
                                                      d.J, F, d.T);
    }
    return cudaGetLastError();
}

}  // namespace mpm
