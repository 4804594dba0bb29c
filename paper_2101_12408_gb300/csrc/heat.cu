// Implicit heat solve with the particle-based Robin boundary term.
//
// Paper section "Temperature Update": with the thermal mass m^T_i of the
// temperature P2G as the mass matrix,
//   (c_p m^T/dt) T + sum_p K V^n_p gradN_i . grad T(x_p) + sum_r h |dA_r| w_ri T(s_r)
//     = (c_p m^T/dt) T^n + sum_r w_ri (h Tbar_r + b_r) |dA_r| + sum_p N_i(x_p) H V^n_p,
// unknowns: nodes with m^T > 0. Readings: the surface weights w_ri are the
// sample's B-spline weights restricted to the unknowns and renormalised (so the
// operator is symmetric and the whole boundary flux reaches the unknowns); the
// printed source term's stray h is dropped. Solved by Jacobi-preconditioned CG
// for the correction from the initial guess T^n.
#include "ctx.h"

namespace mpm {

cudaError_t launch_cg(mpm_ctx* c, int heat);

namespace {

constexpr int NT = 128;

template <typename R>
struct HeatArgs {
    const int *work, *work_gb, *nbr, *cell_start, *scell_start;
    const int4* coord;
    const SceneDev* sc;
    const SceneScal* scal;
    const R* T;
    R* out;
    const R* hinvd;
    const R *pu0, *pu1, *pu2, *Vn;
    const R *su0, *su1, *su2, *sa0, *sa1, *sa2, *swn;
    int check_done;
};

template <typename R>
__device__ __forceinline__ void load_halo_scalar(const int* __restrict__ nbr, int slot, const R* __restrict__ f, R* sh,
                                                 const R* __restrict__ inv, uint8_t* unk) {
    for (int h = threadIdx.x; h < HN; h += blockDim.x) {
        int ns, loc;
        halo_source(nbr, slot, h, ns, loc);
        sh[h] = ns < 0 ? R(0) : f[ns * 64 + loc];
        if (unk) unk[h] = (ns >= 0 && inv[ns * 64 + loc] != R(0)) ? 1 : 0;
    }
}

template <typename R>
__global__ void __launch_bounds__(NT) k_heat_apply(HeatArgs<R> a) {
    __shared__ R Th[HN];
    __shared__ R acc[HN];
    __shared__ uint8_t unk[HN];
    int w = blockIdx.x;
    int slot = a.work[w];
    long long gb = a.work_gb[w];
    int4 bc = a.coord[slot];
    const SceneDev& S = a.sc[bc.w];
    if (!S.thermal) return;
    if (a.check_done && a.scal[bc.w].cg_done) return;
    load_halo_scalar<R>(a.nbr, slot, a.T, Th, a.hinvd, unk);
    for (int h = threadIdx.x; h < HN; h += NT) acc[h] = R(0);
    __syncthreads();
    const R inv_dx = (R)S.inv_dx;
    const R Kc = (R)S.K;
    int beg = a.cell_start[gb * 64], end = a.cell_start[gb * 64 + 64];
    for (int i = beg + threadIdx.x; i < end; i += NT) {
        int lc[3];
        R wgt[3][3], dw[3][3];
        make_stencil_local<R>(a.pu0[i], a.pu1[i], a.pu2[i], inv_dx, lc, wgt, dw);
        R g[3] = {0, 0, 0};
        for (int cz = 0; cz < 3; ++cz)
            for (int cy = 0; cy < 3; ++cy)
                for (int cx = 0; cx < 3; ++cx) {
                    R t = Th[halo_index(lc[0] + cx, lc[1] + cy, lc[2] + cz)];
                    g[0] += t * dw[0][cx] * wgt[1][cy] * wgt[2][cz];
                    g[1] += t * wgt[0][cx] * dw[1][cy] * wgt[2][cz];
                    g[2] += t * wgt[0][cx] * wgt[1][cy] * dw[2][cz];
                }
        R cK = Kc * a.Vn[i];
        g[0] *= cK;
        g[1] *= cK;
        g[2] *= cK;
        for (int cz = 0; cz < 3; ++cz)
            for (int cy = 0; cy < 3; ++cy)
                for (int cx = 0; cx < 3; ++cx)
                    atomicAdd(&acc[halo_index(lc[0] + cx, lc[1] + cy, lc[2] + cz)],
                              g[0] * dw[0][cx] * wgt[1][cy] * wgt[2][cz] + g[1] * wgt[0][cx] * dw[1][cy] * wgt[2][cz] +
                                  g[2] * wgt[0][cx] * wgt[1][cy] * dw[2][cz]);
    }
    int sbeg = a.scell_start[gb * 64], send = a.scell_start[gb * 64 + 64];
    const R hc = (R)S.h;
    for (int j = sbeg + threadIdx.x; j < send; j += NT) {
        R wn = a.swn[j];
        if (wn == R(0)) continue;
        int lc[3];
        R wgt[3][3], dw[3][3];
        make_stencil_local<R>(a.su0[j], a.su1[j], a.su2[j], inv_dx, lc, wgt, dw);
        R ts = 0;
        for (int cz = 0; cz < 3; ++cz)
            for (int cy = 0; cy < 3; ++cy)
                for (int cx = 0; cx < 3; ++cx) {
                    int h = halo_index(lc[0] + cx, lc[1] + cy, lc[2] + cz);
                    if (unk[h]) ts += Th[h] * wgt[0][cx] * wgt[1][cy] * wgt[2][cz];
                }
        R area = sqrt(a.sa0[j] * a.sa0[j] + a.sa1[j] * a.sa1[j] + a.sa2[j] * a.sa2[j]);
        R coef = hc * area * ts * wn * wn;
        for (int cz = 0; cz < 3; ++cz)
            for (int cy = 0; cy < 3; ++cy)
                for (int cx = 0; cx < 3; ++cx) {
                    int h = halo_index(lc[0] + cx, lc[1] + cy, lc[2] + cz);
                    if (unk[h]) atomicAdd(&acc[h], coef * wgt[0][cx] * wgt[1][cy] * wgt[2][cz]);
                }
    }
    __syncthreads();
    for (int h = threadIdx.x; h < HN; h += NT) {
        R val = acc[h];
        if (val == R(0)) continue;
        int ns, loc;
        halo_source(a.nbr, slot, h, ns, loc);
        if (ns >= 0) atomicAdd(&a.out[ns * 64 + loc], val);
    }
}

// right-hand side terms beyond the mass term, float64
struct RhsArgs {
    const int *work, *work_gb, *nbr, *cell_start, *scell_start;
    const int4* coord;
    const SceneDev* sc;
    const double *x0, *x1, *x2, *V0, *J, *F0, *F4, *F8, *F1, *F2, *F3, *F5, *F6, *F7;
    const uint8_t* phase;
    const double *s0, *s1, *s2, *dA0, *dA1, *dA2, *bheat, *Tbar;
    const double* gmT;
    double* rhs;
};

__global__ void __launch_bounds__(NT) k_heat_rhs(RhsArgs a) {
    __shared__ double acc[HN];
    __shared__ uint8_t unk[HN];
    int w = blockIdx.x;
    int slot = a.work[w];
    long long gb = a.work_gb[w];
    int4 bc = a.coord[slot];
    const SceneDev& S = a.sc[bc.w];
    if (!S.thermal) return;
    for (int h = threadIdx.x; h < HN; h += NT) {
        acc[h] = 0.0;
        int ns, loc;
        halo_source(a.nbr, slot, h, ns, loc);
        unk[h] = (ns >= 0 && a.gmT[ns * 64 + loc] > 0.0) ? 1 : 0;
    }
    __syncthreads();
    int ob[3] = {bc.x * BS, bc.y * BS, bc.z * BS};
    if (S.H != 0.0) {
        int beg = a.cell_start[gb * 64], end = a.cell_start[gb * 64 + 64];
        for (int i = beg + threadIdx.x; i < end; i += NT) {
            double u[3] = {(a.x0[i] - S.origin[0]) * S.inv_dx, (a.x1[i] - S.origin[1]) * S.inv_dx,
                           (a.x2[i] - S.origin[2]) * S.inv_dx};
            Stencil<double> st;
            make_stencil<double>(u, S.inv_dx, st);
            double Fd[9] = {a.F0[i], a.F1[i], a.F2[i], a.F3[i], a.F4[i], a.F5[i], a.F6[i], a.F7[i], a.F8[i]};
            double Vn = (a.phase[i] == 0 ? a.J[i] : det3<double>(Fd)) * a.V0[i];
            double c = S.H * Vn;
            for (int cz = 0; cz < 3; ++cz)
                for (int cy = 0; cy < 3; ++cy)
                    for (int cx = 0; cx < 3; ++cx)
                        atomicAdd(&acc[halo_index(st.c[0] - ob[0] + cx, st.c[1] - ob[1] + cy, st.c[2] - ob[2] + cz)],
                                  c * st.w[0][cx] * st.w[1][cy] * st.w[2][cz]);
        }
    }
    int sbeg = a.scell_start[gb * 64], send = a.scell_start[gb * 64 + 64];
    for (int j = sbeg + threadIdx.x; j < send; j += NT) {
        double u[3] = {(a.s0[j] - S.origin[0]) * S.inv_dx, (a.s1[j] - S.origin[1]) * S.inv_dx,
                       (a.s2[j] - S.origin[2]) * S.inv_dx};
        Stencil<double> st;
        make_stencil<double>(u, S.inv_dx, st);
        double wsum = 0.0;
        for (int cz = 0; cz < 3; ++cz)
            for (int cy = 0; cy < 3; ++cy)
                for (int cx = 0; cx < 3; ++cx)
                    if (unk[halo_index(st.c[0] - ob[0] + cx, st.c[1] - ob[1] + cy, st.c[2] - ob[2] + cz)])
                        wsum += st.w[0][cx] * st.w[1][cy] * st.w[2][cz];
        if (!(wsum > 0.0)) continue;
        double area = sqrt(a.dA0[j] * a.dA0[j] + a.dA1[j] * a.dA1[j] + a.dA2[j] * a.dA2[j]);
        double c = (S.h * a.Tbar[j] + a.bheat[j]) * area / wsum;
        for (int cz = 0; cz < 3; ++cz)
            for (int cy = 0; cy < 3; ++cy)
                for (int cx = 0; cx < 3; ++cx) {
                    int h = halo_index(st.c[0] - ob[0] + cx, st.c[1] - ob[1] + cy, st.c[2] - ob[2] + cz);
                    if (unk[h]) atomicAdd(&acc[h], c * st.w[0][cx] * st.w[1][cy] * st.w[2][cz]);
                }
    }
    __syncthreads();
    for (int h = threadIdx.x; h < HN; h += NT) {
        double val = acc[h];
        if (val == 0.0) continue;
        int ns, loc;
        halo_source(a.nbr, slot, h, ns, loc);
        if (ns >= 0) atomicAdd(&a.rhs[ns * 64 + loc], val);
    }
}

// T (R) = T^n on unknowns, u = 0
template <typename R>
__global__ void k_heat_prep(int nb, const double* __restrict__ gTn, const R* __restrict__ hinvd, R* __restrict__ T,
                            R* __restrict__ u) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nb * 64) return;
    T[t] = hinvd[t] != R(0) ? (R)gTn[t] : R(0);
    u[t] = R(0);
}

// CG right-hand side b = rhs_terms - stiff(T^n); |full rhs|^2 for the tolerance
template <typename R>
__global__ void k_heat_b(const int4* __restrict__ coord, const SceneDev* __restrict__ sc, SceneScal* __restrict__ scal,
                         const double* __restrict__ gmT, const double* __restrict__ gTn, const R* __restrict__ stiff,
                         double* __restrict__ rhs) {
    int slot = blockIdx.x, l = threadIdx.x;
    int t = slot * 64 + l;
    int4 bc = coord[slot];
    const SceneDev& S = sc[bc.w];
    double bb = 0.0;
    if (S.thermal && gmT[t] > 0.0) {
        double full = S.cp * gmT[t] / S.dt * gTn[t] + rhs[t];
        bb = full * full;
        rhs[t] = rhs[t] - (double)stiff[t];
    } else {
        rhs[t] = 0.0;
    }
    bb = warp_sum(bb);
    if ((l & 31) == 0 && bb != 0.0) atomicAdd(&scal[bc.w].bnorm, bb);
}

template <typename R>
__global__ void k_heat_finish(int nb, const int4* __restrict__ coord, const SceneDev* __restrict__ sc,
                              const double* __restrict__ gTn, const R* __restrict__ hinvd, const R* __restrict__ x,
                              double* __restrict__ That) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nb * 64) return;
    const SceneDev& S = sc[coord[t >> 6].w];
    That[t] = (S.thermal && hinvd[t] != R(0)) ? gTn[t] + (double)x[t] : 0.0;
}

__global__ void k_heat_begin(SceneScal* scal, const SceneDev* sc, int nsc) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nsc) return;
    SceneScal& c = scal[s];
    c.cg_done = sc[s].thermal ? 0 : 1;
    c.cg_it = 0;
    c.rz = c.rz_new = c.rr = c.pAp = c.bnorm = 0.0;
}

__global__ void k_heat_end(SceneScal* scal, int nsc) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nsc) return;
    scal[s].heat_it = scal[s].cg_it;
}

// full operator for the C ABI: out = P (diag T + stiff)
template <typename R>
__global__ void k_heat_diag(int nb, const R* __restrict__ hinvd, const R* __restrict__ T, R* __restrict__ out) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nb * 64) return;
    R inv = hinvd[t];
    out[t] = inv != R(0) ? T[t] / inv + out[t] : R(0);
}

inline unsigned nblk(long long n, int nt) { return (unsigned)((n + nt - 1) / nt); }

template <typename R>
cudaError_t heat_apply_t(mpm_ctx* c, const void* T, void* out, int check_done) {
    if (c->NW == 0) return cudaSuccess;
    Dev& d = c->d;
    HeatArgs<R> a;
    a.work = d.work;
    a.work_gb = d.work_gb;
    a.nbr = d.nbr;
    a.cell_start = d.cell_start;
    a.scell_start = d.scell_start;
    a.coord = d.slot_coord;
    a.sc = d.sc;
    a.scal = d.scal;
    a.T = (const R*)T;
    a.out = (R*)out;
    a.hinvd = (const R*)d.hinvd;
    a.pu0 = (const R*)d.pu[0];
    a.pu1 = (const R*)d.pu[1];
    a.pu2 = (const R*)d.pu[2];
    a.Vn = (const R*)d.Vn;
    a.su0 = (const R*)d.su[0];
    a.su1 = (const R*)d.su[1];
    a.su2 = (const R*)d.su[2];
    a.sa0 = (const R*)d.sa[0];
    a.sa1 = (const R*)d.sa[1];
    a.sa2 = (const R*)d.sa[2];
    a.swn = (const R*)d.swn;
    a.check_done = check_done;
    MPM_LAUNCH k_heat_apply<R><<<c->NW, NT, 0, c->st>>>(a);
    return cudaGetLastError();
}

template <typename R>
cudaError_t run_heat_t(mpm_ctx* c) {
    Dev& d = c->d;
    cudaStream_t st = c->st;
    int nb = c->NB;
    unsigned g = nblk((long long)nb * 64, 256);
    MPM_LAUNCH k_heat_begin<<<nblk(c->nsc, 128), 128, 0, st>>>(d.scal, d.sc, c->nsc);
    MPM_LAUNCH k_heat_prep<R><<<g, 256, 0, st>>>(nb, d.gTn, (const R*)d.hinvd, (R*)d.hT, (R*)d.hu);
    heat_apply_t<R>(c, d.hT, d.hu, 0);
    cudaMemsetAsync(d.hrhs, 0, sizeof(double) * (size_t)nb * 64, st);
    if (c->NW > 0) {
        RhsArgs a;
        a.work = d.work;
        a.work_gb = d.work_gb;
        a.nbr = d.nbr;
        a.cell_start = d.cell_start;
        a.scell_start = d.scell_start;
        a.coord = d.slot_coord;
        a.sc = d.sc;
        a.x0 = d.x[0];
        a.x1 = d.x[1];
        a.x2 = d.x[2];
        a.V0 = d.V0;
        a.J = d.J;
        a.F0 = d.F[0]; a.F1 = d.F[1]; a.F2 = d.F[2]; a.F3 = d.F[3]; a.F4 = d.F[4];
        a.F5 = d.F[5]; a.F6 = d.F[6]; a.F7 = d.F[7]; a.F8 = d.F[8];
        a.phase = d.phase;
        a.s0 = d.s[0];
        a.s1 = d.s[1];
        a.s2 = d.s[2];
        a.dA0 = d.dA[0];
        a.dA1 = d.dA[1];
        a.dA2 = d.dA[2];
        a.bheat = d.bheat;
        a.Tbar = d.Tbar;
        a.gmT = d.gmT;
        a.rhs = d.hrhs;
        MPM_LAUNCH k_heat_rhs<<<c->NW, NT, 0, st>>>(a);
    }
    MPM_LAUNCH k_heat_b<R><<<nb, 64, 0, st>>>(d.slot_coord, d.sc, d.scal, d.gmT, d.gTn, (const R*)d.hu, d.hrhs);
    cudaError_t e = launch_cg(c, 1);
    if (e != cudaSuccess) return e;
    MPM_LAUNCH k_heat_finish<R><<<g, 256, 0, st>>>(nb, d.slot_coord, d.sc, d.gTn, (const R*)d.hinvd, (const R*)d.hx, d.gThat);
    MPM_LAUNCH k_heat_end<<<nblk(c->nsc, 128), 128, 0, st>>>(d.scal, c->nsc);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_heat_apply(mpm_ctx* c, const void* T, void* out) {
    if (c->rsize == 4) return heat_apply_t<float>(c, T, out, 1);
    return heat_apply_t<double>(c, T, out, 1);
}

cudaError_t launch_heat_full(mpm_ctx* c, const void* T, void* out) {
    // out must be zeroed by the caller
    unsigned g = nblk((long long)c->NB * 64, 256);
    if (c->rsize == 4) {
        heat_apply_t<float>(c, T, out, 0);
        MPM_LAUNCH k_heat_diag<float><<<g, 256, 0, c->st>>>(c->NB, (const float*)c->d.hinvd, (const float*)T, (float*)out);
    } else {
        heat_apply_t<double>(c, T, out, 0);
        MPM_LAUNCH k_heat_diag<double><<<g, 256, 0, c->st>>>(c->NB, (const double*)c->d.hinvd, (const double*)T, (double*)out);
    }
    return cudaGetLastError();
}

cudaError_t run_heat(mpm_ctx* c) {
    if (c->NB == 0) return cudaSuccess;
    bool any = false;
    for (auto& S : c->hsc) any = any || S.thermal;
    if (!any) return cudaSuccess;
    if (c->rsize == 4) return run_heat_t<float>(c);
    return run_heat_t<double>(c);
}

}  // namespace mpm
