// Backward-Euler momentum solve: objective / gradient, Hessian-vector operator,
// Jacobi-preconditioned CG, one-pass Armijo line search, Newton control.
//
// Paper section "Momentum Update" (Eq. disc_force, the discrete energy e(y),
// Eq. fe). With y = x + dt v the backward-Euler equations are the stationarity
// conditions of
//   Phi(v) = sum_i m_i/2 |v_i - v^n_i|^2 - dt sum_i m_i g.v_i + e(x + dt v)
//            + dt mu/2 sum_p V^n_p |sym L_p|^2,     L_p = sum_i v_i gradN_i(x_p)^T,
// liquid J_p = (1 + dt tr L_p) J^n_p, solid F_p = (I + dt L_p) F^n_p, surface
// F^_r = I + dt L(s_r) with energy k_r |cof(F^_r) dA_r|.
// Hessian-vector (the linearisation the paper refers to earlier work for):
//   liquid  dt^2 lambda (J^n)^2 V^0 gradN_i tr(dL)    viscous  dt mu V^n sym(dL) gradN_i
//   solid   dt^2 V^0 dP(F; dL F^n) F^nT gradN_i
//   surface dt^2 dG gradN_i(s_r), dG = -k [dn]x F^ [a]x  (+ -k [n]x dF^ [a]x exact),
//           dn = (I - n n^T) dc/|c|, dc = dcof(F^)[dF^] a, with G = -k [n]x F^ [a]x the
//           gradient of k |cof(F^) a|. The projected mode (the definiteness fix) keeps the
//           Gauss-Newton term and the positive, conformal part of the cofactor curvature
//           n . cof(dF^) a (which has eigenvalues +-|a|), so it is PSD and still stiff
//           against in-plane dilation of the surface.
#include "ctx.h"
#include "polar.cuh"

namespace mpm {

namespace {

constexpr int NT = 128;

struct Ptrs3 { const double* a[3]; };
struct Ptrs9 { const double* a[9]; };
template <typename R> struct RPtr3 { R* a[3]; };
template <typename R> struct RPtr9 { R* a[9]; };
template <typename R> struct RPtr24 { R* a[24]; };
template <typename R> struct RPtr45 { R* a[45]; };

// packed index of the symmetric 9x9 entry (m, l), m <= l
__host__ __device__ constexpr int sym9(int m, int l) { return m * 9 - m * (m - 1) / 2 + (l - m); }

template <typename R>
__device__ __forceinline__ void cross_mat(const R* a, R* M) {
    M[0] = 0; M[1] = -a[2]; M[2] = a[1];
    M[3] = a[2]; M[4] = 0; M[5] = -a[0];
    M[6] = -a[1]; M[7] = a[0]; M[8] = 0;
}

// G = -k [n]x F [a]x
template <typename R>
__device__ __forceinline__ void surf_G(R k, const R* n, const R* F, const R* a, R* G) {
    R An[9], Aa[9], T1[9];
    cross_mat<R>(a, Aa);
    cross_mat<R>(n, An);
    matmul3<R>(F, Aa, T1);
    matmul3<R>(An, T1, G);
#pragma unroll
    for (int q = 0; q < 9; ++q) G[q] *= -k;
}

// unit t1, t2 with (t1, t2, u) right-handed
template <typename R>
__device__ __forceinline__ void tangent_frame(const R* u, R* t1, R* t2) {
    R ax = fabs(u[0]), ay = fabs(u[1]), az = fabs(u[2]);
    int k = ax <= ay ? (ax <= az ? 0 : 2) : (ay <= az ? 1 : 2);
    R e[3] = {R(0), R(0), R(0)};
    e[k] = R(1);
    R d = u[k];
    R t[3] = {e[0] - d * u[0], e[1] - d * u[1], e[2] - d * u[2]};
    R inv = R(1) / sqrt(t[0] * t[0] + t[1] * t[1] + t[2] * t[2]);
    t1[0] = t[0] * inv;
    t1[1] = t[1] * inv;
    t1[2] = t[2] * inv;
    t2[0] = u[1] * t1[2] - u[2] * t1[1];
    t2[1] = u[2] * t1[0] - u[0] * t1[2];
    t2[2] = u[0] * t1[1] - u[1] * t1[0];
}

// Positive (conformal) part of the cofactor curvature n . cof(X) a, added to G:
// with x_ij = t_i . X s_j in frames (t1, t2, n), (s1, s2, a/|a|),
// G += k |a|/2 [(x11 + x22)(t1 s1^T + t2 s2^T) + (x12 - x21)(t1 s2^T - t2 s1^T)].
template <typename R>
__device__ __forceinline__ void add_conformal(R k, const R* n, const R* a, const R* X, R* G) {
    R an = sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
    R ah[3] = {a[0] / an, a[1] / an, a[2] / an};
    R t1[3], t2[3], s1[3], s2[3];
    tangent_frame<R>(n, t1, t2);
    tangent_frame<R>(ah, s1, s2);
    R Xs1[3], Xs2[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        Xs1[i] = X[3 * i] * s1[0] + X[3 * i + 1] * s1[1] + X[3 * i + 2] * s1[2];
        Xs2[i] = X[3 * i] * s2[0] + X[3 * i + 1] * s2[1] + X[3 * i + 2] * s2[2];
    }
    R x11 = t1[0] * Xs1[0] + t1[1] * Xs1[1] + t1[2] * Xs1[2];
    R x22 = t2[0] * Xs2[0] + t2[1] * Xs2[1] + t2[2] * Xs2[2];
    R x12 = t1[0] * Xs2[0] + t1[1] * Xs2[1] + t1[2] * Xs2[2];
    R x21 = t2[0] * Xs1[0] + t2[1] * Xs1[1] + t2[2] * Xs1[2];
    R p = R(0.5) * k * an * (x11 + x22);
    R q = R(0.5) * k * an * (x12 - x21);
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j)
            G[3 * i + j] += p * (t1[i] * s1[j] + t2[i] * s2[j]) + q * (t1[i] * s2[j] - t2[i] * s1[j]);
}

template <typename R>
__device__ __forceinline__ void load_halo_vec_d(const int* __restrict__ nbr, int slot, const double* __restrict__ vec, R (*sh)[HN]) {
    // The halo is stored relative to the velocity of the block's first node,
    // subtracted in float64: velocity gradients sum_i v_i gradN_i^T are unchanged
    // (sum_i gradN_i = 0), but a common translation no longer cancels in R.
    for (int t = threadIdx.x; t < 3 * HN; t += blockDim.x) {
        int c = t / HN, h = t % HN;
        int ns, loc;
        halo_source(nbr, slot, h, ns, loc);
        double ref = vec[slot * 192 + c * 64];
        sh[c][h] = ns < 0 ? R(0) : (R)(vec[ns * 192 + c * 64 + loc] - ref);
    }
}

template <typename A>
__device__ __forceinline__ void flush_halo_vec(const int* __restrict__ nbr, int slot, A (*sh)[HN], A* __restrict__ vec) {
    for (int t = threadIdx.x; t < 3 * HN; t += blockDim.x) {
        int c = t / HN, h = t % HN;
        A val = sh[c][h];
        if (val == A(0)) continue;
        int ns, loc;
        halo_source(nbr, slot, h, ns, loc);
        if (ns >= 0) atomicAdd(&vec[ns * 192 + c * 64 + loc], val);
    }
}

// local stencil of a point: cell relative to the block origin, weights, gradients
template <typename R>
__device__ __forceinline__ void stencil_in_block(const double* p, const SceneDev& S, int4 bc, int lc[3], R w[3][3], R dw[3][3], R f[3]) {
    int ob[3] = {bc.x * BS, bc.y * BS, bc.z * BS};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        double u = (p[a] - S.origin[a]) * S.inv_dx;
        double fl = floor(u);
        lc[a] = (int)fl - ob[a];
        f[a] = (R)(u - 0.5 - (fl - 1.0));
        bspline<R>(f[a], w[a], dw[a]);
#pragma unroll
        for (int k = 0; k < 3; ++k) dw[a][k] *= (R)S.inv_dx;
    }
}

// ======================================================================
// per-step packs for the operator (constant over the Newton iterations)
// ======================================================================
template <typename R>
__global__ void k_pack_volume(int np, Ptrs3 x, const double* __restrict__ J, Ptrs9 F, const double* __restrict__ V0,
                              const double* __restrict__ T, const uint8_t* __restrict__ phase, const int* __restrict__ psc,
                              const SceneDev* __restrict__ sc, RPtr3<R> pu, R* __restrict__ kappa, R* __restrict__ cvisc,
                              RPtr9<R> Fn, R* __restrict__ lmu, R* __restrict__ llam, R* __restrict__ Vn,
                              const int* __restrict__ bslot, int* __restrict__ slot_gen,
                              const int* __restrict__ cell_start, int nw, const int* __restrict__ bw,
                              const int* __restrict__ wrows, const int* __restrict__ wroff, long long opk_cap,
                              R4<R>* __restrict__ opk) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= np) return;
    const SceneDev& S = sc[psc[i]];
    long long rec_at = -1;   // rank-major record slot of this particle
    {
        int c[3];
        for (int a = 0; a < 3; ++a) c[a] = (int)floor((x.a[a][i] - S.origin[a]) * S.inv_dx);
        bool general = phase[i] != 0 || S.mu_l != 0.0;
        long long gb = S.block_base + (c[0] >> 2) + (long long)S.nb[0] * ((c[1] >> 2) + (long long)S.nb[1] * (c[2] >> 2));
        if (general) atomicAdd(&slot_gen[bslot[gb]], 1);
        int lc = (c[0] & 3) + 4 * (c[1] & 3) + 16 * (c[2] & 3);
        int w = bw[gb];
        int k = i - cell_start[gb * 64 + lc];
        if (w >= 0 && w < nw && k >= 0 && k < wrows[w]) {
            long long at = ((long long)wroff[w] + k) * 64 + lc;
            if (at < opk_cap) rec_at = at;
        }
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        double u = (x.a[a][i] - S.origin[a]) * S.inv_dx;
        int c = (int)floor(u);
        pu.a[a][i] = (R)(u - (double)((c >> 2) * BS));
    }
    double dt = S.dt;
    double Jn = J[i], v0 = V0[i];
    bool liq = phase[i] == 0;
    double Fd[9];
    for (int q = 0; q < 9; ++q) Fd[q] = F.a[q][i];
    double detF = det3<double>(Fd);
    Vn[i] = (R)((liq ? Jn : detF) * v0);
    kappa[i] = liq ? (R)(dt * dt * S.lambda_l * Jn * Jn * v0) : R(0);
    cvisc[i] = liq ? (R)(dt * S.mu_l * Jn * v0) : R(0);
    {
        R4<R> rec;
        rec.x = pu.a[0][i];
        rec.y = pu.a[1][i];
        rec.z = pu.a[2][i];
        bool general = !liq || S.mu_l != 0.0;
        rec.w = general ? R(-1) : (R)(dt * dt * S.lambda_l * Jn * Jn * v0);
        if (rec_at >= 0) {
            // pair-interleaved row: cells 2l, 2l+1 as x_A x_B y_A y_B z_A z_B kappa_A kappa_B
            const int lc = (int)(rec_at & 63);
            R* row = reinterpret_cast<R*>(opk + (rec_at - lc)) + 8 * (lc >> 1) + (lc & 1);
            row[0] = rec.x;
            row[2] = rec.y;
            row[4] = rec.z;
            row[6] = rec.w;
        }
    }
    if (!liq) {
        for (int q = 0; q < 9; ++q) Fn.a[q][i] = (R)Fd[q];
        double mu_h, lam_h;
        solid_lame(S, T[i], mu_h, lam_h);
        lmu[i] = (R)mu_h;
        llam[i] = (R)lam_h;
    }
}

template <typename R>
__global__ void k_pack_surface(int ns, Ptrs3 s, Ptrs3 dA, const double* __restrict__ gamma, const int* __restrict__ ssc,
                               const SceneDev* __restrict__ sc, RPtr3<R> su, RPtr3<R> sa, R* __restrict__ sg) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= ns) return;
    const SceneDev& S = sc[ssc[j]];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        double u = (s.a[a][j] - S.origin[a]) * S.inv_dx;
        int c = (int)floor(u);
        su.a[a][j] = (R)(u - (double)((c >> 2) * BS));
        sa.a[a][j] = (R)dA.a[a][j];
    }
    sg[j] = (R)gamma[j];
}

// ======================================================================
// objective + gradient (+ per-iterate caches) at the Newton iterate
// ======================================================================
template <typename R>
struct EvalArgs {
    const int *work, *work_gb, *nbr, *cell_start, *scell_start;
    const int4* coord;
    const SceneDev* sc;
    SceneScal* scal;
    const double* gv;          // iterate (double grid)
    double* grad;              // gradient accumulator (double grid)
    Ptrs3 x;
    const double *J, *V0, *T;
    Ptrs9 F;
    const uint8_t* phase;
    Ptrs3 s, dA;
    const double* gamma;
    int want_grad, want_cache, skip_done;
    int skip_poly;             // non-viscous liquid particles are left to k_eval_cell
    int skip_samples;          // surface samples are left to k_eval_surf
    const int* slot_gen;
    RPtr24<R> scache;          // solid: F (9), R (9), Kinv (6)
    RPtr9<R> sF;               // surface F^
    RPtr3<R> sn;               // surface unit c
    R* sic;                    // 1/|c|
};

// R: arithmetic type; RS: storage type of the per-iterate caches
template <typename R, typename RS>
__global__ void __launch_bounds__(NT) k_eval(EvalArgs<RS> a) {
    __shared__ R vh[3][HN];
    __shared__ double ga[3][HN];
    __shared__ double red[NT / 32];
    int w = blockIdx.x;
    int slot = a.work[w];
    long long gb = a.work_gb[w];
    int4 bc = a.coord[slot];
    const SceneDev& S = a.sc[bc.w];
    if (a.skip_done && a.scal[bc.w].newton_done) return;
    const bool poly = a.skip_poly && S.mu_l == 0.0;
    const bool no_samples = a.skip_samples || a.scell_start[gb * 64] == a.scell_start[gb * 64 + 64];
    if (poly && a.slot_gen[slot] == 0 && no_samples) return;
    load_halo_vec_d<R>(a.nbr, slot, a.gv, vh);
    for (int t = threadIdx.x; t < 3 * HN; t += NT) (&ga[0][0])[t] = 0.0;
    __syncthreads();
    const R dt = (R)S.dt;
    double esum = 0.0;
    int beg = a.cell_start[gb * 64], end = a.cell_start[gb * 64 + 64];
    if (poly && a.slot_gen[slot] == 0) end = beg;
    for (int i = beg + threadIdx.x; i < end; i += NT) {
        if (poly && a.phase[i] == 0) continue;   // k_eval_cell
        double p[3] = {a.x.a[0][i], a.x.a[1][i], a.x.a[2][i]};
        int lc[3];
        R wgt[3][3], dw[3][3], f[3];
        stencil_in_block<R>(p, S, bc, lc, wgt, dw, f);
        R L[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
        for (int cz = 0; cz < 3; ++cz)
            for (int cy = 0; cy < 3; ++cy)
                for (int cx = 0; cx < 3; ++cx) {
                    int h = halo_index(lc[0] + cx, lc[1] + cy, lc[2] + cz);
                    R dN[3] = {dw[0][cx] * wgt[1][cy] * wgt[2][cz], wgt[0][cx] * dw[1][cy] * wgt[2][cz],
                               wgt[0][cx] * wgt[1][cy] * dw[2][cz]};
#pragma unroll
                    for (int q = 0; q < 3; ++q) {
                        R vq = vh[q][h];
                        L[3 * q] += vq * dN[0];
                        L[3 * q + 1] += vq * dN[1];
                        L[3 * q + 2] += vq * dN[2];
                    }
                }
        R M[9];
        double v0 = a.V0[i];
        if (a.phase[i] == 0) {
            R Jn = (R)a.J[i];
            R jm1n = (R)(a.J[i] - 1.0);
            R trL = L[0] + L[4] + L[8];
            R jm1 = jm1n + dt * trL * (R(1) + jm1n);
            R lam = (R)S.lambda_l;
            esum += 0.5 * (double)lam * (double)jm1 * (double)jm1 * v0;
            R Vn = (R)(a.J[i] * v0);
            R mu = (R)S.mu_l;
            R eps[9];
#pragma unroll
            for (int q = 0; q < 3; ++q)
#pragma unroll
                for (int e = 0; e < 3; ++e) eps[3 * q + e] = R(0.5) * (L[3 * q + e] + L[3 * e + q]);
            R e2 = 0;
#pragma unroll
            for (int q = 0; q < 9; ++q) e2 += eps[q] * eps[q];
            esum += 0.5 * (double)dt * (double)mu * (double)Vn * (double)e2;
            R pr = dt * lam * jm1 * Jn * (R)v0;
            R cv = dt * mu * Vn;
#pragma unroll
            for (int q = 0; q < 9; ++q) M[q] = cv * eps[q] + ((q % 4 == 0) ? pr : R(0));
        } else {
            R Fo[9], A1[9], Fc[9];
#pragma unroll
            for (int q = 0; q < 9; ++q) {
                Fo[q] = (R)a.F.a[q][i];
                A1[q] = dt * L[q] + ((q % 4 == 0) ? R(1) : R(0));
            }
            matmul3<R>(A1, Fo, Fc);
            R Rm[9], K[6], sg[3];
            polar3<R>(Fc, Rm, K, sg);
            double Tn = a.T[i];
            double mu_h, lam_h;
            solid_lame(S, Tn, mu_h, lam_h);
            const R mu = (R)mu_h, lam = (R)lam_h;
            R J = det3<R>(Fc);
            esum += ((double)mu * ((double)(sg[0] - 1) * (sg[0] - 1) + (double)(sg[1] - 1) * (sg[1] - 1) +
                                   (double)(sg[2] - 1) * (sg[2] - 1)) +
                     0.5 * (double)lam * (double)(J - 1) * (double)(J - 1)) * v0;
            R C[9], P[9];
            cofactor<R>(Fc, C);
#pragma unroll
            for (int q = 0; q < 9; ++q) P[q] = R(2) * mu * (Fc[q] - Rm[q]) + lam * (J - 1) * C[q];
            matmul3_bt<R>(P, Fo, M);
            R sc = dt * (R)v0;
#pragma unroll
            for (int q = 0; q < 9; ++q) M[q] *= sc;
            if (a.want_cache) {
#pragma unroll
                for (int q = 0; q < 9; ++q) {
                    a.scache.a[q][i] = (RS)Fc[q];
                    a.scache.a[9 + q][i] = (RS)Rm[q];
                }
#pragma unroll
                for (int q = 0; q < 6; ++q) a.scache.a[18 + q][i] = (RS)K[q];
            }
        }
        if (a.want_grad) {
            for (int cz = 0; cz < 3; ++cz)
                for (int cy = 0; cy < 3; ++cy)
                    for (int cx = 0; cx < 3; ++cx) {
                        int h = halo_index(lc[0] + cx, lc[1] + cy, lc[2] + cz);
                        R dN[3] = {dw[0][cx] * wgt[1][cy] * wgt[2][cz], wgt[0][cx] * dw[1][cy] * wgt[2][cz],
                                   wgt[0][cx] * wgt[1][cy] * dw[2][cz]};
#pragma unroll
                        for (int q = 0; q < 3; ++q)
                            atomicAdd(&ga[q][h], (double)(M[3 * q] * dN[0] + M[3 * q + 1] * dN[1] + M[3 * q + 2] * dN[2]));
                    }
        }
    }
    int sbeg = a.scell_start[gb * 64], send = a.scell_start[gb * 64 + 64];
    if (a.skip_samples) send = sbeg;
    for (int j = sbeg + threadIdx.x; j < send; j += NT) {
        double p[3] = {a.s.a[0][j], a.s.a[1][j], a.s.a[2][j]};
        int lc[3];
        R wgt[3][3], dw[3][3], f[3];
        stencil_in_block<R>(p, S, bc, lc, wgt, dw, f);
        R Fh[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
        for (int cz = 0; cz < 3; ++cz)
            for (int cy = 0; cy < 3; ++cy)
                for (int cx = 0; cx < 3; ++cx) {
                    int h = halo_index(lc[0] + cx, lc[1] + cy, lc[2] + cz);
                    R dN[3] = {dw[0][cx] * wgt[1][cy] * wgt[2][cz], wgt[0][cx] * dw[1][cy] * wgt[2][cz],
                               wgt[0][cx] * wgt[1][cy] * dw[2][cz]};
#pragma unroll
                    for (int q = 0; q < 3; ++q) {
                        R vq = dt * vh[q][h];
                        Fh[3 * q] += vq * dN[0];
                        Fh[3 * q + 1] += vq * dN[1];
                        Fh[3 * q + 2] += vq * dN[2];
                    }
                }
        R av[3] = {(R)a.dA.a[0][j], (R)a.dA.a[1][j], (R)a.dA.a[2][j]};
        R C[9];
        cofactor<R>(Fh, C);
        R cv[3] = {C[0] * av[0] + C[1] * av[1] + C[2] * av[2], C[3] * av[0] + C[4] * av[1] + C[5] * av[2],
                   C[6] * av[0] + C[7] * av[1] + C[8] * av[2]};
        R cn = sqrt(cv[0] * cv[0] + cv[1] * cv[1] + cv[2] * cv[2]);
        R k = (R)a.gamma[j];
        esum += (double)k * (double)cn;
        R nv[3] = {cv[0] / cn, cv[1] / cn, cv[2] / cn};
        if (a.want_cache) {
#pragma unroll
            for (int q = 0; q < 9; ++q) a.sF.a[q][j] = (RS)Fh[q];
#pragma unroll
            for (int q = 0; q < 3; ++q) a.sn.a[q][j] = (RS)nv[q];
            a.sic[j] = (RS)(R(1) / cn);
        }
        if (a.want_grad) {
            R G[9];
            surf_G<R>(k * dt, nv, Fh, av, G);
            for (int cz = 0; cz < 3; ++cz)
                for (int cy = 0; cy < 3; ++cy)
                    for (int cx = 0; cx < 3; ++cx) {
                        int h = halo_index(lc[0] + cx, lc[1] + cy, lc[2] + cz);
                        R dN[3] = {dw[0][cx] * wgt[1][cy] * wgt[2][cz], wgt[0][cx] * dw[1][cy] * wgt[2][cz],
                                   wgt[0][cx] * wgt[1][cy] * dw[2][cz]};
#pragma unroll
                        for (int q = 0; q < 3; ++q)
                            atomicAdd(&ga[q][h], (double)(G[3 * q] * dN[0] + G[3 * q + 1] * dN[1] + G[3 * q + 2] * dN[2]));
                    }
        }
    }
    block_atomic_sum<NT>(esum, &a.scal[bc.w].phi_part, red);
    if (a.want_grad) {
        __syncthreads();
        flush_halo_vec<double>(a.nbr, slot, ga, a.grad);
    }
}

// node part of the gradient: m (v - v^n) - dt m g; |P grad|^2 and the kinetic energy
__device__ __forceinline__ void project3(double* v, uint8_t code, const SceneDev& S, int4 bc, int l) {
    if (code & PC_FIXED) {
        v[0] = v[1] = v[2] = 0.0;
        return;
    }
    if (code & PC_SLIPX) v[0] = 0.0;
    if (code & PC_SLIPY) v[1] = 0.0;
    if (code & PC_SLIPZ) v[2] = 0.0;
    if (code & PC_PLANE) {
        double d = v[0] * S.plane_n[0] + v[1] * S.plane_n[1] + v[2] * S.plane_n[2];
        for (int q = 0; q < 3; ++q) v[q] -= d * S.plane_n[q];
    }
    if (code & PC_SPHERE) {
        double x[3], n[3];
        node_position(S, bc, l, x);
        sphere_phi_normal(S, x, n);
        double d = v[0] * n[0] + v[1] * n[1] + v[2] * n[2];
        for (int q = 0; q < 3; ++q) v[q] -= d * n[q];
    }
}

template <typename R>
__device__ __forceinline__ void project3r(R* v, uint8_t code, const SceneDev& S, int4 bc, int l) {
    if (code & PC_FIXED) {
        v[0] = v[1] = v[2] = R(0);
        return;
    }
    if (code & PC_SLIPX) v[0] = R(0);
    if (code & PC_SLIPY) v[1] = R(0);
    if (code & PC_SLIPZ) v[2] = R(0);
    if (code & (PC_PLANE | PC_SPHERE)) {
        R n0, n1, n2;
        if (code & PC_SPHERE) {
            // the sphere's normal at the node, rounded to R
            double x[3], n[3];
            node_position(S, bc, l, x);
            sphere_phi_normal(S, x, n);
            n0 = (R)n[0];
            n1 = (R)n[1];
            n2 = (R)n[2];
        } else if constexpr (sizeof(R) == 4) {
            n0 = S.plane_nf[0];
            n1 = S.plane_nf[1];
            n2 = S.plane_nf[2];
        } else {
            n0 = (R)S.plane_n[0];
            n1 = (R)S.plane_n[1];
            n2 = (R)S.plane_n[2];
        }
        R d = v[0] * n0 + v[1] * n1 + v[2] * n2;
        v[0] -= d * n0;
        v[1] -= d * n1;
        v[2] -= d * n2;
    }
}

__global__ void k_node_grad(const int4* __restrict__ coord, const SceneDev* __restrict__ sc, SceneScal* __restrict__ scal,
                            const double* __restrict__ gm, const double* __restrict__ gvn, const double* __restrict__ gv,
                            const uint8_t* __restrict__ pcode, double* __restrict__ grad, int skip_done) {
    int slot = blockIdx.x, l = threadIdx.x;
    int4 bc = coord[slot];
    const SceneDev& S = sc[bc.w];
    if (skip_done && scal[bc.w].newton_done) return;
    int t = slot * 64 + l;
    double m = gm[t];
    double rr = 0.0, ek = 0.0;
    if (m > 0.0) {
        double gr[3];
        for (int q = 0; q < 3; ++q) {
            int k = slot * 192 + q * 64 + l;
            double v = gv[k], dv = v - gvn[k];
            gr[q] = grad[k] + m * dv - S.dt * m * S.g[q];
            grad[k] = gr[q];
            ek += 0.5 * m * dv * dv - S.dt * m * S.g[q] * v;
        }
        project3(gr, pcode[t], S, bc, l);
        rr = gr[0] * gr[0] + gr[1] * gr[1] + gr[2] * gr[2];
    }
    rr = warp_sum(rr);
    ek = warp_sum(ek);
    if ((l & 31) == 0) {
        // 2 warps per block
        atomicAdd(&scal[bc.w].rr, rr);
        atomicAdd(&scal[bc.w].phi_kin, ek);
    }
}

// ======================================================================
// Hessian-vector operator (the hot kernel): u += K p (stiffness part)
// ======================================================================
template <typename R>
struct ApplyArgs {
    const int *work, *work_gb, *nbr, *cell_start, *scell_start;
    const int4* coord;
    const SceneDev* sc;
    SceneScal* scal;
    const R* p;
    R* u;
    const uint8_t* phase;
    const double* V0;
    RPtr3<R> pu;
    const R *kappa, *cvisc;
    RPtr9<R> Fn;
    const R *lmu, *llam;
    RPtr24<R> scache;
    RPtr3<R> su, sa;
    const R* sg;
    RPtr9<R> sF;
    RPtr3<R> sn;
    const R* sic;
    const R* sKa;             // surface: per-sample records (SREC values: the projected-Hessian map, position)
    RPtr45<R> pK;             // solid: symmetric 9x9 map dL -> M of the projected Hessian (per iterate)
    int use_pK;
    int samples_in_cell;      // projected mode with current maps: k_apply_pair applies the samples
    const int* slot_gen;      // general particles per slot
    const R4<R>* opk;         // rank-major records: position in the block (cells), kappa (< 0: general)
    const int *wrows, *wroff; // per work block: record rows and their offset
    const int *gen_list, *gen_count;   // work blocks with samples or general particles
    int* err;
    int mode;
    int check_done;
    int pap;                  // 1: add p . (H - M) p of the launch to the scene's pAp (p the direction)
};

// ======================================================================
// Per-cell polynomial form of the liquid operator
//
// For a liquid particle without viscosity the operator is rank one,
// u_i += kappa_p tr(dL_p) gradN_i(x_p), and with the in-cell coordinate t in
// [0,1)^3 of the particle (x = (c + t) dx) every 1-D weight and derivative is a
// polynomial of degree <= 2:
//   w = (1/2 - t + t^2/2,  1/2 + t - t^2,  t^2/2),   dw/dt = (-1 + t, 1 - 2t, t).
// So tr(dL)(t) = sum_ijk C_ijk tx^i ty^j tz^k with 26 coefficients (no t^2 t^2 t^2
// term) fixed per cell by the 27 stencil values of p, and the cell's scatter is a
// fixed linear map of the 26 moments M_ijk = sum_p s_p tx^i ty^j tz^k. Each cell
// reads its 81 inputs and writes its 81 outputs once, whatever its particle count;
// per particle only 26 + 26 multiply-adds remain. The transforms below (wT, dT,
// wN, dN) are the 1-D pieces of those two maps; k_apply_pair applies them to two
// cells at once, k_eval_cell and k_curv_cell one cell per thread. Solids, viscous
// liquids and (exact-mode) surface samples take the general per-particle path.
// Shared layout x + 8 y + 52 z: the 32 cells of a warp hit 32 distinct banks.
// ======================================================================

// power coefficients -> from node values (out_k = sum_c v_c W[c][k]) and derivatives
template <typename R>
__device__ __forceinline__ void wT(R v0, R v1, R v2, R& o0, R& o1, R& o2) {
    o0 = R(0.5) * (v0 + v1);
    o1 = v1 - v0;
    o2 = R(0.5) * (v0 + v2) - v1;
}
template <typename R>
__device__ __forceinline__ void dT(R v0, R v1, R v2, R& o0, R& o1) {
    o0 = v1 - v0;
    o1 = v0 - R(2) * v1 + v2;
}
// moments -> node values (n_c = sum_k W[c][k] m_k, n_a = sum_i D[a][i] m_i)
template <typename R>
__device__ __forceinline__ void wN(R m0, R m1, R m2, R& n0, R& n1, R& n2) {
    n0 = R(0.5) * (m0 + m2) - m1;
    n1 = R(0.5) * m0 + m1 - m2;
    n2 = R(0.5) * m2;
}
template <typename R>
__device__ __forceinline__ void dN(R m0, R m1, R& n0, R& n1, R& n2) {
    n0 = m1 - m0;
    n1 = m0 - R(2) * m1;
    n2 = m1;
}

// C += coefficients of tr(dL) (without the 1/dx factor) for the cell at (lx, ly, lz)
template <typename R>
__device__ __forceinline__ void cell_coefficients(R (*ph)[PN], int lx, int ly, int lz, R C[3][3][3]) {
    R Q1[3][3][3], Q2[3][3][3];
    // x component: D along x, W along y and z
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b)
            wT<R>(ph[0][pidx(lx + a, ly + b, lz)], ph[0][pidx(lx + a, ly + b, lz + 1)], ph[0][pidx(lx + a, ly + b, lz + 2)],
                  Q1[a][b][0], Q1[a][b][1], Q1[a][b][2]);
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int k = 0; k < 3; ++k) wT<R>(Q1[a][0][k], Q1[a][1][k], Q1[a][2][k], Q2[a][0][k], Q2[a][1][k], Q2[a][2][k]);
#pragma unroll
    for (int j = 0; j < 3; ++j)
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            R g0, g1;
            dT<R>(Q2[0][j][k], Q2[1][j][k], Q2[2][j][k], g0, g1);
            C[0][j][k] += g0;
            C[1][j][k] += g1;
        }
    // y component: W along x, D along y, W along z
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b)
            wT<R>(ph[1][pidx(lx + a, ly + b, lz)], ph[1][pidx(lx + a, ly + b, lz + 1)], ph[1][pidx(lx + a, ly + b, lz + 2)],
                  Q1[a][b][0], Q1[a][b][1], Q1[a][b][2]);
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int k = 0; k < 3; ++k) dT<R>(Q1[a][0][k], Q1[a][1][k], Q1[a][2][k], Q2[a][0][k], Q2[a][1][k]);
#pragma unroll
    for (int j = 0; j < 2; ++j)
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            R g0, g1, g2;
            wT<R>(Q2[0][j][k], Q2[1][j][k], Q2[2][j][k], g0, g1, g2);
            C[0][j][k] += g0;
            C[1][j][k] += g1;
            C[2][j][k] += g2;
        }
    // z component: W along x and y, D along z
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b)
            dT<R>(ph[2][pidx(lx + a, ly + b, lz)], ph[2][pidx(lx + a, ly + b, lz + 1)], ph[2][pidx(lx + a, ly + b, lz + 2)],
                  Q1[a][b][0], Q1[a][b][1]);
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int k = 0; k < 2; ++k) wT<R>(Q1[a][0][k], Q1[a][1][k], Q1[a][2][k], Q2[a][0][k], Q2[a][1][k], Q2[a][2][k]);
#pragma unroll
    for (int j = 0; j < 3; ++j)
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            R g0, g1, g2;
            wT<R>(Q2[0][j][k], Q2[1][j][k], Q2[2][j][k], g0, g1, g2);
            C[0][j][k] += g0;
            C[1][j][k] += g1;
            C[2][j][k] += g2;
        }
}

// Separable stencil gather / scatter on the padded halo (one axis at a time):
// G_qe = sum_abc p_q(abc) dN_abc/dx_e, and u_q(abc) += sum_e M_qe dN_abc/dx_e.
template <typename R>
__device__ __forceinline__ void gather_grad_sep(R (*ph)[PN], const int* lc, const R (*w)[3], const R (*dw)[3], R* G) {
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        R gx = R(0), gy = R(0), gz = R(0);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            R u0 = R(0), u1 = R(0), u2 = R(0);
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                const R* row = &ph[q][pidx(lc[0] + a, lc[1] + b, lc[2])];
                R p0 = row[0], p1 = row[PZ], p2 = row[2 * PZ];
                R s0 = w[2][0] * p0 + w[2][1] * p1 + w[2][2] * p2;
                R s1 = dw[2][0] * p0 + dw[2][1] * p1 + dw[2][2] * p2;
                u0 += w[1][b] * s0;
                u1 += dw[1][b] * s0;
                u2 += w[1][b] * s1;
            }
            gx += dw[0][a] * u0;
            gy += w[0][a] * u1;
            gz += w[0][a] * u2;
        }
        G[3 * q] = gx;
        G[3 * q + 1] = gy;
        G[3 * q + 2] = gz;
    }
}

// one component q of the two above: row q of the gradient, and the scatter of row q
template <typename R>
__device__ __forceinline__ void gather_grad_row(const R* ph, const int* lc, const R (*w)[3], const R (*dw)[3], R* g) {
    R gx = R(0), gy = R(0), gz = R(0);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        R u0 = R(0), u1 = R(0), u2 = R(0);
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            const R* row = &ph[pidx(lc[0] + a, lc[1] + b, lc[2])];
            R p0 = row[0], p1 = row[PZ], p2 = row[2 * PZ];
            R s0 = w[2][0] * p0 + w[2][1] * p1 + w[2][2] * p2;
            R s1 = dw[2][0] * p0 + dw[2][1] * p1 + dw[2][2] * p2;
            u0 += w[1][b] * s0;
            u1 += dw[1][b] * s0;
            u2 += w[1][b] * s1;
        }
        gx += dw[0][a] * u0;
        gy += w[0][a] * u1;
        gz += w[0][a] * u2;
    }
    g[0] = gx;
    g[1] = gy;
    g[2] = gz;
}

template <typename R>
__device__ __forceinline__ void scatter_sep(R (*ua)[PN], const int* lc, const R (*w)[3], const R (*dw)[3], const R* M) {
#pragma unroll
    for (int q = 0; q < 3; ++q) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            R A0 = M[3 * q] * dw[0][a], A1 = M[3 * q + 1] * w[0][a], A2 = M[3 * q + 2] * w[0][a];
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                R B0 = A0 * w[1][b] + A1 * dw[1][b];
                R B1 = A2 * w[1][b];
                R* row = &ua[q][pidx(lc[0] + a, lc[1] + b, lc[2])];
#pragma unroll
                for (int c = 0; c < 3; ++c) atomicAdd(row + c * PZ, B0 * w[2][c] + B1 * dw[2][c]);
            }
        }
    }
}

// A thread's running sum of products formed in R: compensated (Kahan) in
// float32, plain in float64, handed on in float64 (the CG reductions and the
// operator's p . H p use it).
template <typename R>
struct KSum {
    R s = R(0), c = R(0);   // value s - c
    __device__ void add(R x) {
        if constexpr (sizeof(R) == 4) {
            R y = x - c;
            R t = s + y;
            c = (t - s) - y;
            s = t;
        } else {
            s += x;
        }
    }
    // sum over the warp (valid in lane 0), float32 pairs combined with an
    // error-free two-sum, so the float64 pipe only sees lane 0's conversion
    __device__ double warp_total() const {
        if constexpr (sizeof(R) == 4) {
            R hs = s, hc = c;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                R os = __shfl_down_sync(0xffffffffu, hs, o), oc = __shfl_down_sync(0xffffffffu, hc, o);
                R t = hs + os;
                R bb = t - hs;
                R err = (hs - (t - bb)) + (os - bb);   // hs + os = t + err exactly
                hs = t;
                hc = hc + oc - err;
            }
            return (threadIdx.x & 31) == 0 ? (double)hs - (double)hc : 0.0;
        } else {
            return warp_sum((double)s);
        }
    }
    __device__ void clear() { s = c = R(0); }
};

// general per-particle operator (solid or viscous liquid) on the padded layout

// the exact or projected surface term of sample j for a gathered dF^: G (3x3)
template <typename R>
__device__ __forceinline__ void sample_G(const ApplyArgs<R>& a, int j, const R* dFh, R dt, R* G) {
    R Fh[9], av[3], nv[3];
#pragma unroll
    for (int q = 0; q < 9; ++q) Fh[q] = a.sF.a[q][j];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        av[q] = a.sa.a[q][j];
        nv[q] = a.sn.a[q][j];
    }
    R k = a.sg[j], ic = a.sic[j];
    R dC[9];
    dcofactor<R>(Fh, dFh, dC);
    R dc[3] = {dC[0] * av[0] + dC[1] * av[1] + dC[2] * av[2], dC[3] * av[0] + dC[4] * av[1] + dC[5] * av[2],
               dC[6] * av[0] + dC[7] * av[1] + dC[8] * av[2]};
    R nd = nv[0] * dc[0] + nv[1] * dc[1] + nv[2] * dc[2];
    R dn[3] = {(dc[0] - nd * nv[0]) * ic, (dc[1] - nd * nv[1]) * ic, (dc[2] - nd * nv[2]) * ic};
    surf_G<R>(k * dt * dt, dn, Fh, av, G);
    if (a.mode == MPM_HESS_EXACT) {
        R G2[9];
        surf_G<R>(k * dt * dt, nv, dFh, av, G2);
#pragma unroll
        for (int q = 0; q < 9; ++q) G[q] += G2[q];
    } else {
        add_conformal<R>(k * dt * dt, nv, av, dFh, G);
    }
}

constexpr int NT_CELL = 64;


template <typename R>
__device__ __forceinline__ void load_halo_rows(const int* __restrict__ nbr, int slot, const R* __restrict__ p,
                                               R (*ph)[PN], R (*ua)[PN]) {
    for (int r = threadIdx.x; r < 3 * HE * HE; r += blockDim.x) {
        int c = r / (HE * HE), yz = r % (HE * HE), hy = yz % HE, hz = yz / HE;
        int nmid, nlo, nhi, base;
        halo_row<R>(nbr, slot, hy, hz, nmid, nlo, nhi, base);
        R m0 = R(0), m1 = R(0), m2 = R(0), m3 = R(0);
        if (nmid >= 0) {
            const R* src = p + nmid * 192 + c * 64 + base;
            if constexpr (sizeof(R) == 4) {
                float4 v = *reinterpret_cast<const float4*>(src);
                m0 = v.x; m1 = v.y; m2 = v.z; m3 = v.w;
            } else {
                m0 = src[0]; m1 = src[1]; m2 = src[2]; m3 = src[3];
            }
        }
        int h0 = pidx(0, hy, hz);
        ph[c][h0] = nlo >= 0 ? p[nlo * 192 + c * 64 + base + 3] : R(0);
        ph[c][h0 + 1] = m0;
        ph[c][h0 + 2] = m1;
        ph[c][h0 + 3] = m2;
        ph[c][h0 + 4] = m3;
        ph[c][h0 + 5] = nhi >= 0 ? p[nhi * 192 + c * 64 + base] : R(0);
        if (ua) {
#pragma unroll
            for (int k = 0; k < 6; ++k) ua[c][h0 + k] = R(0);
        }
    }
}

template <typename R>
__device__ __forceinline__ void flush_halo_rows(const int* __restrict__ nbr, int slot, R (*ua)[PN], R* __restrict__ u) {
    for (int r = threadIdx.x; r < 3 * HE * HE; r += blockDim.x) {
        int c = r / (HE * HE), yz = r % (HE * HE), hy = yz % HE, hz = yz / HE;
        int nmid, nlo, nhi, base;
        halo_row<R>(nbr, slot, hy, hz, nmid, nlo, nhi, base);
        int h0 = pidx(0, hy, hz);
        R lo = ua[c][h0], hi = ua[c][h0 + 5];
        R m0 = ua[c][h0 + 1], m1 = ua[c][h0 + 2], m2 = ua[c][h0 + 3], m3 = ua[c][h0 + 4];
        if (nlo >= 0 && lo != R(0)) atomicAdd(&u[nlo * 192 + c * 64 + base + 3], lo);
        if (nhi >= 0 && hi != R(0)) atomicAdd(&u[nhi * 192 + c * 64 + base], hi);
        if (nmid >= 0 && (m0 != R(0) || m1 != R(0) || m2 != R(0) || m3 != R(0))) {
            R* dst = u + nmid * 192 + c * 64 + base;
            if constexpr (sizeof(R) == 4) {
                atomicAdd(reinterpret_cast<float4*>(dst), make_float4(m0, m1, m2, m3));
            } else {
                atomicAdd(dst, m0);
                atomicAdd(dst + 1, m1);
                atomicAdd(dst + 2, m2);
                atomicAdd(dst + 3, m3);
            }
        }
    }
}


// ----------------------------------------------------------------------
// Scatter without shared atomics. Each warp owns 32 cells forming a 4x4x2 brick
// and accumulates into its own z-range of the halo (warp 0: node levels 0..3,
// warp 1: levels 2..5, stored at 4..7), so the two warps never touch the same
// word. Within a warp, for one stencil offset the 32 lanes write 32 distinct
// nodes, and offsets whose z differs by 2 never meet (a warp's cells span two z
// levels), so each phase below is a plain read-add-write by every lane with no
// two lanes on one node; __syncwarp orders the phases.

// every lane of the warp calls it; lanes with act = false only take part in the
// phase ordering (two lanes may never write one node in one phase)
template <typename R>
__device__ __forceinline__ void rmw_phases(R* uq, const R (&N)[3][3][3], int lx, int ly, int zb, bool act = true) {
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            __syncwarp();
            if (act) {
                R* p0 = uq + pidx(lx + a, ly + b, zb);
                R* p2 = uq + pidx(lx + a, ly + b, zb + 2);
                const R v0 = *p0, v2 = *p2;
                *p0 = v0 + N[a][b][0];
                *p2 = v2 + N[a][b][2];
            }
        }
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            __syncwarp();
            if (act) {
                R* p1 = uq + pidx(lx + a, ly + b, zb + 1);
                *p1 += N[a][b][1];
            }
        }
    __syncwarp();
}

// node values (without the 1/dx factor) of the cell's moments, component by
// component, added to the warp's accumulation halo (every lane of the warp calls it)
template <typename R>
__device__ __forceinline__ void cell_scatter_warp(const R (&M)[3][3][3], R (*ua)[UN], int lx, int ly, int zb) {
    R N[3][3][3];
    {
        R T1[2][3][3], T2[2][3][3];
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) wN<R>(M[i][j][0], M[i][j][1], M[i][j][2], T1[i][j][0], T1[i][j][1], T1[i][j][2]);
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int c = 0; c < 3; ++c) wN<R>(T1[i][0][c], T1[i][1][c], T1[i][2][c], T2[i][0][c], T2[i][1][c], T2[i][2][c]);
#pragma unroll
        for (int b = 0; b < 3; ++b)
#pragma unroll
            for (int c = 0; c < 3; ++c) dN<R>(T2[0][b][c], T2[1][b][c], N[0][b][c], N[1][b][c], N[2][b][c]);
    }
    rmw_phases<R>(ua[0], N, lx, ly, zb);
    {
        R T1[3][2][3], T2[3][3][3];
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 2; ++j) wN<R>(M[i][j][0], M[i][j][1], M[i][j][2], T1[i][j][0], T1[i][j][1], T1[i][j][2]);
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int c = 0; c < 3; ++c) dN<R>(T1[i][0][c], T1[i][1][c], T2[i][0][c], T2[i][1][c], T2[i][2][c]);
#pragma unroll
        for (int b = 0; b < 3; ++b)
#pragma unroll
            for (int c = 0; c < 3; ++c) wN<R>(T2[0][b][c], T2[1][b][c], T2[2][b][c], N[0][b][c], N[1][b][c], N[2][b][c]);
    }
    rmw_phases<R>(ua[1], N, lx, ly, zb);
    {
        R T1[3][3][3], T2[3][3][3];
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) dN<R>(M[i][j][0], M[i][j][1], T1[i][j][0], T1[i][j][1], T1[i][j][2]);
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int c = 0; c < 3; ++c) wN<R>(T1[i][0][c], T1[i][1][c], T1[i][2][c], T2[i][0][c], T2[i][1][c], T2[i][2][c]);
#pragma unroll
        for (int b = 0; b < 3; ++b)
#pragma unroll
            for (int c = 0; c < 3; ++c) wN<R>(T2[0][b][c], T2[1][b][c], T2[2][b][c], N[0][b][c], N[1][b][c], N[2][b][c]);
    }
    rmw_phases<R>(ua[2], N, lx, ly, zb);
}

template <typename R>
__device__ __forceinline__ void flush_halo_rows_u(const int* __restrict__ nbr, int slot, R (*ua)[UN], R* __restrict__ u) {
    for (int yz = threadIdx.x; yz < HE * HE; yz += blockDim.x) {
        const int hy = yz % HE, hz = yz / HE;
        int nmid, nlo, nhi, base;
        halo_row<R>(nbr, slot, hy, hz, nmid, nlo, nhi, base);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            R v[6];
#pragma unroll
            for (int k = 0; k < 6; ++k) v[k] = R(0);
            if (hz <= 3) {
                const R* s = &ua[c][pidx(0, hy, hz)];
#pragma unroll
                for (int k = 0; k < 6; ++k) v[k] += s[k];
            }
            if (hz >= 2) {
                const R* s = &ua[c][pidx(0, hy, hz + 2)];
#pragma unroll
                for (int k = 0; k < 6; ++k) v[k] += s[k];
            }
            if (nlo >= 0 && v[0] != R(0)) atomicAdd(&u[nlo * 192 + c * 64 + base + 3], v[0]);
            if (nhi >= 0 && v[5] != R(0)) atomicAdd(&u[nhi * 192 + c * 64 + base], v[5]);
            if (nmid >= 0 && (v[1] != R(0) || v[2] != R(0) || v[3] != R(0) || v[4] != R(0))) {
                R* dst = u + nmid * 192 + c * 64 + base;
                if constexpr (sizeof(R) == 4) {
                    atomicAdd(reinterpret_cast<float4*>(dst), make_float4(v[1], v[2], v[3], v[4]));
                } else {
                    atomicAdd(dst, v[1]);
                    atomicAdd(dst + 1, v[2]);
                    atomicAdd(dst + 2, v[3]);
                    atomicAdd(dst + 3, v[4]);
                }
            }
        }
    }
}

// ======================================================================
// Hessian-vector operator on cells in x-pairs (the production kernel for the
// rank-one liquid particles and the surface samples).
//
// One warp per block of 4x4x4 cells. Lane l = m + 2 ly + 8 lz owns the two
// cells 2l and 2l+1, side by side in x: A at (2m, ly, lz) and B at
// (2m+1, ly, lz). Every step of the per-cell polynomial form above is
// the same for A and B, so the lane carries each quantity as a pair (A in .x, B
// in .y) and uses paired float arithmetic, one instruction for both cells. The
// stencils of A and B cover the x-nodes 2m..2m+2 and 2m+1..2m+3 of a row: the
// lane reads those four nodes as two aligned pairs, and adds A's and B's node
// values into the same four nodes before it writes them. The liquid records of
// a row are stored pair-interleaved (x_A x_B y_A y_B z_A z_B kappa_A kappa_B for
// the cells 2l, 2l+1), so a record pair arrives as four value pairs.
// ======================================================================

// paired arithmetic: float2 uses the paired float instructions, double2 plain pairs
__device__ __forceinline__ float2 vadd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 vmul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 vfma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 vsub(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }
__device__ __forceinline__ double2 vadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 vmul(double2 a, double2 b) { return make_double2(a.x * b.x, a.y * b.y); }
__device__ __forceinline__ double2 vfma(double2 a, double2 b, double2 c) {
    return make_double2(fma(a.x, b.x, c.x), fma(a.y, b.y, c.y));
}
__device__ __forceinline__ double2 vsub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }

template <typename R> struct VPair;
template <> struct VPair<float> {
    using T = float2;
    static __device__ __forceinline__ float2 make(float a, float b) { return make_float2(a, b); }
};
template <> struct VPair<double> {
    using T = double2;
    static __device__ __forceinline__ double2 make(double a, double b) { return make_double2(a, b); }
};

// the scalar transforms (wT, dT, wN, dN) on pairs
template <typename V>
__device__ __forceinline__ void pwT(V v0, V v1, V v2, V& o0, V& o1, V& o2, V h) {
    o0 = vmul(vadd(v0, v1), h);
    o1 = vsub(v1, v0);
    o2 = vsub(vmul(vadd(v0, v2), h), v1);
}
template <typename V>
__device__ __forceinline__ void pdT(V v0, V v1, V v2, V& o0, V& o1, V m2) {
    o0 = vsub(v1, v0);
    o1 = vfma(v1, m2, vadd(v0, v2));
}
template <typename V>
__device__ __forceinline__ void pwN(V m0, V m1, V m2, V& n0, V& n1, V& n2, V h) {
    n0 = vsub(vmul(vadd(m0, m2), h), m1);
    n1 = vfma(m0, h, vsub(m1, m2));
    n2 = vmul(m2, h);
}
template <typename V>
__device__ __forceinline__ void pdN(V m0, V m1, V& n0, V& n1, V& n2, V m2) {
    n0 = vsub(m1, m0);
    n1 = vfma(m1, m2, m0);
    n2 = m1;
}

// the four x-nodes 2m..2m+3 of halo row (y, z) of component q, as the pairs
// (x0, x1) and (x2, x3)
template <typename R>
__device__ __forceinline__ void row_pairs(const R* phq, int x0, int y, int z, typename VPair<R>::T& p01,
                                          typename VPair<R>::T& p23) {
    using V = typename VPair<R>::T;
    const V* r = reinterpret_cast<const V*>(phq + pidx(x0, y, z));
    p01 = r[0];
    p23 = r[1];
}

// C = the coefficients of tr(dL) (without the 1/dx factor) of the cells A and B
// of the pair at (2m, ly, lz): each component's separable transform, the
// derivative axis first (it leaves two coefficients of three).
template <typename R>
__device__ __forceinline__ void pair_coefficients(const R (*ph)[PN], int m, int ly, int lz,
                                                  typename VPair<R>::T (&C)[3][3][3]) {
    using V = typename VPair<R>::T;
    using P = VPair<R>;
    const V h = P::make(R(0.5), R(0.5)), m2 = P::make(R(-2), R(-2));
    const int x0 = 2 * m;
    // x component: D along x, then W along y and z
    {
        V X[2][3][3];
#pragma unroll
        for (int b = 0; b < 3; ++b)
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                V p01, p23;
                row_pairs<R>(ph[0], x0, ly + b, lz + c, p01, p23);
                const V p12 = P::make(p01.y, p23.x);
                pdT<V>(p01, p12, p23, X[0][b][c], X[1][b][c], m2);
            }
        V Y[2][3][3];
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int c = 0; c < 3; ++c) pwT<V>(X[i][0][c], X[i][1][c], X[i][2][c], Y[i][0][c], Y[i][1][c], Y[i][2][c], h);
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) pwT<V>(Y[i][j][0], Y[i][j][1], Y[i][j][2], C[i][j][0], C[i][j][1], C[i][j][2], h);
#pragma unroll
        for (int j = 0; j < 3; ++j)
#pragma unroll
            for (int k = 0; k < 3; ++k) C[2][j][k] = P::make(R(0), R(0));
    }
    // y component: D along y on the node pairs, W along x, then W along z
    {
        V Y01[2][3], Y23[2][3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            V a01[3], a23[3];
#pragma unroll
            for (int b = 0; b < 3; ++b) row_pairs<R>(ph[1], x0, ly + b, lz + c, a01[b], a23[b]);
            pdT<V>(a01[0], a01[1], a01[2], Y01[0][c], Y01[1][c], m2);
            pdT<V>(a23[0], a23[1], a23[2], Y23[0][c], Y23[1][c], m2);
        }
        V X[3][2][3];
#pragma unroll
        for (int j = 0; j < 2; ++j)
#pragma unroll
            for (int c = 0; c < 3; ++c)
                pwT<V>(Y01[j][c], P::make(Y01[j][c].y, Y23[j][c].x), Y23[j][c], X[0][j][c], X[1][j][c], X[2][j][c], h);
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                V g0, g1, g2;
                pwT<V>(X[i][j][0], X[i][j][1], X[i][j][2], g0, g1, g2, h);
                C[i][j][0] = vadd(C[i][j][0], g0);
                C[i][j][1] = vadd(C[i][j][1], g1);
                C[i][j][2] = vadd(C[i][j][2], g2);
            }
    }
    // z component: D along z on the node pairs, W along y, then W along x
    {
        V Z01[3][2], Z23[3][2];
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            V a01[3], a23[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) row_pairs<R>(ph[2], x0, ly + b, lz + c, a01[c], a23[c]);
            pdT<V>(a01[0], a01[1], a01[2], Z01[b][0], Z01[b][1], m2);
            pdT<V>(a23[0], a23[1], a23[2], Z23[b][0], Z23[b][1], m2);
        }
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            V y01[3], y23[3];
            pwT<V>(Z01[0][k], Z01[1][k], Z01[2][k], y01[0], y01[1], y01[2], h);
            pwT<V>(Z23[0][k], Z23[1][k], Z23[2][k], y23[0], y23[1], y23[2], h);
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                V g0, g1, g2;
                pwT<V>(y01[j], P::make(y01[j].y, y23[j].x), y23[j], g0, g1, g2, h);
                C[0][j][k] = vadd(C[0][j][k], g0);
                C[1][j][k] = vadd(C[1][j][k], g1);
                C[2][j][k] = vadd(C[2][j][k], g2);
            }
        }
    }
}

// one component's node values of the pair, from its moments: N[b][c] holds, for
// the halo row (ly + b, zb + c), the values to add at x-nodes 2m..2m+1 (lo) and
// 2m+2..2m+3 (hi), A's and B's contributions summed
template <typename V, typename P>
__device__ __forceinline__ void pair_rows(const V (&Nx)[3][3][3], V (&lo)[3][3], V (&hi)[3][3]) {
#pragma unroll
    for (int b = 0; b < 3; ++b)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const V n0 = Nx[0][b][c], n1 = Nx[1][b][c], n2 = Nx[2][b][c];
            lo[b][c] = P::make(n0.x, n1.x + n0.y);
            hi[b][c] = P::make(n2.x + n1.y, n2.y);
        }
}

// read-add-write of the three components' rows into the lane's accumulation
// levels. Phases: for each y offset b, the z offsets {0, 2} then {1}, the lo pairs
// then the hi pairs; within a phase no two lanes of the warp write one node. The
// components go to separate arrays, so one phase carries all three (six
// independent read-add-writes per lane where z offsets 0 and 2 go together).
template <typename R>
__device__ __forceinline__ void pair_rmw3(R (*ua)[UN], int x0, int ly, int zb,
                                          const typename VPair<R>::T (&lo)[3][3][3],
                                          const typename VPair<R>::T (&hi)[3][3][3]) {
    using V = typename VPair<R>::T;
#pragma unroll
    for (int b = 0; b < 3; ++b) {
#pragma unroll
        for (int half = 0; half < 2; ++half) {
            __syncwarp();
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                V* p0 = reinterpret_cast<V*>(ua[q] + pidx(x0 + 2 * half, ly + b, zb));
                V* p2 = reinterpret_cast<V*>(ua[q] + pidx(x0 + 2 * half, ly + b, zb + 2));
                const V v0 = *p0, v2 = *p2;
                *p0 = vadd(v0, half ? hi[q][b][0] : lo[q][b][0]);
                *p2 = vadd(v2, half ? hi[q][b][2] : lo[q][b][2]);
            }
        }
#pragma unroll
        for (int half = 0; half < 2; ++half) {
            __syncwarp();
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                V* p1 = reinterpret_cast<V*>(ua[q] + pidx(x0 + 2 * half, ly + b, zb + 1));
                *p1 = vadd(*p1, half ? hi[q][b][1] : lo[q][b][1]);
            }
        }
    }
    __syncwarp();
}

// node values (without the 1/dx factor) of the pair's moments, component by
// component, then added to the lane's accumulation levels (every lane calls it)
template <typename R>
__device__ __forceinline__ void pair_scatter(const typename VPair<R>::T (&M)[3][3][3], R (*ua)[UN], int m, int ly,
                                             int zb) {
    using V = typename VPair<R>::T;
    using P = VPair<R>;
    const V h = P::make(R(0.5), R(0.5)), m2 = P::make(R(-2), R(-2));
    const int x0 = 2 * m;
    V N[3][3][3];
    V lo[3][3][3], hi[3][3][3];   // per component
    {   // x: W along z, W along y, D along x
        V T1[2][3][3], T2[2][3][3];
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) pwN<V>(M[i][j][0], M[i][j][1], M[i][j][2], T1[i][j][0], T1[i][j][1], T1[i][j][2], h);
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int c = 0; c < 3; ++c) pwN<V>(T1[i][0][c], T1[i][1][c], T1[i][2][c], T2[i][0][c], T2[i][1][c], T2[i][2][c], h);
#pragma unroll
        for (int b = 0; b < 3; ++b)
#pragma unroll
            for (int c = 0; c < 3; ++c) pdN<V>(T2[0][b][c], T2[1][b][c], N[0][b][c], N[1][b][c], N[2][b][c], m2);
    }
    pair_rows<V, P>(N, lo[0], hi[0]);
    {   // y: W along z, W along x, D along y
        V T1[3][2][3], T2[3][2][3];
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 2; ++j) pwN<V>(M[i][j][0], M[i][j][1], M[i][j][2], T1[i][j][0], T1[i][j][1], T1[i][j][2], h);
#pragma unroll
        for (int j = 0; j < 2; ++j)
#pragma unroll
            for (int c = 0; c < 3; ++c) pwN<V>(T1[0][j][c], T1[1][j][c], T1[2][j][c], T2[0][j][c], T2[1][j][c], T2[2][j][c], h);
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int c = 0; c < 3; ++c) pdN<V>(T2[a][0][c], T2[a][1][c], N[a][0][c], N[a][1][c], N[a][2][c], m2);
    }
    pair_rows<V, P>(N, lo[1], hi[1]);
    {   // z: W along x, W along y, D along z
        V T1[3][3][2], T2[3][3][2];
#pragma unroll
        for (int j = 0; j < 3; ++j)
#pragma unroll
            for (int k = 0; k < 2; ++k) pwN<V>(M[0][j][k], M[1][j][k], M[2][j][k], T1[0][j][k], T1[1][j][k], T1[2][j][k], h);
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int k = 0; k < 2; ++k) pwN<V>(T1[a][0][k], T1[a][1][k], T1[a][2][k], T2[a][0][k], T2[a][1][k], T2[a][2][k], h);
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) pdN<V>(T2[a][b][0], T2[a][b][1], N[a][b][0], N[a][b][1], N[a][b][2], m2);
    }
    pair_rows<V, P>(N, lo[2], hi[2]);
    pair_rmw3<R>(ua, x0, ly, zb, lo, hi);
}

// KRP: record rows staged per bulk copy (2, 4 or 8, chosen by the autotuner in
// cg_solve_t); the sample records share the staging buffer
template <typename R, int KRP>
__global__ void __launch_bounds__(32, sizeof(R) == 4 ? 16 : 8) k_apply_pair(ApplyArgs<R> a) {
    using V = typename VPair<R>::T;
    using P = VPair<R>;
    __shared__ __align__(16) R ph[3][PN];
    __shared__ __align__(16) R ua[3][UN];
    __shared__ __align__(16) R sp[KRP * 256];
    __shared__ __align__(8) uint64_t bar;
    const int w = blockIdx.x;
    const int lane = threadIdx.x;
    // The block's indices and counts are independent loads, issued together; the
    // scene's done flag is read here but tested only once the first record copy
    // and the halo loads are under way, so the two chains of dependent loads
    // overlap.
    const int slot = a.work[w];
    const long long gb = a.work_gb[w];
    const int wrows = a.wrows[w], wroff = a.wroff[w];
    const int4 bc = a.coord[slot];
    const int npart = a.cell_start[gb * 64 + 64] - a.cell_start[gb * 64];
    const int ngen = a.slot_gen[slot];
    const int sbeg = a.scell_start[gb * 64], send = a.scell_start[gb * 64 + 64];
    const int done = a.check_done ? a.scal[bc.w].cg_done : 0;
    const SceneDev& S = a.sc[bc.w];
    // liquid rows of the block: none when every particle takes the general path
    const int rows = (npart > ngen) ? wrows : 0;
    const R* recs = reinterpret_cast<const R*>(a.opk) + (long long)wroff * 256;
    const int nchunk = (rows + KRP - 1) / KRP;
    if (lane == 0) mbar_init(&bar, 1);
    for (int i = lane; i < (int)(3 * UN * sizeof(R) / 16); i += 32)
        reinterpret_cast<int4*>(&ua[0][0])[i] = make_int4(0, 0, 0, 0);
    __syncwarp();
    if (lane == 0 && nchunk > 0) {
        const uint32_t bytes = (uint32_t)(min(KRP, rows) * 256 * sizeof(R));
        mbar_expect_tx(&bar, bytes);
        bulk_g2s(sp, recs, bytes, &bar);
    }
    // the direction's halo: one neighbour lookup per (y, z) row, three components
    for (int yz = lane; yz < HE * HE; yz += 32) {
        const int hy = yz % HE, hz = yz / HE;
        int nmid, nlo, nhi, base;
        halo_row<R>(a.nbr, slot, hy, hz, nmid, nlo, nhi, base);
        const int h0 = pidx(0, hy, hz);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            R m0 = R(0), m1 = R(0), m2 = R(0), m3 = R(0);
            if (nmid >= 0) {
                const R* src = a.p + nmid * 192 + c * 64 + base;
                if constexpr (sizeof(R) == 4) {
                    float4 v = *reinterpret_cast<const float4*>(src);
                    m0 = v.x; m1 = v.y; m2 = v.z; m3 = v.w;
                } else {
                    m0 = src[0]; m1 = src[1]; m2 = src[2]; m3 = src[3];
                }
            }
            ph[c][h0] = nlo >= 0 ? a.p[nlo * 192 + c * 64 + base + 3] : R(0);
            ph[c][h0 + 1] = m0;
            ph[c][h0 + 2] = m1;
            ph[c][h0 + 3] = m2;
            ph[c][h0 + 4] = m3;
            ph[c][h0 + 5] = nhi >= 0 ? a.p[nhi * 192 + c * 64 + base] : R(0);
        }
    }
    __syncwarp();
    if (done) {   // the scene's CG has converged: let the first copy land, then leave
        if (nchunk > 0) mbar_wait_bounded(&bar, 0u, 1LL << 26);
        return;
    }
    const R inv_dx = (R)S.inv_dx;
    const int m = lane & 1, ly = (lane >> 1) & 3, lz = lane >> 3;
    const int zb = lz + 2 * (lz >> 1);   // the lane's accumulation levels (region lz >> 1)
    KSum<R> pap;   // p . (H - M) p of this block's particles and samples
    if (rows > 0) {
        V C[3][3][3], M[3][3][3];
        pair_coefficients<R>(ph, m, ly, lz, C);
        {
            const R s2 = inv_dx * inv_dx;
            const V s2v = P::make(s2, s2);
#pragma unroll
            for (int q = 0; q < 27; ++q) {
                (&C[0][0][0])[q] = vmul((&C[0][0][0])[q], s2v);
                (&M[0][0][0])[q] = P::make(R(0), R(0));
            }
        }
        const V offx = P::make(R(2 * m), R(2 * m + 1)), offy = P::make(R(ly), R(ly)), offz = P::make(R(lz), R(lz));
        V ks = P::make(R(0), R(0)), kc = P::make(R(0), R(0));   // compensated pair sum of s tr
        for (int k = 0; k < nchunk; ++k) {
            const int r0 = k * KRP;
            if (!__all_sync(0xffffffffu, mbar_wait_bounded(&bar, (uint32_t)(k & 1), 1LL << 26))) {
                // give the copy in flight a last bounded wait before the CTA leaves
                if (lane == 0) atomicOr(a.err, ERR_TIMEOUT);
                mbar_wait_bounded(&bar, (uint32_t)(k & 1), 1LL << 20);
                return;
            }
            const int rhi = min(rows, r0 + KRP);
            for (int r = r0; r < rhi; ++r) {
                const V* pr = reinterpret_cast<const V*>(sp + (r - r0) * 256 + 8 * lane);
                const V tx = vsub(pr[0], offx), ty = vsub(pr[1], offy), tz = vsub(pr[2], offz);
                V kap = pr[3];
                kap.x = kap.x > R(0) ? kap.x : R(0);   // empty slot 0, general particle < 0
                kap.y = kap.y > R(0) ? kap.y : R(0);
                // s2 tr(dL)(t) by Horner's rule, z then y then x (no t^2 t^2 t^2 term)
                V E[3];
#pragma unroll
                for (int ii = 0; ii < 3; ++ii) {
                    V D[3];
#pragma unroll
                    for (int j = 0; j < 3; ++j)
                        D[j] = (ii == 2 && j == 2) ? vfma(tz, C[2][2][1], C[2][2][0])
                                                   : vfma(tz, vfma(tz, C[ii][j][2], C[ii][j][1]), C[ii][j][0]);
                    E[ii] = vfma(ty, vfma(ty, D[2], D[1]), D[0]);
                }
                const V tr = vfma(tx, vfma(tx, E[2], E[1]), E[0]);
                const V s = vmul(kap, tr);
                {   // Kahan step on the pair: ks - kc += s tr / s2 (tr carries s2)
                    const V y = vsub(vmul(s, tr), kc);
                    const V t = vadd(ks, y);
                    kc = vsub(vsub(t, ks), y);
                    ks = t;
                }
                const V tz2 = vmul(tz, tz);
                V sx = s;
#pragma unroll
                for (int ii = 0; ii < 3; ++ii) {
                    V sxy = sx;
#pragma unroll
                    for (int j = 0; j < 3; ++j) {
                        M[ii][j][0] = vadd(M[ii][j][0], sxy);
                        M[ii][j][1] = vfma(sxy, tz, M[ii][j][1]);
                        if (!(ii == 2 && j == 2)) M[ii][j][2] = vfma(sxy, tz2, M[ii][j][2]);
                        if (j < 2) sxy = vmul(sxy, ty);
                    }
                    if (ii < 2) sx = vmul(sx, tx);
                }
            }
            __syncwarp();
            if (k + 1 < nchunk && lane == 0) {
                const uint32_t bytes = (uint32_t)(min(KRP, rows - (r0 + KRP)) * 256 * sizeof(R));
                mbar_expect_tx(&bar, bytes);
                bulk_g2s(sp, recs + (long long)(r0 + KRP) * 256, bytes, &bar);
            }
        }
        // s tr carries s2 twice: p . K p = sum kappa s2 tr^2 = (s tr) / s2
        const R inv_s2 = R(1) / (inv_dx * inv_dx);
        pap.add((ks.x - kc.x) * inv_s2);
        pap.add((ks.y - kc.y) * inv_s2);
        pair_scatter<R>(M, ua, m, ly, zb);
    }

    // The block's surface samples (projected mode with current maps), staged by
    // one bulk copy per chunk of SCAP records, in the order of their sorted
    // cells. A pass takes the next ten samples of the chunk, three lanes per
    // sample: lane q gathers row q of dF^, forms row block q of G = K dF^ and
    // the node values of row q of G gradN over the sample's stencil, taken
    // relative to its sorted cell (t clamped to [0, 1]). Samples of one cell are
    // neighbours in the pass; their node values are summed into the first of
    // them (a segmented suffix sum over the lane groups), which alone writes, so
    // the writers of a pass lie in distinct cells. Each adds into its cell's
    // accumulation levels (region sz >> 1, where the cells span two z levels):
    // per stencil offset the writers of a pass write distinct nodes.
    const int nsm = a.samples_in_cell ? send - sbeg : 0;
    if (nsm > 0) {
        constexpr int SCAP = (KRP * 256) / SREC;   // samples per staged chunk
        __shared__ int cell_of[SCAP];               // sorted cell of each staged record
        R* sbuf = sp;
        uint32_t phase = (uint32_t)nchunk;         // bulk copies completed on `bar` so far
        __syncwarp();
        if (lane == 0) {
            const uint32_t bytes = (uint32_t)(min(nsm, SCAP) * SREC * sizeof(R));
            mbar_expect_tx(&bar, bytes);
            bulk_g2s(sbuf, a.sKa + (long long)sbeg * SREC, bytes, &bar);
        }
        const int si = lane / 3, q = lane - 3 * si;
        const int qa = q == 0 ? 1 : 0, qb = q == 2 ? 1 : 2;                 // the other two row blocks
        const int offA = q == 2 ? 27 : 18, offB = q == 0 ? 27 : 36;        // their 3x3 blocks
        const bool trA = q != 0, trB = q == 2;                              // below the diagonal: transposed
        const int c2 = 2 * lane;
        const int scsA = a.scell_start[gb * 64 + c2] - sbeg, scsB = a.scell_start[gb * 64 + c2 + 1] - sbeg;
        const int sceB = a.scell_start[gb * 64 + c2 + 2] - sbeg;
        for (int c0 = 0; c0 < nsm; c0 += SCAP) {
            const int c1 = min(nsm, c0 + SCAP), nc = c1 - c0;
            // the owners of the two cells list their records of this chunk
            for (int j = max(scsA, c0); j < min(scsB, c1); ++j) cell_of[j - c0] = c2;
            for (int j = max(scsB, c0); j < min(sceB, c1); ++j) cell_of[j - c0] = c2 + 1;
            if (!__all_sync(0xffffffffu, mbar_wait_bounded(&bar, phase & 1u, 1LL << 26))) {
                if (lane == 0) atomicOr(a.err, ERR_TIMEOUT);
                mbar_wait_bounded(&bar, phase & 1u, 1LL << 20);
                return;
            }
            ++phase;
            __syncwarp();
            for (int base = 0; base < nc; base += 10) {
                const int k = base + si;
                const int kend = min(nc, base + 10);
                const bool act = lane < 30 && k < kend;
                const int sc = act ? cell_of[k] : -1;   // the sample's cell
                const int scc = sc < 0 ? 0 : sc;
                const int sx = scc & 3, sy = (scc >> 2) & 3, sz = scc >> 4;
                const R* rec = sbuf + (act ? k : 0) * SREC;
                R wgt[3][3], dw[3][3];
                {
                    const R tt[3] = {fmin(fmax(rec[45] - R(sx), R(0)), R(1)), fmin(fmax(rec[46] - R(sy), R(0)), R(1)),
                                     fmin(fmax(rec[47] - R(sz), R(0)), R(1))};
#pragma unroll
                    for (int ax = 0; ax < 3; ++ax) {
                        bspline<R>(tt[ax] + R(0.5), wgt[ax], dw[ax]);
#pragma unroll
                        for (int kk = 0; kk < 3; ++kk) dw[ax][kk] *= inv_dx;
                    }
                }
                const int lc[3] = {sx, sy, sz};
                R g[3] = {R(0), R(0), R(0)};
                if (act) gather_grad_row<R>(ph[q], lc, wgt, dw, g);
                const int l0 = 3 * si < 30 ? 3 * si : 0;
                R gA[3], gB[3];
#pragma unroll
                for (int e = 0; e < 3; ++e) {
                    gA[e] = __shfl_sync(0xffffffffu, g[e], l0 + qa);
                    gB[e] = __shfl_sync(0xffffffffu, g[e], l0 + qb);
                }
                R N[3][3][3];
                if (act) {
                    const R* Dq = rec + 6 * q;
                    const R DM[3][3] = {{Dq[0], Dq[1], Dq[2]}, {Dq[1], Dq[3], Dq[4]}, {Dq[2], Dq[4], Dq[5]}};
                    R bA[9], bB[9];
#pragma unroll
                    for (int mm = 0; mm < 9; ++mm) {
                        bA[mm] = rec[offA + mm];
                        bB[mm] = rec[offB + mm];
                    }
                    R m3[3];
#pragma unroll
                    for (int e = 0; e < 3; ++e) {
                        R acc = R(0);
#pragma unroll
                        for (int f = 0; f < 3; ++f) {
                            const R ka = trA ? bA[3 * f + e] : bA[3 * e + f];
                            const R kb = trB ? bB[3 * f + e] : bB[3 * e + f];
                            acc += DM[e][f] * g[f] + ka * gA[f] + kb * gB[f];
                        }
                        m3[e] = acc;
                    }
                    pap.add(m3[0] * g[0] + m3[1] * g[1] + m3[2] * g[2]);
#pragma unroll
                    for (int aa = 0; aa < 3; ++aa) {
                        const R A0 = m3[0] * dw[0][aa], A1 = m3[1] * wgt[0][aa], A2 = m3[2] * wgt[0][aa];
#pragma unroll
                        for (int bb = 0; bb < 3; ++bb) {
                            const R B0 = A0 * wgt[1][bb] + A1 * dw[1][bb], B1 = A2 * wgt[1][bb];
#pragma unroll
                            for (int cc = 0; cc < 3; ++cc) N[aa][bb][cc] = B0 * wgt[2][cc] + B1 * dw[2][cc];
                        }
                    }
                } else {
#pragma unroll
                    for (int mm = 0; mm < 27; ++mm) (&N[0][0][0])[mm] = R(0);
                }
                // segmented suffix sum over the groups of one cell (a run of at
                // most ten in a pass: steps 1, 2, 4, 8 while some run is longer)
                for (int d = 1; d < 16; d *= 2) {
                    const bool more = act && k + d < kend && cell_of[k + d] == sc;
                    if (!__any_sync(0xffffffffu, more)) break;
                    const int src = lane + 3 * d < 32 ? lane + 3 * d : lane;
#pragma unroll
                    for (int mm = 0; mm < 27; ++mm) {
                        const R t = __shfl_sync(0xffffffffu, (&N[0][0][0])[mm], src);
                        if (more) (&N[0][0][0])[mm] += t;
                    }
                }
                const bool head = act && (k == base || cell_of[k - 1] != sc);
                // component q's accumulation levels of the sample's cell
                rmw_phases<R>(ua[q], N, sx, sy, sz + 2 * (sz >> 1), head);
            }
            __syncwarp();   // the warp is done with this chunk and its cell list
            if (c1 < nsm && lane == 0) {
                const uint32_t bytes = (uint32_t)(min(nsm - c1, SCAP) * SREC * sizeof(R));
                mbar_expect_tx(&bar, bytes);
                bulk_g2s(sbuf, a.sKa + (long long)(sbeg + c1) * SREC, bytes, &bar);
            }
        }
    }
    if (a.pap) {
        const double v = pap.warp_total();
        if (lane == 0 && v != 0.0) atomicAdd(&a.scal[bc.w].pAp, v);
    }
    __syncwarp();
    flush_halo_rows_u<R>(a.nbr, slot, ua, a.u);
}


// the liquid and sample operator with the context's record-row chunk
template <typename R>
void launch_apply_pair(mpm_ctx* c, const ApplyArgs<R>& a, cudaStream_t st, int rows_per_chunk) {
    if (rows_per_chunk == 2) MPM_LAUNCH k_apply_pair<R, 2><<<c->NW, 32, 0, st>>>(a);
    else if (rows_per_chunk == 8) MPM_LAUNCH k_apply_pair<R, 8><<<c->NW, 32, 0, st>>>(a);
    else MPM_LAUNCH k_apply_pair<R, 4><<<c->NW, 32, 0, st>>>(a);
}

// Per-iterate projected Hessian of each solid particle (the reading of the
// paper's "definiteness fix" for solids): the 9x9 Hessian of psi(F) from the
// analytic eigensystem of isotropic energies, with the signed SVD
// F = U diag(s) V^T and psi_k = d psi / d s_k:
//   pair (x, y), third index z: (psi_x - psi_y)/(s_x - s_y) = 2 mu - lambda (J-1) s_z
//     on U sym(e_x e_y) V^T, and (psi_x + psi_y)/(s_x + s_y)
//     = 2 mu - 4 mu / (s_x + s_y) + lambda (J-1) s_z on U skew(e_x e_y) V^T;
//   scaling modes U diag(q) V^T with (eigenvalue, q) of d^2 psi / ds^2;
// negative eigenvalues dropped. Composed with dF = dL F^n and M = dt^2 V0 dP F^nT
// it is the symmetric map dL -> M = dt^2 V0 sum_k lambda_k+ <W_k, dL> W_k with
// W_k = Q_k F^nT, stored as 45 values.
template <typename R>
__global__ void k_solid_hess(int np, const uint8_t* __restrict__ phase, const int* __restrict__ psc,
                             const SceneDev* __restrict__ sc, RPtr24<R> scache, RPtr9<R> Fn, const R* __restrict__ lmu,
                             const R* __restrict__ llam, const double* __restrict__ V0, RPtr45<R> K) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= np || phase[i] == 0) return;
    const SceneDev& S = sc[psc[i]];
    R F[9], Fo[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) {
        F[q] = scache.a[q][i];
        Fo[q] = Fn.a[q][i];
    }
    const R mu = lmu[i], lam = llam[i];
    const R scale = (R)(S.dt * S.dt * V0[i]);
    R u[3][3], V[9], s[3];
    svd3<R>(F, u, V, s);
    const R J = s[0] * s[1] * s[2];
    const R p[3] = {s[1] * s[2], s[0] * s[2], s[0] * s[1]};
    // d^2 psi / ds^2 and its eigen-pairs
    R A[9], Q[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b)
            A[3 * a + b] = lam * p[a] * p[b] + (a == b ? R(2) * mu : lam * (J - R(1)) * s[3 - a - b]);
    for (int sweep = 0; sweep < 12; ++sweep) {
        R off = A[1] * A[1] + A[2] * A[2] + A[5] * A[5];
        R dia = A[0] * A[0] + A[4] * A[4] + A[8] * A[8];
        const R eps = sizeof(R) == 4 ? R(1e-7) : R(1e-16);   // converged to the type's precision
        if (off <= eps * eps * dia) break;
        jacobi_rot(A, Q, 0, 1);
        jacobi_rot(A, Q, 0, 2);
        jacobi_rot(A, Q, 1, 2);
    }
    R Kp[45];
#pragma unroll
    for (int k = 0; k < 45; ++k) Kp[k] = R(0);
    const R h = R(0.70710678118654752440);
    for (int mode = 0; mode < 9; ++mode) {
        R lv, D[9];   // mode matrix in the SVD frame: Q_mode = U D V^T
#pragma unroll
        for (int k = 0; k < 9; ++k) D[k] = R(0);
        if (mode < 3) {
            lv = A[4 * mode];
#pragma unroll
            for (int c = 0; c < 3; ++c) D[4 * c] = Q[3 * c + mode];
        } else {
            const int pr = (mode - 3) >> 1, x = pr == 2 ? 1 : 0, y = pr == 0 ? 1 : 2, z = 3 - x - y;
            const bool twist = (mode - 3) & 1;
            if (!twist) {
                lv = R(2) * mu - lam * (J - R(1)) * s[z];
                D[3 * x + y] = h;
                D[3 * y + x] = h;
            } else {
                R den = s[x] + s[y];
                den = fabs(den) > R(1e-12) ? den : copysign(R(1e-12), den);
                lv = R(2) * mu - R(4) * mu / den + lam * (J - R(1)) * s[z];
                D[3 * x + y] = h;
                D[3 * y + x] = -h;
            }
        }
        if (!(lv > R(0))) continue;
        R Qm[9], W[9];
        // Qm = U D V^T, U_ac = u[c][a]
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                R acc = R(0);
#pragma unroll
                for (int c = 0; c < 3; ++c)
#pragma unroll
                    for (int d = 0; d < 3; ++d) acc += u[c][a] * D[3 * c + d] * V[3 * b + d];
                Qm[3 * a + b] = acc;
            }
        matmul3_bt<R>(Qm, Fo, W);   // W = Qm F^nT
        const R lw = scale * lv;
#pragma unroll
        for (int m = 0; m < 9; ++m)
#pragma unroll
            for (int l = m; l < 9; ++l) Kp[sym9(m, l)] += lw * W[m] * W[l];
    }
#pragma unroll
    for (int k = 0; k < 45; ++k) K.a[k][i] = Kp[k];
}

// Per-iterate symmetric 9x9 map of each surface sample's projected Hessian
// (Gauss-Newton part plus the conformal part of the cofactor curvature), from
// the same cached F^, n, 1/|c| the operator uses: column l is the map applied
// to the l-th unit dF^. The operator then costs 45 loads and 81 multiply-adds
// per sample instead of re-deriving frames and cofactor derivatives.
template <typename R>
__global__ void k_surf_hess(int ns, const int* __restrict__ ssc, const SceneDev* __restrict__ sc, RPtr9<R> sF,
                            RPtr3<R> sa, RPtr3<R> sn, const R* __restrict__ sic, const R* __restrict__ sg, RPtr3<R> su,
                            R* __restrict__ K) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= ns) return;
    const SceneDev& S = sc[ssc[j]];
    const R dt = (R)S.dt;
    R Fh[9], av[3], nv[3];
#pragma unroll
    for (int q = 0; q < 9; ++q) Fh[q] = sF.a[q][j];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        av[q] = sa.a[q][j];
        nv[q] = sn.a[q][j];
    }
    const R k = sg[j] * dt * dt, ic = sic[j];
    for (int l = 0; l < 9; ++l) {
        R X[9] = {R(0), R(0), R(0), R(0), R(0), R(0), R(0), R(0), R(0)};
        X[l] = R(1);
        R dC[9];
        dcofactor<R>(Fh, X, dC);
        R dc[3] = {dC[0] * av[0] + dC[1] * av[1] + dC[2] * av[2], dC[3] * av[0] + dC[4] * av[1] + dC[5] * av[2],
                   dC[6] * av[0] + dC[7] * av[1] + dC[8] * av[2]};
        R nd = nv[0] * dc[0] + nv[1] * dc[1] + nv[2] * dc[2];
        R dn[3] = {(dc[0] - nd * nv[0]) * ic, (dc[1] - nd * nv[1]) * ic, (dc[2] - nd * nv[2]) * ic};
        R G[9];
        surf_G<R>(k, dn, Fh, av, G);
        add_conformal<R>(k, nv, av, X, G);
        for (int m = 0; m <= l; ++m) K[(long long)j * SREC + sample_map_index(m, l)] = G[m];
    }
    for (int q = 0; q < 3; ++q) K[(long long)j * SREC + 45 + q] = su.a[q][j];
}

// level of halo node level z in the two-warp accumulation halo, for writes made
// after both warps finished their phases: levels 0..3 are warp 0's, 4..5 warp 1's
__device__ __forceinline__ int ulevel(int z) { return z <= 3 ? z : z + 2; }

// separable scatter of a 3x3 M (u_q += sum_e M_qe dN/dx_e) into the two-warp
// accumulation halo with shared atomics (samples in the exact mode only)
template <typename R>
__device__ __forceinline__ void scatter_sep_u(R (*ua)[UN], const int* lc, const R (*w)[3], const R (*dw)[3], const R* M) {
#pragma unroll
    for (int q = 0; q < 3; ++q)
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const R A0 = M[3 * q] * dw[0][a], A1 = M[3 * q + 1] * w[0][a], A2 = M[3 * q + 2] * w[0][a];
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                const R B0 = A0 * w[1][b] + A1 * dw[1][b], B1 = A2 * w[1][b];
#pragma unroll
                for (int c = 0; c < 3; ++c)
                    atomicAdd(&ua[q][pidx(lc[0] + a, lc[1] + b, ulevel(lc[2] + c))], B0 * w[2][c] + B1 * dw[2][c]);
            }
        }
}

// Solid particles, viscous liquid particles, and (in the exact mode) surface
// samples. One CTA per block of the compact list, one thread per cell, two warps:
// a thread's general particles share its cell's 27 nodes, so their node values
// add up in registers (the stencil is taken relative to the cell, t clamped to
// [0, 1], as in k_apply_pair), and each warp writes them once per cell into its
// own accumulation levels in conflict-free phases. EXACT_SOLID: solids take the
// exact dP (exact mode with solid buffers), else their projected 9x9 map.
template <typename R, bool EXACT_SOLID>
__global__ void __launch_bounds__(NT_CELL, sizeof(R) == 4 ? 8 : 4) k_apply_general(ApplyArgs<R> a) {
    __shared__ R ph[3][PN];
    __shared__ __align__(16) R ua[3][UN];
    const int w = a.gen_list[blockIdx.x];
    const int slot = a.work[w];
    const long long gb = a.work_gb[w];
    const int4 bc = a.coord[slot];
    if (a.check_done && a.scal[bc.w].cg_done) return;
    const SceneDev& S = a.sc[bc.w];
    for (int i = threadIdx.x; i < (int)(3 * UN * sizeof(R) / 16); i += blockDim.x)
        reinterpret_cast<int4*>(&ua[0][0])[i] = make_int4(0, 0, 0, 0);
    for (int yz = threadIdx.x; yz < HE * HE; yz += blockDim.x) {
        const int hy = yz % HE, hz = yz / HE;
        int nmid, nlo, nhi, base;
        halo_row<R>(a.nbr, slot, hy, hz, nmid, nlo, nhi, base);
        const int h0 = pidx(0, hy, hz);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const R* src = a.p + nmid * 192 + c * 64 + base;
            ph[c][h0] = nlo >= 0 ? a.p[nlo * 192 + c * 64 + base + 3] : R(0);
#pragma unroll
            for (int k = 0; k < 4; ++k) ph[c][h0 + 1 + k] = nmid >= 0 ? src[k] : R(0);
            ph[c][h0 + 5] = nhi >= 0 ? a.p[nhi * 192 + c * 64 + base] : R(0);
        }
    }
    __syncthreads();
    const R dt = (R)S.dt, inv_dx = (R)S.inv_dx;
    const int cell = threadIdx.x, wid = threadIdx.x >> 5;
    const int lx = cell & 3, ly = (cell >> 2) & 3, lz = cell >> 4;
    const int lc[3] = {lx, ly, lz};
    KSum<R> pap;
    R acc[3][3][3][3];
#pragma unroll
    for (int m = 0; m < 81; ++m) (&acc[0][0][0][0])[m] = R(0);
    bool any = false;
    if (a.slot_gen[slot] > 0) {
        const int cb = a.cell_start[gb * 64 + cell], ce = a.cell_start[gb * 64 + cell + 1];
        for (int i = cb; i < ce; ++i) {
            if (!(a.phase[i] != 0 || a.cvisc[i] != R(0))) continue;
            any = true;
            R wgt[3][3], dw[3][3];
            {
                const R tt[3] = {fmin(fmax(a.pu.a[0][i] - R(lx), R(0)), R(1)), fmin(fmax(a.pu.a[1][i] - R(ly), R(0)), R(1)),
                                 fmin(fmax(a.pu.a[2][i] - R(lz), R(0)), R(1))};
#pragma unroll
                for (int ax = 0; ax < 3; ++ax) {
                    bspline<R>(tt[ax] + R(0.5), wgt[ax], dw[ax]);
#pragma unroll
                    for (int k = 0; k < 3; ++k) dw[ax][k] *= inv_dx;
                }
            }
            R dL[9];
            gather_grad_sep<R>(ph, lc, wgt, dw, dL);
            R M[9];
            if (a.phase[i] == 0) {
                const R s = a.kappa[i] * (dL[0] + dL[4] + dL[8]);
                const R cv = a.cvisc[i];
#pragma unroll
                for (int q = 0; q < 3; ++q)
#pragma unroll
                    for (int e = 0; e < 3; ++e) M[3 * q + e] = cv * R(0.5) * (dL[3 * q + e] + dL[3 * e + q]) + (q == e ? s : R(0));
            } else if (!EXACT_SOLID) {
                // projected: the particle's per-iterate 9x9 map
#pragma unroll
                for (int m = 0; m < 9; ++m) M[m] = R(0);
#pragma unroll
                for (int m = 0; m < 9; ++m)
#pragma unroll
                    for (int l = m; l < 9; ++l) {
                        const R kml = a.pK.a[sym9(m, l)][i];
                        M[m] += kml * dL[l];
                        if (l != m) M[l] += kml * dL[m];
                    }
            } else {
                R Fo[9], Fc[9], Rm[9], K[6], dF[9], dP[9];
#pragma unroll
                for (int q = 0; q < 9; ++q) {
                    Fo[q] = a.Fn.a[q][i];
                    Fc[q] = a.scache.a[q][i];
                    Rm[q] = a.scache.a[9 + q][i];
                }
#pragma unroll
                for (int q = 0; q < 6; ++q) K[q] = a.scache.a[18 + q][i];
                matmul3<R>(dL, Fo, dF);
                fcr_dP<R>(Fc, Rm, K, a.lmu[i], a.llam[i], dF, dP);
                matmul3_bt<R>(dP, Fo, M);
                const R sc = dt * dt * (R)a.V0[i];
#pragma unroll
                for (int q = 0; q < 9; ++q) M[q] *= sc;
            }
            R md = R(0);
#pragma unroll
            for (int q = 0; q < 9; ++q) md += M[q] * dL[q];
            pap.add(md);
#pragma unroll
            for (int q = 0; q < 3; ++q)
#pragma unroll
                for (int aa = 0; aa < 3; ++aa) {
                    const R A0 = M[3 * q] * dw[0][aa], A1 = M[3 * q + 1] * wgt[0][aa], A2 = M[3 * q + 2] * wgt[0][aa];
#pragma unroll
                    for (int bb = 0; bb < 3; ++bb) {
                        const R B0 = A0 * wgt[1][bb] + A1 * dw[1][bb], B1 = A2 * wgt[1][bb];
#pragma unroll
                        for (int cc = 0; cc < 3; ++cc) acc[q][aa][bb][cc] += B0 * wgt[2][cc] + B1 * dw[2][cc];
                    }
                }
        }
    }
    if (__any_sync(0xffffffffu, any)) {
#pragma unroll
        for (int q = 0; q < 3; ++q) rmw_phases<R>(ua[q], acc[q], lx, ly, lz + 2 * wid);
    }
    if (!a.samples_in_cell) {
        // samples (exact mode, or maps not current), after both warps' phases
        __syncthreads();
        const int sbeg = a.scell_start[gb * 64], nsm = a.scell_start[gb * 64 + 64] - sbeg;
        for (int k = threadIdx.x; k < nsm; k += blockDim.x) {
            const int j = sbeg + k;
            int slc[3];
            R wgt[3][3], dw[3][3];
            make_stencil_local<R>(a.su.a[0][j], a.su.a[1][j], a.su.a[2][j], inv_dx, slc, wgt, dw);
            R dFh[9];
            gather_grad_sep<R>(ph, slc, wgt, dw, dFh);
            R G[9];
            sample_G<R>(a, j, dFh, dt, G);
            R gd = R(0);
#pragma unroll
            for (int q = 0; q < 9; ++q) gd += G[q] * dFh[q];
            pap.add(gd);
            scatter_sep_u<R>(ua, slc, wgt, dw, G);
        }
    }
    if (a.pap) {
        const double v = pap.warp_total();
        if ((threadIdx.x & 31) == 0 && v != 0.0) atomicAdd(&a.scal[bc.w].pAp, v);
    }
    __syncthreads();
    flush_halo_rows_u<R>(a.nbr, slot, ua, a.u);
}

// Compact list of the work blocks that hold surface samples or general particles.
__global__ void k_gen_flags(int nw, const int* __restrict__ work, const int* __restrict__ work_gb,
                            const int* __restrict__ scell_start, const int* __restrict__ slot_gen, int* __restrict__ flag,
                            int* __restrict__ flag_g) {
    int w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= nw) return;
    long long gb = work_gb[w];
    const bool gen = slot_gen[work[w]] > 0;
    flag[w] = (scell_start[gb * 64 + 64] > scell_start[gb * 64] || gen) ? 1 : 0;
    flag_g[w] = gen ? 1 : 0;
}

__global__ void k_gen_list(int nw, const int* __restrict__ flag, const int* __restrict__ pos, int* __restrict__ list) {
    int w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= nw || !flag[w]) return;
    list[pos[w]] = w;
}

// Surface samples of the float64 objective / gradient and of the line search:
// one warp per block holding samples, padded float64 halos, separable
// gather and scatter (k_eval and k_linesearch leave the samples to these).
template <typename RS>
__global__ void __launch_bounds__(32) k_eval_surf(EvalArgs<RS> a) {
    __shared__ double ph[3][PN];
    __shared__ double ga[3][PN];
    const int w = blockIdx.x;
    const int slot = a.work[w];
    const long long gb = a.work_gb[w];
    const int4 bc = a.coord[slot];
    const SceneDev& S = a.sc[bc.w];
    if (a.skip_done && a.scal[bc.w].newton_done) return;
    const int sbeg = a.scell_start[gb * 64], send = a.scell_start[gb * 64 + 64];
    if (send == sbeg) return;
    load_halo_rows<double>(a.nbr, slot, a.gv, ph, ga);
    __syncthreads();
    const double dt = S.dt;
    double esum = 0.0;
    for (int j = sbeg + threadIdx.x; j < send; j += 32) {
        const double p[3] = {a.s.a[0][j], a.s.a[1][j], a.s.a[2][j]};
        int lc[3];
        double wgt[3][3], dw[3][3], f[3];
        stencil_in_block<double>(p, S, bc, lc, wgt, dw, f);
        double L[9];
        gather_grad_sep<double>(ph, lc, wgt, dw, L);
        double Fh[9];
#pragma unroll
        for (int q = 0; q < 9; ++q) Fh[q] = dt * L[q] + ((q % 4 == 0) ? 1.0 : 0.0);
        const double av[3] = {a.dA.a[0][j], a.dA.a[1][j], a.dA.a[2][j]};
        double C[9];
        cofactor<double>(Fh, C);
        const double cv[3] = {C[0] * av[0] + C[1] * av[1] + C[2] * av[2], C[3] * av[0] + C[4] * av[1] + C[5] * av[2],
                              C[6] * av[0] + C[7] * av[1] + C[8] * av[2]};
        const double cn = sqrt(cv[0] * cv[0] + cv[1] * cv[1] + cv[2] * cv[2]);
        const double k = a.gamma[j];
        esum += k * cn;
        const double ic = 1.0 / cn;
        const double nv[3] = {cv[0] * ic, cv[1] * ic, cv[2] * ic};
        if (a.want_cache) {
#pragma unroll
            for (int q = 0; q < 9; ++q) a.sF.a[q][j] = (RS)Fh[q];
#pragma unroll
            for (int q = 0; q < 3; ++q) a.sn.a[q][j] = (RS)nv[q];
            a.sic[j] = (RS)ic;
        }
        if (a.want_grad) {
            double G[9];
            surf_G<double>(k * dt, nv, Fh, av, G);
            scatter_sep<double>(ga, lc, wgt, dw, G);
        }
    }
    esum = warp_sum(esum);
    if (threadIdx.x == 0 && esum != 0.0) atomicAdd(&a.scal[bc.w].phi_part, esum);
    if (a.want_grad) {
        __syncthreads();
        flush_halo_rows<double>(a.nbr, slot, ga, a.grad);
    }
}

// ======================================================================
// float64 objective / gradient and line search of non-viscous liquid particles,
// thread per cell, with the per-cell polynomial form of the operator:
// tr L(t) = (1/dx) sum C_ijk t^ijk from the iterate's stencil values, and the
// gradient dt lambda (J - 1) J^n V0 gradN_i scattered through 26 moments.
// ======================================================================
struct EvalCellArgs {
    const int *work, *work_gb, *nbr, *cell_start;
    const int4* coord;
    const SceneDev* sc;
    SceneScal* scal;
    const double* gv;
    double* grad;             // null: energy only
    double* grad_l;           // null, or a second target for the same (liquid) gradient
    const double *x0, *x1, *x2, *J, *V0;
    const uint8_t* phase;
    int skip_done;
};

__device__ __forceinline__ void cell_t(const SceneDev& S, int4 bc, int lx, int ly, int lz, double x0, double x1,
                                       double x2, double& tx, double& ty, double& tz) {
    tx = fmin(fmax((x0 - S.origin[0]) * S.inv_dx - (double)(bc.x * BS + lx), 0.0), 1.0);
    ty = fmin(fmax((x1 - S.origin[1]) * S.inv_dx - (double)(bc.y * BS + ly), 0.0), 1.0);
    tz = fmin(fmax((x2 - S.origin[2]) * S.inv_dx - (double)(bc.z * BS + lz), 0.0), 1.0);
}

__global__ void __launch_bounds__(NT_CELL) k_eval_cell(EvalCellArgs a) {
    __shared__ double ph[3][PN];
    __shared__ __align__(16) double ga[3][UN];
    __shared__ double red[NT_CELL / 32];
    int w = blockIdx.x;
    int slot = a.work[w];
    long long gb = a.work_gb[w];
    int4 bc = a.coord[slot];
    const SceneDev& S = a.sc[bc.w];
    if (a.skip_done && a.scal[bc.w].newton_done) return;
    if (S.mu_l != 0.0) return;   // viscous scene: k_eval takes every particle
    for (int i = threadIdx.x; i < (int)(3 * UN * sizeof(double) / 16); i += blockDim.x)
        reinterpret_cast<int4*>(&ga[0][0])[i] = make_int4(0, 0, 0, 0);
    for (int yz = threadIdx.x; yz < HE * HE; yz += blockDim.x) {
        const int hy = yz % HE, hz = yz / HE;
        int nmid, nlo, nhi, base;
        halo_row<double>(a.nbr, slot, hy, hz, nmid, nlo, nhi, base);
        const int h0 = pidx(0, hy, hz);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            ph[c][h0] = nlo >= 0 ? a.gv[nlo * 192 + c * 64 + base + 3] : 0.0;
#pragma unroll
            for (int m = 0; m < 4; ++m) ph[c][h0 + 1 + m] = nmid >= 0 ? a.gv[nmid * 192 + c * 64 + base + m] : 0.0;
            ph[c][h0 + 5] = nhi >= 0 ? a.gv[nhi * 192 + c * 64 + base] : 0.0;
        }
    }
    __syncthreads();
    const int cell = threadIdx.x;
    const int lx = cell & 3, ly = (cell >> 2) & 3, lz = cell >> 4;
    const int cbeg = a.cell_start[gb * 64 + cell], cend = a.cell_start[gb * 64 + cell + 1];
    const double dt = S.dt, lam = S.lambda_l, inv_dx = S.inv_dx;
    double esum = 0.0;
    double M[3][3][3];
#pragma unroll
    for (int q = 0; q < 27; ++q) (&M[0][0][0])[q] = 0.0;
    bool any = false;
    if (cend > cbeg) {
        double C[3][3][3];
#pragma unroll
        for (int q = 0; q < 27; ++q) (&C[0][0][0])[q] = 0.0;
        cell_coefficients<double>(ph, lx, ly, lz, C);
        for (int i = cbeg; i < cend; ++i) {
            if (a.phase[i] != 0) continue;
            any = true;
            double tx, ty, tz;
            cell_t(S, bc, lx, ly, lz, a.x0[i], a.x1[i], a.x2[i], tx, ty, tz);
            // monomials factored as t_x^i (t_y^j t_z^k): the y-z products serve the
            // evaluation and the moments
            const double py[3] = {1.0, ty, ty * ty}, pz[3] = {1.0, tz, tz * tz};
            double yz[3][3];
#pragma unroll
            for (int j = 0; j < 3; ++j)
#pragma unroll
                for (int k = 0; k < 3; ++k) yz[j][k] = py[j] * pz[k];
            double srow[3] = {0.0, 0.0, 0.0};
#pragma unroll
            for (int ii = 0; ii < 3; ++ii)
#pragma unroll
                for (int j = 0; j < 3; ++j)
#pragma unroll
                    for (int k = 0; k < 3; ++k)
                        if (!(ii == 2 && j == 2 && k == 2)) srow[ii] += C[ii][j][k] * yz[j][k];
            double tr = inv_dx * (srow[0] + tx * (srow[1] + tx * srow[2]));
            double Jn = a.J[i], v0 = a.V0[i];
            double jm1 = (Jn - 1.0) + dt * tr * Jn;
            esum += 0.5 * lam * jm1 * jm1 * v0;
            double sp = dt * lam * jm1 * Jn * v0 * inv_dx;
            const double sx[3] = {sp, sp * tx, sp * tx * tx};
#pragma unroll
            for (int ii = 0; ii < 3; ++ii)
#pragma unroll
                for (int j = 0; j < 3; ++j)
#pragma unroll
                    for (int k = 0; k < 3; ++k)
                        if (!(ii == 2 && j == 2 && k == 2)) M[ii][j][k] += sx[ii] * yz[j][k];
        }
    }
    // every lane of a warp takes part in its scatter phases (empty cells add zeros)
    if (a.grad && __any_sync(0xffffffffu, any)) cell_scatter_warp<double>(M, ga, lx, ly, lz + 2 * (threadIdx.x >> 5));
    block_atomic_sum<NT_CELL>(esum, &a.scal[bc.w].phi_part, red);
    if (a.grad) {
        __syncthreads();
        flush_halo_rows_u<double>(a.nbr, slot, ga, a.grad);
        if (a.grad_l) flush_halo_rows_u<double>(a.nbr, slot, ga, a.grad_l);
    }
}

// Line search, liquid part. The liquid energy is exactly quadratic along a
// Newton direction d (J is affine in v), so its change over a step alpha is
// alpha g_l . d + alpha^2/2 d.K_l d, with g_l the float64 liquid gradient at the
// iterate (k_eval_cell keeps a copy) and d.K_l d = sum_p kappa_p (tr L_d)_p^2,
// a sum of non-negative terms formed here in the operator type.
template <typename R>
__global__ void __launch_bounds__(NT_CELL) k_curv_cell(ApplyArgs<R> a) {
    __shared__ R ph[3][PN];
    __shared__ R ua[3][PN];
    __shared__ double red[NT_CELL / 32];
    int w = blockIdx.x;
    int slot = a.work[w];
    long long gb = a.work_gb[w];
    int4 bc = a.coord[slot];
    const SceneDev& S = a.sc[bc.w];
    if (a.scal[bc.w].newton_done) return;
    const int rows = a.wrows[w];
    if (rows == 0) return;
    load_halo_rows<R>(a.nbr, slot, a.p, ph, ua);
    __syncthreads();
    const R inv_dx = (R)S.inv_dx;
    const int cell = threadIdx.x;
    const int lx = cell & 3, ly = (cell >> 2) & 3, lz = cell >> 4;
    const int n = a.cell_start[gb * 64 + cell + 1] - a.cell_start[gb * 64 + cell];
    // the cell's values in the pair-interleaved rows (k_pack_volume)
    const R* recs = reinterpret_cast<const R*>(a.opk + (long long)a.wroff[w] * 64) + 8 * (cell >> 1) + (cell & 1);
    R acc = R(0);
    if (n > 0) {
        R C[3][3][3];
#pragma unroll
        for (int q = 0; q < 27; ++q) (&C[0][0][0])[q] = R(0);
        cell_coefficients<R>(ph, lx, ly, lz, C);
        for (int r = 0; r < n; ++r) {
            const R* rr = recs + (long long)r * 256;
            R4<R> rec;
            rec.x = rr[0];
            rec.y = rr[2];
            rec.z = rr[4];
            rec.w = rr[6];
            if (rec.w < R(0)) continue;
            R tx = fmin(fmax(rec.x - R(lx), R(0)), R(1));
            R ty = fmin(fmax(rec.y - R(ly), R(0)), R(1));
            R tz = fmin(fmax(rec.z - R(lz), R(0)), R(1));
            R py[3] = {R(1), ty, ty * ty}, pz[3] = {R(1), tz, tz * tz};
            R srow[3] = {R(0), R(0), R(0)};
#pragma unroll
            for (int ii = 0; ii < 3; ++ii)
#pragma unroll
                for (int j = 0; j < 3; ++j)
#pragma unroll
                    for (int kk = 0; kk < 3; ++kk)
                        if (!(ii == 2 && j == 2 && kk == 2)) srow[ii] += C[ii][j][kk] * (py[j] * pz[kk]);
            const R tr = inv_dx * (srow[0] + tx * (srow[1] + tx * srow[2]));
            acc += rec.w * tr * tr;
        }
    }
    block_atomic_sum<NT_CELL>((double)acc, const_cast<double*>(&a.scal[bc.w].dkd), red);
}

// ======================================================================
// Jacobi preconditioner of the momentum CG: 1 / m_i on unknown components.
// (Adding the liquid stiffness diagonal sum_p kappa_p (dN_i/dx_a)^2 was measured
// to raise the CG count on the inclined droplets, 170 -> 202 per step: the
// grad-div stiffness leaves divergence-free modes at the mass scale.)
// ======================================================================
// pinv = 1 / (m + pinv) on unknown components (pinv holds zero on entry), 0 elsewhere
template <typename R>
__global__ void k_pinv(int nb, const int4* __restrict__ coord, const SceneDev* __restrict__ sc,
                       const double* __restrict__ gm, const uint8_t* __restrict__ pcode, R* __restrict__ pinv,
                       R* __restrict__ mR) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nb * 64) return;
    int slot = t >> 6, l = t & 63;
    double m = gm[t];
    mR[t] = (R)m;
    uint8_t code = pcode[t];
    for (int c = 0; c < 3; ++c) {
        int k = slot * 192 + c * 64 + l;
        double dg = m + (double)pinv[k];   // pinv holds the stiffness diagonal on entry
        pinv[k] = (m > 0.0 && !(code & PC_FIXED)) ? (R)(1.0 / dg) : R(0);
    }
}

// ======================================================================
// CG vector kernels (one 64-thread CTA per slot; NC = 3 momentum, 1 heat)
// ======================================================================
template <typename R, int NC>
struct CGArgs {
    const int4* coord;
    const SceneDev* sc;
    SceneScal* scal;
    const uint8_t* pcode;     // NC == 3
    const R* inv;             // inverse diagonal (0 = not an unknown)
    const double* gm;         // NC == 3: mass diagonal
    const R* mR;              // NC == 3: mass diagonal in R
    R *x, *r, *p, *u;
    const double* rhs_d;      // for init: b = sign * rhs (double)
    double rhs_sign;
    const R* pinv3;           // NC == 3: inverse diagonal of the projected Hessian, per component
};

// preconditioner entry of node t, component c
template <typename R, int NC>
__device__ __forceinline__ R cg_prec(const CGArgs<R, NC>& a, int slot, int c, int l, int t) {
    if (NC == 3) return a.pinv3[slot * 192 + c * 64 + l];
    return a.inv[t];
}

template <typename R, int NC>
__device__ __forceinline__ void cg_proj(R* v, const CGArgs<R, NC>& a, int t, const SceneDev& S) {
    if (NC == 3) project3r<R>(v, a.pcode[t], S, a.coord[t >> 6], t & 63);
    else if (a.inv[t] == R(0)) v[0] = R(0);
}

template <typename R, int NC>
__device__ __forceinline__ int vidx(int slot, int q, int l) { return NC == 3 ? slot * 192 + q * 64 + l : slot * 64 + l; }

constexpr int CG_SLOTS = 8;             // grid slots per CTA
constexpr int CG_NT = CG_SLOTS * 64;
constexpr int OFF_RR = offsetof(SceneScal, rr) / 8, OFF_RZ = offsetof(SceneScal, rz) / 8,
              OFF_RZN = offsetof(SceneScal, rz_new) / 8, OFF_PAP = offsetof(SceneScal, pAp) / 8,
              OFF_BN = offsetof(SceneScal, bnorm) / 8;

// Per-scene sums of two values over the CTA: warp sums, then one float64 atomic
// per run of equal scenes (slots are ordered scene by scene). scene < 0: no slot.
__device__ __forceinline__ void cta_scene_sum2_warp(double v1, double v2, int scene, SceneScal* scal, int off1, int off2);
__device__ __forceinline__ void cta_scene_sum2(double v1, double v2, int scene, SceneScal* scal, int off1, int off2) {
    cta_scene_sum2_warp(warp_sum(v1), warp_sum(v2), scene, scal, off1, off2);
}

// same, from warp totals held by lane 0 of each warp
__device__ __forceinline__ void cta_scene_sum2_warp(double v1, double v2, int scene, SceneScal* scal, int off1, int off2) {
    __shared__ double s1[CG_NT / 32], s2[CG_NT / 32];
    __shared__ int sid[CG_NT / 32];
    int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        s1[w] = v1;
        s2[w] = v2;
        sid[w] = scene;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int cur = -1;
        double a1 = 0.0, a2 = 0.0;
        for (int k = 0; k <= CG_NT / 32; ++k) {
            int sk = k < CG_NT / 32 ? sid[k] : -2;
            if (sk != cur) {
                if (cur >= 0) {
                    double* base = reinterpret_cast<double*>(&scal[cur]);
                    if (off1 >= 0 && a1 != 0.0) atomicAdd(base + off1, a1);
                    if (off2 >= 0 && a2 != 0.0) atomicAdd(base + off2, a2);
                }
                cur = sk;
                a1 = a2 = 0.0;
            }
            if (k < CG_NT / 32) {
                a1 += s1[k];
                a2 += s2[k];
            }
        }
    }
}

// r = P b, x = 0, z = P(inv r), p = z, u = 0; rz, bnorm (if requested)
template <typename R, int NC>
__global__ void __launch_bounds__(CG_NT) k_cg_init(CGArgs<R, NC> a, int nb, int set_bnorm, int fused_pap) {
    int slot = blockIdx.x * CG_SLOTS + (threadIdx.x >> 6), l = threadIdx.x & 63;
    int scene = -1;
    double bb = 0.0, rz = 0.0;
    if (slot < nb) {
        scene = a.coord[slot].w;
        const SceneDev& S = a.sc[scene];
        if (!a.scal[scene].cg_done) {
            int t = slot * 64 + l;
            R r[NC];
#pragma unroll
            for (int q = 0; q < NC; ++q) r[q] = (R)(a.rhs_sign * a.rhs_d[vidx<R, NC>(slot, q, l)]);
            cg_proj<R, NC>(r, a, t, S);
            R z[NC];
#pragma unroll
            for (int q = 0; q < NC; ++q) z[q] = r[q] * cg_prec<R, NC>(a, slot, q, l, t);
            cg_proj<R, NC>(z, a, t, S);
            R bbl = R(0), rzl = R(0);   // the node's products in R; sums across nodes in float64
#pragma unroll
            for (int q = 0; q < NC; ++q) {
                int k = vidx<R, NC>(slot, q, l);
                a.r[k] = r[q];
                a.x[k] = R(0);
                a.p[k] = z[q];
                a.u[k] = R(0);
                bbl += r[q] * r[q];
                rzl += r[q] * z[q];
            }
            bb = (double)bbl;
            rz = (double)rzl;
        }
    }
    cta_scene_sum2(rz, bb, scene, a.scal, OFF_RZ, set_bnorm ? OFF_BN : -1);
    if (NC == 3 && fused_pap) {
        // p . M p of the first direction p = z (the operator adds p . (H - M) p)
        double mpp = 0.0;
        if (slot < nb && !a.scal[scene].cg_done) {
            const int t = slot * 64 + l;
            R s = R(0);
#pragma unroll
            for (int q = 0; q < NC; ++q) {
                const R pv = a.p[vidx<R, NC>(slot, q, l)];
                s += a.mR[t] * pv * pv;
            }
            mpp = (double)s;
        }
        __syncthreads();
        cta_scene_sum2(mpp, 0.0, scene, a.scal, OFF_PAP, -1);
    }
}


// ---- one CG iteration's vector work as a single cooperative launch ----
// Each thread sums the per-node products of the nodes it visits (KSum). Warps
// stay scene-uniform (a warp covers 32 nodes of one slot and all lanes visit the
// same slots), so a change of scene flushes the warp's sums with one atomic; the
// last scene's sums go through the CTA reduction (cta_scene_sum2).
template <typename R>
struct SceneAcc {
    KSum<R> a1, a2;
    int cur = -1;
    __device__ void add(int scene, R x1, R x2, SceneScal* scal, int off1, int off2) {
        if (scene != cur) {
            flush(scal, off1, off2);
            cur = scene;
        }
        a1.add(x1);
        a2.add(x2);
    }
    __device__ void flush(SceneScal* scal, int off1, int off2) {
        if (cur < 0) return;   // warp-uniform
        double v1 = a1.warp_total(), v2 = a2.warp_total();
        if ((threadIdx.x & 31) == 0) {
            double* base = reinterpret_cast<double*>(&scal[cur]);
            if (off1 >= 0 && v1 != 0.0) atomicAdd(base + off1, v1);
            if (off2 >= 0 && v2 != 0.0) atomicAdd(base + off2, v2);
        }
        a1.clear();
        a2.clear();
    }
};

// Grid-wide barrier of a cooperative launch: bar[0] counts arrivals, bar[1] is
// the generation. The wait is bounded; on timeout ERR_TIMEOUT is set and every
// thread of the CTA gets false.
__device__ bool grid_barrier(unsigned* bar, int* err) {
    __syncthreads();
    int ok = 1;
    if (threadIdx.x == 0) {
        volatile unsigned* gen = bar + 1;
        const unsigned g = *gen;
        __threadfence();
        const unsigned arrived = atomicAdd(bar, 1u);
        if (arrived == gridDim.x - 1) {
            atomicExch(bar, 0u);
            __threadfence();
            atomicAdd(bar + 1, 1u);
        } else {
            long long it = 0;
            while (*gen == g) {
                if (++it > (1LL << 24)) {
                    ok = 0;
                    atomicOr(err, ERR_TIMEOUT);
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
    }
    return __syncthreads_and(ok) != 0;
}

// per-scene CG control: count, test, beta (held in alpha)
__device__ __forceinline__ void cg_check_scene(SceneScal& c, const SceneDev& S, int heat) {
    if (c.cg_done) return;
    c.cg_it += 1;
    double rtol = heat ? S.heat_rtol : S.cg_rtol;
    bool done = !(c.pAp > 0.0) || c.rr <= rtol * rtol * c.bnorm || c.cg_it >= S.max_cg;
    if (done) {
        c.cg_done = 1;
    } else {
        c.alpha = c.rz_new / c.rz;
        c.rz = c.rz_new;
    }
    c.rz_new = 0.0;
    c.rr = 0.0;
    c.pAp = 0.0;
}

// After the operator apply u = K p:
//   A: q = P (D p + u) -> u, pAp
//   B: x += alpha p, r -= alpha q, u = 0, z = P(inv r); rz_new, rr
//      (non-positive curvature: x = p on the first iteration, then stop)
//   C: per-scene control
//   D: p = z + beta p
template <typename R, int NC>
__global__ void __launch_bounds__(CG_NT, 3) k_cg_iter(CGArgs<R, NC> a, int nb, int nsc, int heat, unsigned* bar, int* err) {
    const int nchunks = (nb + CG_SLOTS - 1) / CG_SLOTS;
    const int l = threadIdx.x & 63;
    SceneAcc<R> acc;
    for (int ch = blockIdx.x; ch < nchunks; ch += gridDim.x) {
        const int slot = ch * CG_SLOTS + (threadIdx.x >> 6);
        if (slot >= nb) continue;
        const int scene = a.coord[slot].w;
        const SceneDev& S = a.sc[scene];
        R pql = R(0);   // the node's products in R
        if (!a.scal[scene].cg_done) {
            const int t = slot * 64 + l;
            R q[NC], pv[NC];
            R diag;
            if (NC == 3) diag = a.mR[t];
            else diag = a.inv[t] == R(0) ? R(0) : R(1) / a.inv[t];
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                const int k = vidx<R, NC>(slot, c, l);
                pv[c] = a.p[k];
                q[c] = diag * pv[c] + a.u[k];
            }
            cg_proj<R, NC>(q, a, t, S);
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                a.u[vidx<R, NC>(slot, c, l)] = q[c];
                pql += pv[c] * q[c];
            }
        }
        acc.add(scene, pql, R(0), a.scal, OFF_PAP, -1);
    }
    cta_scene_sum2_warp(acc.a1.warp_total(), acc.a2.warp_total(), acc.cur, a.scal, OFF_PAP, -1);
    if (!grid_barrier(bar, err)) return;
    acc.a1.clear();
    acc.a2.clear();
    acc.cur = -1;
    int ascene = -1;
    R alpha = R(0);
    bool curv_ok = true;
    for (int ch = blockIdx.x; ch < nchunks; ch += gridDim.x) {
        const int slot = ch * CG_SLOTS + (threadIdx.x >> 6);
        if (slot >= nb) continue;
        const int scene = a.coord[slot].w;
        const SceneDev& S = a.sc[scene];
        const SceneScal& sc = a.scal[scene];
        R rzl = R(0), rrl = R(0);
        if (!sc.cg_done) {
            const int t = slot * 64 + l;
            if (scene != ascene) {   // once per scene change, not per node
                const double pAp = sc.pAp;
                curv_ok = pAp > 0.0;
                alpha = curv_ok ? (R)sc.rz / (R)pAp : R(0);   // the step is applied in R
                ascene = scene;
            }
            if (!curv_ok) {
                if (sc.cg_it == 0) {
#pragma unroll
                    for (int c = 0; c < NC; ++c) {
                        const int k = vidx<R, NC>(slot, c, l);
                        a.x[k] = a.p[k];
                    }
                }
#pragma unroll
                for (int c = 0; c < NC; ++c) a.u[vidx<R, NC>(slot, c, l)] = R(0);
            } else {
                R r[NC], z[NC];
#pragma unroll
                for (int c = 0; c < NC; ++c) {
                    const int k = vidx<R, NC>(slot, c, l);
                    a.x[k] += alpha * a.p[k];
                    r[c] = a.r[k] - alpha * a.u[k];
                    a.r[k] = r[c];
                    a.u[k] = R(0);
                }
#pragma unroll
                for (int c = 0; c < NC; ++c) z[c] = r[c] * cg_prec<R, NC>(a, slot, c, l, t);
                cg_proj<R, NC>(z, a, t, S);
#pragma unroll
                for (int c = 0; c < NC; ++c) {
                    rzl += r[c] * z[c];
                    rrl += r[c] * r[c];
                }
            }
        }
        acc.add(scene, rzl, rrl, a.scal, OFF_RZN, OFF_RR);
    }
    cta_scene_sum2_warp(acc.a1.warp_total(), acc.a2.warp_total(), acc.cur, a.scal, OFF_RZN, OFF_RR);
    if (!grid_barrier(bar, err)) return;
    if (blockIdx.x == 0)
        for (int s = threadIdx.x; s < nsc; s += blockDim.x) cg_check_scene(a.scal[s], a.sc[s], heat);
    if (!grid_barrier(bar, err)) return;
    int bscene = -1;
    R beta = R(0);
    for (int ch = blockIdx.x; ch < nchunks; ch += gridDim.x) {
        const int slot = ch * CG_SLOTS + (threadIdx.x >> 6);
        if (slot >= nb) continue;
        const int scene = a.coord[slot].w;
        const SceneDev& S = a.sc[scene];
        const SceneScal& sc = a.scal[scene];
        if (sc.cg_done) continue;
        if (scene != bscene) {
            beta = (R)sc.alpha;   // holds beta here (set by the control phase)
            bscene = scene;
        }
        const int t = slot * 64 + l;
        R z[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) z[c] = a.r[vidx<R, NC>(slot, c, l)] * cg_prec<R, NC>(a, slot, c, l, t);
        cg_proj<R, NC>(z, a, t, S);
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            const int k = vidx<R, NC>(slot, c, l);
            a.p[k] = z[c] + beta * a.p[k];
        }
    }
}

// The momentum CG iteration with p . A p already summed: the operator kernels
// add p . (H - M) p per particle and sample, and the step that formed p (the
// previous iteration's phase D, or k_cg_init) added p . M p, so the iteration
// starts at B:
//   B: q = P (M p + u) on the fly, x += alpha p, r -= alpha q, u = 0,
//      z = P(inv r); rz_new, rr
//   C: per-scene control (zeroes pAp)
//   D: p = z + beta p, and p . M p of the new p into pAp
template <typename R>
__global__ void __launch_bounds__(CG_NT, 3) k_cg_iter2(CGArgs<R, 3> a, int nb, int nsc, unsigned* bar, int* err) {
    const int nchunks = (nb + CG_SLOTS - 1) / CG_SLOTS;
    const int l = threadIdx.x & 63;
    SceneAcc<R> acc;
    int ascene = -1;
    R alpha = R(0);
    bool curv_ok = true;
    for (int ch = blockIdx.x; ch < nchunks; ch += gridDim.x) {
        const int slot = ch * CG_SLOTS + (threadIdx.x >> 6);
        if (slot >= nb) continue;
        const int scene = a.coord[slot].w;
        const SceneDev& S = a.sc[scene];
        const SceneScal& sc = a.scal[scene];
        R rzl = R(0), rrl = R(0);
        if (!sc.cg_done) {
            const int t = slot * 64 + l;
            if (scene != ascene) {   // once per scene change, not per node
                const double pAp = sc.pAp;
                curv_ok = pAp > 0.0;
                alpha = curv_ok ? (R)sc.rz / (R)pAp : R(0);
                ascene = scene;
            }
            if (!curv_ok) {
                if (sc.cg_it == 0) {
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        const int k = slot * 192 + c * 64 + l;
                        a.x[k] = a.p[k];
                    }
                }
#pragma unroll
                for (int c = 0; c < 3; ++c) a.u[slot * 192 + c * 64 + l] = R(0);
            } else {
                const R mr = a.mR[t];
                R pv[3], q[3];
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const int k = slot * 192 + c * 64 + l;
                    pv[c] = a.p[k];
                    q[c] = mr * pv[c] + a.u[k];
                }
                cg_proj<R, 3>(q, a, t, S);
                R r[3], z[3];
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const int k = slot * 192 + c * 64 + l;
                    a.x[k] += alpha * pv[c];
                    r[c] = a.r[k] - alpha * q[c];
                    a.r[k] = r[c];
                    a.u[k] = R(0);
                }
#pragma unroll
                for (int c = 0; c < 3; ++c) z[c] = r[c] * cg_prec<R, 3>(a, slot, c, l, t);
                cg_proj<R, 3>(z, a, t, S);
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    rzl += r[c] * z[c];
                    rrl += r[c] * r[c];
                }
            }
        }
        acc.add(scene, rzl, rrl, a.scal, OFF_RZN, OFF_RR);
    }
    cta_scene_sum2_warp(acc.a1.warp_total(), acc.a2.warp_total(), acc.cur, a.scal, OFF_RZN, OFF_RR);
    if (!grid_barrier(bar, err)) return;
    if (blockIdx.x == 0)
        for (int s = threadIdx.x; s < nsc; s += blockDim.x) cg_check_scene(a.scal[s], a.sc[s], 0);
    if (!grid_barrier(bar, err)) return;
    acc.a1.clear();
    acc.a2.clear();
    acc.cur = -1;
    int bscene = -1;
    R beta = R(0);
    for (int ch = blockIdx.x; ch < nchunks; ch += gridDim.x) {
        const int slot = ch * CG_SLOTS + (threadIdx.x >> 6);
        if (slot >= nb) continue;
        const int scene = a.coord[slot].w;
        const SceneDev& S = a.sc[scene];
        const SceneScal& sc = a.scal[scene];
        R mpp = R(0);
        if (!sc.cg_done) {
            if (scene != bscene) {
                beta = (R)sc.alpha;   // holds beta here (set by the control phase)
                bscene = scene;
            }
            const int t = slot * 64 + l;
            R z[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) z[c] = a.r[slot * 192 + c * 64 + l] * cg_prec<R, 3>(a, slot, c, l, t);
            cg_proj<R, 3>(z, a, t, S);
            const R mr = a.mR[t];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const int k = slot * 192 + c * 64 + l;
                const R pn = z[c] + beta * a.p[k];
                a.p[k] = pn;
                mpp += mr * pn * pn;
            }
        }
        acc.add(scene, mpp, R(0), a.scal, OFF_PAP, -1);
    }
    cta_scene_sum2_warp(acc.a1.warp_total(), acc.a2.warp_total(), acc.cur, a.scal, OFF_PAP, -1);
}

__global__ void k_cg_begin(SceneScal* scal, int nsc, int from_newton) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nsc) return;
    SceneScal& c = scal[s];
    c.cg_done = from_newton ? c.newton_done : 0;
    c.cg_it = 0;
    c.rz = c.rz_new = c.rr = c.pAp = c.bnorm = 0.0;
}

// ======================================================================
// Newton control
// ======================================================================
__global__ void k_newton_begin(SceneScal* scal, int nsc) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nsc) return;
    SceneScal& c = scal[s];
    c.newton_it = 0;
    c.newton_done = 0;
    c.cg_total = 0;
    c.status = 0;
    c.r0 = -1.0;
    c.rnorm = 0.0;
}

__global__ void k_newton_iter_begin(SceneScal* scal, int nsc) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nsc) return;
    SceneScal& c = scal[s];
    if (c.newton_done) return;
    c.rr = 0.0;
    c.phi_kin = 0.0;
    c.phi_part = 0.0;
    c.slope = 0.0;
    c.dkd = 0.0;
    for (int k = 0; k < MAX_LS; ++k) c.dphi[k] = 0.0;
}

__global__ void k_newton_check(SceneScal* scal, const SceneDev* sc, int nsc) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nsc) return;
    SceneScal& c = scal[s];
    if (c.newton_done) return;
    c.rnorm = sqrt(c.rr);
    if (c.r0 < 0.0) c.r0 = c.rnorm;
    if (c.rnorm <= sc[s].newton_tol * fmax(c.r0, 1e-12)) c.newton_done = 1;
    else if (c.newton_it >= sc[s].max_newton) {
        c.newton_done = 1;
        c.status = MPM_ERR_NOT_CONVERGED;
    }
    if (!isfinite(c.rnorm)) {
        c.newton_done = 1;
        c.status = MPM_ERR_NUMERIC;
    }
}

// v = P (v^n + dt g)
__global__ void k_newton_init_v(const int4* __restrict__ coord, const SceneDev* __restrict__ sc, const double* __restrict__ gvn,
                                const uint8_t* __restrict__ pcode, double* __restrict__ gv) {
    int slot = blockIdx.x, l = threadIdx.x;
    int4 bc = coord[slot];
    const SceneDev& S = sc[bc.w];
    int t = slot * 64 + l;
    double v[3];
    for (int q = 0; q < 3; ++q) v[q] = gvn[slot * 192 + q * 64 + l] + S.dt * S.g[q];
    project3(v, pcode[t], S, bc, l);
    for (int q = 0; q < 3; ++q) gv[slot * 192 + q * 64 + l] = v[q];
}

// line search: per-particle energy differences for alpha_k = 2^-k in one pass
template <typename R>
struct LSArgs {
    const int *work, *work_gb, *nbr, *cell_start, *scell_start;
    const int4* coord;
    const SceneDev* sc;
    SceneScal* scal;
    const double* gv;
    const R* d;
    Ptrs3 x;
    const double *J, *V0, *T;
    Ptrs9 F;
    const uint8_t* phase;
    Ptrs3 s, dA;
    const double* gamma;
    int skip_poly;             // non-viscous liquid particles take the closed form (k_curv_cell)
    int skip_samples;          // surface samples are left to k_ls_surf
    const int* slot_gen;
    int k0, k1;                // trials k0..k1-1 (alpha = 2^-k) of this pass; a pass with k0 > 0 runs
                               // only for scenes whose earlier trials all failed (ls_pick < 0)
};

// R: arithmetic type; RD: type of the Newton direction
template <typename R, typename RD>
__global__ void __launch_bounds__(NT) k_linesearch(LSArgs<RD> a) {
    __shared__ R vh[3][HN];
    __shared__ R dh[3][HN];
    __shared__ double red[NT / 32];
    int w = blockIdx.x;
    int slot = a.work[w];
    long long gb = a.work_gb[w];
    int4 bc = a.coord[slot];
    const SceneDev& S = a.sc[bc.w];
    SceneScal& scl = a.scal[bc.w];
    if (scl.newton_done || (a.k0 > 0 && scl.ls_pick >= 0)) return;
    const bool poly = a.skip_poly && S.mu_l == 0.0;
    const bool no_samples = a.skip_samples || a.scell_start[gb * 64] == a.scell_start[gb * 64 + 64];
    if (poly && a.slot_gen[slot] == 0 && no_samples) return;
    load_halo_vec_d<R>(a.nbr, slot, a.gv, vh);
    for (int t = threadIdx.x; t < 3 * HN; t += blockDim.x) {
        int c = t / HN, h = t % HN;
        int ns, loc;
        halo_source(a.nbr, slot, h, ns, loc);
        dh[c][h] = ns < 0 ? R(0) : (R)a.d[ns * 192 + c * 64 + loc];
    }
    __syncthreads();
    const int nls = S.max_ls < MAX_LS ? S.max_ls : MAX_LS;
    const int k1 = a.k1 < nls ? a.k1 : nls;
    const double alpha0 = ldexp(1.0, -a.k0);
    const R dt = (R)S.dt;
    double de[MAX_LS];
#pragma unroll
    for (int k = 0; k < MAX_LS; ++k) de[k] = 0.0;
    int beg = a.cell_start[gb * 64], end = a.cell_start[gb * 64 + 64];
    if (poly && a.slot_gen[slot] == 0) end = beg;
    for (int i = beg + threadIdx.x; i < end; i += NT) {
        if (poly && a.phase[i] == 0) continue;   // k_ls_cell
        double p[3] = {a.x.a[0][i], a.x.a[1][i], a.x.a[2][i]};
        int lc[3];
        R wgt[3][3], dw[3][3], f[3];
        stencil_in_block<R>(p, S, bc, lc, wgt, dw, f);
        R L[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0}, D[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
        for (int cz = 0; cz < 3; ++cz)
            for (int cy = 0; cy < 3; ++cy)
                for (int cx = 0; cx < 3; ++cx) {
                    int h = halo_index(lc[0] + cx, lc[1] + cy, lc[2] + cz);
                    R dN[3] = {dw[0][cx] * wgt[1][cy] * wgt[2][cz], wgt[0][cx] * dw[1][cy] * wgt[2][cz],
                               wgt[0][cx] * wgt[1][cy] * dw[2][cz]};
#pragma unroll
                    for (int q = 0; q < 3; ++q)
#pragma unroll
                        for (int e = 0; e < 3; ++e) {
                            L[3 * q + e] += vh[q][h] * dN[e];
                            D[3 * q + e] += dh[q][h] * dN[e];
                        }
                }
        double v0 = a.V0[i];
        if (a.phase[i] == 0) {
            double Jn = a.J[i];
            R jm1n = (R)(Jn - 1.0);
            R trL = L[0] + L[4] + L[8], trD = D[0] + D[4] + D[8];
            R jm1 = jm1n + dt * trL * (R(1) + jm1n);
            double lam = S.lambda_l;
            double Vn = Jn * v0;
            R el = 0, ed = 0, dd = 0;
#pragma unroll
            for (int q = 0; q < 3; ++q)
#pragma unroll
                for (int e = 0; e < 3; ++e) {
                    R sl = R(0.5) * (L[3 * q + e] + L[3 * e + q]);
                    R sd = R(0.5) * (D[3 * q + e] + D[3 * e + q]);
                    ed += sl * sd;
                    dd += sd * sd;
                }
            (void)el;
            double cvis = 0.5 * S.dt * S.mu_l * Vn;
            double alpha = alpha0;
            for (int k = a.k0; k < k1; ++k) {
                R dJ = (R)alpha * dt * trD * (R)Jn;
                double dE = 0.5 * lam * v0 * (double)dJ * (double)(R(2) * jm1 + dJ);
                dE += cvis * (2.0 * alpha * (double)ed + alpha * alpha * (double)dd);
                de[k] += dE;
                alpha *= 0.5;
            }
        } else {
            R Fo[9], A1[9], Fc[9];
#pragma unroll
            for (int q = 0; q < 9; ++q) {
                Fo[q] = (R)a.F.a[q][i];
                A1[q] = dt * L[q] + ((q % 4 == 0) ? R(1) : R(0));
            }
            matmul3<R>(A1, Fo, Fc);
            double Tn = a.T[i];
            double mu_h, lam_h;
            solid_lame(S, Tn, mu_h, lam_h);
            const R mu = (R)mu_h, lam = (R)lam_h;
            R psi0 = fcr_psi<R>(Fc, mu, lam);
            R alpha = (R)alpha0;
            for (int k = a.k0; k < k1; ++k) {
                R Fa[9];
#pragma unroll
                for (int q = 0; q < 9; ++q) A1[q] = dt * (L[q] + alpha * D[q]) + ((q % 4 == 0) ? R(1) : R(0));
                matmul3<R>(A1, Fo, Fa);
                de[k] += v0 * ((double)fcr_psi<R>(Fa, mu, lam) - (double)psi0);
                alpha *= R(0.5);
            }
        }
    }
    int sbeg = a.scell_start[gb * 64], send = a.scell_start[gb * 64 + 64];
    if (a.skip_samples) send = sbeg;
    for (int j = sbeg + threadIdx.x; j < send; j += NT) {
        double p[3] = {a.s.a[0][j], a.s.a[1][j], a.s.a[2][j]};
        int lc[3];
        R wgt[3][3], dw[3][3], f[3];
        stencil_in_block<R>(p, S, bc, lc, wgt, dw, f);
        R Fh[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1}, Dh[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
        for (int cz = 0; cz < 3; ++cz)
            for (int cy = 0; cy < 3; ++cy)
                for (int cx = 0; cx < 3; ++cx) {
                    int h = halo_index(lc[0] + cx, lc[1] + cy, lc[2] + cz);
                    R dN[3] = {dw[0][cx] * wgt[1][cy] * wgt[2][cz], wgt[0][cx] * dw[1][cy] * wgt[2][cz],
                               wgt[0][cx] * wgt[1][cy] * dw[2][cz]};
#pragma unroll
                    for (int q = 0; q < 3; ++q)
#pragma unroll
                        for (int e = 0; e < 3; ++e) {
                            Fh[3 * q + e] += dt * vh[q][h] * dN[e];
                            Dh[3 * q + e] += dt * dh[q][h] * dN[e];
                        }
                }
        R av[3] = {(R)a.dA.a[0][j], (R)a.dA.a[1][j], (R)a.dA.a[2][j]};
        R C[9], dC[9], CD[9];
        cofactor<R>(Fh, C);
        dcofactor<R>(Fh, Dh, dC);
        cofactor<R>(Dh, CD);
        R c0[3], c1[3], c2[3];
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            c0[q] = C[3 * q] * av[0] + C[3 * q + 1] * av[1] + C[3 * q + 2] * av[2];
            c1[q] = dC[3 * q] * av[0] + dC[3 * q + 1] * av[1] + dC[3 * q + 2] * av[2];
            c2[q] = CD[3 * q] * av[0] + CD[3 * q + 1] * av[1] + CD[3 * q + 2] * av[2];
        }
        R n0 = sqrt(c0[0] * c0[0] + c0[1] * c0[1] + c0[2] * c0[2]);
        double k = a.gamma[j];
        R alpha = (R)alpha0;
        for (int kk = a.k0; kk < k1; ++kk) {
            R dc[3], cn[3];
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                dc[q] = alpha * c1[q] + alpha * alpha * c2[q];
                cn[q] = c0[q] + dc[q];
            }
            R n1 = sqrt(cn[0] * cn[0] + cn[1] * cn[1] + cn[2] * cn[2]);
            R num = R(2) * (c0[0] * dc[0] + c0[1] * dc[1] + c0[2] * dc[2]) + dc[0] * dc[0] + dc[1] * dc[1] + dc[2] * dc[2];
            de[kk] += k * (double)num / ((double)n1 + (double)n0);
            alpha *= R(0.5);
        }
    }
    for (int k = a.k0; k < k1; ++k) block_atomic_sum<NT>(de[k], &scl.dphi[k], red);
}

template <typename RD>
__global__ void __launch_bounds__(32) k_ls_surf(LSArgs<RD> a) {
    __shared__ double pv[3][PN];
    __shared__ double pd[3][PN];
    const int w = blockIdx.x;
    const int slot = a.work[w];
    const long long gb = a.work_gb[w];
    const int4 bc = a.coord[slot];
    const SceneDev& S = a.sc[bc.w];
    SceneScal& scl = a.scal[bc.w];
    if (scl.newton_done || (a.k0 > 0 && scl.ls_pick >= 0)) return;
    const int sbeg = a.scell_start[gb * 64], send = a.scell_start[gb * 64 + 64];
    if (send == sbeg) return;
    load_halo_rows<double>(a.nbr, slot, a.gv, pv, pd);   // pd zeroed, then filled below
    __syncthreads();
    for (int r = threadIdx.x; r < 3 * HE * HE; r += blockDim.x) {
        int c = r / (HE * HE), yz = r % (HE * HE), hy = yz % HE, hz = yz / HE;
        int nmid, nlo, nhi, base;
        halo_row<double>(a.nbr, slot, hy, hz, nmid, nlo, nhi, base);
        int h0 = pidx(0, hy, hz);
        pd[c][h0] = nlo >= 0 ? (double)a.d[nlo * 192 + c * 64 + base + 3] : 0.0;
        for (int k = 0; k < 4; ++k) pd[c][h0 + 1 + k] = nmid >= 0 ? (double)a.d[nmid * 192 + c * 64 + base + k] : 0.0;
        pd[c][h0 + 5] = nhi >= 0 ? (double)a.d[nhi * 192 + c * 64 + base] : 0.0;
    }
    __syncthreads();
    const int nls = S.max_ls < MAX_LS ? S.max_ls : MAX_LS;
    const int k1 = a.k1 < nls ? a.k1 : nls;
    const double dt = S.dt;
    double de[MAX_LS];
#pragma unroll
    for (int k = 0; k < MAX_LS; ++k) de[k] = 0.0;
    for (int j = sbeg + threadIdx.x; j < send; j += 32) {
        const double p[3] = {a.s.a[0][j], a.s.a[1][j], a.s.a[2][j]};
        int lc[3];
        double wgt[3][3], dw[3][3], f[3];
        stencil_in_block<double>(p, S, bc, lc, wgt, dw, f);
        double Lv[9], Ld[9];
        gather_grad_sep<double>(pv, lc, wgt, dw, Lv);
        gather_grad_sep<double>(pd, lc, wgt, dw, Ld);
        double Fh[9], Dh[9];
#pragma unroll
        for (int q = 0; q < 9; ++q) {
            Fh[q] = dt * Lv[q] + ((q % 4 == 0) ? 1.0 : 0.0);
            Dh[q] = dt * Ld[q];
        }
        const double av[3] = {a.dA.a[0][j], a.dA.a[1][j], a.dA.a[2][j]};
        double C[9], dC[9], CD[9];
        cofactor<double>(Fh, C);
        dcofactor<double>(Fh, Dh, dC);
        cofactor<double>(Dh, CD);
        double c0[3], c1[3], c2[3];
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            c0[q] = C[3 * q] * av[0] + C[3 * q + 1] * av[1] + C[3 * q + 2] * av[2];
            c1[q] = dC[3 * q] * av[0] + dC[3 * q + 1] * av[1] + dC[3 * q + 2] * av[2];
            c2[q] = CD[3 * q] * av[0] + CD[3 * q + 1] * av[1] + CD[3 * q + 2] * av[2];
        }
        // |c0 + alpha c1 + alpha^2 c2| - |c0| without cancellation
        const double n0 = sqrt(c0[0] * c0[0] + c0[1] * c0[1] + c0[2] * c0[2]);
        const double k = a.gamma[j];
        double alpha = ldexp(1.0, -a.k0);
#pragma unroll
        for (int kk = 0; kk < MAX_LS; ++kk) {
            if (kk >= a.k0 && kk < k1) {
                double dc[3], cn[3];
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    dc[q] = alpha * c1[q] + alpha * alpha * c2[q];
                    cn[q] = c0[q] + dc[q];
                }
                const double n1 = sqrt(cn[0] * cn[0] + cn[1] * cn[1] + cn[2] * cn[2]);
                const double num = 2.0 * (c0[0] * dc[0] + c0[1] * dc[1] + c0[2] * dc[2]) + dc[0] * dc[0] +
                                   dc[1] * dc[1] + dc[2] * dc[2];
                de[kk] += k * num / (n1 + n0);
                alpha *= 0.5;
            }
        }
    }
#pragma unroll
    for (int k = 0; k < MAX_LS; ++k) {
        const double v = warp_sum(de[k]);
        if (k >= a.k0 && k < k1 && threadIdx.x == 0 && v != 0.0) atomicAdd(&scl.dphi[k], v);
    }
}

// node part of the line search: kinetic + gravity differences, the liquid
// energy's linear term alpha g_l . d, and slope = grad . d
template <typename R>
__global__ void k_ls_nodes(const int4* __restrict__ coord, const SceneDev* __restrict__ sc, SceneScal* __restrict__ scal,
                           const double* __restrict__ gm, const double* __restrict__ gvn, const double* __restrict__ gv,
                           const double* __restrict__ grad, const double* __restrict__ grad_l, const R* __restrict__ d,
                           int k0, int k1in) {
    int slot = blockIdx.x, l = threadIdx.x;
    int4 bc = coord[slot];
    const SceneDev& S = sc[bc.w];
    SceneScal& c = scal[bc.w];
    if (c.newton_done || (k0 > 0 && c.ls_pick >= 0)) return;
    int t = slot * 64 + l;
    double m = gm[t];
    double dv = 0.0, dd = 0.0, gd = 0.0, sl = 0.0, ld = 0.0;
    for (int q = 0; q < 3; ++q) {
        int k = slot * 192 + q * 64 + l;
        double dq = (double)d[k];
        ld += grad_l[k] * dq;   // liquid forces also reach massless halo nodes: d is 0 there
        if (m > 0.0) {
            dv += dq * (gv[k] - gvn[k]);
            dd += dq * dq;
            gd += S.g[q] * dq;
            sl += grad[k] * dq;
        }
    }
    const int nls = S.max_ls < MAX_LS ? S.max_ls : MAX_LS;
    const int k1 = k1in < nls ? k1in : nls;
    double alpha = ldexp(1.0, -k0);
    for (int k = k0; k < k1; ++k) {
        double e = 0.5 * m * (2.0 * alpha * dv + alpha * alpha * dd) - S.dt * alpha * m * gd + alpha * ld;
        e = warp_sum(e);
        if ((l & 31) == 0 && e != 0.0) atomicAdd(&c.dphi[k], e);
        alpha *= 0.5;
    }
    if (k0 == 0) {   // the slope, once per line search
        sl = warp_sum(sl);
        if ((l & 31) == 0 && sl != 0.0) atomicAdd(&c.slope, sl);
    }
}

// Armijo test of trials k0..k1-1 (alpha = 2^-k), the first passing one wins. The
// line search runs in two passes: trials 0 and 1 (alpha = 1, 1/2, which nearly
// every Newton iteration accepts), then, only for scenes where both failed
// (ls_pick < 0 after the first pick), the remaining trials; the result is the
// same as testing all trials in order in one pass.
__global__ void k_ls_pick(SceneScal* scal, const SceneDev* sc, int nsc, int k0, int k1in) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nsc) return;
    SceneScal& c = scal[s];
    if (c.newton_done || (k0 > 0 && c.ls_pick >= 0)) return;
    const int nls = sc[s].max_ls < MAX_LS ? sc[s].max_ls : MAX_LS;
    const int k1 = k1in < nls ? k1in : nls;
    double alpha = ldexp(1.0, -k0);
    int pick = nls;
    for (int k = k0; k < k1; ++k) {
        if (c.dphi[k] + 0.5 * alpha * alpha * c.dkd <= 1e-4 * alpha * c.slope) {
            pick = k;
            break;
        }
        alpha *= 0.5;
    }
    if (pick == nls && k1 < nls) {   // undecided: the next pass tests the rest
        c.ls_pick = -1;
        return;
    }
    c.ls_pick = pick;
    c.cg_total += c.cg_it;
    c.newton_it += 1;
    if (pick == nls) {
        // no trial decreases Phi: keep the iterate and stop (above tolerance)
        c.alpha = 0.0;
        c.newton_done = 1;
        c.status = MPM_ERR_NOT_CONVERGED;
    } else {
        c.alpha = alpha;
    }
}

template <typename R>
__global__ void k_newton_update(const int4* __restrict__ coord, const SceneScal* __restrict__ scal, const R* __restrict__ d,
                                double* __restrict__ gv) {
    int slot = blockIdx.x, l = threadIdx.x;
    int4 bc = coord[slot];
    const SceneScal& c = scal[bc.w];
    if (c.newton_done) return;
    double alpha = c.alpha;
    for (int q = 0; q < 3; ++q) {
        int k = slot * 192 + q * 64 + l;
        gv[k] += alpha * (double)d[k];
    }
}

// Coulomb friction of the slip plane on the end-of-step velocity v~ of one node:
// when v~ presses into the plane (v_n = v~ . n < 0) the plane's normal impulse
// m |v_n| bounds the tangential one by mu_f m |v_n|, so the tangential part t
// shrinks by mu_f |v_n| or stops (|t| <= mu_f |v_n|). The normal part is left
// for the slip projection.
__device__ __forceinline__ void coulomb_node(double* v, const double* n, double mu) {
    double vn = v[0] * n[0] + v[1] * n[1] + v[2] * n[2];
    if (!(vn < 0.0)) return;
    double t[3] = {v[0] - vn * n[0], v[1] - vn * n[1], v[2] - vn * n[2]};
    double tn = sqrt(t[0] * t[0] + t[1] * t[1] + t[2] * t[2]);
    double lim = -mu * vn;
    double s = tn > lim ? 1.0 - lim / tn : 0.0;
    for (int q = 0; q < 3; ++q) v[q] = s * t[q] + vn * n[q];
}

// final explicit force evaluation: vhat = P (v - grad / m), with the plane's
// Coulomb friction before the projection; momentum sums
__global__ void k_newton_final(const int4* __restrict__ coord, const SceneDev* __restrict__ sc, SceneScal* __restrict__ scal,
                               const double* __restrict__ gm, const double* __restrict__ gv, const double* __restrict__ grad,
                               const uint8_t* __restrict__ pcode, double* __restrict__ gvhat) {
    int slot = blockIdx.x, l = threadIdx.x;
    int4 bc = coord[slot];
    const SceneDev& S = sc[bc.w];
    int t = slot * 64 + l;
    double m = gm[t];
    double v[3] = {0, 0, 0};
    if (m > 0.0) {
        for (int q = 0; q < 3; ++q) {
            int k = slot * 192 + q * 64 + l;
            v[q] = gv[k] - grad[k] / m;
        }
        const uint8_t code = pcode[t];
        if (!(code & PC_FIXED) && S.friction > 0.0) {
            if (code & PC_PLANE) coulomb_node(v, S.plane_n, S.friction);
            if (code & PC_SPHERE) {
                double x[3], n[3];
                node_position(S, bc, l, x);
                sphere_phi_normal(S, x, n);
                coulomb_node(v, n, S.friction);
            }
        }
        project3(v, code, S, bc, l);
    }
    for (int q = 0; q < 3; ++q) {
        gvhat[slot * 192 + q * 64 + l] = v[q];
        double mv = warp_sum(m * v[q]);
        if ((l & 31) == 0 && mv != 0.0) atomicAdd(&scal[bc.w].mom[q], mv);
    }
}

__global__ void k_zero_grad_active(int nb, const int4* __restrict__ coord, const SceneScal* __restrict__ scal,
                                   double* __restrict__ grad, double* __restrict__ grad_l) {
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)nb * 192) return;
    if (!scal[coord[t / 192].w].newton_done) {
        grad[t] = 0.0;
        grad_l[t] = 0.0;
    }
}

__global__ void k_zero_mom(SceneScal* scal, int nsc) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nsc) return;
    scal[s].mom[0] = scal[s].mom[1] = scal[s].mom[2] = 0.0;
    scal[s].phi_part = 0.0;
}

// dense <-> grid copies for the C ABI
template <typename Tin, typename Tout>
__global__ void k_dense_to_grid(int nb, const int4* __restrict__ coord, int scene, const SceneDev* __restrict__ sc,
                                const Tin* __restrict__ dense, Tout* __restrict__ grid, int comps) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nb * 64) return;
    int slot = t >> 6, l = t & 63;
    int4 bc = coord[slot];
    const SceneDev& S = sc[bc.w];
    int g[3] = {bc.x * 4 + (l & 3), bc.y * 4 + ((l >> 2) & 3), bc.z * 4 + (l >> 4)};
    bool in = bc.w == scene && g[0] < S.n[0] && g[1] < S.n[1] && g[2] < S.n[2];
    long long node = g[0] + (long long)S.n[0] * (g[1] + (long long)S.n[1] * g[2]);
    for (int q = 0; q < comps; ++q) {
        int k = comps == 1 ? t : slot * 192 + q * 64 + l;
        grid[k] = in ? (Tout)dense[node * comps + q] : Tout(0);
    }
}

template <typename Tin, typename Tout>
__global__ void k_grid_to_dense(int nb, const int4* __restrict__ coord, int scene, const SceneDev* __restrict__ sc,
                                const Tin* __restrict__ grid, Tout* __restrict__ dense, int comps) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nb * 64) return;
    int slot = t >> 6, l = t & 63;
    int4 bc = coord[slot];
    if (bc.w != scene) return;
    const SceneDev& S = sc[bc.w];
    int g[3] = {bc.x * 4 + (l & 3), bc.y * 4 + ((l >> 2) & 3), bc.z * 4 + (l >> 4)};
    if (g[0] >= S.n[0] || g[1] >= S.n[1] || g[2] >= S.n[2]) return;
    long long node = g[0] + (long long)S.n[0] * (g[1] + (long long)S.n[1] * g[2]);
    for (int q = 0; q < comps; ++q) {
        int k = comps == 1 ? t : slot * 192 + q * 64 + l;
        dense[node * comps + q] = (Tout)grid[k];
    }
}

template <typename R>
__global__ void k_project_vec(int nb, const int4* __restrict__ coord, const SceneDev* __restrict__ sc,
                              const uint8_t* __restrict__ pcode, R* __restrict__ vec) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nb * 64) return;
    int slot = t >> 6, l = t & 63;
    const SceneDev& S = sc[coord[slot].w];
    R v[3];
    for (int q = 0; q < 3; ++q) v[q] = vec[slot * 192 + q * 64 + l];
    project3r<R>(v, pcode[t], S, coord[slot], l);
    for (int q = 0; q < 3; ++q) vec[slot * 192 + q * 64 + l] = v[q];
}

// u = P (m p + u)
template <typename R>
__global__ void k_mass_term(int nb, const int4* __restrict__ coord, const SceneDev* __restrict__ sc,
                            const uint8_t* __restrict__ pcode, const double* __restrict__ gm, const R* __restrict__ p,
                            R* __restrict__ u) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nb * 64) return;
    int slot = t >> 6, l = t & 63;
    const SceneDev& S = sc[coord[slot].w];
    R v[3];
    R m = (R)gm[t];
    for (int q = 0; q < 3; ++q) {
        int k = slot * 192 + q * 64 + l;
        v[q] = m * p[k] + u[k];
    }
    project3r<R>(v, pcode[t], S, coord[slot], l);
    for (int q = 0; q < 3; ++q) u[slot * 192 + q * 64 + l] = v[q];
}

inline unsigned nblk(long long n, int nt) { return (unsigned)((n + nt - 1) / nt); }

template <typename R>
EvalArgs<R> make_eval_args(mpm_ctx* c, bool want_grad, bool want_cache, bool skip_done) {
    Dev& d = c->d;
    EvalArgs<R> a;
    a.work = d.work;
    a.work_gb = d.work_gb;
    a.nbr = d.nbr;
    a.cell_start = d.cell_start;
    a.scell_start = d.scell_start;
    a.coord = d.slot_coord;
    a.sc = d.sc;
    a.scal = d.scal;
    a.gv = d.gv;
    a.grad = d.ggrad;
    for (int q = 0; q < 3; ++q) {
        a.x.a[q] = d.x[q];
        a.s.a[q] = d.s[q];
        a.dA.a[q] = d.dA[q];
        a.sn.a[q] = (R*)d.sn[q];
    }
    a.J = d.J;
    a.V0 = d.V0;
    a.T = d.T;
    for (int q = 0; q < 9; ++q) {
        a.F.a[q] = d.F[q];
        a.sF.a[q] = (R*)d.sF[q];
    }
    a.phase = d.phase;
    a.gamma = d.gamma;
    a.want_grad = want_grad;
    a.want_cache = want_cache;
    a.skip_done = skip_done;
    a.skip_poly = 1;
    a.skip_samples = 1;
    a.slot_gen = d.slot_gen;
    for (int q = 0; q < 24; ++q) a.scache.a[q] = (R*)d.scache[q];
    a.sic = (R*)d.sic;
    return a;
}

template <typename R>
ApplyArgs<R> make_apply_args(mpm_ctx* c, const void* p, void* u, int mode, int check_done) {
    Dev& d = c->d;
    ApplyArgs<R> a;
    a.pap = 0;
    a.work = d.work;
    a.work_gb = d.work_gb;
    a.nbr = d.nbr;
    a.cell_start = d.cell_start;
    a.scell_start = d.scell_start;
    a.coord = d.slot_coord;
    a.sc = d.sc;
    a.scal = d.scal;
    a.p = (const R*)p;
    a.u = (R*)u;
    a.phase = d.phase;
    a.V0 = d.V0;
    for (int q = 0; q < 3; ++q) {
        a.pu.a[q] = (R*)d.pu[q];
        a.su.a[q] = (R*)d.su[q];
        a.sa.a[q] = (R*)d.sa[q];
        a.sn.a[q] = (R*)d.sn[q];
    }
    a.kappa = (const R*)d.kappa;
    a.cvisc = (const R*)d.cvisc;
    for (int q = 0; q < 9; ++q) {
        a.Fn.a[q] = (R*)d.Fn[q];
        a.sF.a[q] = (R*)d.sF[q];
    }
    a.lmu = (const R*)d.lame[0];
    a.llam = (const R*)d.lame[1];
    for (int q = 0; q < 24; ++q) a.scache.a[q] = (R*)d.scache[q];
    a.sg = (const R*)d.sg;
    a.sic = (const R*)d.sic;
    a.slot_gen = d.slot_gen;
    a.sKa = (const R*)d.sKa;
    for (int q = 0; q < 45; ++q) a.pK.a[q] = (R*)d.pK[q];
    a.use_pK = (c->pK_valid && mode == MPM_HESS_PROJECTED) ? 1 : 0;
    a.samples_in_cell = (c->sK_valid && mode == MPM_HESS_PROJECTED) ? 1 : 0;
    a.opk = (const R4<R>*)d.opk;
    a.wrows = d.wrows;
    a.wroff = d.wroff;
    if (a.samples_in_cell) {
        a.gen_list = d.gen_list_g;
        a.gen_count = d.gen_pos_g + c->NW;
    } else {
        a.gen_list = d.gen_list;
        a.gen_count = d.gen_pos + c->NW;
    }
    a.err = d.err;
    a.mode = mode;
    a.check_done = check_done;
    return a;
}

template <typename R, int NC>
CGArgs<R, NC> make_cg_args(mpm_ctx* c) {
    Dev& d = c->d;
    CGArgs<R, NC> a;
    a.coord = d.slot_coord;
    a.sc = d.sc;
    a.scal = d.scal;
    a.pcode = d.pcode;
    a.gm = d.gm;
    a.mR = (const R*)d.mR;
    if (NC == 3) {
        a.inv = (const R*)d.invm;
        a.pinv3 = (const R*)d.pinv;
        a.x = (R*)d.cx;
        a.r = (R*)d.cr;
        a.p = (R*)d.cp;
        a.u = (R*)d.cu;
        a.rhs_d = d.ggrad;
        a.rhs_sign = -1.0;
    } else {
        a.inv = (const R*)d.hinvd;
        a.pinv3 = nullptr;
        a.x = (R*)d.hx;
        a.r = (R*)d.hr;
        a.p = (R*)d.hp;
        a.u = (R*)d.hu;
        a.rhs_d = d.hrhs;
        a.rhs_sign = 1.0;
    }
    return a;
}

// rows of a work block's rank-major records: the most particles in one of its cells
__global__ void k_rows(const int* __restrict__ work_gb, const int* __restrict__ cell_start, int* __restrict__ rows) {
    const long long base = (long long)work_gb[blockIdx.x] * 64;
    const int l = threadIdx.x;
    int m = max(cell_start[base + l + 1] - cell_start[base + l], cell_start[base + l + 33] - cell_start[base + l + 32]);
#pragma unroll
    for (int o = 16; o; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (l == 0) rows[blockIdx.x] = m;
}

// Sizes the rank-major operator records for the current sort and grows the
// buffer when it is too small (one host synchronisation per step).
template <typename R>
cudaError_t size_records(mpm_ctx* c) {
    Dev& d = c->d;
    cudaStream_t st = c->st;
    MPM_LAUNCH k_rows<<<c->NW, 32, 0, st>>>(d.work_gb, d.cell_start, d.wrows);
    launch_exclusive_scan(c, d.wrows, d.wroff, c->NW, d.scan_tmp, st);
    cudaMemcpyAsync(c->hcounts + 4, d.wroff + c->NW, sizeof(int), cudaMemcpyDeviceToHost, st);
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return e;
    long long need = (long long)c->hcounts[4] * 64;
    if (need > c->opk_cap) {
        if (d.opk) cudaFree(d.opk);
        d.opk = nullptr;
        c->opk_cap = 0;
        long long cap = need + need / 8 + 4096;
        e = cudaMalloc(&d.opk, (size_t)cap * sizeof(R4<R>));
        if (e != cudaSuccess) return e;
        c->opk_cap = cap;
    }
    return cudaSuccess;
}

template <typename R>
cudaError_t pack_step_t(mpm_ctx* c) {
    Dev& d = c->d;
    cudaStream_t st = c->st;
    cudaMemsetAsync(d.slot_gen, 0, sizeof(int) * (size_t)(c->NB > 0 ? c->NB : 1), st);
    if (c->np > 0 && c->NW > 0) {
        cudaError_t e = size_records<R>(c);
        if (e != cudaSuccess) return e;
        // slots past a cell's last particle stay zero (kappa 0): the operator
        // reads whole rows
        cudaMemsetAsync(d.opk, 0, (size_t)c->hcounts[4] * 64 * sizeof(R4<R>), st);
    }
    if (c->np > 0) {
        RPtr3<R> pu;
        RPtr9<R> Fn;
        for (int q = 0; q < 3; ++q) pu.a[q] = (R*)d.pu[q];
        for (int q = 0; q < 9; ++q) Fn.a[q] = (R*)d.Fn[q];
        Ptrs9 F;
        for (int q = 0; q < 9; ++q) F.a[q] = d.F[q];
        MPM_LAUNCH k_pack_volume<R><<<nblk(c->np, 256), 256, 0, st>>>((int)c->np, Ptrs3{{d.x[0], d.x[1], d.x[2]}}, d.J, F, d.V0, d.T,
                                                           d.phase, d.psc, d.sc, pu, (R*)d.kappa, (R*)d.cvisc, Fn,
                                                           (R*)d.lame[0], (R*)d.lame[1], (R*)d.Vn, d.bslot,
                                                           d.slot_gen, d.cell_start, c->NW, d.bw, d.wrows, d.wroff,
                                                           c->opk_cap, (R4<R>*)d.opk);
    }
    if (c->NW > 0) {
        cudaMemsetAsync(d.pinv, 0, sizeof(R) * (size_t)c->NB * 192, st);
        MPM_LAUNCH k_pinv<R><<<nblk((long long)c->NB * 64, 256), 256, 0, st>>>(c->NB, d.slot_coord, d.sc, d.gm, d.pcode,
                                                                             (R*)d.pinv, (R*)d.mR);
    }
    if (c->ns > 0) {
        RPtr3<R> su, sa;
        for (int q = 0; q < 3; ++q) {
            su.a[q] = (R*)d.su[q];
            sa.a[q] = (R*)d.sa[q];
        }
        MPM_LAUNCH k_pack_surface<R><<<nblk(c->ns, 256), 256, 0, st>>>((int)c->ns, Ptrs3{{d.s[0], d.s[1], d.s[2]}},
                                                            Ptrs3{{d.dA[0], d.dA[1], d.dA[2]}}, d.gamma, d.ssc, d.sc, su,
                                                            sa, (R*)d.sg);
    }
    if (c->NW > 0) {
        MPM_LAUNCH k_gen_flags<<<nblk(c->NW, 256), 256, 0, st>>>(c->NW, d.work, d.work_gb, d.scell_start, d.slot_gen,
                                                               d.gen_flag, d.gen_flag_g);
        launch_exclusive_scan(c, d.gen_flag, d.gen_pos, c->NW, d.scan_tmp, st);
        MPM_LAUNCH k_gen_list<<<nblk(c->NW, 256), 256, 0, st>>>(c->NW, d.gen_flag, d.gen_pos, d.gen_list);
        launch_exclusive_scan(c, d.gen_flag_g, d.gen_pos_g, c->NW, d.scan_tmp, st);
        MPM_LAUNCH k_gen_list<<<nblk(c->NW, 256), 256, 0, st>>>(c->NW, d.gen_flag_g, d.gen_pos_g, d.gen_list_g);
        // the lists' lengths size the general kernel's grid (none: no launch)
        cudaMemcpyAsync(c->hcounts + 5, d.gen_pos + c->NW, sizeof(int), cudaMemcpyDeviceToHost, st);
        cudaMemcpyAsync(c->hcounts + 6, d.gen_pos_g + c->NW, sizeof(int), cudaMemcpyDeviceToHost, st);
        cudaError_t e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return e;
        c->n_gen = c->hcounts[5];
        c->n_gen_g = c->hcounts[6];
    } else {
        c->n_gen = c->n_gen_g = 0;
    }
    return cudaGetLastError();
}

// one CG iteration's vector work: a cooperative launch of k_cg_iter over the
// CTAs that fit on the device at once (grid-stride over the slots)
// CTAs of k_cg_iter that fit on the device at once (queried once per type)
template <typename R, int NC>
cudaError_t cg_iter_capacity(int& grid, int per_sm_cap = 0) {
    static int per_sm[2][2] = {{-1, -1}, {-1, -1}};
    static int n_sm = 0;
    int& occ = per_sm[sizeof(R) == 4 ? 0 : 1][NC == 3 ? 0 : 1];
    if (occ < 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
        // the momentum CG runs the iteration that starts from a summed p . A p
        const void* fn;
        if constexpr (NC == 3) fn = (const void*)k_cg_iter2<R>;
        else fn = (const void*)k_cg_iter<R, NC>;
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, CG_NT, 0);
        if (e != cudaSuccess) return e;
        if (occ < 1) return cudaErrorInvalidConfiguration;
    }
    grid = (per_sm_cap > 0 && per_sm_cap < occ ? per_sm_cap : occ) * n_sm;
    return cudaSuccess;
}

template <typename R, int NC>
cudaError_t launch_cg_iter(mpm_ctx* c, CGArgs<R, NC>& a, int heat) {
    int grid = 0;
    cudaError_t e = cg_iter_capacity<R, NC>(grid, c->cg_ctas_per_sm);
    if (e != cudaSuccess) return e;
    int nb = c->NB, ns = c->nsc;
    int chunks = nblk(nb, CG_SLOTS);
    if (grid > chunks) grid = chunks;
    if (grid < 1) grid = 1;
    unsigned* bar = c->d.cg_bar;
    int* err = c->d.err;
    void* args[] = {(void*)&a, (void*)&nb, (void*)&ns, (void*)&heat, (void*)&bar, (void*)&err};
    void* args2[] = {(void*)&a, (void*)&nb, (void*)&ns, (void*)&bar, (void*)&err};
    // a cooperative launch (all CTAs co-resident), expressed as a launch attribute
    // so that it can also be captured into a CUDA graph
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(CG_NT);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = c->st;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    c->launches++;
    if constexpr (NC == 3) return cudaLaunchKernelExC(&cfg, (const void*)k_cg_iter2<R>, args2);
    else return cudaLaunchKernelExC(&cfg, (const void*)k_cg_iter<R, NC>, args);
}

template <typename R>
cudaError_t cg_solve_t(mpm_ctx* c, int NC_is_heat, int set_bnorm_in_init) {
    // runs CG to completion on every scene that is not done; returns after the host saw all done
    cudaStream_t st = c->st;
    int nb = c->NB;
    int ns = c->nsc;
    Dev& d = c->d;
    int maxit = 0;
    for (auto& S : c->hsc) maxit = maxit > S.max_cg ? maxit : S.max_cg;
    // Autotuner: the first momentum solves of a context each try one launch
    // configuration of the CG loop (CTAs per SM of the vector kernel, iterations per
    // host check); later solves use the one with the least device time per
    // iteration.
    static const int kTune[][2] = {{3, 8}, {2, 8}, {1, 8}, {3, 16}, {2, 16}, {1, 16}};
    constexpr int nTune = (int)(sizeof(kTune) / sizeof(kTune[0]));
    const bool tuning = !NC_is_heat && c->tune_next < nTune;
    if (!NC_is_heat) {
        const int k = tuning ? c->tune_next : c->tune_best;
        c->cg_ctas_per_sm = kTune[k][0];
        c->cg_chunk = kTune[k][1];
    }
    const int chunk = NC_is_heat ? 8 : c->cg_chunk;
    if (tuning) cudaEventRecord(c->tune_ev[0], st);
    cudaError_t e0 = cudaMemsetAsync(d.cg_bar, 0, 2 * sizeof(unsigned), st);
    if (e0 != cudaSuccess) return e0;
    if (NC_is_heat) {
        auto a = make_cg_args<R, 1>(c);
        MPM_LAUNCH k_cg_init<R, 1><<<nblk(nb, CG_SLOTS), CG_NT, 0, st>>>(a, nb, set_bnorm_in_init, 0);
        for (int it = 0; it < maxit; it += chunk) {
            for (int k = 0; k < chunk; ++k) {
                prof_mark_apply(c, true);
                launch_heat_apply(c, d.hp, d.hu);
                prof_mark_apply(c, false);
                e0 = launch_cg_iter<R, 1>(c, a, 1);
                if (e0 != cudaSuccess) return e0;
            }
            cudaMemcpyAsync(c->hscal, d.scal, sizeof(SceneScal) * ns, cudaMemcpyDeviceToHost, st);
            cudaError_t e = cudaStreamSynchronize(st);
            if (e != cudaSuccess) return e;
            prof_collect_applies(c, NC_is_heat != 0);
            bool all = true;
            for (int s = 0; s < ns; ++s) all = all && c->hscal[s].cg_done;
            if (all) break;
        }
    } else {
        auto a = make_cg_args<R, 3>(c);
        auto ap = make_apply_args<R>(c, d.cp, d.cu, MPM_HESS_PROJECTED, 1);
        ap.pap = 1;   // the operator kernels sum p . (H - M) p for the iteration
        MPM_LAUNCH k_cg_init<R, 3><<<nblk(nb, CG_SLOTS), CG_NT, 0, st>>>(a, nb, set_bnorm_in_init, 1);
        // Autotuner, operator tile: the first momentum solve of a context times
        // the liquid and sample operator with 2, 4 and 8 record rows per bulk
        // copy (three applications each on the first CG direction, into the
        // product vector, which is cleared afterwards) and keeps the fastest.
        if (c->op_rows == 0 && c->NW > 0) {
            auto at = ap;
            at.pap = 0;
            at.check_done = 0;
            const int cand[3] = {2, 4, 8};
            float best = 0.f;
            int pick = 4;
            for (int k = 0; k < 3; ++k) {
                launch_apply_pair<R>(c, at, st, cand[k]);   // warm-up
                cudaEventRecord(c->tune_ev[0], st);
                for (int rep = 0; rep < 3; ++rep) launch_apply_pair<R>(c, at, st, cand[k]);
                cudaEventRecord(c->tune_ev[1], st);
                float ms = 0.f;
                if (cudaEventSynchronize(c->tune_ev[1]) == cudaSuccess &&
                    cudaEventElapsedTime(&ms, c->tune_ev[0], c->tune_ev[1]) == cudaSuccess && (k == 0 || ms < best)) {
                    best = ms;
                    pick = cand[k];
                }
            }
            c->op_rows = pick;
            e0 = cudaMemsetAsync(d.cu, 0, (size_t)c->rsize * (size_t)nb * 192, st);
            if (e0 != cudaSuccess) return e0;
        }
        // one chunk of CG iterations: operator apply, then the cooperative vector kernel
        auto enqueue_chunk = [&]() -> cudaError_t {
            for (int k = 0; k < chunk; ++k) {
                prof_mark_apply(c, true);
                if (c->NW > 0) launch_apply_pair<R>(c, ap, st, c->op_rows);
                const int ng = ap.samples_in_cell ? c->n_gen_g : c->n_gen;
                if (ng > 0) {
                    if (ap.use_pK || !c->has_solids) MPM_LAUNCH k_apply_general<R, false><<<ng, NT_CELL, 0, st>>>(ap);
                    else MPM_LAUNCH k_apply_general<R, true><<<ng, NT_CELL, 0, st>>>(ap);
                }
                prof_mark_apply(c, false);
                cudaError_t e = launch_cg_iter<R, 3>(c, a, 0);
                if (e != cudaSuccess) return e;
            }
            return cudaSuccess;
        };
        // The chunk is captured once per solve as a CUDA graph (the operands and
        // grid sizes are fixed for the solve) and replayed until every scene's CG
        // is done; the host reads the per-scene flags between chunks. Without graph
        // support (capture refused) the chunk is launched directly.
        cudaGraphExec_t gexec = nullptr;
        long long per_chunk = 0;
        int nev_chunk = 0;
        if (c->use_graphs) {
            int grid = 0;
            e0 = cg_iter_capacity<R, 3>(grid);   // occupancy query outside the capture
            if (e0 != cudaSuccess) return e0;
            const long long l0 = c->launches;
            const int nev0 = c->nev;
            cudaGraph_t graph = nullptr;
            cudaError_t ec = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
            if (ec == cudaSuccess) {
                cudaError_t eq = enqueue_chunk();
                ec = cudaStreamEndCapture(st, &graph);
                if (eq != cudaSuccess) ec = eq;
            }
            if (ec == cudaSuccess) ec = cudaGraphInstantiate(&gexec, graph, 0);
            if (graph) cudaGraphDestroy(graph);
            if (ec != cudaSuccess) {
                cudaGetLastError();
                c->graph_error = (int)ec;
                if (gexec) cudaGraphExecDestroy(gexec);
                gexec = nullptr;
                c->use_graphs = false;
                c->nev = nev0;
            } else {
                per_chunk = c->launches - l0;
                nev_chunk = c->nev - nev0;
                c->launches = l0;
            }
        }
        for (int it = 0; it < maxit; it += chunk) {
            if (gexec) {
                cudaError_t e = cudaGraphLaunch(gexec, st);
                if (e != cudaSuccess) {
                    cudaGraphExecDestroy(gexec);
                    return e;
                }
                c->launches += per_chunk;
                if (c->prof) c->nev = nev_chunk;   // the graph recorded the chunk's event pairs
            } else {
                e0 = enqueue_chunk();
                if (e0 != cudaSuccess) return e0;
            }
            cudaMemcpyAsync(c->hscal, d.scal, sizeof(SceneScal) * ns, cudaMemcpyDeviceToHost, st);
            cudaError_t e = cudaStreamSynchronize(st);
            if (e != cudaSuccess) {
                if (gexec) cudaGraphExecDestroy(gexec);
                return e;
            }
            prof_collect_applies(c, NC_is_heat != 0);
            bool all = true;
            for (int s = 0; s < ns; ++s) all = all && c->hscal[s].cg_done;
            if (all) break;
        }
        if (gexec) cudaGraphExecDestroy(gexec);
        if (tuning) {
            cudaEventRecord(c->tune_ev[1], st);
            float ms = 0.f;
            int its = 0;
            for (int s = 0; s < ns; ++s) its = its > c->hscal[s].cg_it ? its : c->hscal[s].cg_it;
            if (cudaEventSynchronize(c->tune_ev[1]) == cudaSuccess &&
                cudaEventElapsedTime(&ms, c->tune_ev[0], c->tune_ev[1]) == cudaSuccess && its > 0) {
                const double per_it = ms / its;
                if (c->tune_best < 0 || per_it < c->tune_best_ms) {
                    c->tune_best = c->tune_next;
                    c->tune_best_ms = per_it;
                }
            }
            c->tune_next++;
            if (c->tune_next == nTune && c->tune_best < 0) c->tune_best = 0;
        }
    }
    return cudaGetLastError();
}

template <typename R, typename RS>
cudaError_t eval_t(mpm_ctx* c, bool want_grad, bool want_cache, bool skip_done) {
    if (c->NW == 0) return cudaSuccess;
    auto a = make_eval_args<RS>(c, want_grad, want_cache, skip_done);
    MPM_LAUNCH k_eval<R, RS><<<c->NW, NT, 0, c->st>>>(a);
    if (c->ns > 0) {
        MPM_LAUNCH k_eval_surf<RS><<<c->NW, 32, 0, c->st>>>(a);
        if (want_cache) {
            Dev& dd = c->d;
            RPtr9<RS> sF;
            RPtr3<RS> sa, sn;
            RPtr3<RS> su;
            for (int q = 0; q < 9; ++q) sF.a[q] = (RS*)dd.sF[q];
            for (int q = 0; q < 3; ++q) {
                sa.a[q] = (RS*)dd.sa[q];
                sn.a[q] = (RS*)dd.sn[q];
                su.a[q] = (RS*)dd.su[q];
            }
            MPM_LAUNCH k_surf_hess<RS><<<nblk(c->ns, 128), 128, 0, c->st>>>((int)c->ns, dd.ssc, dd.sc, sF, sa, sn,
                                                                        (const RS*)dd.sic, (const RS*)dd.sg, su,
                                                                        (RS*)dd.sKa);
            c->sK_valid = true;
        }
    }
    if (want_cache && c->has_solids && c->np > 0) {
        Dev& dd = c->d;
        RPtr24<RS> scache;
        RPtr9<RS> Fn;
        RPtr45<RS> K;
        for (int q = 0; q < 24; ++q) scache.a[q] = (RS*)dd.scache[q];
        for (int q = 0; q < 9; ++q) Fn.a[q] = (RS*)dd.Fn[q];
        for (int q = 0; q < 45; ++q) K.a[q] = (RS*)dd.pK[q];
        MPM_LAUNCH k_solid_hess<RS><<<nblk(c->np, 128), 128, 0, c->st>>>((int)c->np, dd.phase, dd.psc, dd.sc, scache, Fn,
                                                                        (const RS*)dd.lame[0], (const RS*)dd.lame[1],
                                                                        dd.V0, K);
        c->pK_valid = true;
    }
    Dev& d = c->d;
    EvalCellArgs e;
    e.work = d.work;
    e.work_gb = d.work_gb;
    e.nbr = d.nbr;
    e.cell_start = d.cell_start;
    e.coord = d.slot_coord;
    e.sc = d.sc;
    e.scal = d.scal;
    e.gv = d.gv;
    e.grad = want_grad ? d.ggrad : nullptr;
    e.grad_l = want_grad && skip_done ? d.ggrad_l : nullptr;   // Newton iterations only
    e.x0 = d.x[0];
    e.x1 = d.x[1];
    e.x2 = d.x[2];
    e.J = d.J;
    e.V0 = d.V0;
    e.phase = d.phase;
    e.skip_done = skip_done;
    MPM_LAUNCH k_eval_cell<<<c->NW, NT_CELL, 0, c->st>>>(e);
    return cudaGetLastError();
}

// objective / gradient in float64 arithmetic, caches stored in the context's type
cudaError_t eval_any(mpm_ctx* c, bool want_grad, bool want_cache, bool skip_done) {
    if (c->rsize == 8) return eval_t<double, double>(c, want_grad, want_cache, skip_done);
    return eval_t<double, float>(c, want_grad, want_cache, skip_done);
}

template <typename R>
cudaError_t newton_t(mpm_ctx* c) {
    Dev& d = c->d;
    cudaStream_t st = c->st;
    int nb = c->NB, ns = c->nsc;
    unsigned gs = nblk(ns, 128);
    MPM_LAUNCH k_newton_begin<<<gs, 128, 0, st>>>(d.scal, ns);
    MPM_LAUNCH k_newton_init_v<<<nb, 64, 0, st>>>(d.slot_coord, d.sc, d.gvn, d.pcode, d.gv);
    int maxn = 0;
    for (auto& S : c->hsc) maxn = maxn > S.max_newton ? maxn : S.max_newton;
    for (int it = 0; it <= maxn; ++it) {
        MPM_LAUNCH k_newton_iter_begin<<<gs, 128, 0, st>>>(d.scal, ns);
        // zero the gradient of scenes still iterating; converged scenes keep the
        // gradient at their final iterate for the closing force evaluation
        MPM_LAUNCH k_zero_grad_active<<<nblk((long long)nb * 192, 256), 256, 0, st>>>(nb, d.slot_coord, d.scal, d.ggrad, d.ggrad_l);
        eval_any(c, true, true, true);
        MPM_LAUNCH k_node_grad<<<nb, 64, 0, st>>>(d.slot_coord, d.sc, d.scal, d.gm, d.gvn, d.gv, d.pcode, d.ggrad, 1);
        MPM_LAUNCH k_newton_check<<<gs, 128, 0, st>>>(d.scal, d.sc, ns);
        cudaMemcpyAsync(c->hscal, d.scal, sizeof(SceneScal) * ns, cudaMemcpyDeviceToHost, st);
        cudaError_t e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return e;
        bool all = true;
        for (int s = 0; s < ns; ++s) all = all && c->hscal[s].newton_done;
        if (all) break;
        MPM_LAUNCH k_cg_begin<<<gs, 128, 0, st>>>(d.scal, ns, 1);
        e = cg_solve_t<R>(c, 0, 1);
        if (e != cudaSuccess) return e;
        if (c->NW > 0) {
            LSArgs<R> a;
            a.work = d.work;
            a.work_gb = d.work_gb;
            a.nbr = d.nbr;
            a.cell_start = d.cell_start;
            a.scell_start = d.scell_start;
            a.coord = d.slot_coord;
            a.sc = d.sc;
            a.scal = d.scal;
            a.gv = d.gv;
            a.d = (const R*)d.cx;
            for (int q = 0; q < 3; ++q) {
                a.x.a[q] = d.x[q];
                a.s.a[q] = d.s[q];
                a.dA.a[q] = d.dA[q];
            }
            a.J = d.J;
            a.V0 = d.V0;
            a.T = d.T;
            for (int q = 0; q < 9; ++q) a.F.a[q] = d.F[q];
            a.phase = d.phase;
            a.gamma = d.gamma;
            a.skip_poly = 1;
            a.skip_samples = 1;
            a.slot_gen = d.slot_gen;
            a.k0 = 0;
            a.k1 = LS_FIRST;
            MPM_LAUNCH k_linesearch<double, R><<<c->NW, NT, 0, st>>>(a);
            if (c->ns > 0) MPM_LAUNCH k_ls_surf<R><<<c->NW, 32, 0, st>>>(a);
            auto cv = make_apply_args<R>(c, d.cx, nullptr, MPM_HESS_PROJECTED, 0);
            MPM_LAUNCH k_curv_cell<R><<<c->NW, NT_CELL, 0, st>>>(cv);
            MPM_LAUNCH k_ls_nodes<R><<<nb, 64, 0, st>>>(d.slot_coord, d.sc, d.scal, d.gm, d.gvn, d.gv, d.ggrad, d.ggrad_l,
                                                        (const R*)d.cx, 0, LS_FIRST);
            MPM_LAUNCH k_ls_pick<<<gs, 128, 0, st>>>(d.scal, d.sc, ns, 0, LS_FIRST);
            // the remaining trials, for scenes whose first two failed
            a.k0 = LS_FIRST;
            a.k1 = MAX_LS;
            MPM_LAUNCH k_linesearch<double, R><<<c->NW, NT, 0, st>>>(a);
            if (c->ns > 0) MPM_LAUNCH k_ls_surf<R><<<c->NW, 32, 0, st>>>(a);
            MPM_LAUNCH k_ls_nodes<R><<<nb, 64, 0, st>>>(d.slot_coord, d.sc, d.scal, d.gm, d.gvn, d.gv, d.ggrad, d.ggrad_l,
                                                        (const R*)d.cx, LS_FIRST, MAX_LS);
            MPM_LAUNCH k_ls_pick<<<gs, 128, 0, st>>>(d.scal, d.sc, ns, LS_FIRST, MAX_LS);
        } else {
            MPM_LAUNCH k_ls_nodes<R><<<nb, 64, 0, st>>>(d.slot_coord, d.sc, d.scal, d.gm, d.gvn, d.gv, d.ggrad, d.ggrad_l,
                                                        (const R*)d.cx, 0, MAX_LS);
            MPM_LAUNCH k_ls_pick<<<gs, 128, 0, st>>>(d.scal, d.sc, ns, 0, MAX_LS);
        }
        MPM_LAUNCH k_newton_update<R><<<nb, 64, 0, st>>>(d.slot_coord, d.scal, (const R*)d.cx, d.gv);
    }
    // final explicit force evaluation: the loop ends right after evaluating the
    // float64 gradient at the final iterate of every scene, so it is in ggrad
    MPM_LAUNCH k_zero_mom<<<gs, 128, 0, st>>>(d.scal, ns);
    MPM_LAUNCH k_newton_final<<<nb, 64, 0, st>>>(d.slot_coord, d.sc, d.scal, d.gm, d.gv, d.ggrad, d.pcode, d.gvhat);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_pack_step(mpm_ctx* c) {
    if (c->rsize == 4) return pack_step_t<float>(c);
    return pack_step_t<double>(c);
}

cudaError_t launch_eval(mpm_ctx* c, bool fp64_math, bool want_cache) {
    Dev& d = c->d;
    int ns = c->nsc;
    MPM_LAUNCH k_newton_begin<<<nblk(ns, 128), 128, 0, c->st>>>(d.scal, ns);
    MPM_LAUNCH k_newton_iter_begin<<<nblk(ns, 128), 128, 0, c->st>>>(d.scal, ns);
    cudaMemsetAsync(d.ggrad, 0, sizeof(double) * (size_t)c->NB * 192, c->st);
    eval_any(c, true, want_cache, false);
    if (c->NB > 0) MPM_LAUNCH k_node_grad<<<c->NB, 64, 0, c->st>>>(d.slot_coord, d.sc, d.scal, d.gm, d.gvn, d.gv, d.pcode, d.ggrad, 0);
    return cudaGetLastError();
}

cudaError_t launch_apply(mpm_ctx* c, const void* p, void* u, int mode) {
    if (c->NW == 0) return cudaSuccess;
    if (c->rsize == 4) {
        auto a = make_apply_args<float>(c, p, u, mode, 0);
        launch_apply_pair<float>(c, a, c->st, c->op_rows);
        const int ng = a.samples_in_cell ? c->n_gen_g : c->n_gen;
        if (ng > 0) {
            if (a.use_pK || !c->has_solids) MPM_LAUNCH k_apply_general<float, false><<<ng, NT_CELL, 0, c->st>>>(a);
            else MPM_LAUNCH k_apply_general<float, true><<<ng, NT_CELL, 0, c->st>>>(a);
        }
    } else {
        auto a = make_apply_args<double>(c, p, u, mode, 0);
        launch_apply_pair<double>(c, a, c->st, c->op_rows);
        const int ng = a.samples_in_cell ? c->n_gen_g : c->n_gen;
        if (ng > 0) {
            if (a.use_pK || !c->has_solids) MPM_LAUNCH k_apply_general<double, false><<<ng, NT_CELL, 0, c->st>>>(a);
            else MPM_LAUNCH k_apply_general<double, true><<<ng, NT_CELL, 0, c->st>>>(a);
        }
    }
    return cudaGetLastError();
}

cudaError_t run_newton(mpm_ctx* c) {
    if (c->NB == 0) return cudaSuccess;
    if (c->rsize == 4) return newton_t<float>(c);
    return newton_t<double>(c);
}

cudaError_t launch_cg(mpm_ctx* c, int heat) {
    if (c->rsize == 4) return cg_solve_t<float>(c, heat, 0);
    return cg_solve_t<double>(c, heat, 0);
}

cudaError_t launch_cg_begin(mpm_ctx* c) {
    MPM_LAUNCH k_cg_begin<<<nblk(c->nsc, 128), 128, 0, c->st>>>(c->d.scal, c->nsc, 0);
    return cudaGetLastError();
}

cudaError_t launch_dense_to_grid(mpm_ctx* c, int scene, const void* dense, void* grid, int comps, int rsize) {
    if (c->NB == 0) return cudaSuccess;
    unsigned g = nblk((long long)c->NB * 64, 256);
    Dev& d = c->d;
    if (rsize == 8)
        MPM_LAUNCH k_dense_to_grid<double, double><<<g, 256, 0, c->st>>>(c->NB, d.slot_coord, scene, d.sc, (const double*)dense, (double*)grid, comps);
    else
        MPM_LAUNCH k_dense_to_grid<float, float><<<g, 256, 0, c->st>>>(c->NB, d.slot_coord, scene, d.sc, (const float*)dense, (float*)grid, comps);
    return cudaGetLastError();
}

cudaError_t launch_grid_to_dense(mpm_ctx* c, int scene, const void* grid, void* dense, int comps, int rsize_in, int rsize_out) {
    if (c->NB == 0) return cudaSuccess;
    unsigned g = nblk((long long)c->NB * 64, 256);
    Dev& d = c->d;
    if (rsize_in == 8 && rsize_out == 8)
        MPM_LAUNCH k_grid_to_dense<double, double><<<g, 256, 0, c->st>>>(c->NB, d.slot_coord, scene, d.sc, (const double*)grid, (double*)dense, comps);
    else if (rsize_in == 4 && rsize_out == 4)
        MPM_LAUNCH k_grid_to_dense<float, float><<<g, 256, 0, c->st>>>(c->NB, d.slot_coord, scene, d.sc, (const float*)grid, (float*)dense, comps);
    else if (rsize_in == 4 && rsize_out == 8)
        MPM_LAUNCH k_grid_to_dense<float, double><<<g, 256, 0, c->st>>>(c->NB, d.slot_coord, scene, d.sc, (const float*)grid, (double*)dense, comps);
    else
        MPM_LAUNCH k_grid_to_dense<double, float><<<g, 256, 0, c->st>>>(c->NB, d.slot_coord, scene, d.sc, (const double*)grid, (float*)dense, comps);
    return cudaGetLastError();
}

cudaError_t launch_project_vec(mpm_ctx* c, void* vec, int rsize) {
    if (c->NB == 0) return cudaSuccess;
    unsigned g = nblk((long long)c->NB * 64, 256);
    Dev& d = c->d;
    if (rsize == 8) MPM_LAUNCH k_project_vec<double><<<g, 256, 0, c->st>>>(c->NB, d.slot_coord, d.sc, d.pcode, (double*)vec);
    else MPM_LAUNCH k_project_vec<float><<<g, 256, 0, c->st>>>(c->NB, d.slot_coord, d.sc, d.pcode, (float*)vec);
    return cudaGetLastError();
}

cudaError_t launch_mass_term(mpm_ctx* c, const void* p, void* u) {
    if (c->NB == 0) return cudaSuccess;
    unsigned g = nblk((long long)c->NB * 64, 256);
    Dev& d = c->d;
    if (c->rsize == 8) MPM_LAUNCH k_mass_term<double><<<g, 256, 0, c->st>>>(c->NB, d.slot_coord, d.sc, d.pcode, d.gm, (const double*)p, (double*)u);
    else MPM_LAUNCH k_mass_term<float><<<g, 256, 0, c->st>>>(c->NB, d.slot_coord, d.sc, d.pcode, d.gm, (const float*)p, (float*)u);
    return cudaGetLastError();
}

}  // namespace mpm
