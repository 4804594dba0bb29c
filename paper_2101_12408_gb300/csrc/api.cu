// C ABI of the library (declared in include/mpm.h): context, particle I/O and
// the four phases of the time step.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>

#include "ctx.h"

namespace mpm {
cudaError_t launch_heat_full(mpm_ctx* c, const void* T, void* out);
}

namespace mpm {

void prof_mark_apply(mpm_ctx* c, bool begin) {
    if (!c->prof || c->nev >= 16) return;
    cudaEventRecord(c->ev[2 * c->nev + (begin ? 0 : 1)], c->st);
    if (!begin) c->nev++;
}

// called after the stream was synchronised
void prof_collect_applies(mpm_ctx* c, bool heat) {
    if (c->prof) {
        for (int i = 0; i < c->nev; ++i) {
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, c->ev[2 * i], c->ev[2 * i + 1]) != cudaSuccess) continue;
            if (heat) {
                c->pr.heat_apply_ms += ms;
                c->pr.heat_apply_launches++;
            } else {
                c->pr.apply_ms += ms;
                c->pr.apply_launches++;
            }
        }
    }
    c->nev = 0;
}

}  // namespace mpm

using namespace mpm;

namespace {

// device time of one phase call (events on the context's stream)
struct PhaseTimer {
    mpm_ctx* c;
    int k;
    PhaseTimer(mpm_ctx* c_, int k_) : c(c_), k(k_) {
        if (c->prof) cudaEventRecord(c->ev[32], c->st);
    }
    ~PhaseTimer() {
        if (!c->prof) return;
        cudaEventRecord(c->ev[33], c->st);
        if (cudaEventSynchronize(c->ev[33]) == cudaSuccess) {
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, c->ev[32], c->ev[33]) == cudaSuccess) c->pr.phase_ms[k] += ms;
        }
    }
};

}  // namespace

namespace {

#define MPM_CUDA(call)                                                                  \
    do {                                                                                \
        cudaError_t e_ = (call);                                                        \
        if (e_ != cudaSuccess) return fail(c, MPM_ERR_CUDA, cudaGetErrorString(e_));    \
    } while (0)

mpm_status fail(mpm_ctx* c, mpm_status s, const char* msg) {
    if (c) c->last_error = msg ? msg : "";
    return s;
}

template <typename T>
cudaError_t dalloc(mpm_ctx* c, T** p, size_t count) {
    void* q = nullptr;
    size_t bytes = count * sizeof(T);
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMalloc(&q, bytes);
    if (e != cudaSuccess) return e;
    c->allocs.push_back(q);
    *p = (T*)q;
    return cudaSuccess;
}

cudaError_t ralloc(mpm_ctx* c, void** p, size_t count) {
    void* q = nullptr;
    size_t bytes = count * (size_t)c->rsize;
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMalloc(&q, bytes);
    if (e != cudaSuccess) return e;
    c->allocs.push_back(q);
    *p = q;
    return cudaSuccess;
}

// staging layouts
__global__ void k_stage_in(int n, int base, int scene, const double* __restrict__ x, const double* __restrict__ v,
                           const double* __restrict__ A, const double* __restrict__ m, const double* __restrict__ V0,
                           const double* __restrict__ J, const double* __restrict__ F, const double* __restrict__ T,
                           const double* __restrict__ gT, const uint8_t* __restrict__ ph, Dev d, int allow_solid) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int k = base + i;
    for (int q = 0; q < 3; ++q) {
        d.x[q][k] = x[3 * i + q];
        d.v[q][k] = v ? v[3 * i + q] : 0.0;
        d.gT[q][k] = gT ? gT[3 * i + q] : 0.0;
    }
    for (int q = 0; q < 9; ++q) {
        d.A[q][k] = A ? A[9 * i + q] : 0.0;
        d.F[q][k] = F ? F[9 * i + q] : ((q % 4 == 0) ? 1.0 : 0.0);
    }
    d.m[k] = m[i];
    d.V0[k] = V0[i];
    d.J[k] = J ? J[i] : 1.0;
    d.T[k] = T ? T[i] : 0.0;
    uint8_t phv = ph ? ph[i] : 0;
    if (phv != 0 && !allow_solid) {   // no solid buffers in this context
        atomicOr(d.err, ERR_SOLID);
        phv = 0;
    }
    d.phase[k] = phv;
    d.pid[k] = i;
    d.psc[k] = scene;
}

__global__ void k_kill_scene(int n, int scene, int* psc) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && psc[i] == scene) psc[i] = -1;
}

__global__ void k_stage_surf_in(int n, int base, int scene, const double* __restrict__ s, const double* __restrict__ dA,
                                const uint8_t* __restrict__ kind, const double* __restrict__ b,
                                const double* __restrict__ Tbar, Dev d) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int k = base + i;
    for (int q = 0; q < 3; ++q) {
        d.s[q][k] = s[3 * i + q];
        d.dA[q][k] = dA[3 * i + q];
    }
    d.kind[k] = kind ? kind[i] : 0;
    d.bheat[k] = b ? b[i] : 0.0;
    d.Tbar[k] = Tbar ? Tbar[i] : 0.0;
    d.sid[k] = i;
    d.ssc[k] = scene;
    d.parent[k] = -1;   // no parent until mpm_resample
}

// gather particle fields back into set order: field id f, comps
__global__ void k_stage_out(int np, int scene, int n, const int* __restrict__ psc, const int* __restrict__ pid,
                            const double* const* __restrict__ src, int comps, double* __restrict__ out) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= np || psc[i] != scene) return;
    int id = pid[i];
    if (id < 0 || id >= n) return;
    for (int q = 0; q < comps; ++q) out[(size_t)id * comps + q] = src[q][i];
}

__global__ void k_stage_out_u8(int np, int scene, int n, const int* __restrict__ psc, const int* __restrict__ pid,
                               const uint8_t* __restrict__ src, uint8_t* __restrict__ out) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= np || psc[i] != scene) return;
    int id = pid[i];
    if (id >= 0 && id < n) out[id] = src[i];
}

__global__ void k_stage_parent(int ns, int np, int scene, int n, const int* __restrict__ ssc, const int* __restrict__ sid,
                               const int* __restrict__ parent, const int* __restrict__ pid, int32_t* __restrict__ out) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= ns || ssc[j] != scene) return;
    int id = sid[j];
    if (id < 0 || id >= n) return;
    int p = parent[j];
    out[id] = (p < 0 || p >= np) ? -1 : pid[p];
}

__global__ void k_check_finite(int n, const double* __restrict__ a, int* err) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && !isfinite(a[i])) atomicOr(err, ERR_NUMERIC);
}

inline unsigned nblk(long long n, int nt) { return (unsigned)((n + nt - 1) / nt); }

mpm_status check_device_error(mpm_ctx* c) {
    cudaError_t e = cudaMemcpyAsync(c->herr, c->d.err, sizeof(int), cudaMemcpyDeviceToHost, c->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
    if (e != cudaSuccess) return fail(c, MPM_ERR_CUDA, cudaGetErrorString(e));
    int err = *c->herr;
    if (err) {
        cudaMemsetAsync(c->d.err, 0, sizeof(int), c->st);
        cudaStreamSynchronize(c->st);
        if (err & ERR_DOMAIN) return fail(c, MPM_ERR_DOMAIN, "a particle or surface sample lies outside cells 1..n-2");
        if (err & ERR_FAR_SURFACE) return fail(c, MPM_ERR_DOMAIN, "a surface sample has no interior particle within 2 dx");
        if (err & ERR_NUMERIC) return fail(c, MPM_ERR_NUMERIC, "non-finite value on the device");
        if (err & ERR_CAPACITY) return fail(c, MPM_ERR_CAPACITY, "more active grid blocks than max_blocks");
        if (err & ERR_TIMEOUT) return fail(c, MPM_ERR_TIMEOUT, "a bounded device wait ran out");
        if (err & ERR_SOLID)
            return fail(c, MPM_ERR_INVALID_ARG, "solid particles in a context created without E0 > 0 or phase change");
    }
    return MPM_OK;
}

size_t staging_doubles(mpm_ctx* c) {
    // two buffers of this size hold every input field of one scene (31 doubles per particle)
    long long mx = 0;
    for (auto& s : c->hsc) {
        long long a = (s.p_end - s.p_begin) * 16;
        long long b = (s.s_end - s.s_begin) * 4;
        mx = mx > a ? mx : a;
        mx = mx > b ? mx : b;
    }
    long long grid = 0;
    for (auto& s : c->hsc) {
        long long g = (long long)s.n[0] * s.n[1] * s.n[2] * 3;
        grid = grid > g ? grid : g;
    }
    return (size_t)(mx > grid ? mx : grid);
}

}  // namespace

extern "C" {

mpm_status mpm_create(const mpm_scene_desc* scenes, int32_t n_scenes, int32_t precision, void* stream, mpm_ctx** out) {
    if (!out || !scenes || n_scenes <= 0) return MPM_ERR_INVALID_ARG;
    *out = nullptr;
    if (precision != MPM_PREC_FP64 && precision != MPM_PREC_FP32_FP64RED) return MPM_ERR_INVALID_ARG;
    mpm_ctx* c = new (std::nothrow) mpm_ctx();
    if (!c) return MPM_ERR_CUDA;
    c->nsc = n_scenes;
    c->prec = precision;
    c->rsize = precision == MPM_PREC_FP64 ? 8 : 4;
    c->st = (cudaStream_t)stream;
    long long bb = 0, pb = 0, sb = 0, bcap = 0;
    bool solids = false;
    for (int k = 0; k < n_scenes; ++k) {
        const mpm_scene_desc& D = scenes[k];
        const mpm_grid_desc& G = D.grid;
        const mpm_params& P = D.params;
        if (G.n[0] < 4 || G.n[1] < 4 || G.n[2] < 4 || !(G.dx > 0) || D.max_particles < 0 || D.max_surface < 0 ||
            !(P.dt > 0) || P.max_ls < 1 || P.max_ls > MAX_LS || P.max_newton < 0 || P.max_cg < 1 ||
            !(P.friction >= 0.0) || !std::isfinite(P.friction) || (P.massless_surface != 0 && P.massless_surface != 1)) {
            delete c;
            return MPM_ERR_INVALID_ARG;
        }
        SceneDev S;
        memset(&S, 0, sizeof(S));
        for (int a = 0; a < 3; ++a) {
            S.n[a] = G.n[a];
            S.nb[a] = (G.n[a] + BS - 1) / BS;
            S.origin[a] = G.origin[a];
            S.g[a] = P.gravity[a];
        }
        S.block_base = bb;
        long long nbl = (long long)S.nb[0] * S.nb[1] * S.nb[2];
        bb += nbl;
        bcap += (D.max_blocks > 0 && D.max_blocks < nbl) ? D.max_blocks : nbl;
        solids = solids || P.E0 > 0.0 || P.phase_change;
        S.dx = G.dx;
        S.inv_dx = 1.0 / G.dx;
        S.dt = P.dt;
        S.rho = P.rho;
        S.lambda_l = P.lambda_l;
        S.mu_l = P.mu_l;
        S.E0 = P.E0;
        S.nu = P.nu;
        S.T0 = P.T0;
        S.T_melt = P.T_melt;
        S.cp = P.cp;
        S.K = P.K;
        S.h = P.h;
        S.H = P.H;
        S.gamma_law = P.gamma_law;
        S.thermal = P.thermal;
        S.phase_change = P.phase_change;
        for (int a = 0; a < 4; ++a) S.gamma_p[a] = P.gamma_p[a];
        S.gamma_lg = P.gamma_lg;
        S.gamma_sl = P.gamma_sl;
        for (int f = 0; f < 6; ++f) S.walls[f] = G.walls[f];
        double nn = std::sqrt(G.plane_n[0] * G.plane_n[0] + G.plane_n[1] * G.plane_n[1] + G.plane_n[2] * G.plane_n[2]);
        S.plane_mode = G.plane_mode;
        if (G.plane_mode && !(nn > 0)) {
            delete c;
            return MPM_ERR_INVALID_ARG;
        }
        for (int a = 0; a < 3; ++a) S.plane_n[a] = G.plane_mode ? G.plane_n[a] / nn : 0.0;
        for (int a = 0; a < 3; ++a) S.plane_nf[a] = (float)S.plane_n[a];
        S.plane_d = G.plane_mode ? G.plane_d / nn : 0.0;
        S.sphere_mode = G.sphere_mode;
        S.sphere_outside = G.sphere_outside ? 1 : 0;
        for (int a = 0; a < 3; ++a) S.sphere_c[a] = G.sphere_mode ? G.sphere[a] : 0.0;
        S.sphere_R = G.sphere_mode ? G.sphere[3] : 0.0;
        if (G.sphere_mode < 0 || G.sphere_mode > 2 || (G.sphere_mode && !(G.sphere[3] > 0.0)) ||
            (G.sphere_mode && !(std::isfinite(G.sphere[0]) && std::isfinite(G.sphere[1]) && std::isfinite(G.sphere[2])))) {
            delete c;
            return MPM_ERR_INVALID_ARG;
        }
        S.newton_tol = P.newton_tol;
        S.cg_rtol = P.cg_rtol;
        S.heat_rtol = P.heat_rtol;
        S.max_newton = P.max_newton;
        S.max_cg = P.max_cg;
        S.max_ls = P.max_ls;
        S.massless = P.massless_surface;
        S.friction = (G.plane_mode == MPM_WALL_SLIP || G.sphere_mode == MPM_WALL_SLIP) ? P.friction : 0.0;
        S.p_begin = pb;
        S.p_end = pb + D.max_particles;
        S.s_begin = sb;
        S.s_end = sb + D.max_surface;
        pb += D.max_particles;
        sb += D.max_surface;
        c->hsc.push_back(S);
    }
    // a re-set scene's new particles are appended; its old ones are dropped by the
    // next sort, or by a compacting sort first when the appended set would not fit
    c->Pcap = pb + 1;
    c->Scap = sb + 1;
    c->total_blocks = bb;
    c->total_cells = bb * 64;
    if (c->Pcap > 0x7fffffffLL || c->total_cells + 1 > 0x7fffffffLL) {
        delete c;
        return MPM_ERR_CAPACITY;
    }
    c->block_cap = bcap;
    c->has_solids = solids;
    // MPM_OP_ROWS=2|4|8 fixes the operator's record rows per bulk copy instead of
    // letting the first momentum solve time them (tests use it to cover each tile)
    if (const char* ev = std::getenv("MPM_OP_ROWS")) {
        const int r = std::atoi(ev);
        if (r == 2 || r == 4 || r == 8) c->op_rows = r;
    }
    Dev& d = c->d;
    long long P = c->Pcap, Sn = c->Scap, NBc = c->total_blocks, NN = bcap * 64;
    long long PS = solids ? P : 1;   // solid-only buffers
    cudaError_t e = cudaSuccess;
#define A_(ptr, T, n) if (e == cudaSuccess) e = dalloc<T>(c, &(ptr), (size_t)(n))
#define R_(ptr, n) if (e == cudaSuccess) e = ralloc(c, &(ptr), (size_t)(n))
    for (int q = 0; q < 3; ++q) {
        A_(d.x[q], double, P); A_(d.v[q], double, P); A_(d.gT[q], double, P);
        A_(d.s[q], double, Sn); A_(d.dA[q], double, Sn); A_(d.bpos[q], double, Sn);
        R_(d.pu[q], P); R_(d.su[q], Sn); R_(d.sa[q], Sn); R_(d.sn[q], Sn);
    }
    for (int q = 0; q < 9; ++q) {
        A_(d.A[q], double, P); A_(d.F[q], double, P);
        R_(d.Fn[q], PS); R_(d.sF[q], Sn);
    }
    for (int q = 0; q < 12; ++q) A_(d.acc[q], double, P);
    for (int q = 0; q < 24; ++q) R_(d.scache[q], PS);
    R_(d.pK[0], 45 * PS);   // one allocation, the 45 entries PS apart
    for (int q = 1; q < 45; ++q) d.pK[q] = (char*)d.pK[0] + (size_t)q * PS * c->rsize;
    A_(d.m, double, P); A_(d.V0, double, P); A_(d.J, double, P); A_(d.T, double, P);
    A_(d.phase, uint8_t, P);
    A_(d.pid, int, P); A_(d.psc, int, P);
    A_(d.scratch_p, double, P); A_(d.scratch_s, double, Sn);
    A_(d.gcount, int, P); A_(d.mt, double, P);
    R_(d.kappa, P); R_(d.cvisc, P); R_(d.lame[0], PS); R_(d.lame[1], PS); R_(d.Vn, P);
    A_(d.bheat, double, Sn); A_(d.Tbar, double, Sn); A_(d.gamma, double, Sn); A_(d.Tr, double, Sn);
    A_(d.kind, uint8_t, Sn);
    A_(d.sid, int, Sn); A_(d.ssc, int, Sn); A_(d.parent, int, Sn);
    R_(d.sg, Sn); R_(d.sic, Sn); R_(d.swn, Sn);
    R_(d.sKa, (size_t)SREC * Sn);   // sample j's record at j * SREC
    A_(d.key, long long, P); A_(d.rank, int, P); A_(d.perm, int, P);
    A_(d.skey, long long, Sn); A_(d.srank, int, Sn); A_(d.sperm, int, Sn);
    A_(d.cell_count, int, c->total_cells + 1); A_(d.cell_start, int, c->total_cells + 1);
    A_(d.scell_count, int, c->total_cells + 1); A_(d.scell_start, int, c->total_cells + 1);
    A_(d.bflag, int, NBc + 1); A_(d.bwork, int, NBc + 1); A_(d.bslot, int, NBc + 1); A_(d.bscan, int, NBc + 1); A_(d.bw, int, NBc + 1);
    A_(d.slot_coord, int4, bcap + 1); A_(d.nbr, int, bcap * 27 + 27); A_(d.work, int, bcap + 1); A_(d.work_gb, int, bcap + 1);
    A_(d.slot_gen, int, bcap + 1); A_(d.wrows, int, bcap + 1); A_(d.wroff, int, bcap + 2);
    A_(d.gen_flag, int, bcap + 1); A_(d.gen_pos, int, bcap + 2); A_(d.gen_list, int, bcap + 1);
    A_(d.gen_flag_g, int, bcap + 1); A_(d.gen_pos_g, int, bcap + 2); A_(d.gen_list_g, int, bcap + 1);
    A_(d.counts, int, 4);
    A_(d.scan_tmp, int, (c->total_cells + 1) / 4096 + 16);
    A_(d.gm, double, NN); A_(d.gmv, double, NN * 3); A_(d.gvn, double, NN * 3); A_(d.gmT, double, NN);
    A_(d.gmTT, double, NN); A_(d.gTn, double, NN); A_(d.gv, double, NN * 3); A_(d.gvhat, double, NN * 3);
    A_(d.gThat, double, NN); A_(d.ggrad, double, NN * 3); A_(d.ggrad_l, double, NN * 3); A_(d.hrhs, double, NN);
    A_(d.pcode, uint8_t, NN);
    R_(d.cx, NN * 3); R_(d.cr, NN * 3); R_(d.cp, NN * 3); R_(d.cu, NN * 3); R_(d.invm, NN); R_(d.pinv, NN * 3); R_(d.mR, NN);
    R_(d.hx, NN); R_(d.hr, NN); R_(d.hp, NN); R_(d.hu, NN); R_(d.hinvd, NN); R_(d.hT, NN);
    size_t stg = staging_doubles(c);
    A_(*(double**)&d.dense_a, double, stg); A_(*(double**)&d.dense_b, double, stg);
    A_(d.sc, SceneDev, n_scenes); A_(d.scal, SceneScal, n_scenes); A_(d.err, int, 1); A_(d.cg_bar, unsigned, 2);
    A_(d.scene_cnt, unsigned long long, n_scenes); A_(d.scene_first, long long, n_scenes);
#undef A_
#undef R_
    for (int k = 0; k < 34 && e == cudaSuccess; ++k) e = cudaEventCreate(&c->ev[k]);
    for (int k = 0; k < 2 && e == cudaSuccess; ++k) e = cudaEventCreate(&c->tune_ev[k]);
    if (e == cudaSuccess) e = cudaMallocHost(&c->hscal, sizeof(SceneScal) * n_scenes);
    if (e == cudaSuccess) e = cudaMallocHost(&c->herr, sizeof(int));
    if (e == cudaSuccess) e = cudaMallocHost(&c->hcounts, sizeof(int) * 8);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d.sc, c->hsc.data(), sizeof(SceneDev) * n_scenes, cudaMemcpyHostToDevice, c->st);
    if (e == cudaSuccess) e = cudaMemsetAsync(d.scal, 0, sizeof(SceneScal) * n_scenes, c->st);
    if (e == cudaSuccess) e = cudaMemsetAsync(d.err, 0, sizeof(int), c->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
    if (e != cudaSuccess) {
        mpm_destroy(c);
        return e == cudaErrorMemoryAllocation ? MPM_ERR_CAPACITY : MPM_ERR_CUDA;
    }
    *out = c;
    return MPM_OK;
}

mpm_status mpm_destroy(mpm_ctx* c) {
    if (!c) return MPM_ERR_INVALID_ARG;
    if (c->st) cudaStreamSynchronize(c->st); else cudaDeviceSynchronize();
    for (void* p : c->allocs) cudaFree(p);
    if (c->d.opk) cudaFree(c->d.opk);
    if (c->tri_buf) cudaFree(c->tri_buf);
    for (int k = 0; k < 34; ++k)
        if (c->ev[k]) cudaEventDestroy(c->ev[k]);
    for (int k = 0; k < 2; ++k)
        if (c->tune_ev[k]) cudaEventDestroy(c->tune_ev[k]);
    if (c->hscal) cudaFreeHost(c->hscal);
    if (c->herr) cudaFreeHost(c->herr);
    if (c->hcounts) cudaFreeHost(c->hcounts);
    delete c;
    return MPM_OK;
}

const char* mpm_last_error(const mpm_ctx* c) { return c ? c->last_error.c_str() : "null context"; }

mpm_status mpm_set_particles(mpm_ctx* c, int32_t scene, int64_t n, const double* x, const double* v, const double* A,
                             const double* m, const double* V0, const double* J, const double* F, const double* T,
                             const double* gradT, const uint8_t* phase) {
    if (!c) return MPM_ERR_INVALID_ARG;
    if (scene < 0 || scene >= c->nsc || n < 0 || (n > 0 && (!x || !m || !V0)))
        return fail(c, MPM_ERR_INVALID_ARG, "mpm_set_particles: bad scene, count or pointer");
    SceneDev& S = c->hsc[scene];
    if (n > S.p_end - S.p_begin) return fail(c, MPM_ERR_CAPACITY, "mpm_set_particles: more particles than max_particles");
    cudaStream_t st = c->st;
    Dev& d = c->d;
    if (c->np > 0) MPM_LAUNCH k_kill_scene<<<nblk(c->np, 256), 256, 0, st>>>((int)c->np, scene, d.psc);
    if (c->np + n > c->Pcap) MPM_CUDA(launch_sort_particles(c));   // drops removed particles
    if (n > 0) {
        // every field is copied (from host or device memory) into the two staging
        // buffers, then one kernel scatters them into the SoA state
        const double* src[9] = {x, v, A, m, V0, J, F, T, gradT};
        size_t comps[9] = {3, 3, 9, 1, 1, 1, 9, 1, 3};
        const double* dptr[9];
        double* bufs[2] = {(double*)d.dense_a, (double*)d.dense_b};
        size_t cap = staging_doubles(c), used[2] = {0, 0};
        for (int f = 0; f < 9; ++f) {
            if (!src[f]) {
                dptr[f] = nullptr;
                continue;
            }
            size_t cnt = comps[f] * (size_t)n;
            int b = used[0] + cnt <= cap ? 0 : 1;
            if (used[b] + cnt > cap) return fail(c, MPM_ERR_CAPACITY, "staging buffer too small");
            double* dst = bufs[b] + used[b];
            used[b] += cnt;
            MPM_CUDA(cudaMemcpyAsync(dst, src[f], cnt * sizeof(double), cudaMemcpyDefault, st));
            dptr[f] = dst;
        }
        uint8_t* ph = nullptr;
        if (phase) {
            // phase bytes go to the tail of the scratch key buffer
            ph = (uint8_t*)d.perm;
            MPM_CUDA(cudaMemcpyAsync(ph, phase, (size_t)n, cudaMemcpyDefault, st));
        }
        MPM_LAUNCH k_stage_in<<<nblk(n, 256), 256, 0, st>>>((int)n, (int)c->np, scene, dptr[0], dptr[1], dptr[2], dptr[3], dptr[4],
                                                  dptr[5], dptr[6], dptr[7], dptr[8], ph, d,
                                                  c->has_solids ? 1 : 0);
        MPM_CUDA(cudaGetLastError());
        // reject non-finite input before any step
        for (int f = 0; f < 9; ++f)
            if (dptr[f]) MPM_LAUNCH k_check_finite<<<nblk(comps[f] * n, 256), 256, 0, st>>>((int)(comps[f] * n), dptr[f], d.err);
        c->np += n;
    }
    c->resampled = false;
    MPM_CUDA(cudaStreamSynchronize(st));
    return check_device_error(c);
}

mpm_status mpm_get_particles(mpm_ctx* c, int32_t scene, int64_t n, double* x, double* v, double* A, double* J,
                             double* F, double* T, double* gradT, uint8_t* phase) {
    if (!c) return MPM_ERR_INVALID_ARG;
    if (scene < 0 || scene >= c->nsc || n < 0) return fail(c, MPM_ERR_INVALID_ARG, "mpm_get_particles: bad scene or count");
    if (n > c->hsc[scene].p_end - c->hsc[scene].p_begin) return fail(c, MPM_ERR_INVALID_ARG, "mpm_get_particles: n above capacity");
    if (n == 0 || c->np == 0) return MPM_OK;
    cudaStream_t st = c->st;
    Dev& d = c->d;
    struct Field { double* out; int comps; double** src; };
    double* srcs[9];
    Field fields[6] = {{x, 3, d.x}, {v, 3, d.v}, {A, 9, d.A}, {F, 9, d.F}, {gradT, 3, d.gT}, {nullptr, 0, nullptr}};
    // device array of source pointers lives in dense_b's head
    for (int f = 0; f < 5; ++f) {
        Field& fd = fields[f];
        if (!fd.out) continue;
        for (int q = 0; q < fd.comps; ++q) srcs[q] = fd.src[q];
        double** dsrc = (double**)d.dense_b;
        MPM_CUDA(cudaMemcpyAsync(dsrc, srcs, sizeof(double*) * fd.comps, cudaMemcpyHostToDevice, st));
        MPM_LAUNCH k_stage_out<<<nblk(c->np, 256), 256, 0, st>>>((int)c->np, scene, (int)n, d.psc, d.pid, (const double* const*)dsrc,
                                                      fd.comps, (double*)d.dense_a);
        MPM_CUDA(cudaMemcpyAsync(fd.out, d.dense_a, sizeof(double) * fd.comps * n, cudaMemcpyDefault, st));
        MPM_CUDA(cudaStreamSynchronize(st));
    }
    double* scal_src[2] = {d.J, d.T};
    double* scal_out[2] = {J, T};
    for (int f = 0; f < 2; ++f) {
        if (!scal_out[f]) continue;
        double** dsrc = (double**)d.dense_b;
        MPM_CUDA(cudaMemcpyAsync(dsrc, &scal_src[f], sizeof(double*), cudaMemcpyHostToDevice, st));
        MPM_LAUNCH k_stage_out<<<nblk(c->np, 256), 256, 0, st>>>((int)c->np, scene, (int)n, d.psc, d.pid, (const double* const*)dsrc, 1,
                                                      (double*)d.dense_a);
        MPM_CUDA(cudaMemcpyAsync(scal_out[f], d.dense_a, sizeof(double) * n, cudaMemcpyDefault, st));
        MPM_CUDA(cudaStreamSynchronize(st));
    }
    if (phase) {
        MPM_LAUNCH k_stage_out_u8<<<nblk(c->np, 256), 256, 0, st>>>((int)c->np, scene, (int)n, d.psc, d.pid, d.phase, (uint8_t*)d.dense_a);
        MPM_CUDA(cudaMemcpyAsync(phase, d.dense_a, (size_t)n, cudaMemcpyDefault, st));
        MPM_CUDA(cudaStreamSynchronize(st));
    }
    return check_device_error(c);
}

mpm_status mpm_set_surface(mpm_ctx* c, int32_t scene, int64_t n, const double* s, const double* dA, const uint8_t* kind,
                           const double* b, const double* Tbar) {
    if (!c) return MPM_ERR_INVALID_ARG;
    if (scene < 0 || scene >= c->nsc || n < 0 || (n > 0 && (!s || !dA)))
        return fail(c, MPM_ERR_INVALID_ARG, "mpm_set_surface: bad scene, count or pointer");
    SceneDev& S = c->hsc[scene];
    if (n > S.s_end - S.s_begin) return fail(c, MPM_ERR_CAPACITY, "mpm_set_surface: more samples than max_surface");
    cudaStream_t st = c->st;
    Dev& d = c->d;
    if (c->ns > 0) MPM_LAUNCH k_kill_scene<<<nblk(c->ns, 256), 256, 0, st>>>((int)c->ns, scene, d.ssc);
    if (c->ns + n > c->Scap) MPM_CUDA(launch_sort_surface(c));   // drops removed samples
    if (n > 0) {
        double* a = (double*)d.dense_a;
        double* bb = (double*)d.dense_b;
        MPM_CUDA(cudaMemcpyAsync(a, s, sizeof(double) * 3 * n, cudaMemcpyDefault, st));
        MPM_CUDA(cudaMemcpyAsync(a + 3 * n, dA, sizeof(double) * 3 * n, cudaMemcpyDefault, st));
        double* db = nullptr;
        double* dT = nullptr;
        if (b) {
            db = bb;
            MPM_CUDA(cudaMemcpyAsync(db, b, sizeof(double) * n, cudaMemcpyDefault, st));
        }
        if (Tbar) {
            dT = bb + n;
            MPM_CUDA(cudaMemcpyAsync(dT, Tbar, sizeof(double) * n, cudaMemcpyDefault, st));
        }
        uint8_t* dk = nullptr;
        if (kind) {
            dk = (uint8_t*)(bb + 2 * n);
            MPM_CUDA(cudaMemcpyAsync(dk, kind, (size_t)n, cudaMemcpyDefault, st));
        }
        MPM_LAUNCH k_stage_surf_in<<<nblk(n, 256), 256, 0, st>>>((int)n, (int)c->ns, scene, a, a + 3 * n, dk, db, dT, d);
        MPM_CUDA(cudaGetLastError());
        MPM_LAUNCH k_check_finite<<<nblk(6 * n, 256), 256, 0, st>>>((int)(6 * n), a, d.err);
        c->ns += n;
    }
    c->resampled = false;
    MPM_CUDA(cudaStreamSynchronize(st));
    return check_device_error(c);
}

mpm_status mpm_get_surface(mpm_ctx* c, int32_t scene, int64_t n, double* s, double* dA, uint8_t* kind, double* gamma,
                           int32_t* parent, double* bpos) {
    if (!c) return MPM_ERR_INVALID_ARG;
    if (scene < 0 || scene >= c->nsc || n < 0) return fail(c, MPM_ERR_INVALID_ARG, "mpm_get_surface: bad scene or count");
    if (n == 0 || c->ns == 0) return MPM_OK;
    cudaStream_t st = c->st;
    Dev& d = c->d;
    struct Field { double* out; int comps; double* src[3]; };
    Field fields[4] = {{s, 3, {d.s[0], d.s[1], d.s[2]}}, {dA, 3, {d.dA[0], d.dA[1], d.dA[2]}},
                       {bpos, 3, {d.bpos[0], d.bpos[1], d.bpos[2]}}, {gamma, 1, {d.gamma, nullptr, nullptr}}};
    for (int f = 0; f < 4; ++f) {
        Field& fd = fields[f];
        if (!fd.out) continue;
        double** dsrc = (double**)d.dense_b;
        MPM_CUDA(cudaMemcpyAsync(dsrc, fd.src, sizeof(double*) * fd.comps, cudaMemcpyHostToDevice, st));
        MPM_LAUNCH k_stage_out<<<nblk(c->ns, 256), 256, 0, st>>>((int)c->ns, scene, (int)n, d.ssc, d.sid, (const double* const*)dsrc,
                                                      fd.comps, (double*)d.dense_a);
        MPM_CUDA(cudaMemcpyAsync(fd.out, d.dense_a, sizeof(double) * fd.comps * n, cudaMemcpyDefault, st));
        MPM_CUDA(cudaStreamSynchronize(st));
    }
    if (kind) {
        MPM_LAUNCH k_stage_out_u8<<<nblk(c->ns, 256), 256, 0, st>>>((int)c->ns, scene, (int)n, d.ssc, d.sid, d.kind, (uint8_t*)d.dense_a);
        MPM_CUDA(cudaMemcpyAsync(kind, d.dense_a, (size_t)n, cudaMemcpyDefault, st));
        MPM_CUDA(cudaStreamSynchronize(st));
    }
    if (parent) {
        MPM_LAUNCH k_stage_parent<<<nblk(c->ns, 256), 256, 0, st>>>((int)c->ns, (int)c->np, scene, (int)n, d.ssc, d.sid, d.parent, d.pid,
                                                         (int32_t*)d.dense_a);
        MPM_CUDA(cudaMemcpyAsync(parent, d.dense_a, sizeof(int32_t) * n, cudaMemcpyDefault, st));
        MPM_CUDA(cudaStreamSynchronize(st));
    }
    return check_device_error(c);
}

mpm_status mpm_generate_surface(mpm_ctx* c, uint64_t seed, double per_cell_area, int64_t* counts) {
    return mpm_generate_surface_method(c, seed, per_cell_area, MPM_ISO_TETRAHEDRA, counts);
}

mpm_status mpm_generate_surface_method(mpm_ctx* c, uint64_t seed, double per_cell_area, int32_t method,
                                       int64_t* counts) {
    if (!c) return MPM_ERR_INVALID_ARG;
    if (!(per_cell_area > 0.0) || !std::isfinite(per_cell_area))
        return fail(c, MPM_ERR_INVALID_ARG, "mpm_generate_surface: per_cell_area must be positive");
    if (method != MPM_ISO_TETRAHEDRA && method != MPM_ISO_CUBES)
        return fail(c, MPM_ERR_INVALID_ARG, "mpm_generate_surface_method: unknown isosurface method");
    if (c->hscene_cnt.size() != (size_t)c->nsc) {
        c->hscene_cnt.assign(c->nsc, 0ull);
        c->hscene_first.assign(c->nsc, 0ll);
    }
    std::vector<long long> cnt(c->nsc, 0);
    int cap_err = 0;
    PhaseTimer timer(c, 0);
    MPM_CUDA(launch_generate_surface(c, (unsigned long long)seed, per_cell_area, method, cnt.data(), &cap_err));
    MPM_CUDA(cudaStreamSynchronize(c->st));
    mpm_status s = check_device_error(c);
    if (s != MPM_OK) return s;
    if (cap_err) return fail(c, MPM_ERR_CAPACITY, "mpm_generate_surface: more samples than max_surface");
    if (counts)
        for (int k = 0; k < c->nsc; ++k) counts[k] = cnt[k];
    return MPM_OK;
}

mpm_status mpm_resample(mpm_ctx* c) {
    if (!c) return MPM_ERR_INVALID_ARG;
    PhaseTimer timer(c, 0);
    cudaStream_t st = c->st;
    MPM_CUDA(launch_sort_particles(c));
    MPM_CUDA(launch_sort_surface(c));
    MPM_CUDA(cudaStreamSynchronize(st));
    mpm_status s = check_device_error(c);
    if (s != MPM_OK) return s;
    MPM_CUDA(launch_nearest_parent(c));
    MPM_CUDA(launch_build_blocks(c));
    s = check_device_error(c);
    if (s != MPM_OK) return s;
    c->resampled = true;
    c->p2g_done = false;
    return MPM_OK;
}

mpm_status mpm_p2g(mpm_ctx* c) {
    if (!c) return MPM_ERR_INVALID_ARG;
    if (!c->resampled) return fail(c, MPM_ERR_INVALID_ARG, "mpm_p2g: call mpm_resample first");
    PhaseTimer timer(c, 1);
    MPM_CUDA(launch_p2g(c));
    MPM_CUDA(launch_pack_step(c));
    c->p2g_done = true;
    return MPM_OK;
}

mpm_status mpm_get_grid(mpm_ctx* c, int32_t scene, int32_t field, double* out) {
    if (!c) return MPM_ERR_INVALID_ARG;
    if (scene < 0 || scene >= c->nsc || !out) return fail(c, MPM_ERR_INVALID_ARG, "mpm_get_grid: bad scene or pointer");
    Dev& d = c->d;
    const double* src = nullptr;
    int comps = 1;
    switch (field) {
        case MPM_FIELD_MASS: src = d.gm; break;
        case MPM_FIELD_MOMENTUM: src = d.gmv; comps = 3; break;
        case MPM_FIELD_VN: src = d.gvn; comps = 3; break;
        case MPM_FIELD_THERMAL_MASS: src = d.gmT; break;
        case MPM_FIELD_TN: src = d.gTn; break;
        case MPM_FIELD_VHAT: src = d.gvhat; comps = 3; break;
        case MPM_FIELD_THAT: src = d.gThat; break;
        case MPM_FIELD_ITERATE: src = d.gv; comps = 3; break;
        default: return fail(c, MPM_ERR_INVALID_ARG, "mpm_get_grid: unknown field");
    }
    const SceneDev& S = c->hsc[scene];
    size_t nodes = (size_t)S.n[0] * S.n[1] * S.n[2];
    cudaStream_t st = c->st;
    MPM_CUDA(cudaMemsetAsync(d.dense_a, 0, sizeof(double) * nodes * comps, st));
    MPM_CUDA(launch_grid_to_dense(c, scene, src, d.dense_a, comps, 8, 8));
    MPM_CUDA(cudaMemcpyAsync(out, d.dense_a, sizeof(double) * nodes * comps, cudaMemcpyDefault, st));
    MPM_CUDA(cudaStreamSynchronize(st));
    return check_device_error(c);
}

mpm_status mpm_set_velocity(mpm_ctx* c, int32_t scene, const double* v) {
    if (!c) return MPM_ERR_INVALID_ARG;
    if (scene < 0 || scene >= c->nsc || !v) return fail(c, MPM_ERR_INVALID_ARG, "mpm_set_velocity: bad scene or pointer");
    if (!c->p2g_done) return fail(c, MPM_ERR_INVALID_ARG, "mpm_set_velocity: call mpm_p2g first");
    Dev& d = c->d;
    const SceneDev& S = c->hsc[scene];
    size_t nodes = (size_t)S.n[0] * S.n[1] * S.n[2];
    cudaStream_t st = c->st;
    MPM_CUDA(cudaMemcpyAsync(d.dense_a, v, sizeof(double) * nodes * 3, cudaMemcpyDefault, st));
    MPM_CUDA(launch_dense_to_grid(c, scene, d.dense_a, d.gv, 3, 8));
    MPM_CUDA(launch_eval(c, false, true));
    MPM_CUDA(cudaStreamSynchronize(st));
    c->step_ready = true;
    return check_device_error(c);
}

mpm_status mpm_energy_gradient(mpm_ctx* c, int32_t scene, double* grad, double* energy) {
    if (!c) return MPM_ERR_INVALID_ARG;
    if (scene < 0 || scene >= c->nsc) return fail(c, MPM_ERR_INVALID_ARG, "mpm_energy_gradient: bad scene");
    if (!c->step_ready) return fail(c, MPM_ERR_INVALID_ARG, "mpm_energy_gradient: call mpm_set_velocity first");
    Dev& d = c->d;
    cudaStream_t st = c->st;
    MPM_CUDA(launch_eval(c, false, true));
    MPM_CUDA(cudaMemcpyAsync(c->hscal, d.scal, sizeof(SceneScal) * c->nsc, cudaMemcpyDeviceToHost, st));
    MPM_CUDA(cudaStreamSynchronize(st));
    if (energy) *energy = c->hscal[scene].phi_kin + c->hscal[scene].phi_part;
    if (grad) {
        const SceneDev& S = c->hsc[scene];
        size_t nodes = (size_t)S.n[0] * S.n[1] * S.n[2];
        MPM_CUDA(cudaMemsetAsync(d.dense_a, 0, sizeof(double) * nodes * 3, st));
        MPM_CUDA(launch_grid_to_dense(c, scene, d.ggrad, d.dense_a, 3, 8, 8));
        MPM_CUDA(cudaMemcpyAsync(grad, d.dense_a, sizeof(double) * nodes * 3, cudaMemcpyDefault, st));
        MPM_CUDA(cudaStreamSynchronize(st));
    }
    return check_device_error(c);
}

mpm_status mpm_apply_hessian(mpm_ctx* c, int32_t scene, const void* dv, void* out, int32_t mode) {
    if (!c) return MPM_ERR_INVALID_ARG;
    if (scene < 0 || scene >= c->nsc || !dv || !out || (mode != MPM_HESS_EXACT && mode != MPM_HESS_PROJECTED))
        return fail(c, MPM_ERR_INVALID_ARG, "mpm_apply_hessian: bad scene, pointer or mode");
    if (!c->step_ready) return fail(c, MPM_ERR_INVALID_ARG, "mpm_apply_hessian: call mpm_set_velocity first");
    Dev& d = c->d;
    cudaStream_t st = c->st;
    const SceneDev& S = c->hsc[scene];
    size_t nodes = (size_t)S.n[0] * S.n[1] * S.n[2];
    size_t rs = c->rsize;
    MPM_CUDA(cudaMemcpyAsync(d.dense_a, dv, rs * nodes * 3, cudaMemcpyDefault, st));
    MPM_CUDA(launch_dense_to_grid(c, scene, d.dense_a, d.cp, 3, c->rsize));
    MPM_CUDA(launch_project_vec(c, d.cp, c->rsize));
    MPM_CUDA(cudaMemsetAsync(d.cu, 0, rs * (size_t)c->NB * 192, st));
    MPM_CUDA(launch_apply(c, d.cp, d.cu, mode));
    MPM_CUDA(launch_mass_term(c, d.cp, d.cu));
    MPM_CUDA(cudaMemsetAsync(d.dense_b, 0, rs * nodes * 3, st));
    MPM_CUDA(launch_grid_to_dense(c, scene, d.cu, d.dense_b, 3, c->rsize, c->rsize));
    MPM_CUDA(cudaMemcpyAsync(out, d.dense_b, rs * nodes * 3, cudaMemcpyDefault, st));
    MPM_CUDA(cudaStreamSynchronize(st));
    return check_device_error(c);
}

mpm_status mpm_heat_apply(mpm_ctx* c, int32_t scene, const void* T, void* out) {
    if (!c) return MPM_ERR_INVALID_ARG;
    if (scene < 0 || scene >= c->nsc || !T || !out) return fail(c, MPM_ERR_INVALID_ARG, "mpm_heat_apply: bad scene or pointer");
    if (!c->p2g_done) return fail(c, MPM_ERR_INVALID_ARG, "mpm_heat_apply: call mpm_p2g first");
    Dev& d = c->d;
    cudaStream_t st = c->st;
    const SceneDev& S = c->hsc[scene];
    size_t nodes = (size_t)S.n[0] * S.n[1] * S.n[2];
    size_t rs = c->rsize;
    MPM_CUDA(cudaMemcpyAsync(d.dense_a, T, rs * nodes, cudaMemcpyDefault, st));
    MPM_CUDA(launch_dense_to_grid(c, scene, d.dense_a, d.hp, 1, c->rsize));
    MPM_CUDA(cudaMemsetAsync(d.hu, 0, rs * (size_t)c->NB * 64, st));
    MPM_CUDA(launch_heat_full(c, d.hp, d.hu));
    MPM_CUDA(cudaMemsetAsync(d.dense_b, 0, rs * nodes, st));
    MPM_CUDA(launch_grid_to_dense(c, scene, d.hu, d.dense_b, 1, c->rsize, c->rsize));
    MPM_CUDA(cudaMemcpyAsync(out, d.dense_b, rs * nodes, cudaMemcpyDefault, st));
    MPM_CUDA(cudaStreamSynchronize(st));
    return check_device_error(c);
}

mpm_status mpm_newton_step(mpm_ctx* c, mpm_stats* stats) {
    if (!c) return MPM_ERR_INVALID_ARG;
    if (!c->p2g_done) return fail(c, MPM_ERR_INVALID_ARG, "mpm_newton_step: call mpm_p2g first");
    cudaStream_t st = c->st;
    {
        PhaseTimer timer(c, 2);
        MPM_CUDA(run_heat(c));
    }
    {
        PhaseTimer timer(c, 3);
        MPM_CUDA(run_newton(c));
    }
    MPM_CUDA(cudaMemcpyAsync(c->hscal, c->d.scal, sizeof(SceneScal) * c->nsc, cudaMemcpyDeviceToHost, st));
    MPM_CUDA(cudaStreamSynchronize(st));
    mpm_status worst = MPM_OK;
    for (int s = 0; s < c->nsc; ++s) {
        const SceneScal& h = c->hscal[s];
        if (stats) {
            stats[s].newton_iters = h.newton_it;
            stats[s].cg_iters = h.cg_total;
            stats[s].heat_iters = h.heat_it;
            stats[s].status = h.status;
            stats[s].residual0 = h.r0;
            stats[s].residual = h.rnorm;
            for (int q = 0; q < 3; ++q) stats[s].momentum[q] = h.mom[q];
        }
        if (h.status != 0 && worst == MPM_OK) worst = (mpm_status)h.status;
        if (c->prof) {
            c->pr.newton_iters += h.newton_it;
            c->pr.cg_iters += h.cg_total;
            c->pr.heat_iters += h.heat_it;
        }
    }
    c->step_ready = true;
    mpm_status e = check_device_error(c);
    if (e != MPM_OK) return e;
    if (worst != MPM_OK) c->last_error = "a scene did not converge (see stats)";
    return worst;
}

mpm_status mpm_g2p(mpm_ctx* c) {
    if (!c) return MPM_ERR_INVALID_ARG;
    if (!c->p2g_done) return fail(c, MPM_ERR_INVALID_ARG, "mpm_g2p: call mpm_newton_step first");
    PhaseTimer timer(c, 4);
    MPM_CUDA(launch_g2p(c));
    c->resampled = false;
    c->p2g_done = false;
    c->step_ready = false;
    return MPM_OK;
}

mpm_status mpm_step(mpm_ctx* c, mpm_stats* stats) {
    mpm_status s = mpm_resample(c);
    if (s != MPM_OK) return s;
    s = mpm_p2g(c);
    if (s != MPM_OK) return s;
    mpm_status sn = mpm_newton_step(c, stats);
    if (sn != MPM_OK && sn != MPM_ERR_NOT_CONVERGED) return sn;
    s = mpm_g2p(c);
    if (s != MPM_OK) return s;
    return sn;
}

mpm_status mpm_sync(mpm_ctx* c) {
    if (!c) return MPM_ERR_INVALID_ARG;
    cudaError_t e = cudaStreamSynchronize(c->st);
    if (e != cudaSuccess) return fail(c, MPM_ERR_CUDA, cudaGetErrorString(e));
    return check_device_error(c);
}

mpm_status mpm_counts(mpm_ctx* c, int64_t* n_particles, int64_t* n_surface, int64_t* n_blocks, int64_t* n_work_blocks) {
    if (!c) return MPM_ERR_INVALID_ARG;
    if (n_particles) *n_particles = c->np;
    if (n_surface) *n_surface = c->ns;
    if (n_blocks) *n_blocks = c->NB;
    if (n_work_blocks) *n_work_blocks = c->NW;
    return MPM_OK;
}

mpm_status mpm_profile_enable(mpm_ctx* c, int32_t enable) {
    if (!c) return MPM_ERR_INVALID_ARG;
    c->prof = enable != 0;
    if (c->prof) {
        memset(&c->pr, 0, sizeof(c->pr));
        c->pr.kernel_launches = -c->launches;   // counts from here
    }
    c->nev = 0;
    return MPM_OK;
}

mpm_status mpm_profile_apply(mpm_ctx* c, int32_t n_applies, int32_t mode, double* ms_per_apply) {
    if (!c) return MPM_ERR_INVALID_ARG;
    if (n_applies < 1 || !ms_per_apply || (mode != MPM_HESS_EXACT && mode != MPM_HESS_PROJECTED))
        return fail(c, MPM_ERR_INVALID_ARG, "mpm_profile_apply: bad count, pointer or mode");
    if (!c->step_ready) return fail(c, MPM_ERR_INVALID_ARG, "mpm_profile_apply: call mpm_newton_step first");
    Dev& d = c->d;
    cudaStream_t st = c->st;
    // the solver's last CG direction at the frozen iterate; the products
    // accumulate in the CG's product vector, which is cleared afterwards
    MPM_CUDA(cudaMemsetAsync(d.cu, 0, (size_t)c->rsize * (size_t)c->NB * 192, st));
    MPM_CUDA(launch_apply(c, d.cp, d.cu, mode));   // warm-up
    MPM_CUDA(cudaEventRecord(c->ev[32], st));
    for (int k = 0; k < n_applies; ++k) MPM_CUDA(launch_apply(c, d.cp, d.cu, mode));
    MPM_CUDA(cudaEventRecord(c->ev[33], st));
    MPM_CUDA(cudaEventSynchronize(c->ev[33]));
    float ms = 0.f;
    MPM_CUDA(cudaEventElapsedTime(&ms, c->ev[32], c->ev[33]));
    *ms_per_apply = (double)ms / n_applies;
    MPM_CUDA(cudaMemsetAsync(d.cu, 0, (size_t)c->rsize * (size_t)c->NB * 192, st));
    MPM_CUDA(cudaStreamSynchronize(st));
    return check_device_error(c);
}

mpm_status mpm_get_profile(mpm_ctx* c, mpm_profile* out) {
    if (!c || !out) return MPM_ERR_INVALID_ARG;
    *out = c->pr;
    out->kernel_launches = c->pr.kernel_launches + c->launches;
    out->cg_ctas_per_sm = c->cg_ctas_per_sm;
    out->cg_chunk = c->cg_chunk;
    out->cg_graphs = c->use_graphs ? 1 : 0;
    out->cg_graph_error = c->graph_error;
    out->op_rows_per_chunk = c->op_rows;
    out->reserved_ = 0;
    return MPM_OK;
}

}  // extern "C"
