// Device-side definitions shared by the library's kernels.
//
// Grid layout: every scene's grid is cut into blocks of 4x4x4 nodes. Only blocks
// touched by a particle stencil are stored ("active blocks", compacted into slots
// 0..NB-1 in global-block order). A scalar grid field stores node l = x + 4y + 16z
// of slot s at s*64 + l; a vector field stores component c at s*192 + c*64 + l.
// Particles are sorted by cell with a block-major cell key, so the particles of a
// block are contiguous. A quadratic B-spline stencil of a particle in cell c
// covers nodes c-1 .. c+1 (nodes sit at cell centres, paper section "Transfer:
// P2G"), so a block's particles touch the block's nodes plus a one-node halo:
// 6x6x6 nodes, staged in shared memory by the kernels that walk a block.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace mpm {

constexpr int BS = 4;       // block edge in nodes / cells
constexpr int BN = 64;      // nodes per block
constexpr int HE = 6;       // halo edge (block + one node each side)
constexpr int HN = 216;     // halo nodes
constexpr int MAX_LS = 16;  // line-search trials (alpha = 2^-k, k < MAX_LS)
constexpr int LS_FIRST = 2; // trials the line search's first pass evaluates (alpha = 1, 1/2)

// Per-scene constants.
struct SceneDev {
    int n[3];
    int nb[3];               // blocks per axis
    long long block_base;    // first global block id of this scene
    double dx, inv_dx;
    double origin[3];
    double dt, g[3], rho, lambda_l, mu_l, E0, nu, T0, T_melt, cp, K, h, H;
    int gamma_law, thermal, phase_change, plane_mode;
    double gamma_p[4], gamma_lg, gamma_sl;
    int walls[6];
    double plane_n[3], plane_d;
    float plane_nf[3], pad_f_;      // plane normal in float32 (the float32 projections)
    double sphere_c[3], sphere_R;   // spherical solid: centre and radius
    int sphere_outside, sphere_mode;
    double newton_tol, cg_rtol, heat_rtol;
    int max_newton, max_cg, max_ls, massless;
    double friction;             // Coulomb coefficient at slip nodes of the plane and the sphere
    long long p_begin, p_end;    // interior particles (set order == storage offset)
    long long s_begin, s_end;    // surface samples
};

// Per-scene solver scalars (float64), live on the device.
struct SceneScal {
    double rr, rz, rz_new, pAp, bnorm, r0, rnorm, slope;
    double phi_kin, phi_part;
    double dphi[MAX_LS];
    double dkd;        // d . K_liquid d of the current Newton direction
    double alpha;
    double mom[3];
    int cg_it, cg_total, newton_it, cg_done, newton_done, ls_pick, status, heat_it;
};

// Device error word bits.
enum : int {
    ERR_DOMAIN = 1,        // particle or sample outside cells 1..n-2
    ERR_FAR_SURFACE = 2,   // no interior particle within dx of a surface sample
    ERR_NUMERIC = 4,
    ERR_CAPACITY = 8,      // more active grid blocks than max_blocks
    ERR_SOLID = 16,        // solid particle without solid buffers
    ERR_TIMEOUT = 32,      // a bounded device wait ran out
};

__device__ __forceinline__ long long cell_key(const SceneDev& S, int cx, int cy, int cz) {
    int bx = cx >> 2, by = cy >> 2, bz = cz >> 2;
    long long gb = S.block_base + bx + (long long)S.nb[0] * (by + (long long)S.nb[1] * bz);
    return gb * 64 + ((cx & 3) + 4 * (cy & 3) + 16 * (cz & 3));
}

// One-axis quadratic B-spline weights for a point at fraction t in [0, 1) of
// its cell (distance to the three nodes c-1, c, c+1 is f, f-1, f-2 with
// f = t + 1/2): w0 = (3/2 - f)^2/2, w1 = 3/4 - (f-1)^2, w2 = (f - 1/2)^2/2.
// dw are d/df (divide by dx for d/dx).
template <typename R>
__device__ __forceinline__ void bspline(R f, R* w, R* dw) {
    R a = R(1.5) - f;
    R b = f - R(1.0);
    R c = f - R(0.5);
    w[0] = R(0.5) * a * a;
    w[1] = R(0.75) - b * b;
    w[2] = R(0.5) * c * c;
    dw[0] = -a;
    dw[1] = R(-2.0) * b;
    dw[2] = c;
}

// Stencil of a point given u = (x - origin)/dx: cell, fraction and weights.
template <typename R>
struct Stencil {
    int c[3];       // cell
    R w[3][3];      // [axis][node]
    R dw[3][3];     // d/dx
};

template <typename R>
__device__ __forceinline__ void make_stencil(const double u[3], R inv_dx, Stencil<R>& st) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        double fl = floor(u[a]);
        st.c[a] = (int)fl;
        // f = u - 1/2 - (c - 1) in [1/2, 3/2)
        R f = (R)(u[a] - 0.5 - (fl - 1.0));
        bspline<R>(f, st.w[a], st.dw[a]);
#pragma unroll
        for (int k = 0; k < 3; ++k) st.dw[a][k] *= inv_dx;
    }
}

// Same from a position relative to a block origin in cell units (float path).
template <typename R>
__device__ __forceinline__ void make_stencil_local(R ux, R uy, R uz, R inv_dx, int lc[3], R w[3][3], R dw[3][3]) {
    R u[3] = {ux, uy, uz};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        // u lies in [0, 4) in exact arithmetic; rounding to R can give exactly 4,
        // which is the right edge of cell 3 (weights 0, 1/2, 1/2): clamp the cell
        R fl = floor(u[a]);
        fl = fl > R(BS - 1) ? R(BS - 1) : (fl < R(0) ? R(0) : fl);
        lc[a] = (int)fl;
        R f = u[a] - fl + R(0.5);
        bspline<R>(f, w[a], dw[a]);
#pragma unroll
        for (int k = 0; k < 3; ++k) dw[a][k] *= inv_dx;
    }
}

// Padded shared-memory layout of a block's 6x6x6 halo: x + 8 y + 52 z, so the 32
// cells of a warp (a 4x4x2 brick) read or write 32 distinct banks.
constexpr int PY = 8, PZ = 52, PN = 312;
__device__ __forceinline__ int pidx(int x, int y, int z) { return x + PY * y + PZ * z; }
// Accumulation halo of a block written by its two warps: warp 0's node levels
// 0..3 at levels 0..3, warp 1's levels 2..5 at 4..7 (the warps never share a word).
constexpr int UZ = 8;
constexpr int UN = PZ * UZ;

// Halo rows along x: the four middle nodes of a row belong to one neighbour block
// and are contiguous there (x fastest), so they move as one vector; the two end
// nodes belong to the x-neighbours.
template <typename R>
__device__ __forceinline__ void halo_row(const int* __restrict__ nbr, int slot, int hy, int hz, int& nmid, int& nlo,
                                         int& nhi, int& base) {
    int oy = hy - 1, oz = hz - 1;
    int by = oy < 0 ? -1 : (oy >= BS ? 1 : 0), bz = oz < 0 ? -1 : (oz >= BS ? 1 : 0);
    const int* nb = nbr + slot * 27 + 3 * (by + 1) + 9 * (bz + 1);
    nlo = nb[0];
    nmid = nb[1];
    nhi = nb[2];
    base = BS * ((oy - BS * by) + BS * (oz - BS * bz));   // local index of x = 0 in the row
}

// Lame coefficients of the solid at temperature T (section "Thermomechanical
// Material Dependence and Phase Change"): shear mu = E(T) / (2 (1 + nu)) with
// E(T) = E0 max(0, (T_melt - T)/(T_melt - T0)); the volumetric coefficient is the
// scene's bulk modulus lambda_l at every temperature (one bulk modulus for the
// liquid and solid phases), so a solid at the melting point stores the liquid's
// energy.
__device__ __forceinline__ void solid_lame(const SceneDev& S, double T, double& mu, double& lam) {
    const double E = S.E0 == 0.0 ? 0.0 : S.E0 * fmax(0.0, (S.T_melt - T) / (S.T_melt - S.T0));
    mu = E / (2.0 * (1.0 + S.nu));
    lam = S.lambda_l;
}

// Signed distance of x to the spherical solid (negative inside the solid) and
// its unit normal (the gradient, pointing into the liquid); the direction is
// (0, 0, 1) from (x - c) at the centre itself.
__device__ __forceinline__ double sphere_phi_normal(const SceneDev& S, const double x[3], double n[3]) {
    double d[3] = {x[0] - S.sphere_c[0], x[1] - S.sphere_c[1], x[2] - S.sphere_c[2]};
    double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    double u[3] = {0.0, 0.0, 1.0};
    if (r > 1e-300) {
        u[0] = d[0] / r;
        u[1] = d[1] / r;
        u[2] = d[2] / r;
    }
    const double sgn = S.sphere_outside ? -1.0 : 1.0;
    for (int a = 0; a < 3; ++a) n[a] = sgn * u[a];
    return S.sphere_outside ? S.sphere_R - r : r - S.sphere_R;
}

// position of node l (0..63) of the block at bc
__device__ __forceinline__ void node_position(const SceneDev& S, int4 bc, int l, double x[3]) {
    x[0] = S.origin[0] + ((double)(bc.x * BS + (l & 3)) + 0.5) * S.dx;
    x[1] = S.origin[1] + ((double)(bc.y * BS + ((l >> 2) & 3)) + 0.5) * S.dx;
    x[2] = S.origin[2] + ((double)(bc.z * BS + (l >> 4)) + 0.5) * S.dx;
}

__device__ __forceinline__ int halo_index(int hx, int hy, int hz) { return hx + HE * (hy + HE * hz); }

// Halo node h (0..215) of block `slot`: which neighbour slot and which local node.
__device__ __forceinline__ void halo_source(const int* __restrict__ nbr, int slot, int h, int& nslot, int& local) {
    int hx = h % HE, hy = (h / HE) % HE, hz = h / (HE * HE);
    int ox = hx - 1, oy = hy - 1, oz = hz - 1;   // node offset from block origin, -1..4
    int bx = ox < 0 ? -1 : (ox >= BS ? 1 : 0);
    int by = oy < 0 ? -1 : (oy >= BS ? 1 : 0);
    int bz = oz < 0 ? -1 : (oz >= BS ? 1 : 0);
    nslot = nbr[slot * 27 + (bx + 1) + 3 * (by + 1) + 9 * (bz + 1)];
    local = (ox - BS * bx) + BS * ((oy - BS * by) + BS * (oz - BS * bz));
}

// 3x3 helpers (row-major m[3*i + j])
template <typename R>
__device__ __forceinline__ void cofactor(const R* F, R* C) {
    C[0] = F[4] * F[8] - F[5] * F[7];
    C[1] = F[5] * F[6] - F[3] * F[8];
    C[2] = F[3] * F[7] - F[4] * F[6];
    C[3] = F[2] * F[7] - F[1] * F[8];
    C[4] = F[0] * F[8] - F[2] * F[6];
    C[5] = F[1] * F[6] - F[0] * F[7];
    C[6] = F[1] * F[5] - F[2] * F[4];
    C[7] = F[2] * F[3] - F[0] * F[5];
    C[8] = F[0] * F[4] - F[1] * F[3];
}

// Directional derivative of the cofactor: dC = d cof(F)[D]
template <typename R>
__device__ __forceinline__ void dcofactor(const R* F, const R* D, R* C) {
    C[0] = D[4] * F[8] + F[4] * D[8] - D[5] * F[7] - F[5] * D[7];
    C[1] = D[5] * F[6] + F[5] * D[6] - D[3] * F[8] - F[3] * D[8];
    C[2] = D[3] * F[7] + F[3] * D[7] - D[4] * F[6] - F[4] * D[6];
    C[3] = D[2] * F[7] + F[2] * D[7] - D[1] * F[8] - F[1] * D[8];
    C[4] = D[0] * F[8] + F[0] * D[8] - D[2] * F[6] - F[2] * D[6];
    C[5] = D[1] * F[6] + F[1] * D[6] - D[0] * F[7] - F[0] * D[7];
    C[6] = D[1] * F[5] + F[1] * D[5] - D[2] * F[4] - F[2] * D[4];
    C[7] = D[2] * F[3] + F[2] * D[3] - D[0] * F[5] - F[0] * D[5];
    C[8] = D[0] * F[4] + F[0] * D[4] - D[1] * F[3] - F[1] * D[3];
}

template <typename R>
__device__ __forceinline__ R det3(const R* F) {
    return F[0] * (F[4] * F[8] - F[5] * F[7]) - F[1] * (F[3] * F[8] - F[5] * F[6]) +
           F[2] * (F[3] * F[7] - F[4] * F[6]);
}

template <typename R>
__device__ __forceinline__ void matmul3(const R* A, const R* B, R* C) {
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) C[3 * i + j] = A[3 * i] * B[j] + A[3 * i + 1] * B[3 + j] + A[3 * i + 2] * B[6 + j];
}

// C = A B^T
template <typename R>
__device__ __forceinline__ void matmul3_bt(const R* A, const R* B, R* C) {
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j)
            C[3 * i + j] = A[3 * i] * B[3 * j] + A[3 * i + 1] * B[3 * j + 1] + A[3 * i + 2] * B[3 * j + 2];
}

// Record of one surface sample for the Hessian operator: its projected-Hessian
// map K (symmetric 9x9 on dF^ flattened row-major, rows 3q..3q+2 belong to
// component q) grouped in 3x3 blocks, then its position in its block:
//   [0, 6)   D0 = K(0,0) upper triangle (00 01 02 11 12 22), [6, 12) D1, [12, 18) D2,
//   [18, 27) O01 = K(0,1) row-major, [27, 36) O02, [36, 45) O12, [45, 48) position,
//   [48, 52) unused: a stride of 52 values puts the records of the samples read
//   together on 8 different shared-memory banks (48 would give 2) and keeps every
//   record 16-byte aligned for the bulk copy.
// The lane computing row block q of G = K dF^ reads D_q and the two off-diagonal
// blocks of its rows (transposed where they lie below the diagonal).
constexpr int SREC = 52;
__host__ __device__ constexpr int sample_map_index(int m, int l) {   // m <= l
    return (m / 3 == l / 3) ? 6 * (m / 3) + (m % 3) * 3 - (m % 3) * ((m % 3) - 1) / 2 + (l % 3 - m % 3)
                            : (m / 3 == 0 ? (l / 3 == 1 ? 18 : 27) : 36) + 3 * (m % 3) + (l % 3);
}

// Four values of one type, 16- (float) or 32-byte (double) aligned: the packed
// per-particle record of the Hessian operator.
template <typename R>
struct alignas(4 * sizeof(R)) R4 {
    R x, y, z, w;
};

// ---- TMA bulk copy global -> shared with an mbarrier (sm_90+ PTX) ----
__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}

// bytes: multiple of 16; dst and src 16-byte aligned
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// bounded wait on an mbarrier phase; false after `limit` polls
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, long long limit) {
    for (long long it = 0; it < limit; ++it)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

// warp + block sum of a double, then one atomicAdd per block
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

template <int NT>
__device__ __forceinline__ void block_atomic_sum(double v, double* target, double* sbuf /* NT/32 */) {
    v = warp_sum(v);
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sbuf[w] = v;
    __syncthreads();
    if (w == 0) {
        double s = lane < NT / 32 ? sbuf[lane] : 0.0;
        s = warp_sum(s);
        if (lane == 0 && s != 0.0) atomicAdd(target, s);
    }
}

}  // namespace mpm
