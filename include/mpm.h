/*
 * mpm.h -- C ABI of the GB300 implicit APIC-MPM surface-energy library.
 *
 * The library advances one or more independent scenes through the time step of
 * "A Momentum-Conserving Implicit Material Point Method for Surface Energies
 * with Spatial Gradients" (arXiv 2101.12408), section "Discretization":
 *   (1) resample the surface (surface + balance particles, mass split),
 *   (2) P2G of momentum and temperature,
 *   (3) grid update: implicit heat solve and backward-Euler Newton-Krylov solve,
 *   (4) G2P with the conservative merge, particle update and phase change.
 * Every step of that path runs in the library's CUDA kernels (sm_103a).
 *
 * Conventions shared by all entry points
 *   - Units and layout: positions in the scene's length unit; the grid of a scene
 *     has n[0] x n[1] x n[2] cells of edge dx starting at `origin`, and one node at
 *     every cell centre (section "Transfer: P2G": nodes at cell centres).
 *     Dense grid arrays are node-major with x fastest: node (i, j, k) has flat index
 *     i + n0 (j + n1 k); vector fields store 3 consecutive components per node.
 *   - Particle arrays are row-major: x is N x 3, A and F are N x 3 x 3 (row = first
 *     index), all float64.
 *   - Pointers: a pointer argument may be host memory or device memory of the
 *     context's device (the CUDA runtime resolves which); the caller owns it and it
 *     only needs to stay valid until the call returns (calls that read or write it
 *     synchronise the context's stream before returning).
 *   - Particles must lie in cells 1 .. n-2 of every axis (their 27-node stencil
 *     stays inside the grid); violations are reported as MPM_ERR_DOMAIN.
 *   - Errors: every entry point returns an mpm_status; mpm_last_error() gives a
 *     one-line reason. Device-side failures (a particle leaving the grid, a surface
 *     sample with no particle within 2 dx, a non-finite value) are recorded in a
 *     device status word and reported by the next call that synchronises.
 *   - Thread safety: one context per host thread; calls on a context are ordered
 *     on its stream.
 */
#ifndef MPM_GB300_H
#define MPM_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mpm_ctx mpm_ctx;

typedef enum {
    MPM_OK = 0,
    MPM_ERR_INVALID_ARG = 1,   /* bad pointer, size, index or parameter */
    MPM_ERR_CAPACITY = 2,      /* more particles / surface samples than created for */
    MPM_ERR_CUDA = 3,          /* a CUDA runtime call failed */
    MPM_ERR_NOT_CONVERGED = 4, /* Newton stopped at max_newton above tolerance */
    MPM_ERR_TIMEOUT = 5,       /* a bounded device wait ran out */
    MPM_ERR_NUMERIC = 6,       /* non-finite value met on the device */
    MPM_ERR_DOMAIN = 7         /* particle or sample outside the valid cells */
} mpm_status;

typedef enum {
    MPM_PREC_FP64 = 0,          /* every operator and vector in float64 */
    MPM_PREC_FP32_FP64RED = 1   /* particle stress / Hessian / heat operators and Krylov
                                   vectors in float32; transfers, grid state, Krylov dot
                                   products, residual norms, line-search energy sums and the
                                   final force evaluation in float64 */
} mpm_precision;

typedef enum {
    MPM_HESS_EXACT = 0,      /* exact second derivative of the objective */
    MPM_HESS_PROJECTED = 1   /* the operator the Newton-CG uses (the paper's "definiteness
                                fix"): each surface sample keeps its Gauss-Newton term and the
                                positive (conformal) part of the cofactor curvature; each solid
                                particle's 9x9 Hessian of psi(F) has its negative eigenvalues
                                set to zero; liquid, viscous and mass terms are unchanged */
} mpm_hess_mode;

typedef enum { MPM_WALL_NONE = 0, MPM_WALL_SLIP = 1, MPM_WALL_STICKY = 2 } mpm_wall;
typedef enum { MPM_GAMMA_CONST = 0, MPM_GAMMA_LINEAR = 1 } mpm_gamma_law;

/* Grid of one scene. Dirichlet velocity conditions (Eq. vbc): the two outer node
 * layers of face f (order x-, x+, y-, y+, z-, z+) follow walls[f]; nodes where the
 * plane's signed distance plane_n . x - plane_d is negative follow plane_mode;
 * nodes inside the spherical solid follow sphere_mode. The sphere (the curved
 * solids of section "Examples") has centre sphere[0..2] and radius sphere[3]; with
 * sphere_outside = 1 the solid is |x - c| > R (a bowl holding the liquid), else
 * |x - c| < R (a ball). A slip node of either solid loses the velocity component
 * along that solid's unit normal at the node (the plane's normal, or (x - c)/|x - c|
 * pointing into the liquid); a sticky node is fixed; a node in both solids, or in
 * a solid and a wall layer, is fixed. Surface samples closer than dx to either
 * solid are solid-liquid. */
typedef struct {
    int32_t n[3];
    double dx;
    double origin[3];
    int32_t walls[6];
    double plane_n[3];
    double plane_d;
    int32_t plane_mode;
    int32_t pad_;
    double sphere[4];
    int32_t sphere_outside;
    int32_t sphere_mode;
} mpm_grid_desc;

/* Physical and solver parameters of one scene (sections "Constitutive Models",
 * "Thermomechanical Material Dependence and Phase Change", "Contact Angle",
 * "Temperature Update"). */
typedef struct {
    double dt;
    double gravity[3];
    double rho;
    double lambda_l;            /* liquid bulk modulus: Psi = lambda/2 (J - 1)^2 */
    double mu_l;                /* liquid viscosity */
    double E0, nu;              /* solid Young's modulus at T <= T0, Poisson ratio */
    double T0, T_melt;          /* E(T) = E0 max(0, (T_melt - T)/(T_melt - T0)) */
    double cp, K, h, H;         /* heat capacity, diffusivity, Robin coefficient, source */
    int32_t gamma_law;          /* MPM_GAMMA_CONST: gamma_lg; MPM_GAMMA_LINEAR:
                                   clamp(gamma_p[0] + gamma_p[1] (T - T0), gamma_p[2], gamma_p[3]) */
    int32_t thermal;            /* 1: heat solve and gamma(T) */
    double gamma_p[4];
    double gamma_lg;            /* liquid-gas coefficient (constant law) */
    double gamma_sl;            /* effective solid-liquid coefficient k_SL - k_SG */
    double newton_tol;          /* stop when |P r| <= newton_tol * max(|P r_0|, 1e-12) */
    double cg_rtol;             /* inner CG relative tolerance */
    double heat_rtol;           /* heat CG tolerance relative to |rhs| */
    int32_t max_newton, max_cg, max_ls;
    int32_t phase_change;       /* 1: melt / freeze at T_melt after G2P */
    double friction;            /* Coulomb coefficient mu_f >= 0 at the slip nodes of the plane and of
                                   the sphere, applied to the end-of-step grid velocity (section
                                   "Examples", inclined ramps): with v~ = v - r/m, n the solid's unit
                                   normal at the node and v_n = v~ . n < 0, the tangential part t
                                   becomes max(0, 1 - mu_f |v_n| / |t|) t; 0 is the frictionless slip */
    int32_t massless_surface;   /* 1: the massless-sample variant the paper compares against (section
                                   "Surface Particle Sampling"): samples carry no mass, no balance
                                   particles, and the parents keep their whole mass. Forces that land
                                   on nodes without mass are lost, so momentum is not conserved */
    int32_t pad_;
} mpm_params;

typedef struct {
    mpm_grid_desc grid;
    mpm_params params;
    int64_t max_particles;      /* capacity of interior particles for this scene */
    int64_t max_surface;        /* capacity of surface samples for this scene */
    int64_t max_blocks;         /* capacity of active 4x4x4-node grid blocks (0: every block of
                                   the grid); exceeding it is MPM_ERR_CAPACITY at mpm_resample */
} mpm_scene_desc;

/* Per-scene statistics of the last mpm_newton_step. */
typedef struct {
    int32_t newton_iters;
    int32_t cg_iters;           /* summed over Newton iterations */
    int32_t heat_iters;
    int32_t status;             /* mpm_status of this scene */
    double residual0;           /* |P r| at the first Newton iterate */
    double residual;            /* |P r| at the last Newton iterate */
    double momentum[3];         /* sum_i m_i v_i of the end-of-step grid velocity (float64) */
    double pad_;
} mpm_stats;

/* Creates a context for `n_scenes` independent scenes advanced together.
 * Allocates every fixed-size device buffer once (particle state, grid, solver
 * vectors, scratch). Two buffers whose size depends on where the particles are
 * grow later, and are kept once grown: the operator's packed particle records,
 * in mpm_p2g when a block's fullest cell needs more rows than the buffer holds,
 * and the triangle buffer of mpm_generate_surface(_method), when a surface has
 * more triangles than it holds. Every other call allocates nothing. `stream` is
 * a cudaStream_t (NULL: the legacy default stream). precision: mpm_precision. */
mpm_status mpm_create(const mpm_scene_desc* scenes, int32_t n_scenes, int32_t precision,
                      void* stream, mpm_ctx** out);
mpm_status mpm_destroy(mpm_ctx* ctx);
const char* mpm_last_error(const mpm_ctx* ctx);

/* Interior particles of one scene (section "Discretization": x, J, v, A, V0, m,
 * T, grad T, plus F and the phase for solids). phase: 0 liquid, 1 solid.
 * Any pointer except x, m, V0 may be NULL (zeros; J = 1, F = I, phase liquid).
 * Arrays are row-major (x: n x 3, A and F: n x 3 x 3) in host or device memory;
 * the call copies them and returns once the caller may reuse them. Host arrays
 * in page-locked memory are copied by DMA at the link's speed, pageable ones
 * through a staging copy. */
mpm_status mpm_set_particles(mpm_ctx* ctx, int32_t scene, int64_t n, const double* x,
                             const double* v, const double* A, const double* m,
                             const double* V0, const double* J, const double* F,
                             const double* T, const double* gradT, const uint8_t* phase);
/* Reads the particles back in the order they were set. NULL pointers are skipped. */
mpm_status mpm_get_particles(mpm_ctx* ctx, int32_t scene, int64_t n, double* x, double* v,
                             double* A, double* J, double* F, double* T, double* gradT,
                             uint8_t* phase);

/* Surface quadrature samples s_r with area-weighted normals dA_r (section
 * "Surface Particle Sampling"), interface kind (0 liquid-gas, 1 solid-liquid),
 * boundary heating b_r and ambient temperature Tbar_r (Eq. heat). kind, b, Tbar
 * may be NULL (zeros). With a solid plane the kind is recomputed by
 * mpm_resample: solid-liquid where the plane distance is below dx. */
mpm_status mpm_set_surface(mpm_ctx* ctx, int32_t scene, int64_t n, const double* s,
                           const double* dA, const uint8_t* kind, const double* b,
                           const double* Tbar);
/* Reads samples back in set order: positions, area normals (carried through the
 * step), kind, surface coefficient gamma_r, the parent particle p(r) (index in
 * mpm_set_particles order) and the balance position b_r. NULL pointers skipped.
 * Samples set by mpm_set_surface or made by mpm_generate_surface have parent -1
 * (and an unset b_r) until the next mpm_resample. */
mpm_status mpm_get_surface(mpm_ctx* ctx, int32_t scene, int64_t n, double* s, double* dA,
                           uint8_t* kind, double* gamma, int32_t* parent, double* bpos);

/* Surface samples generated from the particles (section "Surface Particle
 * Sampling"), replacing every scene's samples; call it before mpm_resample.
 *
 * The level set is the union of spheres of radius 0.867 dx around the interior
 * particles, sampled on the grid nodes (cell centres) as
 * phi = min(distance to the nearest particle, 1.5 dx) - 0.867 dx. Its zero
 * isocontour is triangulated by marching tetrahedra: each cube of 8 nodes is cut
 * into the 6 tetrahedra around its 000-111 diagonal, inside is phi < 0, edge
 * points by linear interpolation, triangles facing outward. Each triangle draws
 * a Poisson count with mean density * area (density = per_cell_area / dx^2,
 * capped at 31) and places that many points uniformly (Osada's construction);
 * every sample carries dA = unit normal / density, so sum |dA| estimates the
 * area without bias. Random numbers come from SplitMix64 seeded with
 * seed ^ (scene * 0x9E3779B97F4A7C15), counter ((6 q + e) 2 + t) 64 + j for
 * triangle t of tetrahedron e of the cube with block-major corner key q, draw j.
 * Kind: solid-liquid where the plane's signed distance is below dx; heating
 * rate b = 0 and ambient temperature T0 on every sample.
 *
 * counts: host array of n_scenes entries receiving each scene's sample count
 * (may be NULL). A scene whose count exceeds its max_surface: MPM_ERR_CAPACITY,
 * samples unchanged. Samples come out in the deterministic enumeration order
 * (cube key, tetrahedron, triangle, draw), which is their set order. */
mpm_status mpm_generate_surface(mpm_ctx* ctx, uint64_t seed, double per_cell_area, int64_t* counts);

/* The isocontour method of mpm_generate_surface_method. */
typedef enum { MPM_ISO_TETRAHEDRA = 0, MPM_ISO_CUBES = 1 } mpm_isosurface;

/* mpm_generate_surface with a choice of triangulation (section "Surface
 * Particle Sampling" names marching cubes, after Chernyaev).
 * MPM_ISO_TETRAHEDRA is mpm_generate_surface itself. MPM_ISO_CUBES is marching
 * cubes: in each cube of 8 nodes the edges that cross the zero level are joined
 * into closed loops face by face (a face with four crossings is resolved by the
 * asymptotic decider: its inside diagonal a, c joins across the face when
 * phi_a phi_c > phi_b phi_d), and each loop becomes a fan of triangles from the
 * crossing of its smallest edge index (edge 4 a + j + 2 k runs along axis a,
 * the other two axes' corner bits j, k in increasing axis order). Loops come
 * from face segments only, so no tunnel through a cube's interior is formed.
 * Triangles face outward; edge points, Poisson counts, Osada points, dA, kind
 * and the seed are as for mpm_generate_surface, except that triangle t of the
 * cube with key q draws counters (12 q + t) 64 + j. Marching cubes makes about
 * a third as many triangles as the tetrahedra; on a union of spheres its area
 * is about 3% smaller (the tetrahedra follow more of the bumps) and it encloses
 * the same volume.
 *
 * method: an mpm_isosurface value, else MPM_ERR_INVALID_ARG. Other arguments,
 * errors and sample order as for mpm_generate_surface. */
mpm_status mpm_generate_surface_method(mpm_ctx* ctx, uint64_t seed, double per_cell_area, int32_t method,
                                       int64_t* counts);

/* (1) Resample: sort by cell, closest interior particle p(r) of each sample
 * (smallest squared distance, ties to the smaller particle index), balance
 * particles b_r = s_r + 2 (x_p(r) - s_r) (Eq. pbal), group sizes |Pi_p| and split
 * masses m~_p = m_p / (2 |Pi_p| + 1) (Eq. cons_mom). */
mpm_status mpm_resample(mpm_ctx* ctx);

/* (2) P2G (section "Transfer: P2G"): grid mass and APIC momentum from interior,
 * surface and balance particles; thermal mass and temperature from interior
 * particles; grid velocity v^n; gamma_r from the grid temperature. */
mpm_status mpm_p2g(mpm_ctx* ctx);

/* Dense float64 copy of one grid field of one scene (length nodes * comps). */
typedef enum {
    MPM_FIELD_MASS = 0, MPM_FIELD_MOMENTUM = 1, MPM_FIELD_VN = 2, MPM_FIELD_THERMAL_MASS = 3,
    MPM_FIELD_TN = 4, MPM_FIELD_VHAT = 5, MPM_FIELD_THAT = 6, MPM_FIELD_ITERATE = 7
} mpm_field;
mpm_status mpm_get_grid(mpm_ctx* ctx, int32_t scene, int32_t field, double* out);

/* Sets the Newton iterate v of one scene (dense float64, nodes x 3) and caches
 * the per-particle state at y = x + dt v (section "Momentum Update"). */
mpm_status mpm_set_velocity(mpm_ctx* ctx, int32_t scene, const double* v);

/* Objective Phi(v) of the backward-Euler system and its gradient dPhi/dv
 * (Eq. disc_force, Eq. fe) at the current iterate: dense float64, nodes x 3,
 * not projected. `energy` (one double) may be NULL. */
mpm_status mpm_energy_gradient(mpm_ctx* ctx, int32_t scene, double* grad, double* energy);

/* Hessian-vector product at the current iterate: out = P H P dv with P the
 * Dirichlet / massless-node projection and H = M + dt^2 d2e/dy2 + dt mu Visc
 * (the linearisation of Eq. fe). dv and out are dense arrays (nodes x 3) of
 * float32 in MPM_PREC_FP32_FP64RED and float64 in MPM_PREC_FP64. mode:
 * mpm_hess_mode. */
mpm_status mpm_apply_hessian(mpm_ctx* ctx, int32_t scene, const void* dv, void* out, int32_t mode);

/* Heat operator (section "Temperature Update"): out = A T with
 * A = c_p m^T/dt + Laplacian (particle quadrature) + Robin (surface quadrature),
 * restricted to nodes with thermal mass. T, out: dense, float32 / float64 as above. */
mpm_status mpm_heat_apply(mpm_ctx* ctx, int32_t scene, const void* T, void* out);

/* (3) Grid update of every scene: heat CG (thermal scenes), then Newton-CG with
 * Armijo line search on Phi, then one explicit force evaluation at the converged
 * iterate. stats: host array of n_scenes entries, or NULL. Returns the worst
 * per-scene status. */
mpm_status mpm_newton_step(mpm_ctx* ctx, mpm_stats* stats);

/* (4) G2P with the conservative merge (section "Transfer: G2P"), particle
 * update x += dt v_p, J / F update, temperature transfer, phase change, and the
 * carried surface samples s += dt v(s), dA <- cof(I + dt grad v(s)) dA. */
mpm_status mpm_g2p(mpm_ctx* ctx);

/* mpm_resample + mpm_p2g + mpm_newton_step + mpm_g2p. */
mpm_status mpm_step(mpm_ctx* ctx, mpm_stats* stats);

/* Waits for the context's stream and reports any device-side error. */
mpm_status mpm_sync(mpm_ctx* ctx);

/* Counts: interior particles, surface samples, active grid blocks (4x4x4 nodes)
 * and blocks holding particles, over all scenes, after the last mpm_resample. */
mpm_status mpm_counts(mpm_ctx* ctx, int64_t* n_particles, int64_t* n_surface,
                      int64_t* n_blocks, int64_t* n_work_blocks);

/* Profiling counters, accumulated while enabled (not part of the paper's method).
 * Kernel durations come from CUDA events recorded on the context's stream around
 * each launch; phase times around each phase call. */
typedef struct {
    int64_t kernel_launches;      /* every kernel the library launched */
    int64_t apply_launches;       /* Hessian-vector operator launches inside Newton-CG */
    double apply_ms;              /* their summed device time */
    int64_t heat_apply_launches;  /* heat operator launches inside the heat CG */
    double heat_apply_ms;
    double phase_ms[5];           /* resample, p2g, heat solve, Newton solve, g2p */
    int64_t newton_iters, cg_iters, heat_iters;
    /* CG launch configuration in use. The first six momentum solves of a context
     * each try one (CTAs per SM of the CG vector kernel x CG iterations between
     * host checks) and later solves keep the fastest per iteration. */
    int32_t cg_ctas_per_sm;       /* 0 before the first solve */
    int32_t cg_chunk;
    int32_t cg_graphs;            /* 1: CG chunks run as CUDA graphs */
    int32_t cg_graph_error;       /* cudaError_t of a refused capture, else 0 */
    /* Hessian operator tile: record rows staged per bulk copy (2, 4 or 8), timed
     * once per context on its first momentum solve; 0 before that solve. The
     * environment variable MPM_OP_ROWS=2|4|8, read by mpm_create, fixes it. */
    int32_t op_rows_per_chunk;
    int32_t reserved_;
} mpm_profile;

/* enable != 0 resets the counters and starts accumulating; 0 stops. */
mpm_status mpm_profile_enable(mpm_ctx* ctx, int32_t enable);
mpm_status mpm_get_profile(mpm_ctx* ctx, mpm_profile* out);

/* Timing of the Hessian-vector operator alone (not part of the paper's method):
 * after one warm-up launch, n_applies back-to-back applications of the operator
 * of mode `mode` (the launches mpm_apply_hessian makes, without its dense copies)
 * to the solver's last CG direction at the iterate the last mpm_newton_step left
 * (call it after mpm_newton_step and before mpm_g2p). *ms_per_apply receives the
 * device time between CUDA events recorded on the context's stream around the
 * n_applies launches, divided by n_applies. Synchronises the stream. */
mpm_status mpm_profile_apply(mpm_ctx* ctx, int32_t n_applies, int32_t mode, double* ms_per_apply);

/* Closest interior particle of each surface sample, computed without allocating.
 *
 * The paper has no counterpart of this entry point: it serves callers that cannot
 * allocate device memory (allocators that forbid cudaMalloc after start-up, hosts
 * that give the library a fixed memory budget) and so cannot create a context. It
 * returns the same parents as mpm_resample: for sample r the index (into x) of the
 * particle with the smallest squared distance, formed as (dx^2 + dy^2) + dz^2 in
 * float64, ties to the smaller index, searched over the 27 cells around the sample
 * and, when none of them holds a particle within dx, over the 125 cells around it.
 *
 * x: n_particles x 3 float64, s: n_samples x 3 float64, parent: n_samples int32, all
 * in memory the device can read / write (device memory, or host memory the device can
 * access); grid: only n, dx and origin are read. stream: a cudaStream_t or NULL.
 * Limits: n_particles <= 524288 and n0 n1 n2 <= 1048576 cells, else MPM_ERR_CAPACITY.
 * Particles must lie in cells 1 .. n-2 and every sample must have a particle within
 * 2 dx (the reach of mpm_resample), else MPM_ERR_DOMAIN (parent = -1 for such
 * samples).
 *
 * Working memory is one fixed device array in the library (about 12.6 MB on every
 * GPU that loads the library, held until the process exits); nothing is allocated or
 * freed. The first call on a device looks up that array's device address and keeps it
 * for the life of the process; make that first call before any stream capture, and
 * do not call this entry point again after a reset of the device (cudaDeviceReset),
 * which the kept address does not survive. Every call reuses the same array and
 * clears the parts that must start at zero, so calls whose work overlaps on the GPU
 * (different streams, or different host threads) race: serialise them. The call
 * reads a status word back and synchronises `stream` before returning. */
mpm_status mpm_nearest_parent_noalloc(const mpm_grid_desc* grid, int64_t n_particles, const double* x,
                                      int64_t n_samples, const double* s, int32_t* parent, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* MPM_GB300_H */
