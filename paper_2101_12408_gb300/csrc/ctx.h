// Host-side context of the library and the launchers of its kernels.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/mpm.h"
#include "common.cuh"

namespace mpm {

// Node projection codes (grid Dirichlet conditions, massless nodes).
enum : uint8_t { PC_FIXED = 1, PC_SLIPX = 2, PC_SLIPY = 4, PC_SLIPZ = 8, PC_PLANE = 16, PC_SPHERE = 32 };

struct Dev {
    // ---- interior particles, float64, sorted by cell (SoA) ----
    double *x[3], *v[3], *A[9], *m, *V0, *J, *F[9], *T, *gT[3];
    uint8_t* phase;
    int *pid, *psc;                 // original index within its scene, scene
    double* scratch_p;              // permutation scratch: particle capacity
    double* scratch_s;              // permutation scratch: sample capacity
    // per-step interior data
    int* gcount;                    // |Pi_p|
    double* mt;                     // split mass
    double* acc[12];                // merged momentum (3) and affine moments (9)
    // operator packs (type R of the context: float or double)
    void* pu[3];                    // position relative to the block origin, in cells
    void* kappa;                    // dt^2 lambda (J^n)^2 V0 (liquid), 0 solid
    void* cvisc;                    // dt mu V^n (liquid), 0 solid
    void* opk;                      // R4 records (block-relative position, kappa; kappa < 0: general
                                    // operator), rank-major per work block: the k-th particle of cell c
                                    // of work block w sits at (wroff[w] + k) * 64 + c
    int* wrows;                     // per work block: record rows (most particles in one of its cells)
    int* wroff;                     // exclusive scan of wrows (+ total)
    int *gen_flag, *gen_pos, *gen_list;   // work blocks with samples or general particles: flag, scan, list
    int *gen_flag_g, *gen_pos_g, *gen_list_g;   // the same for general particles only
    void* Fn[9];                    // F^n (solid)
    void* lame[2];                  // mu, lambda (solid)
    void* scache[24];               // solid per-iterate: F (9), R (9), (tr S I - S)^-1 (6)
    void* Vn;                       // V^n for heat (R)
    // ---- surface samples ----
    double *s[3], *dA[3], *bheat, *Tbar, *gamma, *bpos[3], *Tr;
    uint8_t* kind;
    int *sid, *ssc, *parent;        // parent: sorted interior index
    void* su[3];                    // sample position relative to its block (R)
    void* sa[3];                    // dA (R)
    void* sg;                       // gamma (R)
    void* sF[9];                    // F^ at the iterate (R)
    void* sn[3];                    // unit c (R)
    void* sic;                      // 1/|c| (R)
    void* swn;                      // Robin normaliser 1/sum_j N_j [m^T_j > 0] (R)
    void* sKa;                      // per sample j, SREC values of R at j * SREC: the per-iterate symmetric
                                    // 9x9 projected-Hessian map in 3x3 blocks (sample_map_index), then the
                                    // sample's position in its block (cells) at 45..47
    void* pK[45];                   // the same for a solid particle (R, solid buffers only)
    // ---- sort / blocks ----
    long long* key;                 // interior cell keys
    int* rank;
    int* perm;
    long long* skey;
    int* srank;
    int* sperm;
    int *cell_count, *cell_start;   // interior, over all cells (+1)
    int *scell_count, *scell_start; // surface
    int* bflag;                     // per global block: 1 active
    int* bwork;                     // per global block: 1 holds particles
    int* bslot;                     // per global block: slot or -1
    int* bscan;
    int4* slot_coord;               // bx, by, bz, scene
    int* nbr;                       // 27 neighbour slots per slot
    int* work;                      // work slot list
    int* work_gb;
    int* bw;                        // per global block: its work index (where it holds particles)
    int* slot_gen;                  // per slot: interior particles needing the general operator
    int* counts;                    // [0] NB, [1] NW
    int* scan_tmp;
    // ---- grid (float64) ----
    double *gm, *gmv, *gvn, *gmT, *gmTT, *gTn, *gv, *gvhat, *gThat, *ggrad;
    double* ggrad_l;                // liquid (cell-kernel) part of ggrad, for the line search
    uint8_t* pcode;
    // ---- solver vectors (R) ----
    void *cx, *cr, *cp, *cu, *invm;
    void* pinv;                     // momentum CG preconditioner: 1 / diag(P H P) per component
    void* mR;                       // node mass in R (the CG's mass term)
    void *hx, *hr, *hp, *hu, *hinvd, *hT;   // heat CG (scalar fields)
    double* hrhs;
    // dense staging for the C ABI
    void* dense_a;
    void* dense_b;
    // ---- scalars ----
    SceneDev* sc;
    SceneScal* scal;
    int* err;
    unsigned* cg_bar;               // grid barrier of the cooperative CG kernel (2 words)
    unsigned long long* scene_cnt;  // per scene: generated surface samples
    long long* scene_first;         // per scene: first generated sample
};

}  // namespace mpm

struct mpm_ctx {
    int nsc = 0;
    int prec = 0;
    int rsize = 8;                  // sizeof(R)
    cudaStream_t st = nullptr;
    std::vector<mpm::SceneDev> hsc;
    long long Pcap = 0, Scap = 0, total_blocks = 0, total_cells = 0;
    long long np = 0, ns = 0;       // current totals
    long long block_cap = 0;        // capacity of active blocks (grid slots)
    long long opk_cap = 0;          // capacity of d.opk in records (grown by the per-step pack)
    bool has_solids = false;        // solid-only buffers allocated
    bool sK_valid = false;          // d.sKa holds the maps of the cached iterate
    bool pK_valid = false;          // d.pK holds the solids' maps of the cached iterate
    bool use_graphs = true;         // CG chunks as CUDA graphs (cleared if capture is refused)
    int graph_error = 0;            // the refusal's error code
    // CG launch configuration and its autotuner state
    int cg_ctas_per_sm = 0;         // 0: as many as fit
    int cg_chunk = 8;               // CG iterations per host check
    int tune_next = 0, tune_best = -1;
    int op_rows = 0;                // operator record rows per bulk copy (0: not tuned yet, 4 used)
    double tune_best_ms = 0.0;
    cudaEvent_t tune_ev[2] = {};
    // surface generation: triangle records (grown on demand), per-scene counts
    void* tri_buf = nullptr;
    size_t tri_bytes = 0;
    std::vector<unsigned long long> hscene_cnt;
    std::vector<long long> hscene_first;
    int NB = 0, NW = 0;
    int n_gen = 0, n_gen_g = 0;     // work blocks in the general kernel's lists (with / without samples)
    bool resampled = false, p2g_done = false, step_ready = false;
    mpm::Dev d{};
    mpm::SceneScal* hscal = nullptr;   // pinned mirror
    int* herr = nullptr;               // pinned
    int* hcounts = nullptr;            // pinned
    std::string last_error;
    std::vector<void*> allocs;
    // profiling
    long long launches = 0;
    bool prof = false;
    mpm_profile pr{};
    cudaEvent_t ev[2 * 16 + 2] = {};
    int nev = 0;                       // recorded apply event pairs pending
};

// counts every kernel launch of a context (`c` in scope); usable as a statement prefix
#define MPM_LAUNCH for (int once_ = (c->launches++, 1); once_; once_ = 0)

namespace mpm {

// ---- sort.cu ----
cudaError_t launch_sort_particles(mpm_ctx* c);
cudaError_t launch_sort_surface(mpm_ctx* c);
cudaError_t launch_build_blocks(mpm_ctx* c);   // needs parents (balance particles)
cudaError_t launch_exclusive_scan(mpm_ctx* c, const int* in, int* out, long long n, int* tmp, cudaStream_t st);

// ---- transfer.cu ----
cudaError_t launch_nearest_parent(mpm_ctx* c);
cudaError_t launch_p2g(mpm_ctx* c);
cudaError_t launch_g2p(mpm_ctx* c);

// ---- newton.cu ----
cudaError_t launch_pack_step(mpm_ctx* c);
cudaError_t launch_eval(mpm_ctx* c, bool fp64_math, bool want_cache);
cudaError_t launch_apply(mpm_ctx* c, const void* p, void* u, int mode);
cudaError_t run_newton(mpm_ctx* c);
cudaError_t launch_dense_to_grid(mpm_ctx* c, int scene, const void* dense, void* grid, int comps, int rsize);
cudaError_t launch_grid_to_dense(mpm_ctx* c, int scene, const void* grid, void* dense, int comps, int rsize_in, int rsize_out);
cudaError_t launch_project_vec(mpm_ctx* c, void* vec, int rsize);
cudaError_t launch_mass_term(mpm_ctx* c, const void* p, void* u);

// ---- surfgen.cu ----
// Replaces every scene's surface samples with ones generated on the particles'
// union-of-spheres surface, triangulated by `method` (mpm_isosurface);
// counts[s] receives scene s's count. A count above a scene's max_surface sets
// *capacity_error and leaves the samples unchanged.
cudaError_t launch_generate_surface(mpm_ctx* c, unsigned long long seed, double per_cell_area, int method,
                                    long long* counts, int* capacity_error);

// ---- heat.cu ----
cudaError_t run_heat(mpm_ctx* c);
cudaError_t launch_heat_apply(mpm_ctx* c, const void* T, void* out);

// ---- profiling helpers (api.cu) ----
void prof_mark_apply(mpm_ctx* c, bool begin);
void prof_collect_applies(mpm_ctx* c, bool heat);

}  // namespace mpm
