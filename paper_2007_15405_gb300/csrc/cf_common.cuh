// Shared device definitions of the capfilm CUDA library (sm_103a).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/capfilm.h"

namespace cf {

// Programmatic dependent launch.  The kernels of the step's critical path are
// launched with the programmatic-serialization attribute: the next kernel on
// the stream may be scheduled while its predecessor's last blocks run.  Each
// such kernel first lets its own successor be scheduled (pdl_trigger) and
// then waits until its predecessor has completed with all writes visible
// (pdl_wait), before it touches any memory.  For a normal launch both are
// no-ops.
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Launch a kernel whose first statements are pdl_trigger(); pdl_wait();
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, cudaStream_t s, Args... args) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
}

// D3Q19 (Sec. 3.1): rest, six face neighbours (w = 1/18), twelve edge
// neighbours (w = 1/36); opposite directions are adjacent pairs.
__host__ __device__ constexpr int ex(int i) {
    return i == 1 ? 1 : i == 2 ? -1 : i == 7 ? 1 : i == 8 ? -1 : i == 9 ? 1 : i == 10 ? -1
         : i == 11 ? 1 : i == 12 ? -1 : i == 13 ? 1 : i == 14 ? -1 : 0;
}
__host__ __device__ constexpr int ey(int i) {
    return i == 3 ? 1 : i == 4 ? -1 : i == 7 ? 1 : i == 8 ? -1 : i == 9 ? -1 : i == 10 ? 1
         : i == 15 ? 1 : i == 16 ? -1 : i == 17 ? 1 : i == 18 ? -1 : 0;
}
__host__ __device__ constexpr int ez(int i) {
    return i == 5 ? 1 : i == 6 ? -1 : i == 11 ? 1 : i == 12 ? -1 : i == 13 ? -1 : i == 14 ? 1
         : i == 15 ? 1 : i == 16 ? -1 : i == 17 ? -1 : i == 18 ? 1 : 0;
}
__host__ __device__ constexpr int opp(int i) { return i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1); }
__host__ __device__ constexpr float wgt(int i) {
    return i == 0 ? 1.0f / 3.0f : (i <= 6 ? 1.0f / 18.0f : 1.0f / 36.0f);
}
constexpr int Q = 19;

// Directions 0..18 packed 6 bits each ((ex+1) | (ey+1) << 2 | (ez+1) << 4),
// for code that selects a direction at run time (ek below).
constexpr unsigned long long pack_dirs(int lo) {
    unsigned long long v = 0;
    for (int j = 0; j < 10 && lo + j < Q; ++j) {
        const int k = lo + j;
        v |= (unsigned long long)((ex(k) + 1) | ((ey(k) + 1) << 2) | ((ez(k) + 1) << 4)) << (6 * j);
    }
    return v;
}
constexpr unsigned long long DIRS_LO = pack_dirs(0), DIRS_HI = pack_dirs(10);
__host__ __device__ __forceinline__ void ek(int k, int &x, int &y, int &z) {
    const unsigned c = (unsigned)((k < 10 ? DIRS_LO : DIRS_HI) >> (6 * (k < 10 ? k : k - 10))) & 63u;
    x = (int)(c & 3u) - 1;
    y = (int)((c >> 2) & 3u) - 1;
    z = (int)((c >> 4) & 3u) - 1;
}

// One entry of the cut-link list: link k (1..18) of node n, marked by element T.
// code = n << 5 | (k - 1); n < 2^26 for every lattice cf_create accepts.
__host__ __device__ __forceinline__ int cut_code(long long n, int k) { return (int)(n << 5) | (k - 1); }

// Storage of the populations: float, or half / bfloat16 offsets from the
// rest equilibrium w_i rho of the node (rho kept in float in the density array).
enum Prec { P_F32 = 0, P_F16 = 1, P_BF16 = 2 };
// Half offsets are stored times 2^15: quiescent offsets (~1e-7) then sit in
// half's normal range (above 2^-14) instead of its subnormals, and the largest
// representable offset is still 2 (populations never exceed the density).
constexpr float F16_SCALE = 32768.0f, F16_INV_SCALE = 1.0f / 32768.0f;
inline size_t pop_bytes(int prec) { return prec == P_F32 ? 4 : 2; }

// Momentum exchanged with each membrane element (Sec. 3.1, coupling): summed
// in 64-bit fixed point (units of 2^-40) by integer atomics, which are exact
// and do not depend on the order the contributions arrive in, so runs with
// moving capsules and their restarts repeat bit for bit.  A contribution is
// a float below ~10 in magnitude, so its rounding to 2^-40 lies far below
// its own float precision, and a sum stays far from the 2^63 range.
constexpr float FT_SCALE = 1099511627776.0f;  // 2^40
constexpr double FT_UNIT = 1.0 / 1099511627776.0;
__device__ __forceinline__ void ft_add(long long *a, float v) {
    atomicAdd(reinterpret_cast<unsigned long long *>(a), (unsigned long long)__float2ll_rn(v * FT_SCALE));
}
__device__ __forceinline__ float ft_val(long long v) { return (float)((double)v * FT_UNIT); }

// Parameters of the lattice passes.
struct LBParams {
    int nx, ny, nz, wall;
    long long N;            // nodes
    int zlo, zhi;           // fluid planes [zlo, zhi)
    int zchunk;             // density pass: planes walked per thread (grid.z = fluid planes /
                            // zchunk, strided); batched passes: contiguous planes of a work item
    int zring;              // tau = 1 collide pass: contiguous planes per block (its psi ring)
    int zstride;            // batched passes: z slices of this lattice
    float itau[2], tau[2];  // 1/tau and tau per component
    float G;
    int flags;              // CF_PARTNER_MIRROR, CF_DRY_REMOVE (alternative readings)
    const void *__restrict__ src;    // post-collision populations of the last step
    void *__restrict__ dst;          // post-collision populations of this step
    const float2 *__restrict__ rho_src;  // densities the src populations were encoded with
    const float *__restrict__ src0;  // 16-bit storage: rest populations in float [2][N]
    float *__restrict__ dst0;
    unsigned *__restrict__ step_ctr; // step counter (stochastic-rounding stream)
    const uint32_t *__restrict__ mask;  // cut bits per node
    const int *__restrict__ tri;        // crossed element per node and link [N*18]
    // diffuse-interface coupling (CF_IBM; null otherwise): the membrane force
    // spread to the lattice (ft_add), read and cleared by the collide pass,
    // which also writes the fluid velocity the nodes move with; both only in
    // the blocks of 32 nodes (n / 32) that the spreading flagged
    long long *__restrict__ fibm;       // [3][N]
    float4 *__restrict__ uphys;         // [N] (ux, uy, uz, 0), then the flags: ibm_flags(uphys, N)
    long long *__restrict__ FT;         // element momentum exchange accumulators [3*nfaces] (ft_add)
    const float2 *__restrict__ rec;     // [N][18] bounced (A, B) populations by arriving direction - 1
    const float *__restrict__ wet_el;   // [nfaces] wetting offset of each element's capsule (null: all 0)
    float *__restrict__ out;            // optional [5][N]: rhoA, rhoB, ux, uy, uz
    float2 *__restrict__ rho;           // [N] (rhoA, rhoB) of this step (written by the density pass)
    float2 *__restrict__ psi;           // [N] (psiA, psiB) of this step (written by the density pass)
    float4 *__restrict__ J;             // [N] total momentum of this step (density pass, tau = 1 only);
                                        // the allocation-free step keeps (rho_A, rho_B, psi_A, psi_B)
                                        // of its static scratch here
    unsigned *__restrict__ status;      // device error flags
    // drying (A turned into B): the density pass sums rho_A over the
    // A-majority nodes into block partials, its last block turns them into the
    // fraction the collide pass converts
    double dry_dm;                      // A mass converted per step (0: off)
    double *__restrict__ dry_part;      // [density-pass blocks] partial sums
    unsigned *__restrict__ dry_ctr;     // density-pass blocks finished
    float *__restrict__ dry_eps;        // fraction of this step
};

enum StatusBits : unsigned { ST_OVERFLOW = 1u, ST_NAN = 2u };

// Capsule description on the device.
struct CapDev {
    float kS, C, kB, kV, mass;
    int mode;               // 0 free, 1 frozen, 2 fixed
    int v0, nv, f0, nf;     // global offsets and counts
    int s0, ns;             // node slots [s0, s0 + ns) of the capsule's patches (ns: multiple of 32)
    double V0;              // reference volume
};

// Per-capsule FP64 accumulators (reset each step).
// A_CX..A_CZ hold the node sum relative to the capsule's first node, whose
// position is A_OX..A_OZ; A_VOL the enclosed volume; A_PRE the volume-penalty
// prefactor of Eq. 8 for this step.
enum CapAcc { A_FX = 0, A_FY, A_FZ, A_TX, A_TY, A_TZ, A_AREA, A_VOL, A_CX, A_CY, A_CZ,
              A_FTX, A_FTY, A_FTZ, A_OX, A_OY, A_OZ, A_PRE, A_NACC = 20 };

struct MemParams {
    int nx, ny, nz, wall;
    int ncaps, nfaces, nnodes;
    float zrep, xi, delta0;
    const CapDev *caps;
    const int *faces;        // [3*nf] global node ids
    const int *face_cap;     // [nf]
    const int *node_cap;     // [nv]
    const float *refM;       // [3*nf] inverse reference metric
    const float *refA;       // [nf]
    const float *refDet;     // [nf]
    const int *vf_off;       // [nv+1] vertex -> (face*3+slot) CSR
    const int *vf_ent;
    const float *Xh, *Xl;    // [3*nv] positions of this step as float pairs hi + lo
                             // (per-step displacements are below a float ulp at x ~ 100)
    float *Xnh, *Xnl;        // [3*nv] positions of the next step
    float *V;                // [3*nv] node velocities (written)
    const long long *FT;     // [3*nf] momentum exchanged with the fluid in this step (ft_add)
    const long long *FTprev; // [3*nf] the same, of the previous step
    float *fscr;             // [nf*FS_N] per-element scratch
    float *vscr;             // [nv*4] per-node scratch (gL, gA)
    float *Fcpl;             // [3*nv] coupling force on nodes (readout)
    double *acc;             // [ncaps*A_NACC]
    int *bbox;               // [ncaps*3] mins then [ncaps*3] maxs of this step (written)
    const int *bbox_prev;    // same, of the previous step (Hertz prefilter)
    unsigned *status;        // device error flags
    int any_frozen;
    int inertial;            // CF_INERTIAL: v += F/m, x += v
    // Contact prefilter: each capsule's nodes in patches of 32 neighbouring
    // nodes (Morton order of the shape the capsule was added with); slot s of
    // patch s / 32 holds node perm[s] (-1: padding at a capsule's last patch).
    // The node kernel runs one warp per patch and writes its box.
    const int *perm;         // [nslots]
    int nslots;
    float *pbox;             // [nslots / 32][6]: float min x, y, z, max x, y, z of this step
    // Contact partners of each capsule (lattices with many capsules): nbr[c *
    // CF_NBR_MAX + j], j < nbr_cnt[c], the capsules whose boxes of the previous
    // step come within the contact range, in ascending order; a count above
    // CF_NBR_MAX means "all capsules".  Null: every capsule is checked.
    const int *nbr;
    const int *nbr_cnt;
    // diffuse-interface coupling (CF_IBM; null otherwise): the node update
    // spreads each node's force into fibm [3][N] instead of moving it, and the
    // move kernel steps the nodes with uphys [N] interpolated at their positions
    long long *fibm;
    float4 *uphys;
    long long N;
};
// block flags of the diffuse-interface coupling: byte n / 32 is set when the
// spreading reached node n in this step; they follow the [N] velocities
__host__ __device__ inline uint8_t *ibm_flags(float4 *uphys, long long N) {
    return reinterpret_cast<uint8_t *>(uphys + N);
}
constexpr int CF_NBR_MAX = 48;
constexpr int CF_NBR_MIN_CAPS = 16;  // fewer capsules: no lists, the loop checks them all

// per-element scratch layout (floats)
enum FaceScr { FS_SK = 0, FS_DV = 9, FS_L = 18, FS_AF3 = 27, FS_BEND = 28, FS_N = 37 };

struct CutParams {
    int nx, ny, nz, wall;
    int nfaces;
    const int *faces;
    const float *X;          // positions (float, hi part) the cut links are computed for
    uint32_t *mask;
    int *tri;
    int2 *list;              // one entry per marked link: (cut_code(n, k), T)
    int *count;              // entries appended to `list` (zeroed before)
    long long *FTnext;       // [3*nfaces] exchange accumulator of the next step (zeroed here)
    const float *V;          // [3*nnodes] node velocities
    float4 *uT;              // [nfaces] element velocities (written here)
    int capacity;
    unsigned *status;
    int zero_only;           // fixed capsules: only zero FTnext (the cut links never move)
};

// Reset of the previous cut structure, run by extra blocks of the node-update
// kernel (which touches neither masks nor crossed elements).
struct ClearParams {
    const int2 *list;        // entries of the previous computation
    const int *count;
    int capacity;
    uint32_t *mask;
    int *tri;
    int blocks;              // blocks of the update kernel given to the reset (0: none)
    int *count_next;         // entry counter of the list about to be built: zeroed (may be null)
};

// Bounce records of the cut links for the next streaming (built once per step).
struct PrepParams {
    long long N;
    int prec;                // storage of the populations (cf_precision)
    const void *src;         // post-collision populations about to be streamed
    const float2 *rho;       // (rhoA, rhoB) of the step that produced them
    const uint32_t *mask;
    const int *tri;
    const float4 *uT;        // element velocities (mean of their nodes')
    const int2 *list;        // cut-link entries (cut_code(n, k), T), with repetitions
    const int *count;
    float2 *rec;             // [N][18] bounced (A, B) populations by arriving direction - 1
    long long *FT;           // element momentum exchange accumulators (ft_add)
    int capacity;
    int ref_rho;             // CF_LADD_REF_RHO: Ladd's term with rho_0 = 1
    int blocks;              // blocks striding over the list
};

// The membrane and cut-link kernels of many lattices in one launch: entry i
// holds lattice i's parameters, its blocks are [boff[i], boff[i+1]) of the
// grid.  Travels by value in the launch (64 entries of at most 352 B, the node
// update's, stay under the 32,764-byte launch-parameter limit); larger batches
// take one launch per 64 lattices.
constexpr int CF_SPARSE_CAP = 64;
template <class P>
struct SparseTab {
    int n;
    int boff[CF_SPARSE_CAP + 1];
    P p[CF_SPARSE_CAP];
};
struct UpdateParams {
    MemParams m;
    ClearParams c;
};
constexpr size_t CF_MAX_LAUNCH_PARAMS = 32764;  // bytes of kernel parameters a launch may carry
static_assert(sizeof(SparseTab<UpdateParams>) <= CF_MAX_LAUNCH_PARAMS, "node-update table too large");

__host__ __device__ inline int wrapi(int a, int n) {
    a %= n;
    return a < 0 ? a + n : a;
}

}  // namespace cf

// Host-side launchers (defined in the kernel translation units).
namespace cf {
void set_last_error(const char *msg);  // text returned by cf_last_error() on this thread
// most blocks a density pass of an nx x ny x nz lattice launches
size_t density_blocks_max(int nx, int ny, int nz);
// before_collide (optional): an event the collide pass waits for as well
cudaError_t launch_lb_step(const LBParams &p, int prec, cudaStream_t s, cudaEvent_t before_collide = nullptr);

// Batched lattice passes: many independent lattices in one persistent launch
// per pass.  The per-lattice parameters travel by value in the launch (one
// table per step parity of a captured step pair); the work list holds
// (lattice, x tile, y tile, z slice) items of the chosen tile shape.
// (128 x 248 B fits the 32,764-byte launch-parameter limit with the work-list
// pointer and count; a build with a table of at most 16 lattices keeps the
// launch parameters under 4 KB)
#ifndef CF_BATCH_MAX
#define CF_BATCH_MAX 128
#endif
struct BatchTab {
    LBParams lat[CF_BATCH_MAX];
};
static_assert(sizeof(BatchTab) + sizeof(void *) + sizeof(int) <= CF_MAX_LAUNCH_PARAMS,
              "lattice table too large for one launch");
constexpr int CF_NTILES = 6;  // tile shapes (x width, y depth) of the batched passes
void lb_batch_tile(int tile, int *tx, int *ty);
int lb_batch_resident(int tile, int prec, bool eq);  // blocks of one pass resident on the device
// nlat: lattices in tab
cudaError_t launch_lb_batch(const BatchTab &tab, int nlat, const int4 *work, int nwork, int prec, int tile,
                            cudaStream_t s);
cudaError_t launch_init_film(void *f, float *f0, int prec, float2 *rho, long long N, int nx, int ny,
                             int nz, int wall, float h_top, float rmaj, float rmin, float rmix,
                             const double *jit, const uint8_t *inside, cudaStream_t s);
cudaError_t launch_inside(const uint32_t *mask, uint8_t *inside, int nx, int ny, int nz,
                          cudaStream_t s);
cudaError_t launch_meniscus(const float *out, const uint8_t *inside, float *h, int nx, int ny,
                            int nz, int wall, cudaStream_t s);
// meniscus profile of capsule id from the column heights (one block, FP64):
// out[0..nr) = zeta at r_k = k dr, out[nr] = Z, out[nr+1] = h_inf
cudaError_t launch_meniscus_profile(const float *h, int nx, int ny, const double *acc, const CapDev *caps,
                                    int ncaps, int id, double dr, int nr, double *out, cudaStream_t s);
cudaError_t launch_init_dens(void *f, float *f0, int prec, float2 *rho, long long N, int nx, int ny,
                             int wall, const double *rAB, cudaStream_t s);
cudaError_t launch_mass(const void *f, const float *f0, int prec, const float2 *rho, long long N,
                        double *m2, cudaStream_t s);
// learned warm start: lattice, film plane and densities the set-up kernels use
struct WarmGeom {
    int nx, ny, nz, wall;
    long long N;
    int zm;                       // the film's mixed plane floor(h_top + 1/2)
    double rmaj, rmin, rmix, drho;  // film densities, drho = rmaj - rmin
};
int warm_parts();  // doubles x 4 of partial sums the set-up kernels need
cudaError_t launch_warm_features(const WarmGeom &g, const uint8_t *inside, float lks, float *x, float *mask,
                                 cudaStream_t s);
cudaError_t launch_warm_densities(const WarmGeom &g, const uint8_t *inside, const float *d, double *r,
                                  double *part, cudaStream_t s);
cudaError_t launch_warm_target(const WarmGeom &g, const uint8_t *inside, const float *out, float *t,
                               cudaStream_t s);
cudaError_t launch_field_check(long long N, const float *out, float *snap, double *part, double *res,
                               cudaStream_t s);
// the warm start's U-net on the device (unet_kernels.cu)
struct UNetModel;
cf_status unet_load(const char *path, UNetModel **out);
void unet_free(UNetModel *m);
cf_status unet_forward(const UNetModel *m, const float *feats, int nz, int ny, int nx, float *dens, float *disp,
                       cudaStream_t s);
// membrane kernels 1-3 (positions only) and 4-5 (after the lattice update)
cudaError_t launch_membrane_forces(const MemParams &p, cudaStream_t s, int *nlaunch);
cudaError_t launch_membrane_update(const MemParams &p, const ClearParams &cl, bool any_frozen,
                                   cudaStream_t s, int *nlaunch);
// contact partners of every capsule from the boxes of the previous step
// (writes nbr and nbr_cnt of p; one warp per capsule)
cudaError_t launch_contact_partners(const MemParams &p, int *nbr, int *nbr_cnt, cudaStream_t s, int *nlaunch);
cudaError_t launch_cuts(const CutParams &p, cudaStream_t s, int *nlaunch);
cudaError_t launch_prep(const PrepParams &p, cudaStream_t s, int *nlaunch);
// diffuse-interface coupling: nodes moved with the interpolated fluid velocity
cudaError_t launch_ibm_move(const MemParams &p, cudaStream_t s, int *nl);
// reset of a cut structure (as the node update's extra blocks do)
cudaError_t launch_cut_clear(const ClearParams &cl, cudaStream_t s, int *nl);
// batched forms (one launch per kernel for all lattices of the tables); tv:
// node-kernel blocks (32 nodes), tf: element-kernel blocks (64 elements), cut
// links: cut_blocks(nfaces, lanes) blocks with lanes = cut_lanes(the launch's
// elements), prep: PrepParams.blocks blocks of 256
constexpr int CF_MEM_NODE_BLOCK = 32, CF_MEM_FACE_BLOCK = 64;
int cut_lanes(long long nfaces);
int cut_blocks(int nfaces, int lanes);
cudaError_t launch_membrane_forces_batch(const SparseTab<MemParams> &tv, const SparseTab<MemParams> &tf,
                                         cudaStream_t s, int *nlaunch);
cudaError_t launch_membrane_update_batch(const SparseTab<UpdateParams> &tu, const SparseTab<MemParams> *tfrozen,
                                         cudaStream_t s, int *nlaunch);
cudaError_t launch_cuts_batch(const SparseTab<CutParams> &t, int lanes, cudaStream_t s, int *nlaunch);
cudaError_t launch_prep_batch(const SparseTab<PrepParams> &t, cudaStream_t s, int *nlaunch);
}  // namespace cf
