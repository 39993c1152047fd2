/*
 * capfilm -- C ABI of the GB300 coupled lattice Boltzmann / FEM capsule step.
 *
 * The method is the one of Wouters, Aouane, Sega & Harting, "Capillary
 * interactions between soft capsules protruding through thin fluid films":
 * a two-component Shan-Chen D3Q19 lattice Boltzmann fluid (Sec. 3.1, Eqs. 4,
 * 5, 10) on a substrate, coupled by half-way bounce-back with Ladd's
 * moving-wall term to triangulated elastic capsules (Sec. 3.1, Eqs. 6-9, 11).
 *
 * Conventions
 *  - Lattice units: dx = dt = rho_0 = 1.  Nodes (x, y, z), 0 <= x < nx, ...,
 *    node index n = (z*ny + y)*nx + x.  Periodic in x, y and z; with `wall` set
 *    the plane z = 0 is solid (the substrate, wall at z = 1/2).
 *  - Populations are ordered [component][direction][z][y][x]; component 0 is
 *    the film fluid A, component 1 the covering fluid B.  Direction order:
 *    0 rest; 1..6 = +x,-x,+y,-y,+z,-z; 7..18 = (1,1,0),(-1,-1,0),(1,-1,0),
 *    (-1,1,0),(1,0,1),(-1,0,-1),(1,0,-1),(-1,0,1),(0,1,1),(0,-1,-1),(0,1,-1),
 *    (0,-1,1): opposite directions are adjacent pairs (1,2), (3,4), ...
 *  - Every call returns a cf_status; nothing throws across the ABI.  On error
 *    cf_last_error() returns a thread-local description.
 *  - Host arrays passed in are copied; the caller keeps ownership.  Output
 *    arrays are caller-allocated host buffers of the stated size.
 *  - Device memory is owned by the context.  It is taken from the caller's
 *    allocator when one is given (e.g. PyTorch's caching allocator), otherwise
 *    from cudaMallocAsync on the context's stream.
 *  - All work is queued on the context's stream (desc.stream, or a stream the
 *    context creates).  Readout calls synchronise that stream.
 */
#ifndef CAPFILM_H
#define CAPFILM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    CF_OK = 0,
    CF_EINVAL = 1,     /* bad argument or size                               */
    CF_ENOMEM = 2,     /* device allocation failed                           */
    CF_ECUDA = 3,      /* a CUDA call failed (text in cf_last_error)          */
    CF_ESTATE = 4,     /* call not valid in the current state                */
    CF_ENOTFOUND = 5,  /* unknown capsule id                                 */
    CF_EDIVERGED = 6,  /* non-finite density detected                        */
    CF_EOVERFLOW = 7   /* the cut-link list exceeded its capacity, or an element
                          spans more than 16 lattice units */
} cf_status;

/* Storage of the populations (arithmetic is float32 in every case):
 * CF_FP32       float32 populations;
 * CF_FP16_SHIFT the 18 moving populations as IEEE half offsets
 *               g_i = f_i - w_i rho from the rest equilibrium of the node that
 *               wrote them (rho kept in float32), stored times 2^15 so that
 *               small offsets stay out of half's subnormal range;
 * CF_BF16_SHIFT the same offsets in bfloat16 (unscaled).
 * In both 16-bit modes the offsets are rounded stochastically (a hash of node,
 * step and direction; deterministic from run to run) and the rest population
 * is kept in float32 and takes each node's mass balance, so the stored mass is
 * the collided mass up to float32 rounding.  Population bytes per node drop
 * from 152 to 80. */
typedef enum { CF_FP32 = 0, CF_FP16_SHIFT = 1, CF_BF16_SHIFT = 2 } cf_precision;

/* Capsule modes: FREE moves and deforms (Eq. 9); FROZEN keeps its shape and
 * translates rigidly with the summed force (the frozen-shape protocol of
 * Sec. 4.3); FIXED does not move (the rigid particles of Sec. 4.1). */
typedef enum { CF_FREE = 0, CF_FROZEN = 1, CF_FIXED = 2 } cf_mode;

typedef struct {
    /* returns a device pointer of at least `bytes` bytes usable on `stream`,
     * or NULL on failure */
    void *(*alloc)(size_t bytes, void *stream, void *user);
    void (*free)(void *ptr, void *stream, void *user);
    void *user;
} cf_allocator;

/* Alternative readings of points where the paper is silent (flags of
 * cf_lattice_desc; 0 selects the default readings):
 * CF_INERTIAL        node update v += F_tot/m, x += v instead of the literal
 *                    x += F_tot/m of Eq. 9 with dt = 1 (free and frozen
 *                    capsules; the node velocity enters Ladd's term)
 * CF_LADD_REF_RHO    Ladd's moving-wall term (Sec. 3.1) with the reference
 *                    density rho_0 = 1 instead of the fluid node's density
 * CF_PARTNER_MIRROR  partner density across a cut or substrate link (Sec.
 *                    3.1, last paragraph) = the node's own density instead
 *                    of the mean over the node and its same-side neighbours
 * CF_DRY_REMOVE      drying (cf_remove_mass) removes the A mass instead of
 *                    turning it into B
 * CF_IBM             diffuse-interface (immersed-boundary) coupling instead
 *                    of the paper's cut-link coupling (Sec. 3.1); not part
 *                    of the paper, a variant for comparison: each step the membrane forces (Eqs. 6-8, 11) of every
 *                    node are spread to the 4x4x4 lattice nodes around it
 *                    with Peskin's 4-point kernel, act in the collision as a
 *                    body force shared by the components in proportion to
 *                    their densities, and the nodes then move with the fluid
 *                    velocity (with the half-force shift) interpolated with
 *                    the same kernel.  No lattice link is cut: no bounce-back,
 *                    momentum exchange, Shan-Chen decoupling or wetting offset
 *                    at the membrane, so cf_capsule_force and the lateral
 *                    force read zero; the cut links of the moved membrane
 *                    still give the interior flags of the meniscus readouts.
 *                    Free and fixed capsules only (CF_EINVAL for frozen ones,
 *                    for CF_INERTIAL, and for a batch).  Costs 44 more bytes
 *                    per lattice node. */
enum { CF_INERTIAL = 1, CF_LADD_REF_RHO = 2, CF_PARTNER_MIRROR = 4, CF_DRY_REMOVE = 8, CF_IBM = 16 };

typedef struct {
    int nx, ny, nz;          /* lattice size, each >= 3                        */
    int wall;                /* 1: substrate plane z = 0; 0: fully periodic    */
    double tau[2];           /* BGK relaxation times of A and B (Eq. 4), > 1/2 */
    double G;                /* Shan-Chen coupling G^{AB} = G^{BA} (Eq. 10)    */
    double rep_dz;           /* repulsive plane at z = 1/2 + rep_dz (Sec. 3.2) */
    double xi, delta0;       /* Hertz strength and range (Eq. 11)              */
    int precision;           /* cf_precision                                   */
    const cf_allocator *allocator; /* may be NULL                              */
    void *stream;            /* cudaStream_t or NULL                           */
    int flags;               /* CF_INERTIAL | ... (0: the default readings)    */
} cf_lattice_desc;

typedef struct {
    int nv, nf;              /* nodes and triangular elements                 */
    const double *nodes;     /* host [nv*3], reference (stress-free) shape   */
    const int *faces;        /* host [nf*3], counter-clockwise seen from out */
    double kS;               /* Skalak shear modulus kappa_S (Eq. 6)          */
    double C;                /* Skalak area constant, kappa_A/kappa_S = 1+2C  */
    double kB;               /* Helfrich bending modulus kappa_B (Eq. 7), H0=0 */
    double kV;               /* volume penalty kappa_V (Eq. 8)                */
    double mass;             /* mass per node m_i (Sec. 3.2: 25)              */
    int mode;                /* cf_mode                                       */
    double wet;              /* wetting offset (Sec. 3.1, last paragraph): on
                                every link this membrane cuts, the partner
                                densities interpolated for the Shan-Chen force
                                are rho_A + wet and rho_B - wet (the reaction
                                on the element uses the same); 0 = neutral
                                wetting, the paper's choice; > 0 draws the
                                film fluid A onto the surface.  Finite. */
} cf_capsule_desc;

typedef struct cf_ctx cf_ctx;

/* Thread-local text of the last error of this thread ("" if none). */
const char *cf_last_error(void);

/* Lattice and film set-up (Sec. 3.2).  Allocates the populations and the
 * coupling structures; populations start at zero until cf_set_film.  With
 * tau = 1 for both components the collision stores the equilibria computed
 * from the moments of the density pass (no second pull of the populations);
 * any other tau relaxes the pulled populations.
 * Errors (checked before any CUDA call): CF_EINVAL for a null argument, a
 * dimension below 3, a lattice of 2^26 nodes or more (a cut-list entry holds
 * the node index in 26 bits: at most 67.1 million nodes), tau <= 1/2 or not a
 * number, an unknown precision or flag; then CF_ECUDA (stream or event creation) and
 * CF_ENOMEM (an allocation failed: all blocks obtained are given back). */
cf_status cf_create(const cf_lattice_desc *desc, cf_ctx **out);
/* Frees the context and everything it allocated; a null context is a no-op
 * (CF_OK). */
cf_status cf_destroy(cf_ctx *ctx);

/* Capsule insertion with its elastic moduli (Sec. 3.1, Eqs. 6-8).  The given
 * mesh is the stress-free reference state; *id receives the capsule index
 * (0, 1, ... in insertion order).  Capsules must be added before cf_set_film,
 * which fills their interior with the B-majority fluid. */
cf_status cf_add_capsule(cf_ctx *ctx, const cf_capsule_desc *desc, int *id);
/* The same for n capsules desc[0..n) at once (ids[k] receives the index of
 * desc[k]; ids may be null): the device structures of the membrane are
 * rebuilt once instead of after each capsule, for lattices with many
 * capsules.  Errors as cf_add_capsule, checked for every descriptor before
 * any is added (none is added then). */
cf_status cf_add_capsules(cf_ctx *ctx, const cf_capsule_desc *desc, int n, int *ids);
cf_status cf_set_capsule_mode(cf_ctx *ctx, int id, int mode);

/* Film initialisation (Sec. 3.2): A-majority (rho_maj / rho_min) below the
 * film top h_top, B-majority above, the plane floor(h_top + 1/2) mixed at
 * rho_mix for both, capsule interiors B-majority, all at rest (f_i = w_i rho).
 * jitter: NULL or host [2][nz][ny][nx] added to the densities of A and B. */
cf_status cf_set_film(cf_ctx *ctx, double h_top, double rho_maj, double rho_min,
                      double rho_mix, const double *jitter);

/* Advance n coupled time steps (Sec. 3.1): streaming with bounce-back and
 * Ladd momentum exchange, Shan-Chen forces with interior/exterior
 * decoupling, BGK collision, element forces averaged over two steps, Skalak,
 * Helfrich, volume and Hertz forces, node update, new cut links.  Asynchronous
 * on the context stream; returns CF_EOVERFLOW / CF_EDIVERGED detected by the
 * previous readout or sync. */
cf_status cf_step(cf_ctx *ctx, long long n);

/* Wait for queued work; reports device-side error flags. */
cf_status cf_sync(cf_ctx *ctx);

/* Readouts (Sec. 4.1, 4.3).  Sum over the capsule's nodes of the fluid
 * coupling force of the last step (F) and its torque about the node centroid
 * (T); lateral capillary force between capsules a and b,
 * F = 1/2 (F_b - F_a) . e_ab with e_ab the unit xy vector from a to b
 * (negative = attraction, as in Eq. 3). */
cf_status cf_capsule_force(cf_ctx *ctx, int id, double F[3], double T[3]);
cf_status cf_lateral_force(cf_ctx *ctx, int a, int b, double *F);

/* Node positions (host [nv*3]), surface area and enclosed volume of the mesh
 * the last step's forces were computed on.  Any output may be NULL. */
cf_status cf_capsule_state(cf_ctx *ctx, int id, double *nodes, double *area, double *volume);

/* Densities [2][N] and barycentric velocity u = (j_A + j_B + F/2)/rho [3][N]
 * of the last step (N = nx*ny*nz; solid nodes read 0).  Either may be NULL.
 * *inout_n: the capacity of the buffers in nodes (in) and N (out); a
 * capacity below N returns CF_EINVAL with *inout_n = N and writes nothing. */
cf_status cf_fields(cf_ctx *ctx, double *rho, double *u, size_t *inout_n);

/* Post-collision populations [2][19][N] as float (16-bit storage decoded). */
cf_status cf_populations(cf_ctx *ctx, float *f);

/* Total mass of each component (FP64 sum over the lattice). */
cf_status cf_total_mass(cf_ctx *ctx, double m[2]);

/* Film height per column h[ny][nx]: the first zero of rho_A - rho_B above the
 * substrate, linearly interpolated; NaN where it touches a capsule interior. */
cf_status cf_meniscus_field(cf_ctx *ctx, double *h);

/* Meniscus profile around capsule id (Sec. 4.1, the slice through the
 * particle centre averaged over the four sides), computed on the device in
 * FP64 from the column heights of cf_meniscus_field:
 *  - h_inf, the far-field film height: the mean height of the valid columns
 *    whose (periodic) distance to the nearest capsule centroid is at least
 *    0.9 times the largest such distance;
 *  - from the column nearest to the capsule's xy centroid, the rays +x, -x,
 *    +y and -y are sampled at r_k = k dr, k = 0 .. floor((min(nx,ny)/2)/dr)-1,
 *    by linear interpolation between the two columns that bracket r_k (a
 *    sample touching a NaN column is skipped); zeta_k = mean of the valid
 *    samples - h_inf (NaN when none is valid);
 *  - Z receives the largest valid zeta (the capillary rise; may be NULL).
 * r and zeta have capacity *inout_n (in) and receive *inout_n entries (out);
 * too small returns CF_EINVAL with the needed size.  dr must be positive and
 * at most min(nx, ny)/2 (else CF_EINVAL). */
cf_status cf_meniscus_profile(cf_ctx *ctx, int id, double dr, double *r, double *zeta,
                              size_t *inout_n, double *Z);

/* Meniscus height Z of capsule id: the largest zeta of its profile with
 * dr = 1 (the capillary rise read out in Sec. 4). */
cf_status cf_meniscus_height(cf_ctx *ctx, int id, double *Z);

/* Fit of the meniscus model of Sec. 2 (Eq. 12: zeta(r) = Q K_0(q r), Q the
 * capillary charge, q the inverse capillary length), as done for the
 * equilibrated profile of Sec. 4.1: least squares over the samples (host
 * arrays r[n], zeta[n], e.g. from cf_meniscus_profile) with r > 0,
 * rmin <= r <= rmax and a finite zeta.  For a given q the best Q is linear;
 * q is scanned on 400 logarithmic steps over [1e-3, 3] and refined by
 * golden-section search.  out[0] = Q, out[1] = q, out[2] = rms residual,
 * out[3] = samples used.  K_0 from std::cyl_bessel_k.  Host only, no
 * context.  CF_EINVAL for null arrays or fewer than two samples. */
cf_status cf_meniscus_fit(const double *r, const double *zeta, size_t n, double rmin, double rmax,
                          double out[4]);

/* The lateral capillary force of the theory (Eq. 13) between particles of
 * capillary charges Q1, Q2 at centre distance L: *F = -2 pi q gamma Q1 Q2
 * K_1(q L), negative = attraction.  Host only.  CF_EINVAL unless q, L > 0. */
cf_status cf_capillary_force(double q, double gamma, double Q1, double Q2, double L, double *F);

/* Checkpoint and restart (no counterpart in the paper; the runs reach 2e4 to
 * 5e4 steps).  cf_save writes the state between two steps to `path`: the
 * populations (and 16-bit storage's float rest populations), the densities
 * they were encoded with, the last step's fields, the stochastic-rounding
 * step counter, and with capsules the node positions and velocities, both
 * exchange accumulators (the two-step average), element velocities,
 * per-capsule sums, bounding boxes and the cut-link structure; also the step
 * count and the drying rate.  A versioned binary file (native byte order).
 * cf_load restores it into a context created with the same lattice
 * description and the same capsules added in the same order; the run then
 * continues bit for bit as it would have without the restart (capsules whose
 * motion feeds back through atomic float sums excepted: those runs are not
 * bitwise reproducible even without a restart).  Synchronous.
 * Errors: CF_EINVAL (file cannot be opened, written or read, wrong version,
 * or a context that does not match: the context is then unchanged, except
 * for a truncated file, after which cf_set_film must come again),
 * CF_ESTATE (cf_save before cf_set_film), CF_ECUDA. */
cf_status cf_save(cf_ctx *ctx, const char *path);
cf_status cf_load(cf_ctx *ctx, const char *path);

/* Cut-link structure for the current membrane positions (diagnostics):
 * mask[N] bit (k-1) set when link n -> n + e_k crosses a membrane an odd number
 * of times; tri[N*18] the crossed element (global index) or -1; inside[N]
 * 1 for capsule-interior nodes.  Any output may be NULL. */
cf_status cf_cuts(cf_ctx *ctx, uint32_t *mask, int *tri, uint8_t *inside);

/* Advance n steps like cf_step, without graph replay, timing each phase with
 * CUDA events on the context stream; ms[0..3] receive the mean device time per
 * step of the two lattice passes, of the membrane phase, of the cut-link
 * rebuild and of the bounce-record preparation (milliseconds).  With CF_IBM,
 * ms[0] covers the lattice passes together with the membrane forces and their
 * spreading (which run beside the density pass), ms[1] the interpolation and
 * move of the nodes, and ms[2] = ms[3] = 0.  Synchronises.  For measurement; the
 * populations advance exactly as with cf_step. */
cf_status cf_time_phases(cf_ctx *ctx, long long n, double ms[4]);

/* One lattice time step without capsules that allocates no device memory.
 * The paper has no counterpart: this is for callers that cannot call
 * cudaMalloc (code running inside a framework that owns the device memory as
 * one fixed pool, or that must not allocate once set-up is over).  It applies
 * the same streaming, substrate bounce-back, Shan-Chen force and BGK collision
 * as cf_step does for a lattice without capsules.
 *   src, dst  device pointers, caller-owned, [2][19][nz][ny][nx] float
 *             populations (post-collision) in and out; overlapping ranges
 *             return CF_EINVAL; with a substrate (wall != 0) the plane z = 0
 *             of dst is not written
 *   nx..G     as in cf_lattice_desc; stream: cudaStream_t or NULL
 * The per-node density scratch is a fixed array inside the library, sized for
 * at most 1048576 nodes (16 MiB, held by every GPU that loads the library until
 * the process exits); larger lattices return CF_EINVAL.  Every call looks up
 * the array's device address in the calling thread's current context (the
 * array's host-side name is not a device address); make the first call on a
 * device before any stream capture.  All calls share the array, so
 * calls that overlap on the GPU (other streams, other threads) race; each
 * call overwrites the scratch completely before reading it.  Asynchronous on
 * `stream`. */
cf_status cf_lattice_step_static(const float *src, float *dst, int nx, int ny, int nz, int wall,
                                 const double tau[2], double G, void *stream);

/* Number of kernel launches issued by the last cf_step / cf_time_phases call. */
cf_status cf_launch_count(cf_ctx *ctx, long long *n);

/* Initial state from given densities: rhoA, rhoB host arrays [nz][ny][nx]
 * (copied), populations at rest f_i = w_i rho (Eq. 5 with u = 0); the substrate
 * plane stays empty.  An alternative to cf_set_film for states such as a
 * predicted equilibrium (the learned warm start below); capsules must be added
 * before.  Synchronous. */
cf_status cf_set_densities(cf_ctx *ctx, const double *rhoA, const double *rhoB);

/* Drying: lower the film by turning a mass dmA of component A into component
 * B every step (0 turns it off; the paper keeps each film height fixed, so
 * this rule is a reading of "lowering the film", not a passage of it).  After
 * each collision, every node where A is the majority (rho^A > rho^B, that
 * step's densities) keeps 1 - eps of its A populations and adds eps rho^A w_i
 * to its B populations, eps = dmA / (sum of rho^A over those nodes), at most
 * 1.  The A inventory thus falls by dmA per step and every node keeps its
 * total mass.  The sum is reduced on the device in a fixed order (runs are
 * reproducible).  Not available in a batch (cf_batch_step returns CF_ESTATE).
 * Synchronous.  Errors: CF_EINVAL (dmA negative or not finite), CF_ENOMEM. */
cf_status cf_remove_mass(cf_ctx *ctx, double dmA);

/* ---------------------------------------------------------------- batches
 * A batch steps many independent contexts together, for parameter sweeps such
 * as the paper's series over capsule distance and elastic modulus (Sec. 4):
 * the lattice passes of all of them run as one persistent launch per pass over
 * a work list of (lattice, tile) items, their membrane and cut-link phases as
 * parallel branches, and pairs of steps are replayed from a captured CUDA
 * graph.  Each context advances exactly as cf_step would advance it alone
 * (same arithmetic per node); it stays usable for all readouts, and may also
 * be stepped alone between batch steps.  The batch keeps pointers to the
 * contexts: destroy the batch before any of its contexts. */
typedef struct cf_batch cf_batch;

/* n (1..128) distinct contexts, all after cf_set_film and with the same
 * precision.  Starts with tile shape 1 (32 x 4) and 4 planes per work item.
 * Errors: CF_EINVAL (bad or repeated context, mixed precision), CF_ESTATE. */
cf_status cf_batch_create(cf_ctx *const *ctxs, int n, cf_batch **batch);
cf_status cf_batch_destroy(cf_batch *batch);

/* n steps of every context; returns after they have completed (device errors
 * of any context are reported as by cf_step). */
cf_status cf_batch_step(cf_batch *batch, long long n);

/* As cf_batch_step, and the device time of the n steps in *ms (CUDA events on
 * the batch's own stream). */
cf_status cf_batch_time(cf_batch *batch, long long n, double *ms);

/* As cf_batch_step without graph replay, timing each phase of every step
 * with CUDA events on the batch's stream: ms[0] the two batched lattice
 * passes, ms[1] the phase before them (every context's membrane forces and
 * bounce records), ms[2] the phase after them (node updates and cut links),
 * as mean milliseconds per step.  For measurement; the contexts advance
 * exactly as with cf_batch_step.  Synchronous. */
cf_status cf_batch_time_phases(cf_batch *batch, long long n, double ms[3]);

/* Launch shape of the batched lattice passes: tile in 0..5 selects the block
 * (x width, y depth) = (32,2), (32,4), (32,8), (64,2), (64,4), (128,2);
 * zchunk >= 1 is the number of contiguous planes of a work item (a block
 * walks them; with tau = 1 through its shared-memory ring of
 * pseudopotentials).  Results do not depend on the shape. */
cf_status cf_batch_set_config(cf_batch *batch, int tile, int zchunk);
/* Pipeline groups (1..8): the contexts are split, in order, into this many
 * groups of about equal node count; each group's lattice passes are launches
 * of their own on a stream branch of their own, so the membrane and cut-link
 * phases of one group overlap the lattice passes of another.  Results do not
 * depend on it.  cf_batch_config reports the groups in use (at most the
 * number of contexts). */
cf_status cf_batch_set_groups(cf_batch *batch, int groups);
cf_status cf_batch_config(const cf_batch *batch, int *tile, int *tile_x, int *tile_y, int *zchunk,
                          int *groups);

/* Autotuner: for every tile shape and zchunk in {2, 4, 8} (one group) it
 * replays the captured two-step graph once untimed and then ceil(steps/2)
 * times timed (steps >= 2), keeps the fastest shape, then times the groups
 * 2, 4 and 8 with that shape, and returns the chosen configuration with its
 * time per step (any output may be NULL).  The trials are real steps: every
 * context advances by 2 + 2 ceil(steps/2) steps per configuration tried;
 * the fields readout (cf_fields) is refreshed only by the next
 * cf_batch_step. */
cf_status cf_batch_autotune(cf_batch *batch, int steps, int *tile, int *zchunk, int *groups,
                            double *ms_per_step);

/* Number of kernel launches issued by the last cf_batch_step / cf_batch_time. */
cf_status cf_batch_launch_count(const cf_batch *batch, long long *n);

/* Lateral force (as cf_lateral_force) between capsules a and b of every
 * context of the batch: F[i] for context i (n values, the batch's order). */
cf_status cf_batch_lateral_forces(cf_batch *batch, int a, int b, double *F);

/* ------------------------------------------------------- learned warm start
 * Kernels of a small 3-D convolutional network that predicts an equilibrated
 * density field from the set-up (the paper has no counterpart; its long
 * equilibration runs, Sec. 4, are what the prediction shortens).  All pointers
 * are device pointers owned by the caller; calls are asynchronous on `stream`
 * (cudaStream_t or NULL); bad arguments return CF_EINVAL.
 *   activations  [n][c][nz][ny][nx] bfloat16 (x, y) or float (gradients)
 *   weights      [cout][cin][27] bfloat16, tap = (dz+1)*9 + (dy+1)*3 + (dx+1)
 *   bias         [cout] float
 * A layer is a 3x3x3 convolution with zero padding and dilation dil,
 * 1 <= cin, cout <= 16, followed by a ReLU when relu != 0; products are
 * accumulated in float. */
cf_status cf_conv3d_forward(const void *x, int n, int cin, int nz, int ny, int nx, const void *w,
                            const float *b, int cout, int dil, int relu, void *y, void *stream);

/* Backward of the same layer: gy = dL/dy (float, with respect to the layer's
 * output after its ReLU), y = the forward output (for the ReLU mask; may be NULL
 * when relu == 0).  Writes gx = dL/dx (float; skipped when gx is NULL) and ADDS
 * dL/dw to gw [cout][cin][27] and dL/db to gb [cout] (float, caller zeroes). */
cf_status cf_conv3d_backward(const void *x, int n, int cin, int nz, int ny, int nx, const void *w,
                             int cout, int dil, const void *y, int relu, const float *gy, float *gx,
                             float *gw, float *gb, void *stream);

/* Masked mean squared error of m bfloat16 predictions against float targets:
 * ADDS sum_i mask_i (p_i - t_i)^2 / msum to *loss (device double) and writes
 * grad_i = 2 mask_i (p_i - t_i) / msum (float).  mask may be NULL (all ones). */
cf_status cf_mse(const void *pred, const float *target, const float *mask, long long m, double msum,
                 float *grad, double *loss, void *stream);

/* Adam step t (>= 1) on float master weights w with moments m1, m2 (float, n
 * each), bias-corrected; writes the bfloat16 copy w_bf16 when not NULL. */
cf_status cf_adam(float *w, void *w_bf16, const float *g, float *m1, float *m2, long long n, double lr,
                  double b1, double b2, double eps, int t, void *stream);

/* Conversions float <-> bfloat16 (round to nearest even), n elements. */
cf_status cf_to_bf16(const float *x, void *y, long long n, void *stream);
cf_status cf_from_bf16(const void *x, float *y, long long n, void *stream);

/* ------------------------------------------------ U-net layers (tensor cores)
 * Layers of the warm start's 3-D U-net (the paper has no counterpart; see the
 * warm start above).  Activations are channels-last bfloat16
 * [n][nz][ny][nx][c]; weights bfloat16 [27][cout][cin] (tap = (dz+1)*9 +
 * (dy+1)*3 + (dx+1)); biases and gradients float32.  Every pointer is a
 * device pointer owned by the caller; calls are asynchronous on `stream`;
 * bad shapes return CF_EINVAL (text in cf_last_error).
 *
 * cf_unet_conv: 3x3x3 convolution, zero padding, y = act(b + conv(w, x)),
 * act = ReLU when relu != 0; contracted on the tensor cores (mma.sync
 * m16n8k16, bf16 products, fp32 accumulation).  cin a multiple of 16, cout
 * of 8; b may be NULL; y is float32 when out_f32 != 0, else bfloat16. */
cf_status cf_unet_conv(const void *x, int n, int nz, int ny, int nx, int cin, const void *w, const float *b,
                       int cout, int relu, int out_f32, void *y, void *stream);
/* The same convolution on the 5th-generation tensor cores (tcgen05.mma, M =
 * 128 voxels, N = cout, bf16 operands staged in shared memory, fp32
 * accumulators in tensor memory).  cin a multiple of 16 up to 256, cout a
 * multiple of 16 up to 256 (CF_EINVAL otherwise).  Its waits are bounded:
 * cf_unet_tc_error reports whether one ran out. */
cf_status cf_unet_conv_tc(const void *x, int n, int nz, int ny, int nx, int cin, const void *w, const float *b,
                          int cout, int relu, int out_f32, void *y, void *stream);
/* *err = 1 when a tensor-core convolution launched since the last call gave
 * up a wait (its output is then incomplete), else 0; synchronises the device
 * and clears the flag. */
cf_status cf_unet_tc_error(unsigned *err);
/* wt[26 - t][ci][co] = w[t][co][ci]: with wt as weights, cf_unet_conv of an
 * output gradient (cout channels) gives the input gradient (cin channels). */
cf_status cf_unet_flip(const void *w, int cin, int cout, void *wt, void *stream);
/* Weight and bias gradients for the output gradient gy (bfloat16, cout
 * channels, already masked by the ReLU) and the layer input x: ADDS
 * sum_v gy[v][co] x[v + off(t)][ci] to gw [27][cout][cin] and sum_v gy[v][co]
 * to gb [cout] (gb may be NULL).  The voxels are split into `chunks` ranges;
 * part (at least chunks * 27 * cout * cin floats) receives each range's sums,
 * which are then added in a fixed order: the result is bitwise reproducible.
 * cin a multiple of 16, cout of 8. */
cf_status cf_unet_wgrad(const void *x, const void *gy, int n, int nz, int ny, int nx, int cin, int cout,
                        int chunks, float *part, float *gw, float *gb, void *stream);
/* out[i] = bf16((g[i] + g2[i]) * (y[i] > 0)) (ReLU mask of the layer's
 * output y, bfloat16; no mask when y is NULL; g2 NULL counts as zero), m
 * elements: the gradient of an activation that feeds two layers is the sum. */
cf_status cf_unet_relu_grad(const float *g, const float *g2, const void *y, long long m, void *out,
                            void *stream);
/* Training loss of the U-net's head out (float [n][nz][ny][nx][ch], ch >= 5:
 * channels 0, 1 the density corrections of A and B, channels 2..4 a
 * displacement field) and its gradient g (same shape; channels beyond 4
 * zero).  ADDS to *loss (device double):
 *   wd * sum_{s,c,v} mask[s][v] (out[s][v][c] - t[s][c][v])^2   (t [n][2][V],
 *   mask [n][V]; pass wd = weight / mask sum), plus, when nodes > 0 and
 *   wx > 0, wx / (n nodes) * sum_{s,i} |D_s(X[s][i]) - d[s][i]|^2, D_s the
 *   displacement channels interpolated trilinearly at the node's reference
 *   position X[s][i] (lattice units, float [n][nodes][3], clamped into the
 *   grid) and d the target displacement (float [n][nodes][3]).
 * part: device scratch of at least 304 + n doubles.  Sums are taken in a
 * fixed order (the node gradient by one thread per sample walking its nodes),
 * so the result is bitwise reproducible. */
cf_status cf_unet_loss(const float *out, int n, int nz, int ny, int nx, int ch, const float *t,
                       const float *mask, double wd, const float *X, const float *d, int nodes, double wx,
                       double *part, float *g, double *loss, void *stream);
/* 2x2x2 average pooling of x (bfloat16, fine grid nz x ny x nx, each even)
 * into y, and its gradient (float: gx from the coarse gradient gy). */
cf_status cf_unet_pool(const void *x, int n, int nz, int ny, int nx, int c, void *y, void *stream);
cf_status cf_unet_pool_bwd(const float *gy, int n, int nz, int ny, int nx, int c, float *gx, void *stream);
/* Nearest-neighbour upsampling by 2 of x (bfloat16, coarse grid) to the fine
 * grid nz x ny x nx (each even), and its gradient (float). */
cf_status cf_unet_upsample(const void *x, int n, int nz, int ny, int nx, int c, void *y, void *stream);
cf_status cf_unet_upsample_bwd(const float *gy, int n, int nz, int ny, int nx, int c, float *gx,
                               void *stream);
/* Channel concatenation y[v] = (a[v][0..ca), b[v][0..cb)) of nv voxels
 * (bfloat16), and the split of a float gradient (a or b may be NULL). */
cf_status cf_unet_concat(long long nv, const void *a, int ca, const void *b, int cb, void *y, void *stream);
cf_status cf_unet_split(long long nv, const float *y, int ca, int cb, float *a, float *b, void *stream);
/* Layout changes for one sample: pack channel-first float [c][N] into
 * channels-last bfloat16 [N][cpad] (zero channels beyond c); unpack channels
 * [c0, c0 + c) of channels-last [N][cpad] (bfloat16, or float when x_f32)
 * into channel-first float [c][N]. */
cf_status cf_unet_pack(const float *x, int c, long long N, int cpad, void *y, void *stream);
cf_status cf_unet_unpack(const void *x, int x_f32, int cpad, long long N, int c0, int c, float *y,
                         void *stream);

/* ------------------------------------------------ warm start in the library
 * The trained U-net (the paper has no counterpart: its long equilibration
 * runs, Sec. 4, are what the prediction shortens) loaded onto the device,
 * and the whole warm start of a context: inputs (cf_warm_features), the
 * U-net's density head, the predicted state (cf_warm_apply), then two
 * judging windows of the coupled run with a fallback to the flat film.
 *
 * cf_model_load: weights file "CFUNET01", int32 widths w0 w1 w2, then for
 * the layers e0a e0b e1a e1b ma mb d1a d1b d0a d0b head: int32 cin, cout,
 * float32 weights [27][cout][cin], float32 biases [cout] (native byte
 * order; the shapes must be those of the U-net with these widths).  Weights
 * are stored on the current device in bfloat16.  CF_EINVAL for a missing or
 * malformed file, CF_ENOMEM. */
typedef struct cf_model cf_model;
cf_status cf_model_load(const char *path, cf_model **out);
cf_status cf_model_destroy(cf_model *model);

typedef struct {
    int window;      /* steps of each judging window (>= 1), e.g. 25          */
    double u_limit;  /* largest velocity component allowed, e.g. 0.1          */
    double grow;     /* the mean density change of the second window may be
                        at most grow times the first's, e.g. 1.5              */
    int fallback;    /* 1: restore the flat film when the judgement fails     */
} cf_warm_policy;

/* Warm start of a context (after its capsules are added; lattice sizes
 * divisible by 4): sets the U-net's predicted densities (film h_top,
 * densities rho_maj / rho_min / rho_mix, modulus kS for the input feature),
 * runs 1 + 2 * window steps and judges them: the start is kept when all
 * densities and velocities are finite, no density is negative, no velocity
 * component exceeds u_limit and the density change of the second window is
 * at most grow times the first's; otherwise, with fallback set, the flat
 * film (cf_set_film with `jitter`, which may be NULL) is restored.  *used
 * receives 1 when the prediction was kept, *steps the judging steps taken
 * (either may be NULL).  Synchronous. */
cf_status cf_warmstart(cf_ctx *ctx, const cf_model *model, const cf_warm_policy *policy, double h_top,
                       double rho_maj, double rho_min, double rho_mix, double kS, const double *jitter,
                       int *used, long long *steps);

/* Set-up of the warm start on a context (after its capsules are added; all
 * arrays are device arrays of the caller, [c][nz][ny][nx] float32; the film
 * is the one cf_set_film(h_top, rho_maj, rho_min, rho_mix) would make, and
 * its mixed plane is floor(h_top + 1/2)).  Synchronous; CF_EINVAL for null
 * arrays or bad parameters.
 *
 * cf_warm_features: the network inputs x [4][N] (capsule interior flag; the
 * flat film's phi = +1 below the mixed plane, 0 in it and on the substrate,
 * -1 above and inside capsules; z / nz; log10(kS) + 2) and, if mask is not
 * NULL, the fluid mask [N] (1 outside the capsules and off the substrate). */
cf_status cf_warm_features(cf_ctx *ctx, double h_top, double kS, float *x, float *mask);

/* cf_warm_apply: the state predicted by the network from its corrections d
 * [2][N] (in units of rho_maj - rho_min): the film's densities plus the
 * corrections on the fluid outside the capsules (at least 1e-3), the film's
 * inside them and on the substrate; each component is then scaled on that
 * fluid to the flat film's mass (the run conserves mass, so a start with
 * other masses would relax to another equilibrium).  Populations at rest
 * (Eq. 5 with u = 0), as cf_set_densities.  The sums are reduced on the
 * device in a fixed order. */
cf_status cf_warm_apply(cf_ctx *ctx, double h_top, double rho_maj, double rho_min, double rho_mix,
                        const float *d);

/* cf_warm_target: the training target of the current state (the fields of
 * the last step), t [2][N] = (rho_c - rho_c,film) / (rho_maj - rho_min) on the
 * fluid outside the capsules, 0 elsewhere.  CF_ESTATE before the state is
 * set (cf_set_film, cf_set_densities, cf_warm_apply or cf_load); step first,
 * as the fields are recorded by the steps. */
cf_status cf_warm_target(cf_ctx *ctx, double h_top, double rho_maj, double rho_min, double rho_mix,
                         float *t);

/* cf_field_check: residual statistics of the fields of the last step, for
 * judging a warm start: out[0] = 1 if every density and velocity is finite
 * (else 0), out[1] = smallest density, out[2] = largest |u| component,
 * out[3] = mean |rho - rho_prev| over both components and all nodes, rho_prev
 * being the densities of the previous cf_field_check call on this context
 * (zero for the first).  CF_ESTATE before the state is set; step first, as
 * the fields are recorded by the steps. */
cf_status cf_field_check(cf_ctx *ctx, double out[4]);

#ifdef __cplusplus
}
#endif
#endif
