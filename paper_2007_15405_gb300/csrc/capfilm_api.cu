// Host runtime of the capfilm C ABI (include/capfilm.h).
//
// Owns the device state of one lattice with its capsules, queues the kernels
// of a coupled step on the context stream and replays pairs of steps from a
// captured CUDA graph (a pair returns every double buffer to its starting
// parity, so one graph serves any even number of steps).
#include "../../include/capfilm.h"
#include "cf_common.cuh"

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

using namespace cf;

namespace {

thread_local std::string g_err;

cf_status fail(cf_status s, const std::string &msg) {
    g_err = msg;
    return s;
}

#define CF_CUDA(call)                                                                      \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess)                                                             \
            return fail(CF_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_));     \
    } while (0)

struct HostCapsule {
    int nv, nf, mode;
    double kS, C, kB, kV, mass, wet;
    std::vector<float> X;      // reference positions (float)
    std::vector<int> F;        // local faces
};

}  // namespace

void cf::set_last_error(const char *msg) { g_err = msg; }

namespace {
// IEEE binary16 -> float (host side, for population readouts)
float half_to_float(uint16_t h) {
    const uint32_t sign = (uint32_t)(h >> 15) << 31;
    uint32_t exp = (h >> 10) & 0x1f, man = h & 0x3ff, u;
    if (exp == 0) {
        if (man == 0) u = sign;
        else {  // subnormal
            int e = -1;
            do { ++e; man <<= 1; } while (!(man & 0x400));
            u = sign | ((uint32_t)(127 - 15 - e) << 23) | ((man & 0x3ff) << 13);
        }
    } else if (exp == 31) u = sign | 0x7f800000u | (man << 13);
    else u = sign | ((exp + 127 - 15) << 23) | (man << 13);
    float f;
    std::memcpy(&f, &u, 4);
    return f;
}
}  // namespace

struct cf_ctx {
    cf_lattice_desc d{};
    long long N = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    // second stream for the membrane's position-only kernels, forked from and
    // joined back into `stream` every step
    cudaStream_t stream2 = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    cudaEvent_t ev_batch = nullptr;  // joins this context's work into a batch step
    cf_allocator alloc{};
    bool has_alloc = false;
    std::vector<void *> allocations;

    void *f[2] = {nullptr, nullptr};     // populations (float, or 16-bit offsets)
    float *f0[2] = {nullptr, nullptr};   // 16-bit storage: float rest populations [2][N]
    unsigned *step_ctr = nullptr;
    int fpar = 0;
    float *out = nullptr;
    float2 *rho[2] = {nullptr, nullptr};   // densities paired with each population buffer
    float2 *psi = nullptr;                 // pseudopotentials of the current step
    float4 *J = nullptr;                   // total momentum of the current step (tau = 1)
    uint32_t *mask = nullptr;
    // diffuse-interface coupling (CF_IBM): spread membrane force [3][N] (fixed
    // point), fluid velocity [N] followed by the block flags (ibm_flags), and
    // the all-zero cut bits the lattice reads
    long long *fibm = nullptr;
    float4 *uphys = nullptr;
    uint32_t *mask0 = nullptr;
    bool cuts_stale = false;  // CF_IBM: the cut links lag the positions until a readout needs them
    int *tri = nullptr;
    float2 *rec = nullptr;        // [N][18] bounce records (A, B) by arriving direction
    uint8_t *inside = nullptr;
    int2 *list[2] = {nullptr, nullptr};  // cut-link entries (node << 5 | k - 1, element)
    int *counts = nullptr;  // [2]
    int lpar = 0;
    int capacity = 0;
    unsigned *status = nullptr;
    double *dscratch = nullptr;  // small FP64 scratch (mass)
    double *pscratch = nullptr;  // meniscus profile readout [pcap]
    size_t pcap = 0;
    float *hscratch = nullptr;   // meniscus field [nx*ny]
    double *jit = nullptr;

    // membrane (all capsules concatenated)
    std::vector<HostCapsule> caps;
    int nnodes = 0, nfaces = 0;
    bool any_frozen = false, all_fixed = true;
    float *X[2] = {nullptr, nullptr};  // [hi 3*nv | lo 3*nv] per buffer
    int xpar = 0;
    // momentum exchanged with each element: FT[ftpar] accumulates this step's,
    // FT[1 - ftpar] holds the previous step's (two-step average)
    long long *FT[2] = {nullptr, nullptr};  // fixed point (ft_add)
    int ftpar = 0;
    float4 *uT = nullptr;  // element velocities, recorded with the cut links
    float *wet_el = nullptr;  // [nfaces] wetting offset per element (null when every capsule is neutral)
    float *V = nullptr, *fscr = nullptr, *vscr = nullptr,
          *Fcpl = nullptr, *refM = nullptr, *refA = nullptr, *refDet = nullptr;
    int *faces = nullptr, *face_cap = nullptr, *node_cap = nullptr, *vf_off = nullptr,
        *vf_ent = nullptr, *bbox[2] = {nullptr, nullptr};
    int *perm = nullptr;      // node of each patch slot (-1: padding), see MemParams
    int *nbr = nullptr, *nbr_cnt = nullptr;  // contact partners (CF_NBR_MIN_CAPS capsules or more)
    float *pbox = nullptr;    // patch boxes of this step
    int nslots = 0;
    CapDev *capdev = nullptr;
    double *acc = nullptr;
    std::vector<void *> mem_allocs;

    bool film_set = false;
    long long steps_done = 0;
    long long launches_last = 0;
    int zchunk = 0;
    int zring = 1;

    cudaGraphExec_t graph = nullptr;      // a captured step pair
    cudaGraphExec_t graph_out = nullptr;  // the same, its second step also recording the fields
    int graph_key = -1;
    int graph_launches = 0;  // kernel launches of one graph replay (two steps)

    // learned warm start: partial sums, density snapshot, check results
    double *warm_part = nullptr;
    float *snap = nullptr;
    double *warm_res = nullptr;

    // drying: A mass turned into B per step, and the reduction scratch
    double dry_dm = 0.0;
    double *dry_part = nullptr;
    unsigned *dry_ctr = nullptr;
    float *dry_eps = nullptr;
};

namespace {

// bytes of the block flags of the diffuse-interface coupling (one per 32 nodes)
size_t ibm_flag_bytes(long long N) { return (size_t)((N + 31) / 32 + 15) / 16 * 16; }

// the captured step pairs are stale (the layout or the parities changed)
void drop_graphs(cf_ctx *c) {
    if (c->graph) cudaGraphExecDestroy(c->graph);
    if (c->graph_out) cudaGraphExecDestroy(c->graph_out);
    c->graph = c->graph_out = nullptr;
    c->graph_key = -1;
}

void *dalloc(cf_ctx *c, size_t bytes, bool membrane = false) {
    void *p = nullptr;
    bytes = std::max<size_t>(bytes, 256);
    if (c->has_alloc) {
        p = c->alloc.alloc(bytes, c->stream, c->alloc.user);
    } else {
        if (cudaMallocAsync(&p, bytes, c->stream) != cudaSuccess) p = nullptr;
    }
    if (p) (membrane ? c->mem_allocs : c->allocations).push_back(p);
    return p;
}

void dfree(cf_ctx *c, void *p) {
    if (!p) return;
    if (c->has_alloc) c->alloc.free(p, c->stream, c->alloc.user);
    else cudaFreeAsync(p, c->stream);
}

cf_status check_status(cf_ctx *c) {
    unsigned st = 0;
    CF_CUDA(cudaMemcpyAsync(&st, c->status, sizeof(unsigned), cudaMemcpyDeviceToHost, c->stream));
    CF_CUDA(cudaStreamSynchronize(c->stream));
    if (st) {
        CF_CUDA(cudaMemsetAsync(c->status, 0, sizeof(unsigned), c->stream));
        if (st & ST_NAN) return fail(CF_EDIVERGED, "non-finite density in the lattice");
        if (st & ST_OVERFLOW)
            return fail(CF_EOVERFLOW, "cut-link list exceeded its capacity, or an element spans more "
                                      "than 16 lattice units (or has a non-finite position)");
    }
    return CF_OK;
}

LBParams lb_params(cf_ctx *c, bool with_out) {
    LBParams p{};
    p.nx = c->d.nx; p.ny = c->d.ny; p.nz = c->d.nz; p.wall = c->d.wall;
    p.N = c->N;
    p.zlo = c->d.wall ? 1 : 0;
    p.zhi = c->d.nz;
    p.zchunk = c->zchunk;
    p.zring = c->zring;
    for (int k = 0; k < 2; ++k) {
        p.tau[k] = (float)c->d.tau[k];
        p.itau[k] = (float)(1.0 / c->d.tau[k]);
    }
    p.G = (float)c->d.G;
    p.flags = c->d.flags;
    p.src = c->f[c->fpar];
    p.dst = c->f[1 - c->fpar];
    p.rho_src = c->rho[c->fpar];
    p.src0 = c->f0[c->fpar];
    p.dst0 = c->f0[1 - c->fpar];
    p.step_ctr = c->step_ctr;
    // with the diffuse-interface coupling no link is cut for the fluid
    p.mask = c->mask0 ? c->mask0 : c->mask;
    p.tri = c->tri;
    p.fibm = c->fibm;
    p.uphys = c->uphys;
    p.FT = c->FT[c->ftpar];
    p.out = with_out ? c->out : nullptr;
    p.rho = c->rho[1 - c->fpar];
    p.psi = c->psi;
    p.J = c->J;
    p.rec = c->rec;
    p.wet_el = c->wet_el;
    p.status = c->status;
    p.dry_dm = c->dry_dm;
    p.dry_part = c->dry_part;
    p.dry_ctr = c->dry_ctr;
    p.dry_eps = c->dry_eps;
    return p;
}

MemParams mem_params(cf_ctx *c) {
    MemParams p{};
    p.nx = c->d.nx; p.ny = c->d.ny; p.nz = c->d.nz; p.wall = c->d.wall;
    p.ncaps = (int)c->caps.size();
    p.nfaces = c->nfaces;
    p.nnodes = c->nnodes;
    p.zrep = (float)(0.5 + c->d.rep_dz);
    p.xi = (float)c->d.xi;
    p.delta0 = (float)c->d.delta0;
    p.caps = c->capdev;
    p.faces = c->faces;
    p.face_cap = c->face_cap;
    p.node_cap = c->node_cap;
    p.refM = c->refM; p.refA = c->refA; p.refDet = c->refDet;
    p.vf_off = c->vf_off; p.vf_ent = c->vf_ent;
    p.Xh = c->X[c->xpar];
    p.Xl = c->X[c->xpar] + 3 * (size_t)c->nnodes;
    p.Xnh = c->X[1 - c->xpar];
    p.Xnl = c->X[1 - c->xpar] + 3 * (size_t)c->nnodes;
    p.V = c->V;
    p.FT = c->FT[c->ftpar];
    p.FTprev = c->FT[1 - c->ftpar];
    p.fscr = c->fscr;
    p.vscr = c->vscr;
    p.Fcpl = c->Fcpl;
    p.acc = c->acc;
    p.bbox = c->bbox[c->xpar];
    p.bbox_prev = c->bbox[1 - c->xpar];
    p.status = c->status;
    p.any_frozen = c->any_frozen ? 1 : 0;
    p.inertial = (c->d.flags & CF_INERTIAL) ? 1 : 0;
    p.perm = c->perm;
    p.nslots = c->nslots;
    p.pbox = c->pbox;
    p.nbr = c->nbr;
    p.nbr_cnt = c->nbr_cnt;
    p.fibm = c->fibm;
    p.uphys = c->uphys;
    p.N = c->N;
    return p;
}

// Cut links of positions X into the list other than lpar (the caller flips lpar)
CutParams cut_params(cf_ctx *c, const float *X) {
    const int cur = 1 - c->lpar;
    CutParams q{};
    q.nx = c->d.nx; q.ny = c->d.ny; q.nz = c->d.nz; q.wall = c->d.wall;
    q.nfaces = c->nfaces;
    q.faces = c->faces;
    q.X = X;
    q.mask = c->mask;
    q.tri = c->tri;
    q.list = c->list[cur];
    q.count = c->counts + cur;
    q.FTnext = c->FT[1 - c->ftpar];
    q.V = c->V;
    q.uT = c->uT;
    q.capacity = c->capacity;
    q.status = c->status;
    return q;
}

// Cut links for positions X (cur list lpar, clears the other list's nodes).
// zeroed: the node update has already zeroed the new list's entry counter
cf_status enqueue_cuts(cf_ctx *c, const float *X, int *nl, bool zeroed = false) {
    if (c->nfaces == 0) return CF_OK;
    const int cur = 1 - c->lpar;
    const CutParams q = cut_params(c, X);
    if (!zeroed) CF_CUDA(cudaMemsetAsync(c->counts + cur, 0, sizeof(int), c->stream));
    CF_CUDA(launch_cuts(q, c->stream, nl));
    c->lpar = cur;
    return CF_OK;
}

// bounce records of the cut links for this step's streaming
PrepParams prep_params(cf_ctx *c, int blocks) {
    PrepParams q{};
    q.N = c->N;
    q.prec = c->d.precision;
    q.src = c->f[c->fpar];
    q.rho = c->rho[c->fpar];
    q.mask = c->mask;
    q.tri = c->tri;
    q.uT = c->uT;
    q.list = c->list[c->lpar];
    q.count = c->counts + c->lpar;
    q.rec = c->rec;
    q.FT = c->FT[c->ftpar];
    q.capacity = c->capacity;
    q.ref_rho = (c->d.flags & CF_LADD_REF_RHO) ? 1 : 0;
    q.blocks = blocks;
    return q;
}

// reset of the cut structure about to be rebuilt, by `blocks` extra blocks of
// the node update (none for fixed capsules, whose cut links never move)
ClearParams clear_params(cf_ctx *c, int blocks) {
    ClearParams cl{};
    if (!c->all_fixed) {
        cl.list = c->list[c->lpar];
        cl.count = c->counts + c->lpar;
        cl.capacity = c->capacity;
        cl.mask = c->mask;
        cl.tri = c->tri;
        cl.blocks = blocks;
        cl.count_next = c->counts + (1 - c->lpar);  // the cut links' memset, done by the update
    }
    return cl;
}

// One coupled step on the stream (also used under graph capture).  ev, when
// given, receives five events: ev[4] step start, ev[0] after the bounce
// records, ev[1] after the lattice update, ev[2] after the node update, ev[3]
// after the cut links.
//
//   stream   prep -> density -> collide ----join-> update (+ cut reset) [-> frozen] -> cut links
//   stream2       \-> memsets -> elements -> nodes -> bending -/
//
// The membrane's position-only kernels run beside the lattice update; the
// node update waits for both.
// The membrane half before the lattice update: fork the position-only
// membrane kernels onto stream2 and prepare the bounce records on the stream.
cf_status enqueue_pre(cf_ctx *c, int *nl) {
    if (c->nnodes == 0) return CF_OK;
    // fork: elastic, volume and bending forces of the current positions
    CF_CUDA(cudaEventRecord(c->ev_fork, c->stream));
    CF_CUDA(cudaStreamWaitEvent(c->stream2, c->ev_fork, 0));
    const int nc = (int)c->caps.size();
    int *bb = c->bbox[c->xpar];
    CF_CUDA(cudaMemsetAsync(c->acc, 0, sizeof(double) * A_NACC * nc, c->stream2));
    CF_CUDA(cudaMemsetAsync(bb, 0x7f, sizeof(int) * 3 * nc, c->stream2));
    CF_CUDA(cudaMemsetAsync(bb + 3 * nc, 0x80, sizeof(int) * 3 * nc, c->stream2));
    if (c->nbr) {  // partners from the previous step's boxes, read by the node update
        MemParams q = mem_params(c);
        q.nbr = nullptr;
        CF_CUDA(launch_contact_partners(q, c->nbr, c->nbr_cnt, c->stream2, nl));
    }
    CF_CUDA(launch_membrane_forces(mem_params(c), c->stream2, nl));
    CF_CUDA(cudaEventRecord(c->ev_join, c->stream2));
    // bounce records of the cut links for this step's streaming
    CF_CUDA(launch_prep(prep_params(c, 2 * 152), c->stream, nl));
    return CF_OK;
}

// The membrane half after the lattice update (whose populations are now in
// f[fpar]): join stream2, node update with the reset of the old cut
// structure, new cut links; ev2 (optional) is recorded after the node update.
cf_status enqueue_post(cf_ctx *c, int *nl, cudaEvent_t ev2 = nullptr) {
    const bool mem = c->nnodes > 0;
    if (mem) {
        CF_CUDA(cudaStreamWaitEvent(c->stream, c->ev_join, 0));
        // extra blocks of the update reset the cut structure about to be rebuilt
        CF_CUDA(launch_membrane_update(mem_params(c), clear_params(c, 304), c->any_frozen, c->stream, nl));
        c->xpar = 1 - c->xpar;
    }
    if (ev2) CF_CUDA(cudaEventRecord(ev2, c->stream));
    if (mem) {
        if (!c->all_fixed) {
            // also zeroes the exchange accumulator of the next step
            cf_status s = enqueue_cuts(c, c->X[c->xpar], nl, true);
            if (s != CF_OK) return s;
        } else {
            CF_CUDA(cudaMemsetAsync(c->FT[1 - c->ftpar], 0, sizeof(long long) * 3 * (size_t)c->nfaces,
                                    c->stream));
        }
        c->ftpar = 1 - c->ftpar;
    }
    return CF_OK;
}

// One step with the diffuse-interface coupling (CF_IBM):
//
//   stream   -------------------------------------> density --join-> collide -> move
//   stream2  \-> memsets -> elements -> nodes -> bending -> update: spread -/
//
// The membrane forces of the current positions are spread, beside the
// density pass, before the collision that applies them; the nodes then move
// with this step's fluid velocity.  The lattice sees no cut link: the cut
// links only give the interior flags of the readouts, which rebuild them
// (refresh_cuts) for the positions of the moment.
cf_status enqueue_step_ibm(cf_ctx *c, bool with_out, int *nl, cudaEvent_t *ev) {
    if (ev) CF_CUDA(cudaEventRecord(ev[4], c->stream));
    const bool mem = c->nnodes > 0;
    if (mem) {
        CF_CUDA(cudaEventRecord(c->ev_fork, c->stream));
        CF_CUDA(cudaStreamWaitEvent(c->stream2, c->ev_fork, 0));
        const int nc = (int)c->caps.size();
        int *bb = c->bbox[c->xpar];
        CF_CUDA(cudaMemsetAsync(c->acc, 0, sizeof(double) * A_NACC * nc, c->stream2));
        CF_CUDA(cudaMemsetAsync(bb, 0x7f, sizeof(int) * 3 * nc, c->stream2));
        CF_CUDA(cudaMemsetAsync(bb + 3 * nc, 0x80, sizeof(int) * 3 * nc, c->stream2));
        CF_CUDA(cudaMemsetAsync(ibm_flags(c->uphys, c->N), 0, ibm_flag_bytes(c->N), c->stream2));
        if (c->nbr) {
            MemParams q = mem_params(c);
            q.nbr = nullptr;
            CF_CUDA(launch_contact_partners(q, c->nbr, c->nbr_cnt, c->stream2, nl));
        }
        CF_CUDA(launch_membrane_forces(mem_params(c), c->stream2, nl));
        CF_CUDA(launch_membrane_update(mem_params(c), ClearParams{}, false, c->stream2, nl));
        CF_CUDA(cudaEventRecord(c->ev_join, c->stream2));
    }
    if (ev) CF_CUDA(cudaEventRecord(ev[0], c->stream));
    CF_CUDA(launch_lb_step(lb_params(c, with_out), c->d.precision, c->stream, mem ? c->ev_join : nullptr));
    *nl += 2;
    c->fpar = 1 - c->fpar;
    if (ev) CF_CUDA(cudaEventRecord(ev[1], c->stream));
    if (mem) {
        CF_CUDA(launch_ibm_move(mem_params(c), c->stream, nl));
        c->xpar = 1 - c->xpar;
    }
    if (ev) CF_CUDA(cudaEventRecord(ev[2], c->stream));
    if (mem && !c->all_fixed) c->cuts_stale = true;
    if (ev) CF_CUDA(cudaEventRecord(ev[3], c->stream));
    return CF_OK;
}

// Cut links of the current positions, where the steps have left them behind
// (CF_IBM): reset of the old structure, then the cut-link kernel.
cf_status refresh_cuts(cf_ctx *c) {
    if (!c->cuts_stale) return CF_OK;
    c->cuts_stale = false;
    int nl = 0;
    CF_CUDA(launch_cut_clear(clear_params(c, 304), c->stream, &nl));
    return enqueue_cuts(c, c->X[c->xpar], &nl, true);
}

// interior flags of the current positions (readouts)
cf_status inside_flags(cf_ctx *c) {
    if (!c->nfaces) return CF_OK;
    cf_status s = refresh_cuts(c);
    if (s != CF_OK) return s;
    CF_CUDA(launch_inside(c->mask, c->inside, c->d.nx, c->d.ny, c->d.nz, c->stream));
    return CF_OK;
}

cf_status enqueue_step(cf_ctx *c, bool with_out, int *nl, cudaEvent_t *ev = nullptr) {
    if (c->fibm) return enqueue_step_ibm(c, with_out, nl, ev);
    if (ev) CF_CUDA(cudaEventRecord(ev[4], c->stream));
    cf_status s = enqueue_pre(c, nl);
    if (s != CF_OK) return s;
    if (ev) CF_CUDA(cudaEventRecord(ev[0], c->stream));
    CF_CUDA(launch_lb_step(lb_params(c, with_out), c->d.precision, c->stream));
    *nl += 2;
    c->fpar = 1 - c->fpar;
    if (ev) CF_CUDA(cudaEventRecord(ev[1], c->stream));
    s = enqueue_post(c, nl, ev ? ev[2] : nullptr);
    if (s != CF_OK) return s;
    if (ev) CF_CUDA(cudaEventRecord(ev[3], c->stream));
    return CF_OK;
}

// The captured step pair of the context's current parities (out: its second
// step also records the fields); captured on first use, both dropped when the
// parities or the layout change.
cf_status step_graph(cf_ctx *c, bool out, cudaGraphExec_t *ge) {
    const int key = c->fpar | (c->xpar << 1) | (c->lpar << 2) | (c->ftpar << 3);
    if (c->graph_key != key) drop_graphs(c);
    cudaGraphExec_t &slot = out ? c->graph_out : c->graph;
    if (!slot) {
        cudaGraph_t g;
        CF_CUDA(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
        int nlg = 0;
        cf_status s1 = enqueue_step(c, false, &nlg);
        cf_status s2 = s1 == CF_OK ? enqueue_step(c, out, &nlg) : s1;
        cudaError_t e = cudaStreamEndCapture(c->stream, &g);
        if (s2 != CF_OK) return s2;
        if (e != cudaSuccess) return fail(CF_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e));
        e = cudaGraphInstantiate(&slot, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return fail(CF_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
        c->graph_key = key;
        c->graph_launches = nlg;
    }
    *ge = slot;
    return CF_OK;
}

void choose_launch(cf_ctx *c) {
    // blocks of 32 x 4 columns; each thread walks zchunk planes (strided), so
    // the grid holds about 48 blocks per SM (8 waves of the density pass at 6
    // resident blocks, 6 of the collide pass at 8: measured best between 25
    // and 80 blocks per SM on the 128x64x64 and 256x256x96 lattices)
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) sms = 152;
    const int cols = ((c->d.nx + 31) / 32) * ((c->d.ny + 3) / 4);
    const int nzf = c->d.nz - (c->d.wall ? 1 : 0);
    const int target = sms * 48;
    const int gz = std::max(1, std::min(nzf, (target + cols - 1) / cols));
    c->zchunk = std::max(1, (nzf + gz - 1) / gz);
    if (const char *e = std::getenv("CAPFILM_ZCHUNK")) {  // manual override for launch sweeps
        const int v = std::atoi(e);
        if (v > 0) c->zchunk = std::min(v, nzf);
    }
    // tau = 1 collide pass: each block walks zring contiguous planes through its
    // pseudopotential ring (halo loads amortised over the planes); as many as
    // keep about two waves of resident blocks (8 per SM), at most 16
    const int waves2 = 2 * 8 * sms;
    c->zring = std::max(1, std::min(16, (int)((long long)cols * nzf / waves2)));
    if (const char *e = std::getenv("CAPFILM_ZRING")) {
        const int v = std::atoi(e);
        if (v > 0) c->zring = std::min(v, nzf);
    }
}

cf_status build_membrane(cf_ctx *c) {
    for (void *p : c->mem_allocs) dfree(c, p);
    c->mem_allocs.clear();
    const int nc = (int)c->caps.size();
    int nv = 0, nf = 0;
    for (auto &h : c->caps) { nv += h.nv; nf += h.nf; }
    c->nnodes = nv;
    c->nfaces = nf;
    c->any_frozen = false;
    c->all_fixed = true;
    for (auto &h : c->caps) {
        c->any_frozen |= h.mode == CF_FROZEN;
        c->all_fixed &= h.mode == CF_FIXED;
    }
    std::vector<double> X(3 * (size_t)nv);
    std::vector<float> refM(3 * (size_t)nf), refA(nf), refDet(nf);
    std::vector<int> faces(3 * (size_t)nf), face_cap(nf), node_cap(nv);
    std::vector<CapDev> cd(nc);
    std::vector<std::vector<int>> vf(nv);
    int v0 = 0, f0 = 0;
    for (int k = 0; k < nc; ++k) {
        const HostCapsule &h = c->caps[k];
        CapDev &d = cd[k];
        d.kS = (float)h.kS; d.C = (float)h.C; d.kB = (float)h.kB; d.kV = (float)h.kV;
        d.mass = (float)h.mass; d.mode = h.mode;
        d.v0 = v0; d.nv = h.nv; d.f0 = f0; d.nf = h.nf;
        double V0 = 0.0;
        for (int i = 0; i < h.nv; ++i) {
            for (int a = 0; a < 3; ++a) X[3 * (size_t)(v0 + i) + a] = h.X[3 * i + a];
            node_cap[v0 + i] = k;
        }
        for (int f = 0; f < h.nf; ++f) {
            const int ia = h.F[3 * f], ib = h.F[3 * f + 1], ic = h.F[3 * f + 2];
            faces[3 * (size_t)(f0 + f)] = v0 + ia;
            faces[3 * (size_t)(f0 + f) + 1] = v0 + ib;
            faces[3 * (size_t)(f0 + f) + 2] = v0 + ic;
            face_cap[f0 + f] = k;
            vf[v0 + ia].push_back(3 * (f0 + f) + 0);
            vf[v0 + ib].push_back(3 * (f0 + f) + 1);
            vf[v0 + ic].push_back(3 * (f0 + f) + 2);
            double a[3], b[3], cc[3], u[3], w[3];
            for (int q = 0; q < 3; ++q) {
                a[q] = h.X[3 * ia + q]; b[q] = h.X[3 * ib + q]; cc[q] = h.X[3 * ic + q];
                u[q] = b[q] - a[q]; w[q] = cc[q] - a[q];
            }
            const double g11 = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
            const double g12 = u[0] * w[0] + u[1] * w[1] + u[2] * w[2];
            const double g22 = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
            const double det = g11 * g22 - g12 * g12;
            refM[3 * (size_t)(f0 + f)] = (float)(g22 / det);
            refM[3 * (size_t)(f0 + f) + 1] = (float)(-g12 / det);
            refM[3 * (size_t)(f0 + f) + 2] = (float)(g11 / det);
            refDet[f0 + f] = (float)det;
            refA[f0 + f] = (float)(0.5 * std::sqrt(det));
            const double n0 = b[1] * cc[2] - b[2] * cc[1], n1 = b[2] * cc[0] - b[0] * cc[2],
                         n2 = b[0] * cc[1] - b[1] * cc[0];
            V0 += (a[0] * n0 + a[1] * n1 + a[2] * n2) / 6.0;
        }
        d.V0 = V0;
        v0 += h.nv;
        f0 += h.nf;
    }
    std::vector<int> vf_off(nv + 1, 0), vf_ent;
    for (int v = 0; v < nv; ++v) {
        vf_off[v + 1] = vf_off[v] + (int)vf[v].size();
        for (int e : vf[v]) vf_ent.push_back(e);
    }
    // contact patches: each capsule's nodes in Morton order of their positions
    // (10 bits per axis over the capsule's box), 32 slots per patch
    std::vector<int> perm;
    for (int k = 0; k < nc; ++k) {
        CapDev &d = cd[k];
        double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
        for (int i = d.v0; i < d.v0 + d.nv; ++i)
            for (int a = 0; a < 3; ++a) {
                lo[a] = std::min(lo[a], X[3 * (size_t)i + a]);
                hi[a] = std::max(hi[a], X[3 * (size_t)i + a]);
            }
        std::vector<std::pair<unsigned long long, int>> key(d.nv);
        for (int i = 0; i < d.nv; ++i) {
            unsigned long long m = 0;
            for (int a = 0; a < 3; ++a) {
                const double span = hi[a] - lo[a];
                const double t = span > 0.0 ? (X[3 * (size_t)(d.v0 + i) + a] - lo[a]) / span : 0.0;
                const unsigned q = (unsigned)std::min(1023.0, std::max(0.0, std::floor(t * 1024.0)));
                for (int bit = 0; bit < 10; ++bit) m |= (unsigned long long)((q >> bit) & 1u) << (3 * bit + a);
            }
            key[i] = {m, d.v0 + i};
        }
        std::sort(key.begin(), key.end());
        d.s0 = (int)perm.size();
        d.ns = 32 * ((d.nv + 31) / 32);
        for (int i = 0; i < d.ns; ++i) perm.push_back(i < d.nv ? key[i].second : -1);
    }
    c->nslots = (int)perm.size();
    auto up = [&](void *dst, const void *src, size_t bytes) -> cudaError_t {
        return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, c->stream);
    };
#define MALLOC_M(ptr, T, n)                                                          \
    do {                                                                             \
        ptr = (T *)dalloc(c, sizeof(T) * (size_t)(n), true);                         \
        if (!ptr) return fail(CF_ENOMEM, "device allocation failed (membrane)");     \
    } while (0)
    MALLOC_M(c->X[0], float, 6 * nv);
    MALLOC_M(c->X[1], float, 6 * nv);
    MALLOC_M(c->V, float, 3 * nv);
    MALLOC_M(c->Fcpl, float, 3 * nv);
    MALLOC_M(c->vscr, float, 4 * nv);
    MALLOC_M(c->FT[0], long long, 3 * nf);
    MALLOC_M(c->FT[1], long long, 3 * nf);
    MALLOC_M(c->uT, float4, nf);
    MALLOC_M(c->fscr, float, (size_t)FS_N * nf);
    MALLOC_M(c->refM, float, 3 * nf);
    MALLOC_M(c->refA, float, nf);
    MALLOC_M(c->refDet, float, nf);
    MALLOC_M(c->faces, int, 3 * nf);
    MALLOC_M(c->face_cap, int, nf);
    MALLOC_M(c->node_cap, int, nv);
    MALLOC_M(c->vf_off, int, nv + 1);
    MALLOC_M(c->vf_ent, int, vf_ent.size());
    MALLOC_M(c->bbox[0], int, 6 * nc);
    MALLOC_M(c->bbox[1], int, 6 * nc);
    MALLOC_M(c->capdev, CapDev, nc);
    MALLOC_M(c->perm, int, c->nslots);
    MALLOC_M(c->pbox, float, 6 * (c->nslots / 32));
    c->nbr = c->nbr_cnt = nullptr;
    if (nc >= CF_NBR_MIN_CAPS) {
        MALLOC_M(c->nbr, int, (size_t)CF_NBR_MAX * nc);
        MALLOC_M(c->nbr_cnt, int, nc);
    }
    MALLOC_M(c->acc, double, A_NACC * nc);
    c->wet_el = nullptr;
    bool any_wet = false;
    for (auto &h : c->caps) any_wet |= h.wet != 0.0;
    if (any_wet) {
        MALLOC_M(c->wet_el, float, nf);
        std::vector<float> we(nf);
        for (int f = 0; f < nf; ++f) we[f] = (float)c->caps[face_cap[f]].wet;
        CF_CUDA(up(c->wet_el, we.data(), sizeof(float) * we.size()));
    }
#undef MALLOC_M
    c->xpar = 0;
    {   // bounding boxes of the initial shapes (read as the previous step's)
        std::vector<int> bb(6 * (size_t)nc);
        for (int k = 0; k < nc; ++k) {
            for (int a = 0; a < 3; ++a) { bb[3 * k + a] = INT_MAX; bb[3 * nc + 3 * k + a] = INT_MIN; }
            for (int i = cd[k].v0; i < cd[k].v0 + cd[k].nv; ++i)
                for (int a = 0; a < 3; ++a) {
                    bb[3 * k + a] = std::min(bb[3 * k + a], (int)std::floor(X[3 * (size_t)i + a]));
                    bb[3 * nc + 3 * k + a] = std::max(bb[3 * nc + 3 * k + a], (int)std::ceil(X[3 * (size_t)i + a]));
                }
        }
        CF_CUDA(up(c->bbox[0], bb.data(), sizeof(int) * bb.size()));
        CF_CUDA(up(c->bbox[1], bb.data(), sizeof(int) * bb.size()));
    }
    {   // hi + lo float pairs (the inputs are float-rounded, so lo starts at 0)
        std::vector<float> hl(6 * (size_t)nv, 0.f);
        for (size_t i = 0; i < X.size(); ++i) {
            hl[i] = (float)X[i];
            hl[X.size() + i] = (float)(X[i] - (double)hl[i]);
        }
        CF_CUDA(up(c->X[0], hl.data(), sizeof(float) * hl.size()));
        CF_CUDA(up(c->X[1], hl.data(), sizeof(float) * hl.size()));
    }
    CF_CUDA(cudaMemsetAsync(c->V, 0, sizeof(float) * 3 * nv, c->stream));
    CF_CUDA(cudaMemsetAsync(c->Fcpl, 0, sizeof(float) * 3 * nv, c->stream));
    CF_CUDA(cudaMemsetAsync(c->FT[0], 0, sizeof(long long) * 3 * nf, c->stream));
    CF_CUDA(cudaMemsetAsync(c->FT[1], 0, sizeof(long long) * 3 * nf, c->stream));
    c->ftpar = 0;
    CF_CUDA(cudaMemsetAsync(c->acc, 0, sizeof(double) * A_NACC * nc, c->stream));
    CF_CUDA(up(c->refM, refM.data(), sizeof(float) * refM.size()));
    CF_CUDA(up(c->refA, refA.data(), sizeof(float) * refA.size()));
    CF_CUDA(up(c->refDet, refDet.data(), sizeof(float) * refDet.size()));
    CF_CUDA(up(c->faces, faces.data(), sizeof(int) * faces.size()));
    CF_CUDA(up(c->face_cap, face_cap.data(), sizeof(int) * face_cap.size()));
    CF_CUDA(up(c->node_cap, node_cap.data(), sizeof(int) * node_cap.size()));
    CF_CUDA(up(c->vf_off, vf_off.data(), sizeof(int) * vf_off.size()));
    CF_CUDA(up(c->vf_ent, vf_ent.data(), sizeof(int) * vf_ent.size()));
    CF_CUDA(up(c->capdev, cd.data(), sizeof(CapDev) * cd.size()));
    CF_CUDA(up(c->perm, perm.data(), sizeof(int) * perm.size()));
    // cut-link lists: one entry per end node of each crossing (link, element);
    // an element of edge < 1 crosses a few links, 24 entries per element is a
    // wide bound (overflow raises CF_EOVERFLOW)
    c->capacity = (int)std::min<long long>(36LL * c->N, 24LL * nf + 4096);
    for (int k = 0; k < 2; ++k) {
        c->list[k] = (int2 *)dalloc(c, sizeof(int2) * (size_t)c->capacity, true);
        if (!c->list[k]) return fail(CF_ENOMEM, "device allocation failed (cut lists)");
    }
    // bounce records, dense per node: written and read only at cut links
    c->rec = (float2 *)dalloc(c, sizeof(float2) * 18 * (size_t)c->N, true);
    if (!c->rec) return fail(CF_ENOMEM, "device allocation failed (cut records)");
    // start from a clean cut structure
    CF_CUDA(cudaMemsetAsync(c->mask, 0, sizeof(uint32_t) * c->N, c->stream));
    CF_CUDA(cudaMemsetAsync(c->tri, 0x7f, sizeof(int) * 18 * (size_t)c->N, c->stream));
    CF_CUDA(cudaMemsetAsync(c->counts, 0, sizeof(int) * 2, c->stream));
    // 0x7f7f7f7f is not INT_MAX but any value above every element index works
    int nl = 0;
    cf_status s = enqueue_cuts(c, c->X[c->xpar], &nl);
    if (s != CF_OK) return s;
    CF_CUDA(launch_inside(c->mask, c->inside, c->d.nx, c->d.ny, c->d.nz, c->stream));
    drop_graphs(c);
    return CF_OK;
}

cf_status sync_ok(cf_ctx *c) {
    CF_CUDA(cudaStreamSynchronize(c->stream));
    return check_status(c);
}

}  // namespace

extern "C" {

const char *cf_last_error(void) { return g_err.c_str(); }

cf_status cf_create(const cf_lattice_desc *desc, cf_ctx **out) {
    if (!desc || !out) return fail(CF_EINVAL, "null argument");
    if (desc->nx < 3 || desc->ny < 3 || desc->nz < 3) return fail(CF_EINVAL, "lattice dimensions must be >= 3");
    // a cut-list entry holds the node index in 26 bits (cut_code); population
    // offsets within one component (at most 18 N) then stay 32-bit
    if ((long long)desc->nx * desc->ny * desc->nz >= (1LL << 26))
        return fail(CF_EINVAL, "lattice too large (N >= 2^26 nodes)");
    if (!(desc->tau[0] > 0.5) || !(desc->tau[1] > 0.5)) return fail(CF_EINVAL, "tau must exceed 1/2");
    if (desc->precision != CF_FP32 && desc->precision != CF_FP16_SHIFT &&
        desc->precision != CF_BF16_SHIFT)
        return fail(CF_EINVAL, "unsupported precision");
    if (desc->flags & ~(CF_INERTIAL | CF_LADD_REF_RHO | CF_PARTNER_MIRROR | CF_DRY_REMOVE | CF_IBM))
        return fail(CF_EINVAL, "unknown flag");
    if ((desc->flags & CF_IBM) && (desc->flags & CF_INERTIAL))
        return fail(CF_EINVAL, "CF_INERTIAL does not apply to the diffuse-interface coupling (CF_IBM)");
    cf_ctx *c = new cf_ctx();
    c->d = *desc;
    c->N = (long long)desc->nx * desc->ny * desc->nz;
    if (desc->allocator) {
        c->alloc = *desc->allocator;
        c->has_alloc = c->alloc.alloc && c->alloc.free;
    }
    if (desc->stream) c->stream = (cudaStream_t)desc->stream;
    else {
        if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete c;
            return fail(CF_ECUDA, "cudaStreamCreate failed");
        }
        c->own_stream = true;
    }
    if (cudaStreamCreateWithFlags(&c->stream2, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_batch, cudaEventDisableTiming) != cudaSuccess) {
        cf_destroy(c);
        return fail(CF_ECUDA, "stream / event creation failed");
    }
    const long long N = c->N;
    const size_t pb = pop_bytes(desc->precision);
    c->f[0] = dalloc(c, pb * 38 * N);
    c->f[1] = dalloc(c, pb * 38 * N);
    c->out = (float *)dalloc(c, sizeof(float) * 5 * N);
    c->f0[0] = (float *)dalloc(c, sizeof(float) * 2 * N);
    c->f0[1] = (float *)dalloc(c, sizeof(float) * 2 * N);
    c->step_ctr = (unsigned *)dalloc(c, sizeof(unsigned));
    c->rho[0] = (float2 *)dalloc(c, sizeof(float2) * N);
    c->rho[1] = (float2 *)dalloc(c, sizeof(float2) * N);
    c->psi = (float2 *)dalloc(c, sizeof(float2) * N);
    // tau = 1 for both components: the density pass also stores the momentum
    const bool tau1 = (float)desc->tau[0] == 1.f && (float)desc->tau[1] == 1.f;
    c->J = tau1 ? (float4 *)dalloc(c, sizeof(float4) * N) : nullptr;
    c->mask = (uint32_t *)dalloc(c, sizeof(uint32_t) * N);
    c->tri = (int *)dalloc(c, sizeof(int) * 18 * N);
    c->inside = (uint8_t *)dalloc(c, N);
    c->counts = (int *)dalloc(c, sizeof(int) * 2);
    c->status = (unsigned *)dalloc(c, sizeof(unsigned));
    c->dscratch = (double *)dalloc(c, sizeof(double) * 8);
    c->hscratch = (float *)dalloc(c, sizeof(float) * desc->nx * desc->ny);
    const bool ibm = (desc->flags & CF_IBM) != 0;
    if (ibm) {
        c->fibm = (long long *)dalloc(c, sizeof(long long) * 3 * N);
        c->uphys = (float4 *)dalloc(c, sizeof(float4) * N + ibm_flag_bytes(N));
        c->mask0 = (uint32_t *)dalloc(c, sizeof(uint32_t) * N);
    }
    if ((ibm && (!c->fibm || !c->uphys || !c->mask0)) || !c->f[0] || !c->f[1] || !c->f0[0] || !c->f0[1] || !c->step_ctr || !c->out || !c->rho[0] || !c->rho[1] || !c->psi || (tau1 && !c->J) || !c->mask || !c->tri || !c->inside ||
        !c->counts || !c->status || !c->dscratch || !c->hscratch) {
        cf_destroy(c);
        return fail(CF_ENOMEM, "device allocation failed");
    }
    cudaMemsetAsync(c->f[0], 0, pb * 38 * N, c->stream);
    cudaMemsetAsync(c->f[1], 0, pb * 38 * N, c->stream);
    cudaMemsetAsync(c->f0[0], 0, sizeof(float) * 2 * N, c->stream);
    cudaMemsetAsync(c->f0[1], 0, sizeof(float) * 2 * N, c->stream);
    cudaMemsetAsync(c->step_ctr, 0, sizeof(unsigned), c->stream);
    cudaMemsetAsync(c->rho[0], 0, sizeof(float2) * N, c->stream);
    cudaMemsetAsync(c->rho[1], 0, sizeof(float2) * N, c->stream);
    cudaMemsetAsync(c->psi, 0, sizeof(float2) * N, c->stream);
    cudaMemsetAsync(c->out, 0, sizeof(float) * 5 * N, c->stream);
    cudaMemsetAsync(c->mask, 0, sizeof(uint32_t) * N, c->stream);
    cudaMemsetAsync(c->tri, 0x7f, sizeof(int) * 18 * N, c->stream);
    cudaMemsetAsync(c->inside, 0, N, c->stream);
    cudaMemsetAsync(c->counts, 0, sizeof(int) * 2, c->stream);
    cudaMemsetAsync(c->status, 0, sizeof(unsigned), c->stream);
    if (ibm) {
        cudaMemsetAsync(c->fibm, 0, sizeof(long long) * 3 * N, c->stream);
        cudaMemsetAsync(c->uphys, 0, sizeof(float4) * N + ibm_flag_bytes(N), c->stream);
        cudaMemsetAsync(c->mask0, 0, sizeof(uint32_t) * N, c->stream);
    }
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        cf_destroy(c);
        return fail(CF_ECUDA, std::string("set-up: ") + cudaGetErrorString(e));
    }
    choose_launch(c);
    *out = c;
    return CF_OK;
}

cf_status cf_destroy(cf_ctx *c) {
    if (!c) return CF_OK;
    if (c->stream) cudaStreamSynchronize(c->stream);
    drop_graphs(c);
    for (void *p : c->mem_allocs) dfree(c, p);
    for (void *p : c->allocations) dfree(c, p);
    if (c->jit) dfree(c, c->jit);
    if (c->pscratch) dfree(c, c->pscratch);
    if (c->stream) cudaStreamSynchronize(c->stream);
    if (c->stream2) { cudaStreamSynchronize(c->stream2); cudaStreamDestroy(c->stream2); }
    if (c->ev_fork) cudaEventDestroy(c->ev_fork);
    if (c->ev_join) cudaEventDestroy(c->ev_join);
    if (c->ev_batch) cudaEventDestroy(c->ev_batch);
    if (c->own_stream) cudaStreamDestroy(c->stream);
    delete c;
    return CF_OK;
}

// one capsule descriptor as host data (validated)
static cf_status host_capsule(const cf_capsule_desc *d, HostCapsule &h) {
    if (!d->nodes || !d->faces) return fail(CF_EINVAL, "null argument");
    if (d->nv < 4 || d->nf < 4) return fail(CF_EINVAL, "capsule mesh too small");
    if (d->mode < 0 || d->mode > 2) return fail(CF_EINVAL, "bad capsule mode");
    if (!(d->mass > 0)) return fail(CF_EINVAL, "node mass must be positive");
    if (!std::isfinite(d->wet)) return fail(CF_EINVAL, "wetting offset must be finite");
    h.nv = d->nv; h.nf = d->nf; h.mode = d->mode;
    h.kS = d->kS; h.C = d->C; h.kB = d->kB; h.kV = d->kV; h.mass = d->mass; h.wet = d->wet;
    h.X.resize(3 * (size_t)d->nv);
    for (size_t i = 0; i < h.X.size(); ++i) h.X[i] = (float)d->nodes[i];
    h.F.assign(d->faces, d->faces + 3 * (size_t)d->nf);
    for (int v : h.F)
        if (v < 0 || v >= d->nv) return fail(CF_EINVAL, "face index out of range");
    return CF_OK;
}

cf_status cf_add_capsules(cf_ctx *c, const cf_capsule_desc *d, int n, int *ids) {
    if (!c || !d || n < 1) return fail(CF_EINVAL, "null argument");
    if (c->film_set) return fail(CF_ESTATE, "capsules must be added before cf_set_film");
    std::vector<HostCapsule> hs(n);
    for (int k = 0; k < n; ++k) {
        cf_status s = host_capsule(d + k, hs[k]);
        if (s != CF_OK) return s;
        if (c->fibm && hs[k].mode == CF_FROZEN)
            return fail(CF_EINVAL, "frozen capsules need the cut-link coupling (not CF_IBM)");
    }
    const size_t n0 = c->caps.size();
    for (auto &h : hs) c->caps.push_back(std::move(h));
    cf_status s = build_membrane(c);
    if (s != CF_OK) { c->caps.resize(n0); return s; }
    if (ids)
        for (int k = 0; k < n; ++k) ids[k] = (int)(n0 + k);
    return sync_ok(c);
}

cf_status cf_add_capsule(cf_ctx *c, const cf_capsule_desc *d, int *id) {
    if (!c || !d) return fail(CF_EINVAL, "null argument");
    return cf_add_capsules(c, d, 1, id);
}

cf_status cf_set_capsule_mode(cf_ctx *c, int id, int mode) {
    if (!c) return fail(CF_EINVAL, "null context");
    if (id < 0 || id >= (int)c->caps.size()) return fail(CF_ENOTFOUND, "unknown capsule");
    if (mode < 0 || mode > 2) return fail(CF_EINVAL, "bad capsule mode");
    if (c->fibm && mode == CF_FROZEN)
        return fail(CF_EINVAL, "frozen capsules need the cut-link coupling (not CF_IBM)");
    CF_CUDA(cudaStreamSynchronize(c->stream));
    c->caps[id].mode = mode;
    CapDev d;
    CF_CUDA(cudaMemcpy(&d, c->capdev + id, sizeof(CapDev), cudaMemcpyDeviceToHost));
    d.mode = mode;
    CF_CUDA(cudaMemcpy(c->capdev + id, &d, sizeof(CapDev), cudaMemcpyHostToDevice));
    c->any_frozen = false;
    c->all_fixed = true;
    for (auto &h : c->caps) {
        c->any_frozen |= h.mode == CF_FROZEN;
        c->all_fixed &= h.mode == CF_FIXED;
    }
    drop_graphs(c);
    return CF_OK;
}

cf_status cf_remove_mass(cf_ctx *c, double dm) {
    if (!c) return fail(CF_EINVAL, "null context");
    if (!(dm >= 0.0) || !std::isfinite(dm)) return fail(CF_EINVAL, "the mass per step must be finite and >= 0");
    if (dm > 0.0 && !c->dry_part) {
        // one partial sum per density-pass block
        const size_t nb = density_blocks_max(c->d.nx, c->d.ny, c->d.nz);
        c->dry_part = (double *)dalloc(c, sizeof(double) * nb);
        c->dry_ctr = (unsigned *)dalloc(c, sizeof(unsigned));
        c->dry_eps = (float *)dalloc(c, sizeof(float));
        if (!c->dry_part || !c->dry_ctr || !c->dry_eps) return fail(CF_ENOMEM, "device allocation failed (drying)");
        CF_CUDA(cudaMemsetAsync(c->dry_ctr, 0, sizeof(unsigned), c->stream));
        CF_CUDA(cudaMemsetAsync(c->dry_eps, 0, sizeof(float), c->stream));
    }
    CF_CUDA(cudaStreamSynchronize(c->stream));
    c->dry_dm = dm;
    drop_graphs(c);
    return CF_OK;
}

cf_status cf_set_film(cf_ctx *c, double h_top, double rmaj, double rmin, double rmix,
                      const double *jitter) {
    if (!c) return fail(CF_EINVAL, "null context");
    const long long N = c->N;
    const double *djit = nullptr;
    if (jitter) {
        if (!c->jit) {
            c->jit = (double *)dalloc(c, sizeof(double) * 2 * N);
            if (!c->jit) return fail(CF_ENOMEM, "device allocation failed (jitter)");
            c->allocations.pop_back();  // freed explicitly
        }
        CF_CUDA(cudaMemcpyAsync(c->jit, jitter, sizeof(double) * 2 * N, cudaMemcpyHostToDevice, c->stream));
        djit = c->jit;
    }
    if (cf_status si = inside_flags(c); si != CF_OK) return si;
    CF_CUDA(launch_init_film(c->f[c->fpar], c->f0[c->fpar], c->d.precision, c->rho[c->fpar], N, c->d.nx, c->d.ny, c->d.nz, c->d.wall, (float)h_top,
                             (float)rmaj, (float)rmin, (float)rmix, djit, c->inside, c->stream));
    c->film_set = true;
    return sync_ok(c);
}

cf_status cf_set_densities(cf_ctx *c, const double *rhoA, const double *rhoB) {
    if (!c || !rhoA || !rhoB) return fail(CF_EINVAL, "null argument");
    const long long N = c->N;
    if (!c->jit) {
        c->jit = (double *)dalloc(c, sizeof(double) * 2 * N);
        if (!c->jit) return fail(CF_ENOMEM, "device allocation failed (densities)");
        c->allocations.pop_back();  // freed explicitly
    }
    CF_CUDA(cudaMemcpyAsync(c->jit, rhoA, sizeof(double) * N, cudaMemcpyHostToDevice, c->stream));
    CF_CUDA(cudaMemcpyAsync(c->jit + N, rhoB, sizeof(double) * N, cudaMemcpyHostToDevice, c->stream));
    CF_CUDA(launch_init_dens(c->f[c->fpar], c->f0[c->fpar], c->d.precision, c->rho[c->fpar], N, c->d.nx,
                             c->d.ny, c->d.wall, c->jit, c->stream));
    c->film_set = true;
    return sync_ok(c);
}

// ------------------------------------------------ learned warm start set-up
namespace {
WarmGeom warm_geom(const cf_ctx *c, double h_top, double rmaj, double rmin, double rmix) {
    WarmGeom g{};
    g.nx = c->d.nx; g.ny = c->d.ny; g.nz = c->d.nz; g.wall = c->d.wall;
    g.N = c->N;
    g.zm = (int)std::floor(h_top + 0.5);
    g.rmaj = rmaj; g.rmin = rmin; g.rmix = rmix; g.drho = rmaj - rmin;
    return g;
}
cf_status warm_scratch(cf_ctx *c) {
    if (!c->warm_part) {
        c->warm_part = (double *)dalloc(c, sizeof(double) * 4 * (size_t)warm_parts());
        c->warm_res = (double *)dalloc(c, sizeof(double) * 4);
        c->snap = (float *)dalloc(c, sizeof(float) * 2 * (size_t)c->N);
        if (!c->warm_part || !c->warm_res || !c->snap) return fail(CF_ENOMEM, "device allocation failed (warm start)");
        CF_CUDA(cudaMemsetAsync(c->snap, 0, sizeof(float) * 2 * (size_t)c->N, c->stream));
    }
    if (!c->jit) {
        c->jit = (double *)dalloc(c, sizeof(double) * 2 * c->N);
        if (!c->jit) return fail(CF_ENOMEM, "device allocation failed (densities)");
        c->allocations.pop_back();  // freed explicitly
    }
    return CF_OK;
}
}  // namespace

cf_status cf_warm_features(cf_ctx *c, double h_top, double kS, float *x, float *mask) {
    if (!c || !x) return fail(CF_EINVAL, "null argument");
    if (!(kS > 0.0)) return fail(CF_EINVAL, "kS must be positive");
    if (cf_status si = inside_flags(c); si != CF_OK) return si;
    const WarmGeom g = warm_geom(c, h_top, 0.0, 0.0, 0.0);
    CF_CUDA(launch_warm_features(g, c->inside, (float)(std::log10(kS) + 2.0), x, mask, c->stream));
    return sync_ok(c);
}

cf_status cf_warm_apply(cf_ctx *c, double h_top, double rmaj, double rmin, double rmix, const float *d) {
    if (!c || !d) return fail(CF_EINVAL, "null argument");
    if (!(rmaj > rmin)) return fail(CF_EINVAL, "rho_maj must exceed rho_min");
    cf_status s = warm_scratch(c);
    if (s != CF_OK) return s;
    if (cf_status si = inside_flags(c); si != CF_OK) return si;
    const WarmGeom g = warm_geom(c, h_top, rmaj, rmin, rmix);
    CF_CUDA(launch_warm_densities(g, c->inside, d, c->jit, c->warm_part, c->stream));
    CF_CUDA(launch_init_dens(c->f[c->fpar], c->f0[c->fpar], c->d.precision, c->rho[c->fpar], c->N, c->d.nx,
                             c->d.ny, c->d.wall, c->jit, c->stream));
    c->film_set = true;
    return sync_ok(c);
}

cf_status cf_warm_target(cf_ctx *c, double h_top, double rmaj, double rmin, double rmix, float *t) {
    if (!c || !t) return fail(CF_EINVAL, "null argument");
    if (!(rmaj > rmin)) return fail(CF_EINVAL, "rho_maj must exceed rho_min");
    if (!c->film_set) return fail(CF_ESTATE, "no fields before the first step");
    if (cf_status si = inside_flags(c); si != CF_OK) return si;
    const WarmGeom g = warm_geom(c, h_top, rmaj, rmin, rmix);
    CF_CUDA(launch_warm_target(g, c->inside, c->out, t, c->stream));
    return sync_ok(c);
}

cf_status cf_field_check(cf_ctx *c, double out[4]) {
    if (!c || !out) return fail(CF_EINVAL, "null argument");
    if (!c->film_set) return fail(CF_ESTATE, "no fields before the first step");
    cf_status s = warm_scratch(c);
    if (s != CF_OK) return s;
    CF_CUDA(launch_field_check(c->N, c->out, c->snap, c->warm_part, c->warm_res, c->stream));
    CF_CUDA(cudaMemcpyAsync(out, c->warm_res, sizeof(double) * 4, cudaMemcpyDeviceToHost, c->stream));
    return sync_ok(c);
}

cf_status cf_step(cf_ctx *c, long long n) {
    if (!c) return fail(CF_EINVAL, "null context");
    if (!c->film_set) return fail(CF_ESTATE, "cf_set_film must come before cf_step");
    if (n < 0) return fail(CF_EINVAL, "negative step count");
    if (n == 0) return CF_OK;
    // Steps come from captured step pairs (each returns every double buffer
    // to its parity), the last step recording the fields: an even count ends
    // with the pair whose second step records them, an odd count with one
    // plain recording step.
    int nl = 0;
    long long left = n;
    auto key_of = [](const cf_ctx *x) { return x->fpar | (x->xpar << 1) | (x->lpar << 2) | (x->ftpar << 3); };
    if (left >= 4 && c->graph && c->graph_key != key_of(c)) {
        // every double buffer flips each step, so one plain step brings the
        // context to the parity of the captured graphs (no capture here)
        cf_status s = enqueue_step(c, false, &nl);
        if (s != CF_OK) return s;
        --left;
    }
    if (left >= 3) {
        const bool odd = (left & 1) != 0;
        const long long pairs = left / 2;
        for (long long k = 0; k < pairs; ++k) {
            const bool out = !odd && k == pairs - 1;
            cudaGraphExec_t ge = nullptr;
            cf_status s = step_graph(c, out, &ge);
            if (s != CF_OK) return s;
            CF_CUDA(cudaGraphLaunch(ge, c->stream));
            nl += c->graph_launches;
        }
        left -= 2 * pairs;
    }
    while (left > 0) {
        cf_status s = enqueue_step(c, left == 1, &nl);
        if (s != CF_OK) return s;
        --left;
    }
    c->steps_done += n;
    c->launches_last = nl;
    return CF_OK;
}

cf_status cf_time_phases(cf_ctx *c, long long n, double ms[4]) {
    if (!c || !ms || n <= 0) return fail(CF_EINVAL, "bad argument");
    if (!c->film_set) return fail(CF_ESTATE, "cf_set_film must come before cf_time_phases");
    std::vector<cudaEvent_t> ev(5 * (size_t)n);
    for (auto &e : ev) CF_CUDA(cudaEventCreate(&e));
    int nl = 0;
    cf_status st = CF_OK;
    for (long long k = 0; k < n && st == CF_OK; ++k) st = enqueue_step(c, k == n - 1, &nl, &ev[5 * k]);
    CF_CUDA(cudaStreamSynchronize(c->stream));
    ms[0] = ms[1] = ms[2] = ms[3] = 0.0;
    for (long long k = 0; k < n && st == CF_OK; ++k) {
        for (int q = 0; q < 3; ++q) {
            float t = 0.f;
            CF_CUDA(cudaEventElapsedTime(&t, ev[5 * k + q], ev[5 * k + q + 1]));
            ms[q] += t / n;
        }
        float t = 0.f;
        CF_CUDA(cudaEventElapsedTime(&t, ev[5 * k + 4], ev[5 * k]));
        ms[3] += t / n;
    }
    for (auto &e : ev) cudaEventDestroy(e);
    if (st != CF_OK) return st;
    c->steps_done += n;
    c->launches_last = nl;
    return check_status(c);
}

cf_status cf_sync(cf_ctx *c) {
    if (!c) return fail(CF_EINVAL, "null context");
    return sync_ok(c);
}

cf_status cf_launch_count(cf_ctx *c, long long *n) {
    if (!c || !n) return fail(CF_EINVAL, "null argument");
    *n = c->launches_last;
    return CF_OK;
}

static cf_status read_acc(cf_ctx *c, std::vector<double> &acc) {
    const int nc = (int)c->caps.size();
    acc.assign((size_t)A_NACC * nc, 0.0);
    if (!nc) return CF_OK;
    CF_CUDA(cudaMemcpyAsync(acc.data(), c->acc, sizeof(double) * acc.size(), cudaMemcpyDeviceToHost, c->stream));
    return sync_ok(c);
}

cf_status cf_capsule_force(cf_ctx *c, int id, double F[3], double T[3]) {
    if (!c) return fail(CF_EINVAL, "null context");
    if (id < 0 || id >= (int)c->caps.size()) return fail(CF_ENOTFOUND, "unknown capsule");
    std::vector<double> acc;
    cf_status s = read_acc(c, acc);
    if (s != CF_OK) return s;
    for (int a = 0; a < 3; ++a) {
        if (F) F[a] = acc[(size_t)id * A_NACC + A_FX + a];
        if (T) T[a] = acc[(size_t)id * A_NACC + A_TX + a];
    }
    return CF_OK;
}

cf_status cf_lateral_force(cf_ctx *c, int a, int b, double *F) {
    if (!c || !F) return fail(CF_EINVAL, "null argument");
    const int nc = (int)c->caps.size();
    if (a < 0 || a >= nc || b < 0 || b >= nc || a == b) return fail(CF_ENOTFOUND, "unknown capsule pair");
    std::vector<double> acc;
    cf_status s = read_acc(c, acc);
    if (s != CF_OK) return s;
    const double *A = &acc[(size_t)a * A_NACC], *B = &acc[(size_t)b * A_NACC];
    double dx = (B[A_OX] + B[A_CX] / c->caps[b].nv) - (A[A_OX] + A[A_CX] / c->caps[a].nv);
    double dy = (B[A_OY] + B[A_CY] / c->caps[b].nv) - (A[A_OY] + A[A_CY] / c->caps[a].nv);
    dx -= c->d.nx * std::floor(dx / c->d.nx + 0.5);
    dy -= c->d.ny * std::floor(dy / c->d.ny + 0.5);
    const double L = std::sqrt(dx * dx + dy * dy);
    if (!(L > 0)) return fail(CF_EINVAL, "capsule centroids coincide in the xy plane");
    *F = 0.5 * ((B[A_FX] - A[A_FX]) * dx + (B[A_FY] - A[A_FY]) * dy) / L;
    return CF_OK;
}

cf_status cf_capsule_state(cf_ctx *c, int id, double *nodes, double *area, double *volume) {
    if (!c) return fail(CF_EINVAL, "null context");
    if (id < 0 || id >= (int)c->caps.size()) return fail(CF_ENOTFOUND, "unknown capsule");
    int v0 = 0;
    for (int k = 0; k < id; ++k) v0 += c->caps[k].nv;
    const int nv = c->caps[id].nv;
    if (nodes) {
        std::vector<float> h(3 * (size_t)nv), l(3 * (size_t)nv);
        CF_CUDA(cudaMemcpyAsync(h.data(), c->X[c->xpar] + 3 * (size_t)v0, sizeof(float) * h.size(),
                                cudaMemcpyDeviceToHost, c->stream));
        CF_CUDA(cudaMemcpyAsync(l.data(), c->X[c->xpar] + 3 * (size_t)c->nnodes + 3 * (size_t)v0,
                                sizeof(float) * l.size(), cudaMemcpyDeviceToHost, c->stream));
        cf_status s = sync_ok(c);
        if (s != CF_OK) return s;
        for (size_t i = 0; i < h.size(); ++i) nodes[i] = (double)h[i] + (double)l[i];
    }
    if (area || volume) {
        std::vector<double> acc;
        cf_status s = read_acc(c, acc);
        if (s != CF_OK) return s;
        if (area) *area = acc[(size_t)id * A_NACC + A_AREA];
        if (volume) *volume = acc[(size_t)id * A_NACC + A_VOL];
    }
    return CF_OK;
}

cf_status cf_fields(cf_ctx *c, double *rho, double *u, size_t *inout_n) {
    if (!c || !inout_n) return fail(CF_EINVAL, "null argument");
    const long long N = c->N;
    if (*inout_n < (size_t)N) {
        *inout_n = (size_t)N;
        return fail(CF_EINVAL, "field buffers too small (need " + std::to_string(N) + " nodes)");
    }
    *inout_n = (size_t)N;
    std::vector<float> h(5 * (size_t)N);
    CF_CUDA(cudaMemcpyAsync(h.data(), c->out, sizeof(float) * h.size(), cudaMemcpyDeviceToHost, c->stream));
    cf_status s = sync_ok(c);
    if (s != CF_OK) return s;
    if (rho) for (long long i = 0; i < 2 * N; ++i) rho[i] = h[i];
    if (u) for (long long i = 0; i < 3 * N; ++i) u[i] = h[2 * N + i];
    return CF_OK;
}

cf_status cf_populations(cf_ctx *c, float *f) {
    if (!c || !f) return fail(CF_EINVAL, "null argument");
    const long long N = c->N;
    if (c->d.precision == CF_FP32) {
        CF_CUDA(cudaMemcpyAsync(f, c->f[c->fpar], sizeof(float) * 38 * N, cudaMemcpyDeviceToHost, c->stream));
        return sync_ok(c);
    }
    // 16-bit offsets: f_i = g_i + w_i rho (rho of the node that wrote them)
    std::vector<uint16_t> g(38 * (size_t)N);
    std::vector<float2> d((size_t)N);
    std::vector<float> r0(2 * (size_t)N);
    CF_CUDA(cudaMemcpyAsync(g.data(), c->f[c->fpar], 2 * g.size(), cudaMemcpyDeviceToHost, c->stream));
    CF_CUDA(cudaMemcpyAsync(r0.data(), c->f0[c->fpar], sizeof(float) * r0.size(), cudaMemcpyDeviceToHost, c->stream));
    CF_CUDA(cudaMemcpyAsync(d.data(), c->rho[c->fpar], sizeof(float2) * d.size(), cudaMemcpyDeviceToHost, c->stream));
    cf_status s = sync_ok(c);
    if (s != CF_OK) return s;
    const bool bf = c->d.precision == CF_BF16_SHIFT;
    for (int comp = 0; comp < 2; ++comp)
        for (int i = 0; i < Q; ++i) {
            const float w = i == 0 ? 1.0f / 3.0f : (i <= 6 ? 1.0f / 18.0f : 1.0f / 36.0f);
            for (long long n = 0; n < N; ++n) {
                if (i == 0) {  // rest populations are kept in float
                    f[((size_t)comp * Q) * N + n] = r0[(size_t)comp * N + n];
                    continue;
                }
                const uint16_t h = g[((size_t)comp * Q + i) * N + n];
                float v;
                if (bf) { uint32_t u = (uint32_t)h << 16; std::memcpy(&v, &u, 4); }
                else v = half_to_float(h) * F16_INV_SCALE;
                f[((size_t)comp * Q + i) * N + n] = v + w * (comp ? d[n].y : d[n].x);
            }
        }
    return CF_OK;
}

cf_status cf_total_mass(cf_ctx *c, double m[2]) {
    if (!c || !m) return fail(CF_EINVAL, "null argument");
    CF_CUDA(cudaMemsetAsync(c->dscratch, 0, sizeof(double) * 2, c->stream));
    CF_CUDA(launch_mass(c->f[c->fpar], c->f0[c->fpar], c->d.precision, c->rho[c->fpar], c->N, c->dscratch,
                        c->stream));
    CF_CUDA(cudaMemcpyAsync(m, c->dscratch, sizeof(double) * 2, cudaMemcpyDeviceToHost, c->stream));
    return sync_ok(c);
}

cf_status cf_meniscus_field(cf_ctx *c, double *h) {
    if (!c || !h) return fail(CF_EINVAL, "null argument");
    const int nxy = c->d.nx * c->d.ny;
    if (cf_status si = inside_flags(c); si != CF_OK) return si;
    CF_CUDA(launch_meniscus(c->out, c->inside, c->hscratch, c->d.nx, c->d.ny, c->d.nz, c->d.wall, c->stream));
    std::vector<float> hf(nxy);
    CF_CUDA(cudaMemcpyAsync(hf.data(), c->hscratch, sizeof(float) * nxy, cudaMemcpyDeviceToHost, c->stream));
    cf_status s = sync_ok(c);
    if (s != CF_OK) return s;
    for (int i = 0; i < nxy; ++i) h[i] = hf[i];
    return CF_OK;
}

static size_t profile_samples(const cf_ctx *c, double dr) {
    return (size_t)std::floor((double)(std::min(c->d.nx, c->d.ny) / 2) / dr + 1e-9);
}

cf_status cf_meniscus_profile(cf_ctx *c, int id, double dr, double *r, double *zeta, size_t *inout_n,
                              double *Z) {
    if (!c || !inout_n) return fail(CF_EINVAL, "null argument");
    const int nc = (int)c->caps.size();
    if (id < 0 || id >= nc) return fail(CF_ENOTFOUND, "unknown capsule");
    if (!(dr > 0.0) || !std::isfinite(dr) || dr > std::min(c->d.nx, c->d.ny) / 2)
        return fail(CF_EINVAL, "dr must be positive and at most half the smaller lateral size");
    const size_t nr = profile_samples(c, dr);
    if (*inout_n < nr || !r || !zeta) { *inout_n = nr; return fail(CF_EINVAL, "profile buffer too small"); }
    if (c->pcap < nr + 2) {
        if (c->pscratch) dfree(c, c->pscratch);
        c->pscratch = (double *)dalloc(c, sizeof(double) * (nr + 2));
        if (!c->pscratch) { c->pcap = 0; return fail(CF_ENOMEM, "device allocation failed (profile)"); }
        c->allocations.pop_back();  // freed explicitly
        c->pcap = nr + 2;
    }
    if (cf_status si = inside_flags(c); si != CF_OK) return si;
    CF_CUDA(launch_meniscus(c->out, c->inside, c->hscratch, c->d.nx, c->d.ny, c->d.nz, c->d.wall, c->stream));
    CF_CUDA(launch_meniscus_profile(c->hscratch, c->d.nx, c->d.ny, c->acc, c->capdev, nc, id, dr, (int)nr,
                                    c->pscratch, c->stream));
    std::vector<double> out(nr + 2);
    CF_CUDA(cudaMemcpyAsync(out.data(), c->pscratch, sizeof(double) * out.size(), cudaMemcpyDeviceToHost,
                            c->stream));
    cf_status s = sync_ok(c);
    if (s != CF_OK) return s;
    for (size_t k = 0; k < nr; ++k) {
        r[k] = (double)k * dr;
        zeta[k] = out[k];
    }
    *inout_n = nr;
    if (Z) *Z = out[nr];
    return CF_OK;
}

// ------------------------------------------------ warm start in the library
struct cf_model {
    UNetModel *m = nullptr;
};

extern "C" cf_status cf_model_load(const char *path, cf_model **out) {
    if (!path || !out) return fail(CF_EINVAL, "null argument");
    UNetModel *m = nullptr;
    const cf_status s = unet_load(path, &m);
    if (s != CF_OK) return s;
    *out = new cf_model{m};
    return CF_OK;
}

extern "C" cf_status cf_model_destroy(cf_model *model) {
    if (!model) return CF_OK;
    unet_free(model->m);
    delete model;
    return CF_OK;
}

extern "C" cf_status cf_warmstart(cf_ctx *c, const cf_model *model, const cf_warm_policy *pol, double h_top,
                                  double rmaj, double rmin, double rmix, double kS, const double *jitter, int *used,
                                  long long *steps) {
    if (!c || !model || !pol) return fail(CF_EINVAL, "null argument");
    if (pol->window < 1 || !(pol->grow > 0.0) || !(pol->u_limit > 0.0))
        return fail(CF_EINVAL, "bad warm-start policy (window >= 1, grow > 0, u_limit > 0)");
    if (c->d.nx % 4 || c->d.ny % 4 || c->d.nz % 4) return fail(CF_EINVAL, "the U-net needs lattice sizes divisible by 4");
    const long long N = c->N;
    float *feats = (float *)dalloc(c, sizeof(float) * 4 * (size_t)N);
    float *dens = (float *)dalloc(c, sizeof(float) * 2 * (size_t)N);
    if (!feats || !dens) return fail(CF_ENOMEM, "device allocation failed (warm start)");
    c->allocations.pop_back();
    c->allocations.pop_back();
    auto release = [&]() { dfree(c, feats); dfree(c, dens); };
    cf_status s = cf_warm_features(c, h_top, kS, feats, nullptr);
    if (s == CF_OK) s = unet_forward(model->m, feats, c->d.nz, c->d.ny, c->d.nx, dens, nullptr, c->stream);
    if (s == CF_OK) s = cf_warm_apply(c, h_top, rmaj, rmin, rmix, dens);
    if (s != CF_OK) { release(); return s; }
    // judge the predicted start over two windows: finite, no negative
    // density, velocities below u_limit, and a density change that decays
    double ck[3][4];
    s = cf_step(c, 1);
    if (s == CF_OK) s = cf_field_check(c, ck[0]);
    for (int w = 1; w <= 2 && s == CF_OK; ++w) {
        s = cf_step(c, pol->window);
        if (s == CF_OK) s = cf_field_check(c, ck[w]);
    }
    release();
    if (s != CF_OK && s != CF_EDIVERGED) return s;
    bool ok = s == CF_OK;
    for (int w = 1; w <= 2 && ok; ++w) ok = ck[w][0] == 1.0 && ck[w][1] >= 0.0 && ck[w][2] <= pol->u_limit;
    ok = ok && ck[2][3] <= pol->grow * ck[1][3];
    if (!ok && pol->fallback) {
        s = cf_set_film(c, h_top, rmaj, rmin, rmix, jitter);
        if (s != CF_OK) return s;
    }
    if (used) *used = ok ? 1 : 0;
    if (steps) *steps = 2LL * pol->window + 1;
    return CF_OK;
}

// ------------------------------------------- theory of the capillary force
namespace {
// sum of squared residuals of zeta ~ Q K0(q r) at the best Q for this q
double fit_residual(const std::vector<double> &r, const std::vector<double> &z, double q, double *Qbest) {
    double zk = 0.0, kk = 0.0;
    std::vector<double> k0(r.size());
    for (size_t i = 0; i < r.size(); ++i) {
        k0[i] = std::cyl_bessel_k(0.0, q * r[i]);
        zk += z[i] * k0[i];
        kk += k0[i] * k0[i];
    }
    const double Q = kk > 0.0 ? zk / kk : 0.0;
    double S = 0.0;
    for (size_t i = 0; i < r.size(); ++i) S += (z[i] - Q * k0[i]) * (z[i] - Q * k0[i]);
    if (Qbest) *Qbest = Q;
    return S;
}
}  // namespace

extern "C" cf_status cf_meniscus_fit(const double *r, const double *zeta, size_t n, double rmin, double rmax,
                                     double out[4]) {
    if (!r || !zeta || !out) return fail(CF_EINVAL, "null argument");
    std::vector<double> rr, zz;
    for (size_t i = 0; i < n; ++i)
        if (r[i] > 0.0 && r[i] >= rmin && r[i] <= rmax && std::isfinite(zeta[i])) {
            rr.push_back(r[i]);
            zz.push_back(zeta[i]);
        }
    if (rr.size() < 2) return fail(CF_EINVAL, "fewer than two finite profile samples in [rmin, rmax]");
    // coarse scan of ln q over [ln 1e-3, ln 3], then golden-section refinement
    const int NS = 400;
    const double a0 = std::log(1e-3), a1 = std::log(3.0);
    int best = 0;
    double bestS = HUGE_VAL;
    for (int i = 0; i < NS; ++i) {
        const double S = fit_residual(rr, zz, std::exp(a0 + (a1 - a0) * i / (NS - 1)), nullptr);
        if (S < bestS) { bestS = S; best = i; }
    }
    double lo = a0 + (a1 - a0) * std::max(best - 1, 0) / (NS - 1);
    double hi = a0 + (a1 - a0) * std::min(best + 1, NS - 1) / (NS - 1);
    const double phi = 0.5 * (std::sqrt(5.0) - 1.0);
    double x1 = hi - phi * (hi - lo), x2 = lo + phi * (hi - lo);
    double f1 = fit_residual(rr, zz, std::exp(x1), nullptr), f2 = fit_residual(rr, zz, std::exp(x2), nullptr);
    for (int it = 0; it < 200 && hi - lo > 1e-15; ++it) {
        if (f1 < f2) {
            hi = x2; x2 = x1; f2 = f1;
            x1 = hi - phi * (hi - lo);
            f1 = fit_residual(rr, zz, std::exp(x1), nullptr);
        } else {
            lo = x1; x1 = x2; f1 = f2;
            x2 = lo + phi * (hi - lo);
            f2 = fit_residual(rr, zz, std::exp(x2), nullptr);
        }
    }
    const double q = std::exp(0.5 * (lo + hi));
    double Q = 0.0;
    const double S = fit_residual(rr, zz, q, &Q);
    out[0] = Q;
    out[1] = q;
    out[2] = std::sqrt(S / rr.size());
    out[3] = (double)rr.size();
    return CF_OK;
}

extern "C" cf_status cf_capillary_force(double q, double gamma, double Q1, double Q2, double L, double *F) {
    if (!F) return fail(CF_EINVAL, "null argument");
    if (!(q > 0.0) || !(L > 0.0)) return fail(CF_EINVAL, "q and L must be positive");
    const double pi = 3.14159265358979323846;
    *F = -2.0 * pi * q * gamma * Q1 * Q2 * std::cyl_bessel_k(1.0, q * L);
    return CF_OK;
}

// ------------------------------------------------------------ checkpoints
namespace {
struct CkptHeader {
    char magic[8];  // "CFCKPT01"
    uint32_t version;
    int32_t nx, ny, nz, wall, precision;
    int32_t ncaps, nnodes, nfaces, capacity;
    int32_t fpar, xpar, lpar, ftpar;
    int32_t count;  // entries of the current cut-link list
    int64_t steps_done;
    double dry_dm;
};
constexpr uint32_t CKPT_VERSION = 2;  // 2: element momentum exchange in fixed point

// the device arrays of the state between two steps, in file order
struct CkptPart {
    void *dev;
    size_t bytes;
};
std::vector<CkptPart> ckpt_parts(cf_ctx *c, int count) {
    const long long N = c->N;
    std::vector<CkptPart> v;
    v.push_back({c->f[c->fpar], pop_bytes(c->d.precision) * 38 * (size_t)N});
    if (c->d.precision != CF_FP32) v.push_back({c->f0[c->fpar], sizeof(float) * 2 * (size_t)N});
    v.push_back({c->rho[c->fpar], sizeof(float2) * (size_t)N});
    v.push_back({c->out, sizeof(float) * 5 * (size_t)N});
    v.push_back({c->step_ctr, sizeof(unsigned)});
    if (c->nnodes > 0) {
        const size_t nv = c->nnodes, nf = c->nfaces, nc = c->caps.size();
        v.push_back({c->X[c->xpar], sizeof(float) * 6 * nv});
        v.push_back({c->V, sizeof(float) * 3 * nv});
        v.push_back({c->FT[0], sizeof(long long) * 3 * nf});
        v.push_back({c->FT[1], sizeof(long long) * 3 * nf});
        v.push_back({c->uT, sizeof(float4) * nf});
        v.push_back({c->acc, sizeof(double) * A_NACC * nc});
        v.push_back({c->bbox[0], sizeof(int) * 6 * nc});
        v.push_back({c->bbox[1], sizeof(int) * 6 * nc});
        v.push_back({c->mask, sizeof(uint32_t) * (size_t)N});
        v.push_back({c->tri, sizeof(int) * 18 * (size_t)N});
        v.push_back({c->list[c->lpar], sizeof(int2) * (size_t)count});
    }
    return v;
}
}  // namespace

cf_status cf_save(cf_ctx *c, const char *path) {
    if (!c || !path) return fail(CF_EINVAL, "null argument");
    if (!c->film_set) return fail(CF_ESTATE, "nothing to save before cf_set_film");
    cf_status s = refresh_cuts(c);  // the checkpoint holds the cut links of its positions
    if (s == CF_OK) s = sync_ok(c);
    if (s != CF_OK) return s;
    CkptHeader h{};
    std::memcpy(h.magic, "CFCKPT01", 8);
    h.version = CKPT_VERSION;
    h.nx = c->d.nx; h.ny = c->d.ny; h.nz = c->d.nz; h.wall = c->d.wall; h.precision = c->d.precision;
    h.ncaps = (int)c->caps.size(); h.nnodes = c->nnodes; h.nfaces = c->nfaces; h.capacity = c->capacity;
    h.fpar = c->fpar; h.xpar = c->xpar; h.lpar = c->lpar; h.ftpar = c->ftpar;
    h.steps_done = c->steps_done;
    h.dry_dm = c->dry_dm;
    int count = 0;
    if (c->nnodes > 0) CF_CUDA(cudaMemcpy(&count, c->counts + c->lpar, sizeof(int), cudaMemcpyDeviceToHost));
    h.count = count;
    FILE *fp = std::fopen(path, "wb");
    if (!fp) return fail(CF_EINVAL, std::string("cannot open for writing: ") + path);
    bool ok = std::fwrite(&h, sizeof h, 1, fp) == 1;
    std::vector<char> buf;
    for (const CkptPart &part : ckpt_parts(c, count)) {
        if (!ok) break;
        buf.resize(part.bytes);
        if (cudaMemcpy(buf.data(), part.dev, part.bytes, cudaMemcpyDeviceToHost) != cudaSuccess) {
            std::fclose(fp);
            return fail(CF_ECUDA, "device copy failed while saving");
        }
        ok = std::fwrite(buf.data(), 1, part.bytes, fp) == part.bytes;
    }
    ok = (std::fclose(fp) == 0) && ok;
    if (!ok) return fail(CF_EINVAL, std::string("write failed: ") + path);
    return CF_OK;
}

cf_status cf_load(cf_ctx *c, const char *path) {
    if (!c || !path) return fail(CF_EINVAL, "null argument");
    FILE *fp = std::fopen(path, "rb");
    if (!fp) return fail(CF_EINVAL, std::string("cannot open: ") + path);
    CkptHeader h{};
    if (std::fread(&h, sizeof h, 1, fp) != 1 || std::memcmp(h.magic, "CFCKPT01", 8) != 0 ||
        h.version != CKPT_VERSION) {
        std::fclose(fp);
        return fail(CF_EINVAL, "not a checkpoint of this version");
    }
    if (h.nx != c->d.nx || h.ny != c->d.ny || h.nz != c->d.nz || h.wall != c->d.wall ||
        h.precision != c->d.precision || h.ncaps != (int)c->caps.size() || h.nnodes != c->nnodes ||
        h.nfaces != c->nfaces || h.capacity != c->capacity || h.count < 0 || h.count > c->capacity ||
        (h.fpar | h.xpar | h.lpar | h.ftpar) & ~1) {
        std::fclose(fp);
        return fail(CF_EINVAL, "checkpoint does not match this context (lattice, precision or capsules)");
    }
    cf_status s = sync_ok(c);
    if (s != CF_OK) { std::fclose(fp); return s; }
    c->fpar = h.fpar; c->xpar = h.xpar; c->lpar = h.lpar; c->ftpar = h.ftpar;
    std::vector<char> buf;
    for (const CkptPart &part : ckpt_parts(c, h.count)) {
        buf.resize(part.bytes);
        if (std::fread(buf.data(), 1, part.bytes, fp) != part.bytes) {
            std::fclose(fp);
            c->film_set = false;  // partly loaded: unusable until set up again
            return fail(CF_EINVAL, "checkpoint is truncated");
        }
        if (cudaMemcpy(part.dev, buf.data(), part.bytes, cudaMemcpyHostToDevice) != cudaSuccess) {
            std::fclose(fp);
            c->film_set = false;
            return fail(CF_ECUDA, "device copy failed while loading");
        }
    }
    std::fclose(fp);
    if (c->nnodes > 0) CF_CUDA(cudaMemcpy(c->counts + c->lpar, &h.count, sizeof(int), cudaMemcpyHostToDevice));
    c->steps_done = h.steps_done;
    c->film_set = true;
    drop_graphs(c);
    return cf_remove_mass(c, h.dry_dm);
}

cf_status cf_meniscus_height(cf_ctx *c, int id, double *Z) {
    if (!c || !Z) return fail(CF_EINVAL, "null argument");
    size_t n = profile_samples(c, 1.0);
    std::vector<double> r(std::max<size_t>(n, 1)), zeta(std::max<size_t>(n, 1));
    return cf_meniscus_profile(c, id, 1.0, r.data(), zeta.data(), &n, Z);
}

cf_status cf_cuts(cf_ctx *c, uint32_t *mask, int *tri, uint8_t *inside) {
    if (!c) return fail(CF_EINVAL, "null context");
    if (cf_status si = refresh_cuts(c); si != CF_OK) return si;
    const long long N = c->N;
    if (mask) CF_CUDA(cudaMemcpyAsync(mask, c->mask, sizeof(uint32_t) * N, cudaMemcpyDeviceToHost, c->stream));
    if (tri) CF_CUDA(cudaMemcpyAsync(tri, c->tri, sizeof(int) * 18 * N, cudaMemcpyDeviceToHost, c->stream));
    if (inside) {
        CF_CUDA(launch_inside(c->mask, c->inside, c->d.nx, c->d.ny, c->d.nz, c->stream));
        CF_CUDA(cudaMemcpyAsync(inside, c->inside, N, cudaMemcpyDeviceToHost, c->stream));
    }
    cf_status s = sync_ok(c);
    if (s != CF_OK) return s;
    if (tri)
        for (long long i = 0; i < 18 * N; ++i)
            if (tri[i] >= c->nfaces || tri[i] < 0) tri[i] = -1;
    return CF_OK;
}

}  // extern "C"

// ----------------------------------------------------------------- batches
// A batch steps many contexts together: their membrane halves run as
// parallel branches, their lattice passes as one persistent launch per pass.
// With groups > 1 the contexts are split into groups of about equal node
// count, each with its own lattice launches on a stream branch of its own,
// so that the membrane phases of one group overlap the lattice passes of
// another.
constexpr int CF_MAX_GROUPS = 8;
struct cf_batch {
    std::vector<cf_ctx *> ctx;
    int prec = 0;
    cudaStream_t stream = nullptr;
    cudaEvent_t ev_fork = nullptr;
    int tile = 1, zchunk = 4;     // tile shape index and contiguous planes per work item
    int groups = 1;               // pipeline groups
    int4 *work = nullptr;          // device work list of all lattices (one launch)
    int nwork = 0;
    std::vector<int> zstride;      // per lattice
    std::vector<int> gbeg;                 // [groups + 1] context ranges of the groups
    std::vector<cudaStream_t> gstream;     // [CF_MAX_GROUPS] stream branch per group
    std::vector<cudaEvent_t> gev;          // [CF_MAX_GROUPS] after the group's lattice passes
    std::vector<cudaStream_t> gmem;        // [CF_MAX_GROUPS] the group's position-only membrane kernels
    std::vector<cudaEvent_t> gfork, gjoin; // [CF_MAX_GROUPS] around them
    std::vector<int4 *> gwork;             // per group: work list (lattice index within the group)
    std::vector<int> gnwork;
    cudaGraphExec_t graph = nullptr;      // a captured step pair of all groups
    cudaGraphExec_t graph_out = nullptr;  // the same, its second step also recording the fields
    std::vector<int> graph_key;    // parities of all contexts at capture
    int graph_launches = 0;
    long long launches_last = 0;
};

namespace {

// the captured step pairs are stale (the layout or the parities changed)
void batch_drop_graphs(cf_batch *b) {
    if (b->graph) cudaGraphExecDestroy(b->graph);
    if (b->graph_out) cudaGraphExecDestroy(b->graph_out);
    b->graph = b->graph_out = nullptr;
    b->graph_key.clear();
}

// work items (lattice index - base, x tile, y tile, z slice) of contexts [i0, i1)
void batch_items(cf_batch *b, size_t i0, size_t i1, int base, std::vector<int4> &w) {
    int tx, ty;
    lb_batch_tile(b->tile, &tx, &ty);
    for (size_t i = i0; i < i1; ++i) {
        const cf_ctx *c = b->ctx[i];
        for (int zs = 0; zs < b->zstride[i]; ++zs)
            for (int ty_ = 0; ty_ < (c->d.ny + ty - 1) / ty; ++ty_)
                for (int tx_ = 0; tx_ < (c->d.nx + tx - 1) / tx; ++tx_)
                    w.push_back(make_int4((int)i - base, tx_, ty_, zs));
    }
}

cf_status upload_work(const std::vector<int4> &w, int4 **dev) {
    if (*dev) cudaFree(*dev);
    *dev = nullptr;
    CF_CUDA(cudaMalloc(dev, sizeof(int4) * std::max<size_t>(w.size(), 1)));
    CF_CUDA(cudaMemcpy(*dev, w.data(), sizeof(int4) * w.size(), cudaMemcpyHostToDevice));
    return CF_OK;
}

cf_status batch_build_work(cf_batch *b) {
    const size_t n = b->ctx.size();
    b->zstride.assign(n, 1);
    for (size_t i = 0; i < n; ++i) {
        const cf_ctx *c = b->ctx[i];
        const int nzf = c->d.nz - (c->d.wall ? 1 : 0);
        b->zstride[i] = std::max(1, (nzf + b->zchunk - 1) / b->zchunk);
    }
    std::vector<int4> w;
    batch_items(b, 0, n, 0, w);
    cf_status s = upload_work(w, &b->work);
    if (s != CF_OK) return s;
    b->nwork = (int)w.size();
    // groups: G contiguous context ranges, each non-empty, boundary k placed
    // where the node count before it is nearest to k / G of the total
    const int G = std::max(1, std::min(b->groups, (int)n));
    std::vector<long long> cum(n + 1, 0);
    for (size_t i = 0; i < n; ++i) cum[i + 1] = cum[i] + b->ctx[i]->N;
    b->gbeg.assign(1, 0);
    for (int k = 1; k < G; ++k) {
        const int lo = b->gbeg.back() + 1, hi = (int)n - (G - k);
        int bi = lo;
        for (int i = lo; i <= hi; ++i)
            if (std::llabs(cum[i] * G - cum[n] * k) < std::llabs(cum[bi] * G - cum[n] * k)) bi = i;
        b->gbeg.push_back(bi);
    }
    b->gbeg.push_back((int)n);
    const int ng = (int)b->gbeg.size() - 1;
    b->gnwork.assign(ng, 0);
    if (b->gwork.size() < (size_t)ng) b->gwork.resize(ng, nullptr);
    for (int g = 0; g < ng; ++g) {
        std::vector<int4> wg;
        batch_items(b, b->gbeg[g], b->gbeg[g + 1], b->gbeg[g], wg);
        s = upload_work(wg, &b->gwork[g]);
        if (s != CF_OK) return s;
        b->gnwork[g] = (int)wg.size();
    }
    batch_drop_graphs(b);
    return CF_OK;
}

// The membrane and cut-link kernels of contexts [i0, i1) as one launch per
// kernel (per 64 contexts).  Before the lattice passes: the position-only
// membrane kernels fork onto the group's membrane stream `sm` (joined by the
// node update), the bounce records go on the lattice stream `s`.
cf_status batch_pre(cf_batch *b, int g, int i0, int i1, cudaStream_t s, int *nl) {
    static SparseTab<MemParams> tv, tf;  // copied into each launch
    static SparseTab<PrepParams> tp;
    std::vector<cf_ctx *> mem;
    for (int i = i0; i < i1; ++i)
        if (b->ctx[i]->nnodes > 0) mem.push_back(b->ctx[i]);
    CF_CUDA(cudaEventRecord(b->gfork[g], s));
    CF_CUDA(cudaStreamWaitEvent(b->gmem[g], b->gfork[g], 0));
    // bounce-record blocks per context: about four per SM over the group
    const int pb = std::max(4, std::min(304, (int)((4 * 152 + mem.size() - 1) / std::max<size_t>(mem.size(), 1))));
    for (size_t j0 = 0; j0 < mem.size(); j0 += CF_SPARSE_CAP) {
        const int n = (int)std::min<size_t>(CF_SPARSE_CAP, mem.size() - j0);
        tv.n = tf.n = tp.n = n;
        tv.boff[0] = tf.boff[0] = tp.boff[0] = 0;
        for (int j = 0; j < n; ++j) {
            cf_ctx *c = mem[j0 + j];
            tv.p[j] = tf.p[j] = mem_params(c);
            tv.boff[j + 1] = tv.boff[j] + c->nslots / CF_MEM_NODE_BLOCK;  // one warp per patch
            tf.boff[j + 1] = tf.boff[j] + (c->nfaces + CF_MEM_FACE_BLOCK - 1) / CF_MEM_FACE_BLOCK;
            tp.p[j] = prep_params(c, pb);
            tp.boff[j + 1] = tp.boff[j] + pb;
        }
        for (int j = 0; j < n; ++j) {  // lattices with many capsules: their contact partners first
            cf_ctx *c = mem[j0 + j];
            if (!c->nbr) continue;
            MemParams q = mem_params(c);
            q.nbr = nullptr;
            CF_CUDA(launch_contact_partners(q, c->nbr, c->nbr_cnt, b->gmem[g], nl));
        }
        CF_CUDA(launch_membrane_forces_batch(tv, tf, b->gmem[g], nl));
        CF_CUDA(launch_prep_batch(tp, s, nl));
    }
    CF_CUDA(cudaEventRecord(b->gjoin[g], b->gmem[g]));
    return CF_OK;
}

// After the lattice passes of contexts [i0, i1) (whose populations are now in
// f[fpar]): node update with the reset of the old cut structure, then the cut
// links of the new positions (fixed capsules: only the next step's exchange
// accumulator is zeroed).
cf_status batch_post(cf_batch *b, int g, int i0, int i1, cudaStream_t s, int *nl) {
    static SparseTab<UpdateParams> tu;
    static SparseTab<MemParams> tz;
    static SparseTab<CutParams> tc;
    std::vector<cf_ctx *> mem;
    for (int i = i0; i < i1; ++i)
        if (b->ctx[i]->nnodes > 0) mem.push_back(b->ctx[i]);
    CF_CUDA(cudaStreamWaitEvent(s, b->gjoin[g], 0));
    const int cb = 32;  // reset blocks per context
    for (size_t j0 = 0; j0 < mem.size(); j0 += CF_SPARSE_CAP) {
        const int n = (int)std::min<size_t>(CF_SPARSE_CAP, mem.size() - j0);
        tu.n = n;
        tz.n = 0;
        tu.boff[0] = tz.boff[0] = 0;
        for (int j = 0; j < n; ++j) {
            cf_ctx *c = mem[j0 + j];
            tu.p[j].m = mem_params(c);
            tu.p[j].c = clear_params(c, cb);
            const int nb = (c->nnodes + CF_MEM_NODE_BLOCK - 1) / CF_MEM_NODE_BLOCK;
            tu.boff[j + 1] = tu.boff[j] + nb + tu.p[j].c.blocks;
            if (c->any_frozen) {
                tz.p[tz.n] = tu.p[j].m;
                tz.boff[tz.n + 1] = tz.boff[tz.n] + nb;
                ++tz.n;
            }
        }
        CF_CUDA(launch_membrane_update_batch(tu, tz.n ? &tz : nullptr, s, nl));
    }
    for (cf_ctx *c : mem) c->xpar = 1 - c->xpar;
    for (size_t j0 = 0; j0 < mem.size(); j0 += CF_SPARSE_CAP) {
        const int n = (int)std::min<size_t>(CF_SPARSE_CAP, mem.size() - j0);
        long long faces = 0;
        for (int j = 0; j < n; ++j) faces += mem[j0 + j]->nfaces;
        const int lanes = cut_lanes(faces);
        tc.n = n;
        tc.boff[0] = 0;
        for (int j = 0; j < n; ++j) {
            cf_ctx *c = mem[j0 + j];
            if (!c->all_fixed) {
                tc.p[j] = cut_params(c, c->X[c->xpar]);  // entry counter zeroed by the update
                c->lpar = 1 - c->lpar;
            } else {
                tc.p[j] = CutParams{};
                tc.p[j].nfaces = c->nfaces;
                tc.p[j].FTnext = c->FT[1 - c->ftpar];
                tc.p[j].zero_only = 1;
            }
            tc.boff[j + 1] = tc.boff[j] + cut_blocks(c->nfaces, lanes);
        }
        CF_CUDA(launch_cuts_batch(tc, lanes, s, nl));
    }
    for (cf_ctx *c : mem) c->ftpar = 1 - c->ftpar;
    return CF_OK;
}

// one step with the contexts in pipeline groups (see cf_batch)
cf_status batch_enqueue_groups(cf_batch *b, bool with_out, int *nl) {
    CF_CUDA(cudaEventRecord(b->ev_fork, b->stream));
    const int ng = (int)b->gbeg.size() - 1;
    static BatchTab tab;  // copied into each launch
    for (int g = 0; g < ng; ++g) {
        cudaStream_t gs = b->gstream[g];
        CF_CUDA(cudaStreamWaitEvent(gs, b->ev_fork, 0));
        cf_status s = batch_pre(b, g, b->gbeg[g], b->gbeg[g + 1], gs, nl);
        if (s != CF_OK) return s;
        for (int i = b->gbeg[g]; i < b->gbeg[g + 1]; ++i) {
            LBParams &l = tab.lat[i - b->gbeg[g]];
            l = lb_params(b->ctx[i], with_out);
            l.zstride = b->zstride[i];
            l.zchunk = b->zchunk;
        }
        CF_CUDA(launch_lb_batch(tab, b->gbeg[g + 1] - b->gbeg[g], b->gwork[g], b->gnwork[g], b->prec, b->tile, gs));
        *nl += 2;
        for (int i = b->gbeg[g]; i < b->gbeg[g + 1]; ++i) b->ctx[i]->fpar = 1 - b->ctx[i]->fpar;
        s = batch_post(b, g, b->gbeg[g], b->gbeg[g + 1], gs, nl);
        if (s != CF_OK) return s;
        CF_CUDA(cudaEventRecord(b->gev[g], gs));
        CF_CUDA(cudaStreamWaitEvent(b->stream, b->gev[g], 0));
    }
    return CF_OK;
}

// one step of every context of the batch, enqueued on the batch stream; ev,
// when given, receives four events on the batch stream: ev[0] step start,
// ev[1] before and ev[2] after the lattice passes, ev[3] step end (the
// lattice passes of all contexts then run as one launch per pass, whatever
// the group setting)
cf_status batch_enqueue_step(cf_batch *b, bool with_out, int *nl, cudaEvent_t *ev = nullptr) {
    if (!ev && b->gbeg.size() > 2) return batch_enqueue_groups(b, with_out, nl);
    if (ev) CF_CUDA(cudaEventRecord(ev[0], b->stream));
    const int n = (int)b->ctx.size();
    cf_status s = batch_pre(b, 0, 0, n, b->stream, nl);
    if (s != CF_OK) return s;
    static BatchTab tab;  // copied into the launch
    for (size_t i = 0; i < b->ctx.size(); ++i) {
        tab.lat[i] = lb_params(b->ctx[i], with_out);
        tab.lat[i].zstride = b->zstride[i];
        tab.lat[i].zchunk = b->zchunk;  // contiguous planes per work item
    }
    if (ev) CF_CUDA(cudaEventRecord(ev[1], b->stream));
    CF_CUDA(launch_lb_batch(tab, (int)b->ctx.size(), b->work, b->nwork, b->prec, b->tile, b->stream));
    *nl += 2;
    if (ev) CF_CUDA(cudaEventRecord(ev[2], b->stream));
    for (cf_ctx *c : b->ctx) c->fpar = 1 - c->fpar;
    s = batch_post(b, 0, 0, n, b->stream, nl);
    if (s != CF_OK) return s;
    if (ev) CF_CUDA(cudaEventRecord(ev[3], b->stream));
    return CF_OK;
}

std::vector<int> batch_key(const cf_batch *b) {
    std::vector<int> k;
    for (const cf_ctx *c : b->ctx) k.push_back(c->fpar | (c->xpar << 1) | (c->lpar << 2) | (c->ftpar << 3));
    return k;
}

// the captured two-step graph for the contexts' current parities
// The captured step pair of the contexts' current parities (out: its second
// step also records the fields); captured on first use, both dropped when the
// parities or the layout change.
cf_status batch_graph(cf_batch *b, bool out = false) {
    const std::vector<int> key = batch_key(b);
    if (b->graph_key != key) batch_drop_graphs(b);
    cudaGraphExec_t &slot = out ? b->graph_out : b->graph;
    if (!slot) {
        cudaGraph_t g;
        CF_CUDA(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
        int nlg = 0;
        cf_status s1 = batch_enqueue_step(b, false, &nlg);
        cf_status s2 = s1 == CF_OK ? batch_enqueue_step(b, out, &nlg) : s1;
        cudaError_t e = cudaStreamEndCapture(b->stream, &g);
        if (s2 != CF_OK) return s2;
        if (e != cudaSuccess) return fail(CF_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e));
        e = cudaGraphInstantiate(&slot, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return fail(CF_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
        b->graph_key = key;
        b->graph_launches = nlg;
    }
    return CF_OK;
}

// work a context still has in flight on its own stream comes first (the batch
// step runs all of its kernels on the batch's streams)
cf_status batch_join_contexts(cf_batch *b) {
    for (cf_ctx *c : b->ctx) {
        CF_CUDA(cudaEventRecord(c->ev_batch, c->stream));
        CF_CUDA(cudaStreamWaitEvent(b->stream, c->ev_batch, 0));
    }
    return CF_OK;
}

// pairs graph replays (2 * pairs steps; the fields readout is not refreshed)
cf_status batch_replay(cf_batch *b, int pairs) {
    cf_status s = batch_join_contexts(b);
    if (s != CF_OK) return s;
    s = batch_graph(b);
    if (s != CF_OK) return s;
    for (int k = 0; k < pairs; ++k) CF_CUDA(cudaGraphLaunch(b->graph, b->stream));
    for (cf_ctx *c : b->ctx) c->steps_done += 2 * pairs;
    b->launches_last = (long long)pairs * b->graph_launches;
    return CF_OK;
}

cf_status batch_run(cf_batch *b, long long n) {
    for (cf_ctx *c : b->ctx)
        if (c->dry_dm > 0.0) return fail(CF_ESTATE, "drying (cf_remove_mass) is not available in a batch");
    // as cf_step: captured step pairs, the last step recording the fields
    int nl = 0;
    cf_status sj = batch_join_contexts(b);
    if (sj != CF_OK) return sj;
    long long left = n;
    if (left >= 4 && b->graph && b->graph_key != batch_key(b)) {
        // one plain step brings every context to the captured graphs' parity
        cf_status s = batch_enqueue_step(b, false, &nl);
        if (s != CF_OK) return s;
        --left;
    }
    if (left >= 3) {
        const bool odd = (left & 1) != 0;
        const long long pairs = left / 2;
        for (long long k = 0; k < pairs; ++k) {
            const bool out = !odd && k == pairs - 1;
            cf_status s = batch_graph(b, out);
            if (s != CF_OK) return s;
            CF_CUDA(cudaGraphLaunch(out ? b->graph_out : b->graph, b->stream));
            nl += b->graph_launches;
        }
        left -= 2 * pairs;
    }
    while (left > 0) {
        cf_status s = batch_enqueue_step(b, left == 1, &nl);
        if (s != CF_OK) return s;
        --left;
    }
    for (cf_ctx *c : b->ctx) c->steps_done += n;
    b->launches_last = nl;
    return CF_OK;
}

cf_status batch_sync(cf_batch *b) {
    CF_CUDA(cudaStreamSynchronize(b->stream));
    for (cf_ctx *c : b->ctx) {
        cf_status s = sync_ok(c);
        if (s != CF_OK) return s;
    }
    return CF_OK;
}

}  // namespace

extern "C" {

cf_status cf_batch_create(cf_ctx *const *ctxs, int n, cf_batch **out) {
    if (!ctxs || !out || n <= 0) return fail(CF_EINVAL, "bad argument");
    if (n > CF_BATCH_MAX)
        return fail(CF_EINVAL, "at most " + std::to_string(CF_BATCH_MAX) + " contexts per batch");
    for (int i = 0; i < n; ++i) {
        if (!ctxs[i]) return fail(CF_EINVAL, "null context in batch");
        if (!ctxs[i]->film_set) return fail(CF_ESTATE, "cf_set_film must come before cf_batch_create");
        if (ctxs[i]->fibm) return fail(CF_EINVAL, "the diffuse-interface coupling (CF_IBM) is not available in a batch");
        if (ctxs[i]->d.precision != ctxs[0]->d.precision)
            return fail(CF_EINVAL, "all contexts of a batch need the same precision");
        for (int j = 0; j < i; ++j)
            if (ctxs[j] == ctxs[i]) return fail(CF_EINVAL, "a context appears twice in the batch");
    }
    cf_batch *b = new cf_batch();
    b->ctx.assign(ctxs, ctxs + n);
    b->prec = ctxs[0]->d.precision;
    b->gstream.assign(CF_MAX_GROUPS, nullptr);
    b->gev.assign(CF_MAX_GROUPS, nullptr);
    b->gmem.assign(CF_MAX_GROUPS, nullptr);
    b->gfork.assign(CF_MAX_GROUPS, nullptr);
    b->gjoin.assign(CF_MAX_GROUPS, nullptr);
    bool ok = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) == cudaSuccess &&
              cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming) == cudaSuccess;
    for (int g = 0; ok && g < CF_MAX_GROUPS; ++g)
        ok = cudaStreamCreateWithFlags(&b->gstream[g], cudaStreamNonBlocking) == cudaSuccess &&
             cudaEventCreateWithFlags(&b->gev[g], cudaEventDisableTiming) == cudaSuccess &&
             cudaStreamCreateWithFlags(&b->gmem[g], cudaStreamNonBlocking) == cudaSuccess &&
             cudaEventCreateWithFlags(&b->gfork[g], cudaEventDisableTiming) == cudaSuccess &&
             cudaEventCreateWithFlags(&b->gjoin[g], cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
        cf_batch_destroy(b);
        return fail(CF_ECUDA, "stream / event creation failed");
    }
    // every context's pending work completes before the first batch step
    for (cf_ctx *c : b->ctx) {
        cf_status s = sync_ok(c);
        if (s != CF_OK) { cf_batch_destroy(b); return s; }
    }
    cf_status s = batch_build_work(b);
    if (s != CF_OK) { cf_batch_destroy(b); return s; }
    *out = b;
    return CF_OK;
}

cf_status cf_batch_destroy(cf_batch *b) {
    if (!b) return CF_OK;
    if (b->stream) cudaStreamSynchronize(b->stream);
    batch_drop_graphs(b);
    if (b->work) cudaFree(b->work);
    for (int4 *w : b->gwork)
        if (w) cudaFree(w);
    for (cudaStream_t gs : b->gstream)
        if (gs) cudaStreamDestroy(gs);
    for (cudaStream_t gs : b->gmem)
        if (gs) cudaStreamDestroy(gs);
    for (cudaEvent_t e : b->gev)
        if (e) cudaEventDestroy(e);
    for (cudaEvent_t e : b->gfork)
        if (e) cudaEventDestroy(e);
    for (cudaEvent_t e : b->gjoin)
        if (e) cudaEventDestroy(e);
    if (b->ev_fork) cudaEventDestroy(b->ev_fork);
    if (b->stream) cudaStreamDestroy(b->stream);
    delete b;
    return CF_OK;
}

cf_status cf_batch_set_config(cf_batch *b, int tile, int zchunk) {
    if (!b || tile < 0 || tile >= CF_NTILES || zchunk < 1) return fail(CF_EINVAL, "bad argument");
    CF_CUDA(cudaStreamSynchronize(b->stream));
    b->tile = tile;
    b->zchunk = zchunk;
    return batch_build_work(b);
}

cf_status cf_batch_set_groups(cf_batch *b, int groups) {
    if (!b || groups < 1 || groups > CF_MAX_GROUPS) return fail(CF_EINVAL, "bad argument");
    CF_CUDA(cudaStreamSynchronize(b->stream));
    b->groups = groups;
    return batch_build_work(b);
}

cf_status cf_batch_config(const cf_batch *b, int *tile, int *tile_x, int *tile_y, int *zchunk, int *groups) {
    if (!b) return fail(CF_EINVAL, "null batch");
    int tx, ty;
    lb_batch_tile(b->tile, &tx, &ty);
    if (tile) *tile = b->tile;
    if (tile_x) *tile_x = tx;
    if (tile_y) *tile_y = ty;
    if (zchunk) *zchunk = b->zchunk;
    if (groups) *groups = (int)b->gbeg.size() - 1;
    return CF_OK;
}

cf_status cf_batch_step(cf_batch *b, long long n) {
    if (!b) return fail(CF_EINVAL, "null batch");
    if (n < 0) return fail(CF_EINVAL, "negative step count");
    if (n == 0) return CF_OK;
    cf_status s = batch_run(b, n);
    if (s != CF_OK) return s;
    return batch_sync(b);
}

cf_status cf_batch_time(cf_batch *b, long long n, double *ms) {
    if (!b || !ms || n <= 0) return fail(CF_EINVAL, "bad argument");
    cudaEvent_t e0, e1;
    CF_CUDA(cudaEventCreate(&e0));
    CF_CUDA(cudaEventCreate(&e1));
    CF_CUDA(cudaEventRecord(e0, b->stream));
    cf_status s = batch_run(b, n);
    CF_CUDA(cudaEventRecord(e1, b->stream));
    CF_CUDA(cudaEventSynchronize(e1));
    float t = 0.f;
    CF_CUDA(cudaEventElapsedTime(&t, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (s != CF_OK) return s;
    *ms = t;
    return batch_sync(b);
}

cf_status cf_batch_time_phases(cf_batch *b, long long n, double ms[3]) {
    if (!b || !ms || n <= 0) return fail(CF_EINVAL, "bad argument");
    for (cf_ctx *c : b->ctx)
        if (c->dry_dm > 0.0) return fail(CF_ESTATE, "drying (cf_remove_mass) is not available in a batch");
    std::vector<cudaEvent_t> ev(4 * (size_t)n);
    for (auto &e : ev) CF_CUDA(cudaEventCreate(&e));
    int nl = 0;
    cf_status st = batch_join_contexts(b);
    for (long long k = 0; k < n && st == CF_OK; ++k) st = batch_enqueue_step(b, k == n - 1, &nl, &ev[4 * k]);
    CF_CUDA(cudaStreamSynchronize(b->stream));
    ms[0] = ms[1] = ms[2] = 0.0;
    for (long long k = 0; k < n && st == CF_OK; ++k) {
        float t = 0.f;
        CF_CUDA(cudaEventElapsedTime(&t, ev[4 * k + 1], ev[4 * k + 2]));
        ms[0] += t / n;
        CF_CUDA(cudaEventElapsedTime(&t, ev[4 * k], ev[4 * k + 1]));
        ms[1] += t / n;
        CF_CUDA(cudaEventElapsedTime(&t, ev[4 * k + 2], ev[4 * k + 3]));
        ms[2] += t / n;
    }
    for (auto &e : ev) cudaEventDestroy(e);
    if (st != CF_OK) return st;
    for (cf_ctx *c : b->ctx) c->steps_done += n;
    b->launches_last = nl;
    return batch_sync(b);
}

cf_status cf_batch_autotune(cf_batch *b, int steps, int *tile_out, int *zchunk_out, int *groups_out,
                            double *ms_out) {
    if (!b || steps < 2) return fail(CF_EINVAL, "bad argument");
    const int zcs[3] = {2, 4, 8};
    const int gs[4] = {1, 2, 4, 8};
    const int pairs = (steps + 1) / 2;
    double best = 1e300;
    int bt = b->tile, bz = b->zchunk, bg = b->groups;
    cudaEvent_t e0, e1;
    CF_CUDA(cudaEventCreate(&e0));
    CF_CUDA(cudaEventCreate(&e1));
    // one configuration: capture and one untimed replay, then `pairs` timed replays
    auto trial = [&](int t, int zc, int g, float *ms) -> cf_status {
        b->groups = g;
        cf_status st = cf_batch_set_config(b, t, zc);
        if (st == CF_OK) st = batch_replay(b, 1);
        if (st != CF_OK) return st;
        CF_CUDA(cudaEventRecord(e0, b->stream));
        st = batch_replay(b, pairs);
        if (st != CF_OK) return st;
        CF_CUDA(cudaEventRecord(e1, b->stream));
        CF_CUDA(cudaEventSynchronize(e1));
        CF_CUDA(cudaEventElapsedTime(ms, e0, e1));
        return CF_OK;
    };
    cf_status s = CF_OK;
    // the launch shape of the lattice passes with one group, then the groups
    for (int t = 0; t < CF_NTILES && s == CF_OK; ++t)
        for (int zc : zcs) {
            float ms = 0.f;
            s = trial(t, zc, 1, &ms);
            if (s != CF_OK) break;
            if (ms < best) { best = ms; bt = t; bz = zc; bg = 1; }
        }
    for (int g : gs) {
        if (s != CF_OK || g == 1 || g > (int)b->ctx.size()) continue;
        float ms = 0.f;
        s = trial(bt, bz, g, &ms);
        if (s == CF_OK && ms < best) { best = ms; bg = g; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (s == CF_OK) s = batch_sync(b);
    if (s != CF_OK) return s;
    b->groups = bg;
    s = cf_batch_set_config(b, bt, bz);
    if (s != CF_OK) return s;
    if (tile_out) *tile_out = bt;
    if (zchunk_out) *zchunk_out = bz;
    if (groups_out) *groups_out = (int)b->gbeg.size() - 1;
    if (ms_out) *ms_out = best / (2 * pairs);
    return CF_OK;
}

cf_status cf_batch_lateral_forces(cf_batch *b, int a, int bb, double *F) {
    if (!b || !F) return fail(CF_EINVAL, "null argument");
    for (size_t i = 0; i < b->ctx.size(); ++i) {
        cf_status s = cf_lateral_force(b->ctx[i], a, bb, F + i);
        if (s != CF_OK) return s;
    }
    return CF_OK;
}

cf_status cf_batch_launch_count(const cf_batch *b, long long *n) {
    if (!b || !n) return fail(CF_EINVAL, "null argument");
    *n = b->launches_last;
    return CF_OK;
}

}  // extern "C"
