// Membrane phase of the coupled step and cut-link geometry (sm_103a).
//
// All capsules are concatenated: global node and element indices, with the
// owning capsule per element and per node.  The membrane phase of one step
// (Sec. 3.1, Eqs. 6-9, 11) is five kernels, one thread per element or node of
// all capsules:
//   1. k_mem_elements  per element: Skalak strain forces (Eq. 6), volume
//      gradient terms (Eq. 8), cotangent-Laplacian contributions of the
//      bending energy; FP64 area and volume
//   2. k_mem_nodes     per node: mean-curvature vector and node area, gradients
//      of the bending energy with respect to them; FP64 centroid, bounding box
//   3. k_mem_bending   per element: back-propagation of the bending energy (Eq. 7)
//   4. k_mem_update    per node: gathers of all element contributions (node ->
//      element CSR, no atomics) including the two-step average of the momentum
//      exchanged with the fluid, Hertz forces (Eq. 11), node update (Eq. 9);
//      FP64 sums of force, torque and total force
//   5. k_mem_frozen    (frozen capsules only) rigid translation with the
//      summed force.
// Kernels 1-3 depend on the positions only, so they run on a second stream
// while the lattice update of the same step runs; kernel 4 joins both.  The
// cut links of the moved membrane are rebuilt by k_cut_faces after
// k_mem_update has reset the previous ones; the density pass of the next step
// prepares the bounce records of the cut links.
// With the diffuse-interface coupling (CF_IBM) kernel 4 runs before the
// collide pass and spreads each node's force to the lattice with Peskin's
// 4-point kernel instead of moving it; k_ibm_move then moves the nodes with
// the fluid velocity of the step, interpolated with the same kernel.
#include "cf_common.cuh"
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cfloat>
#include <climits>
#include <algorithm>
#include <cooperative_groups.h>

namespace cf {
namespace cg = cooperative_groups;

struct f3 { float x, y, z; };
__device__ __forceinline__ f3 ld3(const float *p, int i) { return {p[3 * i], p[3 * i + 1], p[3 * i + 2]}; }
__device__ __forceinline__ f3 operator-(f3 a, f3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
__device__ __forceinline__ f3 operator+(f3 a, f3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
__device__ __forceinline__ f3 operator*(float s, f3 a) { return {s * a.x, s * a.y, s * a.z}; }
__device__ __forceinline__ float dot(f3 a, f3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ f3 cross(f3 a, f3 b) {
    return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
__device__ __forceinline__ void st3(float *p, f3 v) { p[0] = v.x; p[1] = v.y; p[2] = v.z; }
// Node positions are float pairs hi + lo (|lo| <= ulp(hi)/2, ~48-bit
// precision): per-step displacements (~1e-5) are below the float ulp at
// x ~ 100, and GB300's FP64 pipe runs at a small fraction of the FP32 rate, so
// positions are advanced with an exact two-sum and all geometry uses
// differences (hi_a - hi_b) + (lo_a - lo_b) in float.
struct pf { f3 h, l; };
__device__ __forceinline__ pf ldp(const float *H, const float *L, int i) { return {ld3(H, i), ld3(L, i)}; }
__device__ __forceinline__ f3 pdiff(const pf &a, const pf &b) {
    return {(a.h.x - b.h.x) + (a.l.x - b.l.x), (a.h.y - b.h.y) + (a.l.y - b.l.y),
            (a.h.z - b.h.z) + (a.l.z - b.l.z)};
}
// (h, l) += v exactly up to the pair's precision (Knuth two-sum, renormalised)
__device__ __forceinline__ void pf_add(float &h, float &l, float v) {
    const float s = h + v;
    const float bb = s - h;
    const float err = (h - (s - bb)) + (v - bb);
    const float t = l + err;
    const float h2 = s + t;
    l = t - (h2 - s);
    h = h2;
}
__device__ __forceinline__ void st_pos(float *H, float *L, int i, const pf &x, f3 v) {
    float hx = x.h.x, hy = x.h.y, hz = x.h.z, lx = x.l.x, ly = x.l.y, lz = x.l.z;
    pf_add(hx, lx, v.x); pf_add(hy, ly, v.y); pf_add(hz, lz, v.z);
    st3(H + 3 * i, f3{hx, hy, hz});
    st3(L + 3 * i, f3{lx, ly, lz});
}

// Per-capsule sums: a warp that holds one capsule (the usual case, capsules
// are contiguous) adds its 32 terms in float by shuffles and books the partial
// with one FP64 atomic; mixed warps book per lane.  The accumulators are FP64.
__device__ __forceinline__ void acc_add(double *acc, int cap, int slot, float v, bool valid) {
    const unsigned full = 0xffffffffu;
    const int key = valid ? cap : -1;
    const int k0 = __shfl_sync(full, key, 0);
    if (__all_sync(full, key == k0)) {
        float s = valid ? v : 0.f;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(full, s, o);
        if ((threadIdx.x & 31) == 0 && k0 >= 0) atomicAdd(acc + k0 * A_NACC + slot, (double)s);
    } else if (valid) {
        atomicAdd(acc + cap * A_NACC + slot, (double)v);
    }
}

__device__ __forceinline__ void acc_minmax(int *bbox, int ncaps, int cap, f3 x, bool valid) {
    const unsigned full = 0xffffffffu;
    const int key = valid ? cap : -1;
    const int k0 = __shfl_sync(full, key, 0);
    const float lo[3] = {valid ? x.x : 3.0e38f, valid ? x.y : 3.0e38f, valid ? x.z : 3.0e38f};
    const float hi[3] = {valid ? x.x : -3.0e38f, valid ? x.y : -3.0e38f, valid ? x.z : -3.0e38f};
    if (__all_sync(full, key == k0)) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            float mn = lo[a], mx = hi[a];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                mn = fminf(mn, __shfl_xor_sync(full, mn, o));
                mx = fmaxf(mx, __shfl_xor_sync(full, mx, o));
            }
            if ((threadIdx.x & 31) == 0 && k0 >= 0) {
                atomicMin(bbox + 3 * k0 + a, (int)floorf(mn));
                atomicMax(bbox + 3 * ncaps + 3 * k0 + a, (int)ceilf(mx));
            }
        }
    } else if (valid) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            atomicMin(bbox + 3 * cap + a, (int)floorf(lo[a]));
            atomicMax(bbox + 3 * ncaps + 3 * cap + a, (int)ceilf(hi[a]));
        }
    }
}

// cot of the angle at o between o->p and o->q, with gradients w.r.t. p, q
__device__ __forceinline__ float cot_grad(f3 o, f3 p, f3 q, f3 &dp, f3 &dq) {
    const f3 u = p - o, w = q - o;
    const f3 n = cross(u, w);
    const float s = sqrtf(dot(n, n)), d = dot(u, w);
    const float uu = dot(u, u), ww = dot(w, w);
    const float is = 1.0f / s, c2 = d * is * is;
    // ds/du = (ww u - d w)/s, ds/dw = (uu w - d u)/s
    dp = is * w - c2 * (is * (ww * u - d * w));
    dq = is * u - c2 * (is * (uu * w - d * u));
    return d * is;
}
__device__ __forceinline__ float cot_only(f3 o, f3 p, f3 q) {
    const f3 u = p - o, w = q - o;
    const f3 n = cross(u, w);
    return dot(u, w) / sqrtf(dot(n, n));
}

// Phase 1 for element f (global index): area and volume terms returned.
__device__ __forceinline__ void face_pass(const MemParams &p, const CapDev &cp, int f, float &area,
                                          float &vol) {
    const int ia = p.faces[3 * f], ib = p.faces[3 * f + 1], ic = p.faces[3 * f + 2];
    const pf pa = ldp(p.Xh, p.Xl, ia), pb = ldp(p.Xh, p.Xl, ib), pc = ldp(p.Xh, p.Xl, ic);
    const pf po = ldp(p.Xh, p.Xl, cp.v0);  // capsule origin: its first node
    // element geometry in coordinates local to its first node (translation invariant)
    const f3 a{0.f, 0.f, 0.f}, b = pdiff(pb, pa), c = pdiff(pc, pa);
    const f3 ra = pdiff(pa, po);
    float *S = p.fscr + (long long)f * FS_N;
    const f3 u = b - a, w = c - a;
    const f3 nrm = cross(u, w);
    const float Af = 0.5f * sqrtf(dot(nrm, nrm));
    area = Af;
    vol = dot(ra, nrm) * (1.f / 6.f);  // (x_a - o) . (u x w) / 6, summed in FP64
    if (cp.mode != 0) return;
    // Skalak (Eq. 6): I1 = tr(G0^-1 g) - 2, I2 = det g / det G0 - 1
    const float g11 = dot(u, u), g12 = dot(u, w), g22 = dot(w, w);
    const float m11 = p.refM[3 * f], m12 = p.refM[3 * f + 1], m22 = p.refM[3 * f + 2];
    const float idet = 1.0f / p.refDet[f];
    const float I1 = m11 * g11 + 2.f * m12 * g12 + m22 * g22 - 2.f;
    const float I2 = (g11 * g22 - g12 * g12) * idet - 1.f;
    const float A0 = p.refA[f];
    const float dW1 = 0.25f * cp.kS * (2.f * I1 + 2.f);
    const float dW2 = 0.25f * cp.kS * (-2.f + 2.f * cp.C * I2);
    const f3 gb = A0 * (dW1 * (2.f * (m11 * u + m12 * w)) + dW2 * (2.f * idet * (g22 * u - g12 * w)));
    const f3 gc = A0 * (dW1 * (2.f * (m12 * u + m22 * w)) + dW2 * (2.f * idet * (g11 * w - g12 * u)));
    st3(S + FS_SK + 0, gb + gc);
    st3(S + FS_SK + 3, -1.f * gb);
    st3(S + FS_SK + 6, -1.f * gc);
    // volume gradient terms (x_b x x_c etc.); their per-node sums are
    // translation invariant on a closed mesh, so positions are taken relative
    // to the capsule's first node to avoid cancellation
    const f3 rb = ra + b, rc = ra + c;
    st3(S + FS_DV + 0, cross(rb, rc));
    st3(S + FS_DV + 3, cross(rc, ra));
    st3(S + FS_DV + 6, cross(ra, rb));
    // bending, first pass: cotangents, Laplacian contributions, A_f/3
    const float cta = cot_only(a, b, c), ctb = cot_only(b, c, a), ctc = cot_only(c, a, b);
    st3(S + FS_L + 0, ctc * (b - a) + ctb * (c - a));
    st3(S + FS_L + 3, cta * (c - b) + ctc * (a - b));
    st3(S + FS_L + 6, ctb * (a - c) + cta * (b - c));
    S[FS_AF3] = Af / 3.f;
}

// Node -> element entries are visited eight at a time with all loads issued
// before use (the gather is latency-bound).
constexpr int VU = 8;

__device__ __forceinline__ void node_bending_grad(const MemParams &p, const CapDev &cp, int v) {
    f3 L{0.f, 0.f, 0.f};
    float A = 0.f;
    const int e0 = p.vf_off[v], e1 = p.vf_off[v + 1];
    for (int eb = e0; eb < e1; eb += VU) {
        int ent[VU];
#pragma unroll
        for (int j = 0; j < VU; ++j) ent[j] = eb + j < e1 ? __ldg(p.vf_ent + eb + j) : -1;
#pragma unroll
        for (int j = 0; j < VU; ++j) {
            if (ent[j] < 0) continue;
            const int f = ent[j] / 3, sl = ent[j] - 3 * f;
            const float *S = p.fscr + (long long)f * FS_N;
            L = L + ld3(S + FS_L, sl);
            A += S[FS_AF3];
        }
    }
    const float iA = 1.f / A;
    st3(p.vscr + 4 * v, (0.25f * cp.kB * iA) * L);
    p.vscr[4 * v + 3] = -0.125f * cp.kB * dot(L, L) * iA * iA;
}

// Phase 3 for element f: back-propagation of the bending energy.
__device__ __forceinline__ void face_bending(const MemParams &p, int f) {
    const int ia = p.faces[3 * f], ib = p.faces[3 * f + 1], ic = p.faces[3 * f + 2];
    const pf pa = ldp(p.Xh, p.Xl, ia);
    const f3 a{0.f, 0.f, 0.f}, b = pdiff(ldp(p.Xh, p.Xl, ib), pa), c = pdiff(ldp(p.Xh, p.Xl, ic), pa);
    float *S = p.fscr + (long long)f * FS_N;
    f3 da_p, da_q, db_p, db_q, dc_p, dc_q;
    const float cta = cot_grad(a, b, c, da_p, da_q);  // p=b, q=c
    const float ctb = cot_grad(b, c, a, db_p, db_q);  // p=c, q=a
    const float ctc = cot_grad(c, a, b, dc_p, dc_q);  // p=a, q=b
    const f3 gLa = ld3(p.vscr + 4 * ia, 0), gLb = ld3(p.vscr + 4 * ib, 0), gLc = ld3(p.vscr + 4 * ic, 0);
    const float gAf = (p.vscr[4 * ia + 3] + p.vscr[4 * ib + 3] + p.vscr[4 * ic + 3]) * (1.f / 3.f);
    const float gam_a = dot(gLb - gLc, c - b);
    const float gam_b = dot(gLa - gLc, c - a);
    const float gam_c = dot(gLa - gLb, b - a);
    f3 ga = ctc * (gLb - gLa) + ctb * (gLc - gLa);
    f3 gb = ctc * (gLa - gLb) + cta * (gLc - gLb);
    f3 gc = ctb * (gLa - gLc) + cta * (gLb - gLc);
    gb = gb + gam_a * da_p; gc = gc + gam_a * da_q; ga = ga - gam_a * (da_p + da_q);
    gc = gc + gam_b * db_p; ga = ga + gam_b * db_q; gb = gb - gam_b * (db_p + db_q);
    ga = ga + gam_c * dc_p; gb = gb + gam_c * dc_q; gc = gc - gam_c * (dc_p + dc_q);
    // node areas A_v = sum A_f / 3: dA_f/db, dA_f/dc
    const f3 u = b - a, w = c - a;
    const f3 nrm = cross(u, w);
    const float s = sqrtf(dot(nrm, nrm)), d = dot(u, w), uu = dot(u, u), ww = dot(w, w);
    const f3 dAb = (0.5f / s) * (ww * u - d * w);
    const f3 dAc = (0.5f / s) * (uu * w - d * u);
    gb = gb + gAf * dAb; gc = gc + gAf * dAc; ga = ga - gAf * (dAb + dAc);
    st3(S + FS_BEND + 0, -1.f * ga);
    st3(S + FS_BEND + 3, -1.f * gb);
    st3(S + FS_BEND + 6, -1.f * gc);
}

__device__ __forceinline__ float hertz(float xi, float d0, float d) {
    const float o = d0 - d;
    return xi * o * sqrtf(o);
}

// Phase 4 for node v: coupling, elastic and Hertz forces.
__device__ __forceinline__ void node_forces(const MemParams &p, const CapDev &cp, int cap, int v,
                                            float pre, const pf &x, f3 &Fc, f3 &Ft) {
    Fc = f3{0.f, 0.f, 0.f};
    f3 Fe{0.f, 0.f, 0.f}, Fi{0.f, 0.f, 0.f}, dv{0.f, 0.f, 0.f};
    const bool el = cp.mode == 0;
    const int e0 = p.vf_off[v], e1 = p.vf_off[v + 1];
    // entries GU at a time, every load unconditional (entries past the end
    // repeat the first one with weight 0), so that they are all in flight at once
    constexpr int GU = 4;
    for (int eb = e0; eb < e1; eb += GU) {
        int f[GU], sl[GU];
        float w[GU];
#pragma unroll
        for (int j = 0; j < GU; ++j) {
            const bool ok = eb + j < e1;
            const int e = __ldg(p.vf_ent + (ok ? eb + j : e0));
            f[j] = e / 3;
            sl[j] = e - 3 * f[j];
            w[j] = ok ? 1.f : 0.f;
        }
        f3 ft[GU];
#pragma unroll
        for (int j = 0; j < GU; ++j) {  // exchange of this step and the previous one, summed exactly
            const long long *a = p.FT + 3 * f[j], *b = p.FTprev + 3 * f[j];
            ft[j] = f3{ft_val(a[0] + b[0]), ft_val(a[1] + b[1]), ft_val(a[2] + b[2])};
        }
        if (el) {
            f3 fe[GU], fd[GU];
#pragma unroll
            for (int j = 0; j < GU; ++j) {
                const float *S = p.fscr + (long long)f[j] * FS_N;
                fe[j] = ld3(S + FS_SK, sl[j]) + ld3(S + FS_BEND, sl[j]);
                fd[j] = ld3(S + FS_DV, sl[j]);
            }
#pragma unroll
            for (int j = 0; j < GU; ++j) {
                Fe = Fe + w[j] * fe[j];
                dv = dv + w[j] * fd[j];
            }
        }
#pragma unroll
        for (int j = 0; j < GU; ++j) Fc = Fc + w[j] * ft[j];
    }
    Fc = (0.5f / 3.f) * Fc;  // two-step average, a third to each node of the element
    if (el) Fe = Fe + pre * dv;
    // Hertz (Eq. 11): substrate plane
    if (p.wall) {
        const float d = (x.h.z - p.zrep) + x.l.z;
        if (d < p.delta0) Fi.z += hertz(p.xi, p.delta0, d);
    }
    // Hertz: nodes of other capsules, in three filters: the other capsule's
    // bounding box of the previous step widened by one lattice unit (nodes
    // move far less per step), per periodic image of this node; then the
    // boxes of that capsule's 32-node patches at this step's positions
    // (written by the node kernel) widened by delta0; then the distance of
    // each node of an overlapping patch.  With the image shift applied to
    // this node, each pair closer than delta0 is met in exactly one image
    // (the lattice spans more than 2 delta0 in x and y).
    const float pad = p.delta0 + 1.0f, ppad = p.delta0 + 1e-3f;
    // the partner list (if any) holds, in ascending order, every capsule whose
    // box test below can pass, so the sum runs over the same capsules in the
    // same order as a loop over all of them
    const int nlist = p.nbr ? __ldg(p.nbr_cnt + cap) : 0;
    const bool all = !p.nbr || nlist > CF_NBR_MAX;
    const int ncand = all ? p.ncaps : nlist;
    for (int j = 0; j < ncand; ++j) {
        const int c2 = all ? j : __ldg(p.nbr + cap * CF_NBR_MAX + j);
        if (c2 == cap) continue;
        const int *lo = p.bbox_prev + 3 * c2, *hi = p.bbox_prev + 3 * p.ncaps + 3 * c2;
        if (x.h.z < lo[2] - pad || x.h.z > hi[2] + pad) continue;
        for (int sy = -1; sy <= 1; ++sy)
            for (int sx = -1; sx <= 1; ++sx) {
                const float ox = (float)(sx * p.nx), oy = (float)(sy * p.ny);
                const float qx = x.h.x + ox, qy = x.h.y + oy;
                if (qx < lo[0] - pad || qx > hi[0] + pad) continue;
                if (qy < lo[1] - pad || qy > hi[1] + pad) continue;
                const CapDev c2d = p.caps[c2];
                for (int q = c2d.s0 >> 5; q < (c2d.s0 + c2d.ns) >> 5; ++q) {
                    const float *B = p.pbox + 6 * q;
                    if (qx < B[0] - ppad || qx > B[3] + ppad || qy < B[1] - ppad || qy > B[4] + ppad ||
                        x.h.z < B[2] - ppad || x.h.z > B[5] + ppad)
                        continue;
                    for (int j = 0; j < 32; ++j) {
                        const int w = __ldg(p.perm + 32 * q + j);
                        if (w < 0) break;  // padding ends the capsule's last patch
                        f3 dd = pdiff(x, ldp(p.Xh, p.Xl, w));
                        dd.x += ox;
                        dd.y += oy;
                        const float d = sqrtf(dot(dd, dd));
                        if (d < p.delta0 && d > 0.f) Fi = Fi + (hertz(p.xi, p.delta0, d) / d) * dd;
                    }
                }
            }
    }
    Ft = Fc + Fe + Fi;
}

// Threads per block of the membrane kernels: small blocks spread the few
// thousand latency-bound threads over all SMs.
constexpr int MT = CF_MEM_FACE_BLOCK;  // element kernels
constexpr int MV = CF_MEM_NODE_BLOCK;  // node kernels

// Each kernel body takes its block index within its own capsule set (bid), so
// that one launch can serve the capsule sets of many lattices: the batched
// form of a kernel finds its lattice from the table's block offsets.
__device__ __forceinline__ int tab_find(const int *boff, int n, int b) {
    int lo = 0, hi = n - 1;  // the last table entry whose blocks start at or before b
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (boff[mid] <= b) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}
#define CF_BATCHED(name, body, P, bound)                                              \
    __global__ void __launch_bounds__(bound) name(const __grid_constant__ SparseTab<P> t) { \
        const int i = tab_find(t.boff, t.n, (int)blockIdx.x);                        \
        body(t.p[i], (int)blockIdx.x - t.boff[i]);                                   \
    }

// 0. per-capsule accumulators and bounding boxes of this step: zero and empty
//    (one block per capsule set)
__device__ __forceinline__ void mem_reset_body(const MemParams &p, int) {
    for (int i = threadIdx.x; i < p.ncaps * A_NACC; i += blockDim.x) p.acc[i] = 0.0;
    for (int i = threadIdx.x; i < 3 * p.ncaps; i += blockDim.x) {
        p.bbox[i] = 0x7f7f7f7f;                  // the byte patterns of the single-lattice
        p.bbox[3 * p.ncaps + i] = (int)0x80808080u;  // step's memsets
    }
}

// 1. elements: Skalak, volume and first bending terms, FP64 area and volume
__device__ __forceinline__ void mem_elements_body(const MemParams &p, int bid) {
    const int f = bid * MT + threadIdx.x;
    const bool valid = f < p.nfaces;
    const int cap = p.face_cap[valid ? f : 0];
    float area = 0.f, vol = 0.f;
    if (valid) face_pass(p, p.caps[cap], f, area, vol);
    acc_add(p.acc, cap, A_AREA, area, valid);
    acc_add(p.acc, cap, A_VOL, vol, valid);
}

// 2. nodes, one warp per 32-node patch: bending gradients, centroid
//    (relative to the capsule's first node), bounding boxes of the capsule
//    and of the patch.  Lane 0 of a patch always holds a node, so padding
//    lanes take its capsule and every warp sums for one capsule.
__device__ __forceinline__ void mem_nodes_body(const MemParams &p, int bid) {
    const int v = p.perm[bid * MV + threadIdx.x];
    const bool valid = v >= 0;
    const int vv = valid ? v : p.perm[bid * MV];
    const int cap = p.node_cap[vv];
    const CapDev cp = p.caps[cap];
    if (valid && cp.mode == 0) node_bending_grad(p, cp, vv);
    const pf x = ldp(p.Xh, p.Xl, vv);
    const f3 r = pdiff(x, ldp(p.Xh, p.Xl, cp.v0));
    if (valid && vv == cp.v0) {
        double *A = p.acc + cap * A_NACC;
        A[A_OX] = (double)x.h.x + x.l.x;
        A[A_OY] = (double)x.h.y + x.l.y;
        A[A_OZ] = (double)x.h.z + x.l.z;
        // volume penalty prefactor -kV (V - V0) / V0 / 6 (Eq. 8); V is the
        // FP64 sum of the element terms (relative to the first node), complete
        // since the element kernel ran
        A[A_PRE] = -(double)cp.kV * (A[A_VOL] - cp.V0) / cp.V0 / 6.0;
    }
    acc_add(p.acc, cap, A_CX, r.x, valid);
    acc_add(p.acc, cap, A_CY, r.y, valid);
    acc_add(p.acc, cap, A_CZ, r.z, valid);
    acc_minmax(p.bbox, p.ncaps, cap, x.h, valid);
    // the patch's box (the padding lanes repeat lane 0's node)
    float b[6] = {x.h.x, x.h.y, x.h.z, x.h.x, x.h.y, x.h.z};
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            b[a] = fminf(b[a], __shfl_xor_sync(0xffffffffu, b[a], o));
            b[3 + a] = fmaxf(b[3 + a], __shfl_xor_sync(0xffffffffu, b[3 + a], o));
        }
    if (threadIdx.x < 6) {
        float vb = b[0];
#pragma unroll
        for (int a = 1; a < 6; ++a) vb = threadIdx.x == a ? b[a] : vb;
        p.pbox[6 * bid + threadIdx.x] = vb;
    }
}

// 3. elements: bending back-propagation
__device__ __forceinline__ void mem_bending_body(const MemParams &p, int bid) {
    const int f = bid * MT + threadIdx.x;
    if (f < p.nfaces && p.caps[p.face_cap[f]].mode == 0) face_bending(p, f);
}

// 4. nodes: coupling, elastic and Hertz forces, node update (Eq. 9), FP64
//    sums of force, torque and total force.  Blocks past the nodes undo the
//    previous cut structure (each entry of the previous list names one marked
//    link: its mask word and crossed element are reset) before the cut links
//    of the new positions are marked.
// reset of the cut structure of list cl.list: block bid of cl.blocks
__device__ __forceinline__ void cut_clear_body(const ClearParams &cl, int bid) {
    const int cnt = min(*cl.count, cl.capacity);
    for (int i = bid * MV + threadIdx.x; i < cnt; i += cl.blocks * MV) {
        const int2 e = cl.list[i];
        const long long n = (long long)((unsigned)e.x >> 5);
        cl.mask[n] = 0u;
        cl.tri[n * 18 + (e.x & 31)] = 0x7fffffff;
    }
}

// ------------------------------------------------ diffuse-interface coupling
// Peskin's 4-point kernel (Peskin, "The immersed boundary method", Acta
// Numerica 2002): phi(r) = (3 - 2r + sqrt(1 + 4r - 4r^2)) / 8 on [0, 1] and
// (5 - 2r - sqrt(-7 + 12r - 4r^2)) / 8 on [1, 2], which equals 1/2 - phi(2 - r)
// there.  A coordinate with integer part f and fraction t in [0, 1] reaches
// the nodes f-1 .. f+2 at distances 1+t, t, 1-t, 2-t, so its four weights are
// 1/2 - phi(1-t), phi(t), phi(1-t), 1/2 - phi(t): two square roots, and the
// weights sum to one.
__device__ __forceinline__ float peskin_inner(float r) {
    return 0.125f * (3.f - 2.f * r + sqrtf(1.f + 4.f * r * (1.f - r)));
}
// first node b (= floor(x) - 1) and weights of one coordinate x = h + l
__device__ __forceinline__ void ibm_axis(float h, float l, int &b, float (&w)[4]) {
    float fl = floorf(h);
    float t = (h - fl) + l;  // h - fl is exact; |l| <= ulp(h) / 2
    if (t < 0.f) { t += 1.f; fl -= 1.f; }
    else if (t >= 1.f) { t -= 1.f; fl += 1.f; }
    // a non-finite position (reported by the cut-link kernel) still gives
    // in-range nodes: fmaxf drops a NaN, the clamp keeps the int conversion defined
    b = (int)fminf(fmaxf(fl, -1e8f), 1e8f) - 1;
    const float p0 = peskin_inner(t), p1 = peskin_inner(1.f - t);
    w[0] = 0.5f - p1; w[1] = p0; w[2] = p1; w[3] = 0.5f - p0;
}
// The 4 x 4 x 4 nodes around x (periodic; substrate nodes skipped) with their
// weights: f(lattice index, weight) for each
template <class Fn>
__device__ __forceinline__ void ibm_stencil(const MemParams &p, const pf &x, Fn f) {
    int b[3];
    float w[3][4];
    ibm_axis(x.h.x, x.l.x, b[0], w[0]);
    ibm_axis(x.h.y, x.l.y, b[1], w[1]);
    ibm_axis(x.h.z, x.l.z, b[2], w[2]);
#pragma unroll
    for (int kz = 0; kz < 4; ++kz) {
        const int z = wrapi(b[2] + kz, p.nz);
        if (p.wall && z == 0) continue;
#pragma unroll
        for (int ky = 0; ky < 4; ++ky) {
            const long long row = ((long long)z * p.ny + wrapi(b[1] + ky, p.ny)) * p.nx;
#pragma unroll
            for (int kx = 0; kx < 4; ++kx) f(row + wrapi(b[0] + kx, p.nx), (w[0][kx] * w[1][ky]) * w[2][kz]);
        }
    }
}

// The forces F of the warp's nodes at x spread to the lattice, their stencil
// nodes flagged.  Each contribution F_a w is rounded to fixed point (ft_add),
// so the sums do not depend on the order of the atomics.  The warp takes its
// nodes one after another; lane l adds stencil column kx = l % 4 of the rows
// (kz, ky) in group g = l / 4, so that an atomic instruction writes 8 runs of
// 4 consecutive lattice nodes instead of 32 scattered ones.  Per node the six
// passes cover the component a = pass / 2 and the rows ky = g % 4,
// kz = g / 4 + 2 (pass % 2).  Called by the whole (32-thread) warp.
struct IbmNode { int b[3]; float w[3][4]; float F[3]; };
__device__ __forceinline__ void ibm_spread_warp(const MemParams &p, bool valid, const pf &x, f3 F) {
    __shared__ IbmNode sn[32];
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    if (valid) {
        IbmNode &m = sn[lane];
        ibm_axis(x.h.x, x.l.x, m.b[0], m.w[0]);
        ibm_axis(x.h.y, x.l.y, m.b[1], m.w[1]);
        ibm_axis(x.h.z, x.l.z, m.b[2], m.w[2]);
        m.F[0] = F.x; m.F[1] = F.y; m.F[2] = F.z;
    }
    __syncwarp();
    long long *fb = p.fibm;
    const long long N = p.N;
    uint8_t *flag = ibm_flags(p.uphys, N);
    const int kx = lane & 3, g = lane >> 2, ky = g & 3, kz0 = g >> 2;
    unsigned todo = __ballot_sync(full, valid);
    while (todo) {
        const int j = __ffs(todo) - 1;
        todo &= todo - 1;
        const IbmNode &m = sn[j];
        const long long xn = wrapi(m.b[0] + kx, p.nx);
        const long long yrow = wrapi(m.b[1] + ky, p.ny);
        const float wxy = m.w[0][kx] * m.w[1][ky];
#pragma unroll
        for (int h = 0; h < 2; ++h) {  // rows kz = kz0 and kz0 + 2
            const int kz = kz0 + 2 * h;
            const int z = wrapi(m.b[2] + kz, p.nz);
            if (p.wall && z == 0) continue;  // substrate nodes take no force
            const long long n = ((long long)z * p.ny + yrow) * p.nx + xn;
            const float wt = wxy * m.w[2][kz];
#pragma unroll
            for (int a = 0; a < 3; ++a) ft_add(fb + a * N + n, m.F[a] * wt);
            flag[n >> 5] = 1;
        }
    }
    __syncwarp();
}

// IBM: the diffuse-interface spreading may be on (single-lattice kernel only)
template <bool IBM = false>
__device__ __forceinline__ void mem_update_body(const MemParams &p, const ClearParams &cl, int bid) {
    if (cl.count_next && bid == 0 && threadIdx.x == 0) *cl.count_next = 0;
    const int node_blocks = (p.nnodes + MV - 1) / MV;
    if (bid >= node_blocks) {
        cut_clear_body(cl, bid - node_blocks);
        return;
    }
    const int v = bid * MV + threadIdx.x;
    const bool valid = v < p.nnodes;
    const int vv = valid ? v : 0;
    const int cap = p.node_cap[vv];
    const CapDev cp = p.caps[cap];
    const double *A = p.acc + cap * A_NACC;
    f3 Fc{0.f, 0.f, 0.f}, Ft{0.f, 0.f, 0.f}, r{0.f, 0.f, 0.f};
    const pf x = ldp(p.Xh, p.Xl, vv);
    if (valid) {
        const float pre = (float)A[A_PRE];
        node_forces(p, cp, cap, vv, pre, x, Fc, Ft);
        st3(p.Fcpl + 3 * vv, Fc);
        if (p.fibm) {
            // spread below by the whole warp; the node moves after the lattice update (k_ibm_move)
        } else if (cp.mode == 0) {
            // Eq. 9 with dt = 1 (v = F/m), or with CF_INERTIAL v += F/m
            f3 vel = (1.f / cp.mass) * Ft;
            if (p.inertial) vel = vel + ld3(p.V, vv);
            st3(p.V + 3 * vv, vel);
            st_pos(p.Xnh, p.Xnl, vv, x, vel);
        } else if (cp.mode == 2) {
            st3(p.V + 3 * vv, f3{0.f, 0.f, 0.f});
            st_pos(p.Xnh, p.Xnl, vv, x, f3{0.f, 0.f, 0.f});
        }
        const float ic = 1.f / cp.nv;
        const f3 cen{(float)A[A_CX] * ic, (float)A[A_CY] * ic, (float)A[A_CZ] * ic};
        r = pdiff(x, ldp(p.Xh, p.Xl, cp.v0)) - cen;
    }
    const f3 tq = cross(r, Fc);
    double *Aw = p.acc;
    acc_add(Aw, cap, A_FX, Fc.x, valid);
    acc_add(Aw, cap, A_FY, Fc.y, valid);
    acc_add(Aw, cap, A_FZ, Fc.z, valid);
    acc_add(Aw, cap, A_TX, tq.x, valid);
    acc_add(Aw, cap, A_TY, tq.y, valid);
    acc_add(Aw, cap, A_TZ, tq.z, valid);
    acc_add(Aw, cap, A_FTX, Ft.x, valid);
    acc_add(Aw, cap, A_FTY, Ft.y, valid);
    acc_add(Aw, cap, A_FTZ, Ft.z, valid);
    if (IBM && p.fibm) ibm_spread_warp(p, valid, x, Ft);
}
__device__ __forceinline__ void mem_update_body(const UpdateParams &u, int bid) { mem_update_body(u.m, u.c, bid); }

// 5. frozen shapes: rigid translation with the summed force
__device__ __forceinline__ void mem_frozen_body(const MemParams &p, int bid) {
    const int v = bid * MV + threadIdx.x;
    if (v >= p.nnodes) return;
    const int cap = p.node_cap[v];
    const CapDev cp = p.caps[cap];
    if (cp.mode != 1) return;
    const double *A = p.acc + cap * A_NACC;
    const double sc = 1.0 / ((double)cp.mass * cp.nv);
    f3 vel{(float)(A[A_FTX] * sc), (float)(A[A_FTY] * sc), (float)(A[A_FTZ] * sc)};
    if (p.inertial) vel = vel + ld3(p.V, v);
    st3(p.V + 3 * v, vel);
    st_pos(p.Xnh, p.Xnl, v, ldp(p.Xh, p.Xl, v), vel);
}

__global__ void __launch_bounds__(MT) k_mem_elements(const MemParams p) { mem_elements_body(p, blockIdx.x); }
__global__ void __launch_bounds__(MV) k_mem_nodes(const MemParams p) { mem_nodes_body(p, blockIdx.x); }
__global__ void __launch_bounds__(MT) k_mem_bending(const MemParams p) { mem_bending_body(p, blockIdx.x); }
// IBM: spreading for the diffuse-interface coupling (its own instantiation)
template <bool IBM>
__global__ void __launch_bounds__(MV) k_mem_update(const MemParams p, const ClearParams cl) {
    pdl_trigger();
    pdl_wait();
    mem_update_body<IBM>(p, cl, blockIdx.x);
}
__global__ void __launch_bounds__(MV) k_mem_frozen(const MemParams p) { mem_frozen_body(p, blockIdx.x); }

// Diffuse-interface coupling: each free node moves with the fluid velocity of
// this step interpolated at its position with the spreading kernel (substrate
// nodes carry zero velocity); fixed nodes stay.
__global__ void __launch_bounds__(MV) k_ibm_move(const MemParams p) {
    const int v = blockIdx.x * MV + threadIdx.x;
    if (v >= p.nnodes) return;
    const pf x = ldp(p.Xh, p.Xl, v);
    f3 u{0.f, 0.f, 0.f};
    if (p.caps[p.node_cap[v]].mode == 0) {
        const float4 *up = p.uphys;
        ibm_stencil(p, x, [&](long long n, float w) {
            const float4 q = __ldg(up + n);
            u = u + w * f3{q.x, q.y, q.z};
        });
    }
    st3(p.V + 3 * v, u);
    st_pos(p.Xnh, p.Xnl, v, x, u);
}

__global__ void __launch_bounds__(MV) k_cut_clear(const ClearParams cl) {
    if (cl.count_next && blockIdx.x == 0 && threadIdx.x == 0) *cl.count_next = 0;
    cut_clear_body(cl, blockIdx.x);
}

cudaError_t launch_cut_clear(const ClearParams &cl, cudaStream_t s, int *nl) {
    if (cl.blocks <= 0) return cudaSuccess;
    k_cut_clear<<<(unsigned)cl.blocks, MV, 0, s>>>(cl);
    *nl += 1;
    return cudaGetLastError();
}

cudaError_t launch_ibm_move(const MemParams &p, cudaStream_t s, int *nl) {
    k_ibm_move<<<(unsigned)((p.nnodes + MV - 1) / MV), MV, 0, s>>>(p);
    *nl += 1;
    return cudaGetLastError();
}

__global__ void __launch_bounds__(MT) k_mem_reset_b(const __grid_constant__ SparseTab<MemParams> t) {
    mem_reset_body(t.p[blockIdx.x], 0);
}
CF_BATCHED(k_mem_elements_b, mem_elements_body, MemParams, MT)
CF_BATCHED(k_mem_nodes_b, mem_nodes_body, MemParams, MV)
CF_BATCHED(k_mem_bending_b, mem_bending_body, MemParams, MT)
CF_BATCHED(k_mem_frozen_b, mem_frozen_body, MemParams, MV)
__global__ void __launch_bounds__(MV) k_mem_update_b(const __grid_constant__ SparseTab<UpdateParams> t) {
    pdl_trigger();
    pdl_wait();
    const int i = tab_find(t.boff, t.n, (int)blockIdx.x);
    mem_update_body(t.p[i], (int)blockIdx.x - t.boff[i]);
}

// One warp per capsule c: the capsules c2 != c (ascending) whose box of the
// previous step, widened by the contact range plus one unit, overlaps c's box
// widened by one unit (nodes move far less than a unit per step) in some
// periodic image along x and y: a superset of the capsules the node loop's
// box test can accept for a node of c.
__global__ void __launch_bounds__(32) k_contact_partners(const MemParams p, int *nbr, int *nbr_cnt) {
    const int c = blockIdx.x;
    const int lane = threadIdx.x;
    const int *lo = p.bbox_prev, *hi = p.bbox_prev + 3 * p.ncaps;
    const float pad = p.delta0 + 2.0f;
    const float cl[3] = {(float)lo[3 * c], (float)lo[3 * c + 1], (float)lo[3 * c + 2]};
    const float ch[3] = {(float)hi[3 * c], (float)hi[3 * c + 1], (float)hi[3 * c + 2]};
    int count = 0;
    for (int b = 0; b < p.ncaps; b += 32) {
        const int c2 = b + lane;
        bool ok = false;
        if (c2 < p.ncaps && c2 != c) {
            const float l2[3] = {(float)lo[3 * c2], (float)lo[3 * c2 + 1], (float)lo[3 * c2 + 2]};
            const float h2[3] = {(float)hi[3 * c2], (float)hi[3 * c2 + 1], (float)hi[3 * c2 + 2]};
            if (ch[2] >= l2[2] - pad && cl[2] <= h2[2] + pad) {
                for (int sy = -1; sy <= 1 && !ok; ++sy)
                    for (int sx = -1; sx <= 1 && !ok; ++sx) {
                        const float ox = (float)(sx * p.nx), oy = (float)(sy * p.ny);
                        ok = ch[0] + ox >= l2[0] - pad && cl[0] + ox <= h2[0] + pad &&
                             ch[1] + oy >= l2[1] - pad && cl[1] + oy <= h2[1] + pad;
                    }
            }
        }
        const unsigned m = __ballot_sync(0xffffffffu, ok);
        const int at = count + __popc(m & ((1u << lane) - 1u));
        if (ok && at < CF_NBR_MAX) nbr[c * CF_NBR_MAX + at] = c2;
        count += __popc(m);
    }
    if (lane == 0) nbr_cnt[c] = count;  // above CF_NBR_MAX: the node loop checks every capsule
}

cudaError_t launch_contact_partners(const MemParams &p, int *nbr, int *nbr_cnt, cudaStream_t s, int *nl) {
    k_contact_partners<<<p.ncaps, 32, 0, s>>>(p, nbr, nbr_cnt);
    *nl += 1;
    return cudaGetLastError();
}

cudaError_t launch_membrane_forces(const MemParams &p, cudaStream_t s, int *nl) {
    const unsigned gf = (unsigned)((p.nfaces + MT - 1) / MT), gs = (unsigned)(p.nslots / MV);
    k_mem_elements<<<gf, MT, 0, s>>>(p);
    k_mem_nodes<<<gs, MV, 0, s>>>(p);
    k_mem_bending<<<gf, MT, 0, s>>>(p);
    *nl += 3;
    return cudaGetLastError();
}

cudaError_t launch_membrane_update(const MemParams &p, const ClearParams &cl, bool any_frozen,
                                   cudaStream_t s, int *nl) {
    const unsigned gv = (unsigned)((p.nnodes + MV - 1) / MV);
    if (p.fibm) launch_pdl(k_mem_update<true>, dim3(gv + (unsigned)cl.blocks), dim3(MV), s, p, cl);
    else launch_pdl(k_mem_update<false>, dim3(gv + (unsigned)cl.blocks), dim3(MV), s, p, cl);
    *nl += 1;
    if (any_frozen) {
        k_mem_frozen<<<gv, MV, 0, s>>>(p);
        *nl += 1;
    }
    return cudaGetLastError();
}

// Batched forms: tv holds node-kernel block offsets, tf element-kernel ones
cudaError_t launch_membrane_forces_batch(const SparseTab<MemParams> &tv, const SparseTab<MemParams> &tf,
                                         cudaStream_t s, int *nl) {
    if (tv.n == 0) return cudaSuccess;
    k_mem_reset_b<<<tv.n, MT, 0, s>>>(tv);
    if (tf.boff[tf.n] > 0) k_mem_elements_b<<<tf.boff[tf.n], MT, 0, s>>>(tf);
    k_mem_nodes_b<<<tv.boff[tv.n], MV, 0, s>>>(tv);
    if (tf.boff[tf.n] > 0) k_mem_bending_b<<<tf.boff[tf.n], MT, 0, s>>>(tf);
    *nl += 4;
    return cudaGetLastError();
}

cudaError_t launch_membrane_update_batch(const SparseTab<UpdateParams> &tu, const SparseTab<MemParams> *tfz,
                                         cudaStream_t s, int *nl) {
    if (tu.n == 0) return cudaSuccess;
    launch_pdl(k_mem_update_b, dim3((unsigned)tu.boff[tu.n]), dim3(MV), s, tu);
    *nl += 1;
    if (tfz && tfz->n > 0) {
        k_mem_frozen_b<<<tfz->boff[tfz->n], MV, 0, s>>>(*tfz);
        *nl += 1;
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------- cut links
// Orientation det[b-a; c-a; d-a] in FP32 with a certainty margin, and in FP64
// for the undecided cases.  Coordinates stay within a few lattice units of each
// other, so the FP32 value is accurate to ~1e-5.
__device__ __forceinline__ float orient_f(f3 a, f3 b, f3 c, f3 d) {
    return dot(b - a, cross(c - a, d - a));
}
__device__ __forceinline__ double orient_d(f3 a, f3 b, f3 c, f3 d) {
    const double r1x = (double)b.x - a.x, r1y = (double)b.y - a.y, r1z = (double)b.z - a.z;
    const double r2x = (double)c.x - a.x, r2y = (double)c.y - a.y, r2z = (double)c.z - a.z;
    const double r3x = (double)d.x - a.x, r3y = (double)d.y - a.y, r3z = (double)d.z - a.z;
    const double nx = r2y * r3z - r2z * r3y, ny = r2z * r3x - r2x * r3z, nz = r2x * r3y - r2y * r3x;
    return r1x * nx + r1y * ny + r1z * nz;
}
constexpr float OEPS = 1e-4f;

// FP64 decisions are rare and kept out of line: GB300's FP64 pipe is a small
// fraction of its FP32 rate, and an inlined fallback may be if-converted.
__device__ __noinline__ bool side_of_d(f3 A, f3 B, f3 C, f3 P) { return orient_d(A, B, C, P) >= 0.0; }

// segment P->Q, already known to have its end points on opposite sides of the
// plane, crosses triangle ABC (sign(0) = + convention on the edge tests)
__device__ __noinline__ bool edges_pass_d(f3 P, f3 Qp, f3 A, f3 B, f3 C) {
    const double S1 = orient_d(P, Qp, A, B), S2 = orient_d(P, Qp, B, C), S3 = orient_d(P, Qp, C, A);
    return ((S1 >= 0.0) == (S2 >= 0.0)) && ((S2 >= 0.0) == (S3 >= 0.0));
}
__device__ __forceinline__ bool edges_pass(f3 P, f3 Qp, f3 A, f3 B, f3 C) {
    const float s1 = orient_f(P, Qp, A, B), s2 = orient_f(P, Qp, B, C), s3 = orient_f(P, Qp, C, A);
    if (fabsf(s1) > OEPS && fabsf(s2) > OEPS && fabsf(s3) > OEPS)
        return ((s1 >= 0.f) == (s2 >= 0.f)) && ((s2 >= 0.f) == (s3 >= 0.f));
    return edges_pass_d(P, Qp, A, B, C);
}

// L lanes per element (the launches use L = 1 when they have elements enough
// to fill the GPU, else the warp-per-element form below).  A link (P, P+e_k), k in the nine positive directions,
// can cross the element only where its crossing point lies in the element's
// bounding box: along an axis a with e_a = 0 the start node lies in the box,
// along an axis with e_a = +1 (-1) in the box widened by one unit below
// (above).  The lanes walk that range of start nodes for each direction
// (widened by 1e-3, so the candidates cover every crossing the exact tests
// can find; an element of the usual size has about twenty), lane j of the
// element taking candidates j, j + L, ..., and give each candidate the exact
// tests: plane sides of both end points
// (orientation against the element, sign(0) = +, FP32 with a margin and FP64
// otherwise) and, where they differ, the three edge orientations.  A crossing
// toggles the cut bit of the link at both of its end nodes, keeps the
// smallest crossing element there, and appends one list entry per end node.
// Lane 0 also records the element's velocity (the mean of its nodes', for
// Ladd's term of the next streaming) and zeroes the element's
// momentum-exchange accumulator of the next step.
constexpr int CUT_TPB = 128;  // threads per block

// periodic index, with the common in-range case first
__device__ __forceinline__ int wrap_fast(int a, int n) { return (unsigned)a < (unsigned)n ? a : wrapi(a, n); }
__device__ __forceinline__ long long node_at(const CutParams &p, int x, int y, int z) {
    return ((long long)wrap_fast(z, p.nz) * p.ny + wrap_fast(y, p.ny)) * p.nx + wrap_fast(x, p.nx);
}

// plane side (sign(0) = +) of P against the element ABC with normal nrm =
// (B-A) x (C-A): the orientation det[B-A; C-A; P-A] = nrm . (P-A), in float
// within ~1e-6 of its exact value for nodes within a few units of A, so the
// margin sends every close case to the FP64 test
__device__ __forceinline__ bool plane_side(const f3 &nrm, const f3 &A, const f3 &B, const f3 &C,
                                           const f3 &P) {
    const float d = dot(nrm, P - A);
    return fabsf(d) > OEPS ? d >= 0.f : side_of_d(A, B, C, P);
}

// one candidate link (direction k from start node (x, y, z)) of element T
__device__ __forceinline__ void cut_candidate(const CutParams &p, int T, const f3 &A, const f3 &B, const f3 &C,
                                              const f3 &nrm, int k, const int (&e)[3], int x, int y, int z) {
    // links touching the substrate plane z = 0 are not fluid links
    if (p.wall && (wrap_fast(z, p.nz) == 0 || wrap_fast(z + e[2], p.nz) == 0)) return;
    const f3 P{(float)x, (float)y, (float)z};
    const f3 Qp{(float)(x + e[0]), (float)(y + e[1]), (float)(z + e[2])};
    if (plane_side(nrm, A, B, C, P) == plane_side(nrm, A, B, C, Qp) || !edges_pass(P, Qp, A, B, C)) return;
    const long long n0 = node_at(p, x, y, z), n1 = node_at(p, x + e[0], y + e[1], z + e[2]);
    const int k2 = opp(k);
    atomicXor(p.mask + n0, 1u << (k - 1));
    atomicMin(p.tri + n0 * 18 + (k - 1), T);
    atomicXor(p.mask + n1, 1u << (k2 - 1));
    atomicMin(p.tri + n1 * 18 + (k2 - 1), T);
    // one counter update for the lanes that append together (all of a block's
    // lanes belong to one lattice, so they share the counter)
    const cg::coalesced_group g = cg::coalesced_threads();
    int base = 0;
    if (g.thread_rank() == 0) base = atomicAdd(p.count, 2 * (int)g.size());
    const int idx = g.shfl(base, 0) + 2 * (int)g.thread_rank();
    if (idx + 1 < p.capacity) {
        p.list[idx] = make_int2(cut_code(n0, k), T);
        p.list[idx + 1] = make_int2(cut_code(n1, k2), T);
    } else {
        atomicOr(p.status, ST_OVERFLOW);
    }
}

// The same tests with one warp per element, for launches with few elements:
// lanes 0-8 take one direction each and compute its range of start nodes, a
// warp prefix sum hands every lane one (direction, start node) candidate, 32
// per pass, and each pass appends its crossings with one counter update.
__device__ __forceinline__ void cut_faces_warp_body(const CutParams &p, int bid) {
    const unsigned full = 0xffffffffu;
    const int lane = (int)(threadIdx.x & 31);
    const int T = bid * (CUT_TPB / 32) + (int)(threadIdx.x >> 5);
    if (T >= p.nfaces) return;  // the whole warp
    if (p.zero_only) {  // fixed capsules: the cut links stay, the accumulator is zeroed
        if (lane < 3) p.FTnext[3 * T + lane] = 0;
        return;
    }
    const int ia = p.faces[3 * T], ib = p.faces[3 * T + 1], ic = p.faces[3 * T + 2];
    if (lane == 0) {
        const float ux = (p.V[3 * ia] + p.V[3 * ib] + p.V[3 * ic]) * (1.0f / 3.0f);
        const float uy = (p.V[3 * ia + 1] + p.V[3 * ib + 1] + p.V[3 * ic + 1]) * (1.0f / 3.0f);
        const float uz = (p.V[3 * ia + 2] + p.V[3 * ib + 2] + p.V[3 * ic + 2]) * (1.0f / 3.0f);
        p.uT[T] = make_float4(ux, uy, uz, 0.f);
    } else if (lane < 4) {
        p.FTnext[3 * T + lane - 1] = 0;
    }
    // the decision is taken on the float (hi) positions
    const f3 A = ld3(p.X, ia), B = ld3(p.X, ib), C = ld3(p.X, ic);
    const float emin[3] = {fminf(A.x, fminf(B.x, C.x)), fminf(A.y, fminf(B.y, C.y)),
                           fminf(A.z, fminf(B.z, C.z))};
    const float emax[3] = {fmaxf(A.x, fmaxf(B.x, C.x)), fmaxf(A.y, fmaxf(B.y, C.y)),
                           fmaxf(A.z, fmaxf(B.z, C.z))};
    // an element spanning more than 16 units (or with a non-finite position)
    // is an error, not a workload: it would hand the warp unbounded candidates
    if (!(emax[0] - emin[0] <= 16.f && emax[1] - emin[1] <= 16.f && emax[2] - emin[2] <= 16.f)) {
        if (lane == 0) atomicOr(p.status, ST_OVERFLOW);
        return;
    }
    // lane d < 9: start-node range of direction k = 2d + 1
    const float pad = 1e-3f;
    int rlo[3] = {0, 0, 0}, rn[3] = {0, 0, 0};
    int cnt = 0;
    if (lane < 9) {
        int e[3];
        ek(2 * lane + 1, e[0], e[1], e[2]);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const float lo = (e[a] > 0 ? emin[a] - 1.f : emin[a]) - pad;
            const float hi = (e[a] < 0 ? emax[a] + 1.f : emax[a]) + pad;
            rlo[a] = (int)ceilf(lo);
            rn[a] = max(0, (int)floorf(hi) - rlo[a] + 1);
        }
        cnt = rn[0] * rn[1] * rn[2];
    }
    int incl = cnt;
#pragma unroll
    for (int o = 1; o < 16; o <<= 1) {
        const int t = __shfl_up_sync(full, incl, o);
        if (lane >= o) incl += t;
    }
    const int total = __shfl_sync(full, incl, 8);
    const f3 nrm = cross(B - A, C - A);
    for (int j0 = 0; j0 < total; j0 += 32) {
        const int j = j0 + lane;
        // direction of candidate j: the number of directions whose inclusive
        // prefix is at most j
        int dsel = 0;
#pragma unroll
        for (int d = 0; d < 9; ++d) dsel += __shfl_sync(full, incl, d) <= j ? 1 : 0;
        const int src = min(dsel, 8);
        const int base = __shfl_sync(full, incl - cnt, src);
        const int lx = __shfl_sync(full, rlo[0], src), ly = __shfl_sync(full, rlo[1], src),
                  lz = __shfl_sync(full, rlo[2], src);
        const int nx_ = __shfl_sync(full, rn[0], src), ny_ = __shfl_sync(full, rn[1], src);
        bool hit = false;
        long long n0 = 0, n1 = 0;
        const int k = 2 * src + 1;
        if (j < total) {
            // start node idx of the direction's range, x fastest
            const int idx = j - base;
            const int nxy = nx_ * ny_;
            // (idx + 1/2) / nxy lies at least 1/(2 nxy) from an integer, far
            // above the error of the fast quotient, so truncation is exact
            const int iz = (int)__fdividef((float)idx + 0.5f, (float)nxy);
            const int r = idx - iz * nxy;
            const int iy = (int)__fdividef((float)r + 0.5f, (float)nx_);
            const int x = lx + r - iy * nx_, y = ly + iy, z = lz + iz;
            int kx, ky, kz;
            ek(k, kx, ky, kz);
            // links touching the substrate plane z = 0 are not fluid links
            if (!(p.wall && (wrap_fast(z, p.nz) == 0 || wrap_fast(z + kz, p.nz) == 0))) {
                const f3 P{(float)x, (float)y, (float)z};
                const f3 Qp{(float)(x + kx), (float)(y + ky), (float)(z + kz)};
                hit = plane_side(nrm, A, B, C, P) != plane_side(nrm, A, B, C, Qp) &&
                      edges_pass(P, Qp, A, B, C);
            }
            if (hit) {
                n0 = node_at(p, x, y, z);
                n1 = node_at(p, x + kx, y + ky, z + kz);
            }
        }
        const unsigned hits = __ballot_sync(full, hit);
        if (!hits) continue;
        const int leader = __ffs(hits) - 1;
        int at = 0;
        if (lane == leader) at = atomicAdd(p.count, 2 * __popc(hits));
        at = __shfl_sync(full, at, leader);
        if (hit) {
            const int k2 = opp(k);
            atomicXor(p.mask + n0, 1u << (k - 1));
            atomicMin(p.tri + n0 * 18 + (k - 1), T);
            atomicXor(p.mask + n1, 1u << (k2 - 1));
            atomicMin(p.tri + n1 * 18 + (k2 - 1), T);
            const int idx = at + 2 * __popc(hits & ((1u << lane) - 1u));
            if (idx + 1 < p.capacity) {
                p.list[idx] = make_int2(cut_code(n0, k), T);
                p.list[idx + 1] = make_int2(cut_code(n1, k2), T);
            } else {
                atomicOr(p.status, ST_OVERFLOW);
            }
        }
    }
}


template <int L>
__device__ __forceinline__ void cut_faces_body(const CutParams &p, int bid) {
    const int t = bid * CUT_TPB + (int)threadIdx.x;
    const int T = t / L, sub = t % L;
    if (T >= p.nfaces) return;
    if (sub == 0) {
        p.FTnext[3 * T] = 0;
        p.FTnext[3 * T + 1] = 0;
        p.FTnext[3 * T + 2] = 0;
    }
    if (p.zero_only) return;  // fixed capsules: the cut links stay, the accumulator is zeroed
    const int ia = p.faces[3 * T], ib = p.faces[3 * T + 1], ic = p.faces[3 * T + 2];
    if (sub == 0) {
        const float ux = (p.V[3 * ia] + p.V[3 * ib] + p.V[3 * ic]) * (1.0f / 3.0f);
        const float uy = (p.V[3 * ia + 1] + p.V[3 * ib + 1] + p.V[3 * ic + 1]) * (1.0f / 3.0f);
        const float uz = (p.V[3 * ia + 2] + p.V[3 * ib + 2] + p.V[3 * ic + 2]) * (1.0f / 3.0f);
        p.uT[T] = make_float4(ux, uy, uz, 0.f);
    }
    // the decision is taken on the float (hi) positions
    const f3 A = ld3(p.X, ia), B = ld3(p.X, ib), C = ld3(p.X, ic);
    const float emin[3] = {fminf(A.x, fminf(B.x, C.x)), fminf(A.y, fminf(B.y, C.y)),
                           fminf(A.z, fminf(B.z, C.z))};
    const float emax[3] = {fmaxf(A.x, fmaxf(B.x, C.x)), fmaxf(A.y, fmaxf(B.y, C.y)),
                           fmaxf(A.z, fmaxf(B.z, C.z))};
    // an element spanning more than 16 units (or with a non-finite position)
    // is an error, not a workload: it would hand the lanes unbounded candidates
    if (!(emax[0] - emin[0] <= 16.f && emax[1] - emin[1] <= 16.f && emax[2] - emin[2] <= 16.f)) {
        if (sub == 0) atomicOr(p.status, ST_OVERFLOW);
        return;
    }
    const float pad = 1e-3f;
    const f3 nrm = cross(B - A, C - A);
    for (int d = 0; d < 9; ++d) {
        const int k = 2 * d + 1;
        int e[3];
        ek(k, e[0], e[1], e[2]);
        int rlo[3], rn[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const float lo = (e[a] > 0 ? emin[a] - 1.f : emin[a]) - pad;
            const float hi = (e[a] < 0 ? emax[a] + 1.f : emax[a]) + pad;
            rlo[a] = (int)ceilf(lo);
            rn[a] = max(0, (int)floorf(hi) - rlo[a] + 1);
        }
        if constexpr (L == 1) {
            for (int z = rlo[2]; z < rlo[2] + rn[2]; ++z)
                for (int y = rlo[1]; y < rlo[1] + rn[1]; ++y)
                    for (int x = rlo[0]; x < rlo[0] + rn[0]; ++x) cut_candidate(p, T, A, B, C, nrm, k, e, x, y, z);
        } else {
            const int nxy = rn[0] * rn[1], total = nxy * rn[2];
            for (int j = sub; j < total; j += L) {
                const int iz = j / nxy, r = j - iz * nxy, iy = r / rn[0];
                cut_candidate(p, T, A, B, C, nrm, k, e, rlo[0] + r - iy * rn[0], rlo[1] + iy, rlo[2] + iz);
            }
        }
    }
}

template <int L>
__device__ __forceinline__ void cut_faces_any(const CutParams &p, int bid) {
    if constexpr (L == 32) cut_faces_warp_body(p, bid);
    else cut_faces_body<L>(p, bid);
}
template <int L>
__global__ void __launch_bounds__(CUT_TPB) k_cut_faces(const CutParams p) {
    pdl_trigger();
    pdl_wait();
    cut_faces_any<L>(p, blockIdx.x);
}
template <int L>
__global__ void __launch_bounds__(CUT_TPB) k_cut_faces_b(const __grid_constant__ SparseTab<CutParams> t) {
    pdl_trigger();
    pdl_wait();
    const int i = tab_find(t.boff, t.n, (int)blockIdx.x);
    cut_faces_any<L>(t.p[i], (int)blockIdx.x - t.boff[i]);
}

// lanes per element: one thread per element once the launch has some 40k
// elements, else a warp per element (measured: 10k elements of one capsule
// pair 16 us with warps against 44 us with threads; 82k elements of eight
// sweep lattices 56 us with threads against 79 us with warps; 655k elements
// of the 64-lattice sweep 0.32 ms against 0.64 ms)
int cut_lanes(long long nfaces) { return nfaces >= 40960 ? 1 : 32; }
int cut_blocks(int nfaces, int lanes) { return (int)(((long long)nfaces * lanes + CUT_TPB - 1) / CUT_TPB); }

cudaError_t launch_cuts(const CutParams &p, cudaStream_t s, int *nl) {
    const int L = cut_lanes(p.nfaces);
    const dim3 g(cut_blocks(p.nfaces, L)), b(CUT_TPB);
    if (L == 1) launch_pdl(k_cut_faces<1>, g, b, s, p);
    else launch_pdl(k_cut_faces<32>, g, b, s, p);
    *nl += 1;
    return cudaGetLastError();
}

cudaError_t launch_cuts_batch(const SparseTab<CutParams> &t, int lanes, cudaStream_t s, int *nl) {
    if (t.n == 0 || t.boff[t.n] == 0) return cudaSuccess;
    const dim3 g((unsigned)t.boff[t.n]), b(CUT_TPB);
    if (lanes == 1) launch_pdl(k_cut_faces_b<1>, g, b, s, t);
    else launch_pdl(k_cut_faces_b<32>, g, b, s, t);
    *nl += 1;
    return cudaGetLastError();
}

// Post-collision population (component c, direction k) of node n, decoded
// (16-bit storage holds the offset from w_k rho of the node).
__device__ __forceinline__ float pop_at(const PrepParams &p, int c, int k, long long n, float rho) {
    const long long i = ((long long)c * Q + k) * p.N + n;
    if (p.prec == P_F16)
        return __half2float(static_cast<const __half *>(p.src)[i]) * F16_INV_SCALE + wgt(k) * rho;
    if (p.prec == P_BF16)
        return __bfloat162float(static_cast<const __nv_bfloat16 *>(p.src)[i]) + wgt(k) * rho;
    return static_cast<const float *>(p.src)[i];
}

// Bounce records for the next streaming, one thread per entry of the cut-link
// list: the population a cut node sent towards the membrane comes back with
// Ladd's term -2 w_k rho (e_k . u_T)/c_s^2 (rho: the node's density = sum of
// its post-collision populations; u_T: velocity of the crossed element, the
// mean of its nodes' velocities); the momentum each bounce exchanges with the element,
// sum_c (2 f*_k - corr), is booked on it (Sec. 3.1, coupling paragraph).  A link
// crossed by several elements has one entry per element: the entry of the
// smallest one (the element kept in tri) writes the record, and a link whose
// crossings cancelled out (even count, cut bit clear) writes none.
__device__ __forceinline__ void cut_prep_body(const PrepParams &p, int bid) {
    const int cnt = min(*p.count, p.capacity);
    for (int i = bid * (int)blockDim.x + (int)threadIdx.x; i < cnt; i += p.blocks * (int)blockDim.x) {
        const int2 e = __ldg(p.list + i);
        const long long n = (long long)((unsigned)e.x >> 5);
        const int k1 = e.x & 31, k = k1 + 1, T = e.y;
        // every load the entry needs is issued before its checks (the
        // addresses are valid for any entry), so the loads overlap
        const uint32_t m = __ldg(p.mask + n);
        const int t = __ldg(p.tri + n * 18 + k1);
        // the node's density: the sum of its post-collision populations equals
        // the density of the step that produced them (BGK conserves mass)
        const float2 dn = __ldg(p.rho + n);
        const float4 u = __ldg(p.uT + T);  // recorded by k_cut_faces
        const float foa = pop_at(p, 0, k, n, dn.x), fob = pop_at(p, 1, k, n, dn.y);
        if (!((m >> k1) & 1u) || t != T) continue;
        int kx, ky, kz;
        ek(k, kx, ky, kz);
        const float eu = kx * u.x + ky * u.y + kz * u.z;
        const float w6 = 6.0f * wgt(k);
        const float ra = p.ref_rho ? 1.f : dn.x, rb = p.ref_rho ? 1.f : dn.y;  // CF_LADD_REF_RHO
        const float ca = w6 * ra * eu, cb = w6 * rb * eu;
        p.rec[n * 18 + (opp(k) - 1)] = make_float2(foa - ca, fob - cb);
        const float sx = (2.0f * foa - ca) + (2.0f * fob - cb);
        if (kx) ft_add(p.FT + 3 * T + 0, kx * sx);
        if (ky) ft_add(p.FT + 3 * T + 1, ky * sx);
        if (kz) ft_add(p.FT + 3 * T + 2, kz * sx);
    }
}

__global__ void __launch_bounds__(256) k_cut_prep(const PrepParams p) {
    pdl_trigger();
    pdl_wait();
    cut_prep_body(p, blockIdx.x);
}
__global__ void __launch_bounds__(256) k_cut_prep_b(const __grid_constant__ SparseTab<PrepParams> t) {
    pdl_trigger();
    pdl_wait();
    const int i = tab_find(t.boff, t.n, (int)blockIdx.x);
    cut_prep_body(t.p[i], (int)blockIdx.x - t.boff[i]);
}

cudaError_t launch_prep(const PrepParams &p, cudaStream_t s, int *nl) {
    launch_pdl(k_cut_prep, dim3((unsigned)p.blocks), dim3(256), s, p);
    *nl += 1;
    return cudaGetLastError();
}

cudaError_t launch_prep_batch(const SparseTab<PrepParams> &t, cudaStream_t s, int *nl) {
    if (t.n == 0 || t.boff[t.n] == 0) return cudaSuccess;
    launch_pdl(k_cut_prep_b, dim3((unsigned)t.boff[t.n]), dim3(256), s, t);
    *nl += 1;
    return cudaGetLastError();
}

}  // namespace cf
