// Membrane phase of the coupled step and cut-link geometry (sm_103a).
//
// All capsules are concatenated: global node and element indices, with the
// owning capsule per element and per node.  One step of the membrane phase
// (Sec. 3.1, Eqs. 6-9, 11) is four short kernels:
//   k_faces     per element: two-step average of the exchanged momentum,
//               Skalak strain forces (Eq. 6), volume gradient terms (Eq. 8),
//               cotangent-Laplacian contributions for the bending energy,
//               FP64 per-capsule area and volume
//   k_vert1     per node: mean-curvature vector and node area, gradients of
//               the bending energy with respect to them; FP64 centroid and
//               integer bounding box per capsule
//   k_bend      per element: back-propagation of the bending energy (Eq. 7)
//   k_vert2     per node: gathers of all element contributions (vertex->element
//               CSR, no atomics), Hertz forces (Eq. 11), node update (Eq. 9),
//               FP64 per-capsule force/torque sums
// plus k_frozen for rigidly translated capsules.  The cut links for the moved
// membrane are then rebuilt by k_cut_clear and k_cut_faces.
#include "cf_common.cuh"
#include <cfloat>

namespace cf {

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
struct d3 { double x, y, z; };
__device__ __forceinline__ d3 ld3d(const double *p, int i) { return {p[3 * i], p[3 * i + 1], p[3 * i + 2]}; }
__device__ __forceinline__ f3 fdiff(d3 a, d3 b) {  // float(a - b), exact difference first
    return {(float)(a.x - b.x), (float)(a.y - b.y), (float)(a.z - b.z)};
}
__device__ __forceinline__ f3 tof(d3 a) { return {(float)a.x, (float)a.y, (float)a.z}; }

// Warp-aggregated FP64 add into per-capsule accumulators: lanes sharing the
// capsule id combine first, one atomic per group.
__device__ __forceinline__ void acc_add(double *acc, int cap, int slot, double v, bool valid) {
    const unsigned full = 0xffffffffu;
    const int key = valid ? cap : -1;
    const unsigned grp = __match_any_sync(full, key);
    const int leader = __ffs(grp) - 1;
    const int lane = threadIdx.x & 31;
    double s = 0.0;
#pragma unroll 4
    for (int src = 0; src < 32; ++src) {  // all lanes shuffle together
        const double o = __shfl_sync(full, v, src);
        if ((grp >> src) & 1u) s += o;
    }
    if (lane == leader && valid) atomicAdd(acc + cap * A_NACC + slot, s);
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

__global__ void k_faces(const MemParams p) {
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = f < p.nfaces;
    const int ff = valid ? f : 0;
    const int cap = p.face_cap[ff];
    const CapDev cp = p.caps[cap];
    const int ia = p.faces[3 * ff], ib = p.faces[3 * ff + 1], ic = p.faces[3 * ff + 2];
    const d3 da = ld3d(p.X, ia), db = ld3d(p.X, ib), dc = ld3d(p.X, ic);
    // element geometry in coordinates local to its first node (translation invariant)
    const f3 a{0.f, 0.f, 0.f}, b = fdiff(db, da), c = fdiff(dc, da);
    float *S = p.fscr + (long long)ff * FS_N;
    double area = 0.0, vol = 0.0;
    if (valid) {
        // two-step average of the momentum exchanged with this element
        const f3 ft = ld3(p.FT, ff), fp = ld3(p.FTprev, ff);
        st3(S + FS_FBAR, 0.5f * (ft + fp));
        st3(p.FTprev + 3 * ff, ft);
        st3(p.FT + 3 * ff, f3{0.f, 0.f, 0.f});
        const f3 u = b - a, w = c - a;
        const f3 nrm = cross(u, w);
        const float Af = 0.5f * sqrtf(dot(nrm, nrm));
        area = Af;
        // volume term in FP64 relative to the first node (translation invariant)
        {
            const double ux = u.x, uy = u.y, uz = u.z, wx = w.x, wy = w.y, wz = w.z;
            const double ax = da.x, ay = da.y, az = da.z;
            // x_a . (x_b x x_c) = x_a . (u x w) + ... ; use (a, a+u, a+w):
            // a.(b x c) = a.((a+u) x (a+w)) = a.(u x w) (a.(a x .) = 0)
            const double cx = uy * wz - uz * wy, cy = uz * wx - ux * wz, cz = ux * wy - uy * wx;
            vol = (ax * cx + ay * cy + az * cz) / 6.0;
        }
        if (cp.mode == 0) {
            // Skalak (Eq. 6): I1 = tr(G0^-1 g) - 2, I2 = det g / det G0 - 1
            const float g11 = dot(u, u), g12 = dot(u, w), g22 = dot(w, w);
            const float m11 = p.refM[3 * ff], m12 = p.refM[3 * ff + 1], m22 = p.refM[3 * ff + 2];
            const float idet = 1.0f / p.refDet[ff];
            const float I1 = m11 * g11 + 2.f * m12 * g12 + m22 * g22 - 2.f;
            const float I2 = (g11 * g22 - g12 * g12) * idet - 1.f;
            const float A0 = p.refA[ff];
            const float dW1 = 0.25f * cp.kS * (2.f * I1 + 2.f);
            const float dW2 = 0.25f * cp.kS * (-2.f + 2.f * cp.C * I2);
            const f3 gb = A0 * (dW1 * (2.f * (m11 * u + m12 * w)) + dW2 * (2.f * idet * (g22 * u - g12 * w)));
            const f3 gc = A0 * (dW1 * (2.f * (m12 * u + m22 * w)) + dW2 * (2.f * idet * (g11 * w - g12 * u)));
            st3(S + FS_SK + 0, gb + gc);
            st3(S + FS_SK + 3, -1.f * gb);
            st3(S + FS_SK + 6, -1.f * gc);
            // volume gradient terms (x_b x x_c etc.); their per-node sums are
            // translation invariant on a closed mesh, so positions are taken
            // relative to the capsule's first node to avoid cancellation
            const d3 o = ld3d(p.X, cp.v0);
            const f3 ra = fdiff(da, o), rb = fdiff(db, o), rc = fdiff(dc, o);
            st3(S + FS_DV + 0, cross(rb, rc));
            st3(S + FS_DV + 3, cross(rc, ra));
            st3(S + FS_DV + 6, cross(ra, rb));
            // bending, first pass: cotangents, Laplacian contributions, A_f/3
            const float cta = cot_only(a, b, c), ctb = cot_only(b, c, a), ctc = cot_only(c, a, b);
            st3(S + FS_L + 0, ctc * (b - a) + ctb * (c - a));
            st3(S + FS_L + 3, cta * (c - b) + ctc * (a - b));
            st3(S + FS_L + 6, ctb * (a - c) + cta * (b - c));
            S[FS_AF3] = Af / 3.f;
            S[FS_COT] = cta; S[FS_COT + 1] = ctb; S[FS_COT + 2] = ctc;
        }
    }
    acc_add(p.acc, cap, A_AREA, area, valid);
    acc_add(p.acc, cap, A_VOL, vol, valid);
}

__global__ void k_vert1(const MemParams p) {
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = v < p.nnodes;
    const int vv = valid ? v : 0;
    const int cap = p.node_cap[vv];
    const CapDev cp = p.caps[cap];
    const d3 x = ld3d(p.X, vv);
    if (valid && cp.mode == 0) {
        f3 L{0.f, 0.f, 0.f};
        float A = 0.f;
        for (int e = p.vf_off[vv]; e < p.vf_off[vv + 1]; ++e) {
            const int ent = p.vf_ent[e];
            const int f = ent / 3, sl = ent % 3;
            const float *S = p.fscr + (long long)f * FS_N;
            L = L + ld3(S + FS_L, sl);
            A += S[FS_AF3];
        }
        // E = kB/8 |L|^2 / A (Eq. 7, H0 = 0): dE/dL and dE/dA
        const float iA = 1.f / A;
        st3(p.vscr + 4 * vv, (0.25f * cp.kB * iA) * L);
        p.vscr[4 * vv + 3] = -0.125f * cp.kB * dot(L, L) * iA * iA;
    }
    acc_add(p.acc, cap, A_CX, x.x, valid);
    acc_add(p.acc, cap, A_CY, x.y, valid);
    acc_add(p.acc, cap, A_CZ, x.z, valid);
    if (valid) {  // bbox: mins [3*ncaps] then maxs [3*ncaps]
        atomicMin(p.bbox + 3 * cap + 0, (int)floor(x.x));
        atomicMin(p.bbox + 3 * cap + 1, (int)floor(x.y));
        atomicMin(p.bbox + 3 * cap + 2, (int)floor(x.z));
        atomicMax(p.bbox + 3 * p.ncaps + 3 * cap + 0, (int)ceil(x.x));
        atomicMax(p.bbox + 3 * p.ncaps + 3 * cap + 1, (int)ceil(x.y));
        atomicMax(p.bbox + 3 * p.ncaps + 3 * cap + 2, (int)ceil(x.z));
    }
}

__global__ void k_bend(const MemParams p) {
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= p.nfaces) return;
    const int cap = p.face_cap[f];
    if (p.caps[cap].mode != 0) return;
    const int ia = p.faces[3 * f], ib = p.faces[3 * f + 1], ic = p.faces[3 * f + 2];
    const d3 pa = ld3d(p.X, ia);
    const f3 a{0.f, 0.f, 0.f}, b = fdiff(ld3d(p.X, ib), pa), c = fdiff(ld3d(p.X, ic), pa);
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
    (void)cta; (void)ctb; (void)ctc;
}

__device__ __forceinline__ float hertz(float xi, float d0, float d) {
    const float o = d0 - d;
    return xi * o * sqrtf(o);
}

__global__ void k_vert2(const MemParams p) {
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = v < p.nnodes;
    const int vv = valid ? v : 0;
    const int cap = p.node_cap[vv];
    const CapDev cp = p.caps[cap];
    const d3 x = ld3d(p.X, vv);
    f3 Fc{0.f, 0.f, 0.f}, Fe{0.f, 0.f, 0.f}, Fi{0.f, 0.f, 0.f};
    if (valid) {
        const bool el = cp.mode == 0;
        f3 dv{0.f, 0.f, 0.f};
        for (int e = p.vf_off[vv]; e < p.vf_off[vv + 1]; ++e) {
            const int ent = p.vf_ent[e];
            const int f = ent / 3, sl = ent % 3;
            const float *S = p.fscr + (long long)f * FS_N;
            Fc = Fc + ld3(S + FS_FBAR, 0);
            if (el) {
                Fe = Fe + ld3(S + FS_SK, sl) + ld3(S + FS_BEND, sl);
                dv = dv + ld3(S + FS_DV, sl);
            }
        }
        Fc = (1.f / 3.f) * Fc;
        if (el) {
            const double V = p.acc[cap * A_NACC + A_VOL];
            const float pre = (float)(-(double)cp.kV * (V - cp.V0) / cp.V0 / 6.0);
            Fe = Fe + pre * dv;
        }
        // Hertz (Eq. 11): substrate plane
        if (p.wall) {
            const float d = (float)(x.z - (double)p.zrep);
            if (d < p.delta0) Fi.z += hertz(p.xi, p.delta0, d);
        }
        // Hertz: nodes of other capsules (bounding boxes prefilter)
        for (int c2 = 0; c2 < p.ncaps; ++c2) {
            if (c2 == cap) continue;
            const int *lo = p.bbox + 3 * c2, *hi = p.bbox + 3 * p.ncaps + 3 * c2;
            if (x.z < lo[2] - p.delta0 || x.z > hi[2] + p.delta0) continue;
            for (int sy = -1; sy <= 1; ++sy)
                for (int sx = -1; sx <= 1; ++sx) {
                    const double ox = sx * p.nx, oy = sy * p.ny;
                    if (x.x + ox < lo[0] - p.delta0 || x.x + ox > hi[0] + p.delta0) continue;
                    if (x.y + oy < lo[1] - p.delta0 || x.y + oy > hi[1] + p.delta0) continue;
                    const CapDev c2d = p.caps[c2];
                    for (int w = c2d.v0; w < c2d.v0 + c2d.nv; ++w) {
                        const d3 y = ld3d(p.X, w);
                        f3 dd = fdiff(x, y);
                        dd.x -= p.nx * floorf(dd.x / p.nx + 0.5f);
                        dd.y -= p.ny * floorf(dd.y / p.ny + 0.5f);
                        const float d = sqrtf(dot(dd, dd));
                        if (d < p.delta0 && d > 0.f) Fi = Fi + (hertz(p.xi, p.delta0, d) / d) * dd;
                    }
                }
        }
    }
    const f3 Ft = Fc + Fe + Fi;
    if (valid) {
        st3(p.Fcpl + 3 * vv, Fc);
        if (cp.mode == 0) {
            const f3 vel = (1.f / cp.mass) * Ft;
            st3(p.V + 3 * vv, vel);
            p.Xn[3 * vv] = x.x + vel.x;
            p.Xn[3 * vv + 1] = x.y + vel.y;
            p.Xn[3 * vv + 2] = x.z + vel.z;
        } else if (cp.mode == 2) {
            st3(p.V + 3 * vv, f3{0.f, 0.f, 0.f});
            p.Xn[3 * vv] = x.x;
            p.Xn[3 * vv + 1] = x.y;
            p.Xn[3 * vv + 2] = x.z;
        }
    }
    // per-capsule FP64 sums: coupling force, its torque about the centroid, total force
    const double icnt = 1.0 / cp.nv;
    const double rx = x.x - p.acc[cap * A_NACC + A_CX] * icnt;
    const double ry = x.y - p.acc[cap * A_NACC + A_CY] * icnt;
    const double rz = x.z - p.acc[cap * A_NACC + A_CZ] * icnt;
    acc_add(p.acc, cap, A_FX, Fc.x, valid);
    acc_add(p.acc, cap, A_FY, Fc.y, valid);
    acc_add(p.acc, cap, A_FZ, Fc.z, valid);
    acc_add(p.acc, cap, A_TX, ry * Fc.z - rz * Fc.y, valid);
    acc_add(p.acc, cap, A_TY, rz * Fc.x - rx * Fc.z, valid);
    acc_add(p.acc, cap, A_TZ, rx * Fc.y - ry * Fc.x, valid);
    acc_add(p.acc, cap, A_FTX, Ft.x, valid);
    acc_add(p.acc, cap, A_FTY, Ft.y, valid);
    acc_add(p.acc, cap, A_FTZ, Ft.z, valid);
}

__global__ void k_frozen(const MemParams p) {
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= p.nnodes) return;
    const int cap = p.node_cap[v];
    const CapDev cp = p.caps[cap];
    if (cp.mode != 1) return;
    const double s = 1.0 / ((double)cp.mass * cp.nv);
    const f3 vel{(float)(p.acc[cap * A_NACC + A_FTX] * s), (float)(p.acc[cap * A_NACC + A_FTY] * s),
                 (float)(p.acc[cap * A_NACC + A_FTZ] * s)};
    st3(p.V + 3 * v, vel);
    const d3 x = ld3d(p.X, v);
    p.Xn[3 * v] = x.x + vel.x;
    p.Xn[3 * v + 1] = x.y + vel.y;
    p.Xn[3 * v + 2] = x.z + vel.z;
}

cudaError_t launch_membrane(const MemParams &p, bool any_frozen, cudaStream_t s, int *nl) {
    const int bt = 128;
    const int gf = (p.nfaces + bt - 1) / bt, gv = (p.nnodes + bt - 1) / bt;
    k_faces<<<gf, bt, 0, s>>>(p);
    k_vert1<<<gv, bt, 0, s>>>(p);
    k_bend<<<gf, bt, 0, s>>>(p);
    k_vert2<<<gv, bt, 0, s>>>(p);
    *nl += 4;
    if (any_frozen) { k_frozen<<<gv, bt, 0, s>>>(p); *nl += 1; }
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

// segment P->Q crosses triangle ABC (sign(0) = + convention)
__device__ bool seg_tri(f3 P, f3 Qp, f3 A, f3 B, f3 C) {
    const float EPS = 1e-4f;
    const float dp = orient_f(A, B, C, P), dq = orient_f(A, B, C, Qp);
    if (fabsf(dp) > EPS && fabsf(dq) > EPS) {
        if ((dp >= 0.f) == (dq >= 0.f)) return false;
        const float s1 = orient_f(P, Qp, A, B), s2 = orient_f(P, Qp, B, C), s3 = orient_f(P, Qp, C, A);
        if (fabsf(s1) > EPS && fabsf(s2) > EPS && fabsf(s3) > EPS)
            return ((s1 >= 0.f) == (s2 >= 0.f)) && ((s2 >= 0.f) == (s3 >= 0.f));
    }
    const double Dp = orient_d(A, B, C, P), Dq = orient_d(A, B, C, Qp);
    if ((Dp >= 0.0) == (Dq >= 0.0)) return false;
    const double S1 = orient_d(P, Qp, A, B), S2 = orient_d(P, Qp, B, C), S3 = orient_d(P, Qp, C, A);
    return ((S1 >= 0.0) == (S2 >= 0.0)) && ((S2 >= 0.0) == (S3 >= 0.0));
}

__global__ void k_cut_clear(const CutParams p) {
    const int prev = *p.prev_count;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < prev && i < p.capacity;
         i += gridDim.x * blockDim.x) {
        const int n = p.prev_list[i];
        p.mask[n] = 0u;
        p.touched[n] = 0u;
#pragma unroll
        for (int k = 0; k < 18; ++k) p.tri[(long long)n * 18 + k] = 0x7fffffff;
    }
}

__device__ __forceinline__ void mark(const CutParams &p, int x, int y, int z, int k, int T) {
    const long long n = ((long long)wrapi(z, p.nz) * p.ny + wrapi(y, p.ny)) * p.nx + wrapi(x, p.nx);
    atomicXor(p.mask + n, 1u << (k - 1));
    atomicMin(p.tri + n * 18 + (k - 1), T);
    if (atomicExch(p.touched + n, 1u) == 0u) {
        const int idx = atomicAdd(p.count, 1);
        if (idx < p.capacity) p.list[idx] = (int)n;
        else atomicOr(p.status, ST_OVERFLOW);
    }
}

// one warp per element: all links (x, x+e_k), k in the nine positive
// directions, starting within one unit of the element's bounding box
__global__ void k_cut_faces(const CutParams p) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp >= p.nfaces) return;
    const int T = warp;
    const f3 A = tof(ld3d(p.X, p.faces[3 * T])), B = tof(ld3d(p.X, p.faces[3 * T + 1])),
             C = tof(ld3d(p.X, p.faces[3 * T + 2]));
    const int lx = (int)ceilf(fminf(A.x, fminf(B.x, C.x)) - 1.f), hx = (int)floorf(fmaxf(A.x, fmaxf(B.x, C.x)) + 1.f);
    const int ly = (int)ceilf(fminf(A.y, fminf(B.y, C.y)) - 1.f), hy = (int)floorf(fmaxf(A.y, fmaxf(B.y, C.y)) + 1.f);
    const int lz = (int)ceilf(fminf(A.z, fminf(B.z, C.z)) - 1.f), hz = (int)floorf(fmaxf(A.z, fmaxf(B.z, C.z)) + 1.f);
    const int sx = hx - lx + 1, sy = hy - ly + 1, sz = hz - lz + 1;
    const int total = sx * sy * sz * 9;
    constexpr int POS[9] = {1, 3, 5, 7, 9, 11, 13, 15, 17};
    for (int t = lane; t < total; t += 32) {
        const int d = t % 9;
        const int node = t / 9;
        const int x = lx + node % sx, y = ly + (node / sx) % sy, z = lz + node / (sx * sy);
        int k = 1, kx = 0, ky = 0, kz = 0;
#pragma unroll
        for (int j = 0; j < 9; ++j)
            if (j == d) { k = POS[j]; kx = ex(POS[j]); ky = ey(POS[j]); kz = ez(POS[j]); }
        if (p.wall && (wrapi(z, p.nz) == 0 || wrapi(z + kz, p.nz) == 0)) continue;
        const f3 P{(float)x, (float)y, (float)z};
        const f3 Qp{(float)(x + kx), (float)(y + ky), (float)(z + kz)};
        if (seg_tri(P, Qp, A, B, C)) {
            mark(p, x, y, z, k, T);
            mark(p, x + kx, y + ky, z + kz, opp(k), T);
        }
    }
}

cudaError_t launch_cuts(const CutParams &p, int prev_hint, cudaStream_t s, int *nl) {
    (void)prev_hint;
    k_cut_clear<<<152, 256, 0, s>>>(p);
    const long long threads = (long long)p.nfaces * 32;
    k_cut_faces<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(p);
    *nl += 2;
    return cudaGetLastError();
}

}  // namespace cf
