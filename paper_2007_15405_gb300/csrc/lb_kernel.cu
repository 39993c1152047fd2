// Two-component Shan-Chen lattice Boltzmann step (sm_103a), two passes.
//
// The lattice part of a coupled time step (Sec. 3.1): pull-streaming of both
// components with half-way bounce-back on the substrate and on membrane-cut
// links (Ladd's moving-wall term), the momentum those bounces exchange with
// the membrane elements, the densities and pseudopotentials
// psi = 1 - exp(-rho), the Shan-Chen force (Eq. 10) with the interior/exterior
// decoupling, and the BGK collision (Eqs. 4-5) with the velocity-shift forcing.
//
//   k_density     per node: sum the 38 streamed populations, write
//                 (rho_A, rho_B) and (psi_A, psi_B) as two float2, and for
//                 tau = 1 the total momentum J as a float4
//   k_collide_eq  tau = 1: read rho, psi, J of the node and the
//                 pseudopotentials of the 18 neighbours (float2, L1/L2
//                 resident), Shan-Chen force, velocity shift, store the
//                 equilibria (BGK with tau = 1)
//   k_collide     any tau: gather the 38 streamed populations again, then as
//                 above with the BGK relaxation of the pulled populations
//
// Layout: populations f[c][i][z][y][x] (float, or 16-bit offsets with float
// rest populations), two buffers (src -> dst); threads map to x so every
// gather is a coalesced row.  Both passes are barrier-free.  DRAM traffic per
// node update with tau = 1: 152 B of population reads and 32 B of density,
// pseudopotential and momentum writes in the density pass, 36 B of reads and
// 152 B of population writes in the collide pass.  Gather addresses are the
// node index plus per-direction offsets with the periodic wrap folded into
// per-node deltas.
//
// With the diffuse-interface coupling (CF_IBM, own instantiations of the
// single-lattice collide passes) the collide pass also adds the membrane
// force spread to the node, shared by the components in proportion to their
// densities, and writes the fluid velocity the membrane nodes move with; the
// lattice then sees no cut link.
#include "cf_common.cuh"
#include "../../include/capfilm.h"

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <math_constants.h>
#include <algorithm>
#include <cstdint>

namespace cf {

constexpr int BX = 32, BY = 4;  // thread block: one row segment of 32 x 4 rows
// resident blocks per SM the collide pass is compiled for (its register cap)
#ifndef CF_COLLIDE_MINB
#define CF_COLLIDE_MINB 5
#endif
#ifndef CF_COLLIDE16_MINB  // the same for 16-bit storage
#define CF_COLLIDE16_MINB 4
#endif

__device__ __forceinline__ float psi_of(float r) { return -expm1f(-r); }

// Population storage.  Float stores f_i itself.  Half and bfloat16 store,
// for the 18 moving directions, the offset g_i = f_i - w_i rho from the rest
// equilibrium of the node that wrote it (rho from that step's density array):
// the offsets are O(w rho |u|), so 16 bits resolve f_i far better than
// storing f_i directly, and the population traffic is halved.  The offsets
// are rounded stochastically (a counter-based hash of node, step and
// direction picks the rounding): at a stationary interface the offsets repeat
// from step to step, and round-to-nearest errors would add up linearly.  The
// rest population stays in float and takes the node's mass balance after the
// moving offsets are rounded, so every node stores exactly its mass.
template <typename T> struct Pop;
template <> struct Pop<float> {
    static constexpr bool shifted = false;
    __device__ static float ld(const float *p) { return __ldg(p); }
    // store v, return the value stored
    __device__ static float st(float *p, float v, uint32_t) { *p = v; return v; }
};
__device__ __forceinline__ uint32_t mix32(uint32_t x) {
    x ^= x >> 16; x *= 0x7feb352du; x ^= x >> 15; x *= 0x846ca68bu; x ^= x >> 16;
    return x;
}
// stochastic rounding of v to bfloat16: random bits below its 8-bit mantissa,
// then truncation of the magnitude
__device__ __forceinline__ __nv_bfloat16 sr_bf16(float v, uint32_t r) {
    uint32_t b = __float_as_uint(v);
    if ((b & 0x7f800000u) != 0x7f800000u) b += r & 0xffffu;
    return __ushort_as_bfloat16((unsigned short)(b >> 16));
}
// stochastic rounding of v to half: random bits below its 10-bit mantissa
// (13 float bits in the normal range), then round toward zero
__device__ __forceinline__ __half sr_f16(float v, uint32_t r) {
    uint32_t b = __float_as_uint(v);
    if ((b & 0x7f800000u) != 0x7f800000u) b = (b + (r & 0x1fffu)) & ~0x1fffu;
    return __float2half_rz(__uint_as_float(b));
}
// Two offsets at once: cvt.rs rounds x into the high and y into the low
// 16 bits of the result, stochastically, with the high and low 16 bits of r
// as their random bits (unbiased: measured round-up frequencies equal the
// fractional parts).  put2 stores the halves, val2 returns (x, y) as stored.
template <> struct Pop<__half> {
    static constexpr bool shifted = true;
    static constexpr float scale = F16_SCALE, inv_scale = F16_INV_SCALE;  // stored = offset x scale
    __device__ static float ld(const __half *p) { return __half2float(__ldg(p)) * F16_INV_SCALE; }
    __device__ static float st(__half *p, float v, uint32_t r) {
        const __half h = sr_f16(v * F16_SCALE, r);
        *p = h;
        return __half2float(h) * F16_INV_SCALE;
    }
    __device__ static uint32_t cvt2(float x, float y, uint32_t r) {
        uint32_t d;
        asm("cvt.rs.satfinite.f16x2.f32 %0, %1, %2, %3;"
            : "=r"(d) : "f"(x * F16_SCALE), "f"(y * F16_SCALE), "r"(r));
        return d;
    }
    __device__ static float2 val2(uint32_t d) {
        const float2 f = __half22float2(*reinterpret_cast<const __half2 *>(&d));  // (low, high)
        return make_float2(f.y * F16_INV_SCALE, f.x * F16_INV_SCALE);
    }
    // the same with x and y already scaled, and the stored values in scaled units
    __device__ static uint32_t cvt2s(float xs, float ys, uint32_t r) {
        uint32_t d;
        asm("cvt.rs.satfinite.f16x2.f32 %0, %1, %2, %3;" : "=r"(d) : "f"(xs), "f"(ys), "r"(r));
        return d;
    }
    __device__ static float2 raw2(uint32_t d) {
        const float2 f = __half22float2(*reinterpret_cast<const __half2 *>(&d));
        return make_float2(f.y, f.x);
    }
    __device__ static void put2(__half *px, __half *py, uint32_t d) {
        *reinterpret_cast<unsigned short *>(px) = (unsigned short)(d >> 16);
        *reinterpret_cast<unsigned short *>(py) = (unsigned short)(d & 0xffffu);
    }
};
template <> struct Pop<__nv_bfloat16> {
    static constexpr bool shifted = true;
    static constexpr float scale = 1.0f, inv_scale = 1.0f;
    __device__ static float ld(const __nv_bfloat16 *p) { return __bfloat162float(__ldg(p)); }
    __device__ static float st(__nv_bfloat16 *p, float v, uint32_t r) {
        const __nv_bfloat16 h = sr_bf16(v, r);
        *p = h;
        return __bfloat162float(h);
    }
    __device__ static uint32_t cvt2(float x, float y, uint32_t r) {
        uint32_t d;
        asm("cvt.rs.satfinite.bf16x2.f32 %0, %1, %2, %3;" : "=r"(d) : "f"(x), "f"(y), "r"(r));
        return d;
    }
    __device__ static float2 val2(uint32_t d) {  // a bfloat16 is the high half of a float
        return make_float2(__uint_as_float(d & 0xffff0000u), __uint_as_float(d << 16));
    }
    __device__ static uint32_t cvt2s(float x, float y, uint32_t r) { return cvt2(x, y, r); }
    __device__ static float2 raw2(uint32_t d) { return val2(d); }
    __device__ static void put2(__nv_bfloat16 *px, __nv_bfloat16 *py, uint32_t d) {
        *reinterpret_cast<unsigned short *>(px) = (unsigned short)(d >> 16);
        *reinterpret_cast<unsigned short *>(py) = (unsigned short)(d & 0xffffu);
    }
};

// Offsets from node n to its neighbour at -e in each axis (periodic).
struct Deltas {
    int n;                 // node index
    int dxm, dxp;          // to x-1, x+1
    int dym, dyp;          // to y-1, y+1 (in nodes)
    int dzm, dzp;          // to z-1, z+1 (in nodes)
    bool wlo, whi;         // z-1 / z+1 is the substrate
};

__device__ __forceinline__ Deltas deltas(const LBParams &p, int x, int y, int z) {
    Deltas d;
    const int nx = p.nx, ny = p.ny, nxy = p.nx * p.ny;
    d.n = (z * ny + y) * nx + x;
    d.dxm = x == 0 ? nx - 1 : -1;
    d.dxp = x == nx - 1 ? -(nx - 1) : 1;
    d.dym = y == 0 ? (ny - 1) * nx : -nx;
    d.dyp = y == ny - 1 ? -(ny - 1) * nx : nx;
    d.dzm = z == 0 ? (p.nz - 1) * nxy : -nxy;
    d.dzp = z == p.nz - 1 ? -(p.nz - 1) * nxy : nxy;
    d.wlo = p.wall && z == 1;
    d.whi = p.wall && z == p.nz - 1;
    return d;
}

// offset of node x + s (s in {-1,0,1}^3) relative to n
__device__ __forceinline__ int nb_off(const Deltas &d, int sx, int sy, int sz) {
    int o = 0;
    o += sx == -1 ? d.dxm : sx == 1 ? d.dxp : 0;
    o += sy == -1 ? d.dym : sy == 1 ? d.dyp : 0;
    o += sz == -1 ? d.dzm : sz == 1 ? d.dzp : 0;
    return o;
}

// offset of the source of pulled direction i (node x - e_i, or the node's own
// opposite population where x - e_i is the substrate), relative to src + n
__device__ __forceinline__ int src_off(const Deltas &d, int N, int i) {
    if ((ez(i) == 1 && d.wlo) || (ez(i) == -1 && d.whi)) return opp(i) * N;
    return i * N + nb_off(d, -ex(i), -ey(i), -ez(i));
}
// node offset of that source
__device__ __forceinline__ int src_node_off(const Deltas &d, int i) {
    if ((ez(i) == 1 && d.wlo) || (ez(i) == -1 && d.whi)) return 0;
    return nb_off(d, -ex(i), -ey(i), -ez(i));
}

// Post-streaming populations of the node: coalesced gathers, then the
// bounce-back values of its membrane-cut links.
template <typename T>
__device__ __forceinline__ uint32_t pull(const LBParams &p, const Deltas &d, float (&fa)[Q],
                                         float (&fb)[Q]) {
    const int N = (int)p.N;
    const T *sA = static_cast<const T *>(p.src) + d.n;
    const T *sB = static_cast<const T *>(p.src) + (long long)Q * N + d.n;
    const uint32_t m = __ldg(p.mask + d.n);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        if (Pop<T>::shifted && i == 0) {  // rest populations are kept in float
            fa[0] = __ldg(p.src0 + d.n);
            fb[0] = __ldg(p.src0 + N + d.n);
            continue;
        }
        const int o = src_off(d, N, i);
        fa[i] = Pop<T>::ld(sA + o);
        fb[i] = Pop<T>::ld(sB + o);
        if (Pop<T>::shifted) {  // decode with the density of the source node
            const float2 r = __ldg(p.rho_src + d.n + src_node_off(d, i));
            fa[i] += wgt(i) * r.x;
            fb[i] += wgt(i) * r.y;
        }
    }
    if (m) {
        // membrane-cut links: the bounced populations (Ladd's moving-wall term
        // included) were prepared for this step by k_cut_prep
        const float2 *R = p.rec + (long long)d.n * 18;
#pragma unroll
        for (int k = 1; k < Q; ++k) {
            if ((m >> (k - 1)) & 1u) {
                const float2 v = __ldg(R + opp(k) - 1);
                fa[opp(k)] = v.x;
                fb[opp(k)] = v.y;
            }
        }
    }
    return m;
}

// z range of the fluid planes a thread walks (grid.z splits the column).
// REV maps the blocks in reverse order: the collide pass then starts on the
// tiles the density pass touched last (still in L2), and the next density pass
// starts on the tiles the collide pass wrote last.
template <bool REV = false>
__device__ __forceinline__ bool node_of(const LBParams &p, int &x, int &y, int &z) {
    const int bx = REV ? (int)(gridDim.x - 1 - blockIdx.x) : (int)blockIdx.x;
    const int by = REV ? (int)(gridDim.y - 1 - blockIdx.y) : (int)blockIdx.y;
    const int bz = REV ? (int)(gridDim.z - 1 - blockIdx.z) : (int)blockIdx.z;
    x = bx * BX + threadIdx.x;
    y = by * BY + threadIdx.y;
    z = p.zlo + bz;
    return x < p.nx && y < p.ny;
}

// Density pass of one node: streamed populations -> rho, psi, and with MOM the
// total momentum J = sum_c sum_i f_i^c e_i for the tau = 1 collision.  Returns
// rho_A if A is the majority there, else 0 (the node's share of the drying sum).
template <typename T, bool MOM = false>
__device__ __forceinline__ float density_node(const LBParams &p, const Deltas &d) {
    float fa[Q], fb[Q];
    pull<T>(p, d, fa, fb);
    float ra = 0.f, rb = 0.f;
#pragma unroll
    for (int i = 0; i < Q; ++i) { ra += fa[i]; rb += fb[i]; }
    p.rho[d.n] = make_float2(ra, rb);
    p.psi[d.n] = make_float2(psi_of(ra), psi_of(rb));
    if (MOM) {
        float j[3] = {0.f, 0.f, 0.f};
#pragma unroll
        for (int i = 1; i < Q; i += 2) {  // opposite pairs (i, i+1), both components
            const float dj = (fa[i] - fa[i + 1]) + (fb[i] - fb[i + 1]);
            j[0] += ex(i) * dj; j[1] += ey(i) * dj; j[2] += ez(i) * dj;
        }
        p.J[d.n] = make_float4(j[0], j[1], j[2], 0.f);
    }
    return ra > rb ? ra : 0.f;
}

// Drying: the sum of rho_A over the A-majority nodes.  Each block of the
// density pass writes its partial sum; the last block to finish adds the
// partials in index order (so the result does not depend on the order the
// blocks ran in) and writes eps = dm / sum, at most 1, for the collide pass.
__device__ __forceinline__ void dry_reduce(const LBParams &p, float s) {
    __shared__ double part[BY];
    __shared__ bool last;
    double v = s;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (threadIdx.x == 0) part[threadIdx.y] = v;  // a block row is one warp
    __syncthreads();
    const unsigned nb = gridDim.x * gridDim.y * gridDim.z;
    if (threadIdx.x == 0 && threadIdx.y == 0) {
        double b = 0.0;
        for (int k = 0; k < BY; ++k) b += part[k];
        p.dry_part[(blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x] = b;
        __threadfence();
        last = atomicAdd(p.dry_ctr, 1u) == nb - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double a = 0.0;
    for (unsigned i = threadIdx.y * BX + threadIdx.x; i < nb; i += BX * BY) a += __ldcg(p.dry_part + i);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    __syncthreads();
    if (threadIdx.x == 0) part[threadIdx.y] = a;
    __syncthreads();
    if (threadIdx.x == 0 && threadIdx.y == 0) {
        double S = 0.0;
        for (int k = 0; k < BY; ++k) S += part[k];
        *p.dry_eps = S > 0.0 ? (float)fmin(1.0, p.dry_dm / S) : 0.f;
        *p.dry_ctr = 0u;  // ready for the next step
    }
}

// resident blocks per SM the density pass is compiled for: its 38 gathers are
// issued back to back, so the register cap sets how many nodes are in flight
#ifndef CF_DENSITY_MINB
#define CF_DENSITY_MINB 8
#endif
#ifndef CF_DENSITY_MOM_MINB  // the same when it also sums the momentum
#define CF_DENSITY_MOM_MINB 6
#endif

// DRY: also the drying sum (the whole block must reach the reduction);
// MOM: also the total momentum (tau = 1 collision)
template <typename T, bool DRY = false, bool MOM = false>
__global__ void __launch_bounds__(BX *BY, MOM ? CF_DENSITY_MOM_MINB : CF_DENSITY_MINB) k_density(const LBParams p) {
    pdl_trigger();
    pdl_wait();
    if (Pop<T>::shifted && blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0 &&
        threadIdx.x == 0 && threadIdx.y == 0)
        atomicAdd(p.step_ctr, 1u);  // read by the collide pass that follows
    int x, y, z;
    if (!DRY) {
        if (!node_of(p, x, y, z)) return;
        for (; z < p.zhi; z += gridDim.z) density_node<T, MOM>(p, deltas(p, x, y, z));
        return;
    }
    float s = 0.f;
    if (node_of(p, x, y, z))
        for (; z < p.zhi; z += gridDim.z) s += density_node<T, MOM>(p, deltas(p, x, y, z));
    dry_reduce(p, s);
}

// Shan-Chen force on both components at a node (Eq. 10 with G^{AB} = G^{BA} = G,
// G^{AA} = G^{BB} = 0), with the decoupling across cut and substrate links:
// there the partner's pseudopotential comes from the mean density over this
// node and its neighbours reached through uncut fluid links (on a membrane
// link plus the capsule's wetting offset, +wet for A and -wet for B), and
// the reaction goes to the crossed element.
__device__ __forceinline__ void sc_force(const LBParams &p, const Deltas &d, uint32_t m, float ra, float rb,
                                         float pa, float pb, float (&FA)[3], float (&FB)[3]) {
    const int n = d.n;
    // sum_k w_k psi'(x+e_k) e_k, summed over opposite pairs (k, k+1) as
    // w_k e_k (psi'(x+e_k) - psi'(x-e_k)): the difference of two nearby
    // pseudopotentials is exact in float, so the rounding error of the sum
    // scales with the (small) gradient instead of the pseudopotentials
    float sa[3] = {0.f, 0.f, 0.f}, sb[3] = {0.f, 0.f, 0.f};
    if (!m && !d.wlo && !d.whi) {
#pragma unroll
        for (int k = 1; k < Q; k += 2) {
            const float2 q1 = __ldg(p.psi + n + nb_off(d, ex(k), ey(k), ez(k)));
            const float2 q2 = __ldg(p.psi + n + nb_off(d, -ex(k), -ey(k), -ez(k)));
            const float da = q1.x - q2.x, db = q1.y - q2.y;
            sa[0] += wgt(k) * ex(k) * da; sa[1] += wgt(k) * ey(k) * da; sa[2] += wgt(k) * ez(k) * da;
            sb[0] += wgt(k) * ex(k) * db; sb[1] += wgt(k) * ey(k) * db; sb[2] += wgt(k) * ez(k) * db;
        }
    } else {
        // partner densities across a cut or substrate link: mean over this
        // node and its neighbours reached through uncut fluid links (with
        // CF_PARTNER_MIRROR the node's own densities)
        float ia = ra, ib = rb, cnt = 1.f;
        if (!(p.flags & CF_PARTNER_MIRROR)) {
#pragma unroll
            for (int k = 1; k < Q; ++k) {
                const bool solid = (ez(k) == 1 && d.whi) || (ez(k) == -1 && d.wlo);
                const bool cut = (m >> (k - 1)) & 1u;
                if (!solid && !cut) {
                    const float2 q = __ldg(p.rho + n + nb_off(d, ex(k), ey(k), ez(k)));
                    ia += q.x; ib += q.y; cnt += 1.f;
                }
            }
        }
        const float ma = ia / cnt, mb = ib / cnt;
        const float qa_eff = psi_of(ma), qb_eff = psi_of(mb);
        float qA[Q], qB[Q];  // partner pseudopotentials per direction
#pragma unroll
        for (int k = 1; k < Q; ++k) {
            const bool solid = (ez(k) == 1 && d.whi) || (ez(k) == -1 && d.wlo);
            const bool cut = (m >> (k - 1)) & 1u;
            float qa, qb;
            if (solid || cut) {
                qa = qa_eff; qb = qb_eff;
                if (cut && !solid) {
                    const int el = __ldg(p.tri + (long long)n * 18 + (k - 1));
                    if (p.wet_el) {
                        // wetting of the crossed element's capsule: offset of the
                        // interpolated densities, +wet for A and -wet for B
                        const float w = __ldg(p.wet_el + el);
                        if (w != 0.f) { qa = psi_of(ma + w); qb = psi_of(mb - w); }
                    }
                    // reaction of the decoupled interaction on the crossed element
                    const float r = p.G * wgt(k) * (pa * qb + pb * qa);
                    if (ex(k)) ft_add(p.FT + 3 * el + 0, ex(k) * r);
                    if (ey(k)) ft_add(p.FT + 3 * el + 1, ey(k) * r);
                    if (ez(k)) ft_add(p.FT + 3 * el + 2, ez(k) * r);
                }
            } else {
                const float2 q = __ldg(p.psi + n + nb_off(d, ex(k), ey(k), ez(k)));
                qa = q.x; qb = q.y;
            }
            qA[k] = qa; qB[k] = qb;
        }
#pragma unroll
        for (int k = 1; k < Q; k += 2) {
            const float da = qA[k] - qA[k + 1], db = qB[k] - qB[k + 1];
            sa[0] += wgt(k) * ex(k) * da; sa[1] += wgt(k) * ey(k) * da; sa[2] += wgt(k) * ez(k) * da;
            sb[0] += wgt(k) * ex(k) * db; sb[1] += wgt(k) * ey(k) * db; sb[2] += wgt(k) * ez(k) * db;
        }
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        FA[a] = -p.G * pa * sb[a];
        FB[a] = -p.G * pb * sa[a];
    }
}

// Diffuse-interface coupling (CF_IBM): the membrane force spread to node n
// acts on the fluid as a body force, shared by the components in proportion
// to their densities.  The accumulator is cleared for the next spreading.
// Only in blocks the spreading reached (elsewhere the accumulator is zero).
__device__ __forceinline__ bool ibm_reached(const LBParams &p, int n) {
    return p.fibm && __ldg(ibm_flags(p.uphys, p.N) + (n >> 5));
}
// The loads are issued with the node's own loads, ahead of the Shan-Chen
// stencil's gathers (ibm_load); the force is added after it (ibm_apply).
struct IbmForce { long long f[3]; };
__device__ __forceinline__ IbmForce ibm_load(const LBParams &p, int n) {
    const long long *f = p.fibm + n;
    return {{f[0], f[p.N], f[2 * p.N]}};
}
__device__ __forceinline__ void ibm_apply(const LBParams &p, int n, float ra, float rb, const IbmForce &q,
                                          float (&FA)[3], float (&FB)[3]) {
    long long *f = p.fibm + n;
    f[0] = 0; f[p.N] = 0; f[2 * p.N] = 0;
    const float sa = ra / (ra + rb), sb = rb / (ra + rb);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float F = ft_val(q.f[a]);
        FA[a] += sa * F;
        FB[a] += sb * F;
    }
}

// Post-collision populations of node n from the equilibria at (rho, u^eq)
// (Eq. 5): BGK relaxation of the pulled fa, fb, or with EQ (tau = 1 for both
// components) the equilibria themselves.  Float storage: the rest population
// takes the mass balance of the equilibria.  16-bit storage: offsets from w_i
// rho, stochastically rounded, and the float rest population takes what the
// rounded moving populations leave of the mass.  With DRY, an A-majority node
// keeps 1 - eps of its A populations and adds eps rho_A w_i to its B ones.
template <typename T, bool DRY, bool EQ>
__device__ __forceinline__ void store_post(const LBParams &p, int n, float ra, float rb, const float (&ua)[3],
                                           const float (&ub)[3], const float (&fa)[Q], const float (&fb)[Q]) {
    float ca = 1.f, cb = 0.f;  // drying: A kept, B gained per unit weight
    if (DRY && ra > rb) {
        const float e = __ldg(p.dry_eps);
        ca = 1.f - e;
        cb = (p.flags & CF_DRY_REMOVE) ? 0.f : e * ra;  // removed, or turned into B
    }
    const float ka = 1.0f - 1.5f * (ua[0] * ua[0] + ua[1] * ua[1] + ua[2] * ua[2]);
    const float kb = 1.0f - 1.5f * (ub[0] * ub[0] + ub[1] * ub[1] + ub[2] * ub[2]);
    const int N = (int)p.N;
    T *__restrict__ dA = static_cast<T *>(p.dst) + n;
    T *__restrict__ dB = static_cast<T *>(p.dst) + (long long)Q * N + n;
    const float ta = p.itau[0], tb = p.itau[1];
    // Eq. 5 for opposite pairs: f^eq_{i,i+1} = w rho (ka + 4.5 eu^2 +- 3 eu); the
    // rest population takes the mass balance (sum_i f^eq_i = rho) so that the
    // float32 weights (which sum to 1 + 1.5e-8) create no mass
    float qa0 = ra, qb0 = rb;
    if constexpr (!Pop<T>::shifted) {
#pragma unroll
        for (int i = 1; i < Q; i += 2) {
            const float eua = ex(i) * ua[0] + ey(i) * ua[1] + ez(i) * ua[2];
            const float eub = ex(i) * ub[0] + ey(i) * ub[1] + ez(i) * ub[2];
            const float wa = wgt(i) * ra, wb = wgt(i) * rb;
            const float sa_ = wa * (ka + 4.5f * eua * eua), sb_ = wb * (kb + 4.5f * eub * eub);
            const float qa1 = sa_ + 3.0f * wa * eua, qa2 = sa_ - 3.0f * wa * eua;
            const float qb1 = sb_ + 3.0f * wb * eub, qb2 = sb_ - 3.0f * wb * eub;
            qa0 -= qa1 + qa2;
            qb0 -= qb1 + qb2;
            float va1 = EQ ? qa1 : fa[i] - (fa[i] - qa1) * ta, va2 = EQ ? qa2 : fa[i + 1] - (fa[i + 1] - qa2) * ta;
            float vb1 = EQ ? qb1 : fb[i] - (fb[i] - qb1) * tb, vb2 = EQ ? qb2 : fb[i + 1] - (fb[i + 1] - qb2) * tb;
            if (DRY) {
                va1 *= ca; va2 *= ca;
                vb1 += wgt(i) * cb; vb2 += wgt(i) * cb;
            }
            Pop<T>::st(dA + i * N, va1, 0u);
            Pop<T>::st(dA + (i + 1) * N, va2, 0u);
            Pop<T>::st(dB + i * N, vb1, 0u);
            Pop<T>::st(dB + (i + 1) * N, vb2, 0u);
        }
        float va0 = EQ ? qa0 : fa[0] - (fa[0] - qa0) * ta, vb0 = EQ ? qb0 : fb[0] - (fb[0] - qb0) * tb;
        if (DRY) {
            va0 *= ca;
            vb0 += wgt(0) * cb;
        }
        Pop<T>::st(dA, va0, 0u);
        Pop<T>::st(dB, vb0, 0u);
    } else if constexpr (EQ && !DRY) {
        // tau = 1, no drying: the offsets f^eq_i - w_i rho = w_i rho (kappa +
        // 4.5 eu^2 +- 3 eu), kappa = -1.5 u^2, computed directly (no
        // cancellation against w_i rho) with the storage scale folded into
        // w_i rho; stochastically rounded as below.  The rest population takes
        // the mass balance rho - sum_i w_i rho - sum_i stored offsets, the
        // weight sum being 12 w_1 (the float weights: w_1 = 1/18, w_7 = w_1 / 2
        // exactly), so the rounding of w_1 rho is unbiased.
        uint32_t rs = mix32((uint32_t)n * 0x9e3779b9u ^ mix32(*p.step_ctr));
        const float S = Pop<T>::scale;
        const float kA = -1.5f * (ua[0] * ua[0] + ua[1] * ua[1] + ua[2] * ua[2]);
        const float kB = -1.5f * (ub[0] * ub[0] + ub[1] * ub[1] + ub[2] * ub[2]);
        const float raS = ra * S, rbS = rb * S;
        float sumA = 0.f, sumB = 0.f;  // stored offsets, scaled
#pragma unroll
        for (int i = 1; i < Q; i += 2) {
            const float eua = ex(i) * ua[0] + ey(i) * ua[1] + ez(i) * ua[2];
            const float eub = ex(i) * ub[0] + ey(i) * ub[1] + ez(i) * ub[2];
            const float waS = wgt(i) * raS, wbS = wgt(i) * rbS;
            const float ca = kA + 4.5f * eua * eua, cb = kB + 4.5f * eub * eub;
            const float ta = 3.0f * eua, tb = 3.0f * eub;
            rs = rs * 1664525u + 1013904223u;
            const uint32_t hA = Pop<T>::cvt2s(waS * (ca + ta), waS * (ca - ta), rs ^ (rs >> 16));
            rs = rs * 1664525u + 1013904223u;
            const uint32_t hB = Pop<T>::cvt2s(wbS * (cb + tb), wbS * (cb - tb), rs ^ (rs >> 16));
            Pop<T>::put2(dA + i * N, dA + (i + 1) * N, hA);
            Pop<T>::put2(dB + i * N, dB + (i + 1) * N, hB);
            const float2 sA = Pop<T>::raw2(hA), sB = Pop<T>::raw2(hB);
            sumA += sA.x + sA.y;
            sumB += sB.x + sB.y;
        }
        const float w1 = wgt(1);
        p.dst0[n] = (ra - 12.0f * (w1 * ra)) - sumA * Pop<T>::inv_scale;
        p.dst0[N + n] = (rb - 12.0f * (w1 * rb)) - sumB * Pop<T>::inv_scale;
    } else {
        // 16-bit offsets from w_i rho, stochastically rounded; the float rest
        // population takes what the rounded moving populations leave of the mass
        uint32_t rs = mix32((uint32_t)n * 0x9e3779b9u ^ mix32(*p.step_ctr));
        float ma = ra, mb = rb;  // mass left for the rest populations
        if (DRY) {
            ma = ca * ra;
            mb = rb + cb;
        }
#pragma unroll
        for (int i = 1; i < Q; i += 2) {
            const float eua = ex(i) * ua[0] + ey(i) * ua[1] + ez(i) * ua[2];
            const float eub = ex(i) * ub[0] + ey(i) * ub[1] + ez(i) * ub[2];
            const float wa = wgt(i) * ra, wb = wgt(i) * rb;
            const float sa_ = wa * (ka + 4.5f * eua * eua), sb_ = wb * (kb + 4.5f * eub * eub);
            const float qa1 = sa_ + 3.0f * wa * eua, qa2 = sa_ - 3.0f * wa * eua;
            const float qb1 = sb_ + 3.0f * wb * eub, qb2 = sb_ - 3.0f * wb * eub;
            float va1 = EQ ? qa1 : fa[i] - (fa[i] - qa1) * ta, va2 = EQ ? qa2 : fa[i + 1] - (fa[i + 1] - qa2) * ta;
            float vb1 = EQ ? qb1 : fb[i] - (fb[i] - qb1) * tb, vb2 = EQ ? qb2 : fb[i + 1] - (fb[i + 1] - qb2) * tb;
            if (DRY) {
                va1 *= ca; va2 *= ca;
                vb1 += wgt(i) * cb; vb2 += wgt(i) * cb;
            }
            // an LCG step per pair draws its rounding bits; the xor-shift mixes
            // the well-distributed high bits into the low half
            rs = rs * 1664525u + 1013904223u;
            const uint32_t hA = Pop<T>::cvt2(va1 - wa, va2 - wa, rs ^ (rs >> 16));
            rs = rs * 1664525u + 1013904223u;
            const uint32_t hB = Pop<T>::cvt2(vb1 - wb, vb2 - wb, rs ^ (rs >> 16));
            Pop<T>::put2(dA + i * N, dA + (i + 1) * N, hA);
            Pop<T>::put2(dB + i * N, dB + (i + 1) * N, hB);
            const float2 sA = Pop<T>::val2(hA), sB = Pop<T>::val2(hB);
            ma -= (sA.x + wa) + (sA.y + wa);
            mb -= (sB.x + wb) + (sB.y + wb);
        }
        p.dst0[n] = ma;
        p.dst0[N + n] = mb;
    }
}

// Collision of one node for any tau: pull again, Shan-Chen force, velocity
// shift, BGK (Eqs. 4-5), store.
// IBM: the diffuse-interface body force may be present (single-lattice passes;
// the batched passes compile it out)
template <typename T, bool DRY = false, bool IBM = false>
__device__ __forceinline__ void collide_node(const LBParams &p, const Deltas &d) {
    float fa[Q], fb[Q];
    const uint32_t m = pull<T>(p, d, fa, fb);
    const int n = d.n;
    const float2 mr = __ldg(p.rho + n), mp = __ldg(p.psi + n);
    const float ra = mr.x, rb = mr.y, pa = mp.x, pb = mp.y;
    const bool ibm = IBM && ibm_reached(p, n);
    IbmForce fi{};
    if (ibm) fi = ibm_load(p, n);
    float FA[3], FB[3];
    sc_force(p, d, m, ra, rb, pa, pb, FA, FB);
    if (ibm) ibm_apply(p, n, ra, rb, fi, FA, FB);
    float ja[3] = {0.f, 0.f, 0.f}, jb[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int i = 1; i < Q; i += 2) {  // opposite pairs (i, i+1)
        const float da = fa[i] - fa[i + 1], db = fb[i] - fb[i + 1];
        ja[0] += ex(i) * da; ja[1] += ey(i) * da; ja[2] += ez(i) * da;
        jb[0] += ex(i) * db; jb[1] += ey(i) * db; jb[2] += ez(i) * db;
    }
    // velocity shift: common velocity weighted by 1/tau, u^{c,eq} = u' + tau^c F^c / rho^c
    const float iden = 1.0f / (ra * p.itau[0] + rb * p.itau[1]);
    const float sfa = p.tau[0] / ra, sfb = p.tau[1] / rb;
    float ua[3], ub[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float up = (ja[a] * p.itau[0] + jb[a] * p.itau[1]) * iden;
        ua[a] = up + sfa * FA[a];
        ub[a] = up + sfb * FB[a];
    }
    if (p.out || ibm) {
        const float rt = ra + rb;
        const float u[3] = {(ja[0] + jb[0] + 0.5f * (FA[0] + FB[0])) / rt,
                            (ja[1] + jb[1] + 0.5f * (FA[1] + FB[1])) / rt,
                            (ja[2] + jb[2] + 0.5f * (FA[2] + FB[2])) / rt};
        if (p.out) {
            p.out[n] = ra;
            p.out[p.N + n] = rb;
            p.out[2 * p.N + n] = u[0];
            p.out[3 * p.N + n] = u[1];
            p.out[4 * p.N + n] = u[2];
        }
        if (ibm) p.uphys[n] = make_float4(u[0], u[1], u[2], 0.f);
    }
    if (!(ra + rb < 1e30f)) atomicOr(p.status, ST_NAN);
    store_post<T, DRY, false>(p, n, ra, rb, ua, ub, fa, fb);
}

// Collision of one node with tau = 1 for both components: BGK then stores the
// equilibria themselves, which need only the moments.  The density pass has
// stored the total momentum J = sum_c sum_i f_i^c e_i, so the populations are
// not pulled a second time.  The common velocity is u' = J / (rho_A + rho_B)
// and u^{c,eq} = u' + F^c / rho^c (the velocity shift with tau = 1).
// ibm: the node's spread force is in FA, FB (its velocity goes to uphys)
template <typename T, bool DRY>
__device__ __forceinline__ void collide_eq_finish(const LBParams &p, int n, float ra, float rb, const float4 J4,
                                                  const float (&FA)[3], const float (&FB)[3], bool ibm) {
    const float J[3] = {J4.x, J4.y, J4.z};
    const float rt = ra + rb, iden = 1.0f / rt, ia = 1.0f / ra, ib = 1.0f / rb;
    float ua[3], ub[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float up = J[a] * iden;
        ua[a] = up + ia * FA[a];
        ub[a] = up + ib * FB[a];
    }
    if (p.out || ibm) {
        const float u[3] = {(J[0] + 0.5f * (FA[0] + FB[0])) / rt, (J[1] + 0.5f * (FA[1] + FB[1])) / rt,
                            (J[2] + 0.5f * (FA[2] + FB[2])) / rt};
        if (p.out) {
            p.out[n] = ra;
            p.out[p.N + n] = rb;
            p.out[2 * p.N + n] = u[0];
            p.out[3 * p.N + n] = u[1];
            p.out[4 * p.N + n] = u[2];
        }
        if (ibm) p.uphys[n] = make_float4(u[0], u[1], u[2], 0.f);
    }
    if (!(ra + rb < 1e30f)) atomicOr(p.status, ST_NAN);
    float unused[Q];  // the equilibria need no pulled populations
    store_post<T, DRY, true>(p, n, ra, rb, ua, ub, unused, unused);
}

// the node's own inputs of the tau = 1 collision, loaded together ahead of
// the Shan-Chen stencil's gathers
struct NodeOwn {
    uint32_t m;
    float2 r, q;
    float4 J;
};
__device__ __forceinline__ NodeOwn node_own(const LBParams &p, long long n) {
    return {__ldg(p.mask + n), __ldg(p.rho + n), __ldg(p.psi + n), __ldg(p.J + n)};
}

template <typename T, bool DRY = false, bool IBM = false>
__device__ __forceinline__ void collide_eq_node(const LBParams &p, const Deltas &d, const NodeOwn &o) {
    const int n = d.n;
    const uint32_t m = o.m;
    const float2 mr = o.r, mp = o.q;
    const float4 J4 = o.J;
    const bool ibm = IBM && ibm_reached(p, n);
    IbmForce fi{};
    if (ibm) fi = ibm_load(p, n);
    float FA[3], FB[3];
    sc_force(p, d, m, mr.x, mr.y, mp.x, mp.y, FA, FB);
    if (ibm) ibm_apply(p, n, mr.x, mr.y, fi, FA, FB);
    collide_eq_finish<T, DRY>(p, n, mr.x, mr.y, J4, FA, FB, ibm);
}

// the planes zb, zb + zs, ... below ze of column (x, y)
template <typename T, bool DRY = false, bool IBM = false>
__device__ __forceinline__ void collide_eq_column(const LBParams &p, int x, int y, int zb, int ze, int zs) {
    for (int z = zb; z < ze; z += zs) {
        const Deltas d = deltas(p, x, y, z);
        collide_eq_node<T, DRY, IBM>(p, d, node_own(p, d.n));
    }
}

// ---------------------------------------------------------------------------
// tau = 1 collide pass with the pseudopotentials staged in shared memory.
// A block owns a TX x TY column tile and walks a contiguous run of planes; a
// ring of four planes of psi (the tile plus a one-node halo, periodic wrap)
// holds the planes z-1, z, z+1 the Shan-Chen stencil of plane z reads, while
// cp.async fills the fourth with plane z+2.  The 18 neighbour pseudopotentials
// of a node then come from shared memory at fixed offsets instead of 18 global
// gathers.  Nodes next to a cut or substrate link take the general stencil
// (sc_force, global loads), which also forms the partner densities.
template <int TX, int TY> struct PsiRing {
    float2 v[4][TY + 2][TX + 2];
};

__device__ __forceinline__ void cp_async8(void *smem, const void *gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// plane z (any integer; the data wraps periodically) of the tile at (x0, y0)
// into ring slot z & 3
template <int TX, int TY>
__device__ __forceinline__ void ring_load(const LBParams &p, PsiRing<TX, TY> &R, int z, int x0, int y0) {
    const int nx = p.nx, ny = p.ny;
    const int gz = ((unsigned)z < (unsigned)p.nz) ? z : wrapi(z, p.nz);
    const float2 *plane = p.psi + (long long)gz * nx * ny;
    float2(*dst)[TX + 2] = R.v[z & 3];
    for (int e = threadIdx.y * TX + threadIdx.x; e < (TY + 2) * (TX + 2); e += TX * TY) {
        const int ly = e / (TX + 2), lx = e - ly * (TX + 2);
        int gx = x0 + lx - 1, gy = y0 + ly - 1;
        if ((unsigned)gx >= (unsigned)nx) gx = wrapi(gx, nx);
        if ((unsigned)gy >= (unsigned)ny) gy = wrapi(gy, ny);
        cp_async8(&dst[ly][lx], plane + (long long)gy * nx + gx);
    }
}

template <typename T, bool DRY, int TX, int TY, bool IBM = false>
__device__ __forceinline__ void collide_eq_node_ring(const LBParams &p, const Deltas &d,
                                                     const PsiRing<TX, TY> &R, int z) {
    const int n = d.n;
    const int tx = threadIdx.x + 1, ty = threadIdx.y + 1;
    const uint32_t m = __ldg(p.mask + n);
    const float2 mr = __ldg(p.rho + n), mp = R.v[z & 3][ty][tx];
    const float ra = mr.x, rb = mr.y, pa = mp.x, pb = mp.y;
    const bool ibm = IBM && ibm_reached(p, n);
    IbmForce fi{};
    if (ibm) fi = ibm_load(p, n);
    float FA[3], FB[3];
    if (!m && !d.wlo && !d.whi) {
        // the stencil of sc_force over opposite pairs, neighbours from the ring
        float sa[3] = {0.f, 0.f, 0.f}, sb[3] = {0.f, 0.f, 0.f};
#pragma unroll
        for (int k = 1; k < Q; k += 2) {
            const float2 q1 = R.v[(z + ez(k)) & 3][ty + ey(k)][tx + ex(k)];
            const float2 q2 = R.v[(z - ez(k)) & 3][ty - ey(k)][tx - ex(k)];
            const float da = q1.x - q2.x, db = q1.y - q2.y;
            sa[0] += wgt(k) * ex(k) * da; sa[1] += wgt(k) * ey(k) * da; sa[2] += wgt(k) * ez(k) * da;
            sb[0] += wgt(k) * ex(k) * db; sb[1] += wgt(k) * ey(k) * db; sb[2] += wgt(k) * ez(k) * db;
        }
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            FA[a] = -p.G * pa * sb[a];
            FB[a] = -p.G * pb * sa[a];
        }
    } else {
        sc_force(p, d, m, ra, rb, pa, pb, FA, FB);
    }
    if (ibm) ibm_apply(p, n, ra, rb, fi, FA, FB);
    collide_eq_finish<T, DRY>(p, n, ra, rb, __ldg(p.J + n), FA, FB, ibm);
}

// planes [zb, ze) of the tile at (x0, y0); every thread of the block calls it
// with the same arguments (the ring loads and barriers are block-wide)
template <typename T, bool DRY, int TX, int TY, bool IBM = false>
__device__ __forceinline__ void collide_eq_ring(const LBParams &p, PsiRing<TX, TY> &R, int x0, int y0, int zb,
                                                int ze) {
    if (zb >= ze) return;
    const int x = x0 + (int)threadIdx.x, y = y0 + (int)threadIdx.y;
    const bool in = x < p.nx && y < p.ny;
    ring_load<TX, TY>(p, R, zb - 1, x0, y0);
    ring_load<TX, TY>(p, R, zb, x0, y0);
    ring_load<TX, TY>(p, R, zb + 1, x0, y0);
    cp_async_commit();
    cp_async_wait_all();
    __syncthreads();
    for (int z = zb; z < ze; ++z) {
        if (z + 1 < ze) ring_load<TX, TY>(p, R, z + 2, x0, y0);  // for the next plane
        cp_async_commit();
        if (in) collide_eq_node_ring<T, DRY, TX, TY, IBM>(p, deltas(p, x, y, z), R, z);
        cp_async_wait_all();
        __syncthreads();
    }
}

// IBM: with the diffuse-interface body force (its own instantiation, so that
// the lattices without it keep their registers)
template <typename T, bool DRY = false, bool IBM = false>
__global__ void __launch_bounds__(BX *BY, Pop<T>::shifted ? CF_COLLIDE16_MINB : CF_COLLIDE_MINB)
    k_collide(const LBParams p) {
    pdl_trigger();
    pdl_wait();
    int x, y, z;
    if (!node_of<true>(p, x, y, z)) return;
    for (; z < p.zhi; z += gridDim.z) collide_node<T, DRY, IBM>(p, deltas(p, x, y, z));
}

// resident blocks per SM of the tau = 1 collide pass (no second pull: few registers)
#ifndef CF_COLLIDE_EQ_MINB
#define CF_COLLIDE_EQ_MINB 8
#endif

// Blocks in reverse order (the tiles the density pass read last first).
// With CF_PSI_RING set, each block walks zring contiguous planes through its
// pseudopotential ring; by default the neighbour pseudopotentials are global
// gathers (L1/L2 hits) and threads walk planes strided by grid.z like the
// density pass (measured faster on the GB300: the ring's loads and barriers
// cost more than the gathers they replace).
#ifndef CF_PSI_RING
#define CF_PSI_RING 0
#endif
template <typename T, bool DRY = false, bool IBM = false>
__global__ void __launch_bounds__(BX *BY, CF_COLLIDE_EQ_MINB) k_collide_eq(const LBParams p) {
    pdl_trigger();
    pdl_wait();
#if CF_PSI_RING
    __shared__ PsiRing<BX, BY> R;
    const int bx = (int)(gridDim.x - 1 - blockIdx.x), by = (int)(gridDim.y - 1 - blockIdx.y);
    const int bz = (int)(gridDim.z - 1 - blockIdx.z);
    const int zb = p.zlo + bz * p.zring, ze = min(p.zhi, zb + p.zring);
    collide_eq_ring<T, DRY, BX, BY, IBM>(p, R, bx * BX, by * BY, zb, ze);
#else
    int x, y, z;
    if (!node_of<true>(p, x, y, z)) return;
    collide_eq_column<T, DRY, IBM>(p, x, y, z, p.zhi, (int)gridDim.z);
#endif
}

size_t density_blocks_max(int nx, int ny, int nz) {
    return (size_t)((nx + BX - 1) / BX) * ((ny + BY - 1) / BY) * nz;
}

namespace {
// before_collide (optional): the collide pass also waits for this event (a
// plain launch then, the density pass stays programmatic)
template <typename T, bool DRY, bool IBM>
void lb_passes(const LBParams &p, dim3 grid, dim3 block, cudaStream_t s, bool eq, cudaEvent_t before_collide) {
    if (eq) {
        launch_pdl(k_density<T, DRY, true>, grid, block, s, p);
#if CF_PSI_RING
        const int zr = std::max(1, p.zring);
        const dim3 gc(grid.x, grid.y, (unsigned)((p.zhi - p.zlo + zr - 1) / zr));
#else
        const dim3 gc = grid;
#endif
        if (before_collide) {
            cudaStreamWaitEvent(s, before_collide, 0);
            k_collide_eq<T, DRY, IBM><<<gc, block, 0, s>>>(p);
        } else {
            launch_pdl(k_collide_eq<T, DRY, IBM>, gc, block, s, p);
        }
    } else {
        launch_pdl(k_density<T, DRY>, grid, block, s, p);
        if (before_collide) {
            cudaStreamWaitEvent(s, before_collide, 0);
            k_collide<T, DRY, IBM><<<grid, block, 0, s>>>(p);
        } else {
            launch_pdl(k_collide<T, DRY, IBM>, grid, block, s, p);
        }
    }
}
template <typename T>
void lb_passes(const LBParams &p, dim3 grid, dim3 block, cudaStream_t s, bool dry, bool eq, cudaEvent_t ev) {
    const bool ibm = p.fibm != nullptr;
    if (dry) {
        if (ibm) lb_passes<T, true, true>(p, grid, block, s, eq, ev);
        else lb_passes<T, true, false>(p, grid, block, s, eq, ev);
    } else {
        if (ibm) lb_passes<T, false, true>(p, grid, block, s, eq, ev);
        else lb_passes<T, false, false>(p, grid, block, s, eq, ev);
    }
}
}  // namespace

cudaError_t launch_lb_step(const LBParams &p, int prec, cudaStream_t s, cudaEvent_t before_collide) {
    const int nzf = p.zhi - p.zlo;
    const int gz = p.zchunk > 0 ? (nzf + p.zchunk - 1) / p.zchunk : nzf;
    dim3 grid((p.nx + BX - 1) / BX, (p.ny + BY - 1) / BY, gz), block(BX, BY);
    const bool dry = p.dry_dm > 0.0;
    // tau = 1 for both components: the collide pass takes the density pass's momentum
    const bool eq = p.J != nullptr && p.tau[0] == 1.f && p.tau[1] == 1.f;
    if (prec == P_F16) lb_passes<__half>(p, grid, block, s, dry, eq, before_collide);
    else if (prec == P_BF16) lb_passes<__nv_bfloat16>(p, grid, block, s, dry, eq, before_collide);
    else lb_passes<float>(p, grid, block, s, dry, eq, before_collide);
    return cudaGetLastError();
}

// ------------------------------------------------------------ batched passes
// One persistent launch per pass for many independent lattices (a parameter
// sweep).  Blocks stride over the work list of (lattice, x tile, y tile,
// z slice) items; a thread walks the planes z0, z0 + zstride, ... of its
// column.  The per-node arithmetic is that of the single-lattice passes, so
// a lattice stepped in a batch follows the same trajectory as alone.  The
// collide pass walks the list backwards (the tiles the density pass read last
// are still in L2).  Tile shapes (x width x y depth, the block shape) are
// compiled in and chosen by the autotuner of the batch.  EQ: every lattice has
// tau = 1, and the passes are those of the tau = 1 collision (momentum from
// the density pass, no second pull).
// work item (lattice, x tile, y tile, z slice): slice s covers the planes
// [zlo + s zchunk, zlo + (s + 1) zchunk) of its lattice
template <typename T, int TX, int TY, bool EQ>
__global__ void __launch_bounds__(TX *TY) k_density_batch(const __grid_constant__ BatchTab tab,
                                                          const int4 *__restrict__ work, int nwork) {
    for (int w = blockIdx.x; w < nwork; w += gridDim.x) {
        const int4 it = __ldg(work + w);
        const LBParams &p = tab.lat[it.x];
        if (Pop<T>::shifted && it.y == 0 && it.z == 0 && it.w == 0 && threadIdx.x == 0 &&
            threadIdx.y == 0)
            atomicAdd(p.step_ctr, 1u);  // read by the collide pass that follows
        const int x = it.y * TX + (int)threadIdx.x, y = it.z * TY + (int)threadIdx.y;
        if (x >= p.nx || y >= p.ny) continue;
        const int zb = p.zlo + it.w * p.zchunk, ze = min(p.zhi, zb + p.zchunk);
        for (int z = zb; z < ze; ++z) density_node<T, EQ>(p, deltas(p, x, y, z));
    }
}

// the collide pass walks the work list backwards; with EQ (tau = 1) through
// the pseudopotential ring (block-wide: every thread takes part in each item)
#ifndef CF_COLLIDE_BATCH_EQ_MINB  // resident blocks per SM of the tau = 1 batched collide (128 threads)
#define CF_COLLIDE_BATCH_EQ_MINB 8
#endif
template <typename T, int TX, int TY, bool EQ>
__global__ void __launch_bounds__(TX *TY, (TX * TY >= 256 ? 2 : (EQ ? CF_COLLIDE_BATCH_EQ_MINB : 5))) k_collide_batch(
    const __grid_constant__ BatchTab tab, const int4 *__restrict__ work, int nwork) {
    __shared__ PsiRing<TX, (EQ && CF_PSI_RING != 0) ? TY : 1> R;
    for (int w = blockIdx.x; w < nwork; w += gridDim.x) {
        const int4 it = __ldg(work + (nwork - 1 - w));
        const LBParams &p = tab.lat[it.x];
        const int zb = p.zlo + it.w * p.zchunk, ze = min(p.zhi, zb + p.zchunk);
        if constexpr (EQ && CF_PSI_RING != 0) {
            collide_eq_ring<T, false, TX, TY>(p, R, it.y * TX, it.z * TY, zb, ze);
        } else if constexpr (EQ) {
            const int x = it.y * TX + (int)threadIdx.x, y = it.z * TY + (int)threadIdx.y;
            if (x >= p.nx || y >= p.ny) continue;
            collide_eq_column<T>(p, x, y, zb, ze, 1);
        } else {
            const int x = it.y * TX + (int)threadIdx.x, y = it.z * TY + (int)threadIdx.y;
            if (x >= p.nx || y >= p.ny) continue;
            for (int z = zb; z < ze; ++z) collide_node<T>(p, deltas(p, x, y, z));
        }
    }
}

namespace {
constexpr int TILE_X[CF_NTILES] = {32, 32, 32, 64, 64, 128};
constexpr int TILE_Y[CF_NTILES] = {2, 4, 8, 2, 4, 2};

template <typename T, int TX, int TY>
void batch_kernels(bool eq, const void *&kd, const void *&kc) {
    if (eq) {
        kd = reinterpret_cast<const void *>(&k_density_batch<T, TX, TY, true>);
        kc = reinterpret_cast<const void *>(&k_collide_batch<T, TX, TY, true>);
    } else {
        kd = reinterpret_cast<const void *>(&k_density_batch<T, TX, TY, false>);
        kc = reinterpret_cast<const void *>(&k_collide_batch<T, TX, TY, false>);
    }
}

template <typename T>
void batch_kernels_t(int tile, bool eq, const void *&kd, const void *&kc) {
    switch (tile) {
    case 0: batch_kernels<T, 32, 2>(eq, kd, kc); break;
    case 1: batch_kernels<T, 32, 4>(eq, kd, kc); break;
    case 2: batch_kernels<T, 32, 8>(eq, kd, kc); break;
    case 3: batch_kernels<T, 64, 2>(eq, kd, kc); break;
    case 4: batch_kernels<T, 64, 4>(eq, kd, kc); break;
    default: batch_kernels<T, 128, 2>(eq, kd, kc); break;
    }
}

void batch_kernel_ptrs(int tile, int prec, bool eq, const void *&kd, const void *&kc) {
    if (prec == P_F16) batch_kernels_t<__half>(tile, eq, kd, kc);
    else if (prec == P_BF16) batch_kernels_t<__nv_bfloat16>(tile, eq, kd, kc);
    else batch_kernels_t<float>(tile, eq, kd, kc);
}

// tau = 1 in every lattice of the table (the tau = 1 passes apply)
bool batch_eq(const BatchTab &tab, int nlat) {
    for (int i = 0; i < nlat; ++i)
        if (!tab.lat[i].J || tab.lat[i].tau[0] != 1.f || tab.lat[i].tau[1] != 1.f) return false;
    return nlat > 0;
}
}  // namespace

void lb_batch_tile(int tile, int *tx, int *ty) {
    tile = std::min(std::max(tile, 0), CF_NTILES - 1);
    *tx = TILE_X[tile];
    *ty = TILE_Y[tile];
}

int lb_batch_resident(int tile, int prec, bool eq) {
    static int cache[2][3][CF_NTILES] = {};
    tile = std::min(std::max(tile, 0), CF_NTILES - 1);
    prec = std::min(std::max(prec, 0), 2);
    int &c = cache[eq ? 1 : 0][prec][tile];
    if (c == 0) {
        const void *kd, *kc;
        batch_kernel_ptrs(tile, prec, eq, kd, kc);
        int dev = 0, sms = 0, per_sm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kc, TILE_X[tile] * TILE_Y[tile], 0);
        c = sms * std::max(per_sm, 1);
    }
    return c;
}

cudaError_t launch_lb_batch(const BatchTab &tab, int nlat, const int4 *work, int nwork, int prec, int tile,
                            cudaStream_t s) {
    tile = std::min(std::max(tile, 0), CF_NTILES - 1);
    const bool eq = batch_eq(tab, nlat);
    const void *kd, *kc;
    batch_kernel_ptrs(tile, prec, eq, kd, kc);
    const dim3 block(TILE_X[tile], TILE_Y[tile]);
    // enough blocks to cover the list, at most a few waves of resident blocks
    const unsigned grid = (unsigned)std::max(1, std::min(nwork, 4 * lb_batch_resident(tile, prec, eq)));
    void *args[] = {const_cast<BatchTab *>(&tab), &work, &nwork};
    cudaError_t e = cudaLaunchKernel(kd, dim3(grid), block, args, 0, s);
    if (e != cudaSuccess) return e;
    return cudaLaunchKernel(kc, dim3(grid), block, args, 0, s);
}

// ------------------------------------------------------------ film set-up
template <typename T>
__device__ __forceinline__ void init_rest(T *f, float *f0, float2 *rho, long long N, long long n,
                                          const double (&r)[2]);

template <typename T>
__global__ void k_init_film(T *f, float *f0, float2 *rho, long long N, int nx, int ny, int nz,
                           int wall, float h_top, float rmaj, float rmin, float rmix,
                           const double *jit, const uint8_t *inside) {
    const long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (n >= N) return;
    const int z = (int)(n / ((long long)nx * ny));
    const int zm = (int)floorf(h_top + 0.5f);
    double r[2];
    if (wall && z == 0) { r[0] = r[1] = 0.0; }
    else {
        if (inside[n]) { r[0] = rmin; r[1] = rmaj; }
        else if (z < zm) { r[0] = rmaj; r[1] = rmin; }
        else if (z == zm) { r[0] = rmix; r[1] = rmix; }
        else { r[0] = rmin; r[1] = rmaj; }
        if (jit) { r[0] += jit[n]; r[1] += jit[N + n]; }
    }
    init_rest<T>(f, f0, rho, N, n, r);
}

// Rest state f_i = w_i rho of node n for the densities r[2] (16-bit storage:
// zero offsets and the float rest population from the mass balance).
template <typename T>
__device__ __forceinline__ void init_rest(T *f, float *f0, float2 *rho, long long N, long long n,
                                          const double (&r)[2]) {
    float ra = 0.f, rb = 0.f;
    if (Pop<T>::shifted) {  // rest state: zero offsets from w_i rho, float rest populations
        ra = (float)r[0];
        rb = (float)r[1];
        float ma = ra, mb = rb;
#pragma unroll
        for (int i = 1; i < Q; ++i) {
            Pop<T>::st(f + (long long)i * N + n, 0.f, 0u);
            Pop<T>::st(f + (long long)(Q + i) * N + n, 0.f, 0u);
            ma -= wgt(i) * ra;
            mb -= wgt(i) * rb;
        }
        f0[n] = ma;
        f0[N + n] = mb;
    } else {
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const double w = i == 0 ? 1.0 / 3.0 : (i <= 6 ? 1.0 / 18.0 : 1.0 / 36.0);
            const float fa = (float)(w * r[0]), fb = (float)(w * r[1]);
            Pop<T>::st(f + (long long)i * N + n, fa, 0u);
            Pop<T>::st(f + (long long)(Q + i) * N + n, fb, 0u);
            ra += fa;
            rb += fb;
        }
    }
    rho[n] = make_float2(ra, rb);  // density of the initial state
}

// Rest state from given densities rAB [2][N] (the substrate plane empty).
template <typename T>
__global__ void k_init_dens(T *f, float *f0, float2 *rho, long long N, int nx, int ny, int wall,
                            const double *rAB) {
    const long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (n >= N) return;
    const int z = (int)(n / ((long long)nx * ny));
    double r[2] = {rAB[n], rAB[N + n]};
    if (wall && z == 0) r[0] = r[1] = 0.0;
    init_rest<T>(f, f0, rho, N, n, r);
}

cudaError_t launch_init_dens(void *f, float *f0, int prec, float2 *rho, long long N, int nx, int ny,
                             int wall, const double *rAB, cudaStream_t s) {
    const unsigned g = (unsigned)((N + 255) / 256);
    if (prec == P_F16)
        k_init_dens<<<g, 256, 0, s>>>(static_cast<__half *>(f), f0, rho, N, nx, ny, wall, rAB);
    else if (prec == P_BF16)
        k_init_dens<<<g, 256, 0, s>>>(static_cast<__nv_bfloat16 *>(f), f0, rho, N, nx, ny, wall, rAB);
    else
        k_init_dens<<<g, 256, 0, s>>>(static_cast<float *>(f), f0, rho, N, nx, ny, wall, rAB);
    return cudaGetLastError();
}

cudaError_t launch_init_film(void *f, float *f0, int prec, float2 *rho, long long N, int nx, int ny,
                             int nz, int wall, float h_top, float rmaj, float rmin, float rmix,
                             const double *jit, const uint8_t *inside, cudaStream_t s) {
    const unsigned g = (unsigned)((N + 255) / 256);
    if (prec == P_F16)
        k_init_film<<<g, 256, 0, s>>>(static_cast<__half *>(f), f0, rho, N, nx, ny, nz, wall, h_top,
                                      rmaj, rmin, rmix, jit, inside);
    else if (prec == P_BF16)
        k_init_film<<<g, 256, 0, s>>>(static_cast<__nv_bfloat16 *>(f), f0, rho, N, nx, ny, nz, wall,
                                      h_top, rmaj, rmin, rmix, jit, inside);
    else
        k_init_film<<<g, 256, 0, s>>>(static_cast<float *>(f), f0, rho, N, nx, ny, nz, wall, h_top,
                                      rmaj, rmin, rmix, jit, inside);
    return cudaGetLastError();
}

// interior flags: parity of cut +z links walked up each column
__global__ void k_inside(const uint32_t *mask, uint8_t *inside, int nx, int ny, int nz) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nx * ny) return;
    int in = 0;
    for (int z = 0; z < nz; ++z) {
        const long long n = (long long)z * nx * ny + c;
        inside[n] = (uint8_t)in;
        if (mask[n] & (1u << 4)) in ^= 1;
    }
}

cudaError_t launch_inside(const uint32_t *mask, uint8_t *inside, int nx, int ny, int nz,
                          cudaStream_t s) {
    k_inside<<<(nx * ny + 127) / 128, 128, 0, s>>>(mask, inside, nx, ny, nz);
    return cudaGetLastError();
}

// film height per column from the recorded densities
__global__ void k_meniscus(const float *out, const uint8_t *inside, float *h, int nx, int ny,
                           int nz, int wall) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nx * ny) return;
    const long long N = (long long)nx * ny * nz;
    float res = __int_as_float(0x7fc00000);
    for (int z = wall ? 1 : 0; z + 1 < nz; ++z) {
        const long long n0 = (long long)z * nx * ny + c, n1 = n0 + (long long)nx * ny;
        const float p0 = out[n0] - out[N + n0], p1 = out[n1] - out[N + n1];
        if (p0 > 0.f && p1 <= 0.f) {
            if (!inside[n0] && !inside[n1]) res = z + p0 / (p0 - p1);
            break;
        }
    }
    h[c] = res;
}

cudaError_t launch_meniscus(const float *out, const uint8_t *inside, float *h, int nx, int ny,
                            int nz, int wall, cudaStream_t s) {
    k_meniscus<<<(nx * ny + 127) / 128, 128, 0, s>>>(out, inside, h, nx, ny, nz, wall);
    return cudaGetLastError();
}

// Meniscus profile of capsule `id` (Sec. 4.1) from the column heights h
// [ny][nx] (NaN where no valid interface): one block, FP64.
//  - centroids: the FP64 node sums of the last step (per-capsule accumulators)
//  - h_inf: mean of the valid columns whose periodic distance to the nearest
//    capsule centroid is at least 0.9 of the largest such distance
//  - rays from the column nearest to the centroid along +x, -x, +y, -y,
//    sampled at r_k = k dr with linear interpolation between the bracketing
//    columns (invalid where either is NaN); zeta_k = ray mean - h_inf
//  - out[0..nr) = zeta, out[nr] = Z (largest valid zeta), out[nr+1] = h_inf
constexpr int PROF_THREADS = 256;

__device__ __forceinline__ double block_sum(double v, double *red) {
    red[threadIdx.x] = v;
    __syncthreads();
    for (int o = PROF_THREADS / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    const double r = red[0];
    __syncthreads();
    return r;
}
__device__ __forceinline__ double block_max(double v, double *red) {
    red[threadIdx.x] = v;
    __syncthreads();
    for (int o = PROF_THREADS / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + o]);
        __syncthreads();
    }
    const double r = red[0];
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(PROF_THREADS) k_meniscus_profile(
    const float *__restrict__ h, int nx, int ny, const double *__restrict__ acc, const CapDev *__restrict__ caps,
    int ncaps, int id, double dr, int nr, double *__restrict__ out) {
    __shared__ double red[PROF_THREADS];
    auto centre = [&](int k, double &cx, double &cy) {
        const double *a = acc + (size_t)k * A_NACC;
        const double nv = (double)caps[k].nv;
        cx = a[A_OX] + a[A_CX] / nv;
        cy = a[A_OY] + a[A_CY] / nv;
    };
    auto nearest = [&](int x, int y) {
        double best = CUDART_INF;
        for (int k = 0; k < ncaps; ++k) {
            double cx, cy;
            centre(k, cx, cy);
            double dx = x - cx, dy = y - cy;
            dx -= nx * floor(dx / nx + 0.5);
            dy -= ny * floor(dy / ny + 0.5);
            best = fmin(best, sqrt(dx * dx + dy * dy));
        }
        return best;
    };
    const int ncol = nx * ny;
    double m = 0.0;
    for (int c = threadIdx.x; c < ncol; c += PROF_THREADS)
        if (!isnan(h[c])) m = fmax(m, nearest(c % nx, c / nx));
    const double dmax = block_max(m, red);
    double hs = 0.0, hc = 0.0;
    for (int c = threadIdx.x; c < ncol; c += PROF_THREADS) {
        const float v = h[c];
        if (!isnan(v) && nearest(c % nx, c / nx) >= 0.9 * dmax) { hs += v; hc += 1.0; }
    }
    const double S = block_sum(hs, red), Cn = block_sum(hc, red);
    const double hinf = Cn > 0.0 ? S / Cn : CUDART_NAN;
    double cx, cy;
    centre(id, cx, cy);
    const int x0 = (int)lround(cx), y0 = (int)lround(cy);
    for (int k = threadIdx.x; k < nr; k += PROF_THREADS) {
        const double rk = k * dr;
        const int j0 = (int)floor(rk);
        const double t = rk - j0;
        double s = 0.0;
        int cnt = 0;
        for (int q = 0; q < 4; ++q) {
            const int sx = q == 0 ? 1 : q == 1 ? -1 : 0, sy = q == 2 ? 1 : q == 3 ? -1 : 0;
            const int xa = wrapi(x0 + sx * j0, nx), ya = wrapi(y0 + sy * j0, ny);
            const int xb = wrapi(x0 + sx * (j0 + 1), nx), yb = wrapi(y0 + sy * (j0 + 1), ny);
            const double ha = h[ya * nx + xa], hb = h[yb * nx + xb];
            const double v = t == 0.0 ? ha : (1.0 - t) * ha + t * hb;
            if (!isnan(v)) { s += v; ++cnt; }
        }
        out[k] = cnt ? s / cnt - hinf : CUDART_NAN;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double Z = CUDART_NAN;
        for (int k = 0; k < nr; ++k)
            if (!isnan(out[k]) && (isnan(Z) || out[k] > Z)) Z = out[k];
        out[nr] = Z;
        out[nr + 1] = hinf;
    }
}

cudaError_t launch_meniscus_profile(const float *h, int nx, int ny, const double *acc, const CapDev *caps,
                                    int ncaps, int id, double dr, int nr, double *out, cudaStream_t s) {
    k_meniscus_profile<<<1, PROF_THREADS, 0, s>>>(h, nx, ny, acc, caps, ncaps, id, dr, nr, out);
    return cudaGetLastError();
}

// FP64 mass of each component (decoded populations)
template <typename T>
__global__ void k_mass(const T *f, const float *f0, const float2 *rho, long long N, double *m2) {
    double s[2] = {0.0, 0.0};
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < N;
         n += (long long)gridDim.x * blockDim.x) {
        if (Pop<T>::shifted) {
            const float2 r = rho[n];
            s[0] += f0[n];
            s[1] += f0[N + n];
#pragma unroll
            for (int i = 1; i < Q; ++i) {
                s[0] += Pop<T>::ld(f + (long long)i * N + n) + wgt(i) * r.x;
                s[1] += Pop<T>::ld(f + (long long)(Q + i) * N + n) + wgt(i) * r.y;
            }
        } else {
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                s[0] += Pop<T>::ld(f + (long long)i * N + n);
                s[1] += Pop<T>::ld(f + (long long)(Q + i) * N + n);
            }
        }
    }
    for (int c = 0; c < 2; ++c) {
        double v = s[c];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) == 0) atomicAdd(m2 + c, v);
    }
}

cudaError_t launch_mass(const void *f, const float *f0, int prec, const float2 *rho, long long N,
                        double *m2, cudaStream_t s) {
    if (prec == P_F16) k_mass<<<304, 256, 0, s>>>(static_cast<const __half *>(f), f0, rho, N, m2);
    else if (prec == P_BF16)
        k_mass<<<304, 256, 0, s>>>(static_cast<const __nv_bfloat16 *>(f), f0, rho, N, m2);
    else k_mass<<<304, 256, 0, s>>>(static_cast<const float *>(f), f0, rho, N, m2);
    return cudaGetLastError();
}

}  // namespace cf

// ------------------------------------------- lattice update with static scratch
// Some callers cannot allocate device memory: code that runs inside a host
// framework which owns the whole device allocation (a fixed pool handed out
// once, or an allocator that may not be called from the thread doing the
// stepping), or code that must not allocate between a set-up phase and the
// stepping loop.  cf_lattice_step_static advances a lattice without capsules
// one step with the same arithmetic as the density and collide passes above,
// taking the per-node density scratch from a fixed array compiled into this
// library instead of allocating it.  The array holds the densities of at most
// CF_STATIC_MAX_NODES nodes; every GPU that loads the library keeps it
// (16 MiB) until the process exits.
namespace cf {

constexpr long long CF_STATIC_MAX_NODES = 1LL << 20;
static __device__ __align__(256) float4 g_static_dens[CF_STATIC_MAX_NODES];

__global__ void __launch_bounds__(BX *BY) k_density_static(const LBParams p) {
    int x, y, z;
    if (!node_of(p, x, y, z)) return;
    const int N = (int)p.N;
    for (; z < p.zhi; z += gridDim.z) {
        const Deltas d = deltas(p, x, y, z);
        const float *src = static_cast<const float *>(p.src);
        const float *sA = src + d.n, *sB = src + (long long)Q * N + d.n;
        float ra = 0.f, rb = 0.f;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const int o = src_off(d, N, i);
            ra += __ldg(sA + o);
            rb += __ldg(sB + o);
        }
        p.J[d.n] = make_float4(ra, rb, psi_of(ra), psi_of(rb));
    }
}

// Shan-Chen force (substrate links use the interpolated partner density),
// velocity shift, BGK, store: the collide pass without membrane links.
__device__ __forceinline__ void collide_node_static(const LBParams &p, const Deltas &d) {
    const int N = (int)p.N, n = d.n;
    float fa[Q], fb[Q];
    {
        const float *src = static_cast<const float *>(p.src);
        const float *sA = src + n, *sB = src + (long long)Q * N + n;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const int o = src_off(d, N, i);
            fa[i] = __ldg(sA + o);
            fb[i] = __ldg(sB + o);
        }
    }
    const float4 me = p.J[n];
    const float ra = me.x, rb = me.y, pa = me.z, pb = me.w;
    float sa[3] = {0.f, 0.f, 0.f}, sb[3] = {0.f, 0.f, 0.f};  // summed over opposite pairs
    if (!d.wlo && !d.whi) {
#pragma unroll
        for (int k = 1; k < Q; k += 2) {
            const float4 q1 = p.J[n + nb_off(d, ex(k), ey(k), ez(k))];
            const float4 q2 = p.J[n + nb_off(d, -ex(k), -ey(k), -ez(k))];
            const float da = q1.z - q2.z, db = q1.w - q2.w;
            sa[0] += wgt(k) * ex(k) * da; sa[1] += wgt(k) * ey(k) * da; sa[2] += wgt(k) * ez(k) * da;
            sb[0] += wgt(k) * ex(k) * db; sb[1] += wgt(k) * ey(k) * db; sb[2] += wgt(k) * ez(k) * db;
        }
    } else {
        float ia = ra, ib = rb, cnt = 1.f;
#pragma unroll
        for (int k = 1; k < Q; ++k) {
            const bool solid = (ez(k) == 1 && d.whi) || (ez(k) == -1 && d.wlo);
            if (!solid) {
                const float4 q = p.J[n + nb_off(d, ex(k), ey(k), ez(k))];
                ia += q.x; ib += q.y; cnt += 1.f;
            }
        }
        const float qa_eff = psi_of(ia / cnt), qb_eff = psi_of(ib / cnt);
        float qA[Q], qB[Q];
#pragma unroll
        for (int k = 1; k < Q; ++k) {
            const bool solid = (ez(k) == 1 && d.whi) || (ez(k) == -1 && d.wlo);
            if (solid) { qA[k] = qa_eff; qB[k] = qb_eff; }
            else {
                const float4 q = p.J[n + nb_off(d, ex(k), ey(k), ez(k))];
                qA[k] = q.z; qB[k] = q.w;
            }
        }
#pragma unroll
        for (int k = 1; k < Q; k += 2) {
            const float da = qA[k] - qA[k + 1], db = qB[k] - qB[k + 1];
            sa[0] += wgt(k) * ex(k) * da; sa[1] += wgt(k) * ey(k) * da; sa[2] += wgt(k) * ez(k) * da;
            sb[0] += wgt(k) * ex(k) * db; sb[1] += wgt(k) * ey(k) * db; sb[2] += wgt(k) * ez(k) * db;
        }
    }
    const float FA[3] = {-p.G * pa * sb[0], -p.G * pa * sb[1], -p.G * pa * sb[2]};
    const float FB[3] = {-p.G * pb * sa[0], -p.G * pb * sa[1], -p.G * pb * sa[2]};
    float ja[3] = {0.f, 0.f, 0.f}, jb[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int i = 1; i < Q; i += 2) {
        const float da = fa[i] - fa[i + 1], db = fb[i] - fb[i + 1];
        ja[0] += ex(i) * da; ja[1] += ey(i) * da; ja[2] += ez(i) * da;
        jb[0] += ex(i) * db; jb[1] += ey(i) * db; jb[2] += ez(i) * db;
    }
    const float den = ra * p.itau[0] + rb * p.itau[1];
    float ua[3], ub[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float up = (ja[a] * p.itau[0] + jb[a] * p.itau[1]) / den;
        ua[a] = up + p.tau[0] * FA[a] / ra;
        ub[a] = up + p.tau[1] * FB[a] / rb;
    }
    const float ka = 1.0f - 1.5f * (ua[0] * ua[0] + ua[1] * ua[1] + ua[2] * ua[2]);
    const float kb = 1.0f - 1.5f * (ub[0] * ub[0] + ub[1] * ub[1] + ub[2] * ub[2]);
    float *__restrict__ dA = static_cast<float *>(p.dst) + n;
    float *__restrict__ dB = static_cast<float *>(p.dst) + (long long)Q * N + n;
    const float ta = p.itau[0], tb = p.itau[1];
    float qa0 = ra, qb0 = rb;
#pragma unroll
    for (int i = 1; i < Q; i += 2) {
        const float eua = ex(i) * ua[0] + ey(i) * ua[1] + ez(i) * ua[2];
        const float eub = ex(i) * ub[0] + ey(i) * ub[1] + ez(i) * ub[2];
        const float wa = wgt(i) * ra, wb = wgt(i) * rb;
        const float sa_ = wa * (ka + 4.5f * eua * eua), sb_ = wb * (kb + 4.5f * eub * eub);
        const float qa1 = sa_ + 3.0f * wa * eua, qa2 = sa_ - 3.0f * wa * eua;
        const float qb1 = sb_ + 3.0f * wb * eub, qb2 = sb_ - 3.0f * wb * eub;
        qa0 -= qa1 + qa2;
        qb0 -= qb1 + qb2;
        dA[i * N] = fa[i] - (fa[i] - qa1) * ta;
        dA[(i + 1) * N] = fa[i + 1] - (fa[i + 1] - qa2) * ta;
        dB[i * N] = fb[i] - (fb[i] - qb1) * tb;
        dB[(i + 1) * N] = fb[i + 1] - (fb[i + 1] - qb2) * tb;
    }
    dA[0] = fa[0] - (fa[0] - qa0) * ta;
    dB[0] = fb[0] - (fb[0] - qb0) * tb;
}

__global__ void __launch_bounds__(BX *BY) k_collide_static(const LBParams p) {
    int x, y, z;
    if (!node_of(p, x, y, z)) return;
    for (; z < p.zhi; z += gridDim.z) collide_node_static(p, deltas(p, x, y, z));
}

// Device address of the static scratch in the current context (the array's
// name is only a host-side stand-in).  Looked up on every call: the lookup is
// a cheap host call, and a cached address could belong to a context that has
// since been destroyed (cudaDeviceReset) or to another context on the device.
static float4 *static_dens_address(cudaError_t *err) {
    void *ptr = nullptr;
    *err = cudaGetSymbolAddress(&ptr, g_static_dens);
    return *err == cudaSuccess ? static_cast<float4 *>(ptr) : nullptr;
}

}  // namespace cf

extern "C" cf_status cf_lattice_step_static(const float *src, float *dst, int nx, int ny, int nz,
                                            int wall, const double tau[2], double G, void *stream) {
    using namespace cf;
    if (!src || !dst || !tau) { set_last_error("null argument"); return CF_EINVAL; }
    if (nx < 3 || ny < 3 || nz < 3) { set_last_error("lattice dimensions must be >= 3"); return CF_EINVAL; }
    const long long N = (long long)nx * ny * nz;
    if (N > CF_STATIC_MAX_NODES) {
        set_last_error("cf_lattice_step_static: lattice larger than the static scratch "
                       "(at most 1048576 nodes)");
        return CF_EINVAL;
    }
    if (!(tau[0] > 0.5) || !(tau[1] > 0.5)) { set_last_error("tau must exceed 1/2"); return CF_EINVAL; }
    {   // the collide pass reads src around every node while it writes dst
        const uintptr_t a0 = (uintptr_t)src, b0 = (uintptr_t)dst;
        const uintptr_t bytes = (uintptr_t)(2 * Q * N) * sizeof(float);
        if (a0 < b0 + bytes && b0 < a0 + bytes) {
            set_last_error("cf_lattice_step_static: src and dst overlap");
            return CF_EINVAL;
        }
    }
    cudaError_t e = cudaSuccess;
    float4 *dens = static_dens_address(&e);
    if (!dens) {
        set_last_error(cudaGetErrorString(e));
        return CF_ECUDA;
    }
    LBParams p{};
    p.nx = nx; p.ny = ny; p.nz = nz; p.wall = wall ? 1 : 0;
    p.N = N;
    p.zlo = p.wall ? 1 : 0;
    p.zhi = nz;
    p.zchunk = 1;
    for (int k = 0; k < 2; ++k) { p.tau[k] = (float)tau[k]; p.itau[k] = (float)(1.0 / tau[k]); }
    p.G = (float)G;
    p.src = src;
    p.dst = dst;
    p.J = dens;
    const cudaStream_t s = (cudaStream_t)stream;
    // both kernels stride over the planes by gridDim.z, so grid.z stays
    // within the 65535 launch limit for any accepted lattice
    dim3 grid((nx + BX - 1) / BX, (ny + BY - 1) / BY, std::min(p.zhi - p.zlo, 65535)), block(BX, BY);
    k_density_static<<<grid, block, 0, s>>>(p);
    k_collide_static<<<grid, block, 0, s>>>(p);
    e = cudaGetLastError();
    if (e != cudaSuccess) { set_last_error(cudaGetErrorString(e)); return CF_ECUDA; }
    return CF_OK;
}
