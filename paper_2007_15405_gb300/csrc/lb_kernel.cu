// Fused two-component Shan-Chen lattice Boltzmann step (sm_103a).
//
// One launch performs, for every fluid node, the whole lattice part of a time
// step of the coupled method (Sec. 3.1): pull-streaming of both components
// with half-way bounce-back on the substrate and on membrane-cut links (Ladd's
// moving-wall term), the momentum those bounces exchange with the membrane
// elements, the densities and pseudopotentials psi = 1 - exp(-rho), the
// Shan-Chen force (Eq. 10) with the interior/exterior decoupling, and the BGK
// collision (Eqs. 4-5) with the velocity-shift forcing.
//
// Layout: populations f[c][i][z][y][x] (float), two buffers (src -> dst).
// Each CTA owns a TX x TY column tile and marches through a chunk of z planes.
// The densities and pseudopotentials of three consecutive planes (tile plus a
// one-node halo) live in a shared-memory ring, so the Shan-Chen stencil needs
// no second pass over the populations: each population is read once and
// written once per step (304 bytes per node update), plus the halo recomputes
// which neighbouring tiles/chunks fetch concurrently (L2 hits).  Alternate z
// chunks march in opposite directions so that the planes two chunks share are
// loaded at the same time.
#include "cf_common.cuh"

namespace cf {

template <int TX, int TY>
struct Ring {
    float rho[3][2][TY + 2][TX + 2];
    float psi[3][2][TY + 2][TX + 2];
};

__device__ __forceinline__ int slot3(int z) { return ((z % 3) + 3) % 3; }
__device__ __forceinline__ float psi_of(float r) { return -expm1f(-r); }

// plane zu (unwrapped) is solid when the substrate is on
__device__ __forceinline__ bool solid_plane(const LBParams &p, int zu) {
    return p.wall && (wrapi(zu, p.nz) == 0);
}

// Pull the 2 x 19 post-streaming populations of node (x, y, z) (z wrapped,
// fluid).  OWNER: this thread owns the node and books the momentum exchange.
template <bool OWNER>
__device__ __forceinline__ void pull_node(const LBParams &p, int x, int y, int z, float (&fa)[Q],
                                          float (&fb)[Q], uint32_t &m) {
    const int nx = p.nx, ny = p.ny, nz = p.nz;
    const long long N = p.N;
    const int xm = x == 0 ? nx - 1 : x - 1, xp = x == nx - 1 ? 0 : x + 1;
    const int ym = y == 0 ? ny - 1 : y - 1, yp = y == ny - 1 ? 0 : y + 1;
    const int zm = z == 0 ? nz - 1 : z - 1, zp = z == nz - 1 ? 0 : z + 1;
    const long long n = ((long long)z * ny + y) * nx + x;
    const float *__restrict__ sA = p.src;
    const float *__restrict__ sB = p.src + (long long)Q * N;
    m = p.mask[n];
    const bool wall_below = p.wall && zm == 0;  // pulling from z-1 hits the substrate
    const bool wall_above = p.wall && zp == 0;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        // source node x - e_i
        const int sx = ex(i) == 1 ? xm : ex(i) == -1 ? xp : x;
        const int sy = ey(i) == 1 ? ym : ey(i) == -1 ? yp : y;
        const int sz = ez(i) == 1 ? zm : ez(i) == -1 ? zp : z;
        const bool wb = (ez(i) == 1 && wall_below) || (ez(i) == -1 && wall_above);
        long long s;
        int d;
        if (wb) { s = n; d = opp(i); }
        else { s = ((long long)sz * ny + sy) * nx + sx; d = i; }
        fa[i] = __ldg(sA + (long long)d * N + s);
        fb[i] = __ldg(sB + (long long)d * N + s);
    }
    if (m) {
        // membrane-cut links: bounce back what this node sent towards the
        // membrane, with Ladd's term -2 w_k rho (e_k . u_T)/c_s^2, where rho
        // is this node's density (= sum of its post-collision populations)
        // and u_T the mean velocity of the crossed element's three nodes.
        float rwa = 0.f, rwb = 0.f;
#pragma unroll
        for (int j = 0; j < Q; ++j) {
            rwa += __ldg(sA + (long long)j * N + n);
            rwb += __ldg(sB + (long long)j * N + n);
        }
#pragma unroll
        for (int k = 1; k < Q; ++k) {
            if ((m >> (k - 1)) & 1u) {
                const int T = __ldg(p.tri + n * 18 + (k - 1));
                const int a = __ldg(p.faces + 3 * T), b = __ldg(p.faces + 3 * T + 1),
                          c = __ldg(p.faces + 3 * T + 2);
                const float ux = (p.V[3 * a] + p.V[3 * b] + p.V[3 * c]) * (1.0f / 3.0f);
                const float uy = (p.V[3 * a + 1] + p.V[3 * b + 1] + p.V[3 * c + 1]) * (1.0f / 3.0f);
                const float uz = (p.V[3 * a + 2] + p.V[3 * b + 2] + p.V[3 * c + 2]) * (1.0f / 3.0f);
                const float eu = ex(k) * ux + ey(k) * uy + ez(k) * uz;
                const float foa = __ldg(sA + (long long)k * N + n);
                const float fob = __ldg(sB + (long long)k * N + n);
                const float ca = 6.0f * wgt(k) * rwa * eu;
                const float cb = 6.0f * wgt(k) * rwb * eu;
                fa[opp(k)] = foa - ca;
                fb[opp(k)] = fob - cb;
                if (OWNER) {
                    const float sx = (2.0f * foa - ca) + (2.0f * fob - cb);
                    if (ex(k)) atomicAdd(p.FT + 3 * T + 0, ex(k) * sx);
                    if (ey(k)) atomicAdd(p.FT + 3 * T + 1, ey(k) * sx);
                    if (ez(k)) atomicAdd(p.FT + 3 * T + 2, ez(k) * sx);
                }
            }
        }
    }
}

template <int TX, int TY>
__device__ __forceinline__ void store_ring(Ring<TX, TY> &R, int sl, int cy, int cx, float ra, float rb) {
    R.rho[sl][0][cy][cx] = ra;
    R.rho[sl][1][cy][cx] = rb;
    R.psi[sl][0][cy][cx] = psi_of(ra);
    R.psi[sl][1][cy][cx] = psi_of(rb);
}

// Densities of the halo ring of plane zu (unwrapped) into the shared ring.
template <int TX, int TY>
__device__ __forceinline__ void load_halo(const LBParams &p, Ring<TX, TY> &R, int zu, int x0, int y0) {
    constexpr int NH = 2 * (TX + 2) + 2 * TY;
    const int t = threadIdx.y * TX + threadIdx.x;
    const int z = wrapi(zu, p.nz);
    const int sl = slot3(zu);
    for (int h = t; h < NH; h += TX * TY) {
        int cx, cy;
        if (h < TX + 2) { cx = h; cy = 0; }
        else if (h < 2 * (TX + 2)) { cx = h - (TX + 2); cy = TY + 1; }
        else if (h < 2 * (TX + 2) + TY) { cx = 0; cy = 1 + h - 2 * (TX + 2); }
        else { cx = TX + 1; cy = 1 + h - 2 * (TX + 2) - TY; }
        const int x = wrapi(x0 - 1 + cx, p.nx), y = wrapi(y0 - 1 + cy, p.ny);
        float fa[Q], fb[Q];
        uint32_t m;
        pull_node<false>(p, x, y, z, fa, fb, m);
        float ra = 0.f, rb = 0.f;
#pragma unroll
        for (int i = 0; i < Q; ++i) { ra += fa[i]; rb += fb[i]; }
        store_ring(R, sl, cy, cx, ra, rb);
    }
}

// Shan-Chen force with decoupling, velocity shift, BGK, store.
template <int TX, int TY>
__device__ __forceinline__ void collide_node(const LBParams &p, const Ring<TX, TY> &R, int zu, int x,
                                             int y, const float (&fa)[Q], const float (&fb)[Q],
                                             uint32_t m) {
    const int cx = threadIdx.x + 1, cy = threadIdx.y + 1;
    const int z = wrapi(zu, p.nz);
    const int s0 = slot3(zu), sm = slot3(zu - 1), sp = slot3(zu + 1);
    const float ra = R.rho[s0][0][cy][cx], rb = R.rho[s0][1][cy][cx];
    const float pa = R.psi[s0][0][cy][cx], pb = R.psi[s0][1][cy][cx];
    const bool wall_lo = solid_plane(p, zu - 1), wall_hi = solid_plane(p, zu + 1);
    float sa[3] = {0.f, 0.f, 0.f}, sb[3] = {0.f, 0.f, 0.f};  // sum_k w_k psi'(x+e_k) e_k
    const long long n = ((long long)z * p.ny + y) * p.nx + x;
    if (!m && !wall_lo && !wall_hi) {
#pragma unroll
        for (int k = 1; k < Q; ++k) {
            const int sl = ez(k) == 1 ? sp : ez(k) == -1 ? sm : s0;
            const float qa = R.psi[sl][0][cy + ey(k)][cx + ex(k)];
            const float qb = R.psi[sl][1][cy + ey(k)][cx + ex(k)];
            sa[0] += wgt(k) * ex(k) * qa; sa[1] += wgt(k) * ey(k) * qa; sa[2] += wgt(k) * ez(k) * qa;
            sb[0] += wgt(k) * ex(k) * qb; sb[1] += wgt(k) * ey(k) * qb; sb[2] += wgt(k) * ez(k) * qb;
        }
    } else {
        // partner densities across a cut or substrate link: mean over this
        // node and its neighbours reached through uncut fluid links
        float ia = ra, ib = rb, cnt = 1.f;
#pragma unroll
        for (int k = 1; k < Q; ++k) {
            const bool solid = (ez(k) == 1 && wall_hi) || (ez(k) == -1 && wall_lo);
            const bool cut = (m >> (k - 1)) & 1u;
            if (!solid && !cut) {
                const int sl = ez(k) == 1 ? sp : ez(k) == -1 ? sm : s0;
                ia += R.rho[sl][0][cy + ey(k)][cx + ex(k)];
                ib += R.rho[sl][1][cy + ey(k)][cx + ex(k)];
                cnt += 1.f;
            }
        }
        const float qa_eff = psi_of(ia / cnt), qb_eff = psi_of(ib / cnt);
#pragma unroll
        for (int k = 1; k < Q; ++k) {
            const bool solid = (ez(k) == 1 && wall_hi) || (ez(k) == -1 && wall_lo);
            const bool cut = (m >> (k - 1)) & 1u;
            float qa, qb;
            if (solid || cut) {
                qa = qa_eff; qb = qb_eff;
                if (cut && !solid) {
                    // reaction of the decoupled interaction on the crossed element
                    const int T = __ldg(p.tri + n * 18 + (k - 1));
                    const float r = p.G * wgt(k) * (pa * qb_eff + pb * qa_eff);
                    if (ex(k)) atomicAdd(p.FT + 3 * T + 0, ex(k) * r);
                    if (ey(k)) atomicAdd(p.FT + 3 * T + 1, ey(k) * r);
                    if (ez(k)) atomicAdd(p.FT + 3 * T + 2, ez(k) * r);
                }
            } else {
                const int sl = ez(k) == 1 ? sp : ez(k) == -1 ? sm : s0;
                qa = R.psi[sl][0][cy + ey(k)][cx + ex(k)];
                qb = R.psi[sl][1][cy + ey(k)][cx + ex(k)];
            }
            sa[0] += wgt(k) * ex(k) * qa; sa[1] += wgt(k) * ey(k) * qa; sa[2] += wgt(k) * ez(k) * qa;
            sb[0] += wgt(k) * ex(k) * qb; sb[1] += wgt(k) * ey(k) * qb; sb[2] += wgt(k) * ez(k) * qb;
        }
    }
    // Eq. 10 with G^{AB} = G^{BA} = G, G^{AA} = G^{BB} = 0
    const float FA[3] = {-p.G * pa * sb[0], -p.G * pa * sb[1], -p.G * pa * sb[2]};
    const float FB[3] = {-p.G * pb * sa[0], -p.G * pb * sa[1], -p.G * pb * sa[2]};
    float ja[3] = {0.f, 0.f, 0.f}, jb[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int i = 1; i < Q; ++i) {
        ja[0] += ex(i) * fa[i]; ja[1] += ey(i) * fa[i]; ja[2] += ez(i) * fa[i];
        jb[0] += ex(i) * fb[i]; jb[1] += ey(i) * fb[i]; jb[2] += ez(i) * fb[i];
    }
    // velocity shift: common velocity weighted by 1/tau, u^{c,eq} = u' + tau^c F^c / rho^c
    const float den = ra * p.itau[0] + rb * p.itau[1];
    float ua[3], ub[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float up = (ja[a] * p.itau[0] + jb[a] * p.itau[1]) / den;
        ua[a] = up + p.tau[0] * FA[a] / ra;
        ub[a] = up + p.tau[1] * FB[a] / rb;
    }
    if (p.out) {
        const float rt = ra + rb;
        p.out[n] = ra;
        p.out[p.N + n] = rb;
        p.out[2 * p.N + n] = (ja[0] + jb[0] + 0.5f * (FA[0] + FB[0])) / rt;
        p.out[3 * p.N + n] = (ja[1] + jb[1] + 0.5f * (FA[1] + FB[1])) / rt;
        p.out[4 * p.N + n] = (ja[2] + jb[2] + 0.5f * (FA[2] + FB[2])) / rt;
    }
    if (!(ra + rb < 1e30f)) atomicOr(p.status, ST_NAN);
    const float uua = ua[0] * ua[0] + ua[1] * ua[1] + ua[2] * ua[2];
    const float uub = ub[0] * ub[0] + ub[1] * ub[1] + ub[2] * ub[2];
    float *__restrict__ dA = p.dst;
    float *__restrict__ dB = p.dst + (long long)Q * p.N;
    // Eq. 5; the rest population takes the mass balance (sum_i f^eq_i = rho)
    // so that the float32 weights (which sum to 1 + 1.5e-8) create no mass
    float qa0 = ra, qb0 = rb;
#pragma unroll
    for (int i = 1; i < Q; ++i) {
        const float eua = ex(i) * ua[0] + ey(i) * ua[1] + ez(i) * ua[2];
        const float eub = ex(i) * ub[0] + ey(i) * ub[1] + ez(i) * ub[2];
        const float qa = wgt(i) * ra * (1.0f + 3.0f * eua + 4.5f * eua * eua - 1.5f * uua);
        const float qb = wgt(i) * rb * (1.0f + 3.0f * eub + 4.5f * eub * eub - 1.5f * uub);
        qa0 -= qa;
        qb0 -= qb;
        dA[(long long)i * p.N + n] = fa[i] - (fa[i] - qa) * p.itau[0];
        dB[(long long)i * p.N + n] = fb[i] - (fb[i] - qb) * p.itau[1];
    }
    dA[n] = fa[0] - (fa[0] - qa0) * p.itau[0];
    dB[n] = fb[0] - (fb[0] - qb0) * p.itau[1];
}

template <int TX, int TY>
__global__ void __launch_bounds__(TX *TY, 2) k_lb_fused(const LBParams p) {
    __shared__ Ring<TX, TY> R;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int chunk = blockIdx.z;
    const int z0 = p.zlo + chunk * p.zchunk;
    const int z1 = min(z0 + p.zchunk, p.zhi);
    if (z0 >= z1) return;
    const int dir = (chunk & 1) ? -1 : 1;
    const int zs = dir > 0 ? z0 : z1 - 1;
    const int cnt = z1 - z0;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int x = wrapi(x0 + tx, p.nx), y = wrapi(y0 + ty, p.ny);
    const bool active = (x0 + tx < p.nx) && (y0 + ty < p.ny);

    float ca[Q], cb[Q], na[Q], nb[Q];
    uint32_t cm = 0, nm = 0;

    // plane before the chunk (densities only)
    {
        const int zu = zs - dir;
        if (!solid_plane(p, zu)) {
            pull_node<false>(p, x, y, wrapi(zu, p.nz), na, nb, nm);
            float ra = 0.f, rb = 0.f;
#pragma unroll
            for (int i = 0; i < Q; ++i) { ra += na[i]; rb += nb[i]; }
            store_ring(R, slot3(zu), ty + 1, tx + 1, ra, rb);
            load_halo(p, R, zu, x0, y0);
        }
    }
    // first plane of the chunk
    {
        if (active) pull_node<true>(p, x, y, wrapi(zs, p.nz), ca, cb, cm);
        else pull_node<false>(p, x, y, wrapi(zs, p.nz), ca, cb, cm);
        float ra = 0.f, rb = 0.f;
#pragma unroll
        for (int i = 0; i < Q; ++i) { ra += ca[i]; rb += cb[i]; }
        store_ring(R, slot3(zs), ty + 1, tx + 1, ra, rb);
        load_halo(p, R, zs, x0, y0);
    }
    for (int s = 0; s < cnt; ++s) {
        const int zu = zs + s * dir;
        const int zn = zu + dir;
        if (s + 1 < cnt || !solid_plane(p, zn)) {
            const bool keep = s + 1 < cnt;
            if (keep && active) pull_node<true>(p, x, y, wrapi(zn, p.nz), na, nb, nm);
            else pull_node<false>(p, x, y, wrapi(zn, p.nz), na, nb, nm);
            float ra = 0.f, rb = 0.f;
#pragma unroll
            for (int i = 0; i < Q; ++i) { ra += na[i]; rb += nb[i]; }
            store_ring(R, slot3(zn), ty + 1, tx + 1, ra, rb);
            load_halo(p, R, zn, x0, y0);
        }
        __syncthreads();
        if (active) collide_node<TX, TY>(p, R, zu, x, y, ca, cb, cm);
#pragma unroll
        for (int i = 0; i < Q; ++i) { ca[i] = na[i]; cb[i] = nb[i]; }
        cm = nm;
        __syncthreads();
    }
}

cudaError_t launch_lb_step(const LBParams &p, int variant, cudaStream_t s) {
    const int nzf = p.zhi - p.zlo;
    const int nch = (nzf + p.zchunk - 1) / p.zchunk;
    if (variant == 1) {
        dim3 grid((p.nx + 31) / 32, (p.ny + 7) / 8, nch), block(32, 8);
        k_lb_fused<32, 8><<<grid, block, 0, s>>>(p);
    } else {
        dim3 grid((p.nx + 31) / 32, (p.ny + 3) / 4, nch), block(32, 4);
        k_lb_fused<32, 4><<<grid, block, 0, s>>>(p);
    }
    return cudaGetLastError();
}

// ------------------------------------------------------------ film set-up
__global__ void k_init_film(float *f, long long N, int nx, int ny, int nz, int wall, float h_top,
                           float rmaj, float rmin, float rmix, const double *jit,
                           const uint8_t *inside) {
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
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const double w = i == 0 ? 1.0 / 3.0 : (i <= 6 ? 1.0 / 18.0 : 1.0 / 36.0);
        f[(long long)i * N + n] = (float)(w * r[0]);
        f[(long long)(Q + i) * N + n] = (float)(w * r[1]);
    }
}

cudaError_t launch_init_film(float *f, long long N, int nx, int ny, int nz, int wall, float h_top,
                             float rmaj, float rmin, float rmix, const double *jit,
                             const uint8_t *inside, cudaStream_t s) {
    k_init_film<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(f, N, nx, ny, nz, wall, h_top, rmaj,
                                                             rmin, rmix, jit, inside);
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

// FP64 mass of each component
__global__ void k_mass(const float *f, long long N, double *m2) {
    double s[2] = {0.0, 0.0};
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < N;
         n += (long long)gridDim.x * blockDim.x) {
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            s[0] += f[(long long)i * N + n];
            s[1] += f[(long long)(Q + i) * N + n];
        }
    }
    for (int c = 0; c < 2; ++c) {
        double v = s[c];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) == 0) atomicAdd(m2 + c, v);
    }
}

cudaError_t launch_mass(const float *f, long long N, double *m2, cudaStream_t s) {
    k_mass<<<304, 256, 0, s>>>(f, N, m2);
    return cudaGetLastError();
}

}  // namespace cf
