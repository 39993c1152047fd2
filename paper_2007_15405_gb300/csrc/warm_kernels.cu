// Kernels of the learned warm start (sm_103a): a small 3-D convolutional
// network trained on equilibrated fields of the coupled method and used to
// predict an initial density field.
//
// Layers are 3x3x3 convolutions with zero padding and a dilation, at most 16
// input and 16 output channels, followed by a ReLU or by nothing.
// Activations and weights are stored in bfloat16, every product is
// accumulated in float32, gradients and the optimiser's master weights are
// float32.  Layout: activations [n][c][nz][ny][nx], weights [cout][cin][27]
// (tap = (dz+1)*9 + (dy+1)*3 + (dx+1)).  With at most 16 x 16 channels each
// voxel's contraction is 27 * cin * cout multiply-adds, too few to fill
// tensor-core tiles, so the layers run on the FP32 pipes: one thread per
// voxel holds all output channels in registers, the layer's weights sit in
// shared memory.
#include "cf_common.cuh"
#include "../../include/capfilm.h"

#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>

namespace cf {

constexpr int MAXC = 16;       // channels per layer, at most
constexpr int CONV_T = 128;    // threads per block (voxel kernels)

struct ConvShape {
    int n, cin, cout, nz, ny, nx, dil;
    long long V;               // voxels per sample
};

__device__ __forceinline__ float bf(const __nv_bfloat16 *p, long long i) { return __bfloat162float(p[i]); }

// offset (dz, dy, dx) of tap t, times the dilation
__device__ __forceinline__ void tap_off(int t, int dil, int &dz, int &dy, int &dx) {
    dz = (t / 9 - 1) * dil;
    dy = ((t / 3) % 3 - 1) * dil;
    dx = (t % 3 - 1) * dil;
}

__global__ void __launch_bounds__(CONV_T) k_conv_fwd(ConvShape s, const __nv_bfloat16 *__restrict__ x,
                                                    const __nv_bfloat16 *__restrict__ w,
                                                    const float *__restrict__ b, int relu,
                                                    __nv_bfloat16 *__restrict__ y) {
    __shared__ float ws[MAXC * MAXC * 27];
    const int nw = s.cout * s.cin * 27;
    for (int i = threadIdx.x; i < nw; i += blockDim.x) ws[i] = bf(w, i);
    __syncthreads();
    const long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (g >= s.n * s.V) return;
    const int smp = (int)(g / s.V);
    const long long v = g - smp * s.V;
    const int z = (int)(v / ((long long)s.ny * s.nx)), yy = (int)((v / s.nx) % s.ny), xx = (int)(v % s.nx);
    float acc[MAXC];
#pragma unroll
    for (int co = 0; co < MAXC; ++co) acc[co] = co < s.cout ? b[co] : 0.f;
    for (int ci = 0; ci < s.cin; ++ci) {
        const __nv_bfloat16 *xc = x + ((long long)smp * s.cin + ci) * s.V;
        for (int t = 0; t < 27; ++t) {
            int dz, dy, dx;
            tap_off(t, s.dil, dz, dy, dx);
            const int zz = z + dz, y2 = yy + dy, x2 = xx + dx;
            if (zz < 0 || zz >= s.nz || y2 < 0 || y2 >= s.ny || x2 < 0 || x2 >= s.nx) continue;
            const float xv = bf(xc, ((long long)zz * s.ny + y2) * s.nx + x2);
            const float *wt = ws + ci * 27 + t;
#pragma unroll
            for (int co = 0; co < MAXC; ++co)
                if (co < s.cout) acc[co] += wt[co * s.cin * 27] * xv;
        }
    }
#pragma unroll
    for (int co = 0; co < MAXC; ++co)
        if (co < s.cout) {
            const float o = relu ? fmaxf(acc[co], 0.f) : acc[co];
            y[((long long)smp * s.cout + co) * s.V + v] = __float2bfloat16_rn(o);
        }
}

// gradient with respect to the layer input: each input voxel gathers from the
// output voxels it fed, gy masked by the ReLU of the layer's output
__global__ void __launch_bounds__(CONV_T) k_conv_bwd_data(ConvShape s, const __nv_bfloat16 *__restrict__ w,
                                                         const __nv_bfloat16 *__restrict__ y, int relu,
                                                         const float *__restrict__ gy,
                                                         float *__restrict__ gx) {
    __shared__ float ws[MAXC * MAXC * 27];
    const int nw = s.cout * s.cin * 27;
    for (int i = threadIdx.x; i < nw; i += blockDim.x) ws[i] = bf(w, i);
    __syncthreads();
    const long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (g >= s.n * s.V) return;
    const int smp = (int)(g / s.V);
    const long long v = g - smp * s.V;
    const int z = (int)(v / ((long long)s.ny * s.nx)), yy = (int)((v / s.nx) % s.ny), xx = (int)(v % s.nx);
    float acc[MAXC];
#pragma unroll
    for (int ci = 0; ci < MAXC; ++ci) acc[ci] = 0.f;
    for (int co = 0; co < s.cout; ++co) {
        const long long base = ((long long)smp * s.cout + co) * s.V;
        for (int t = 0; t < 27; ++t) {
            int dz, dy, dx;
            tap_off(t, s.dil, dz, dy, dx);
            const int zz = z - dz, y2 = yy - dy, x2 = xx - dx;  // output voxel fed through tap t
            if (zz < 0 || zz >= s.nz || y2 < 0 || y2 >= s.ny || x2 < 0 || x2 >= s.nx) continue;
            const long long u = ((long long)zz * s.ny + y2) * s.nx + x2;
            float gv = gy[base + u];
            if (relu && !(bf(y, base + u) > 0.f)) gv = 0.f;
            const float *wt = ws + co * s.cin * 27 + t;
#pragma unroll
            for (int ci = 0; ci < MAXC; ++ci)
                if (ci < s.cin) acc[ci] += wt[ci * 27] * gv;
        }
    }
#pragma unroll
    for (int ci = 0; ci < MAXC; ++ci)
        if (ci < s.cin) gx[((long long)smp * s.cin + ci) * s.V + v] = acc[ci];
}

// Gradient with respect to weights and bias.  A block takes a range of
// voxels; its threads are the (input channel, tap) pairs.  Per chunk of WCH
// voxels the block stages the masked output gradient of every output channel
// and the voxels' sample and coordinates in shared memory; every thread then
// adds gy'[co][v] x[ci][v + tap] over the chunk for all co, and books each
// weight with one atomic at the end.  The bias gradient rides on the centre
// tap of input channel 0.
constexpr int WCH = 128;  // voxels staged per chunk
__global__ void k_conv_bwd_weight(ConvShape s, const __nv_bfloat16 *__restrict__ x,
                                  const __nv_bfloat16 *__restrict__ y, int relu,
                                  const float *__restrict__ gy, long long per_block,
                                  float *__restrict__ gw, float *__restrict__ gb) {
    __shared__ float gs[MAXC][WCH];
    __shared__ int cs[WCH], cz[WCH], cy[WCH], cx[WCH];  // sample and coordinates
    const int tid = threadIdx.x;
    const bool active = tid < s.cin * 27;
    const int ci = active ? tid / 27 : 0, t = tid % 27;
    int dz = 0, dy = 0, dx = 0;
    tap_off(t, s.dil, dz, dy, dx);
    const bool bias = active && ci == 0 && t == 13;
    float acc[MAXC], accb[MAXC];
#pragma unroll
    for (int co = 0; co < MAXC; ++co) { acc[co] = 0.f; accb[co] = 0.f; }
    const long long total = s.n * s.V;
    const long long g0 = blockIdx.x * per_block, g1 = min(total, g0 + per_block);
    for (long long c0 = g0; c0 < g1; c0 += WCH) {
        const int m = (int)min((long long)WCH, g1 - c0);
        __syncthreads();
        for (int j = tid; j < m; j += blockDim.x) {
            const long long g = c0 + j;
            const int smp = (int)(g / s.V);
            const long long v = g - smp * s.V;
            cs[j] = smp;
            cz[j] = (int)(v / ((long long)s.ny * s.nx));
            cy[j] = (int)((v / s.nx) % s.ny);
            cx[j] = (int)(v % s.nx);
        }
        for (int i = tid; i < s.cout * WCH; i += blockDim.x) {
            const int co = i / WCH, j = i % WCH;
            float gv = 0.f;
            if (j < m) {
                const long long g = c0 + j;
                const int smp = (int)(g / s.V);
                const long long idx = ((long long)smp * s.cout + co) * s.V + (g - smp * s.V);
                gv = gy[idx];
                if (relu && !(bf(y, idx) > 0.f)) gv = 0.f;
            }
            gs[co][j] = gv;
        }
        __syncthreads();
        if (!active) continue;
        for (int j = 0; j < m; ++j) {
            const int zz = cz[j] + dz, y2 = cy[j] + dy, x2 = cx[j] + dx;
            float xv = 0.f;
            if (zz >= 0 && zz < s.nz && y2 >= 0 && y2 < s.ny && x2 >= 0 && x2 < s.nx)
                xv = bf(x, ((long long)cs[j] * s.cin + ci) * s.V + ((long long)zz * s.ny + y2) * s.nx + x2);
#pragma unroll
            for (int co = 0; co < MAXC; ++co)
                if (co < s.cout) {
                    acc[co] += gs[co][j] * xv;
                    if (bias) accb[co] += gs[co][j];
                }
        }
    }
    if (!active) return;
#pragma unroll
    for (int co = 0; co < MAXC; ++co)
        if (co < s.cout) {
            atomicAdd(gw + (co * s.cin + ci) * 27 + t, acc[co]);
            if (bias) atomicAdd(gb + co, accb[co]);
        }
}

// masked mean squared error: loss += sum mask (p - q)^2 / msum, grad = 2 mask (p - q) / msum
__global__ void k_mse(const __nv_bfloat16 *__restrict__ pred, const float *__restrict__ target,
                      const float *__restrict__ mask, long long m, float inv_msum,
                      float *__restrict__ grad, double *__restrict__ loss) {
    double part = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < m;
         i += (long long)gridDim.x * blockDim.x) {
        const float k = mask ? mask[i] : 1.f;
        const float d = bf(pred, i) - target[i];
        grad[i] = 2.f * k * d * inv_msum;
        part += (double)(k * d * d * inv_msum);
    }
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(loss, part);
}

// Adam on float master weights (bias-corrected moments), bfloat16 copies
__global__ void k_adam(float *__restrict__ w, __nv_bfloat16 *__restrict__ wb, const float *__restrict__ g,
                       float *__restrict__ m1, float *__restrict__ m2, long long n, float lr, float b1,
                       float b2, float eps, float c1, float c2) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float a = b1 * m1[i] + (1.f - b1) * gi;
        const float q = b2 * m2[i] + (1.f - b2) * gi * gi;
        m1[i] = a;
        m2[i] = q;
        const float wi = w[i] - lr * (a * c1) / (sqrtf(q * c2) + eps);
        w[i] = wi;
        if (wb) wb[i] = __float2bfloat16_rn(wi);
    }
}

__global__ void k_to_bf16(const float *__restrict__ x, __nv_bfloat16 *__restrict__ y, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        y[i] = __float2bfloat16_rn(x[i]);
}

__global__ void k_from_bf16(const __nv_bfloat16 *__restrict__ x, float *__restrict__ y, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        y[i] = __bfloat162float(x[i]);
}

// ----------------------------------------------- warm-start set-up kernels
// The network's inputs, the state set from its prediction and its training
// targets are per-node functions of the lattice and the film; the residual
// check reduces the fields.  Block sums go to per-block partials, which every
// consumer adds in index order (results do not depend on block scheduling).
constexpr int WB = 256;           // threads per block of these kernels
constexpr int WARM_BLOCKS = 608;  // blocks (4 per SM), fixed so partials fit a known size

__device__ __forceinline__ int warm_z(const WarmGeom &g, long long n) {
    return (int)(n / ((long long)g.nx * g.ny));
}
// the flat film's phi: +1 below the mixed plane, 0 in it, -1 above and inside
// capsules, 0 on the substrate plane
__device__ __forceinline__ float warm_phi(const WarmGeom &g, int z, bool ins) {
    float phi = z < g.zm ? 1.f : z == g.zm ? 0.f : -1.f;
    if (ins) phi = -1.f;
    if (g.wall && z == 0) phi = 0.f;
    return phi;
}
// the flat film's densities (no jitter) from its phi
__device__ __forceinline__ void warm_film(const WarmGeom &g, float phi, int z, double &fa, double &fb) {
    fa = phi > 0.5f ? g.rmaj : phi < -0.5f ? g.rmin : g.rmix;
    fb = phi > 0.5f ? g.rmin : phi < -0.5f ? g.rmaj : g.rmix;
    if (g.wall && z == 0) fa = fb = 0.0;
}

__global__ void __launch_bounds__(WB) k_warm_features(WarmGeom g, const uint8_t *__restrict__ inside, float lks,
                                                      float *__restrict__ x, float *__restrict__ mask) {
    const long long N = g.N;
    for (long long n = blockIdx.x * (long long)WB + threadIdx.x; n < N; n += (long long)gridDim.x * WB) {
        const int z = warm_z(g, n);
        const bool ins = inside[n] != 0;
        x[n] = ins ? 1.f : 0.f;
        x[N + n] = warm_phi(g, z, ins);
        x[2 * N + n] = (float)z / (float)g.nz;
        x[3 * N + n] = lks;
        if (mask) mask[n] = (!ins && z >= (g.wall ? 1 : 0)) ? 1.f : 0.f;
    }
}

// sum of 4 doubles over the block into part[4 * blockIdx.x + j]
__device__ __forceinline__ void block_sum4(double (&v)[4], double *part) {
    __shared__ double sh[WB / 32][4];
#pragma unroll
    for (int j = 0; j < 4; ++j)
        for (int o = 16; o > 0; o >>= 1) v[j] += __shfl_xor_sync(0xffffffffu, v[j], o);
    if ((threadIdx.x & 31) == 0)
        for (int j = 0; j < 4; ++j) sh[threadIdx.x >> 5][j] = v[j];
    __syncthreads();
    if (threadIdx.x < 4) {
        double s = 0.0;
        for (int w = 0; w < WB / 32; ++w) s += sh[w][threadIdx.x];
        part[4 * blockIdx.x + threadIdx.x] = s;
    }
}

// predicted densities: the film plus the corrections on the fluid outside
// the capsules (at least 1e-3), the film inside and on the substrate; sums of
// the film's and the prediction's masses on that fluid
__global__ void __launch_bounds__(WB) k_warm_dens(WarmGeom g, const uint8_t *__restrict__ inside,
                                                  const float *__restrict__ d, double *__restrict__ r,
                                                  double *__restrict__ part) {
    const long long N = g.N;
    double v[4] = {0.0, 0.0, 0.0, 0.0};  // film A, predicted A, film B, predicted B
    for (long long n = blockIdx.x * (long long)WB + threadIdx.x; n < N; n += (long long)gridDim.x * WB) {
        const int z = warm_z(g, n);
        const bool ins = inside[n] != 0;
        double fa, fb;
        warm_film(g, warm_phi(g, z, ins), z, fa, fb);
        const bool free = !ins && !(g.wall && z == 0);
        const double ra = free ? fmax(fa + g.drho * (double)d[n], 1e-3) : fa;
        const double rb = free ? fmax(fb + g.drho * (double)d[N + n], 1e-3) : fb;
        r[n] = ra;
        r[N + n] = rb;
        if (free) { v[0] += fa; v[1] += ra; v[2] += fb; v[3] += rb; }
    }
    block_sum4(v, part);
}

// scale each component on the free fluid to the film's mass
__global__ void __launch_bounds__(WB) k_warm_rescale(WarmGeom g, const uint8_t *__restrict__ inside,
                                                     const double *__restrict__ part, int nparts,
                                                     double *__restrict__ r) {
    double t[4] = {0.0, 0.0, 0.0, 0.0};
    for (int b = 0; b < nparts; ++b)
        for (int j = 0; j < 4; ++j) t[j] += part[4 * b + j];
    const double sa = t[1] > 0.0 ? t[0] / t[1] : 1.0, sb = t[3] > 0.0 ? t[2] / t[3] : 1.0;
    const long long N = g.N;
    for (long long n = blockIdx.x * (long long)WB + threadIdx.x; n < N; n += (long long)gridDim.x * WB) {
        const int z = warm_z(g, n);
        if (inside[n] != 0 || (g.wall && z == 0)) continue;
        r[n] *= sa;
        r[N + n] *= sb;
    }
}

// training targets: (rho_c - rho_c,film) / (rho_maj - rho_min) on the fluid
// outside the capsules, 0 elsewhere; rho_c from the recorded fields
__global__ void __launch_bounds__(WB) k_warm_target(WarmGeom g, const uint8_t *__restrict__ inside,
                                                    const float *__restrict__ out, float *__restrict__ t) {
    const long long N = g.N;
    for (long long n = blockIdx.x * (long long)WB + threadIdx.x; n < N; n += (long long)gridDim.x * WB) {
        const int z = warm_z(g, n);
        const bool ins = inside[n] != 0;
        double fa, fb;
        warm_film(g, warm_phi(g, z, ins), z, fa, fb);
        const bool m = !ins && z >= (g.wall ? 1 : 0);
        t[n] = m ? (float)(((double)out[n] - fa) / g.drho) : 0.f;
        t[N + n] = m ? (float)(((double)out[N + n] - fb) / g.drho) : 0.f;
    }
}

// residual check: finite flag, smallest density, largest |u| component, sum
// of |rho - snapshot| over both components; the snapshot takes the densities
__global__ void __launch_bounds__(WB) k_field_check(long long N, const float *__restrict__ out,
                                                    float *__restrict__ snap, double *__restrict__ part) {
    double v[4] = {1.0, 1e300, 0.0, 0.0};
    for (long long i = blockIdx.x * (long long)WB + threadIdx.x; i < 5 * N; i += (long long)gridDim.x * WB) {
        const float q = out[i];
        if (!isfinite(q)) v[0] = 0.0;
        if (i < 2 * N) {
            v[1] = fmin(v[1], (double)q);
            v[3] += fabs((double)q - (double)snap[i]);
            snap[i] = q;
        } else {
            v[2] = fmax(v[2], fabs((double)q));
        }
    }
    // reduce: min for the flag and the smallest density, max for |u|, sum
    __shared__ double sh[WB / 32][4];
    for (int o = 16; o > 0; o >>= 1) {
        v[0] = fmin(v[0], __shfl_xor_sync(0xffffffffu, v[0], o));
        v[1] = fmin(v[1], __shfl_xor_sync(0xffffffffu, v[1], o));
        v[2] = fmax(v[2], __shfl_xor_sync(0xffffffffu, v[2], o));
        v[3] += __shfl_xor_sync(0xffffffffu, v[3], o);
    }
    if ((threadIdx.x & 31) == 0)
        for (int j = 0; j < 4; ++j) sh[threadIdx.x >> 5][j] = v[j];
    __syncthreads();
    if (threadIdx.x == 0) {
        double a[4] = {sh[0][0], sh[0][1], sh[0][2], sh[0][3]};
        for (int w = 1; w < WB / 32; ++w) {
            a[0] = fmin(a[0], sh[w][0]); a[1] = fmin(a[1], sh[w][1]);
            a[2] = fmax(a[2], sh[w][2]); a[3] += sh[w][3];
        }
        for (int j = 0; j < 4; ++j) part[4 * blockIdx.x + j] = a[j];
    }
}

__global__ void k_field_check_final(const double *__restrict__ part, int nparts, long long N,
                                    double *__restrict__ res) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double a[4] = {1.0, 1e300, 0.0, 0.0};
    for (int b = 0; b < nparts; ++b) {
        a[0] = fmin(a[0], part[4 * b]); a[1] = fmin(a[1], part[4 * b + 1]);
        a[2] = fmax(a[2], part[4 * b + 2]); a[3] += part[4 * b + 3];
    }
    res[0] = a[0]; res[1] = a[1]; res[2] = a[2]; res[3] = a[3] / (2.0 * (double)N);
}

cudaError_t launch_warm_features(const WarmGeom &g, const uint8_t *inside, float lks, float *x, float *mask,
                                 cudaStream_t s) {
    k_warm_features<<<WARM_BLOCKS, WB, 0, s>>>(g, inside, lks, x, mask);
    return cudaGetLastError();
}

cudaError_t launch_warm_densities(const WarmGeom &g, const uint8_t *inside, const float *d, double *r,
                                  double *part, cudaStream_t s) {
    k_warm_dens<<<WARM_BLOCKS, WB, 0, s>>>(g, inside, d, r, part);
    k_warm_rescale<<<WARM_BLOCKS, WB, 0, s>>>(g, inside, part, WARM_BLOCKS, r);
    return cudaGetLastError();
}

cudaError_t launch_warm_target(const WarmGeom &g, const uint8_t *inside, const float *out, float *t,
                               cudaStream_t s) {
    k_warm_target<<<WARM_BLOCKS, WB, 0, s>>>(g, inside, out, t);
    return cudaGetLastError();
}

cudaError_t launch_field_check(long long N, const float *out, float *snap, double *part, double *res,
                               cudaStream_t s) {
    k_field_check<<<WARM_BLOCKS, WB, 0, s>>>(N, out, snap, part);
    k_field_check_final<<<1, 32, 0, s>>>(part, WARM_BLOCKS, N, res);
    return cudaGetLastError();
}

int warm_parts() { return WARM_BLOCKS; }

namespace {
cf_status conv_check(int n, int cin, int cout, int nz, int ny, int nx, int dil) {
    if (n < 1 || cin < 1 || cout < 1 || cin > MAXC || cout > MAXC || nz < 1 || ny < 1 || nx < 1 || dil < 1) {
        set_last_error("conv3d: need 1 <= channels <= 16, positive sizes and dilation");
        return CF_EINVAL;
    }
    return CF_OK;
}
ConvShape shape(int n, int cin, int cout, int nz, int ny, int nx, int dil) {
    ConvShape s{n, cin, cout, nz, ny, nx, dil, (long long)nz * ny * nx};
    return s;
}
cf_status cuda_status(cudaError_t e) {
    if (e == cudaSuccess) return CF_OK;
    set_last_error(cudaGetErrorString(e));
    return CF_ECUDA;
}
unsigned blocks_for(long long m) { return (unsigned)std::min<long long>((m + 255) / 256, 152LL * 16); }
}  // namespace

}  // namespace cf

using namespace cf;

extern "C" {

cf_status cf_conv3d_forward(const void *x, int n, int cin, int nz, int ny, int nx, const void *w,
                            const float *b, int cout, int dil, int relu, void *y, void *stream) {
    cf_status st = conv_check(n, cin, cout, nz, ny, nx, dil);
    if (st != CF_OK) return st;
    if (!x || !w || !b || !y) { set_last_error("conv3d: null pointer"); return CF_EINVAL; }
    const ConvShape s = shape(n, cin, cout, nz, ny, nx, dil);
    const long long m = s.n * s.V;
    k_conv_fwd<<<(unsigned)((m + CONV_T - 1) / CONV_T), CONV_T, 0, (cudaStream_t)stream>>>(
        s, static_cast<const __nv_bfloat16 *>(x), static_cast<const __nv_bfloat16 *>(w), b, relu,
        static_cast<__nv_bfloat16 *>(y));
    return cuda_status(cudaGetLastError());
}

cf_status cf_conv3d_backward(const void *x, int n, int cin, int nz, int ny, int nx, const void *w,
                             int cout, int dil, const void *y, int relu, const float *gy, float *gx,
                             float *gw, float *gb, void *stream) {
    cf_status st = conv_check(n, cin, cout, nz, ny, nx, dil);
    if (st != CF_OK) return st;
    if (!x || !w || !gy || !gw || !gb || (relu && !y)) { set_last_error("conv3d: null pointer"); return CF_EINVAL; }
    const ConvShape s = shape(n, cin, cout, nz, ny, nx, dil);
    const long long m = s.n * s.V;
    const cudaStream_t cs = (cudaStream_t)stream;
    const auto *xb = static_cast<const __nv_bfloat16 *>(x);
    const auto *wb = static_cast<const __nv_bfloat16 *>(w);
    const auto *yb = static_cast<const __nv_bfloat16 *>(y);
    if (gx)
        k_conv_bwd_data<<<(unsigned)((m + CONV_T - 1) / CONV_T), CONV_T, 0, cs>>>(s, wb, yb, relu, gy, gx);
    // about 4 * 152 blocks of (cin * 27) threads, each over a contiguous voxel range
    const long long nb = std::min<long long>(608, (m + WCH - 1) / WCH);
    const long long per = ((m + nb - 1) / nb + WCH - 1) / WCH * WCH;
    const int threads = std::max(((cin * 27 + 31) / 32) * 32, 128);
    k_conv_bwd_weight<<<(unsigned)((m + per - 1) / per), threads, 0, cs>>>(s, xb, yb, relu, gy, per, gw, gb);
    return cuda_status(cudaGetLastError());
}

cf_status cf_mse(const void *pred, const float *target, const float *mask, long long m, double msum,
                 float *grad, double *loss, void *stream) {
    if (!pred || !target || !grad || !loss || m < 1 || !(msum > 0)) {
        set_last_error("mse: bad argument");
        return CF_EINVAL;
    }
    k_mse<<<blocks_for(m), 256, 0, (cudaStream_t)stream>>>(static_cast<const __nv_bfloat16 *>(pred), target,
                                                            mask, m, (float)(1.0 / msum), grad, loss);
    return cuda_status(cudaGetLastError());
}

cf_status cf_adam(float *w, void *w_bf16, const float *g, float *m1, float *m2, long long n, double lr,
                  double b1, double b2, double eps, int t, void *stream) {
    if (!w || !g || !m1 || !m2 || n < 1 || t < 1) { set_last_error("adam: bad argument"); return CF_EINVAL; }
    const float c1 = (float)(1.0 / (1.0 - std::pow(b1, t))), c2 = (float)(1.0 / (1.0 - std::pow(b2, t)));
    k_adam<<<blocks_for(n), 256, 0, (cudaStream_t)stream>>>(w, static_cast<__nv_bfloat16 *>(w_bf16), g, m1, m2,
                                                             n, (float)lr, (float)b1, (float)b2, (float)eps,
                                                             c1, c2);
    return cuda_status(cudaGetLastError());
}

cf_status cf_to_bf16(const float *x, void *y, long long n, void *stream) {
    if (!x || !y || n < 0) { set_last_error("to_bf16: bad argument"); return CF_EINVAL; }
    if (n == 0) return CF_OK;
    k_to_bf16<<<blocks_for(n), 256, 0, (cudaStream_t)stream>>>(x, static_cast<__nv_bfloat16 *>(y), n);
    return cuda_status(cudaGetLastError());
}

cf_status cf_from_bf16(const void *x, float *y, long long n, void *stream) {
    if (!x || !y || n < 0) { set_last_error("from_bf16: bad argument"); return CF_EINVAL; }
    if (n == 0) return CF_OK;
    k_from_bf16<<<blocks_for(n), 256, 0, (cudaStream_t)stream>>>(static_cast<const __nv_bfloat16 *>(x), y, n);
    return cuda_status(cudaGetLastError());
}

}  // extern "C"
