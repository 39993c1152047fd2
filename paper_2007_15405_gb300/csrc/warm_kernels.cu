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
