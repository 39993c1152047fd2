// Tensor-core layers of the learned warm start's 3-D U-net (sm_103a).
//
// Activations are channels-last bfloat16, a[n][z][y][x][c], with the channel
// count a multiple of 16; weights are bfloat16 [27][cout][cin] (tap-major,
// tap = (dz+1)*9 + (dy+1)*3 + (dx+1)); biases, gradients of the weights and
// the optimiser's master weights are float32.
//
// A 3x3x3 convolution with zero padding is an implicit GEMM: output voxels
// are the rows (M), output channels the columns (N), and (tap, input
// channel) the contraction (K).  Each warp computes a 16-voxel x 32-channel
// tile with mma.sync m16n8k16 (bf16 in, fp32 accumulate): per tap and per
// 16 input channels it loads one A fragment (16 voxels x 16 channels, the
// tap-shifted voxels' channel rows, contiguous in the channels-last layout)
// and four B fragments (16 channels x 8 outputs, contiguous in the
// [27][cout][cin] layout).  The input gradient is the same kernel with the
// weights mirrored in space and transposed in channels.  The weight gradient
// is a GEMM over the voxels (M = output channels, N = input channels, K =
// voxels), split into a fixed number of voxel chunks whose partial sums are
// reduced in a fixed order afterwards, so training is bitwise reproducible.
#include "cf_common.cuh"
#include "../../include/capfilm.h"

#include <cuda_bf16.h>

#include <algorithm>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <vector>

namespace cf {

namespace {

__device__ __forceinline__ void mma_bf16(float (&c)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ uint32_t ld32(const __nv_bfloat16 *p) { return __ldg(reinterpret_cast<const uint32_t *>(p)); }
__device__ __forceinline__ uint32_t pack2(__nv_bfloat16 lo, __nv_bfloat16 hi) {
    return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

struct Grid3 {
    int n, nz, ny, nx;
    long long V;  // voxels per sample
};

// linear voxel index of (sample s, z, y, x) shifted by tap t, or -1 outside
__device__ __forceinline__ long long shifted(const Grid3 &g, int s, int z, int y, int x, int t) {
    const int zz = z + t / 9 - 1, yy = y + (t / 3) % 3 - 1, xx = x + t % 3 - 1;
    if ((unsigned)zz >= (unsigned)g.nz || (unsigned)yy >= (unsigned)g.ny || (unsigned)xx >= (unsigned)g.nx)
        return -1;
    return (long long)s * g.V + ((long long)zz * g.ny + yy) * g.nx + xx;
}

constexpr int CW = 4;  // warps per block of the convolution

// y[v][co] = act(b[co] + sum_t sum_ci w[t][co][ci] x[v + off(t)][ci]); a warp
// owns 16 voxels x 32 output channels (cout a multiple of 8; channels beyond
// cout are skipped).  OUTF: float output, else bfloat16.
template <bool OUTF>
__global__ void __launch_bounds__(32 * CW) k_conv_mma(Grid3 g, const __nv_bfloat16 *__restrict__ x, int cin,
                                                     const __nv_bfloat16 *__restrict__ w,
                                                     const float *__restrict__ b, int cout, int relu,
                                                     void *__restrict__ yout) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int gi = lane >> 2, ti = lane & 3;
    const long long total = (long long)g.n * g.V;
    const long long v0 = ((long long)blockIdx.x * CW + warp) * 16;
    const int co0 = blockIdx.y * 32;
    if (v0 >= total) return;
    // the two voxel rows this thread loads (gi and gi + 8)
    int s[2], z[2], y[2], xx[2];
    bool ok[2];
    for (int r = 0; r < 2; ++r) {
        const long long v = v0 + gi + 8 * r;
        ok[r] = v < total;
        const long long vv = ok[r] ? v : 0;
        s[r] = (int)(vv / g.V);
        const long long l = vv - (long long)s[r] * g.V;
        z[r] = (int)(l / ((long long)g.ny * g.nx));
        y[r] = (int)((l / g.nx) % g.ny);
        xx[r] = (int)(l % g.nx);
    }
    float acc[4][4];
    for (int j = 0; j < 4; ++j)
        for (int q = 0; q < 4; ++q) acc[j][q] = 0.f;
    for (int t = 0; t < 27; ++t) {
        long long src[2];
        for (int r = 0; r < 2; ++r) src[r] = ok[r] ? shifted(g, s[r], z[r], y[r], xx[r], t) : -1;
        const __nv_bfloat16 *wt = w + (size_t)t * cout * cin;
        for (int c0 = 0; c0 < cin; c0 += 16) {
            uint32_t a[4];
            a[0] = src[0] >= 0 ? ld32(x + src[0] * cin + c0 + 2 * ti) : 0u;
            a[1] = src[1] >= 0 ? ld32(x + src[1] * cin + c0 + 2 * ti) : 0u;
            a[2] = src[0] >= 0 ? ld32(x + src[0] * cin + c0 + 2 * ti + 8) : 0u;
            a[3] = src[1] >= 0 ? ld32(x + src[1] * cin + c0 + 2 * ti + 8) : 0u;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int co = co0 + 8 * j + gi;
                if (co0 + 8 * j >= cout) break;
                uint32_t bb[2];
                const __nv_bfloat16 *wr = wt + (size_t)co * cin + c0 + 2 * ti;
                bb[0] = ld32(wr);
                bb[1] = ld32(wr + 8);
                mma_bf16(acc[j], a, bb);
            }
        }
    }
    // epilogue: rows gi / gi + 8, columns 2 ti, 2 ti + 1 of each 8-channel block
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int c = co0 + 8 * j + 2 * ti;
        if (co0 + 8 * j >= cout) break;
        const float b0 = b ? b[c] : 0.f, b1 = b ? b[c + 1] : 0.f;
        for (int r = 0; r < 2; ++r) {
            if (!ok[r]) continue;
            const long long v = v0 + gi + 8 * r;
            float o0 = acc[j][2 * r] + b0, o1 = acc[j][2 * r + 1] + b1;
            if (relu) { o0 = fmaxf(o0, 0.f); o1 = fmaxf(o1, 0.f); }
            if (OUTF) {
                float *yo = static_cast<float *>(yout) + v * cout + c;
                yo[0] = o0;
                yo[1] = o1;
            } else {
                __nv_bfloat16 *yo = static_cast<__nv_bfloat16 *>(yout) + v * cout + c;
                *reinterpret_cast<uint32_t *>(yo) = pack2(__float2bfloat16_rn(o0), __float2bfloat16_rn(o1));
            }
        }
    }
}

// ------------------------------------------------------------------------
// The same convolution on the 5th-generation tensor cores (tcgen05).  A block
// owns 128 consecutive voxels (the MMA's M) and all cout output channels (N).
// For each of the 27 taps the block stages the shifted input rows A_t
// [128][cin] (zero rows outside the grid) and the tap's weights B_t
// [cout][cin] in shared memory, as K-major operands without swizzle: 8-row x
// 16-byte core matrices, K blocks adjacent (128 B apart), row blocks
// cin * 16 B apart.  One thread issues the tap's cin / 16 MMAs (M = 128,
// N = cout, K = 16, bf16 inputs, fp32 accumulation in tensor memory) and
// commits them to the stage's mbarrier; two stages let the loads of one tap
// overlap the MMAs of the previous one.  The epilogue reads the accumulators
// from tensor memory (each warp its 32 rows), adds the bias, applies the ReLU
// and stores bfloat16 (or float) rows.  Waits are bounded: a wait that runs
// out sets *err and the block frees its tensor memory and returns.
__device__ unsigned g_tc_err;  // a tensor-core convolution gave up a wait

namespace tc {

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory operand descriptor: start >> 4 (bits 0-13), leading byte
// offset >> 4 (16-29), stride byte offset >> 4 (32-45), descriptor version 1
// (46-47), no swizzle (61-63 = 0)
__device__ __forceinline__ uint64_t desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((saddr >> 4) & 0x3fffu) | ((uint64_t)((lbo >> 4) & 0x3fffu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3fffu) << 32) | (1ull << 46);
}
// instruction descriptor of kind::f16: fp32 accumulator (bits 4-5 = 1), bf16 A
// and B (7-9 = 1, 10-12 = 1), both K-major, N >> 3 (17-22), M >> 4 (24-28)
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
// bounded wait for the phase of parity `phase`; false when the limit ran out
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, unsigned phase) {
    const uint32_t a = smem_u32(bar);
    for (int it = 0; it < (1 << 20); ++it) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(a), "r"(phase)
            : "memory");
        if (done) return true;
    }
    return false;
}

template <bool OUTF>
__global__ void __launch_bounds__(128, 1) k_conv_tc(Grid3 g, const __nv_bfloat16 *__restrict__ x, int cin,
                                                    const __nv_bfloat16 *__restrict__ w,
                                                    const float *__restrict__ b, int cout, int relu,
                                                    void *__restrict__ yout, unsigned *__restrict__ err) {
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ uint64_t bar[2];
    __shared__ uint32_t tmem_base;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const long long total = (long long)g.n * g.V;
    const long long v0 = (long long)blockIdx.x * 128;
    const int kb = cin / 8;                       // 16-byte chunks per row
    const uint32_t a_bytes = 128u * cin * 2u, b_bytes = (uint32_t)cout * cin * 2u;
    const uint32_t stage_bytes = a_bytes + b_bytes;
    const int ncols = cout <= 32 ? 32 : (cout <= 64 ? 64 : (cout <= 128 ? 128 : 256));
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "r"(ncols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base;
    const uint32_t idesc = idesc_bf16(128, cout);
    // this thread's row of A: voxel v0 + tid, its coordinates decoded once
    const long long vr = v0 + tid;
    const bool vin = vr < total;
    int rz = 0, ry = 0, rx = 0;
    long long sbase = 0;
    if (vin) {
        const long long sm = vr / g.V, l = vr - sm * g.V;
        sbase = sm * g.V;
        rz = (int)(l / ((long long)g.ny * g.nx));
        const int rem = (int)(l - (long long)rz * g.ny * g.nx);
        ry = rem / g.nx;
        rx = rem - ry * g.nx;
    }
    unsigned char *const arow = smem + ((tid >> 3) * kb) * 128 + (tid & 7) * 16;  // chunk q at + q * 128
    bool ok = true;
    for (int t = 0; t < 27 && ok; ++t) {
        const int st = t & 1;
        unsigned char *sa = smem + st * stage_bytes, *sb = sa + a_bytes;
        if (t >= 2) ok = mbar_wait(&bar[st], ((t - 2) >> 1) & 1);  // the MMAs of tap t - 2 read this stage
        if (__syncthreads_and(ok) == 0) { ok = false; break; }
        // A_t: the thread's row shifted by tap t (zero outside the grid), all cin channels
        {
            const int zz = rz + t / 9 - 1, yy = ry + (t / 3) % 3 - 1, xx = rx + t % 3 - 1;
            const bool in = vin && (unsigned)zz < (unsigned)g.nz && (unsigned)yy < (unsigned)g.ny &&
                            (unsigned)xx < (unsigned)g.nx;
            const uint4 *src =
                reinterpret_cast<const uint4 *>(x + (sbase + ((long long)zz * g.ny + yy) * g.nx + xx) * cin);
            unsigned char *dst = arow + st * stage_bytes;
            for (int q = 0; q < kb; ++q)
                *reinterpret_cast<uint4 *>(dst + q * 128) = in ? __ldg(src + q) : make_uint4(0u, 0u, 0u, 0u);
        }
        // B_t: weights w[t][co][ci], row co
        const __nv_bfloat16 *wt = w + (size_t)t * cout * cin;
        for (int i = tid; i < cout * kb; i += 128) {
            const int r = i / kb, q = i - r * kb;
            const uint4 val = __ldg(reinterpret_cast<const uint4 *>(wt + (size_t)r * cin) + q);
            *reinterpret_cast<uint4 *>(sb + ((r >> 3) * kb + q) * 128 + (r & 7) * 16) = val;
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // visible to the tensor cores
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t a0 = smem_u32(sa), b0 = smem_u32(sb), sbo = (uint32_t)cin * 16u;
            for (int ks = 0; ks < cin / 16; ++ks) {
                const uint64_t ad = desc(a0 + ks * 256u, 128u, sbo), bd = desc(b0 + ks * 256u, 128u, sbo);
                const uint32_t acc = (t > 0 || ks > 0) ? 1u : 0u;
                asm volatile(
                    "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                    " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                    "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
                    : "memory");
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_u32(&bar[st]))
                         : "memory");
        }
    }
    // the last commit covers every MMA issued before it (taps 25 and 26 both)
    if (ok) ok = mbar_wait(&bar[0], 1) && mbar_wait(&bar[1], 0);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (__syncthreads_and(ok)) {
        const long long v = v0 + warp * 32 + lane;
        for (int c = 0; c < cout; c += 8) {
            uint32_t r[8];
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];\n"
                : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                : "r"(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            if (v >= total) continue;
            float o[8];
            for (int j = 0; j < 8; ++j) {
                o[j] = __uint_as_float(r[j]) + (b ? b[c + j] : 0.f);
                if (relu) o[j] = fmaxf(o[j], 0.f);
            }
            if (OUTF) {
                float4 *yo = reinterpret_cast<float4 *>(static_cast<float *>(yout) + v * cout + c);
                yo[0] = make_float4(o[0], o[1], o[2], o[3]);
                yo[1] = make_float4(o[4], o[5], o[6], o[7]);
            } else {
                uint4 pk;
                pk.x = pack2(__float2bfloat16_rn(o[0]), __float2bfloat16_rn(o[1]));
                pk.y = pack2(__float2bfloat16_rn(o[2]), __float2bfloat16_rn(o[3]));
                pk.z = pack2(__float2bfloat16_rn(o[4]), __float2bfloat16_rn(o[5]));
                pk.w = pack2(__float2bfloat16_rn(o[6]), __float2bfloat16_rn(o[7]));
                *reinterpret_cast<uint4 *>(static_cast<__nv_bfloat16 *>(yout) + v * cout + c) = pk;
            }
        }
    } else if (tid == 0) {
        atomicOr(err, 1u);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols) : "memory");
}

}  // namespace tc

// wt[26 - t][ci][co] = w[t][co][ci]: the input gradient is the convolution of
// the output gradient with the weights mirrored in space, channels transposed
__global__ void k_flip(const __nv_bfloat16 *__restrict__ w, int cin, int cout, __nv_bfloat16 *__restrict__ wt) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const long long nW = 27LL * cout * cin;
    if (i >= nW) return;
    const int t = (int)(i / ((long long)cout * cin));
    const int co = (int)((i / cin) % cout), ci = (int)(i % cin);
    wt[((size_t)(26 - t) * cin + ci) * cout + co] = w[i];
}

// Weight gradient, chunk `blockIdx.z` of the voxels: part[chunk][t][co][ci] =
// sum over the chunk's voxels v of gy[v][co] x[v + off(t)][ci].  A warp owns
// 16 output x 32 input channels of one tap (blockIdx.y = tap * ceil(cout/16)
// + output-channel block, blockIdx.x * CW + warp = input-channel block of
// 32); channels beyond cout / cin are skipped.
__global__ void __launch_bounds__(32 * CW) k_wgrad_mma(Grid3 g, const __nv_bfloat16 *__restrict__ x, int cin,
                                                      const __nv_bfloat16 *__restrict__ gy, int cout,
                                                      long long chunk, float *__restrict__ part) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int gi = lane >> 2, ti = lane & 3;
    const int cob = (cout + 15) / 16;
    const int t = blockIdx.y / cob, co0 = (blockIdx.y % cob) * 16;
    const int ci0 = (blockIdx.x * CW + warp) * 32;
    if (ci0 >= cin) return;
    const long long total = (long long)g.n * g.V;
    const long long vb = (long long)blockIdx.z * chunk, ve = min(total, vb + chunk);
    float acc[4][4];
    for (int j = 0; j < 4; ++j)
        for (int q = 0; q < 4; ++q) acc[j][q] = 0.f;
    for (long long k0 = vb; k0 < ve; k0 += 16) {
        // the four voxels of this thread's fragment columns: k0 + 2 ti + {0, 1, 8, 9}
        long long vv[4], src[4];
        for (int q = 0; q < 4; ++q) {
            vv[q] = k0 + 2 * ti + (q & 1) + 8 * (q >> 1);
            src[q] = -1;
            if (vv[q] < ve) {
                const int s = (int)(vv[q] / g.V);
                const long long l = vv[q] - (long long)s * g.V;
                src[q] = shifted(g, s, (int)(l / ((long long)g.ny * g.nx)), (int)((l / g.nx) % g.ny),
                                 (int)(l % g.nx), t);
            }
        }
        const __nv_bfloat16 zero = __float2bfloat16_rn(0.f);
        uint32_t a[4];
        for (int r = 0; r < 2; ++r) {  // A[m = co][k = voxel]: rows gi, gi + 8 (zero beyond cout)
            const int co = co0 + gi + 8 * r;
            const bool cok = co < cout;
            const __nv_bfloat16 e0 = cok && vv[0] < ve ? gy[vv[0] * cout + co] : zero;
            const __nv_bfloat16 e1 = cok && vv[1] < ve ? gy[vv[1] * cout + co] : zero;
            const __nv_bfloat16 e2 = cok && vv[2] < ve ? gy[vv[2] * cout + co] : zero;
            const __nv_bfloat16 e3 = cok && vv[3] < ve ? gy[vv[3] * cout + co] : zero;
            a[r] = pack2(e0, e1);
            a[r + 2] = pack2(e2, e3);
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {  // B[k = voxel][n = ci]: column gi of block j
            const int ci = ci0 + 8 * j + gi;
            if (ci0 + 8 * j >= cin) break;
            uint32_t bb[2];
            const __nv_bfloat16 e0 = src[0] >= 0 ? x[src[0] * cin + ci] : zero;
            const __nv_bfloat16 e1 = src[1] >= 0 ? x[src[1] * cin + ci] : zero;
            const __nv_bfloat16 e2 = src[2] >= 0 ? x[src[2] * cin + ci] : zero;
            const __nv_bfloat16 e3 = src[3] >= 0 ? x[src[3] * cin + ci] : zero;
            bb[0] = pack2(e0, e1);
            bb[1] = pack2(e2, e3);
            mma_bf16(acc[j], a, bb);
        }
    }
    float *pt = part + ((size_t)blockIdx.z * 27 + t) * cout * cin;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int ci = ci0 + 8 * j + 2 * ti;
        if (ci0 + 8 * j >= cin) break;
        for (int r = 0; r < 2; ++r) {
            const int co = co0 + gi + 8 * r;
            if (co >= cout) continue;
            pt[(size_t)co * cin + ci] = acc[j][2 * r];
            pt[(size_t)co * cin + ci + 1] = acc[j][2 * r + 1];
        }
    }
}

// gw[i] += sum over the chunks in order of part[chunk][i]
__global__ void k_wgrad_reduce(const float *__restrict__ part, int chunks, long long nW, float *__restrict__ gw) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= nW) return;
    float s = 0.f;
    for (int k = 0; k < chunks; ++k) s += part[(size_t)k * nW + i];
    gw[i] += s;
}

// gb[co] += sum over all voxels of gy[v][co], one block per channel, fixed order
__global__ void k_bias_grad(const __nv_bfloat16 *__restrict__ gy, long long total, int cout, float *__restrict__ gb) {
    __shared__ float red[256];
    const int co = blockIdx.x;
    float s = 0.f;
    for (long long v = threadIdx.x; v < total; v += blockDim.x) s += __bfloat162float(gy[v * cout + co]);
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) gb[co] += red[0];
}

// out = bf16((g + g2) * (y > 0)) with y the layer's output (ReLU mask), or
// without the mask when y is null; g2 (a second gradient reaching the same
// activation, e.g. through a skip connection) may be null
__global__ void k_relu_grad(const float *__restrict__ g, const float *__restrict__ g2,
                            const __nv_bfloat16 *__restrict__ y, long long m, __nv_bfloat16 *__restrict__ out) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= m) return;
    float v = g[i] + (g2 ? g2[i] : 0.f);
    if (y && !(__bfloat162float(y[i]) > 0.f)) v = 0.f;
    out[i] = __float2bfloat16_rn(v);
}

// Loss of the U-net's head (float [n][V][ch], channels 0, 1: density
// corrections; 2, 3, 4: displacement field) and its gradient g (same shape):
//   density:      wd / msum * sum_{s,c,v} mask (out_c - t_c)^2,  t [n][2][V], mask [n][V]
//   displacement: wx / nodes * sum_{s,i} |D(X_i) - d_i|^2, D the displacement
//                 channels interpolated trilinearly at the node's reference
//                 position X_i (lattice units, clamped inside the grid),
//                 d_i the node's target displacement
// The density part is elementwise; the displacement part is taken by one
// thread per sample walking its nodes in order (the gradient scatter is then
// in a fixed order); the loss is summed per block and then in block order.
__global__ void k_loss_density(int n, long long V, int ch, const float *__restrict__ out,
                               const float *__restrict__ t, const float *__restrict__ mask, double scale,
                               float *__restrict__ g, double *__restrict__ part) {
    __shared__ double red[256];
    const long long tot = (long long)n * V;
    double acc = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < tot;
         i += (long long)gridDim.x * blockDim.x) {
        const int s = (int)(i / V);
        const long long v = i - (long long)s * V;
        const float m = mask[i];
        for (int c = 0; c < ch; ++c) g[i * ch + c] = 0.f;
        for (int c = 0; c < 2; ++c) {
            const float d = out[i * ch + c] - t[((long long)s * 2 + c) * V + v];
            acc += scale * m * d * d;
            g[i * ch + c] = (float)(2.0 * scale * m * d);
        }
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

__global__ void k_loss_nodes(int n, int nz, int ny, int nx, int ch, const float *__restrict__ out,
                             const float *__restrict__ X, const float *__restrict__ d, int nodes, double scale,
                             float *__restrict__ g, double *__restrict__ part) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    const long long V = (long long)nz * ny * nx;
    const float *o = out + (long long)s * V * ch;
    float *gs = g + (long long)s * V * ch;
    double acc = 0.0;
    for (int i = 0; i < nodes; ++i) {
        const float *xi = X + ((long long)s * nodes + i) * 3;
        const float px = fminf(fmaxf(xi[0], 0.f), nx - 1.001f), py = fminf(fmaxf(xi[1], 0.f), ny - 1.001f),
                    pz = fminf(fmaxf(xi[2], 0.f), nz - 1.001f);
        const int x0 = (int)px, y0 = (int)py, z0 = (int)pz;
        const float fx = px - x0, fy = py - y0, fz = pz - z0;
        float D[3] = {0.f, 0.f, 0.f};
        for (int k = 0; k < 8; ++k) {
            const int dx = k & 1, dy = (k >> 1) & 1, dz = k >> 2;
            const float wgt = (dx ? fx : 1.f - fx) * (dy ? fy : 1.f - fy) * (dz ? fz : 1.f - fz);
            const long long v = ((long long)(z0 + dz) * ny + (y0 + dy)) * nx + (x0 + dx);
            for (int a = 0; a < 3; ++a) D[a] += wgt * o[v * ch + 2 + a];
        }
        float r[3];
        for (int a = 0; a < 3; ++a) {
            r[a] = D[a] - d[((long long)s * nodes + i) * 3 + a];
            acc += scale * (double)r[a] * r[a];
        }
        for (int k = 0; k < 8; ++k) {
            const int dx = k & 1, dy = (k >> 1) & 1, dz = k >> 2;
            const float wgt = (dx ? fx : 1.f - fx) * (dy ? fy : 1.f - fy) * (dz ? fz : 1.f - fz);
            const long long v = ((long long)(z0 + dz) * ny + (y0 + dy)) * nx + (x0 + dx);
            for (int a = 0; a < 3; ++a) gs[v * ch + 2 + a] += (float)(2.0 * scale) * wgt * r[a];
        }
    }
    part[s] = acc;
}

__global__ void k_loss_sum(const double *__restrict__ part, int np, double *__restrict__ loss) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < np; ++i) s += part[i];
        *loss += s;
    }
}

// 2x2x2 average pooling, channels-last, fine grid (nz, ny, nx) even
template <typename T>
__device__ __forceinline__ float toF(T v);
template <> __device__ __forceinline__ float toF<float>(float v) { return v; }
template <> __device__ __forceinline__ float toF<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }

__global__ void k_pool(Grid3 f, int c, const __nv_bfloat16 *__restrict__ x, __nv_bfloat16 *__restrict__ y) {
    const int cz = f.nz / 2, cy = f.ny / 2, cx = f.nx / 2;
    const long long Vc = (long long)cz * cy * cx, tot = f.n * Vc * c;
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= tot) return;
    const int ch = (int)(i % c);
    const long long v = i / c;
    const int s = (int)(v / Vc);
    const long long l = v - s * Vc;
    const int Z = (int)(l / ((long long)cy * cx)), Y = (int)((l / cx) % cy), X = (int)(l % cx);
    float a = 0.f;
    for (int d = 0; d < 8; ++d) {
        const int z = 2 * Z + (d >> 2), yy = 2 * Y + ((d >> 1) & 1), xx = 2 * X + (d & 1);
        a += __bfloat162float(x[((s * f.V) + ((long long)z * f.ny + yy) * f.nx + xx) * c + ch]);
    }
    y[i] = __float2bfloat16_rn(0.125f * a);
}

// gradient of the pooling: every fine voxel gets 1/8 of its coarse voxel's
__global__ void k_pool_bwd(Grid3 f, int c, const float *__restrict__ gy, float *__restrict__ gx) {
    const long long tot = f.n * f.V * c;
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= tot) return;
    const int ch = (int)(i % c);
    const long long v = i / c;
    const int s = (int)(v / f.V);
    const long long l = v - s * f.V;
    const int z = (int)(l / ((long long)f.ny * f.nx)), yy = (int)((l / f.nx) % f.ny), xx = (int)(l % f.nx);
    const int cz = f.nz / 2, cy = f.ny / 2, cx = f.nx / 2;
    const long long Vc = (long long)cz * cy * cx;
    gx[i] = 0.125f * gy[(s * Vc + ((long long)(z / 2) * cy + yy / 2) * cx + xx / 2) * c + ch];
}

// nearest-neighbour upsampling by 2 from the coarse grid of the fine grid f
__global__ void k_upsample(Grid3 f, int c, const __nv_bfloat16 *__restrict__ x, __nv_bfloat16 *__restrict__ y) {
    const long long tot = f.n * f.V * c;
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= tot) return;
    const int ch = (int)(i % c);
    const long long v = i / c;
    const int s = (int)(v / f.V);
    const long long l = v - s * f.V;
    const int z = (int)(l / ((long long)f.ny * f.nx)), yy = (int)((l / f.nx) % f.ny), xx = (int)(l % f.nx);
    const int cy = f.ny / 2, cx = f.nx / 2;
    const long long Vc = (long long)(f.nz / 2) * cy * cx;
    y[i] = x[(s * Vc + ((long long)(z / 2) * cy + yy / 2) * cx + xx / 2) * c + ch];
}

// gradient of the upsampling: each coarse voxel sums its eight fine ones
__global__ void k_upsample_bwd(Grid3 f, int c, const float *__restrict__ gy, float *__restrict__ gx) {
    const int cz = f.nz / 2, cy = f.ny / 2, cx = f.nx / 2;
    const long long Vc = (long long)cz * cy * cx, tot = f.n * Vc * c;
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= tot) return;
    const int ch = (int)(i % c);
    const long long v = i / c;
    const int s = (int)(v / Vc);
    const long long l = v - s * Vc;
    const int Z = (int)(l / ((long long)cy * cx)), Y = (int)((l / cx) % cy), X = (int)(l % cx);
    float a = 0.f;
    for (int d = 0; d < 8; ++d) {
        const int z = 2 * Z + (d >> 2), yy = 2 * Y + ((d >> 1) & 1), xx = 2 * X + (d & 1);
        a += gy[((s * f.V) + ((long long)z * f.ny + yy) * f.nx + xx) * c + ch];
    }
    gx[i] = a;
}

// channel concatenation y[v] = (a[v][0..ca), b[v][0..cb)) and its split
template <typename T>
__global__ void k_concat(long long nv, const T *__restrict__ a, int ca, const T *__restrict__ b, int cb,
                         T *__restrict__ y) {
    const int c = ca + cb;
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= nv * c) return;
    const long long v = i / c;
    const int ch = (int)(i % c);
    y[i] = ch < ca ? a[v * ca + ch] : b[v * cb + ch - ca];
}
template <typename T>
__global__ void k_split(long long nv, const T *__restrict__ y, int ca, int cb, T *__restrict__ a, T *__restrict__ b) {
    const int c = ca + cb;
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= nv * c) return;
    const long long v = i / c;
    const int ch = (int)(i % c);
    if (ch < ca) { if (a) a[v * ca + ch] = y[i]; }
    else if (b) b[v * cb + ch - ca] = y[i];
}

// channel-first float [c][N] (one sample) <-> channels-last [N][cpad]
__global__ void k_pack(const float *__restrict__ x, int c, long long N, int cpad, __nv_bfloat16 *__restrict__ y) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= N * cpad) return;
    const long long v = i / cpad;
    const int ch = (int)(i % cpad);
    y[i] = __float2bfloat16_rn(ch < c ? x[(size_t)ch * N + v] : 0.f);
}
template <typename T>
__global__ void k_unpack(const T *__restrict__ x, int cpad, long long N, int c0, int c, float *__restrict__ y) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= N * c) return;
    const int ch = (int)(i / N);
    const long long v = i % N;
    y[i] = toF<T>(x[v * cpad + c0 + ch]);
}

inline unsigned nblk(long long n, int t = 256) { return (unsigned)((n + t - 1) / t); }
constexpr int LOSS_BLOCKS = 304;  // blocks of the density loss (two per SM)

cf_status ucheck(cudaError_t e) {
    if (e != cudaSuccess) {
        set_last_error(cudaGetErrorString(e));
        return CF_ECUDA;
    }
    return CF_OK;
}

cf_status bad(const char *m) {
    set_last_error(m);
    return CF_EINVAL;
}

bool grid_ok(int n, int nz, int ny, int nx) { return n >= 1 && nz >= 1 && ny >= 1 && nx >= 1; }

}  // namespace

// ------------------------------------------------------- the model on device
// The U-net's parameters (bfloat16 weights [27][cout][cin], float biases) in
// layer order e0a e0b e1a e1b ma mb d1a d1b d0a d0b head, for inference
// inside the library (cf_warmstart).
struct UNetModel {
    int w0 = 0, w1 = 0, w2 = 0;
    int cin[11] = {}, cout[11] = {};
    __nv_bfloat16 *w[11] = {};
    float *b[11] = {};
};

void unet_free(UNetModel *m) {
    if (!m) return;
    for (int k = 0; k < 11; ++k) {
        if (m->w[k]) cudaFree(m->w[k]);
        if (m->b[k]) cudaFree(m->b[k]);
    }
    delete m;
}

namespace {
__global__ void k_f32_to_bf16(const float *__restrict__ x, __nv_bfloat16 *__restrict__ y, long long n) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < n) y[i] = __float2bfloat16_rn(x[i]);
}
}  // namespace

// File: "CFUNET01", int32 w0 w1 w2, then per layer int32 cin, cout, float32
// weights [27][cout][cin], float32 biases [cout] (native byte order).
cf_status unet_load(const char *path, UNetModel **out) {
    FILE *fp = std::fopen(path, "rb");
    if (!fp) { set_last_error("cf_model_load: cannot open the file"); return CF_EINVAL; }
    char magic[8];
    int32_t wd[3];
    UNetModel *m = new UNetModel();
    auto fail_ = [&](const char *msg, cf_status st) { std::fclose(fp); unet_free(m); set_last_error(msg); return st; };
    if (std::fread(magic, 1, 8, fp) != 8 || std::memcmp(magic, "CFUNET01", 8) != 0 || std::fread(wd, 4, 3, fp) != 3)
        return fail_("cf_model_load: not a U-net weight file", CF_EINVAL);
    m->w0 = wd[0]; m->w1 = wd[1]; m->w2 = wd[2];
    const int W0 = wd[0], W1 = wd[1], W2 = wd[2];
    const int ecin[11] = {16, W0, W0, W1, W1, W2, W1 + W2, W1, W0 + W1, W0, W0};
    const int ecout[11] = {W0, W0, W1, W1, W2, W2, W1, W1, W0, W0, 16};
    for (int k = 0; k < 11; ++k) {
        int32_t cc[2];
        if (std::fread(cc, 4, 2, fp) != 2 || cc[0] != ecin[k] || cc[1] != ecout[k] || cc[0] % 16 || cc[1] % 16)
            return fail_("cf_model_load: layer shapes do not match the U-net", CF_EINVAL);
        m->cin[k] = cc[0];
        m->cout[k] = cc[1];
        const size_t nw = 27ull * cc[0] * cc[1];
        std::vector<float> hw(nw), hb(cc[1]);
        if (std::fread(hw.data(), 4, nw, fp) != nw || std::fread(hb.data(), 4, (size_t)cc[1], fp) != (size_t)cc[1])
            return fail_("cf_model_load: file truncated", CF_EINVAL);
        float *tmp = nullptr;
        if (cudaMalloc(&m->w[k], nw * 2) != cudaSuccess || cudaMalloc(&m->b[k], (size_t)cc[1] * 4) != cudaSuccess ||
            cudaMalloc(&tmp, nw * 4) != cudaSuccess) {
            if (tmp) cudaFree(tmp);
            return fail_("cf_model_load: device allocation failed", CF_ENOMEM);
        }
        cudaMemcpy(tmp, hw.data(), nw * 4, cudaMemcpyHostToDevice);
        cudaMemcpy(m->b[k], hb.data(), (size_t)cc[1] * 4, cudaMemcpyHostToDevice);
        k_f32_to_bf16<<<nblk((long long)nw), 256>>>(tmp, m->w[k], (long long)nw);
        const cudaError_t e = cudaDeviceSynchronize();
        cudaFree(tmp);
        if (e != cudaSuccess) return fail_(cudaGetErrorString(e), CF_ECUDA);
    }
    std::fclose(fp);
    *out = m;
    return CF_OK;
}

// Forward of one lattice (nz, ny, nx multiples of 4) from its features
// [4][N] (float, channel-first): density corrections dens [2][N] and the
// displacement field disp [3][N] (float, channel-first; either may be null).
// Temporaries come from cudaMallocAsync on the stream.
cf_status unet_forward(const UNetModel *m, const float *feats, int nz, int ny, int nx, float *dens, float *disp,
                       cudaStream_t s) {
    if (nz % 4 || ny % 4 || nx % 4) { set_last_error("the U-net needs lattice sizes divisible by 4"); return CF_EINVAL; }
    const long long N = (long long)nz * ny * nx, N1 = N / 8, N2 = N / 64;
    const int W0 = m->w0, W1 = m->w1, W2 = m->w2;
    std::vector<void *> bufs;
    auto alloc = [&](size_t bytes) -> void * {
        void *p = nullptr;
        if (cudaMallocAsync(&p, std::max<size_t>(bytes, 256), s) != cudaSuccess) return nullptr;
        bufs.push_back(p);
        return p;
    };
    auto bf = [&](long long n) { return static_cast<__nv_bfloat16 *>(alloc((size_t)n * 2)); };
    __nv_bfloat16 *x = bf(N * 16), *e0a = bf(N * W0), *e0b = bf(N * W0), *p1 = bf(N1 * W0), *e1a = bf(N1 * W1),
                  *e1b = bf(N1 * W1), *p2 = bf(N2 * W1), *ma = bf(N2 * W2), *mb = bf(N2 * W2), *u1 = bf(N1 * W2),
                  *c1 = bf(N1 * (W1 + W2)), *d1a = bf(N1 * W1), *d1b = bf(N1 * W1), *u0 = bf(N * W1),
                  *c0 = bf(N * (W0 + W1)), *d0a = bf(N * W0), *d0b = bf(N * W0);
    float *head = static_cast<float *>(alloc((size_t)N * 16 * 4));
    cf_status st = CF_OK;
    for (void *p : bufs)
        if (!p) st = CF_ENOMEM;
    // every layer on the tcgen05 convolution where its channel counts allow (all of the default widths)
    auto conv = [&](int k, const void *in, int gz, int gy, int gx, void *out, int f32) {
        if (st != CF_OK) return;
        const int ci = m->cin[k], co = m->cout[k], relu = k == 10 ? 0 : 1;
        if (ci % 16 == 0 && ci <= 256 && co % 16 == 0 && co <= 256)
            st = cf_unet_conv_tc(in, 1, gz, gy, gx, ci, m->w[k], m->b[k], co, relu, f32, out, s);
        else
            st = cf_unet_conv(in, 1, gz, gy, gx, ci, m->w[k], m->b[k], co, relu, f32, out, s);
    };
    if (st == CF_OK) st = cf_unet_pack(feats, 4, N, 16, x, s);
    conv(0, x, nz, ny, nx, e0a, 0);
    conv(1, e0a, nz, ny, nx, e0b, 0);
    if (st == CF_OK) st = cf_unet_pool(e0b, 1, nz, ny, nx, W0, p1, s);
    conv(2, p1, nz / 2, ny / 2, nx / 2, e1a, 0);
    conv(3, e1a, nz / 2, ny / 2, nx / 2, e1b, 0);
    if (st == CF_OK) st = cf_unet_pool(e1b, 1, nz / 2, ny / 2, nx / 2, W1, p2, s);
    conv(4, p2, nz / 4, ny / 4, nx / 4, ma, 0);
    conv(5, ma, nz / 4, ny / 4, nx / 4, mb, 0);
    if (st == CF_OK) st = cf_unet_upsample(mb, 1, nz / 2, ny / 2, nx / 2, W2, u1, s);
    if (st == CF_OK) st = cf_unet_concat(N1, e1b, W1, u1, W2, c1, s);
    conv(6, c1, nz / 2, ny / 2, nx / 2, d1a, 0);
    conv(7, d1a, nz / 2, ny / 2, nx / 2, d1b, 0);
    if (st == CF_OK) st = cf_unet_upsample(d1b, 1, nz, ny, nx, W1, u0, s);
    if (st == CF_OK) st = cf_unet_concat(N, e0b, W0, u0, W1, c0, s);
    conv(8, c0, nz, ny, nx, d0a, 0);
    conv(9, d0a, nz, ny, nx, d0b, 0);
    conv(10, d0b, nz, ny, nx, head, 1);
    if (st == CF_OK && dens) st = cf_unet_unpack(head, 1, 16, N, 0, 2, dens, s);
    if (st == CF_OK && disp) st = cf_unet_unpack(head, 1, 16, N, 2, 3, disp, s);
    for (void *p : bufs)
        if (p) cudaFreeAsync(p, s);
    if (st == CF_ENOMEM) set_last_error("device allocation failed (U-net activations)");
    return st;
}

}  // namespace cf

using namespace cf;

extern "C" {

cf_status cf_unet_conv(const void *x, int n, int nz, int ny, int nx, int cin, const void *w, const float *b,
                       int cout, int relu, int out_f32, void *y, void *stream) {
    if (!x || !w || !y) return bad("null argument");
    if (!grid_ok(n, nz, ny, nx) || cin < 16 || cin % 16 || cout < 8 || cout % 8)
        return bad("cf_unet_conv: bad shape (cin a multiple of 16, cout of 8)");
    const Grid3 g{n, nz, ny, nx, (long long)nz * ny * nx};
    const long long rows = (long long)n * g.V;
    const dim3 grid((unsigned)((rows + 16 * CW - 1) / (16 * CW)), (unsigned)((cout + 31) / 32));
    const cudaStream_t s = (cudaStream_t)stream;
    const auto *xb = static_cast<const __nv_bfloat16 *>(x);
    const auto *wb = static_cast<const __nv_bfloat16 *>(w);
    if (out_f32) k_conv_mma<true><<<grid, 32 * CW, 0, s>>>(g, xb, cin, wb, b, cout, relu, y);
    else k_conv_mma<false><<<grid, 32 * CW, 0, s>>>(g, xb, cin, wb, b, cout, relu, y);
    return ucheck(cudaGetLastError());
}

cf_status cf_unet_conv_tc(const void *x, int n, int nz, int ny, int nx, int cin, const void *w, const float *b,
                          int cout, int relu, int out_f32, void *y, void *stream) {
    if (!x || !w || !y) return bad("null argument");
    if (!grid_ok(n, nz, ny, nx) || cin < 16 || cin % 16 || cin > 256 || cout < 16 || cout % 16 || cout > 256)
        return bad("cf_unet_conv_tc: bad shape (cin and cout multiples of 16 up to 256)");
    const Grid3 g{n, nz, ny, nx, (long long)nz * ny * nx};
    const long long rows = (long long)n * g.V;
    // the two operand stages; at least 228 KB * ncols / 512 so that the blocks
    // resident on an SM never ask for more than its 512 tensor-memory columns
    const int ncols = cout <= 32 ? 32 : (cout <= 64 ? 64 : (cout <= 128 ? 128 : 256));
    const size_t smem = std::max(2 * ((size_t)128 * cin * 2 + (size_t)cout * cin * 2),
                                 (size_t)228 * 1024 * ncols / 512 + 1024);
    const cudaStream_t s = (cudaStream_t)stream;
    const auto *xb = static_cast<const __nv_bfloat16 *>(x);
    const auto *wb = static_cast<const __nv_bfloat16 *>(w);
    unsigned *err = nullptr;
    cudaError_t e = cudaGetSymbolAddress(reinterpret_cast<void **>(&err), g_tc_err);
    if (e != cudaSuccess) return ucheck(e);
    const unsigned blocks = (unsigned)((rows + 127) / 128);
    if (out_f32) {
        e = cudaFuncSetAttribute(tc::k_conv_tc<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess) tc::k_conv_tc<true><<<blocks, 128, smem, s>>>(g, xb, cin, wb, b, cout, relu, y, err);
    } else {
        e = cudaFuncSetAttribute(tc::k_conv_tc<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess) tc::k_conv_tc<false><<<blocks, 128, smem, s>>>(g, xb, cin, wb, b, cout, relu, y, err);
    }
    if (e != cudaSuccess) return ucheck(e);
    return ucheck(cudaGetLastError());
}

cf_status cf_unet_tc_error(unsigned *err) {
    if (!err) return bad("null argument");
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpyFromSymbol(err, g_tc_err, sizeof(unsigned));
    const unsigned zero = 0;
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_tc_err, &zero, sizeof(unsigned));
    return ucheck(e);
}

cf_status cf_unet_flip(const void *w, int cin, int cout, void *wt, void *stream) {
    if (!w || !wt || cin < 1 || cout < 1) return bad("bad argument");
    const long long nW = 27LL * cin * cout;
    k_flip<<<nblk(nW), 256, 0, (cudaStream_t)stream>>>(static_cast<const __nv_bfloat16 *>(w), cin, cout,
                                                       static_cast<__nv_bfloat16 *>(wt));
    return ucheck(cudaGetLastError());
}

cf_status cf_unet_wgrad(const void *x, const void *gy, int n, int nz, int ny, int nx, int cin, int cout,
                        int chunks, float *part, float *gw, float *gb, void *stream) {
    if (!x || !gy || !part || !gw) return bad("null argument");
    if (!grid_ok(n, nz, ny, nx) || cin < 16 || cin % 16 || cout < 8 || cout % 8 || chunks < 1)
        return bad("cf_unet_wgrad: bad shape (cin a multiple of 16, cout of 8)");
    const Grid3 g{n, nz, ny, nx, (long long)nz * ny * nx};
    const long long total = (long long)n * g.V;
    long long chunk = (total + chunks - 1) / chunks;
    chunk = (chunk + 15) / 16 * 16;
    const int nch = (int)((total + chunk - 1) / chunk);
    const cudaStream_t s = (cudaStream_t)stream;
    const dim3 grid((unsigned)(((cin + 31) / 32 + CW - 1) / CW), (unsigned)(27 * ((cout + 15) / 16)), (unsigned)nch);
    k_wgrad_mma<<<grid, 32 * CW, 0, s>>>(g, static_cast<const __nv_bfloat16 *>(x), cin,
                                         static_cast<const __nv_bfloat16 *>(gy), cout, chunk, part);
    const long long nW = 27LL * cin * cout;
    k_wgrad_reduce<<<nblk(nW), 256, 0, s>>>(part, nch, nW, gw);
    if (gb) k_bias_grad<<<cout, 256, 0, s>>>(static_cast<const __nv_bfloat16 *>(gy), total, cout, gb);
    return ucheck(cudaGetLastError());
}

cf_status cf_unet_relu_grad(const float *g, const float *g2, const void *y, long long m, void *out, void *stream) {
    if (!g || !out || m < 0) return bad("bad argument");
    k_relu_grad<<<nblk(m), 256, 0, (cudaStream_t)stream>>>(g, g2, static_cast<const __nv_bfloat16 *>(y), m,
                                                          static_cast<__nv_bfloat16 *>(out));
    return ucheck(cudaGetLastError());
}

cf_status cf_unet_loss(const float *out, int n, int nz, int ny, int nx, int ch, const float *t, const float *mask,
                       double wd, const float *X, const float *d, int nodes, double wx, double *part,
                       float *g, double *loss, void *stream) {
    if (!out || !t || !mask || !part || !g || !loss || !grid_ok(n, nz, ny, nx) || ch < 5)
        return bad("cf_unet_loss: bad argument (head of at least 5 channels)");
    if (nodes > 0 && (!X || !d)) return bad("cf_unet_loss: node arrays missing");
    const cudaStream_t s = (cudaStream_t)stream;
    const long long V = (long long)nz * ny * nx;
    // msum: the mask sum, reduced on the host's request beforehand (scale
    // passed as wd / msum by the caller)
    k_loss_density<<<LOSS_BLOCKS, 256, 0, s>>>(n, V, ch, out, t, mask, wd, g, part);
    k_loss_sum<<<1, 1, 0, s>>>(part, LOSS_BLOCKS, loss);
    if (nodes > 0 && wx > 0.0) {
        k_loss_nodes<<<(n + 31) / 32, 32, 0, s>>>(n, nz, ny, nx, ch, out, X, d, nodes, wx / ((double)n * nodes),
                                                  g, part + LOSS_BLOCKS);
        k_loss_sum<<<1, 1, 0, s>>>(part + LOSS_BLOCKS, n, loss);
    }
    return ucheck(cudaGetLastError());
}

cf_status cf_unet_pool(const void *x, int n, int nz, int ny, int nx, int c, void *y, void *stream) {
    if (!x || !y || !grid_ok(n, nz, ny, nx) || c < 1 || nz % 2 || ny % 2 || nx % 2)
        return bad("cf_unet_pool: bad shape (even grid)");
    const Grid3 f{n, nz, ny, nx, (long long)nz * ny * nx};
    k_pool<<<nblk(f.n * f.V / 8 * c), 256, 0, (cudaStream_t)stream>>>(f, c, static_cast<const __nv_bfloat16 *>(x),
                                                                   static_cast<__nv_bfloat16 *>(y));
    return ucheck(cudaGetLastError());
}

cf_status cf_unet_pool_bwd(const float *gy, int n, int nz, int ny, int nx, int c, float *gx, void *stream) {
    if (!gy || !gx || !grid_ok(n, nz, ny, nx) || c < 1 || nz % 2 || ny % 2 || nx % 2)
        return bad("cf_unet_pool_bwd: bad shape (even grid)");
    const Grid3 f{n, nz, ny, nx, (long long)nz * ny * nx};
    k_pool_bwd<<<nblk(f.n * f.V * c), 256, 0, (cudaStream_t)stream>>>(f, c, gy, gx);
    return ucheck(cudaGetLastError());
}

cf_status cf_unet_upsample(const void *x, int n, int nz, int ny, int nx, int c, void *y, void *stream) {
    if (!x || !y || !grid_ok(n, nz, ny, nx) || c < 1 || nz % 2 || ny % 2 || nx % 2)
        return bad("cf_unet_upsample: bad shape (even fine grid)");
    const Grid3 f{n, nz, ny, nx, (long long)nz * ny * nx};
    k_upsample<<<nblk(f.n * f.V * c), 256, 0, (cudaStream_t)stream>>>(f, c, static_cast<const __nv_bfloat16 *>(x),
                                                                    static_cast<__nv_bfloat16 *>(y));
    return ucheck(cudaGetLastError());
}

cf_status cf_unet_upsample_bwd(const float *gy, int n, int nz, int ny, int nx, int c, float *gx, void *stream) {
    if (!gy || !gx || !grid_ok(n, nz, ny, nx) || c < 1 || nz % 2 || ny % 2 || nx % 2)
        return bad("cf_unet_upsample_bwd: bad shape (even fine grid)");
    const Grid3 f{n, nz, ny, nx, (long long)nz * ny * nx};
    k_upsample_bwd<<<nblk(f.n * f.V / 8 * c), 256, 0, (cudaStream_t)stream>>>(f, c, gy, gx);
    return ucheck(cudaGetLastError());
}

cf_status cf_unet_concat(long long nv, const void *a, int ca, const void *b, int cb, void *y, void *stream) {
    if (!a || !b || !y || nv < 0 || ca < 1 || cb < 1) return bad("bad argument");
    k_concat<<<nblk(nv * (ca + cb)), 256, 0, (cudaStream_t)stream>>>(
        nv, static_cast<const __nv_bfloat16 *>(a), ca, static_cast<const __nv_bfloat16 *>(b), cb,
        static_cast<__nv_bfloat16 *>(y));
    return ucheck(cudaGetLastError());
}

cf_status cf_unet_split(long long nv, const float *y, int ca, int cb, float *a, float *b, void *stream) {
    if (!y || nv < 0 || ca < 1 || cb < 1) return bad("bad argument");
    k_split<<<nblk(nv * (ca + cb)), 256, 0, (cudaStream_t)stream>>>(nv, y, ca, cb, a, b);
    return ucheck(cudaGetLastError());
}

cf_status cf_unet_pack(const float *x, int c, long long N, int cpad, void *y, void *stream) {
    if (!x || !y || N < 0 || c < 1 || cpad < c) return bad("bad argument");
    k_pack<<<nblk(N * cpad), 256, 0, (cudaStream_t)stream>>>(x, c, N, cpad, static_cast<__nv_bfloat16 *>(y));
    return ucheck(cudaGetLastError());
}

cf_status cf_unet_unpack(const void *x, int x_f32, int cpad, long long N, int c0, int c, float *y, void *stream) {
    if (!x || !y || N < 0 || c < 1 || c0 < 0 || c0 + c > cpad) return bad("bad argument");
    if (x_f32)
        k_unpack<float><<<nblk(N * c), 256, 0, (cudaStream_t)stream>>>(static_cast<const float *>(x), cpad, N, c0, c, y);
    else
        k_unpack<__nv_bfloat16><<<nblk(N * c), 256, 0, (cudaStream_t)stream>>>(
            static_cast<const __nv_bfloat16 *>(x), cpad, N, c0, c, y);
    return ucheck(cudaGetLastError());
}

}  // extern "C"
