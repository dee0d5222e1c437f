// Kernels of the learned warm start: a 3-D convolutional encoder-decoder on channels-last BF16
// tensors with FP32 accumulation.  The convolution the network runs is the tcgen05 kernel of
// nn_tc.cu; this file keeps the warp-level mma.sync (m16n8k16 BF16) formulation of the same
// convolution as the measured baseline (conv3d_mma) and the weight gradient.
//
// conv3d (3x3x3, zero padding one voxel) as an implicit GEMM: out[v][n] = b[n] +
//   sum_{tap, k} in[v + off(tap)][k] * B[tap][n][k].  Forward: B = W^T stored [27][Cout][Cin].
//   The data gradient is the same kernel on dY with B = W stored [27][Cin][Cout] and the taps
//   flipped.  Tiles of 64 voxels x 64 (or 32) outputs per 128-thread block, K staged 32 (or 16)
//   channels at a time through shared memory with cp.async (zero-fill outside the grid), A and B
//   fragments by ldmatrix.
// Weight gradient: dW[tap][i][o] = sum_v in[v + off(tap)][i] dY[v][o], a GEMM over voxels
//   (split over blocks, FP32 atomics), both operands read from voxel-major tiles by
//   ldmatrix.trans.
// Pooling, upsampling, concatenation, ReLU masks, the 1x1x1 head, the MSE loss, Adam and the
// input features are plain elementwise kernels.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "nn.h"

namespace hrt {
namespace nn {

typedef __nv_bfloat16 bf16;

// ---------------------------------------------------------------- PTX helpers
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, bool valid) {
    const int n = valid ? 16 : 0;   // 0 source bytes: the 16 shared bytes are zero-filled
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(smem_u32(smem)), "l"(gmem), "r"(n));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

__device__ __forceinline__ void ldsm_x4(uint32_t& r0, uint32_t& r1, uint32_t& r2, uint32_t& r3, const void* p) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(smem_u32(p)));
}
__device__ __forceinline__ void ldsm_x4_t(uint32_t& r0, uint32_t& r1, uint32_t& r2, uint32_t& r3, const void* p) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(smem_u32(p)));
}
__device__ __forceinline__ void mma16816(float* d, const uint32_t* a, uint32_t b0, uint32_t b1) {
    asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                 "{%0,%1,%2,%3};\n"
                 : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
                 : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ int tap_dz(int t) { return t / 9 - 1; }
__device__ __forceinline__ int tap_dy(int t) { return (t / 3) % 3 - 1; }
__device__ __forceinline__ int tap_dx(int t) { return t % 3 - 1; }

// ---------------------------------------------------------------- implicit-GEMM convolution
// KS = channels staged per step (16 or 32); BN = outputs per block (32 or 64).
template <int KS, int BN>
__global__ void __launch_bounds__(128) k_conv3d(const bf16* __restrict__ in, const bf16* __restrict__ B,
                                                const float* __restrict__ bias, bf16* __restrict__ out, int D, int H,
                                                int W, int Cin, int Cout, int flip, int relu) {
    constexpr int BM = 64;
    constexpr int LDA = KS + 8;   // padded rows: conflict-free ldmatrix
    __shared__ __align__(16) bf16 As[2][BM * LDA];
    __shared__ __align__(16) bf16 Bs[2][BN * LDA];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wm = warp & 1, wn = warp >> 1;          // 2 x 2 warps
    constexpr int WN = BN / 2;                        // outputs per warp
    constexpr int NT = WN / 8;                        // n8 tiles per warp
    const long long V = (long long)D * H * W;
    const long long v0 = (long long)blockIdx.x * BM;
    const int n0 = blockIdx.y * BN;
    const int nb = blockIdx.z;                        // sample in the batch
    const bf16* inb = in + (long long)nb * V * Cin;
    bf16* outb = out + (long long)nb * V * Cout;

    float acc[2][NT][4];
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < NT; ++b)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[a][b][c] = 0.f;

    const int kchunks = Cin / KS;
    const int nsteps = 27 * kchunks;
    constexpr int CPR = KS / 8;                       // 16-byte chunks per row

    auto load_stage = [&](int step, int buf) {
        const int tap = step / kchunks;
        const int k0 = (step % kchunks) * KS;
        const int btap = flip ? 26 - tap : tap;
        const int dz = tap_dz(tap), dy = tap_dy(tap), dx = tap_dx(tap);
        for (int c = tid; c < BM * CPR; c += 128) {
            const int m = c / CPR, part = c % CPR;
            const long long v = v0 + m;
            bool ok = v < V;
            long long src = 0;
            if (ok) {
                const int x = (int)(v % W), y = (int)((v / W) % H), z = (int)(v / ((long long)W * H));
                const int zz = z + dz, yy = y + dy, xx = x + dx;
                ok = zz >= 0 && zz < D && yy >= 0 && yy < H && xx >= 0 && xx < W;
                src = (((long long)zz * H + yy) * W + xx) * Cin + k0 + part * 8;
            }
            cp_async16(&As[buf][m * LDA + part * 8], ok ? (const void*)(inb + src) : (const void*)inb, ok);
        }
        for (int c = tid; c < BN * CPR; c += 128) {
            const int n = c / CPR, part = c % CPR;
            const bool ok = n0 + n < Cout;
            const long long src = ((long long)btap * Cout + n0 + n) * Cin + k0 + part * 8;
            cp_async16(&Bs[buf][n * LDA + part * 8], ok ? (const void*)(B + src) : (const void*)B, ok);
        }
        cp_async_commit();
    };

    load_stage(0, 0);
    for (int step = 0; step < nsteps; ++step) {
        const int buf = step & 1;
        if (step + 1 < nsteps) {
            load_stage(step + 1, buf ^ 1);
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < KS; kk += 16) {
            uint32_t af[2][4];
#pragma unroll
            for (int mt = 0; mt < 2; ++mt) {
                const int q = lane >> 3, r = lane & 7;
                const int row = wm * 32 + mt * 16 + r + (q & 1) * 8;
                const int col = kk + (q >> 1) * 8;
                ldsm_x4(af[mt][0], af[mt][1], af[mt][2], af[mt][3], &As[buf][row * LDA + col]);
            }
#pragma unroll
            for (int nt = 0; nt < NT; nt += 2) {
                const int q = lane >> 3, r = lane & 7;
                const int row = wn * WN + nt * 8 + r + (q >> 1) * 8;
                const int col = kk + (q & 1) * 8;
                uint32_t b0, b1, b2, b3;
                ldsm_x4(b0, b1, b2, b3, &Bs[buf][row * LDA + col]);
#pragma unroll
                for (int mt = 0; mt < 2; ++mt) {
                    mma16816(acc[mt][nt], af[mt], b0, b1);
                    mma16816(acc[mt][nt + 1], af[mt], b2, b3);
                }
            }
        }
        __syncthreads();
    }
    // epilogue: bias, ReLU, BF16 store
#pragma unroll
    for (int mt = 0; mt < 2; ++mt) {
#pragma unroll
        for (int half = 0; half < 2; ++half) {
            const long long v = v0 + wm * 32 + mt * 16 + (lane >> 2) + half * 8;
            if (v >= V) continue;
#pragma unroll
            for (int nt = 0; nt < NT; ++nt) {
                const int n = n0 + wn * WN + nt * 8 + (lane & 3) * 2;
                if (n >= Cout) continue;
                float a0 = acc[mt][nt][half * 2] + (bias ? bias[n] : 0.f);
                float a1 = acc[mt][nt][half * 2 + 1] + (bias ? bias[n + 1] : 0.f);
                if (relu) {
                    a0 = fmaxf(a0, 0.f);
                    a1 = fmaxf(a1, 0.f);
                }
                *reinterpret_cast<__nv_bfloat162*>(outb + v * Cout + n) = __floats2bfloat162_rn(a0, a1);
            }
        }
    }
}

cudaError_t conv3d_mma(const bf16* in, const bf16* Bw, const float* bias, bf16* out, int N, int D, int H, int W, int Cin,
                       int Cout, bool flip, bool relu, cudaStream_t s) {
    if (Cin % 16 != 0 || Cout % 32 != 0) return cudaErrorInvalidValue;
    const long long V = (long long)D * H * W;
    const dim3 grid((unsigned)((V + 63) / 64), (unsigned)((Cout + 63) / 64), (unsigned)N);
    if (Cout % 64 == 0) {
        if (Cin % 32 == 0) k_conv3d<32, 64><<<grid, 128, 0, s>>>(in, Bw, bias, out, D, H, W, Cin, Cout, flip, relu);
        else k_conv3d<16, 64><<<grid, 128, 0, s>>>(in, Bw, bias, out, D, H, W, Cin, Cout, flip, relu);
    } else {
        const dim3 g2((unsigned)((V + 63) / 64), (unsigned)(Cout / 32), (unsigned)N);
        if (Cin % 32 == 0) k_conv3d<32, 32><<<g2, 128, 0, s>>>(in, Bw, bias, out, D, H, W, Cin, Cout, flip, relu);
        else k_conv3d<16, 32><<<g2, 128, 0, s>>>(in, Bw, bias, out, D, H, W, Cin, Cout, flip, relu);
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------- weight gradient
// dW[tap][i][o] += sum_{v in this block's voxels} in[v + off(tap)][i] * dy[v][o].
// Block: 64 input channels (M) x 64 output channels (N), 32 voxels per K step.
__global__ void __launch_bounds__(128) k_conv3d_wgrad(const bf16* __restrict__ in, const bf16* __restrict__ dy,
                                                      float* __restrict__ dw, int D, int H, int W, int Cin, int Cout,
                                                      int nsplit, int nbatch) {
    constexpr int BKV = 32;          // voxels per step
    constexpr int BM = 64, BN = 64;
    constexpr int LDA = BM + 8, LDB = BN + 8;
    __shared__ __align__(16) bf16 As[2][BKV * LDA];   // [voxel][i]
    __shared__ __align__(16) bf16 Bs[2][BKV * LDB];   // [voxel][o]
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wm = warp & 1, wn = warp >> 1;
    const int tap = blockIdx.x;
    const int mblocks = (Cin + BM - 1) / BM;
    const int i0 = (blockIdx.y % mblocks) * BM;
    const int o0 = (blockIdx.y / mblocks) * BN;
    const int split = blockIdx.z;
    const int dz = tap_dz(tap), dyy = tap_dy(tap), dx = tap_dx(tap);
    const long long V = (long long)D * H * W;
    const long long total = V * nbatch;
    const long long per = ((total + nsplit - 1) / nsplit + BKV - 1) / BKV * BKV;
    const long long vbeg = (long long)split * per;
    const long long vend = vbeg + per < total ? vbeg + per : total;
    float acc[2][4][4];
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[a][b][c] = 0.f;
    if (vbeg >= vend) return;
    const int nsteps = (int)((vend - vbeg + BKV - 1) / BKV);

    auto load_stage = [&](int step, int buf) {
        const long long vb = vbeg + (long long)step * BKV;
        for (int c = tid; c < BKV * (BM / 8); c += 128) {
            const int k = c / (BM / 8), part = c % (BM / 8);
            const long long g = vb + k;
            bool ok = g < vend && i0 + part * 8 < Cin;
            long long src = 0;
            if (ok) {
                const long long nb = g / V, v = g % V;
                const int x = (int)(v % W), y = (int)((v / W) % H), z = (int)(v / ((long long)W * H));
                const int zz = z + dz, yy = y + dyy, xx = x + dx;
                ok = zz >= 0 && zz < D && yy >= 0 && yy < H && xx >= 0 && xx < W;
                src = ((nb * D + zz) * H + yy) * (long long)W * Cin + (long long)xx * Cin + i0 + part * 8;
            }
            cp_async16(&As[buf][k * LDA + part * 8], ok ? (const void*)(in + src) : (const void*)in, ok);
        }
        for (int c = tid; c < BKV * (BN / 8); c += 128) {
            const int k = c / (BN / 8), part = c % (BN / 8);
            const long long g = vb + k;
            const bool ok = g < vend && o0 + part * 8 < Cout;
            const long long src = g * Cout + o0 + part * 8;
            cp_async16(&Bs[buf][k * LDB + part * 8], ok ? (const void*)(dy + src) : (const void*)dy, ok);
        }
        cp_async_commit();
    };

    load_stage(0, 0);
    for (int step = 0; step < nsteps; ++step) {
        const int buf = step & 1;
        if (step + 1 < nsteps) {
            load_stage(step + 1, buf ^ 1);
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BKV; kk += 16) {
            uint32_t af[2][4];
#pragma unroll
            for (int mt = 0; mt < 2; ++mt) {
                const int q = lane >> 3, r = lane & 7;
                const int krow = kk + r + (q >> 1) * 8;
                const int col = wm * 32 + mt * 16 + (q & 1) * 8;
                ldsm_x4_t(af[mt][0], af[mt][1], af[mt][2], af[mt][3], &As[buf][krow * LDA + col]);
            }
#pragma unroll
            for (int nt = 0; nt < 4; nt += 2) {
                const int q = lane >> 3, r = lane & 7;
                const int krow = kk + r + (q & 1) * 8;
                const int col = wn * 32 + nt * 8 + (q >> 1) * 8;
                uint32_t b0, b1, b2, b3;
                ldsm_x4_t(b0, b1, b2, b3, &Bs[buf][krow * LDB + col]);
#pragma unroll
                for (int mt = 0; mt < 2; ++mt) {
                    mma16816(acc[mt][nt], af[mt], b0, b1);
                    mma16816(acc[mt][nt + 1], af[mt], b2, b3);
                }
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int half = 0; half < 2; ++half) {
            const int i = i0 + wm * 32 + mt * 16 + (lane >> 2) + half * 8;
            if (i >= Cin) continue;
#pragma unroll
            for (int nt = 0; nt < 4; ++nt) {
                const int o = o0 + wn * 32 + nt * 8 + (lane & 3) * 2;
                if (o >= Cout) continue;
                float* dst = dw + ((long long)tap * Cin + i) * Cout + o;
                atomicAdd(dst, acc[mt][nt][half * 2]);
                atomicAdd(dst + 1, acc[mt][nt][half * 2 + 1]);
            }
        }
}

cudaError_t conv3d_wgrad_mma(const bf16* in, const bf16* dy, float* dw, int N, int D, int H, int W, int Cin, int Cout,
                             cudaStream_t s) {
    if (Cin % 8 != 0 || Cout % 8 != 0) return cudaErrorInvalidValue;
    const long long total = (long long)D * H * W * N;
    int nsplit = (int)(total / 4096);
    nsplit = nsplit < 1 ? 1 : (nsplit > 64 ? 64 : nsplit);
    const int mblocks = (Cin + 63) / 64, nblocks = (Cout + 63) / 64;
    const dim3 grid(27, (unsigned)(mblocks * nblocks), (unsigned)nsplit);
    k_conv3d_wgrad<<<grid, 128, 0, s>>>(in, dy, dw, D, H, W, Cin, Cout, nsplit, N);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- elementwise kernels
#define GRID_STRIDE(i, n) for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < (n); i += (long long)gridDim.x * blockDim.x)

static unsigned blocks_for(long long n) {
    const long long b = (n + 255) / 256;
    return (unsigned)(b < 1 ? 1 : (b > 65535 * 8 ? 65535 * 8 : b));
}

__global__ void k_bias_grad(const bf16* __restrict__ dy, float* __restrict__ db, long long V, int C) {
    // one block per channel group of 32 channels; threads stride over voxels
    __shared__ float part[8][32];
    const int c = blockIdx.y * 32 + (threadIdx.x & 31);
    float s = 0.f;
    if (c < C)
        for (long long v = (long long)blockIdx.x * 8 + (threadIdx.x >> 5); v < V; v += (long long)gridDim.x * 8)
            s += __bfloat162float(dy[v * C + c]);
    part[threadIdx.x >> 5][threadIdx.x & 31] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        float t = 0.f;
        for (int w = 0; w < 8; ++w) t += part[w][threadIdx.x];
        if (c < C) atomicAdd(db + c, t);
    }
}

cudaError_t bias_grad(const bf16* dy, float* db, long long V, int C, cudaStream_t s) {
    const dim3 grid(256, (unsigned)((C + 31) / 32));
    k_bias_grad<<<grid, 256, 0, s>>>(dy, db, V, C);
    return cudaGetLastError();
}

// Channels-last tensors with C % 8 == 0: each thread moves 8 channels (16 bytes) of one voxel.
__device__ __forceinline__ void unpack8(const uint4& u, float* f) {
    const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&u);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const float2 t = __bfloat1622float2(h[i]);
        f[2 * i] = t.x;
        f[2 * i + 1] = t.y;
    }
}
__device__ __forceinline__ uint4 pack8(const float* f) {
    uint4 u;
    __nv_bfloat162* h = reinterpret_cast<__nv_bfloat162*>(&u);
#pragma unroll
    for (int i = 0; i < 4; ++i) h[i] = __floats2bfloat162_rn(f[2 * i], f[2 * i + 1]);
    return u;
}
__device__ __forceinline__ uint4 ld8(const bf16* p) { return *reinterpret_cast<const uint4*>(p); }
__device__ __forceinline__ void st8(bf16* p, const uint4& u) { *reinterpret_cast<uint4*>(p) = u; }

__global__ void k_relu_mask(bf16* __restrict__ g, const bf16* __restrict__ h, long long n8) {
    GRID_STRIDE(i, n8) {
        float gv[8], hv[8];
        unpack8(ld8(g + 8 * i), gv);
        unpack8(ld8(h + 8 * i), hv);
#pragma unroll
        for (int k = 0; k < 8; ++k)
            if (!(hv[k] > 0.f)) gv[k] = 0.f;
        st8(g + 8 * i, pack8(gv));
    }
}

cudaError_t relu_mask(bf16* g, const bf16* h, long long n, cudaStream_t s) {
    if (n % 8) return cudaErrorInvalidValue;
    k_relu_mask<<<blocks_for(n / 8), 256, 0, s>>>(g, h, n / 8);
    return cudaGetLastError();
}

// 2x2x2 average pooling: one thread per (output voxel, 8 channels)
__global__ void k_pool2(const bf16* __restrict__ x, bf16* __restrict__ y, int N, int D, int H, int W, int C) {
    const int d = D / 2, h = H / 2, w = W / 2, C8 = C / 8;
    const long long n = (long long)N * d * h * w * C8;
    GRID_STRIDE(i, n) {
        const int c = (int)(i % C8) * 8;
        long long r = i / C8;
        const int xx = (int)(r % w); r /= w;
        const int yy = (int)(r % h); r /= h;
        const int zz = (int)(r % d);
        const long long nb = r / d;
        float s8[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b)
                for (int e = 0; e < 2; ++e) {
                    float v[8];
                    unpack8(ld8(x + (((nb * D + 2 * zz + a) * H + 2 * yy + b) * W + 2 * xx + e) * C + c), v);
#pragma unroll
                    for (int k = 0; k < 8; ++k) s8[k] += v[k];
                }
#pragma unroll
        for (int k = 0; k < 8; ++k) s8[k] *= 0.125f;
        st8(y + i * 8, pack8(s8));
    }
}

__global__ void k_pool2_back(const bf16* __restrict__ dy, bf16* __restrict__ dx, int N, int D, int H, int W, int C,
                             int accumulate) {
    const int C8 = C / 8;
    const long long n = (long long)N * D * H * W * C8;
    GRID_STRIDE(i, n) {
        const int c = (int)(i % C8) * 8;
        long long r = i / C8;
        const int xx = (int)(r % W); r /= W;
        const int yy = (int)(r % H); r /= H;
        const int zz = (int)(r % D);
        const long long nb = r / D;
        float g[8];
        unpack8(ld8(dy + (((nb * (D / 2) + zz / 2) * (H / 2) + yy / 2) * (W / 2) + xx / 2) * C + c), g);
        if (accumulate) {
            float o[8];
            unpack8(ld8(dx + i * 8), o);
#pragma unroll
            for (int k = 0; k < 8; ++k) g[k] = 0.125f * g[k] + o[k];
        } else {
#pragma unroll
            for (int k = 0; k < 8; ++k) g[k] *= 0.125f;
        }
        st8(dx + i * 8, pack8(g));
    }
}

// nearest 2x upsampling of x [N][D/2][H/2][W/2][C1] into channels [0, C1) of y [N][D][H][W][Ctot]
__global__ void k_up2_into(const bf16* __restrict__ x, bf16* __restrict__ y, int N, int D, int H, int W, int C1,
                           int Ctot) {
    const int C8 = C1 / 8;
    const long long n = (long long)N * D * H * W * C8;
    GRID_STRIDE(i, n) {
        const int c = (int)(i % C8) * 8;
        long long r = i / C8;
        const int xx = (int)(r % W); r /= W;
        const int yy = (int)(r % H); r /= H;
        const int zz = (int)(r % D);
        const long long nb = r / D;
        st8(y + (((nb * D + zz) * H + yy) * W + xx) * Ctot + c,
            ld8(x + (((nb * (D / 2) + zz / 2) * (H / 2) + yy / 2) * (W / 2) + xx / 2) * C1 + c));
    }
}

// copy s [N*V][C2] into channels [off, off + C2) of y [N*V][Ctot]
__global__ void k_copy_into(const bf16* __restrict__ s, bf16* __restrict__ y, long long NV, int C2, int off, int Ctot) {
    const int C8 = C2 / 8;
    GRID_STRIDE(i, NV * C8) {
        const long long v = i / C8;
        const int c = (int)(i % C8) * 8;
        st8(y + v * Ctot + off + c, ld8(s + i * 8));
    }
}

// gradient of the concat: channels [0, C1) summed over each 2x2x2 block into dx (upsampling
// gradient), channels [C1, Ctot) added into dskip
__global__ void k_concat_back(const bf16* __restrict__ g, bf16* __restrict__ dx, bf16* __restrict__ dskip, int N, int D,
                              int H, int W, int C1, int Ctot) {
    const int d = D / 2, h = H / 2, w = W / 2, C18 = C1 / 8;
    const long long n1 = (long long)N * d * h * w * C18;
    GRID_STRIDE(i, n1) {
        const int c = (int)(i % C18) * 8;
        long long r = i / C18;
        const int xx = (int)(r % w); r /= w;
        const int yy = (int)(r % h); r /= h;
        const int zz = (int)(r % d);
        const long long nb = r / d;
        float s8[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b)
                for (int e = 0; e < 2; ++e) {
                    float v[8];
                    unpack8(ld8(g + (((nb * D + 2 * zz + a) * H + 2 * yy + b) * W + 2 * xx + e) * Ctot + c), v);
#pragma unroll
                    for (int k = 0; k < 8; ++k) s8[k] += v[k];
                }
        st8(dx + i * 8, pack8(s8));
    }
    const int C28 = (Ctot - C1) / 8;
    const long long n2 = (long long)N * D * H * W * C28;
    GRID_STRIDE(j, n2) {
        const long long v = j / C28;
        const int c = (int)(j % C28) * 8;
        float a8[8], b8[8];
        unpack8(ld8(dskip + j * 8), a8);
        unpack8(ld8(g + v * Ctot + C1 + c), b8);
#pragma unroll
        for (int k = 0; k < 8; ++k) a8[k] += b8[k];
        st8(dskip + j * 8, pack8(a8));
    }
}

cudaError_t pool2(const bf16* x, bf16* y, int N, int D, int H, int W, int C, cudaStream_t s) {
    if (C % 8) return cudaErrorInvalidValue;
    k_pool2<<<blocks_for((long long)N * D * H * W * C / 64), 256, 0, s>>>(x, y, N, D, H, W, C);
    return cudaGetLastError();
}
cudaError_t pool2_back(const bf16* dy, bf16* dx, int N, int D, int H, int W, int C, bool accumulate, cudaStream_t s) {
    if (C % 8) return cudaErrorInvalidValue;
    k_pool2_back<<<blocks_for((long long)N * D * H * W * C / 8), 256, 0, s>>>(dy, dx, N, D, H, W, C, accumulate);
    return cudaGetLastError();
}
cudaError_t concat_up(const bf16* low, const bf16* skip, bf16* y, int N, int D, int H, int W, int C1, int C2,
                      cudaStream_t s) {
    if (C1 % 8 || C2 % 8) return cudaErrorInvalidValue;
    k_up2_into<<<blocks_for((long long)N * D * H * W * C1 / 8), 256, 0, s>>>(low, y, N, D, H, W, C1, C1 + C2);
    k_copy_into<<<blocks_for((long long)N * D * H * W * C2 / 8), 256, 0, s>>>(skip, y, (long long)N * D * H * W, C2,
                                                                            C1, C1 + C2);
    return cudaGetLastError();
}
cudaError_t concat_up_back(const bf16* g, bf16* dlow, bf16* dskip, int N, int D, int H, int W, int C1, int C2,
                           cudaStream_t s) {
    if (C1 % 8 || C2 % 8) return cudaErrorInvalidValue;
    k_concat_back<<<blocks_for((long long)N * D * H * W * (C1 + C2) / 8), 256, 0, s>>>(g, dlow, dskip, N, D, H, W, C1,
                                                                                      C1 + C2);
    return cudaGetLastError();
}

// 1x1x1 head: y[v] = b + sum_c h[v][c] w[c] (FP32 out); loss 0.5 mean((y - t)^2) and dy
__global__ void k_head(const bf16* __restrict__ h, const float* __restrict__ w, const float* __restrict__ b,
                       float* __restrict__ y, long long NV, int C) {
    GRID_STRIDE(v, NV) {
        float s = b[0];
        for (int c = 0; c < C; c += 8) {
            float hv[8];
            unpack8(ld8(h + v * C + c), hv);
#pragma unroll
            for (int k = 0; k < 8; ++k) s += hv[k] * w[c + k];
        }
        y[v] = s;
    }
}

__global__ void k_loss(const float* __restrict__ y, const float* __restrict__ t, float* __restrict__ dy,
                       double* __restrict__ loss, long long NV) {
    double part = 0.0;
    GRID_STRIDE(v, NV) {
        const float e = y[v] - t[v];
        dy[v] = e / (float)NV;
        part += 0.5 * (double)e * (double)e;
    }
    for (int o = 16; o > 0; o >>= 1) part += __shfl_down_sync(0xffffffffu, part, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(loss, part / (double)NV);
}

// head backward: dh[v][c] = dy[v] w[c]; dw[c] += sum_v h[v][c] dy[v]; db += sum_v dy[v].  A thread
// keeps one group of 8 channels and strides over voxels, summing its share of dw (and db) in
// registers; the block adds the threads' sums in shared memory, then one atomic per channel.
__global__ void k_head_back(const bf16* __restrict__ h, const float* __restrict__ w, const float* __restrict__ dy,
                            bf16* __restrict__ dh, float* __restrict__ dw, float* __restrict__ db, long long NV, int C) {
    extern __shared__ float sacc[];   // [C + 1]
    for (int c = threadIdx.x; c <= C; c += blockDim.x) sacc[c] = 0.f;
    __syncthreads();
    const int C8 = C / 8, per = (int)blockDim.x / C8;        // voxels a block takes per round
    const int cg = (int)threadIdx.x % C8, row = (int)threadIdx.x / C8;
    if (row < per) {
        float wv[8], acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f}, accb = 0.f;
#pragma unroll
        for (int k = 0; k < 8; ++k) wv[k] = w[cg * 8 + k];
        for (long long v = (long long)blockIdx.x * per + row; v < NV; v += (long long)gridDim.x * per) {
            const float g = dy[v];
            float hv[8], o[8];
            unpack8(ld8(h + v * C + cg * 8), hv);
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                o[k] = g * wv[k];
                acc[k] += hv[k] * g;
            }
            st8(dh + v * C + cg * 8, pack8(o));
            accb += g;
        }
#pragma unroll
        for (int k = 0; k < 8; ++k) atomicAdd(&sacc[cg * 8 + k], acc[k]);
        if (cg == 0) atomicAdd(&sacc[C], accb);
    }
    __syncthreads();
    for (int c = threadIdx.x; c < C; c += blockDim.x) atomicAdd(dw + c, sacc[c]);
    if (threadIdx.x == 0) atomicAdd(db, sacc[C]);
}

cudaError_t head_forward(const bf16* h, const float* w, const float* b, float* y, long long NV, int C, cudaStream_t s) {
    if (C % 8) return cudaErrorInvalidValue;
    k_head<<<blocks_for(NV), 256, 0, s>>>(h, w, b, y, NV, C);
    return cudaGetLastError();
}
cudaError_t mse_loss(const float* y, const float* t, float* dy, double* loss, long long NV, cudaStream_t s) {
    k_loss<<<blocks_for(NV), 256, 0, s>>>(y, t, dy, loss, NV);
    return cudaGetLastError();
}
cudaError_t head_backward(const bf16* h, const float* w, const float* dy, bf16* dh, float* dw, float* db, long long NV,
                          int C, cudaStream_t s) {
    if (C % 8 || C / 8 > 256) return cudaErrorInvalidValue;
    unsigned g = blocks_for(NV * (C / 8));
    if (g > 1024) g = 1024;
    k_head_back<<<g, 256, sizeof(float) * (C + 1), s>>>(h, w, dy, dh, dw, db, NV, C);
    return cudaGetLastError();
}

// Adam (Kingma & Ba 2015) on FP32 master weights, then the two BF16 copies of every conv
// weight: W [27][Cin][Cout] (data gradient) and W^T [27][Cout][Cin] (forward).
__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m, float* __restrict__ v,
                       long long n, float lr, float b1, float b2, float eps, float c1, float c2) {
    GRID_STRIDE(i, n) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

cudaError_t adam(float* p, const float* g, float* m, float* v, long long n, float lr, int step, cudaStream_t s) {
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
    k_adam<<<blocks_for(n), 256, 0, s>>>(p, g, m, v, n, lr, b1, b2, 1e-8f, c1, c2);
    return cudaGetLastError();
}

__global__ void k_weights_bf16(const float* __restrict__ w, bf16* __restrict__ wb, bf16* __restrict__ wt, int cin_real,
                               int Cin, int Cout) {
    const long long n = 27LL * Cin * Cout;
    GRID_STRIDE(i, n) {
        const int o = (int)(i % Cout);
        const long long r = i / Cout;
        const int ci = (int)(r % Cin);
        const int tap = (int)(r / Cin);
        const float val = ci < cin_real ? w[((long long)tap * cin_real + ci) * Cout + o] : 0.f;
        wb[i] = __float2bfloat16(val);
        wt[((long long)tap * Cout + o) * Cin + ci] = __float2bfloat16(val);
    }
}

cudaError_t weights_bf16(const float* w, bf16* wb, bf16* wt, int cin_real, int Cin, int Cout, cudaStream_t s) {
    k_weights_bf16<<<blocks_for(27LL * Cin * Cout), 256, 0, s>>>(w, wb, wt, cin_real, Cin, Cout);
    return cudaGetLastError();
}

// Bp [Cin/8][Cout/BN][27][BN][8] from B [27][Cout][Cin]
__global__ void k_pack_tma_weights(const bf16* __restrict__ B, bf16* __restrict__ Bp, int Cin, int Cout, int BN) {
    GRID_STRIDE(i, 27LL * Cin * Cout) {
        long long r = i;
        const int c = (int)(r % 8);
        r /= 8;
        const int n = (int)(r % BN);
        r /= BN;
        const int tap = (int)(r % 27);
        r /= 27;
        const int nt = (int)(r % (Cout / BN));
        const int c8 = (int)(r / (Cout / BN));
        Bp[i] = B[((long long)tap * Cout + nt * BN + n) * Cin + c8 * 8 + c];
    }
}

cudaError_t pack_tma_weights(const bf16* B, bf16* Bp, int Cin, int Cout, cudaStream_t s) {
    if (Cin <= 0 || Cout <= 0 || Cin % 8 != 0 || Cout % 32 != 0) return cudaErrorInvalidValue;
    k_pack_tma_weights<<<blocks_for(27LL * Cin * Cout), 256, 0, s>>>(B, Bp, Cin, Cout, tma_tile_n(Cout));
    return cudaGetLastError();
}

// uniform(-bound, bound) initial weights from Philox-free integer hashing (splitmix64)
__device__ __forceinline__ unsigned long long splitmix64(unsigned long long x) {
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}

__global__ void k_init_uniform(float* p, long long n, float bound, unsigned long long seed) {
    GRID_STRIDE(i, n) {
        const unsigned long long r = splitmix64(seed ^ (unsigned long long)i * 0x100000001B3ull);
        const float u = (float)(r >> 40) * (1.f / 16777216.f);
        p[i] = (2.f * u - 1.f) * bound;
    }
}

cudaError_t init_uniform(float* p, long long n, float bound, unsigned long long seed, cudaStream_t s) {
    k_init_uniform<<<blocks_for(n), 256, 0, s>>>(p, n, bound, seed);
    return cudaGetLastError();
}

// float [NV][cin] -> BF16 [NV][Cpad] (zero channels beyond cin)
__global__ void k_pack_input(const float* __restrict__ x, bf16* __restrict__ y, long long NV, int cin, int Cpad) {
    GRID_STRIDE(i, NV * Cpad) {
        const long long v = i / Cpad;
        const int c = (int)(i % Cpad);
        y[i] = __float2bfloat16(c < cin ? x[v * cin + c] : 0.f);
    }
}

cudaError_t pack_input(const float* x, bf16* y, long long NV, int cin, int Cpad, cudaStream_t s) {
    k_pack_input<<<blocks_for(NV * Cpad), 256, 0, s>>>(x, y, NV, cin, Cpad);
    return cudaGetLastError();
}

__global__ void k_bf16_to_f32(const bf16* __restrict__ x, float* __restrict__ y, long long n) {
    GRID_STRIDE(i, n) y[i] = __bfloat162float(x[i]);
}
__global__ void k_f32_to_bf16(const float* __restrict__ x, bf16* __restrict__ y, long long n) {
    GRID_STRIDE(i, n) y[i] = __float2bfloat16(x[i]);
}
cudaError_t bf16_to_f32(const bf16* x, float* y, long long n, cudaStream_t s) {
    k_bf16_to_f32<<<blocks_for(n), 256, 0, s>>>(x, y, n);
    return cudaGetLastError();
}
cudaError_t f32_to_bf16(const float* x, bf16* y, long long n, cudaStream_t s) {
    k_f32_to_bf16<<<blocks_for(n), 256, 0, s>>>(x, y, n);
    return cudaGetLastError();
}

}  // namespace nn
}  // namespace hrt
