// 3x3x3 'same' convolution of the learned warm start on the 5th-generation tensor cores: an
// implicit GEMM out[v][n] = act(b[n] + sum_{tap, k} in[v + off(tap)][k] * B[tap][n][k]) with the
// FP32 accumulator in tensor memory.
//
// Per block (128 threads): a tile of 128 voxels (the MMA's M) x BN outputs (its N).  The K loop
// runs over (tap, KC-channel chunk) stages: every thread gathers its voxel's KC channels at the
// tap offset (zero outside the grid) and a share of the B rows into shared memory with
// cp.async, in the no-swizzle K-major core-matrix layout (8 rows x 16 bytes per core matrix,
// 128 bytes apart along K, KC * 16 bytes apart per 8 rows); one thread issues KC / 16
// tcgen05.mma (M = 128, N = BN, K = 16, BF16 in, FP32 accumulate) and commits them to the
// stage's mbarrier.  Two stage buffers: the gather of stage s + 1 overlaps the MMAs of stage s,
// and a buffer is refilled only after the mbarrier shows its MMAs complete.  The epilogue reads
// each voxel's row of the accumulator (tensor-memory lane = voxel) with tcgen05.ld, adds the
// bias, applies ReLU and stores BF16.  Every wait is bounded (2 s): past it the block records
// an error, frees its tensor memory and returns.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "nn.h"
#include "tcgen05.cuh"

namespace hrt {
namespace nn {

typedef __nv_bfloat16 bf16;

__device__ int g_tc_error = 0;          // set by a block whose wait gave up

namespace {

constexpr uint64_t WAIT_LIMIT_NS = 2000000000ull;

__device__ __forceinline__ void cp_async16_zfill(uint32_t smem, const void* gmem, bool valid) {
    const int n = valid ? 16 : 0;       // 0 source bytes: the 16 shared bytes are zero-filled
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(smem), "l"(gmem), "r"(n) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// byte offset of (row, 16-byte chunk along K) in a KC-wide no-swizzle K-major tile
template <int KC>
__device__ __forceinline__ uint32_t core_off(int row, int chunk) {
    return (uint32_t)((row >> 3) * (KC * 16) + chunk * 128 + (row & 7) * 16);
}

}  // namespace

template <int KC, int BN>
__global__ void __launch_bounds__(128) k_conv3d_tc(const bf16* __restrict__ in, const bf16* __restrict__ B,
                                                   const float* __restrict__ bias, bf16* __restrict__ out, int D, int H,
                                                   int W, int Cin, int Cout, int flip, int relu) {
    constexpr int BM = 128;
    constexpr int A_BYTES = BM * KC * 2, B_BYTES = BN * KC * 2;
    constexpr uint32_t NCOLS = BN < 32 ? 32 : BN;
    constexpr int CH = KC / 8;                      // 16-byte chunks per row and stage
    extern __shared__ __align__(1024) unsigned char smem[];
    const uint32_t sA = tc::smem_addr(smem);
    const uint32_t sB = sA + 2 * A_BYTES;
    const uint32_t bar0 = sB + 2 * B_BYTES;         // two 8-byte mbarriers
    const uint32_t slot = bar0 + 16;                // tensor-memory address written by the allocation
    const int tid = threadIdx.x, warp = tid >> 5;
    const long long V = (long long)D * H * W;
    const long long v0 = (long long)blockIdx.x * BM;
    const int n0 = blockIdx.y * BN;
    const bf16* inb = in + (long long)blockIdx.z * V * Cin;
    bf16* outb = out + (long long)blockIdx.z * V * Cout;

    if (warp == 0) {
        tc::tmem_alloc(slot, NCOLS);
        tc::tmem_relinquish();
    }
    if (tid == 0) {
        tc::mbar_init(bar0, 1);
        tc::mbar_init(bar0 + 8, 1);
        tc::fence_mbar_init();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    uint32_t tmem;
    asm volatile("ld.shared.u32 %0, [%1];" : "=r"(tmem) : "r"(slot) : "memory");

    // this thread's voxel (row tid of the tile) and its grid position
    const long long v = v0 + tid;
    const bool vin = v < V;
    int x = 0, y = 0, z = 0;
    if (vin) {
        x = (int)(v % W);
        y = (int)((v / W) % H);
        z = (int)(v / ((long long)W * H));
    }
    const int kchunks = Cin / KC;
    const int S = 27 * kchunks;

    auto load = [&](int s, int buf) {
        const int tap = s / kchunks, k0 = (s % kchunks) * KC;
        const int btap = flip ? 26 - tap : tap;
        const int zz = z + tap / 9 - 1, yy = y + (tap / 3) % 3 - 1, xx = x + tap % 3 - 1;
        const bool ok = vin && zz >= 0 && zz < D && yy >= 0 && yy < H && xx >= 0 && xx < W;
        const bf16* src = ok ? inb + (((long long)zz * H + yy) * W + xx) * Cin + k0 : inb;
        const uint32_t a = sA + buf * A_BYTES;
#pragma unroll
        for (int c = 0; c < CH; ++c) cp_async16_zfill(a + core_off<KC>(tid, c), ok ? (const void*)(src + c * 8) : src, ok);
        const uint32_t b = sB + buf * B_BYTES;
        for (int q = tid; q < BN * CH; q += 128) {
            const int n = q / CH, c = q % CH;
            const bool okb = n0 + n < Cout;
            const bf16* bs = okb ? B + ((long long)btap * Cout + n0 + n) * Cin + k0 + c * 8 : B;
            cp_async16_zfill(b + core_off<KC>(n, c), bs, okb);
        }
        cp_async_commit();
    };

    constexpr uint32_t IDESC = tc::idesc_bf16_f32(BM, BN);
    bool failed = false;
    load(0, 0);
    for (int s = 0; s < S; ++s) {
        const int buf = s & 1;
        cp_async_wait_all();
        tc::fence_proxy_async_smem();
        if (__syncthreads_or(failed ? 1 : 0)) {
            failed = true;
            break;
        }
        if (tid == 0) {
            tc::fence_after_sync();
            const uint32_t a = sA + buf * A_BYTES, b = sB + buf * B_BYTES;
#pragma unroll
            for (int kk = 0; kk < KC / 16; ++kk)
                tc::mma_bf16(tmem, tc::smem_desc(a + kk * 256, 128, KC * 16), tc::smem_desc(b + kk * 256, 128, KC * 16),
                             IDESC, (s > 0 || kk > 0) ? 1u : 0u);
            tc::mma_commit(bar0 + 8 * buf);
        }
        if (s + 1 < S) {
            // the other buffer is free once the MMAs of stage s - 1 are complete
            if (s >= 1 && !tc::mbar_wait(bar0 + 8 * (buf ^ 1), (uint32_t)((s - 1) >> 1) & 1u, WAIT_LIMIT_NS)) failed = true;
            if (!failed) load(s + 1, buf ^ 1);
        }
    }
    if (!failed) {
        const int last = S - 1;
        if (!tc::mbar_wait(bar0 + 8 * (last & 1), (uint32_t)(last >> 1) & 1u, WAIT_LIMIT_NS)) failed = true;
    }
    failed = __syncthreads_or(failed ? 1 : 0) != 0;
    if (!failed) {
        tc::fence_after_sync();
        const uint32_t row_addr = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll 1
        for (int c0 = 0; c0 < BN; c0 += 16) {
            float acc[16];
            tc::tmem_ld16(row_addr + (uint32_t)c0, acc);
            if (vin) {
                __align__(16) __nv_bfloat162 o[8];
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const int n = n0 + c0 + 2 * i;
                    float a0 = acc[2 * i] + (bias ? bias[n] : 0.f);
                    float a1 = acc[2 * i + 1] + (bias ? bias[n + 1] : 0.f);
                    if (relu) {
                        a0 = fmaxf(a0, 0.f);
                        a1 = fmaxf(a1, 0.f);
                    }
                    o[i] = __floats2bfloat162_rn(a0, a1);
                }
                uint4* dst = reinterpret_cast<uint4*>(outb + v * Cout + n0 + c0);
                dst[0] = *reinterpret_cast<const uint4*>(&o[0]);
                dst[1] = *reinterpret_cast<const uint4*>(&o[4]);
            }
        }
    } else if (tid == 0) {
        atomicExch(&g_tc_error, 1);
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, NCOLS);
}

// Dynamic shared memory per block: the two stage buffers, padded when needed so that no more
// blocks are resident on an SM than its 512 tensor-memory columns serve (an allocation then never
// waits for another block).
template <int KC, int BN>
static cudaError_t launch_tc(const bf16* in, const bf16* Bw, const float* bias, bf16* out, int N, int D, int H, int W,
                             int Cin, int Cout, bool flip, bool relu, cudaStream_t s) {
    constexpr int NCOLS = BN < 32 ? 32 : BN;
    constexpr int MAX_RESIDENT = 512 / NCOLS;
    static int smem = 0;
    if (smem == 0) {
        int bytes = 2 * 128 * KC * 2 + 2 * BN * KC * 2 + 32;
        cudaError_t e = cudaFuncSetAttribute(k_conv3d_tc<KC, BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        if (e != cudaSuccess) return e;
        for (;;) {
            int per_sm = 0;
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_conv3d_tc<KC, BN>, 128, bytes);
            if (e != cudaSuccess) return e;
            if (per_sm <= MAX_RESIDENT) break;
            bytes += 4096;
            if (bytes > 200 * 1024) return cudaErrorInvalidConfiguration;
        }
        smem = bytes;
    }
    const long long V = (long long)D * H * W;
    const dim3 grid((unsigned)((V + 127) / 128), (unsigned)(Cout / BN), (unsigned)N);
    k_conv3d_tc<KC, BN><<<grid, 128, smem, s>>>(in, Bw, bias, out, D, H, W, Cin, Cout, flip, relu);
    return cudaGetLastError();
}

template <int KC>
static cudaError_t dispatch_bn(const bf16* in, const bf16* Bw, const float* bias, bf16* out, int N, int D, int H, int W,
                               int Cin, int Cout, bool flip, bool relu, cudaStream_t s) {
    if (Cout % 128 == 0) return launch_tc<KC, 128>(in, Bw, bias, out, N, D, H, W, Cin, Cout, flip, relu, s);
    if (Cout % 64 == 0) return launch_tc<KC, 64>(in, Bw, bias, out, N, D, H, W, Cin, Cout, flip, relu, s);
    return launch_tc<KC, 32>(in, Bw, bias, out, N, D, H, W, Cin, Cout, flip, relu, s);
}

cudaError_t conv3d(const bf16* in, const bf16* Bw, const float* bias, bf16* out, int N, int D, int H, int W, int Cin,
                   int Cout, bool flip, bool relu, cudaStream_t s) {
    if (Cin % 16 != 0 || Cout % 32 != 0 || Cin <= 0 || Cout <= 0) return cudaErrorInvalidValue;
    if (Cin % 64 == 0) return dispatch_bn<64>(in, Bw, bias, out, N, D, H, W, Cin, Cout, flip, relu, s);
    if (Cin % 32 == 0) return dispatch_bn<32>(in, Bw, bias, out, N, D, H, W, Cin, Cout, flip, relu, s);
    return dispatch_bn<16>(in, Bw, bias, out, N, D, H, W, Cin, Cout, flip, relu, s);
}

cudaError_t tc_status(int* failed, cudaStream_t s) {
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return e;
    return cudaMemcpyFromSymbol(failed, g_tc_error, sizeof(int));
}

}  // namespace nn
}  // namespace hrt
