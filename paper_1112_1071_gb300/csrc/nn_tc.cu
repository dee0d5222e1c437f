// 3x3x3 'same' convolution of the learned warm start on the 5th-generation tensor cores: an
// implicit GEMM out[v][n] = act(b[n] + sum_{tap, k} in[v + off(tap)][k] * B[tap][n][k]) with the
// FP32 accumulator in tensor memory.
//
// Per block (128 threads): a brick of 16 (y) x 8 (x) voxels of one z plane is the MMA's M = 128
// (row = 8 y + x = tensor-memory lane), BN outputs its N.  For each chunk of 16 input channels
// the block loads a halo of 3 (z) x 18 (y) x 10 (x) voxels, as three x-shifted copies laid out in
// the no-swizzle K-major core-matrix layout (8 voxels along x x 16 bytes of channels per core
// matrix, the chunk's two core matrices 128 bytes apart, one 8-voxel group per (copy, z, y) 256
// bytes apart), and the weights of TG taps (all 27, or 9 when BN = 128) in the same layout.  The
// A operand of tap (dz, dy, dx) is 16 consecutive groups of the dx copy starting at (dz, dy): a
// shared-memory descriptor, no copy per tap; the input is read from L2 about 4 times instead of
// 27.  After one cp.async wait and one barrier a single thread issues the TG tcgen05.mma of the
// phase back to back (M = 128, N = BN, K = 16, BF16 in, FP32 accumulate) and commits them to an
// mbarrier, which every thread waits on before the next phase overwrites the operands; other
// resident blocks overlap their loads with these MMAs.  The epilogue reads each voxel's row of
// the accumulator with tcgen05.ld, adds the bias, applies ReLU and stores BF16.  Every wait is
// bounded (2 s): past it the block records an error, frees its tensor memory and returns.
#include <cuda.h>          // CUtensorMap and its enums (the encoder is fetched from the driver at run time)
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <atomic>
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
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

constexpr int BRICK_Y = 16, BRICK_X = 8, HALO_Y = BRICK_Y + 2;
constexpr int KC = 16;                              // input channels per halo
constexpr int GROUP = KC * 16;                      // one 8-voxel group: two core matrices
constexpr int HALO_GROUPS = 3 * 3 * HALO_Y;         // (dx copy, z, y)
constexpr int HALO_BYTES = HALO_GROUPS * GROUP;

// taps per phase: all 27 while their weights take at most 32 KB, else 9 (one z plane of taps)
template <int BN>
constexpr int taps_per_phase() { return 27 * BN * KC * 2 <= 32768 ? 27 : 9; }
template <int BN>
constexpr int smem_bytes() { return HALO_BYTES + taps_per_phase<BN>() * BN * KC * 2 + 16; }

}  // namespace

template <int BN>
__global__ void __launch_bounds__(128) k_conv3d_tc(const bf16* __restrict__ in, const bf16* __restrict__ B,
                                                   const float* __restrict__ bias, bf16* __restrict__ out, int D, int H,
                                                   int W, int Cin, int Cout, int flip, int relu) {
    constexpr uint32_t NCOLS = BN < 32 ? 32 : BN;
    constexpr int TG = taps_per_phase<BN>();
    constexpr int B_TILE = BN * KC * 2;             // one tap's weights
    extern __shared__ __align__(1024) unsigned char smem[];
    const uint32_t sH = tc::smem_addr(smem);
    const uint32_t sB = sH + HALO_BYTES;
    const uint32_t bar = sB + TG * B_TILE;          // one 8-byte mbarrier
    const uint32_t slot = bar + 8;                  // tensor-memory address written by the allocation
    const int tid = threadIdx.x, warp = tid >> 5;
    const int nbx = (W + BRICK_X - 1) / BRICK_X, nby = (H + BRICK_Y - 1) / BRICK_Y;
    const int x0 = (blockIdx.x % nbx) * BRICK_X;
    const int y0 = ((blockIdx.x / nbx) % nby) * BRICK_Y;
    const int z0 = blockIdx.x / (nbx * nby);
    const int n0 = blockIdx.y * BN;
    const long long V = (long long)D * H * W;
    const bf16* inb = in + (long long)blockIdx.z * V * Cin;
    bf16* outb = out + (long long)blockIdx.z * V * Cout;

    if (warp == 0) {
        tc::tmem_alloc(slot, NCOLS);
        tc::tmem_relinquish();
    }
    if (tid == 0) {
        tc::mbar_init(bar, 1);
        tc::fence_mbar_init();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    uint32_t tmem;
    asm volatile("ld.shared.u32 %0, [%1];" : "=r"(tmem) : "r"(slot) : "memory");

    // halo of channels k0 .. k0 + 15: thread -> (group parity, voxel xr, 16-byte chunk c); each
    // pass covers 8 groups, 21 passes the 162 groups (the last partly)
    auto load_halo = [&](int k0) {
        const int c = tid & 1, xr = (tid >> 1) & 7, gsub = tid >> 4;
        for (int g = gsub; g < HALO_GROUPS; g += 8) {
            const int hy = g % HALO_Y, hz = (g / HALO_Y) % 3, dxc = g / (3 * HALO_Y);
            const int xx = x0 + xr + dxc - 1, yy = y0 + hy - 1, zz = z0 + hz - 1;
            const bool ok = xx >= 0 && xx < W && yy >= 0 && yy < H && zz >= 0 && zz < D;
            const bf16* src = ok ? inb + (((long long)zz * H + yy) * W + xx) * Cin + k0 + c * 8 : inb;
            asm volatile("cp.async.ca.shared.global [%0], [%1], 16, %2;\n" ::"r"(sH + g * GROUP + c * 128 + xr * 16),
                         "l"(src), "r"(ok ? 16 : 0)
                         : "memory");
        }
    };
    // weights of taps t0 .. t0 + TG - 1 for channels k0 .. k0 + 15: tile (tap) -> rows n -> 2 chunks
    auto load_b = [&](int t0, int k0) {
        for (int q = tid; q < TG * BN * 2; q += 128) {
            const int c = q & 1, n = (q >> 1) % BN, t = q / (2 * BN);
            const int btap = flip ? 26 - (t0 + t) : t0 + t;
            const bf16* bs = B + ((long long)btap * Cout + n0 + n) * Cin + k0 + c * 8;
            cp_async16_zfill(sB + t * B_TILE + (n >> 3) * GROUP + c * 128 + (n & 7) * 16, bs, true);
        }
    };

    constexpr uint32_t IDESC = tc::idesc_bf16_f32(128, BN);
    const int kchunks = Cin / KC;
    const int phases = kchunks * (27 / TG);
    bool failed = false;
    for (int ph = 0; ph < phases && !failed; ++ph) {
        const int ci = ph / (27 / TG), t0 = (ph % (27 / TG)) * TG;
        // the operands of the previous phase are free once its MMAs are complete
        if (ph > 0 && !tc::mbar_wait(bar, (uint32_t)(ph - 1) & 1u, WAIT_LIMIT_NS)) failed = true;
        if (!failed) {
            if (t0 == 0) load_halo(ci * KC);
            load_b(t0, ci * KC);
        }
        cp_async_commit();
        cp_async_wait<0>();
        tc::fence_proxy_async_smem();
        if (__syncthreads_or(failed ? 1 : 0)) {
            failed = true;
            break;
        }
        if (tid == 0) {
            tc::fence_after_sync();
#pragma unroll 1
            for (int t = 0; t < TG; ++t) {
                const int tap = t0 + t;
                const int dz = tap / 9, dy = (tap / 3) % 3, dx = tap % 3;          // 0..2 = offset + 1
                const uint32_t a = sH + ((dx * 3 + dz) * HALO_Y + dy) * GROUP;
                tc::mma_bf16(tmem, tc::smem_desc(a, 128, GROUP), tc::smem_desc(sB + t * B_TILE, 128, GROUP), IDESC,
                             (ph > 0 || t > 0) ? 1u : 0u);
            }
            tc::mma_commit(bar);
        }
    }
    if (!failed && !tc::mbar_wait(bar, (uint32_t)(phases - 1) & 1u, WAIT_LIMIT_NS)) failed = true;
    failed = __syncthreads_or(failed ? 1 : 0) != 0;
    if (!failed) {
        tc::fence_after_sync();
        const int yy = y0 + tid / BRICK_X, xx = x0 + tid % BRICK_X;
        const bool vin = yy < H && xx < W;
        const long long v = ((long long)z0 * H + yy) * W + xx;
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

// Dynamic shared memory per block: halo and weights, padded when needed so that no more blocks
// are resident on an SM than its 512 tensor-memory columns serve (an allocation then never
// waits for another block).
template <int BN>
static cudaError_t launch_tc(const bf16* in, const bf16* Bw, const float* bias, bf16* out, int N, int D, int H, int W,
                             int Cin, int Cout, bool flip, bool relu, cudaStream_t s) {
    constexpr int NCOLS = BN < 32 ? 32 : BN;
    constexpr int MAX_RESIDENT = 512 / NCOLS;
    // the attribute belongs to the current device's context: set it on every launch
    cudaError_t e = cudaFuncSetAttribute(k_conv3d_tc<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (e != cudaSuccess) return e;
    // residency-capped size, computed once per instantiation (host threads may race to fill it
    // with the same value)
    static std::atomic<int> smem_cached{0};
    int smem = smem_cached.load(std::memory_order_relaxed);
    if (smem == 0) {
        int bytes = smem_bytes<BN>();
        for (;;) {
            int per_sm = 0;
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_conv3d_tc<BN>, 128, bytes);
            if (e != cudaSuccess) return e;
            if (per_sm <= MAX_RESIDENT) break;
            bytes += 4096;
            if (bytes > 200 * 1024) return cudaErrorInvalidConfiguration;
        }
        smem = bytes;
        smem_cached.store(bytes, std::memory_order_relaxed);
    }
    const unsigned bricks = (unsigned)(((W + BRICK_X - 1) / BRICK_X) * ((H + BRICK_Y - 1) / BRICK_Y) * D);
    const dim3 grid(bricks, (unsigned)(Cout / BN), (unsigned)N);
    k_conv3d_tc<BN><<<grid, 128, smem, s>>>(in, Bw, bias, out, D, H, W, Cin, Cout, flip, relu);
    return cudaGetLastError();
}

cudaError_t conv3d_phased(const bf16* in, const bf16* Bw, const float* bias, bf16* out, int N, int D, int H, int W,
                          int Cin, int Cout, bool flip, bool relu, cudaStream_t s) {
    if (Cin % 16 != 0 || Cout % 32 != 0 || Cin <= 0 || Cout <= 0) return cudaErrorInvalidValue;
    if (Cout % 128 == 0) return launch_tc<128>(in, Bw, bias, out, N, D, H, W, Cin, Cout, flip, relu, s);
    if (Cout % 64 == 0) return launch_tc<64>(in, Bw, bias, out, N, D, H, W, Cin, Cout, flip, relu, s);
    return launch_tc<32>(in, Bw, bias, out, N, D, H, W, Cin, Cout, flip, relu, s);
}

// ---------------------------------------------------------------- TMA-fed, pipelined convolution
// The same implicit GEMM as k_conv3d_tc, arranged for Blackwell's asynchronous units.  A
// persistent CTA per SM walks its share of (image, z, 16 x 8 brick, output-channel tile) work
// items with three roles: one thread loads, per 16-channel chunk, the halo (one TMA box of 10 x
// 18 x 3 voxels per 8-channel half) and all 27 taps' weights (one bulk copy per 8-channel half
// from the packed layout of pack_tma_weights) into one of the shared-memory stages; one thread issues the chunk's 27 MMAs into one of two tensor-memory accumulators as
// soon as the stage has landed and hands the stage back when they complete; four epilogue warps
// drain the other accumulator (bias, ReLU, BF16 store) meanwhile.  The loads of the next chunks
// thus overlap the MMAs of this one, and a tile's epilogue the next tile's MMAs.  A TMA box of 8
// channels (16 bytes) x voxels along x puts each voxel's 8 channels in one 16-byte row, so 8
// consecutive voxels of one (z, y) row are a no-swizzle K-major core matrix; the box holds 10
// voxels along x, so the three x shifts of a tap are the same box read 0, 16 or 32 bytes further
// into each 160-byte row (the stride byte offset of the operand descriptor), and the halo is
// loaded once, not three times; the second channel half lies one region further (its leading
// byte offset).  The packed weights land as [tap][output channel][8 channels], 8 output channels
// per core matrix, so a chunk's weights are 2 bulk copies, not 2 x 27 x BN 16-byte rows.  Every wait
// gives up after WAIT_LIMIT_NS (or when another role has given up): the block records the error,
// lets its own loads and MMAs drain (bounded), frees its tensor memory and returns.
constexpr int TM_THREADS = 192;                     // warps 0-3 epilogue, 4 TMA, 5 MMA

// NT = 16 x 8-voxel tiles side by side along x per work item: they share one halo and one fetch
// of the weights (the weights are most of a stage's bytes)
template <int BN, int NT>
struct TmShape {
    static constexpr int HX = NT * BRICK_X + 2;     // halo voxels along x
    static constexpr int ROW = HX * 16;             // one (z, y) row of one channel half
    static constexpr int HALF_BYTES = 3 * HALO_Y * ROW;            // one channel half of the halo
    static constexpr int HALF = (HALF_BYTES + 127) & ~127;         // its region, 128-byte aligned
    static constexpr int WHALF = 27 * BN * 16;      // one channel half of all taps' weights
    static constexpr int STAGE = 2 * HALF + 2 * WHALF;
    static constexpr int TX = 2 * HALF_BYTES + 2 * WHALF;          // bytes a stage's loads deliver
    static constexpr int FIT = (227 * 1024 - 1024 - 128) / STAGE;  // stages that fit in 227 KB
    static constexpr int STAGES = FIT > 4 ? 4 : FIT;
    static constexpr int SMEM = STAGES * STAGE + 1024 + 128;       // + alignment slack, barriers
    static constexpr uint32_t NCOLS = 2 * NT * BN;  // two accumulators of NT tiles each
    static_assert(STAGES >= 2, "two stages at least");
    static_assert(NCOLS == 64 || NCOLS == 128 || NCOLS == 256, "tensor memory columns: a power of two");
};

template <int BN, int NT>
__global__ void __launch_bounds__(TM_THREADS, 1)
    k_conv3d_tma(const __grid_constant__ CUtensorMap act, const bf16* __restrict__ Bp, const float* __restrict__ bias, bf16* __restrict__ out, int N, int D, int H, int W, int Cin, int Cout,
                 int flip, int relu) {
    using S = TmShape<BN, NT>;
    constexpr int STAGE = S::STAGE, WHALF = S::WHALF, TM_STAGES = S::STAGES, TM_HALF = S::HALF, TM_ROW = S::ROW;
    constexpr uint32_t NCOLS = S::NCOLS;
    constexpr uint32_t IDESC = tc::idesc_bf16_f32(128, BN);
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    const uint32_t raw = tc::smem_addr(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    const uint32_t sbar = base + TM_STAGES * STAGE;
    unsigned char* const gbar = smem_raw + (sbar - raw);
    auto full = [&](int st) { return sbar + 8u * st; };
    auto empty = [&](int st) { return sbar + 8u * (TM_STAGES + st); };
    auto accf = [&](int b) { return sbar + 8u * (2 * TM_STAGES + b); };
    auto acce = [&](int b) { return sbar + 8u * (2 * TM_STAGES + 2 + b); };
    const uint32_t drain = sbar + 8u * (2 * TM_STAGES + 4);
    const uint32_t slot = sbar + 8u * (2 * TM_STAGES + 5);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(gbar + 8 * (2 * TM_STAGES + 5) + 4);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    if (tid == 0) {
        for (int st = 0; st < TM_STAGES; ++st) {
            tc::mbar_init(full(st), 1);
            tc::mbar_init(empty(st), 1);
        }
        for (int b = 0; b < 2; ++b) {
            tc::mbar_init(accf(b), 1);
            tc::mbar_init(acce(b), 128);
        }
        tc::mbar_init(drain, 1);
        *abort_flag = 0;
        tc::fence_mbar_init();
    }
    if (warp == 0) {
        tc::tmem_alloc(slot, NCOLS);
        tc::tmem_relinquish();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    uint32_t tmem;
    asm volatile("ld.shared.u32 %0, [%1];" : "=r"(tmem) : "r"(slot) : "memory");

    // a bounded wait that also gives up once another role has (drains wait out their time)
    auto wait = [&](uint32_t bar, uint32_t parity, bool drain_wait = false) -> bool {
        const uint64_t t0 = tc::global_ns();
        for (;;) {
            uint32_t done;
            asm volatile(
                "{\n\t.reg .pred p;\n\t"
                "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                "selp.u32 %0, 1, 0, p;\n\t}"
                : "=r"(done)
                : "r"(bar), "r"(parity)
                : "memory");
            if (done) return true;
            if ((*abort_flag && !drain_wait) || tc::global_ns() - t0 > WAIT_LIMIT_NS) {
                *abort_flag = 1;
                atomicExch(&g_tc_error, 1);
                return false;
            }
        }
    };

    const int nbx = (W + NT * BRICK_X - 1) / (NT * BRICK_X), nby = (H + BRICK_Y - 1) / BRICK_Y, ntn = Cout / BN;
    const long long ntiles = (long long)N * D * nby * nbx * ntn;
    const int kchunks = Cin / KC;
    auto decode = [&](long long t, int& b, int& z, int& y0, int& x0, int& n0) {
        n0 = (int)(t % ntn) * BN;
        t /= ntn;
        x0 = (int)(t % nbx) * (NT * BRICK_X);
        t /= nbx;
        y0 = (int)(t % nby) * BRICK_Y;
        t /= nby;
        z = (int)(t % D);
        b = (int)(t / D);
    };

    if (warp == 4) {
        // ---------------------------------------------------------------- TMA producer
        if (lane == 0) {
            tc::tma_prefetch_map(&act);
            long long it = 0;
            bool ok = true;
            for (long long t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
                int b, z, y0, x0, n0;
                decode(t, b, z, y0, x0, n0);
                for (int c = 0; c < kchunks && ok; ++c, ++it) {
                    const int st = (int)(it % TM_STAGES);
                    const uint32_t use = (uint32_t)(it / TM_STAGES);
                    if (!wait(empty(st), (use & 1u) ^ 1u)) {
                        ok = false;
                        break;
                    }
                    const uint32_t sb = base + st * STAGE;
                    tc::mbar_arrive_expect_tx(full(st), (uint32_t)S::TX);
                    for (int h = 0; h < 2; ++h)
                        tc::tma_load_5d(sb + h * TM_HALF, &act, c * KC + h * 8, x0 - 1, y0 - 1, z - 1, b, full(st));
                    for (int h = 0; h < 2; ++h)
                        tc::bulk_load(sb + 2 * TM_HALF + h * WHALF,
                                      Bp + ((long long)(c * 2 + h) * ntn + n0 / BN) * (27 * BN * 8), WHALF, full(st));
                }
            }
            // no copy may still be landing when the block leaves: wait for the last stages issued
            for (long long k = it - TM_STAGES; k < it; ++k)
                if (k >= 0) wait(full((int)(k % TM_STAGES)), (uint32_t)((k / TM_STAGES) & 1), true);
        }
    } else if (warp == 5) {
        // ---------------------------------------------------------------- MMA issuer
        if (lane == 0) {
            long long it = 0;
            int j = 0;
            bool ok = true;
            for (long long t = blockIdx.x; t < ntiles && ok; t += gridDim.x, ++j) {
                const int buf = j & 1;
                if (!wait(acce(buf), (((uint32_t)j >> 1) & 1u) ^ 1u)) break;
                tc::fence_after_sync();
                const uint32_t acc = tmem + (uint32_t)(buf * NT * BN);
                for (int c = 0; c < kchunks; ++c, ++it) {
                    const int st = (int)(it % TM_STAGES);
                    if (!wait(full(st), (uint32_t)((it / TM_STAGES) & 1))) {
                        ok = false;
                        break;
                    }
                    tc::fence_after_sync();
                    const uint32_t sb = base + st * STAGE;
                    // the stage's descriptors once; each tap adds a constant to their address
                    // field (shared addresses < 2^18, so the 14-bit field never carries)
                    const uint64_t a0 = tc::smem_desc(sb, TM_HALF, TM_ROW);
                    const uint64_t b0 = tc::smem_desc(sb + 2 * TM_HALF, WHALF, 128);
#pragma unroll
                    for (int tap = 0; tap < 27; ++tap) {
                        const int dz = tap / 9, dy = (tap / 3) % 3, dx = tap % 3;
                        const uint32_t boff = (flip ? (26 - tap) * BN : tap * BN);   // x 16 bytes >> 4
#pragma unroll
                        for (int u = 0; u < NT; ++u) {
                            const uint32_t aoff = ((dz * HALO_Y + dy) * TM_ROW + (u * BRICK_X + dx) * 16) >> 4;
                            tc::mma_bf16(acc + (uint32_t)(u * BN), a0 + aoff, b0 + boff, IDESC,
                                         (c > 0 || tap > 0) ? 1u : 0u);
                        }
                    }
                    tc::mma_commit(empty(st));          // the stage is free once these MMAs complete
                }
                if (ok) tc::mma_commit(accf(buf));
            }
            // every MMA this thread issued has completed before tensor memory is freed
            tc::mma_commit(drain);
            wait(drain, 0u, true);
        }
    } else {
        // ---------------------------------------------------------------- epilogue (warps 0-3)
        int j = 0;
        const long long V = (long long)D * H * W;
        for (long long t = blockIdx.x; t < ntiles; t += gridDim.x, ++j) {
            const int buf = j & 1;
            bool got = true;
            if (lane == 0) got = wait(accf(buf), ((uint32_t)j >> 1) & 1u);
            if (!__shfl_sync(0xffffffffu, got ? 1 : 0, 0)) break;
            tc::fence_after_sync();
            int b, z, y0, x0, n0;
            decode(t, b, z, y0, x0, n0);
            bf16* outb = out + (long long)b * V * Cout;
#pragma unroll 1
            for (int u = 0; u < NT; ++u) {
                const int yy = y0 + tid / BRICK_X, xx = x0 + u * BRICK_X + tid % BRICK_X;
                const bool vin = yy < H && xx < W;
                const long long v = ((long long)z * H + yy) * W + xx;
                const uint32_t row_addr = tmem + (uint32_t)((buf * NT + u) * BN) + ((uint32_t)(warp * 32) << 16);
#pragma unroll 1
                for (int c0 = 0; c0 < BN; c0 += 16) {
                    float accv[16];
                    tc::tmem_ld16(row_addr + (uint32_t)c0, accv);
                    if (vin) {
                        __align__(16) __nv_bfloat162 o[8];
#pragma unroll
                        for (int i = 0; i < 8; ++i) {
                            const int n = n0 + c0 + 2 * i;
                            float a0 = accv[2 * i] + (bias ? bias[n] : 0.f);
                            float a1 = accv[2 * i + 1] + (bias ? bias[n + 1] : 0.f);
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
            }
            tc::fence_before_sync();
            tc::mbar_arrive(acce(buf));
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, NCOLS);
}

namespace {
typedef CUresult (*EncodeTiled)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiled encode_tiled() {
    static std::atomic<void*> fn{nullptr};
    void* f = fn.load(std::memory_order_acquire);
    if (!f) {
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        fn.store(f, std::memory_order_release);
    }
    return reinterpret_cast<EncodeTiled>(f);
}
}  // namespace

template <int BN, int NT>
static cudaError_t launch_tma(const bf16* in, const bf16* Bp, const float* bias, bf16* out, int N, int D, int H, int W,
                              int Cin, int Cout, bool flip, bool relu, cudaStream_t s) {
    using S = TmShape<BN, NT>;
    EncodeTiled enc = encode_tiled();
    if (!enc) return cudaErrorNotSupported;
    CUtensorMap act;
    const cuuint64_t adim[5] = {(cuuint64_t)Cin, (cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)D, (cuuint64_t)N};
    const cuuint64_t astr[4] = {(cuuint64_t)Cin * 2, (cuuint64_t)W * Cin * 2, (cuuint64_t)H * W * Cin * 2,
                                (cuuint64_t)D * H * W * Cin * 2};
    const cuuint32_t abox[5] = {8, (cuuint32_t)S::HX, HALO_Y, 3, 1};
    const cuuint32_t ones[5] = {1, 1, 1, 1, 1};
    if (enc(&act, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, const_cast<bf16*>(in), adim, astr, abox, ones,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return cudaErrorInvalidValue;
    constexpr int SMEM = S::SMEM;
    cudaError_t e = cudaFuncSetAttribute(k_conv3d_tma<BN, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    const long long ntiles =
        (long long)N * D * ((H + BRICK_Y - 1) / BRICK_Y) * ((W + NT * BRICK_X - 1) / (NT * BRICK_X)) * (Cout / BN);
    const int grid = (int)(ntiles < sms ? ntiles : sms);
    k_conv3d_tma<BN, NT><<<grid, TM_THREADS, SMEM, s>>>(act, Bp, bias, out, N, D, H, W, Cin, Cout, flip ? 1 : 0,
                                                    relu ? 1 : 0);
    return cudaGetLastError();
}

// The TMA-fed kernel whenever the packed weights are given (tiles of 64 output channels when
// Cout % 64 == 0, else 32), the per-phase kernel otherwise.
cudaError_t conv3d(const bf16* in, const bf16* Bw, const bf16* Bp, const float* bias, bf16* out, int N, int D, int H,
                   int W, int Cin, int Cout, bool flip, bool relu, cudaStream_t s) {
    if (Cin % 16 != 0 || Cout % 32 != 0 || Cin <= 0 || Cout <= 0) return cudaErrorInvalidValue;
    if (Bp && encode_tiled()) {
        const bool two = W > BRICK_X;       // two tiles per weight fetch unless the grid is one tile wide
        if (tma_tile_n(Cout) == 64)
            return two ? launch_tma<64, 2>(in, Bp, bias, out, N, D, H, W, Cin, Cout, flip, relu, s)
                       : launch_tma<64, 1>(in, Bp, bias, out, N, D, H, W, Cin, Cout, flip, relu, s);
        return two ? launch_tma<32, 2>(in, Bp, bias, out, N, D, H, W, Cin, Cout, flip, relu, s)
                   : launch_tma<32, 1>(in, Bp, bias, out, N, D, H, W, Cin, Cout, flip, relu, s);
    }
    return conv3d_phased(in, Bw, bias, out, N, D, H, W, Cin, Cout, flip, relu, s);
}

// ---------------------------------------------------------------- weight gradient
// dW[tap][i][o] += sum_v in[v + off(tap)][i] dY[v][o]: per block a GEMM with M = 128 rows of
// (tap, input channel) -- TPG = 128 / CB taps of a block of CB input channels --, N = BN output
// channels and K = a contiguous range of voxels (split over blocks; FP32 atomics at the end).
// Both operands are read voxel by voxel with their channels contiguous, the MN-major form:
// every 16-byte load (8 channels of one voxel) is one row of a core matrix (8 voxels along K x 16
// bytes along M or N), core matrices 128 bytes apart along K (the descriptor's leading byte
// offset, as in the K-major operands of the convolution) and KV * 16 bytes apart along M/N (its
// stride byte offset).
// KV = 64 voxels per stage (four K = 16 MMAs), two stage buffers, one mbarrier per buffer.
constexpr int WG_KV = 64;

template <int BN>
__global__ void __launch_bounds__(128) k_conv3d_wgrad_tc(const bf16* __restrict__ in, const bf16* __restrict__ dy,
                                                         float* __restrict__ dw, int D, int H, int W, int Cin, int Cout,
                                                         int CB, int nsplit, int nbatch) {
    constexpr uint32_t NCOLS = BN < 32 ? 32 : BN;
    constexpr int A_BYTES = 128 * WG_KV * 2, B_BYTES = BN * WG_KV * 2;
    constexpr int MN_STRIDE = WG_KV / 8 * 128;       // between 8-row groups along M (or N)
    extern __shared__ __align__(1024) unsigned char smem[];
    const uint32_t sA = tc::smem_addr(smem);
    const uint32_t sB = sA + 2 * A_BYTES;
    const uint32_t bar0 = sB + 2 * B_BYTES;
    const uint32_t slot = bar0 + 16;
    const int tid = threadIdx.x, warp = tid >> 5;
    const int TPG = 128 / CB;                        // taps per block
    const int ngroups = (27 + TPG - 1) / TPG;
    const int tap0 = (blockIdx.x % ngroups) * TPG;
    const int i0 = (blockIdx.x / ngroups) * CB;
    const int o0 = blockIdx.y * BN;
    const long long V = (long long)D * H * W, total = V * nbatch;
    const long long per = ((total + nsplit - 1) / nsplit + WG_KV - 1) / WG_KV * WG_KV;
    const long long vbeg = (long long)blockIdx.z * per;
    const long long vend = vbeg + per < total ? vbeg + per : total;

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

    // thread -> voxel kv = tid / 2 of the stage, row chunks (tid & 1) * 8 .. + 7 of the 16
    const int kv = tid >> 1, rc0 = (tid & 1) * 8;
    auto load = [&](long long v0, int buf) {
        const long long v = v0 + kv;
        const bool vin = v < vend;
        int x = 0, y = 0, z = 0;
        long long base = 0;
        if (vin) {
            const long long b = v / V, r = v - b * V;
            x = (int)(r % W);
            y = (int)((r / W) % H);
            z = (int)(r / ((long long)W * H));
            base = b * V;
        }
        const uint32_t a = sA + buf * A_BYTES + (kv >> 3) * 128 + (kv & 7) * 16;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int row0 = (rc0 + q) * 8;                 // first of the chunk's 8 rows
            const int t = row0 / CB, tap = tap0 + t, i = i0 + row0 % CB;
            bool ok = vin && t < TPG && tap < 27;
            const bf16* src = in;
            if (ok) {
                const int zz = z + tap / 9 - 1, yy = y + (tap / 3) % 3 - 1, xx = x + tap % 3 - 1;
                ok = zz >= 0 && zz < D && yy >= 0 && yy < H && xx >= 0 && xx < W;
                if (ok) src = in + (base + ((long long)zz * H + yy) * W + xx) * Cin + i;
            }
            cp_async16_zfill(a + (row0 >> 3) * MN_STRIDE, src, ok);
        }
        const uint32_t b = sB + buf * B_BYTES + (kv >> 3) * 128 + (kv & 7) * 16;
        for (int ng = (tid & 1); ng < BN / 8; ng += 2) {
            const bool ok = vin;
            cp_async16_zfill(b + ng * MN_STRIDE, ok ? (const void*)(dy + v * Cout + o0 + ng * 8) : (const void*)dy, ok);
        }
        cp_async_commit();
    };

    // instruction descriptor: FP32 D, BF16 A and B, both MN-major (bits 15 and 16), M = 128, N = BN
    constexpr uint32_t IDESC = tc::idesc_bf16_f32(128, BN) | (1u << 15) | (1u << 16);
    const int S = (int)((vend - vbeg + WG_KV - 1) / WG_KV);
    bool failed = false;
    if (S > 0) load(vbeg, 0);
    for (int s = 0; s < S; ++s) {
        const int buf = s & 1;
        cp_async_wait<0>();
        tc::fence_proxy_async_smem();
        if (__syncthreads_or(failed ? 1 : 0)) {
            failed = true;
            break;
        }
        if (tid == 0) {
            tc::fence_after_sync();
            const uint32_t a = sA + buf * A_BYTES, b = sB + buf * B_BYTES;
#pragma unroll
            for (int kk = 0; kk < WG_KV / 16; ++kk)
                tc::mma_bf16(tmem, tc::smem_desc(a + kk * 256, 128, MN_STRIDE), tc::smem_desc(b + kk * 256, 128, MN_STRIDE),
                             IDESC, (s > 0 || kk > 0) ? 1u : 0u);
            tc::mma_commit(bar0 + 8 * buf);
        }
        if (s + 1 < S) {
            if (s >= 1 && !tc::mbar_wait(bar0 + 8 * (buf ^ 1), (uint32_t)((s - 1) >> 1) & 1u, WAIT_LIMIT_NS)) failed = true;
            if (!failed) load(vbeg + (long long)(s + 1) * WG_KV, buf ^ 1);
        }
    }
    if (!failed && S > 0 && !tc::mbar_wait(bar0 + 8 * ((S - 1) & 1), (uint32_t)((S - 1) >> 1) & 1u, WAIT_LIMIT_NS))
        failed = true;
    cp_async_wait<0>();
    failed = __syncthreads_or(failed ? 1 : 0) != 0;
    if (!failed && S > 0) {
        tc::fence_after_sync();
        const int t = tid / CB, tap = tap0 + t, i = i0 + tid % CB;
        const bool valid = t < TPG && tap < 27;
        const uint32_t row_addr = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll 1
        for (int c0 = 0; c0 < BN; c0 += 16) {
            float acc[16];
            tc::tmem_ld16(row_addr + (uint32_t)c0, acc);
            if (valid) {
                float* dst = dw + ((long long)tap * Cin + i) * Cout + o0 + c0;
#pragma unroll
                for (int j = 0; j < 16; ++j) atomicAdd(dst + j, acc[j]);
            }
        }
    } else if (failed && tid == 0) {
        atomicExch(&g_tc_error, 1);
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, NCOLS);
}

template <int BN>
static cudaError_t launch_wgrad_tc(const bf16* in, const bf16* dy, float* dw, int N, int D, int H, int W, int Cin,
                                   int Cout, int CB, cudaStream_t s) {
    constexpr int NCOLS = BN < 32 ? 32 : BN;
    constexpr int MAX_RESIDENT = 512 / NCOLS;
    cudaError_t e = cudaFuncSetAttribute(k_conv3d_wgrad_tc<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (e != cudaSuccess) return e;
    static std::atomic<int> smem_cached{0};
    int smem = smem_cached.load(std::memory_order_relaxed);
    if (smem == 0) {
        int bytes = 2 * (128 + BN) * WG_KV * 2 + 32;
        for (;;) {
            int per_sm = 0;
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_conv3d_wgrad_tc<BN>, 128, bytes);
            if (e != cudaSuccess) return e;
            if (per_sm <= MAX_RESIDENT) break;
            bytes += 4096;
            if (bytes > 200 * 1024) return cudaErrorInvalidConfiguration;
        }
        smem = bytes;
        smem_cached.store(bytes, std::memory_order_relaxed);
    }
    const int TPG = 128 / CB;
    const int blocks_mn = ((27 + TPG - 1) / TPG) * (Cin / CB) * (Cout / BN);
    const long long total = (long long)D * H * W * N;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    // voxel splits: enough blocks for four waves, at least 8 stages per block
    long long nsplit = ((long long)sms * 8 + blocks_mn - 1) / blocks_mn;
    const long long max_split = (total + 8 * WG_KV - 1) / (8 * WG_KV);
    if (nsplit > max_split) nsplit = max_split;
    if (nsplit < 1) nsplit = 1;
    const dim3 grid((unsigned)(((27 + TPG - 1) / TPG) * (Cin / CB)), (unsigned)(Cout / BN), (unsigned)nsplit);
    k_conv3d_wgrad_tc<BN><<<grid, 128, smem, s>>>(in, dy, dw, D, H, W, Cin, Cout, CB, (int)nsplit, N);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- weight gradient, brick form
// dW[tap][i][o] = sum_v in[v + off(tap)][i] dY[v][o] summed brick by brick (16 x 8 voxels of one
// z-plane).  A CTA owns one dz plane of taps (9 taps), NB input channels and up to 128 output
// channels, and a range of bricks.  Per brick TMA lands the dY brick (the MMA's A: M = 128 rows of
// output channels -- rows past the real ones read zeroed regions --, K = 128 voxels, MN-major: a
// core matrix is 8 voxels x 8 channels) and the input's halo plane z + dz - 1 (B: N = NB input
// channels; a tap's (dy, dx) shift is only a start offset into the 18 x 10-voxel plane, so the
// halo is loaded once for its 9 taps).  One thread issues 9 taps x 8 K-steps of tcgen05.mma into
// nine tensor-memory accumulators that run over all the CTA's bricks; at the end four warps add
// them into dW with FP32 atomics.  Waits are bounded as in k_conv3d_tma.
constexpr int WH_THREADS = 192;                           // warps 0-3 epilogue, 4 TMA, 5 MMA
constexpr int WH_ROW = (BRICK_X + 2) * 16;                // one halo row of 8 channels: 160 bytes
constexpr int WH_HBYTES = HALO_Y * WH_ROW;                // one 8-channel halo plane: 2880 bytes
constexpr int WH_HREG = (WH_HBYTES + 127) & ~127;         // its region, 128-byte aligned
constexpr int WH_DREG = BRICK_X * BRICK_Y * 16;           // one 8-channel dY brick: 2048 bytes
constexpr int WH_DY = 16 * WH_DREG;                       // 128 output-channel rows: 32 KB

// T = the transposed roles, for layers with more input than output channels: the halo view is A
// (M = 128 input channels, zeroed rows past the real ones) and the dY brick B (N = NB output
// channels); the accumulators then hold dW^T per tap.
template <int NB, bool T>
struct WhShape {
    static constexpr int HREGS = T ? 16 : NB / 8;     // halo regions (8 input channels each)
    static constexpr int DREGS = T ? NB / 8 : 16;     // dY regions (8 output channels each)
    static constexpr int HALO = HREGS * WH_HREG;
    static constexpr int HALO_AL = (HALO + 1023) & ~1023;
    static constexpr int STAGE = HALO_AL + DREGS * WH_DREG;
    static constexpr int STAGES = 4;
    static constexpr int SMEM = STAGES * STAGE + 1024 + 128;
    static constexpr uint32_t NCOLS = 9 * NB <= 256 ? 256 : 512;
    static_assert(SMEM <= 227 * 1024, "shared memory");
};

template <int NB, bool T>
__global__ void __launch_bounds__(WH_THREADS, 1)
    k_conv3d_wgrad_tma(const __grid_constant__ CUtensorMap act, const __grid_constant__ CUtensorMap dym,
                       float* __restrict__ dw, int N, int D, int H, int W, int Cin, int Cout, int nci, int nco,
                       int nsplit) {
    using S = WhShape<NB, T>;
    constexpr int STAGE = S::STAGE, WS = S::STAGES;
    constexpr uint32_t NCOLS = S::NCOLS;
    // FP32 D, BF16 A and B, both MN-major (bits 15 and 16), M = 128, N = NB
    constexpr uint32_t IDESC = tc::idesc_bf16_f32(128, NB) | (1u << 15) | (1u << 16);
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    const uint32_t raw = tc::smem_addr(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    const uint32_t sbar = base + WS * STAGE;
    unsigned char* const gbar = smem_raw + (sbar - raw);
    auto full = [&](int st) { return sbar + 8u * st; };
    auto empty = [&](int st) { return sbar + 8u * (WS + st); };
    const uint32_t accf = sbar + 8u * (2 * WS);
    const uint32_t drain = sbar + 8u * (2 * WS + 1);
    const uint32_t slot = sbar + 8u * (2 * WS + 2);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(gbar + 8 * (2 * WS + 2) + 4);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    // this CTA: (dz, input-channel block, output-channel block, split)
    int c = blockIdx.x;
    const int split = c % nsplit;
    c /= nsplit;
    const int cob = c % nco;
    c /= nco;
    const int cib = c % nci;
    const int dz = c / nci;
    const int ci0 = cib * (T ? 128 : NB), co0 = cob * (T ? NB : 128);
    const int mreal = T ? min(128, Cin - ci0) : min(128, Cout - co0);   // M rows that are real
    const int nbx = (W + BRICK_X - 1) / BRICK_X, nby = (H + BRICK_Y - 1) / BRICK_Y;
    const long long nbricks = (long long)N * D * nby * nbx;
    const long long b0 = nbricks * split / nsplit, b1 = nbricks * (split + 1) / nsplit;

    if (tid == 0) {
        for (int st = 0; st < WS; ++st) {
            tc::mbar_init(full(st), 1);
            tc::mbar_init(empty(st), 1);
        }
        tc::mbar_init(accf, 1);
        tc::mbar_init(drain, 1);
        *abort_flag = 0;
        tc::fence_mbar_init();
    }
    // the M operand's regions of rows past mreal stay zero in every stage
    for (int st = 0; st < WS; ++st) {
        const int reg = T ? WH_HREG : WH_DREG;
        const int from = (T ? 0 : S::HALO_AL) + (mreal / 8) * reg, to = (T ? 0 : S::HALO_AL) + 16 * reg;
        uint4* z = reinterpret_cast<uint4*>(smem_raw + (base - raw) + st * STAGE + from);
        for (int q = tid; q < (to - from) / 16; q += WH_THREADS) z[q] = make_uint4(0u, 0u, 0u, 0u);
    }
    tc::fence_proxy_async_smem();
    if (warp == 0) {
        tc::tmem_alloc(slot, NCOLS);
        tc::tmem_relinquish();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    uint32_t tmem;
    asm volatile("ld.shared.u32 %0, [%1];" : "=r"(tmem) : "r"(slot) : "memory");

    auto wait = [&](uint32_t bar, uint32_t parity, bool drain_wait = false) -> bool {
        const uint64_t t0 = tc::global_ns();
        for (;;) {
            uint32_t done;
            asm volatile(
                "{\n\t.reg .pred p;\n\t"
                "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                "selp.u32 %0, 1, 0, p;\n\t}"
                : "=r"(done)
                : "r"(bar), "r"(parity)
                : "memory");
            if (done) return true;
            if ((*abort_flag && !drain_wait) || tc::global_ns() - t0 > WAIT_LIMIT_NS) {
                *abort_flag = 1;
                atomicExch(&g_tc_error, 1);
                return false;
            }
        }
    };
    auto decode = [&](long long t, int& b, int& z, int& y0, int& x0) {
        x0 = (int)(t % nbx) * BRICK_X;
        t /= nbx;
        y0 = (int)(t % nby) * BRICK_Y;
        t /= nby;
        z = (int)(t % D);
        b = (int)(t / D);
    };

    if (warp == 4) {
        // ---------------------------------------------------------------- TMA producer
        if (lane == 0) {
            tc::tma_prefetch_map(&act);
            tc::tma_prefetch_map(&dym);
            const int hg = T ? mreal / 8 : NB / 8, dg = T ? NB / 8 : mreal / 8;   // boxes per stage
            const uint32_t tx = (uint32_t)(hg * WH_HBYTES + dg * WH_DREG);
            long long it = 0;
            for (long long t = b0; t < b1; ++t, ++it) {
                const int st = (int)(it % WS);
                if (!wait(empty(st), ((uint32_t)(it / WS) & 1u) ^ 1u)) break;
                int b, z, y0, x0;
                decode(t, b, z, y0, x0);
                const uint32_t sb = base + st * STAGE;
                tc::mbar_arrive_expect_tx(full(st), tx);
                for (int g = 0; g < hg; ++g)
                    tc::tma_load_5d(sb + g * WH_HREG, &act, ci0 + 8 * g, x0 - 1, y0 - 1, z + dz - 1, b, full(st));
                for (int g = 0; g < dg; ++g)
                    tc::tma_load_5d(sb + S::HALO_AL + g * WH_DREG, &dym, co0 + 8 * g, x0, y0, z, b, full(st));
            }
            // no copy may still be landing when the block leaves
            for (long long k = it - WS; k < it; ++k)
                if (k >= 0) wait(full((int)(k % WS)), (uint32_t)((k / WS) & 1), true);
        }
    } else if (warp == 5) {
        // ---------------------------------------------------------------- MMA issuer
        if (lane == 0) {
            long long it = 0;
            bool ok = true;
            for (long long t = b0; t < b1; ++t, ++it) {
                const int st = (int)(it % WS);
                if (!wait(full(st), (uint32_t)((it / WS) & 1))) {
                    ok = false;
                    break;
                }
                tc::fence_after_sync();
                const uint32_t sb = base + st * STAGE;
                // dY brick: 8-voxel core matrices 128 B apart along K, 8-channel regions apart
                // along M or N; halo: the tap's view of the plane, 8-voxel rows 160 B apart
                const uint64_t d0 = tc::smem_desc(sb + S::HALO_AL, 128, WH_DREG);
                const uint64_t h0 = tc::smem_desc(sb, WH_ROW, WH_HREG);
#pragma unroll
                for (int tap = 0; tap < 9; ++tap) {
                    const int dy = tap / 3, dx = tap % 3;
#pragma unroll
                    for (int kk = 0; kk < 8; ++kk) {
                        const uint32_t doff = (kk * 256) >> 4;
                        const uint32_t hoff = (((2 * kk + dy) * (BRICK_X + 2) + dx) * 16) >> 4;
                        if constexpr (T)
                            tc::mma_bf16(tmem + (uint32_t)(tap * NB), h0 + hoff, d0 + doff, IDESC,
                                         (t > b0 || kk > 0) ? 1u : 0u);
                        else
                            tc::mma_bf16(tmem + (uint32_t)(tap * NB), d0 + doff, h0 + hoff, IDESC,
                                         (t > b0 || kk > 0) ? 1u : 0u);
                    }
                }
                tc::mma_commit(empty(st));
            }
            if (ok && b1 > b0) tc::mma_commit(accf);
            else if (ok) tc::mbar_arrive(accf);
            tc::mma_commit(drain);
            wait(drain, 0u, true);
        }
    } else {
        // ---------------------------------------------------------------- epilogue (warps 0-3)
        bool got = true;
        if (lane == 0) got = wait(accf, 0u);
        got = __shfl_sync(0xffffffffu, got ? 1 : 0, 0) != 0;
        if (got && b1 > b0) {
            tc::fence_after_sync();
            const int m = warp * 32 + lane;               // this lane's M row
            const uint32_t row = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll 1
            for (int tap = 0; tap < 9; ++tap) {
                const int tp = dz * 9 + tap;
#pragma unroll 1
                for (int c0 = 0; c0 < NB; c0 += 16) {
                    float v[16];
                    tc::tmem_ld16(row + (uint32_t)(tap * NB + c0), v);
                    if (m < mreal) {
                        if constexpr (T) {       // row = input channel, columns = output channels
                            float* dst = dw + ((long long)tp * Cin + ci0 + m) * Cout + co0 + c0;
#pragma unroll
                            for (int q = 0; q < 16; ++q) atomicAdd(dst + q, v[q]);
                        } else {                 // row = output channel, columns = input channels
                            float* dst = dw + ((long long)tp * Cin + ci0 + c0) * Cout + co0 + m;
#pragma unroll
                            for (int q = 0; q < 16; ++q) atomicAdd(dst + (long long)q * Cout, v[q]);
                        }
                    }
                }
            }
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, NCOLS);
}

template <int NB, bool T>
static cudaError_t launch_wgrad_tma(const bf16* in, const bf16* dy, float* dw, int N, int D, int H, int W, int Cin,
                                    int Cout, cudaStream_t s) {
    using S = WhShape<NB, T>;
    EncodeTiled enc = encode_tiled();
    if (!enc) return cudaErrorNotSupported;
    CUtensorMap act, dym;
    const cuuint32_t ones[5] = {1, 1, 1, 1, 1};
    const cuuint64_t adim[5] = {(cuuint64_t)Cin, (cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)D, (cuuint64_t)N};
    const cuuint64_t astr[4] = {(cuuint64_t)Cin * 2, (cuuint64_t)W * Cin * 2, (cuuint64_t)H * W * Cin * 2,
                                (cuuint64_t)D * H * W * Cin * 2};
    const cuuint32_t abox[5] = {8, BRICK_X + 2, HALO_Y, 1, 1};
    if (enc(&act, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, const_cast<bf16*>(in), adim, astr, abox, ones,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return cudaErrorInvalidValue;
    const cuuint64_t ddim[5] = {(cuuint64_t)Cout, (cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)D, (cuuint64_t)N};
    const cuuint64_t dstr[4] = {(cuuint64_t)Cout * 2, (cuuint64_t)W * Cout * 2, (cuuint64_t)H * W * Cout * 2,
                                (cuuint64_t)D * H * W * Cout * 2};
    const cuuint32_t dbox[5] = {8, BRICK_X, BRICK_Y, 1, 1};
    if (enc(&dym, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, const_cast<bf16*>(dy), ddim, dstr, dbox, ones,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return cudaErrorInvalidValue;
    cudaError_t e =
        cudaFuncSetAttribute(k_conv3d_wgrad_tma<NB, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, S::SMEM);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    const int nci = T ? (Cin + 127) / 128 : Cin / NB, nco = T ? Cout / NB : (Cout + 127) / 128;
    const long long nbricks = (long long)N * D * ((H + BRICK_Y - 1) / BRICK_Y) * ((W + BRICK_X - 1) / BRICK_X);
    const int cols = 3 * nci * nco;
    // one wave of one CTA per SM, at least 4 bricks per CTA
    long long nsplit = sms / cols;
    if (nsplit < 1) nsplit = 1;
    if (nsplit > nbricks / 4) nsplit = nbricks / 4 > 0 ? nbricks / 4 : 1;
    k_conv3d_wgrad_tma<NB, T><<<(unsigned)(cols * nsplit), WH_THREADS, S::SMEM, s>>>(act, dym, dw, N, D, H, W, Cin,
                                                                                    Cout, nci, nco, (int)nsplit);
    return cudaGetLastError();
}

cudaError_t conv3d_wgrad(const bf16* in, const bf16* dy, float* dw, int N, int D, int H, int W, int Cin, int Cout,
                         cudaStream_t s) {
    // the brick form, its MMA rows (128) on the wider side: output channels (input channels in
    // blocks of 32) or, with more input than output channels, input channels (output channels in
    // blocks of 32); 16 input channels (the first layer) on the stacked-tap kernel below, which
    // is faster there
    if (encode_tiled() && Cin % 32 == 0 && Cout % 8 == 0) {
        if (Cin > Cout && Cout % 32 == 0) return launch_wgrad_tma<32, true>(in, dy, dw, N, D, H, W, Cin, Cout, s);
        return launch_wgrad_tma<32, false>(in, dy, dw, N, D, H, W, Cin, Cout, s);
    }
    // channel blocks of CB <= 128 rows stacked with 128 / CB taps; other shapes on mma.sync
    const int CB = Cin <= 128 ? Cin : 64;
    if (Cin % 16 != 0 || Cout % 32 != 0 || Cin % CB != 0 || 128 % CB != 0 && Cin > 128)
        return conv3d_wgrad_mma(in, dy, dw, N, D, H, W, Cin, Cout, s);
    if (Cout % 128 == 0) return launch_wgrad_tc<128>(in, dy, dw, N, D, H, W, Cin, Cout, CB, s);
    if (Cout % 64 == 0) return launch_wgrad_tc<64>(in, dy, dw, N, D, H, W, Cin, Cout, CB, s);
    return launch_wgrad_tc<32>(in, dy, dw, N, D, H, W, Cin, Cout, CB, s);
}

cudaError_t tc_status(int* failed, cudaStream_t s) {
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return e;
    return cudaMemcpyFromSymbol(failed, g_tc_error, sizeof(int));
}

}  // namespace nn
}  // namespace hrt
