// hrt_quantile_ratio_noalloc: the convergence quantile of a Lucy iteration for callers that
// cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: a host framework whose allocator has already reserved
// the device memory (a caching allocator or a fixed arena) leaves nothing for a library to take,
// and latency-bound callers cannot afford the device-wide synchronisation cudaMalloc/cudaFree
// may impose.  This entry point needs no allocation at all: its only scratch is the fixed
// file-scope array below, which every GPU that loads the library holds until the process exits.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "../../include/hrt.h"

namespace {

// Scratch: a 256-bin radix histogram and four words of select state
// (prefix of the answer, rank still to find, number of cells with dust, answer).
constexpr int NA_BINS = 256;
struct NoAllocScratch {
    unsigned int hist[NA_BINS];
    unsigned long long state[4];
};
static __device__ __align__(256) NoAllocScratch g_scratch;

constexpr int MAX_DEVICES = 64;
std::mutex g_mutex;
NoAllocScratch* g_addr[MAX_DEVICES] = {nullptr};

__device__ __forceinline__ bool key_of(const double* prev, const double* cur, const float* rho, long long c,
                                       unsigned long long& key) {
    if (!(rho[c] > 0.f)) return false;
    const double a = prev[c], b = cur[c];
    double R = fmax(a / b, b / a);
    if (!(R == R)) R = __longlong_as_double(0x7ff0000000000000ll);
    key = (unsigned long long)__double_as_longlong(R);
    return true;
}

__global__ void na_init(NoAllocScratch* s) {
    for (int i = threadIdx.x; i < NA_BINS; i += blockDim.x) s->hist[i] = 0u;
    if (threadIdx.x == 0) s->state[0] = s->state[1] = s->state[2] = s->state[3] = 0ull;
}

__global__ void __launch_bounds__(256) na_count(const float* rho, long long n, NoAllocScratch* s) {
    unsigned long long cnt = 0;
    for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x)
        cnt += rho[c] > 0.f;
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_down_sync(0xffffffffu, cnt, o);
    if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(&s->state[2], cnt);
}

// rank of the nearest-rank p-quantile among the cells with dust
__global__ void na_rank(double p, NoAllocScratch* s) {
    const unsigned long long m = s->state[2];
    long long k = m > 0 ? (long long)ceil(p * (double)m) - 1 : 0;
    if (k < 0) k = 0;
    if (m > 0 && k > (long long)m - 1) k = (long long)m - 1;
    s->state[1] = (unsigned long long)k;
}

__global__ void __launch_bounds__(256) na_hist(const double* prev, const double* cur, const float* rho, long long n,
                                               int shift, NoAllocScratch* s) {
    __shared__ unsigned int h[NA_BINS];
    h[threadIdx.x] = 0u;
    __syncthreads();
    const unsigned long long prefix = s->state[0];
    const unsigned long long himask = (shift >= 56) ? 0ull : (~0ull << (shift + 8));
    for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
        unsigned long long key;
        if (key_of(prev, cur, rho, c, key) && (key & himask) == (prefix & himask))
            atomicAdd(&h[(key >> shift) & 255ull], 1u);
    }
    __syncthreads();
    if (h[threadIdx.x]) atomicAdd(&s->hist[threadIdx.x], h[threadIdx.x]);
}

__global__ void na_pick(int shift, NoAllocScratch* s, double* out) {
    if (threadIdx.x != 0) return;
    unsigned long long k = s->state[1], cum = 0;
    int b = 0;
    for (; b < NA_BINS - 1; ++b) {
        if (cum + s->hist[b] > k) break;
        cum += s->hist[b];
    }
    s->state[0] |= ((unsigned long long)b) << shift;
    s->state[1] = k - cum;
    for (int i = 0; i < NA_BINS; ++i) s->hist[i] = 0u;
    if (shift == 0) {
        const double nan = __longlong_as_double(0x7ff8000000000000ll);
        *out = s->state[2] > 0 ? __longlong_as_double((long long)s->state[0]) : nan;
    }
}

// Device address of the scratch array for the current device, looked up once per device.
NoAllocScratch* scratch_for_current_device(int* err) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) {
        cudaGetLastError();
        *err = HRT_ECUDA;
        return nullptr;
    }
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_addr[dev]) {
        void* ptr = nullptr;
        if (cudaGetSymbolAddress(&ptr, g_scratch) != cudaSuccess || !ptr) {
            cudaGetLastError();
            *err = HRT_ECUDA;
            return nullptr;
        }
        g_addr[dev] = static_cast<NoAllocScratch*>(ptr);
    }
    return g_addr[dev];
}

}  // namespace

extern "C" int hrt_quantile_ratio_noalloc(int64_t n, const double* d_prev, const double* d_cur, const float* d_rho,
                                          double p, double* d_out, void* stream) {
    if (n < 1 || n > HRT_NOALLOC_MAX_CELLS) return HRT_EINVAL;
    if (!d_prev || !d_cur || !d_rho || !d_out) return HRT_EINVAL;
    if (!(p > 0.0 && p <= 1.0)) return HRT_EINVAL;
    // an error left by earlier work on this thread is the caller's: report it apart and leave it
    if (cudaPeekAtLastError() != cudaSuccess) return HRT_ESTATE;
    int err = HRT_OK;
    NoAllocScratch* s = scratch_for_current_device(&err);
    if (!s) return err;
    const cudaStream_t st = (cudaStream_t)stream;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) {
        cudaGetLastError();
        return HRT_ECUDA;
    }
    const long long need = (n + 255) / 256;
    const int grid = (int)(need < (long long)sms * 8 ? need : (long long)sms * 8);
    na_init<<<1, 256, 0, st>>>(s);
    na_count<<<grid, 256, 0, st>>>(d_rho, n, s);
    na_rank<<<1, 1, 0, st>>>(p, s);
    for (int shift = 56; shift >= 0; shift -= 8) {
        na_hist<<<grid, 256, 0, st>>>(d_prev, d_cur, d_rho, n, shift, s);
        na_pick<<<1, 32, 0, st>>>(shift, s, d_out);
    }
    if (cudaGetLastError() != cudaSuccess) return HRT_ECUDA;
    return HRT_OK;
}
