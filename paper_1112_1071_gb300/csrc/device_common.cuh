// Device-side building blocks of the packet propagation: counter-based random numbers,
// dust properties at a frequency, table sampling, directions and Henyey-Greenstein scattering.
// Single precision except where noted; all quantities in the library's scaled length unit
// (the grid's outer extent L0 = 1).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>
#include <math_constants.h>

#include "hrt_types.h"

namespace hrt {

// ---------------------------------------------------------------- Philox4x32-10
// Salmon, Moraes, Dror & Shaw (2011): ten rounds of two 32x32->64 multiplications with the
// key bumped by the Weyl constants between rounds.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) {
            k.x += 0x9E3779B9u;
            k.y += 0xBB67AE85u;
        }
        const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    }
    return c;
}

// Uniform deviate in (0, 1] on the 2^-24 lattice: ((x >> 8) + 1) 2^-24, exact in FP32.
__device__ __forceinline__ float u01(uint32_t x) { return __uint2float_rn((x >> 8) + 1u) * 0x1p-24f; }

// Packet stream: draw n uses word n mod 4 of block philox((n/4, packet, iteration, model), seed).
struct PacketRng {
    uint2 key;
    uint32_t pkt, iter, model, n;
    uint4 buf;
    __device__ __forceinline__ void init(uint2 k, uint32_t p, uint32_t it, uint32_t m) {
        key = k; pkt = p; iter = it; model = m; n = 0;
    }
    __device__ __forceinline__ float next() {
        const uint32_t s = n & 3u;
        if (s == 0) buf = philox4x32_10(make_uint4(n >> 2, pkt, iter, model), key);
        const uint32_t w = s == 0 ? buf.x : (s == 1 ? buf.y : (s == 2 ? buf.z : buf.w));
        ++n;
        return u01(w);
    }
};

// ---------------------------------------------------------------- dust at a frequency
// chi log-log between nodes, albedo linear in log nu (nodes in log space on the device).
struct DustAt {
    float chi;      // extinction (cm^2/g)
    float kappa;    // absorption (1 - albedo) chi
    float albedo;
};

__device__ __forceinline__ int find_interval(const float* __restrict__ x, int n, float v) {
    // largest j in [0, n-2] with x[j] <= v (clamped)
    int lo = 0, hi = n - 1;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(x + mid) <= v) lo = mid; else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ DustAt dust_at(const DevDust& d, float nu) {
    const float ln = logf(nu);
    const int j = find_interval(d.lnu, d.nnu, ln);
    float t = (ln - __ldg(d.lnu + j)) * __ldg(d.inv_dlnu + j);
    t = fminf(fmaxf(t, 0.f), 1.f);
    const float lc = __ldg(d.lchi + j) + t * (__ldg(d.lchi + j + 1) - __ldg(d.lchi + j));
    const float a = __ldg(d.alb + j) + t * (__ldg(d.alb + j + 1) - __ldg(d.alb + j));
    DustAt r;
    r.chi = expf(lc);
    r.albedo = a;
    r.kappa = (1.f - a) * r.chi;
    return r;
}

// ---------------------------------------------------------------- table sampling
// Piecewise-constant pdf on each interval: interval j = largest j with cdf[j] < u, then
// linear placement inside it.
__device__ __forceinline__ float sample_table(const float* __restrict__ x, const float* __restrict__ cdf, int n,
                                              float u) {
    int lo = 0, hi = n - 1;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(cdf + mid) < u) lo = mid; else hi = mid;
    }
    const float c0 = __ldg(cdf + lo), c1 = __ldg(cdf + lo + 1);
    const float x0 = __ldg(x + lo), x1 = __ldg(x + lo + 1);
    const float f = (c1 > c0) ? (u - c0) / (c1 - c0) : 0.f;
    return x0 + f * (x1 - x0);
}

// smallest index s with cdf[s] >= u (cdf[n-1] == 1)
template <typename T>
__device__ __forceinline__ int64_t select_cdf(const T* __restrict__ cdf, int64_t n, T u) {
    int64_t lo = 0, hi = n - 1;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (cdf[mid] >= u) hi = mid; else lo = mid + 1;
    }
    return lo;
}

// ---------------------------------------------------------------- directions
__device__ __forceinline__ float3 isotropic_dir(float u1, float u2) {
    const float mu = 2.f * u1 - 1.f;
    const float st = sqrtf(fmaxf(0.f, 1.f - mu * mu));
    float s, c;
    sincospif(2.f * u2, &s, &c);
    return make_float3(st * c, st * s, mu);
}

// Henyey-Greenstein cos(Theta) by inversion of its cumulative distribution.
__device__ __forceinline__ float hg_mu(float g, float u) {
    if (g == 0.f) return 2.f * u - 1.f;
    const float a = (1.f - g * g) / (1.f - g + 2.f * g * u);
    const float mu = (1.f + g * g - a * a) / (2.f * g);
    return fminf(1.f, fmaxf(-1.f, mu));
}

__device__ __forceinline__ float hg_phase(float g, float mu) {
    const float d = 1.f + g * g - 2.f * g * mu;
    return (1.f - g * g) / (4.f * CUDART_PI_F * d * sqrtf(d));
}

// Rotate u by polar angle acos(mu) and azimuth psi = 2 pi u2 about a fixed frame:
// e1 = unit(z x u), or unit(y x u) when |u_z| >= 0.99999; e2 = u x e1.
__device__ __forceinline__ float3 scatter_dir(float3 u, float mu, float u2) {
    float3 e1;
    if (fabsf(u.z) < 0.99999f) e1 = make_float3(-u.y, u.x, 0.f);
    else e1 = make_float3(u.z, 0.f, -u.x);
    const float inv = rsqrtf(e1.x * e1.x + e1.y * e1.y + e1.z * e1.z);
    e1.x *= inv; e1.y *= inv; e1.z *= inv;
    const float3 e2 = make_float3(u.y * e1.z - u.z * e1.y, u.z * e1.x - u.x * e1.z, u.x * e1.y - u.y * e1.x);
    const float st = sqrtf(fmaxf(0.f, 1.f - mu * mu));
    float sp, cp;
    sincospif(2.f * u2, &sp, &cp);
    float3 v = make_float3(mu * u.x + st * (cp * e1.x + sp * e2.x), mu * u.y + st * (cp * e1.y + sp * e2.y),
                           mu * u.z + st * (cp * e1.z + sp * e2.z));
    const float n = rsqrtf(v.x * v.x + v.y * v.y + v.z * v.z);
    v.x *= n; v.y *= n; v.z *= n;
    return v;
}

__device__ __forceinline__ float dot3(float3 a, float3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }

// FP32 -> FP64 widening by integer operations (exact for normal numbers: the exponent is
// rebiased by 1023 - 127 and the 23 fraction bits move up by 29), so that the deposit atomics
// of the walk do not occupy the FP64 pipe; zero, subnormals, infinities and NaN take the
// ordinary conversion.
__device__ __forceinline__ double widen(float v) {
    const uint32_t b = __float_as_uint(v);
    const uint32_t e = (b >> 23) & 0xFFu;
    if (e - 1u >= 254u) return (double)v;
    const unsigned long long bits = ((unsigned long long)(b >> 31) << 63) |
                                    ((unsigned long long)(e + 896u) << 52) |
                                    ((unsigned long long)(b & 0x7FFFFFu) << 29);
    return __longlong_as_double((long long)bits);
}

}  // namespace hrt
