// Modified random walk (Sect. 2.2; the published diffusion form the paper refers to): geometry
// and path length of one step, FP32.
//
// Deep inside a cell of large optical depth a packet crosses a sphere of radius R0 centred on
// it, inside the cell, in one step.  Diffusion with coefficient D = 1 / (3 rho chi_t) per unit
// path length (chi_t the Rosseland mean of the transport extinction chi_nu (1 - albedo g))
// from the centre of a sphere with an absorbing surface leaves the packet inside after path
// length s with probability
//   P(s) = 2 sum_{n>=1} (-1)^{n+1} exp(-n^2 x),   x = pi^2 D s / R0^2 = pi^2 s / (3 tau0 R0),
// tau0 = rho chi_t R0.  The step's path length solves P(s) = zeta.
#pragma once
#include <math_constants.h>

#include "device_grid.cuh"

namespace hrt {

constexpr float MRW_SHRINK = 0.99f;    // sphere radius / distance to the nearest wall

// Distance from a point at (a, b) in a plane through the z axis (or a point at azimuth) to a
// wall through the origin whose unit direction in that plane is (c_w, s_w): the perpendicular
// distance |a s_w - b c_w| while the wall's ray is within a quarter turn of the point, else the
// distance to the wall's edge (the origin), the point's own distance h.
__device__ __forceinline__ float ray_wall_distance(float a, float b, float c_w, float s_w, float h) {
    return fmaf(a, c_w, b * s_w) > 0.f ? fabsf(fmaf(a, s_w, -b * c_w)) : h;
}

// Distance from the packet's position to the nearest wall bounding its cell: planes of a
// Cartesian cell; spheres, cones and half-planes of a spherical-polar cell; cylinders, planes and
// half-planes of a cylindrical cell.  The polar axis, r = 0 and R = 0 bound nothing (the cell
// continues through them), nor do the phi walls of a grid with one phi cell.
template <int G>
__device__ __forceinline__ float wall_distance(const DevGrid& g, const Ray& r) {
    if constexpr (G == GRID_CARTESIAN) {
        float d = fminf(r.p.x - __ldg(g.w1 + r.i), __ldg(g.w1 + r.i + 1) - r.p.x);
        d = fminf(d, fminf(r.p.y - __ldg(g.w2 + r.j), __ldg(g.w2 + r.j + 1) - r.p.y));
        return fminf(d, fminf(r.p.z - __ldg(g.w3 + r.k), __ldg(g.w3 + r.k + 1) - r.p.z));
    } else {
        const float R = sqrtf(fmaf(r.p.x, r.p.x, r.p.y * r.p.y));
        float d = F_INF;
        if (g.n3 > 1) {
            // half-plane phi_w: (x, y) against the direction (cos phi_w, sin phi_w)
            d = ray_wall_distance(r.p.x, r.p.y, __ldg(g.cph + r.k), __ldg(g.sph + r.k), R);
            d = fminf(d, ray_wall_distance(r.p.x, r.p.y, __ldg(g.cph + r.k + 1), __ldg(g.sph + r.k + 1), R));
        }
        const float lo = __ldg(g.rw + r.i), hi = __ldg(g.rw + r.i + 1);
        if constexpr (G == GRID_SPHERICAL) {
            const float rad = sqrtf(dot3(r.p, r.p));
            if (lo > 0.f) d = fminf(d, rad - lo);
            d = fminf(d, hi - rad);
            // cone theta_w: (z, R) against the direction (cos theta_w, sin theta_w)
            if (!(r.j == 0 && (g.poles & 1)))
                d = fminf(d, ray_wall_distance(r.p.z, R, __ldg(g.cth + r.j), __ldg(g.sth + r.j), rad));
            if (!(r.j == g.n2 - 1 && (g.poles & 2)))
                d = fminf(d, ray_wall_distance(r.p.z, R, __ldg(g.cth + r.j + 1), __ldg(g.sth + r.j + 1), rad));
        } else {
            if (lo > 0.f) d = fminf(d, R - lo);
            d = fminf(d, hi - R);
            d = fminf(d, fminf(r.p.z - __ldg(g.w2 + r.j), __ldg(g.w2 + r.j + 1) - r.p.z));
        }
        return fmaxf(d, 0.f);
    }
}

// s / R0 with P(s) = zeta, zeta in (0, 1] (0 for zeta = 1), by Newton's method on the log of a
// form of P that converges in a few terms: for x >= ~1 (zeta <= 0.69) the series itself, in
// q = exp(-x); for smaller x Jacobi's transformation
//   1 - P = 2 sqrt(pi / x) sum_{k>=0} exp(-pi^2 (2k + 1)^2 / (4 x)),
// solved for w = 1 / x against 1 - zeta (exact in FP32 for the library's uniforms).
__device__ __forceinline__ float mrw_path(float tau0, float zeta) {
    constexpr float PI2 = CUDART_PI_F * CUDART_PI_F;
    if (!(zeta < 1.f)) return 0.f;
    float x;
    if (zeta <= 0.69f) {
        const float lz = logf(zeta);
        x = logf(2.f / zeta);                    // the first term alone
        for (int it = 0; it < 2; ++it) {      // quadratic convergence from within e^-3x: 2 suffice in FP32
            const float q = expf(-x), q2 = q * q, q3 = q2 * q, q8 = q2 * q2 * q2 * q2;
            const float q15 = q8 * q3 * q3 * q;
            const float S = q * (1.f - q3 + q8 - q15);                // P / 2
            const float dS = -q * (1.f - 4.f * q3 + 9.f * q8 - 16.f * q15);
            x -= (logf(2.f * S) - lz) / (dS / S);
        }
    } else {
        const float l1 = logf(1.f - zeta);
        const float c0 = logf(2.f * sqrtf(CUDART_PI_F));
        float w = fmaxf((c0 - l1) / (0.25f * PI2), 1.f);
        for (int it = 0; it < 3; ++it) {
            const float e = expf(-2.f * PI2 * w);
            const float f = c0 + 0.5f * logf(w) - 0.25f * PI2 * w + log1pf(e) - l1;
            const float df = 0.5f / w - 0.25f * PI2 - 2.f * PI2 * e / (1.f + e);
            w -= f / df;
        }
        x = 1.f / w;
    }
    return 3.f * tau0 * x / PI2;
}

}  // namespace hrt
