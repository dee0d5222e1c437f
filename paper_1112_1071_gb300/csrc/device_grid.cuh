// Cell walks on Cartesian and spherical-polar grids (Sect. 2.1.2, Sect. 2.2).
//
// A Ray carries a position, a unit direction and the integer cell index per axis.  The wall a
// ray leaves through is always found from the integer index and the wall tables, never from
// an accumulated coordinate, and the crossed coordinate is reset onto that wall after every
// crossing (Cartesian: the coordinate itself; spherical: the radius), so rounding does not
// accumulate from cell to cell.
//
// Spherical walls are spheres r_i, cones theta_j (z sin(theta) = R cos(theta), R the
// cylindrical radius; theta = pi/2 is the plane z = 0) and half-planes phi_k.  A root of a
// wall is admissible only when the ray leaves the cell through it (r increasing through the
// outer sphere, decreasing through the inner one; theta decreasing through the lower cone,
// increasing through the upper; phi likewise), which makes the walk robust for packets sitting
// on a wall.  The precision policy of the wall solves is stated with them below.
#pragma once
#include "device_common.cuh"

namespace hrt {

constexpr float F_INF = __builtin_huge_valf();

struct Ray {
    float3 p;
    float3 u;
    float3 inv;          // 1/u per axis (Cartesian), 0 where u = 0
    int32_t i, j, k;     // per-axis cell index
    int32_t ci;          // linear cell index (k n2 + j) n1 + i
};

enum WalkEvent : int32_t { EV_INTERACT = 0, EV_ESCAPE = 1, EV_ABORT = 2, EV_STUCK = 3 };

__device__ __forceinline__ void set_dir(Ray& r, float3 u) {
    r.u = u;
    r.inv = make_float3(u.x != 0.f ? 1.f / u.x : 0.f, u.y != 0.f ? 1.f / u.y : 0.f, u.z != 0.f ? 1.f / u.z : 0.f);
}

__device__ __forceinline__ int32_t lin(const DevGrid& g, int i, int j, int k) { return (k * g.n2 + j) * g.n1 + i; }

// Cell along one axis holding v; on a wall, the cell the motion points into (dv > 0: upper).
__device__ __forceinline__ int locate_axis(const float* __restrict__ w, int n, float v, float dv) {
    if (v < __ldg(w) || v > __ldg(w + n)) return -1;
    int lo = 0, hi = n;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(w + mid) <= v) lo = mid; else hi = mid;
    }
    int i = lo;
    if (hi == n && v == __ldg(w + n)) i = n;
    if (v == __ldg(w + i) && !(dv > 0.f)) i -= 1;
    return (i < 0 || i >= n) ? -1 : i;
}

// ================================================================ Cartesian
__device__ __forceinline__ float cart_exit(const DevGrid& g, const Ray& r, int& axis) {
    float dx = F_INF, dy = F_INF, dz = F_INF;
    if (r.u.x != 0.f) dx = fmaxf((__ldg(g.w1 + r.i + (r.u.x > 0.f)) - r.p.x) * r.inv.x, 0.f);
    if (r.u.y != 0.f) dy = fmaxf((__ldg(g.w2 + r.j + (r.u.y > 0.f)) - r.p.y) * r.inv.y, 0.f);
    if (r.u.z != 0.f) dz = fmaxf((__ldg(g.w3 + r.k + (r.u.z > 0.f)) - r.p.z) * r.inv.z, 0.f);
    // ties go to the lowest axis
    if (dx <= dy && dx <= dz) { axis = 0; return dx; }
    if (dy <= dz) { axis = 1; return dy; }
    axis = 2;
    return dz;
}

// Advance to the wall on `axis` and into the next cell; true when the ray leaves the grid.
__device__ __forceinline__ bool cart_step(const DevGrid& g, Ray& r, float l, int axis) {
    r.p.x += l * r.u.x;
    r.p.y += l * r.u.y;
    r.p.z += l * r.u.z;
    if (axis == 0) {
        const int up = r.u.x > 0.f;
        r.p.x = __ldg(g.w1 + r.i + up);
        r.i += up ? 1 : -1;
        r.ci += up ? 1 : -1;
        return r.i < 0 || r.i >= g.n1;
    } else if (axis == 1) {
        const int up = r.u.y > 0.f;
        r.p.y = __ldg(g.w2 + r.j + up);
        r.j += up ? 1 : -1;
        r.ci += up ? g.n1 : -g.n1;
        return r.j < 0 || r.j >= g.n2;
    } else {
        const int up = r.u.z > 0.f;
        r.p.z = __ldg(g.w3 + r.k + up);
        r.k += up ? 1 : -1;
        r.ci += up ? g.n1 * g.n2 : -g.n1 * g.n2;
        return r.k < 0 || r.k >= g.n3;
    }
}

// The same walk with the next wall of every axis (the wall the ray moves towards) held by the
// caller in wn: cart_next_walls loads them when a ray starts, cart_exit_w equals cart_exit, and
// cart_step_w equals cart_step without branching on the crossed axis, loading only that axis's
// next wall -- one table load per crossing instead of four, the same FP32 operations.
__device__ __forceinline__ float3 cart_next_walls(const DevGrid& g, const Ray& r) {
    return make_float3(__ldg(g.w1 + r.i + (r.u.x > 0.f)), __ldg(g.w2 + r.j + (r.u.y > 0.f)),
                       __ldg(g.w3 + r.k + (r.u.z > 0.f)));
}

__device__ __forceinline__ float cart_exit_w(const Ray& r, float3 wn, int& axis) {
    const float dx = r.u.x != 0.f ? fmaxf((wn.x - r.p.x) * r.inv.x, 0.f) : F_INF;
    const float dy = r.u.y != 0.f ? fmaxf((wn.y - r.p.y) * r.inv.y, 0.f) : F_INF;
    const float dz = r.u.z != 0.f ? fmaxf((wn.z - r.p.z) * r.inv.z, 0.f) : F_INF;
    // ties go to the lowest axis
    const bool bx = dx <= dy && dx <= dz;
    const bool by = !bx && dy <= dz;
    axis = bx ? 0 : (by ? 1 : 2);
    return bx ? dx : (by ? dy : dz);
}

__device__ __forceinline__ bool cart_step_w(const DevGrid& g, Ray& r, float3& wn, float l, int axis) {
    const bool ax = axis == 0, ay = axis == 1;
    const bool az = !ax && !ay;
    r.p.x = ax ? wn.x : r.p.x + l * r.u.x;
    r.p.y = ay ? wn.y : r.p.y + l * r.u.y;
    r.p.z = az ? wn.z : r.p.z + l * r.u.z;
    const float ua = ax ? r.u.x : (ay ? r.u.y : r.u.z);
    const int up = ua > 0.f;
    const int s = up ? 1 : -1;
    r.i += ax ? s : 0;
    r.j += ay ? s : 0;
    r.k += az ? s : 0;
    r.ci += ax ? s : (ay ? s * g.n1 : s * g.n1 * g.n2);
    const bool out = (unsigned)r.i >= (unsigned)g.n1 || (unsigned)r.j >= (unsigned)g.n2 || (unsigned)r.k >= (unsigned)g.n3;
    if (!out) {
        const float* w = ax ? g.w1 : (ay ? g.w2 : g.w3);
        const float v = __ldg(w + (ax ? r.i : (ay ? r.j : r.k)) + up);
        wn.x = ax ? v : wn.x;
        wn.y = ay ? v : wn.y;
        wn.z = az ? v : wn.z;
    }
    return out;
}

__device__ __forceinline__ bool cart_locate(const DevGrid& g, Ray& r) {
    r.i = locate_axis(g.w1, g.n1, r.p.x, r.u.x);
    r.j = locate_axis(g.w2, g.n2, r.p.y, r.u.y);
    r.k = locate_axis(g.w3, g.n3, r.p.z, r.u.z);
    if (r.i < 0 || r.j < 0 || r.k < 0) return false;
    r.ci = lin(g, r.i, r.j, r.k);
    return true;
}

// ================================================================ spherical-polar
// Precision of the wall solves.  Positions and directions are FP32; the distance returned is
// FP32.  What FP32 arithmetic loses is the cancellation in the quadratic's terms when they
// nearly vanish: |p|^2 - r_w^2 for a point close to a sphere, and the discriminant for a ray
// nearly tangent to a sphere or a cone (the root error grows as the rounding of those terms
// divided by the root separation).  So:
//   * |p|^2 - r_w^2 is formed in FP32 with the rounding errors of the squares and sums carried
//     (error-free transformations) against r_w^2 held as an FP32 pair: ~2^-44 |p|^2 instead of
//     2^-23 |p|^2, at the cost of ~20 FP32 operations and no FP64;
//   * the coefficients and discriminant are formed in FP64 (products of FP32 numbers are exact
//     in FP64, so only their sums round) for spheres below r_fp64 and cones with sin(theta)
//     below sin_fp64 (small r and the polar axis), and for the inner sphere or a cone whose FP32
//     discriminant is within 2^-10 of a double root (a grazing ray; for a cone, only when that
//     root can be the exit).  The square root, divisions and root selection then run in FP32 on
//     the accurately rounded coefficients.

// s = a + b exactly as s + e (Knuth); __fadd_rn keeps the compiler from fusing or reordering.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// |p|^2 - (w_hi + w_lo) with the FP32 rounding errors of the squares (fma) and sums carried.
__device__ __forceinline__ float sphere_c(float3 p, float w_hi, float w_lo) {
    const float x2 = __fmul_rn(p.x, p.x), y2 = __fmul_rn(p.y, p.y), z2 = __fmul_rn(p.z, p.z);
    const float ex = fmaf(p.x, p.x, -x2), ey = fmaf(p.y, p.y, -y2), ez = fmaf(p.z, p.z, -z2);
    float s1, e1, s2, e2, s3, e3;
    two_sum(x2, y2, s1, e1);
    two_sum(s1, z2, s2, e2);
    two_sum(s2, -w_hi, s3, e3);
    return __fadd_rn(s3, __fadd_rn(__fadd_rn(__fadd_rn(e1, e2), e3),
                                   __fadd_rn(__fadd_rn(ex, ey), __fsub_rn(ez, w_lo))));
}

// Roots of s^2 + 2 b s + c = 0 given disc = b^2 - c.
// Outer sphere: the far root (always ahead of a point inside), without cancellation:
// -c / (b + sq) when moving outwards, -b + sq otherwise.
__device__ __forceinline__ float sphere_out_root(float b, float c, float disc) {
    const float sq = sqrtf(fmaxf(disc, 0.f));
    const float s = b > 0.f ? -c / (b + sq) : -b + sq;
    return fmaxf(s, 0.f);
}
// Inner sphere: the near root, only while moving inwards (b < 0).
__device__ __forceinline__ float sphere_in_root(float b, float c, float disc) {
    if (disc < 0.f) return F_INF;
    return fmaxf(c / (-b + sqrtf(disc)), 0.f);
}

// FP64 p.u and |p|^2 from FP32 inputs.
struct SphQ64 { double b, rr; };
__device__ __forceinline__ SphQ64 sphere_terms64(const Ray& r) {
    const double px = r.p.x, py = r.p.y, pz = r.p.z;
    SphQ64 q;
    q.rr = fma(px, px, fma(py, py, pz * pz));
    q.b = fma(px, (double)r.u.x, fma(py, (double)r.u.y, pz * (double)r.u.z));
    return q;
}

// Cone coefficients: the ray meets z sin(w) = R cos(w) (both nappes) where
// A s^2 + 2 B s + C = 0; disc = B^2 - A C.
struct ConeQ { float A, B, C, disc; };

// FP32: uR2 = u_x^2 + u_y^2, pu = p_x u_x + p_y u_y and Rp = |p_R| are shared by both cones;
// C = f (p_z sin + Rp cos) with f = p_z sin - Rp cos = r sin(theta_w - theta) formed directly.
__device__ __forceinline__ ConeQ cone_coeffs32(const Ray& r, float uR2, float pu, float Rp, float cw, float sw) {
    const float sw2 = sw * sw, cw2 = cw * cw;
    ConeQ q;
    q.A = r.u.z * r.u.z * sw2 - uR2 * cw2;
    q.B = r.p.z * r.u.z * sw2 - pu * cw2;
    const float f = r.p.z * sw - Rp * cw;
    q.C = f * (r.p.z * sw + Rp * cw);
    q.disc = q.B * q.B - q.A * q.C;
    return q;
}

// FP64 coefficients from the FP32 ray (exact products, rounded sums), rounded to FP32.  Out of
// line with scalar arguments: the call is rare, and an inlined FP64 block would be scheduled
// (and its operands converted) on the common path.
static __device__ __noinline__ ConeQ cone_coeffs64(float px_, float py_, float pz_, float ux_, float uy_, float uz_,
                                                  double cw, double sw) {
    const double px = px_, py = py_, pz = pz_, ux = ux_, uy = uy_, uz = uz_;
    const double sw2 = sw * sw, cw2 = cw * cw;
    const double uR2 = fma(ux, ux, uy * uy), pu = fma(px, ux, py * uy), R2 = fma(px, px, py * py);
    const double A = fma(uz * uz, sw2, -uR2 * cw2);
    const double B = fma(pz * uz, sw2, -pu * cw2);
    const double C = fma(pz * pz, sw2, -R2 * cw2);
    ConeQ q;
    q.A = (float)A; q.B = (float)B; q.C = (float)C;
    q.disc = (float)fma(B, B, -A * C);
    return q;
}

// The smallest root >= -tol on the cone's own nappe through which the ray leaves the cell in
// the given sense (+1: theta decreasing, f increasing), or +inf.
__device__ __forceinline__ float cone_pick(const ConeQ& q, const Ray& r, float cw, float sw, int sense, float tol) {
    if (q.disc < 0.f) return F_INF;
    const float sq = sqrtf(q.disc);
    const float qq = -(q.B + copysignf(sq, q.B));
    float roots[2];
    roots[0] = (q.A != 0.f) ? qq / q.A : F_INF;
    roots[1] = (qq != 0.f) ? q.C / qq : F_INF;
    float best = F_INF;
#pragma unroll
    for (int t = 0; t < 2; ++t) {
        const float s = roots[t];
        if (!(s >= -tol) || !(s < best)) continue;
        const float qz = r.p.z + s * r.u.z;
        if (!(qz * cw > 0.f)) continue;        // other nappe
        const float qx = r.p.x + s * r.u.x, qy = r.p.y + s * r.u.y;
        const float Rq2 = qx * qx + qy * qy;
        if (Rq2 == 0.f) continue;
        // sign of df/ds = u_z sin - cos (q_R . u_R) / |q_R|, scaled by |q_R| > 0 (no division)
        const float dfds = r.u.z * sw * sqrtf(Rq2) - cw * (qx * r.u.x + qy * r.u.y);
        if (sense > 0 ? !(dfds > 0.f) : !(dfds < 0.f)) continue;
        best = fmaxf(s, 0.f);
    }
    return best;
}

__device__ __forceinline__ float phi_root(const Ray& r, float cw, float sw, int sense, float tol) {
    const float nx = -sw, ny = cw;
    const float nu = nx * r.u.x + ny * r.u.y;
    if (nu == 0.f || ((sense > 0) != (nu > 0.f))) return F_INF;
    const float s = -(nx * r.p.x + ny * r.p.y) / nu;
    if (!(s >= -tol)) return F_INF;
    const float qx = r.p.x + s * r.u.x, qy = r.p.y + s * r.u.y;
    if (!(cw * qx + sw * qy > 0.f)) return F_INF;
    return fmaxf(s, 0.f);
}

// Exit through cone wall jw in the given sense (the midplane wall is the plane z = 0); `best`
// is the nearest exit found so far.
__device__ __forceinline__ float cone_wall(const DevGrid& g, const Ray& r, int jw, int sense, float uR2, float pu,
                                          float Rp, float tol, float best) {
    const float cw = __ldg(g.cth + jw), sw = __ldg(g.sth + jw);
    if (cw == 0.f) {           // f = z increases when u_z > 0
        if (r.u.z == 0.f || ((sense > 0) != (r.u.z > 0.f))) return F_INF;
        const float s = -r.p.z / r.u.z;
        return s < -tol ? F_INF : fmaxf(s, 0.f);
    }
    ConeQ q;
    bool fp64 = sw < g.sin_fp64;
    if (!fp64) {
        q = cone_coeffs32(r, uR2, pu, Rp, cw, sw);
        // Grazing: both roots lie within 3.2% of s_c = -B/A (|disc| < 2^-10 B^2 plus its FP32
        // rounding error ~2^-21 B^2 leave sqrt(|disc|) < 0.032 |B|), so the root nearest zero is
        // no closer than 0.96 s_c.  The FP64 redo is needed only where a root can be the exit,
        // not behind the ray and not beyond `best`: a ray running along a cone far from its
        // tangent point stays "grazing" for many steps while that cone is never its exit.
        if (fabsf(q.disc) < 0x1p-10f * q.B * q.B) {
            const float s0 = 0.96f * (-q.B / q.A);
            fp64 = s0 >= -tol && s0 < best;
        }
    }
    if (fp64) q = cone_coeffs64(r.p.x, r.p.y, r.p.z, r.u.x, r.u.y, r.u.z, __ldg(g.cthd + jw), __ldg(g.sthd + jw));
    return cone_pick(q, r, cw, sw, sense, tol);
}

// Distance to the exit of the current cell; axis 0/1/2 = r/theta/phi, dir = +-1.
__device__ __forceinline__ float sph_exit(const DevGrid& g, const Ray& r, int& axis, int& dir) {
    const float rr = dot3(r.p, r.p);
    const float b = dot3(r.p, r.u);
    const float tol = 2e-6f * sqrtf(rr) + 1e-30f;
    // A ray enters the inner sphere only when clearly moving inwards: a ray tangent to the
    // sphere touches it at one point, and FP32 rounding of p.u around zero must not make it
    // cross back and forth there.
    const float b_in = -1e-6f * sqrtf(rr);
    const bool inward = b < b_in && __ldg(g.rw + r.i) > 0.f;
    float best;
    axis = 0; dir = 1;
    if (__ldg(g.rw + r.i + 1) < g.r_fp64) {
        const SphQ64 t = sphere_terms64(r);
        const double ro = __ldg(g.rwd + r.i + 1);
        const double co = fma(-ro, ro, t.rr);
        const float bf = (float)t.b;
        best = sphere_out_root(bf, (float)co, (float)fma(t.b, t.b, -co));
        if (inward) {
            const double ri = __ldg(g.rwd + r.i);
            const double ci = fma(-ri, ri, t.rr);
            const float s = sphere_in_root(bf, (float)ci, (float)fma(t.b, t.b, -ci));
            if (s < best) { best = s; dir = -1; }
        }
    } else {
        const float co = sphere_c(r.p, __ldg(g.r2w + r.i + 1), __ldg(g.r2wl + r.i + 1));
        best = sphere_out_root(b, co, fmaf(b, b, -co));
        if (inward) {
            const float ci = sphere_c(r.p, __ldg(g.r2w + r.i), __ldg(g.r2wl + r.i));
            float disc = fmaf(b, b, -ci);
            float bb = b;
            if (fabsf(disc) < 0x1p-10f * b * b) {           // grazing the inner sphere
                const SphQ64 t = sphere_terms64(r);
                const double ri = __ldg(g.rwd + r.i);
                const double ci64 = fma(-ri, ri, t.rr);
                disc = (float)fma(t.b, t.b, -ci64);
                bb = (float)t.b;
            }
            const float s = sphere_in_root(bb, ci, disc);
            if (s < best) { best = s; dir = -1; }
        }
    }
    // terms shared by both cones of the cell
    const float uR2 = r.u.x * r.u.x + r.u.y * r.u.y;
    const float pu = r.p.x * r.u.x + r.p.y * r.u.y;
    const float Rp = sqrtf(r.p.x * r.p.x + r.p.y * r.p.y);
    // lower wall j is left with theta decreasing (sense +1), upper wall j + 1 increasing (-1)
    if (r.j > 0) {
        const float s = cone_wall(g, r, r.j, +1, uR2, pu, Rp, tol, best);
        if (s < best) { best = s; axis = 1; dir = -1; }
    }
    if (r.j + 1 < g.n2) {
        const float s = cone_wall(g, r, r.j + 1, -1, uR2, pu, Rp, tol, best);
        if (s < best) { best = s; axis = 1; dir = 1; }
    }
    if (g.n3 > 1) {
        float s = phi_root(r, __ldg(g.cph + r.k), __ldg(g.sph + r.k), -1, tol);
        if (s < best) { best = s; axis = 2; dir = -1; }
        s = phi_root(r, __ldg(g.cph + r.k + 1), __ldg(g.sph + r.k + 1), +1, tol);
        if (s < best) { best = s; axis = 2; dir = 1; }
    }
    return best;
}

__device__ __forceinline__ float wrap_2pi(float a) {
    const float twopi = 2.f * CUDART_PI_F;
    if (a < 0.f) a += twopi;
    if (a >= twopi) a -= twopi;
    return a;
}

// theta and phi cells of a point (direction breaks ties on walls)
__device__ __forceinline__ void sph_angles(const DevGrid& g, Ray& r) {
    const float rr = dot3(r.p, r.p);
    const float rad = sqrtf(rr);
    float th, vt, ph, vp;
    if (rad == 0.f) {
        th = acosf(fminf(1.f, fmaxf(-1.f, r.u.z)));
        vt = 0.f;
        ph = wrap_2pi(atan2f(r.u.y, r.u.x));
        vp = 0.f;
    } else {
        th = acosf(fminf(1.f, fmaxf(-1.f, r.p.z / rad)));
        vt = -(r.u.z * rr - r.p.z * dot3(r.p, r.u));
        const float Rc = r.p.x * r.p.x + r.p.y * r.p.y;
        if (Rc == 0.f) { ph = wrap_2pi(atan2f(r.u.y, r.u.x)); vp = 0.f; }
        else { ph = wrap_2pi(atan2f(r.p.y, r.p.x)); vp = r.p.x * r.u.y - r.p.y * r.u.x; }
    }
    int j = locate_axis(g.thw, g.n2, th, vt);
    if (j < 0) j = (th <= __ldg(g.thw)) ? 0 : g.n2 - 1;
    r.j = j;
    int k = 0;
    if (g.n3 > 1) {
        if (ph == 0.f && !(vp > 0.f)) k = g.n3 - 1;
        else {
            k = locate_axis(g.phw, g.n3, ph, vp);
            if (k < 0) k = g.n3 - 1;
        }
    }
    r.k = k;
}

// Cross the inner vacuum hole from a point on or inside the sphere r_0 to its far side.
__device__ __forceinline__ void sph_cross_hole(const DevGrid& g, Ray& r) {
    const double pd[3] = {r.p.x, r.p.y, r.p.z}, ud[3] = {r.u.x, r.u.y, r.u.z};
    const double b = pd[0] * ud[0] + pd[1] * ud[1] + pd[2] * ud[2];
    const double r0 = __ldg(g.rwd);
    const double c = pd[0] * pd[0] + pd[1] * pd[1] + pd[2] * pd[2] - r0 * r0;
    double disc = b * b - c;
    double s = -b + sqrt(disc > 0.0 ? disc : 0.0);
    if (s < 0.0) s = 0.0;
    r.p = make_float3((float)(pd[0] + s * ud[0]), (float)(pd[1] + s * ud[1]), (float)(pd[2] + s * ud[2]));
    r.i = 0;
    sph_angles(g, r);
    r.ci = lin(g, r.i, r.j, r.k);
}

__device__ __forceinline__ bool sph_step(const DevGrid& g, Ray& r, float l, int axis, int dir) {
    r.p.x += l * r.u.x;
    r.p.y += l * r.u.y;
    r.p.z += l * r.u.z;
    if (axis == 0) {
        r.i += dir;
        if (r.i >= g.n1) return true;
        if (r.i < 0) {
            sph_cross_hole(g, r);
            return false;
        }
        // put the point back on the sphere it crossed
        const float rw = __ldg(g.rw + r.i + (dir < 0 ? 1 : 0));
        const float sc = rw * rsqrtf(dot3(r.p, r.p));
        r.p.x *= sc; r.p.y *= sc; r.p.z *= sc;
        r.ci += dir;
        return false;
    }
    if (axis == 1) {
        r.j += dir;
        r.ci += dir * g.n1;
        return false;
    }
    r.k += dir;
    if (r.k < 0) r.k += g.n3;
    if (r.k >= g.n3) r.k -= g.n3;
    r.ci = lin(g, r.i, r.j, r.k);
    return false;
}

__device__ __forceinline__ bool sph_locate(const DevGrid& g, Ray& r) {
    const float rr = dot3(r.p, r.p);
    const float rad = sqrtf(rr);
    const float vr = dot3(r.p, r.u);
    const float r0 = __ldg(g.rw);
    const bool in_hole = (rad == 0.f && r0 > 0.f) || rad < r0 || (rad == r0 && r0 > 0.f && !(vr > 0.f));
    if (in_hole) {
        sph_cross_hole(g, r);
        return true;
    }
    if (rad == 0.f) r.i = 0;
    else {
        r.i = locate_axis(g.rw, g.n1, rad, vr);
        if (r.i < 0) return false;
    }
    sph_angles(g, r);
    r.ci = lin(g, r.i, r.j, r.k);
    return true;
}

// ================================================================ cylindrical-polar (R, z, phi)
// Walls: cylinders R_i about the z axis, planes z_j (the w2 table) and half-planes phi_k; an
// inner vacuum cylinder when R_0 > 0.  A cylinder's quadratic a s^2 + 2 b s + c = 0 has
// a = u_x^2 + u_y^2, b = p_R . u_R and c = |p_R|^2 - R_w^2; c is formed with the rounding errors
// carried as for spheres, and a ray grazing the inner cylinder redoes its discriminant in FP64.

__device__ __forceinline__ float cyl_c(float px, float py, float w_hi, float w_lo) {
    const float x2 = __fmul_rn(px, px), y2 = __fmul_rn(py, py);
    const float ex = fmaf(px, px, -x2), ey = fmaf(py, py, -y2);
    float s1, e1, s2, e2;
    two_sum(x2, y2, s1, e1);
    two_sum(s1, -w_hi, s2, e2);
    return __fadd_rn(s2, __fadd_rn(__fadd_rn(e1, e2), __fsub_rn(__fadd_rn(ex, ey), w_lo)));
}

__device__ __forceinline__ float cyl_exit(const DevGrid& g, const Ray& r, int& axis, int& dir) {
    const float a = r.u.x * r.u.x + r.u.y * r.u.y;
    const float b = r.p.x * r.u.x + r.p.y * r.u.y;
    const float R2 = r.p.x * r.p.x + r.p.y * r.p.y;
    const float tol = 2e-6f * sqrtf(R2 + r.p.z * r.p.z) + 1e-30f;
    float best = F_INF;
    axis = -1;
    dir = 0;
    if (a > 0.f) {
        // outer cylinder: the far root, always ahead of a point inside
        const float co = cyl_c(r.p.x, r.p.y, __ldg(g.r2w + r.i + 1), __ldg(g.r2wl + r.i + 1));
        const float sq = sqrtf(fmaxf(fmaf(b, b, -a * co), 0.f));
        const float s = b > 0.f ? -co / (b + sq) : (-b + sq) / a;
        best = fmaxf(s, 0.f);
        axis = 0;
        dir = 1;
        // inner cylinder, entered only while clearly moving inwards (as for the inner sphere)
        if (b < -1e-6f * sqrtf(R2 * a) && __ldg(g.rw + r.i) > 0.f) {
            const float ci = cyl_c(r.p.x, r.p.y, __ldg(g.r2w + r.i), __ldg(g.r2wl + r.i));
            float disc = fmaf(b, b, -a * ci);
            float bb = b;
            if (fabsf(disc) < 0x1p-10f * b * b) {           // grazing the inner cylinder
                const double px = r.p.x, py = r.p.y, ux = r.u.x, uy = r.u.y;
                const double ad = fma(ux, ux, uy * uy), bd = fma(px, ux, py * uy);
                const double ri = __ldg(g.rwd + r.i);
                const double cd = fma(px, px, fma(py, py, -ri * ri));
                disc = (float)fma(bd, bd, -ad * cd);
                bb = (float)bd;
            }
            if (disc >= 0.f) {
                const float si = fmaxf(ci / (-bb + sqrtf(disc)), 0.f);
                if (si < best) { best = si; dir = -1; }
            }
        }
    }
    if (r.u.z != 0.f) {
        const float zw = r.u.z > 0.f ? __ldg(g.w2 + r.j + 1) : __ldg(g.w2 + r.j);
        const float s = fmaxf((zw - r.p.z) * r.inv.z, 0.f);
        if (s < best) { best = s; axis = 1; dir = r.u.z > 0.f ? 1 : -1; }
    }
    if (g.n3 > 1) {
        float s = phi_root(r, __ldg(g.cph + r.k), __ldg(g.sph + r.k), -1, tol);
        if (s < best) { best = s; axis = 2; dir = -1; }
        s = phi_root(r, __ldg(g.cph + r.k + 1), __ldg(g.sph + r.k + 1), +1, tol);
        if (s < best) { best = s; axis = 2; dir = 1; }
    }
    return best;
}

// Azimuthal cell of a point (direction breaks ties on walls; on the axis, the direction's phi).
__device__ __forceinline__ int phi_cell(const DevGrid& g, const Ray& r) {
    if (g.n3 <= 1) return 0;
    float ph, vp;
    if (r.p.x * r.p.x + r.p.y * r.p.y == 0.f) { ph = wrap_2pi(atan2f(r.u.y, r.u.x)); vp = 0.f; }
    else { ph = wrap_2pi(atan2f(r.p.y, r.p.x)); vp = r.p.x * r.u.y - r.p.y * r.u.x; }
    if (ph == 0.f && !(vp > 0.f)) return g.n3 - 1;
    const int k = locate_axis(g.phw, g.n3, ph, vp);
    return k < 0 ? g.n3 - 1 : k;
}

// Cross the inner vacuum cylinder to its far side (FP64); true when the ray leaves the grid on
// the way (through a z plane, or running along the axis).
__device__ __forceinline__ bool cyl_cross_hole(const DevGrid& g, Ray& r) {
    const double px = r.p.x, py = r.p.y, ux = r.u.x, uy = r.u.y;
    const double a = fma(ux, ux, uy * uy);
    if (!(a > 0.0)) return true;
    const double R0 = __ldg(g.rwd);
    const double b = fma(px, ux, py * uy);
    const double c = fma(px, px, fma(py, py, -R0 * R0));
    const double sq = sqrt(fmax(fma(b, b, -a * c), 0.0));
    double s = b > 0.0 ? -c / (b + sq) : (-b + sq) / a;
    if (s < 0.0) s = 0.0;
    r.p = make_float3((float)(px + s * ux), (float)(py + s * uy), (float)((double)r.p.z + s * (double)r.u.z));
    const int j = locate_axis(g.w2, g.n2, r.p.z, r.u.z);
    if (j < 0) return true;
    r.i = 0;
    r.j = j;
    r.k = phi_cell(g, r);
    r.ci = lin(g, r.i, r.j, r.k);
    return false;
}

__device__ __forceinline__ bool cyl_step(const DevGrid& g, Ray& r, float l, int axis, int dir) {
    r.p.x += l * r.u.x;
    r.p.y += l * r.u.y;
    r.p.z += l * r.u.z;
    if (axis == 0) {
        r.i += dir;
        if (r.i >= g.n1) return true;
        if (r.i < 0) return cyl_cross_hole(g, r);
        // put the point back on the cylinder it crossed
        const float Rw = __ldg(g.rw + r.i + (dir < 0 ? 1 : 0));
        const float sc = Rw * rsqrtf(r.p.x * r.p.x + r.p.y * r.p.y);
        r.p.x *= sc;
        r.p.y *= sc;
        r.ci += dir;
        return false;
    }
    if (axis == 1) {
        r.j += dir;
        if (r.j < 0 || r.j >= g.n2) return true;
        r.p.z = __ldg(g.w2 + r.j + (dir < 0 ? 1 : 0));
        r.ci += dir * g.n1;
        return false;
    }
    r.k += dir;
    if (r.k < 0) r.k += g.n3;
    if (r.k >= g.n3) r.k -= g.n3;
    r.ci = lin(g, r.i, r.j, r.k);
    return false;
}

__device__ __forceinline__ bool cyl_locate(const DevGrid& g, Ray& r) {
    const int j = locate_axis(g.w2, g.n2, r.p.z, r.u.z);
    if (j < 0) return false;
    const float R = sqrtf(r.p.x * r.p.x + r.p.y * r.p.y);
    const float vR = r.p.x * r.u.x + r.p.y * r.u.y;
    const float R0 = __ldg(g.rw);
    if (R0 > 0.f && (R < R0 || (R == R0 && !(vR > 0.f)))) return !cyl_cross_hole(g, r);
    // without a hole the axis R = 0 lies inside the innermost ring (it is not a wall)
    const int i = (R == 0.f && R0 == 0.f) ? 0 : locate_axis(g.rw, g.n1, R, vR);
    if (i < 0) return false;
    r.i = i;
    r.j = j;
    r.k = phi_cell(g, r);
    r.ci = lin(g, r.i, r.j, r.k);
    return true;
}

// ================================================================ dispatch
template <int G>
__device__ __forceinline__ float cell_exit(const DevGrid& g, const Ray& r, int& axis, int& dir) {
    if constexpr (G == GRID_CARTESIAN) {
        const float l = cart_exit(g, r, axis);
        dir = 0;
        return l;
    } else if constexpr (G == GRID_SPHERICAL) {
        return sph_exit(g, r, axis, dir);
    } else {
        return cyl_exit(g, r, axis, dir);
    }
}

template <int G>
__device__ __forceinline__ bool cell_step(const DevGrid& g, Ray& r, float l, int axis, int dir) {
    if constexpr (G == GRID_CARTESIAN) return cart_step(g, r, l, axis);
    else if constexpr (G == GRID_SPHERICAL) return sph_step(g, r, l, axis, dir);
    else return cyl_step(g, r, l, axis, dir);
}

template <int G>
__device__ __forceinline__ bool grid_locate(const DevGrid& g, Ray& r) {
    if constexpr (G == GRID_CARTESIAN) return cart_locate(g, r);
    else if constexpr (G == GRID_SPHERICAL) return sph_locate(g, r);
    else return cyl_locate(g, r);
}

// ================================================================ grid entry from outside
// Cell index of v clamped into [w_0, w_n] (no direction rule: used only at the outer boundary).
__device__ __forceinline__ int clamp_axis(const float* __restrict__ w, int n, float v) {
    if (!(v > __ldg(w))) return 0;
    if (!(v < __ldg(w + n))) return n - 1;
    int lo = 0, hi = n;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(w + mid) <= v) lo = mid; else hi = mid;
    }
    return lo;
}

// Locate a packet that has just crossed the grid's outer boundary inwards (grid_entry, then a
// step of 1e-6 along the ray).  On a ray that enters at a glancing angle that step is a radial
// depth below FP32 rounding of the position, which can leave the point just outside; such a
// point belongs to the boundary cell it is entering, so the outer index is clamped there.
template <int G>
__device__ __forceinline__ bool grid_locate_entry(const DevGrid& g, Ray& r) {
    if (grid_locate<G>(g, r)) return true;
    if constexpr (G == GRID_CARTESIAN) {
        r.i = clamp_axis(g.w1, g.n1, r.p.x);
        r.j = clamp_axis(g.w2, g.n2, r.p.y);
        r.k = clamp_axis(g.w3, g.n3, r.p.z);
    } else if constexpr (G == GRID_SPHERICAL) {
        r.i = clamp_axis(g.rw, g.n1, sqrtf(dot3(r.p, r.p)));
        sph_angles(g, r);
    } else {
        const float R = sqrtf(r.p.x * r.p.x + r.p.y * r.p.y);
        if (R < __ldg(g.rw)) return false;                  // the inner cylinder is not the boundary
        r.i = clamp_axis(g.rw, g.n1, R);
        r.j = clamp_axis(g.w2, g.n2, r.p.z);
        r.k = phi_cell(g, r);
    }
    r.ci = lin(g, r.i, r.j, r.k);
    return true;
}

// Parameter t >= 0 at which p + t u first enters the grid's outer boundary (0 when p is inside),
// or -1 when the ray misses the grid (FP32, scaled lengths).
template <int G>
__device__ __forceinline__ float grid_entry(const DevGrid& g, float3 p, float3 u) {
    float tmin = -F_INF, tmax = F_INF;
    if constexpr (G == GRID_SPHERICAL) {
        const float ro = __ldg(g.rw + g.n1);
        const float b = dot3(p, u), c = fmaf(-ro, ro, dot3(p, p));
        if (c <= 0.f) return 0.f;
        const float disc = b * b - c;
        if (disc < 0.f || b >= 0.f) return -1.f;
        return c / (-b + sqrtf(disc));
    } else {
        const float* ws[3] = {g.w1, g.w2, g.w3};
        const int ns[3] = {g.n1, g.n2, g.n3};
        const float pc[3] = {p.x, p.y, p.z}, uc[3] = {u.x, u.y, u.z};
        if constexpr (G == GRID_CYLINDRICAL) {
            const float ro = __ldg(g.rw + g.n1);
            const float a = u.x * u.x + u.y * u.y, b = p.x * u.x + p.y * u.y;
            const float c = fmaf(-ro, ro, p.x * p.x + p.y * p.y);
            if (a == 0.f) {
                if (c > 0.f) return -1.f;
            } else {
                const float disc = b * b - a * c;
                if (disc < 0.f) return -1.f;
                const float sq = sqrtf(disc);
                tmin = (-b - sq) / a;
                tmax = (-b + sq) / a;
            }
        }
        for (int ax = (G == GRID_CYLINDRICAL ? 2 : 0); ax < 3; ++ax) {
            // Cartesian: x, y, z; cylindrical: only z (the w2 walls)
            const int wa = G == GRID_CYLINDRICAL ? 1 : ax;
            const float* w = ws[wa];
            const float lo = __ldg(w), hi = __ldg(w + ns[wa]);
            if (uc[ax] == 0.f) {
                if (pc[ax] < lo || pc[ax] > hi) return -1.f;
                continue;
            }
            const float t1 = (lo - pc[ax]) / uc[ax], t2 = (hi - pc[ax]) / uc[ax];
            tmin = fmaxf(tmin, fminf(t1, t2));
            tmax = fminf(tmax, fmaxf(t1, t2));
        }
    }
    if (tmax < fmaxf(tmin, 0.f)) return -1.f;
    return fmaxf(tmin, 0.f);
}

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Near-zero crossings (shorter than 1e-6 of the radius) in a row beyond which the ray is
// moved on by a hair: a ray grazing a curved wall within rounding could otherwise cross it back
// and forth without advancing.  A ray that still makes no headway after MAX_WALK_STEPS
// crossings is ended and counted (C_STUCK); the walk therefore always terminates.
constexpr int ZERO_RUN_LIMIT = 16;
constexpr unsigned MAX_WALK_STEPS = 1u << 22;

__device__ __forceinline__ bool tiny_step(const Ray& r, float l) { return l <= 1e-6f * sqrtf(dot3(r.p, r.p)); }

__device__ __forceinline__ void nudge(Ray& r) {
    const float h = 1e-6f * fmaxf(sqrtf(dot3(r.p, r.p)), 1e-6f);
    r.p.x += h * r.u.x;
    r.p.y += h * r.u.y;
    r.p.z += h * r.u.z;
}

// Extinction optical depth from the ray's position to the grid edge (no deposit), each crossing
// counted in ncross; the walk stops once the depth passes tau_stop.  A ray that has not reached
// the edge after MAX_WALK_STEPS crossings is dropped: F_INF.
template <int G>
__device__ __forceinline__ float tau_to_edge(const DevGrid& g, Ray r, float chi, unsigned long long& ncross,
                                             float tau_stop) {
    float tau = 0.f;
    if constexpr (G == GRID_CARTESIAN) {
        // the next wall of every axis in registers, one wall load per crossing (same arithmetic)
        float3 wn = cart_next_walls(g, r);
        for (unsigned steps = 0; steps < MAX_WALK_STEPS; ++steps) {
            int axis;
            const float l = cart_exit_w(r, wn, axis);
            tau += __ldg(g.rhoL + r.ci) * chi * l;
            ++ncross;
            if (tau > tau_stop) return tau;
            if (cart_step_w(g, r, wn, l, axis)) return tau;
        }
        return F_INF;
    }
    int zero_run = 0;
    for (unsigned steps = 0; steps < MAX_WALK_STEPS; ++steps) {
        int axis, dir;
        const float l = cell_exit<G>(g, r, axis, dir);
        tau += __ldg(g.rhoL + r.ci) * chi * l;
        ++ncross;
        if (tau > tau_stop) return tau;
        if (cell_step<G>(g, r, l, axis, dir)) return tau;
        if constexpr (G != GRID_CARTESIAN) {
            if (!tiny_step(r, l)) zero_run = 0;
            else if (++zero_run > ZERO_RUN_LIMIT) { nudge(r); zero_run = 0; }
        }
    }
    return F_INF;
}

}  // namespace hrt
