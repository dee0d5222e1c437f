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
// on a wall.  Sphere solves for small radii and cone solves near the polar axis run in FP64;
// everything else in FP32.
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

__device__ __forceinline__ bool cart_locate(const DevGrid& g, Ray& r) {
    r.i = locate_axis(g.w1, g.n1, r.p.x, r.u.x);
    r.j = locate_axis(g.w2, g.n2, r.p.y, r.u.y);
    r.k = locate_axis(g.w3, g.n3, r.p.z, r.u.z);
    if (r.i < 0 || r.j < 0 || r.k < 0) return false;
    r.ci = lin(g, r.i, r.j, r.k);
    return true;
}

// ================================================================ spherical-polar
// uR2 = u_x^2 + u_y^2, pu = p_x u_x + p_y u_y and Rp = |p_R| are shared by both cones of a cell.
template <typename R>
__device__ __forceinline__ R cone_root(R px, R py, R pz, R ux, R uy, R uz, R uR2, R pu, R Rp, R cw, R sw, int sense,
                                       R tol) {
    const R inf = R(F_INF);
    if (cw == R(0)) {          // the midplane z = 0; f = z increases when u_z > 0
        if (uz == R(0) || ((sense > 0) != (uz > R(0)))) return inf;
        const R s = -pz / uz;
        return s < -tol ? inf : (s > R(0) ? s : R(0));
    }
    const R sw2 = sw * sw, cw2 = cw * cw;
    const R A = uz * uz * sw2 - uR2 * cw2;
    const R B = pz * uz * sw2 - pu * cw2;
    const R f = pz * sw - Rp * cw;              // r sin(theta_w - theta): > 0 above the cone
    const R C = f * (pz * sw + Rp * cw);
    const R disc = B * B - A * C;
    if (disc < R(0)) return inf;
    const R sq = sqrt(disc);
    const R q = -(B + copysign(sq, B));
    R roots[2];
    roots[0] = (A != R(0)) ? q / A : inf;
    roots[1] = (q != R(0)) ? C / q : inf;
    R best = inf;
#pragma unroll
    for (int t = 0; t < 2; ++t) {
        const R s = roots[t];
        if (!(s >= -tol) || !(s < best)) continue;
        const R qz = pz + s * uz;
        if (!(qz * cw > R(0))) continue;        // other nappe
        const R qx = px + s * ux, qy = py + s * uy;
        const R Rq2 = qx * qx + qy * qy;
        if (Rq2 == R(0)) continue;
        // sign of df/ds = u_z sin - cos (q_R . u_R) / |q_R|, scaled by |q_R| > 0 (no division)
        const R dfds = uz * sw * sqrt(Rq2) - cw * (qx * ux + qy * uy);
        if (sense > 0 ? !(dfds > R(0)) : !(dfds < R(0))) continue;
        best = s > R(0) ? s : R(0);
    }
    return best;
}

// outer sphere: the far root (always ahead of a point inside); inner sphere: the near root,
// only while moving inwards.
template <typename R>
__device__ __forceinline__ R sphere_out(R rr, R b, R rw2) {
    const R c = rr - rw2;
    const R disc = b * b - c;
    const R sq = sqrt(disc > R(0) ? disc : R(0));
    // far root without cancellation: -c / (b + sq) when moving outwards, -b + sq otherwise
    const R s = b > R(0) ? -c / (b + sq) : -b + sq;
    return s > R(0) ? s : R(0);
}
template <typename R>
__device__ __forceinline__ R sphere_in(R rr, R b, R rw2) {
    const R c = rr - rw2;
    const R disc = b * b - c;
    if (disc < R(0)) return R(F_INF);
    const R s = c / (-b + sqrt(disc));
    return s > R(0) ? s : R(0);
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

// Exit through cone wall jw in the given sense; FP64 for walls near the polar axis.
__device__ __forceinline__ float cone_wall(const DevGrid& g, const Ray& r, int jw, int sense, float uR2, float pu,
                                          float Rp, float tol) {
    const float sw = __ldg(g.sth + jw);
    if (sw < g.sin_fp64) {
        const double px = r.p.x, py = r.p.y, ux = r.u.x, uy = r.u.y;
        return (float)cone_root<double>(px, py, r.p.z, ux, uy, r.u.z, ux * ux + uy * uy, px * ux + py * uy,
                                        sqrt(px * px + py * py), __ldg(g.cthd + jw), __ldg(g.sthd + jw), sense,
                                        (double)tol);
    }
    return cone_root<float>(r.p.x, r.p.y, r.p.z, r.u.x, r.u.y, r.u.z, uR2, pu, Rp, __ldg(g.cth + jw), sw, sense, tol);
}

// Distance to the exit of the current cell; axis 0/1/2 = r/theta/phi, dir = +-1.
__device__ __forceinline__ float sph_exit(const DevGrid& g, const Ray& r, int& axis, int& dir) {
    const float rr = dot3(r.p, r.p);
    const float b = dot3(r.p, r.u);
    const float tol = 2e-6f * sqrtf(rr) + 1e-30f;
    float best;
    const float rout = __ldg(g.rw + r.i + 1);
    // A ray enters the inner sphere only when clearly moving inwards: a ray tangent to the
    // sphere touches it at one point, and FP32 rounding of p.u around zero must not make it
    // cross back and forth there.
    const float b_in = -1e-6f * sqrtf(rr);
    if (rout < g.r_fp64) {
        const double pd[3] = {r.p.x, r.p.y, r.p.z}, ud[3] = {r.u.x, r.u.y, r.u.z};
        const double rrd = pd[0] * pd[0] + pd[1] * pd[1] + pd[2] * pd[2];
        const double bd = pd[0] * ud[0] + pd[1] * ud[1] + pd[2] * ud[2];
        const double ro = __ldg(g.rwd + r.i + 1), ri = __ldg(g.rwd + r.i);
        best = (float)sphere_out<double>(rrd, bd, ro * ro);
        axis = 0; dir = 1;
        if (ri > 0.0 && bd < (double)b_in) {
            const float s = (float)sphere_in<double>(rrd, bd, ri * ri);
            if (s < best) { best = s; dir = -1; }
        }
    } else {
        best = sphere_out<float>(rr, b, __ldg(g.r2w + r.i + 1));
        axis = 0; dir = 1;
        if (b < b_in && __ldg(g.rw + r.i) > 0.f) {
            const float s = sphere_in<float>(rr, b, __ldg(g.r2w + r.i));
            if (s < best) { best = s; dir = -1; }
        }
    }
    // terms shared by both cones of the cell
    const float uR2 = r.u.x * r.u.x + r.u.y * r.u.y;
    const float pu = r.p.x * r.u.x + r.p.y * r.u.y;
    const float Rp = sqrtf(r.p.x * r.p.x + r.p.y * r.p.y);
    // lower wall j is left with theta decreasing (sense +1), upper wall j + 1 increasing (-1)
    if (r.j > 0) {
        const float s = cone_wall(g, r, r.j, +1, uR2, pu, Rp, tol);
        if (s < best) { best = s; axis = 1; dir = -1; }
    }
    if (r.j + 1 < g.n2) {
        const float s = cone_wall(g, r, r.j + 1, -1, uR2, pu, Rp, tol);
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

// ================================================================ dispatch
template <int G>
__device__ __forceinline__ float cell_exit(const DevGrid& g, const Ray& r, int& axis, int& dir) {
    if constexpr (G == GRID_CARTESIAN) {
        const float l = cart_exit(g, r, axis);
        dir = 0;
        return l;
    } else {
        return sph_exit(g, r, axis, dir);
    }
}

template <int G>
__device__ __forceinline__ bool cell_step(const DevGrid& g, Ray& r, float l, int axis, int dir) {
    if constexpr (G == GRID_CARTESIAN) return cart_step(g, r, l, axis);
    else return sph_step(g, r, l, axis, dir);
}

template <int G>
__device__ __forceinline__ bool grid_locate(const DevGrid& g, Ray& r) {
    if constexpr (G == GRID_CARTESIAN) return cart_locate(g, r);
    else return sph_locate(g, r);
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

// Extinction optical depth from the ray's position to the grid edge (no deposit).
template <int G>
__device__ __forceinline__ float tau_to_edge(const DevGrid& g, Ray r, float chi, unsigned long long& ncross,
                                             float tau_stop) {
    float tau = 0.f;
    int zero_run = 0;
    for (unsigned steps = 0; steps < MAX_WALK_STEPS; ++steps) {
        int axis, dir;
        const float l = cell_exit<G>(g, r, axis, dir);
        tau += __ldg(g.rhoL + r.ci) * chi * l;
        ++ncross;
        if (tau > tau_stop) return tau;
        if (cell_step<G>(g, r, l, axis, dir)) return tau;
        if constexpr (G == GRID_SPHERICAL) {
            if (!tiny_step(r, l)) zero_run = 0;
            else if (++zero_run > ZERO_RUN_LIMIT) { nudge(r); zero_run = 0; }
        }
    }
    return tau;
}

}  // namespace hrt
