// Single-step kernels: one step of the method on many independent inputs with given uniform
// deviates, for element-by-element comparison with a CPU reference.  They call exactly the
// device functions the propagation kernels use.
#include "hrt_internal.h"
#include "packet.cuh"

namespace hrt {

__global__ void k_step_philox(int64_t n, const uint32_t* ctr, const uint32_t* key, uint32_t* out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint4 c = make_uint4(ctr[4 * i], ctr[4 * i + 1], ctr[4 * i + 2], ctr[4 * i + 3]);
        const uint4 r = philox4x32_10(c, make_uint2(key[2 * i], key[2 * i + 1]));
        out[4 * i] = r.x; out[4 * i + 1] = r.y; out[4 * i + 2] = r.z; out[4 * i + 3] = r.w;
    }
}

template <int G>
__global__ void k_step_exit(DevGrid g, int64_t n, const float* pos, const float* dir, const int32_t* cell,
                            float* dist, int32_t* ex, float inv_L0, float L0) {
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
        Ray r;
        r.p = make_float3(pos[3 * q] * inv_L0, pos[3 * q + 1] * inv_L0, pos[3 * q + 2] * inv_L0);
        set_dir(r, make_float3(dir[3 * q], dir[3 * q + 1], dir[3 * q + 2]));
        r.i = cell[3 * q]; r.j = cell[3 * q + 1]; r.k = cell[3 * q + 2];
        r.ci = lin(g, r.i, r.j, r.k);
        int axis, d;
        const float l = cell_exit<G>(g, r, axis, d);
        if constexpr (G == GRID_CARTESIAN) {
            const float ua = axis == 0 ? r.u.x : (axis == 1 ? r.u.y : r.u.z);
            d = ua > 0.f ? 1 : -1;
        }
        dist[q] = l * L0;
        ex[q] = axis * 2 + (d > 0 ? 1 : 0);
    }
}

template <int G>
__global__ void k_step_tau(DevGrid g, DevDust dd, int64_t n, const float* pos, const float* dir, const float* nu,
                           float* tau, float inv_L0) {
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
        Ray r;
        r.p = make_float3(pos[3 * q] * inv_L0, pos[3 * q + 1] * inv_L0, pos[3 * q + 2] * inv_L0);
        set_dir(r, make_float3(dir[3 * q], dir[3 * q + 1], dir[3 * q + 2]));
        unsigned long long nc = 0;
        float t = 0.f;
        if (grid_locate<G>(g, r)) t = tau_to_edge<G>(g, r, dust_at(dd, nu[q]).chi, nc, F_INF);
        tau[q] = t;
    }
}

template <int G>
__global__ void k_step_wall_distance(DevGrid g, int64_t n, const float* pos, const int32_t* cell, float* dist,
                                     float inv_L0, float L0) {
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
        Ray r;
        r.p = make_float3(pos[3 * q] * inv_L0, pos[3 * q + 1] * inv_L0, pos[3 * q + 2] * inv_L0);
        r.i = cell[3 * q]; r.j = cell[3 * q + 1]; r.k = cell[3 * q + 2];
        r.ci = lin(g, r.i, r.j, r.k);
        dist[q] = wall_distance<G>(g, r) * L0;
    }
}

__global__ void k_step_mrw_path(int64_t n, const float* tau0, const float* zeta, float* out) {
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x)
        out[q] = mrw_path(tau0[q], zeta[q]);
}

__global__ void k_step_hg(float gg, int64_t n, const float* din, const float* u1, const float* u2, float* dout) {
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
        const float3 u = make_float3(din[3 * q], din[3 * q + 1], din[3 * q + 2]);
        const float3 v = scatter_dir(u, hg_mu(gg, u1[q]), u2[q]);
        dout[3 * q] = v.x; dout[3 * q + 1] = v.y; dout[3 * q + 2] = v.z;
    }
}

__global__ void k_step_sample(const float* x, const float* cdf, int nx, int64_t n, const int32_t* row, const float* u,
                              float* out) {
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x)
        out[q] = sample_table(x, cdf + (int64_t)row[q] * nx, nx, u[q]);
}

static int blocks_for(int64_t n) {
    const int64_t b = (n + 255) / 256;
    return (int)(b < 1 ? 1 : (b > 4096 ? 4096 : b));
}

cudaError_t launch_step_philox(int64_t n, const uint32_t* ctr, const uint32_t* key, uint32_t* out, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_step_philox<<<blocks_for(n), 256, 0, s>>>(n, ctr, key, out);
    return cudaGetLastError();
}

cudaError_t launch_step_cell_exit(const DevGrid& g, int64_t n, const float* pos, const float* dir, const int32_t* cell,
                                  float* dist, int32_t* ex, float inv_L0, float L0, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    if (g.type == GRID_CARTESIAN)
        k_step_exit<GRID_CARTESIAN><<<blocks_for(n), 256, 0, s>>>(g, n, pos, dir, cell, dist, ex, inv_L0, L0);
    else if (g.type == GRID_CYLINDRICAL)
        k_step_exit<GRID_CYLINDRICAL><<<blocks_for(n), 256, 0, s>>>(g, n, pos, dir, cell, dist, ex, inv_L0, L0);
    else k_step_exit<GRID_SPHERICAL><<<blocks_for(n), 256, 0, s>>>(g, n, pos, dir, cell, dist, ex, inv_L0, L0);
    return cudaGetLastError();
}

cudaError_t launch_step_tau(const DevGrid& g, const DevDust& d, int64_t n, const float* pos, const float* dir,
                            const float* nu, float* tau, float inv_L0, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    if (g.type == GRID_CARTESIAN) k_step_tau<GRID_CARTESIAN><<<blocks_for(n), 256, 0, s>>>(g, d, n, pos, dir, nu, tau, inv_L0);
    else if (g.type == GRID_CYLINDRICAL)
        k_step_tau<GRID_CYLINDRICAL><<<blocks_for(n), 256, 0, s>>>(g, d, n, pos, dir, nu, tau, inv_L0);
    else k_step_tau<GRID_SPHERICAL><<<blocks_for(n), 256, 0, s>>>(g, d, n, pos, dir, nu, tau, inv_L0);
    return cudaGetLastError();
}

cudaError_t launch_step_wall_distance(const DevGrid& g, int64_t n, const float* pos, const int32_t* cell, float* dist,
                                     float inv_L0, float L0, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    if (g.type == GRID_CARTESIAN)
        k_step_wall_distance<GRID_CARTESIAN><<<blocks_for(n), 256, 0, s>>>(g, n, pos, cell, dist, inv_L0, L0);
    else if (g.type == GRID_CYLINDRICAL)
        k_step_wall_distance<GRID_CYLINDRICAL><<<blocks_for(n), 256, 0, s>>>(g, n, pos, cell, dist, inv_L0, L0);
    else k_step_wall_distance<GRID_SPHERICAL><<<blocks_for(n), 256, 0, s>>>(g, n, pos, cell, dist, inv_L0, L0);
    return cudaGetLastError();
}

cudaError_t launch_step_mrw_path(int64_t n, const float* tau0, const float* zeta, float* out, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_step_mrw_path<<<blocks_for(n), 256, 0, s>>>(n, tau0, zeta, out);
    return cudaGetLastError();
}

cudaError_t launch_step_hg(float g, int64_t n, const float* din, const float* u1, const float* u2, float* dout,
                           cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_step_hg<<<blocks_for(n), 256, 0, s>>>(g, n, din, u1, u2, dout);
    return cudaGetLastError();
}

cudaError_t launch_step_sample(const float* x, const float* cdf, int nx, int64_t n, const int32_t* row, const float* u,
                               float* out, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_step_sample<<<blocks_for(n), 256, 0, s>>>(x, cdf, nx, n, row, u, out);
    return cudaGetLastError();
}

}  // namespace hrt
