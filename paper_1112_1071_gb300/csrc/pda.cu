// Partial diffusion approximation (App. A) on spherical-polar grids, FP64.
//
// Cells with dust that the propagation sampled with fewer than n_min packet entries (consecutive
// path segments of one packet in one cell count once) take T^4 from the discrete diffusion
// equation printed in App. A.  That equation, multiplied through by r_i^2 dr_i sin(theta_j)
// dtheta_j dphi_k, is symmetric: every face between cells c and n has one weight
//   W = F / (dtau_c + dtau_n),
//   F = r_face^2 sin(theta_j) dtheta_j dphi_k   (radial faces),
//       r_i dr_i dphi_k sin(theta_face)          (polar faces),
//       r_i dr_i dtheta_j                        (azimuthal faces),
// with dtau the Rosseland optical depth across the cell along that coordinate (rho chi_R dr,
// rho chi_R r dtheta, rho chi_R r sin(theta) dphi; chi_R at the previous iteration's temperature;
// r, theta at cell centres).  Neighbours outside the grid or without dust add no term; phi is
// periodic.  Well-sampled neighbours are boundary values (App. A); a connected region with none
// keeps its Monte-Carlo temperatures.  The symmetric positive definite system sum_n W (x_c - x_n)
// = 0 is solved for x = T^4 by Jacobi-preconditioned conjugate gradients; Adot = E(T) (Eq. 3)
// and the convergence key of the solved cells are then replaced.
#include "hrt_internal.h"
#include "planck.cuh"
#include "temperature.cuh"

namespace hrt {

// Rosseland mean extinction chi_R(T_m) = int dB/dT dnu / int chi^-1 dB/dT dnu, trapezoid rule
// over the dust nodes; one thread per temperature node.
__global__ void k_rosseland(int nnu, const double* __restrict__ nu, const double* __restrict__ chi, int nT,
                            const double* __restrict__ T, double* __restrict__ chiR, double* __restrict__ lnchiR) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= nT) return;
    double num = 0.0, den = 0.0;
    double w0 = planck_dbdt(nu[0], T[m]);
    for (int k = 1; k < nnu; ++k) {
        const double w1 = planck_dbdt(nu[k], T[m]);
        const double dn = nu[k] - nu[k - 1];
        num += 0.5 * (w1 + w0) * dn;
        den += 0.5 * (w1 / chi[k] + w0 / chi[k - 1]) * dn;
        w0 = w1;
    }
    chiR[m] = num / den;
    lnchiR[m] = log(num / den);
}

cudaError_t launch_rosseland(int nnu, const double* nu, const double* chi, int nT, const double* T, double* chiR,
                             double* lnchiR, cudaStream_t s) {
    k_rosseland<<<(nT + 127) / 128, 128, 0, s>>>(nnu, nu, chi, nT, T, chiR, lnchiR);
    return cudaGetLastError();
}

struct Cell3 { int i, j, k; };
__device__ __forceinline__ Cell3 cell3(const PdaJob& J, int64_t c) {
    Cell3 q;
    q.i = (int)(c % J.n1);
    q.j = (int)((c / J.n1) % J.n2);
    q.k = (int)(c / ((int64_t)J.n1 * J.n2));
    return q;
}

// Neighbour across face f (0/1: r +-, 2/3: theta +-, 4/5: phi +-, periodic), -1 outside.
__device__ __forceinline__ int64_t neighbour(const PdaJob& J, Cell3 q, int f) {
    int i = q.i, j = q.j, k = q.k;
    switch (f) {
        case 0: ++i; break;
        case 1: --i; break;
        case 2: ++j; break;
        case 3: --j; break;
        case 4: k = (k + 1) % J.n3; break;
        default: k = (k + J.n3 - 1) % J.n3; break;
    }
    if (i < 0 || i >= J.n1 || j < 0 || j >= J.n2) return -1;
    return ((int64_t)k * J.n2 + j) * J.n1 + i;
}

// Rosseland optical depths across each cell, and the candidate mask.
__global__ void k_pda_dtau(PdaJob J) {
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < J.nc; c += (int64_t)gridDim.x * blockDim.x) {
        const Cell3 q = cell3(J, c);
        const double rho = (double)J.rhoL[c];
        const double rk = rho * loglog(J.T_prev[c], J.lnT, J.lnchiR, J.nT);
        J.dtau[c] = rk * J.dr[q.i];
        J.dtau[J.nc + c] = rk * J.rc[q.i] * J.dth[q.j];
        J.dtau[2 * J.nc + c] = rk * J.rc[q.i] * J.stc[q.j] * J.dph[q.k];
        J.state[c] = (rho > 0.0 && J.visits[c] < J.n_min) ? 1 : 0;
    }
}

// Face weights of the candidate cells; candidates next to a well-sampled dust cell are anchored.
__global__ void k_pda_weights(PdaJob J) {
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < J.nc; c += (int64_t)gridDim.x * blockDim.x) {
        if (J.state[c] == 0) continue;
        const Cell3 q = cell3(J, c);
        bool anchored = false;
        for (int f = 0; f < 6; ++f) {
            const int64_t n = neighbour(J, q, f);
            double w = 0.0;
            if (n >= 0 && J.rhoL[n] > 0.f) {
                const int ax = f >> 1;
                const double den = J.dtau[ax * J.nc + c] + J.dtau[ax * J.nc + n];
                double F;
                if (ax == 0) {
                    const double rf = J.rface[q.i + (f == 0 ? 1 : 0)];
                    F = rf * rf * J.stc[q.j] * J.dth[q.j] * J.dph[q.k];
                } else if (ax == 1) {
                    F = J.rc[q.i] * J.dr[q.i] * J.dph[q.k] * J.stf[q.j + (f == 2 ? 1 : 0)];
                } else {
                    F = J.rc[q.i] * J.dr[q.i] * J.dth[q.j];
                }
                if (den > 0.0) w = F / den;
                if (w > 0.0 && J.state[n] == 0) anchored = true;
            }
            J.W[f * J.nc + c] = w;
        }
        if (anchored) J.state[c] = 2;
    }
}

// One sweep of the anchoring flood: a candidate next to an anchored cell is anchored.
__global__ void k_pda_flood(PdaJob J, int* changed) {
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < J.nc; c += (int64_t)gridDim.x * blockDim.x) {
        if (J.state[c] != 1) continue;
        const Cell3 q = cell3(J, c);
        for (int f = 0; f < 6; ++f) {
            if (!(J.W[f * J.nc + c] > 0.0)) continue;
            const int64_t n = neighbour(J, q, f);
            if (J.state[n] == 2) {
                J.state[c] = 2;
                *changed = 1;
                break;
            }
        }
    }
}

// Block sum of one FP64 value per thread, added to *out by thread 0.
__device__ __forceinline__ void block_add(double v, double* out) {
    __shared__ double part[32];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) part[wid] = v;
    __syncthreads();
    if (wid == 0) {
        v = lane < (int)(blockDim.x >> 5) ? part[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0 && v != 0.0) atomicAdd(out, v);
    }
    __syncthreads();
}

// Conjugate gradients preconditioned by the diagonal (Jacobi): the face weights span many
// decades between optically thin and thick cells, and the diagonal scaling removes most of that.
// Scalars: [0] r.z, [1] p.q, [2] new r.z, [3] r.r, [4] b.b, [5] iterations.
//
// x0 = (T_mc)^4, b from the boundary values, r = b - A x0, z = r / diag, p = z; sums r.z, r.r,
// b.b; counts the cells.
__global__ void __launch_bounds__(256) k_cg_init(PdaJob J) {
    double rz = 0.0, rr = 0.0, bb = 0.0;
    unsigned long long cnt = 0;
    for (int64_t c0 = (int64_t)blockIdx.x * blockDim.x; c0 < J.nc; c0 += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = c0 + threadIdx.x;
        if (c < J.nc) {
            double x = 0.0, r = 0.0, b = 0.0, dg = 0.0;
            if (J.state[c] == 2) {
                const Cell3 q = cell3(J, c);
                const double t = J.T[c];
                x = t * t * t * t;
                double off = 0.0;
                for (int f = 0; f < 6; ++f) {
                    const double w = J.W[f * J.nc + c];
                    if (!(w > 0.0)) continue;
                    const int64_t n = neighbour(J, q, f);
                    const double tn = J.T[n];
                    const double xn = tn * tn * tn * tn;
                    dg += w;
                    if (J.state[n] == 2) off += w * xn;
                    else b += w * xn;
                }
                r = b - (dg * x - off);
                ++cnt;
            }
            const double z = dg > 0.0 ? r / dg : 0.0;
            J.x[c] = x; J.r[c] = r; J.p[c] = z; J.b[c] = b; J.dg[c] = dg;
            rz += r * z;
            rr += r * r;
            bb += b * b;
        }
    }
    block_add(rz, J.scal + 0);
    block_add(rr, J.scal + 3);
    block_add(bb, J.scal + 4);
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_down_sync(0xffffffffu, cnt, o);
    if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(J.count, cnt);
}

// q = A p and the sum p.q
__global__ void __launch_bounds__(256) k_cg_apply(PdaJob J) {
    double pq = 0.0;
    for (int64_t c0 = (int64_t)blockIdx.x * blockDim.x; c0 < J.nc; c0 += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = c0 + threadIdx.x;
        if (c < J.nc) {
            double v = 0.0;
            if (J.state[c] == 2) {
                const Cell3 q = cell3(J, c);
                double off = 0.0;
                for (int f = 0; f < 6; ++f) {
                    const double w = J.W[f * J.nc + c];
                    if (!(w > 0.0)) continue;
                    const int64_t n = neighbour(J, q, f);
                    if (J.state[n] == 2) off += w * J.p[n];
                }
                v = J.dg[c] * J.p[c] - off;
                pq += J.p[c] * v;
            }
            J.q[c] = v;
        }
    }
    block_add(pq, J.scal + 1);
}

// x += alpha p, r -= alpha q (alpha = r.z / p.q), z = r / diag; sums of the new r.z and r.r
__global__ void __launch_bounds__(256) k_cg_update(PdaJob J) {
    const double pq = J.scal[1];
    const double alpha = pq > 0.0 ? J.scal[0] / pq : 0.0;
    double rz = 0.0, rr = 0.0;
    for (int64_t c0 = (int64_t)blockIdx.x * blockDim.x; c0 < J.nc; c0 += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = c0 + threadIdx.x;
        if (c < J.nc && J.state[c] == 2) {
            J.x[c] += alpha * J.p[c];
            const double r = J.r[c] - alpha * J.q[c];
            J.r[c] = r;
            rz += r * (r / J.dg[c]);
            rr += r * r;
        }
    }
    block_add(rz, J.scal + 2);
    block_add(rr, J.scal + 3);
}

// p = z + beta p (beta = new r.z / old r.z)
__global__ void k_cg_direction(PdaJob J) {
    const double beta = J.scal[0] > 0.0 ? J.scal[2] / J.scal[0] : 0.0;
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < J.nc; c += (int64_t)gridDim.x * blockDim.x)
        if (J.state[c] == 2) J.p[c] = J.r[c] / J.dg[c] + beta * J.p[c];
}

// roll the scalars; r.r of this iteration stays in [3] for the host's stopping test
__global__ void k_cg_roll(double* scal) {
    scal[0] = scal[2];
    scal[1] = 0.0;
    scal[2] = 0.0;
    scal[5] += 1.0;
}

__global__ void k_cg_clear_rr(double* scal) { scal[3] = 0.0; }

// T = x^(1/4), Adot = E(T), re-emission row and convergence key of the solved cells.
__global__ void k_pda_finish(PdaJob J) {
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < J.nc; c += (int64_t)gridDim.x * blockDim.x) {
        if (J.state[c] != 2) continue;
        const double T = pow(fmax(J.x[c], 1e-300), 0.25);
        const double A = loglog(T, J.lnT, J.lnE, J.nT);
        J.T[c] = T;
        J.adot[c] = A;
        J.row[c] = nearest_row(T, J.lnT, J.nT);
        double R;
        if (J.quantity == 0) R = fmax(J.T_prev[c] / T, T / J.T_prev[c]);
        else R = J.first ? __longlong_as_double(0x7ff0000000000000ll) : fmax(J.adot_prev[c] / A, A / J.adot_prev[c]);
        if (!(R == R)) R = __longlong_as_double(0x7ff0000000000000ll);
        J.keys[c] = (unsigned long long)__double_as_longlong(R);
    }
}

static int pda_grid(int64_t n) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t need = (n + 255) / 256;
    const int64_t cap = (int64_t)sms * 8;
    return (int)(need < 1 ? 1 : (need < cap ? need : cap));
}

cudaError_t run_pda(const PdaJob& J, double tol, int max_iter, int* host_flag, double* host_scal, PdaStats* st,
                    cudaStream_t s, int* launched) {
    const int grid = pda_grid(J.nc);
    cudaError_t e;
    if ((e = cudaMemsetAsync(J.scal, 0, 8 * sizeof(double), s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(J.count, 0, sizeof(unsigned long long), s)) != cudaSuccess) return e;
    k_pda_dtau<<<grid, 256, 0, s>>>(J);
    k_pda_weights<<<grid, 256, 0, s>>>(J);
    *launched += 2;
    // anchoring flood: each sweep that changes anything anchors at least one more cell
    for (int64_t sweep = 0; sweep < J.nc; ++sweep) {
        if ((e = cudaMemsetAsync(J.flag, 0, sizeof(int), s)) != cudaSuccess) return e;
        k_pda_flood<<<grid, 256, 0, s>>>(J, J.flag);
        *launched += 1;
        if ((e = cudaMemcpyAsync(host_flag, J.flag, sizeof(int), cudaMemcpyDeviceToHost, s)) != cudaSuccess) return e;
        if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
        if (*host_flag == 0) break;
    }
    k_cg_init<<<grid, 256, 0, s>>>(J);
    *launched += 1;
    if ((e = cudaMemcpyAsync(host_scal, J.scal, 8 * sizeof(double), cudaMemcpyDeviceToHost, s)) != cudaSuccess) return e;
    unsigned long long cnt = 0;
    if ((e = cudaMemcpyAsync(&cnt, J.count, sizeof(cnt), cudaMemcpyDeviceToHost, s)) != cudaSuccess) return e;
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
    st->n_cells = (int64_t)cnt;
    st->iterations = 0;
    st->residual = 0.0;
    if (cnt == 0) return cudaGetLastError();
    const double bb = host_scal[4];
    double rr = host_scal[3];
    const double stop = tol * tol * bb;
    int it = 0;
    while (it < max_iter && rr > stop && rr > 0.0) {
        const int chunk = 8;
        for (int u = 0; u < chunk; ++u) {
            k_cg_apply<<<grid, 256, 0, s>>>(J);
            k_cg_clear_rr<<<1, 1, 0, s>>>(J.scal);
            k_cg_update<<<grid, 256, 0, s>>>(J);
            k_cg_direction<<<grid, 256, 0, s>>>(J);
            k_cg_roll<<<1, 1, 0, s>>>(J.scal);
        }
        *launched += 5 * chunk;
        it += chunk;
        if ((e = cudaMemcpyAsync(host_scal, J.scal, 8 * sizeof(double), cudaMemcpyDeviceToHost, s)) != cudaSuccess)
            return e;
        if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
        rr = host_scal[3];
    }
    st->iterations = it;
    st->residual = bb > 0.0 ? sqrt(rr / bb) : 0.0;
    k_pda_finish<<<grid, 256, 0, s>>>(J);
    *launched += 1;
    return cudaGetLastError();
}

}  // namespace hrt
