// Raytracing of the source and dust emission into SEDs and images (Sect. 2.6.3).
//
// Once the temperatures have converged, thermal emission reaches each observer without a
// random walk.  Emission at a point whose column to the grid edge along the observer direction
// is Sigma = int rho ds arrives in SED bin b with
//     L / (4 pi) int_bin p(nu) exp(-chi(nu) Sigma) dnu,
// p the normalised spectrum the packets would sample (piecewise constant between table nodes:
// the source spectrum, or the cell's emissivity row kappa_nu B_nu(T)), chi the extinction.  The
// bin integral is a quadrature on the pieces of the bin between the nodes of p and of chi
// (3-point Gauss-Legendre, nodes and chi tabulated on the host once per pass).  Point sources
// send their luminosity along the one ray from the source (the columns of k_source_columns).
// Dust emission is sampled by rays: ray k picks a cell in proportion to its emission m E(T)
// (Eq. 3) and a point uniform in its volume, from its own Philox stream, and carries
// L_dust / n_rays.  One walk per ray and observer gives Sigma; the quadrature over all bins then
// runs as a separate reduction over rays.  Images take the same weights at the projected point.
#include "propagate_common.cuh"

namespace hrt {

// ---------------------------------------------------------------- emission luminosity and CDF
__global__ void k_rt_lum(RtJob J) {
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < J.nc; c += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(c % J.n1), j = (int)((c / J.n1) % J.n2), k = (int)(c / ((int64_t)J.n1 * J.n2));
        double L = 0.0;
        const double rho = (double)J.rho[c];
        if (rho > 0.0) {
            const double lx = log(J.T[c]);
            double lE;
            if (!(lx > J.lnT[0])) lE = J.lnE[0];
            else if (lx >= J.lnT[J.nT - 1]) lE = J.lnE[J.nT - 1];
            else {
                int lo = 0, hi = J.nT - 1;
                while (hi - lo > 1) {
                    const int mid = (lo + hi) >> 1;
                    if (J.lnT[mid] <= lx) lo = mid; else hi = mid;
                }
                lE = J.lnE[lo] + (lx - J.lnT[lo]) / (J.lnT[lo + 1] - J.lnT[lo]) * (J.lnE[lo + 1] - J.lnE[lo]);
            }
            L = rho * J.va[i] * J.vb[j] * J.vc[k] * exp(lE);
        }
        J.cdf[c] = L;
    }
}

// Inclusive prefix sum of J.cdf in place (FP64), in three steps: block sums, a scan of the block
// sums by one block, and the scan of each block with its offset; then normalisation.
constexpr int SCAN_BLOCK = 1024;

__device__ __forceinline__ double block_inclusive_scan(double v, double* sh) {
    const int t = threadIdx.x;
    sh[t] = v;
    __syncthreads();
    for (int off = 1; off < blockDim.x; off <<= 1) {
        const double add = t >= off ? sh[t - off] : 0.0;
        __syncthreads();
        sh[t] += add;
        __syncthreads();
    }
    return sh[t];
}

__global__ void __launch_bounds__(SCAN_BLOCK) k_scan_blocks(double* x, int64_t n, double* sums) {
    __shared__ double sh[SCAN_BLOCK];
    const int64_t c = (int64_t)blockIdx.x * SCAN_BLOCK + threadIdx.x;
    const double v = c < n ? x[c] : 0.0;
    const double s = block_inclusive_scan(v, sh);
    if (c < n) x[c] = s;
    if (threadIdx.x == SCAN_BLOCK - 1) sums[blockIdx.x] = s;
}

__global__ void __launch_bounds__(SCAN_BLOCK) k_scan_sums(double* sums, int nb, double* total) {
    __shared__ double sh[SCAN_BLOCK];
    double carry = 0.0;
    for (int base = 0; base < nb; base += SCAN_BLOCK) {
        const int b = base + threadIdx.x;
        const double v = b < nb ? sums[b] : 0.0;
        const double s = block_inclusive_scan(v, sh);
        if (b < nb) sums[b] = carry + s - v;     // exclusive offset of block b
        __syncthreads();
        carry += sh[SCAN_BLOCK - 1];
        __syncthreads();
    }
    if (threadIdx.x == 0) *total = carry;
}

__global__ void k_scan_finish(double* x, int64_t n, const double* offs, const double* total) {
    const int64_t c = (int64_t)blockIdx.x * SCAN_BLOCK + threadIdx.x;
    if (c >= n) return;
    const double t = *total;
    double v = t > 0.0 ? (x[c] + offs[blockIdx.x]) / t : 0.0;
    if (c == n - 1) v = 1.0;
    x[c] = v;
}

// ---------------------------------------------------------------- dust rays: columns, images
__device__ __forceinline__ float emission_pdf(const RtJob& J, int row, int j) {
    const float* cdf = J.cdf_emit + (int64_t)row * J.nnu;
    return (__ldg(cdf + j + 1) - __ldg(cdf + j)) * __ldg(J.inv_dnu + j);
}

// sum_q over the dust quadrature nodes of bin b of p_row(j_q) w_q exp(-chi_q Sigma)
__device__ __forceinline__ float dust_bin(const RtJob& J, int row, int b, float sigma) {
    float acc = 0.f;
    for (int q = __ldg(J.qd_off + b); q < __ldg(J.qd_off + b + 1); ++q)
        acc += emission_pdf(J, row, __ldg(J.qd_j + q)) * __ldg(J.qd_w + q) * expf(-__ldg(J.qd_chi + q) * sigma);
    return acc;
}

template <int G>
__global__ void __launch_bounds__(256) k_rt_rays(DevGrid g, DevObs o, RtJob J) {
    unsigned long long ncross = 0;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < J.n_rays; k += (int64_t)gridDim.x * blockDim.x) {
        PacketRng rng;
        rng.init(make_uint2(J.key0, J.key1), (uint32_t)k, J.iter_key, J.model_key);
        const int64_t c = select_cdf<double>(J.cdf, J.nc, (double)rng.next());
        const float f0 = rng.next(), f1 = rng.next(), f2 = rng.next();
        Ray at;
        place_in_cell<G>(g, c, f0, f1, f2, at);
        const int row = min(max(__ldg(J.emit_row + c), 0), J.nT - 1);
        J.row[k] = row;
        for (int ob = 0; ob < o.nobs; ++ob) {
            Ray r = at;
            set_dir(r, make_float3(__ldg(o.n + 3 * ob), __ldg(o.n + 3 * ob + 1), __ldg(o.n + 3 * ob + 2)));
            const float sigma = tau_to_edge<G>(g, r, 1.f, ncross, F_INF);
            J.col[k * o.nobs + ob] = sigma;
            if (o.nimg > 0) {
                const float px = at.p.x * __ldg(o.ex + 3 * ob) + at.p.y * __ldg(o.ex + 3 * ob + 1) + at.p.z * __ldg(o.ex + 3 * ob + 2);
                const float py = at.p.x * __ldg(o.ey + 3 * ob) + at.p.y * __ldg(o.ey + 3 * ob + 1) + at.p.z * __ldg(o.ey + 3 * ob + 2);
                const int ix = (int)floorf((px + o.img_half) * o.img_scale);
                const int iy = (int)floorf((py + o.img_half) * o.img_scale);
                if (ix >= 0 && ix < o.img_nx && iy >= 0 && iy < o.img_ny)
                    for (int l = 0; l < o.nimg; ++l) {
                        const int b = __ldg(o.img_bin + l);
                        if (b < 0) continue;
                        const double w = J.eps4pi * (double)dust_bin(J, row, b, sigma);
                        atomicAdd(J.img + (((int64_t)ob * o.nimg + l) * o.img_ny + iy) * o.img_nx + ix, w);
                    }
            }
        }
    }
    for (int off = 16; off > 0; off >>= 1) ncross += __shfl_down_sync(0xffffffffu, ncross, off);
    if ((threadIdx.x & 31) == 0 && ncross) atomicAdd(J.counters + C_PEEL_CROSSINGS, ncross);
}

// ---------------------------------------------------------------- dust rays: SED bins
// Block (ob, 256 quadrature nodes, chunk of RT_CHUNK rays): each thread sums one node over the
// chunk's rays (FP32), then adds eps/(4 pi) w_q times the sum to its bin (FP64 atomic).
constexpr int RT_CHUNK = 2048;

__global__ void __launch_bounds__(256) k_rt_sed(RtJob J, int nobs) {
    __shared__ float s_col[RT_CHUNK];
    __shared__ int s_row[RT_CHUNK];
    const int ob = blockIdx.x;
    const int q = blockIdx.y * blockDim.x + threadIdx.x;
    const int64_t k0 = (int64_t)blockIdx.z * RT_CHUNK;
    const int nk = (int)min((int64_t)RT_CHUNK, J.n_rays - k0);
    for (int t = threadIdx.x; t < nk; t += blockDim.x) {
        s_col[t] = J.col[(k0 + t) * nobs + ob];
        s_row[t] = J.row[k0 + t];
    }
    __syncthreads();
    if (q >= J.nqd) return;
    const int j = __ldg(J.qd_j + q);
    const float chi = __ldg(J.qd_chi + q);
    const float idn = __ldg(J.inv_dnu + j);
    float acc = 0.f;
    for (int t = 0; t < nk; ++t) {
        const float* cdf = J.cdf_emit + (int64_t)s_row[t] * J.nnu;
        acc += (__ldg(cdf + j + 1) - __ldg(cdf + j)) * expf(-chi * s_col[t]);
    }
    if (acc != 0.f)
        atomicAdd(J.sed + (int64_t)ob * J.nsed + __ldg(J.qd_bin + q), J.eps4pi * (double)(acc * idn * __ldg(J.qd_w + q)));
}

// ---------------------------------------------------------------- point sources
__global__ void k_rt_sources(DevObs o, RtJob J) {
    const int64_t n = (int64_t)J.npoint * o.nobs * J.nqs;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
        const int q = (int)(t % J.nqs);
        const int ob = (int)((t / J.nqs) % o.nobs);
        const int s = (int)(t / ((int64_t)J.nqs * o.nobs));
        const float sigma = J.src_col[s * o.nobs + ob];
        if (sigma < 0.f) continue;                 // source outside the grid
        const int j = J.qs_j[q];
        const double p = ((double)J.spec_cdf[(int64_t)s * J.nspec + j + 1] - (double)J.spec_cdf[(int64_t)s * J.nspec + j]) /
                         (J.spec_nu[j + 1] - J.spec_nu[j]);
        const double w = J.src_L[s] / (4.0 * CUDART_PI) * p * (double)J.qs_w[q] * exp(-(double)J.qs_chi[q] * sigma);
        if (w != 0.0) atomicAdd(J.sed + (int64_t)ob * J.nsed + J.qs_bin[q], w);
    }
}

__global__ void k_rt_source_images(DevObs o, RtJob J) {
    const int64_t n = (int64_t)J.npoint * o.nobs * o.nimg;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
        const int l = (int)(t % o.nimg);
        const int ob = (int)((t / o.nimg) % o.nobs);
        const int s = (int)(t / ((int64_t)o.nimg * o.nobs));
        const float sigma = J.src_col[s * o.nobs + ob];
        const int b = o.img_bin[l];
        if (sigma < 0.f || b < 0) continue;
        const float3 p = make_float3(J.src_pos[3 * s], J.src_pos[3 * s + 1], J.src_pos[3 * s + 2]);
        const float px = p.x * o.ex[3 * ob] + p.y * o.ex[3 * ob + 1] + p.z * o.ex[3 * ob + 2];
        const float py = p.x * o.ey[3 * ob] + p.y * o.ey[3 * ob + 1] + p.z * o.ey[3 * ob + 2];
        const int ix = (int)floorf((px + o.img_half) * o.img_scale);
        const int iy = (int)floorf((py + o.img_half) * o.img_scale);
        if (ix < 0 || ix >= o.img_nx || iy < 0 || iy >= o.img_ny) continue;
        double w = 0.0;
        for (int q = J.qs_off[b]; q < J.qs_off[b + 1]; ++q) {
            const int j = J.qs_j[q];
            const double pj = ((double)J.spec_cdf[(int64_t)s * J.nspec + j + 1] - (double)J.spec_cdf[(int64_t)s * J.nspec + j]) /
                              (J.spec_nu[j + 1] - J.spec_nu[j]);
            w += pj * (double)J.qs_w[q] * exp(-(double)J.qs_chi[q] * sigma);
        }
        w *= J.src_L[s] / (4.0 * CUDART_PI);
        if (w != 0.0) atomicAdd(J.img + (((int64_t)ob * o.nimg + l) * o.img_ny + iy) * o.img_nx + ix, w);
    }
}

// ---------------------------------------------------------------- driver
cudaError_t run_raytrace(const DevGrid& g, const DevObs& o, RtJob J, double* host_total, cudaStream_t s,
                         int* launched) {
    cudaError_t e;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    // point sources
    if (J.npoint > 0 && J.nqs > 0) {
        k_rt_sources<<<sms * 4, 256, 0, s>>>(o, J);
        *launched += 1;
        if (o.nimg > 0) {
            k_rt_source_images<<<(J.npoint * o.nobs * o.nimg + 127) / 128, 128, 0, s>>>(o, J);
            *launched += 1;
        }
    }
    if (J.n_rays <= 0) return cudaGetLastError();
    // emission CDF over cells
    k_rt_lum<<<sms * 8, 256, 0, s>>>(J);
    const int nb = (int)((J.nc + SCAN_BLOCK - 1) / SCAN_BLOCK);
    k_scan_blocks<<<nb, SCAN_BLOCK, 0, s>>>(J.cdf, J.nc, J.scan_sums);
    k_scan_sums<<<1, SCAN_BLOCK, 0, s>>>(J.scan_sums, nb, J.total);
    k_scan_finish<<<nb, SCAN_BLOCK, 0, s>>>(J.cdf, J.nc, J.scan_sums, J.total);
    *launched += 4;
    if ((e = cudaMemcpyAsync(host_total, J.total, sizeof(double), cudaMemcpyDeviceToHost, s)) != cudaSuccess) return e;
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
    if (!(*host_total > 0.0)) return cudaGetLastError();      // no dust emission
    J.eps4pi = *host_total / (double)J.n_rays / (4.0 * CUDART_PI);
    const int grid = (int)std::min<int64_t>((J.n_rays + 255) / 256, (int64_t)sms * 8);
    if (g.type == GRID_CARTESIAN) k_rt_rays<GRID_CARTESIAN><<<grid, 256, 0, s>>>(g, o, J);
    else if (g.type == GRID_CYLINDRICAL) k_rt_rays<GRID_CYLINDRICAL><<<grid, 256, 0, s>>>(g, o, J);
    else k_rt_rays<GRID_SPHERICAL><<<grid, 256, 0, s>>>(g, o, J);
    dim3 sg(o.nobs, (J.nqd + 255) / 256, (unsigned)((J.n_rays + RT_CHUNK - 1) / RT_CHUNK));
    k_rt_sed<<<sg, 256, 0, s>>>(J, o.nobs);
    *launched += 2;
    return cudaGetLastError();
}

}  // namespace hrt
