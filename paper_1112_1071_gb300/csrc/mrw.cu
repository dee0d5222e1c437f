// Tables of the modified random walk (Sect. 2.2), FP64 on the temperature nodes, and the
// per-cell coefficients a pass reads (FP32, at the temperatures the pass starts from):
//   chi_t(T)  = int dB/dT dnu / int chi_nu^-1 (1 - albedo_nu g)^-1 dB/dT dnu   (Rosseland mean of
//               the transport extinction: the diffusion coefficient D = 1 / (3 rho chi_t)),
//   kappa_P(T) = int kappa_nu B_nu dnu / int B_nu dnu   (absorption per unit path length of a field
//               thermalised at T: the deposit of a step, Eq. 2),
// trapezoid rule over the dust nodes; per cell log-log between the nodes, clamped at the ends.
#include "hrt_internal.h"
#include "planck.cuh"
#include "temperature.cuh"

namespace hrt {

// one thread per temperature node
__global__ void k_mrw_tables(int nnu, const double* __restrict__ nu, const double* __restrict__ chi,
                             const double* __restrict__ kappa, const double* __restrict__ alb, double g, int nT,
                             const double* __restrict__ T, double* __restrict__ ln_chit, double* __restrict__ ln_kp) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= nT) return;
    double num = 0.0, den = 0.0, kb = 0.0, bb = 0.0;
    double w0 = planck_dbdt(nu[0], T[m]), b0 = planck_bnu(nu[0], T[m]);
    double it0 = 1.0 / (chi[0] * (1.0 - alb[0] * g));
    for (int k = 1; k < nnu; ++k) {
        const double w1 = planck_dbdt(nu[k], T[m]), b1 = planck_bnu(nu[k], T[m]);
        const double it1 = 1.0 / (chi[k] * (1.0 - alb[k] * g));
        const double h = 0.5 * (nu[k] - nu[k - 1]);
        num += (w1 + w0) * h;
        den += (w1 * it1 + w0 * it0) * h;
        kb += (kappa[k] * b1 + kappa[k - 1] * b0) * h;
        bb += (b1 + b0) * h;
        w0 = w1; b0 = b1; it0 = it1;
    }
    ln_chit[m] = log(num / den);
    ln_kp[m] = log(kb / bb);
}

cudaError_t launch_mrw_tables(int nnu, const double* nu, const double* chi, const double* kappa, const double* alb,
                              double g, int nT, const double* T, double* ln_chit, double* ln_kp, cudaStream_t s) {
    k_mrw_tables<<<(nT + 127) / 128, 128, 0, s>>>(nnu, nu, chi, kappa, alb, g, nT, T, ln_chit, ln_kp);
    return cudaGetLastError();
}

// k[c] = rhoL[c] chi_t(T_c) (inverse transport mean free path per scaled length; 0 without dust),
// kp[c] = kappa_P(T_c)
__global__ void k_mrw_cells(int64_t n, const float* __restrict__ rhoL, const double* __restrict__ T,
                            const double* __restrict__ lnT, const double* __restrict__ ln_chit,
                            const double* __restrict__ ln_kp, int nT, float* __restrict__ k, float* __restrict__ kp) {
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (int64_t)gridDim.x * blockDim.x) {
        const float rho = rhoL[c];
        const double Tc = T[c];
        k[c] = rho > 0.f ? (float)((double)rho * loglog(Tc, lnT, ln_chit, nT)) : 0.f;
        kp[c] = (float)loglog(Tc, lnT, ln_kp, nT);
    }
}

cudaError_t launch_mrw_cells(int64_t n, const float* rhoL, const double* T, const double* lnT, const double* ln_chit,
                             const double* ln_kp, int nT, float* k, float* kp, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t want = (n + 255) / 256;
    const int blocks = (int)(want < (int64_t)sms * 8 ? want : (int64_t)sms * 8);
    k_mrw_cells<<<blocks, 256, 0, s>>>(n, rhoL, T, lnT, ln_chit, ln_kp, nT, k, kp);
    return cudaGetLastError();
}

}  // namespace hrt
