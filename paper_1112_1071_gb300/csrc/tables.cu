// Pre-computed dust and source tables (Sect. 2.1.3: emissivities and Planck means are
// tabulated once; Sect. 2.1.1: packet frequencies reproduce the source spectrum).  Built on
// the device in FP64 when the problem is set up.
//
// E(T_m) = 4 pi int kappa_nu B_nu(T_m) dnu (Eq. 3's left side) by the trapezoid rule over the
// dust frequency nodes; the emissivity row of node m is the normalised cumulative trapezoid
// integral of kappa_nu B_nu(T_m), stored as FP32 for sampling.
#include <math_constants.h>

#include "hrt_internal.h"
#include "planck.cuh"
#include "user_spectrum.h"

namespace hrt {

// one thread per temperature node
__global__ void k_emission_tables(int nnu, const double* __restrict__ nu, const double* __restrict__ kappa, int nT,
                                  const double* __restrict__ T, double* __restrict__ E, double* __restrict__ lnE,
                                  float* __restrict__ cdf) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= nT) return;
    double prev = kappa[0] * planck_bnu(nu[0], T[m]);
    double total = 0.0;
    float* row = cdf + (int64_t)m * nnu;
    row[0] = 0.f;
    // first pass: the total
    for (int k = 1; k < nnu; ++k) {
        const double f = kappa[k] * planck_bnu(nu[k], T[m]);
        total += 0.5 * (f + prev) * (nu[k] - nu[k - 1]);
        prev = f;
    }
    E[m] = 4.0 * CUDART_PI * total;
    lnE[m] = log(E[m]);
    // second pass: normalised running sum
    prev = kappa[0] * planck_bnu(nu[0], T[m]);
    double run = 0.0;
    for (int k = 1; k < nnu; ++k) {
        const double f = kappa[k] * planck_bnu(nu[k], T[m]);
        run += 0.5 * (f + prev) * (nu[k] - nu[k - 1]);
        prev = f;
        row[k] = (float)(run / total);
    }
    row[nnu - 1] = 1.f;
}

cudaError_t launch_emission_tables(int nnu, const double* nu, const double* kappa, int nT, const double* T, double* E,
                                   double* lnE, float* cdf, cudaStream_t s) {
    k_emission_tables<<<(nT + 127) / 128, 128, 0, s>>>(nnu, nu, kappa, nT, T, E, lnE, cdf);
    return cudaGetLastError();
}

// one block per source: the cumulative trapezoid of the spectrum on the source grid,
// normalised so that the in-band part carries all of the luminosity
__global__ void k_source_spectra(int nspec, const double* __restrict__ spec_nu, const double* __restrict__ teff,
                                 const double* __restrict__ user_nu, const double* __restrict__ user_f,
                                 const int* __restrict__ user_off, const int* __restrict__ user_n,
                                 float* __restrict__ spec_cdf) {
    const int s = blockIdx.x;
    if (threadIdx.x != 0) return;
    float* row = spec_cdf + (int64_t)s * nspec;
    auto f_at = [&](int k) -> double {
        if (user_n[s] > 0) return user_spectrum(spec_nu[k], user_nu + user_off[s], user_f + user_off[s], user_n[s]);
        return planck_bnu(spec_nu[k], teff[s]);
    };
    double total = 0.0, prev = f_at(0);
    for (int k = 1; k < nspec; ++k) {
        const double f = f_at(k);
        total += 0.5 * (f + prev) * (spec_nu[k] - spec_nu[k - 1]);
        prev = f;
    }
    row[0] = 0.f;
    double run = 0.0;
    prev = f_at(0);
    for (int k = 1; k < nspec; ++k) {
        const double f = f_at(k);
        run += 0.5 * (f + prev) * (spec_nu[k] - spec_nu[k - 1]);
        prev = f;
        row[k] = total > 0.0 ? (float)(run / total) : (float)k / (float)(nspec - 1);
    }
    row[nspec - 1] = 1.f;
}

cudaError_t launch_source_spectra(int nsrc, int nspec, const double* spec_nu, const double* teff,
                                  const double* user_nu, const double* user_f, const int* user_off, const int* user_n,
                                  float* spec_cdf, cudaStream_t s) {
    if (nsrc <= 0) return cudaSuccess;
    k_source_spectra<<<nsrc, 32, 0, s>>>(nspec, spec_nu, teff, user_nu, user_f, user_off, user_n, spec_cdf);
    return cudaGetLastError();
}

}  // namespace hrt
