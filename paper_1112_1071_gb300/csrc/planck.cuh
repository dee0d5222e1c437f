// The Planck function and its temperature derivative in FP64 (cgs), for the tables built on the
// device: emissivities and E(T) (Eq. 3), Rosseland and Planck means (App. A, the modified
// random walk).
#pragma once
#include <cuda_runtime.h>

namespace hrt {

// cgs, CODATA 2018 exact SI values
constexpr double H_PLANCK = 6.62607015e-27;
constexpr double K_BOLTZ = 1.380649e-16;
constexpr double C_LIGHT = 2.99792458e10;

// B_nu(T) = (2 h nu^3 / c^2) / (exp(h nu / k T) - 1)
__device__ __forceinline__ double planck_bnu(double nu, double T) {
    const double x = H_PLANCK * nu / (K_BOLTZ * T);
    if (x > 700.0) return 0.0;
    return 2.0 * H_PLANCK * nu * nu * nu / (C_LIGHT * C_LIGHT) / expm1(x);
}

// dB_nu/dT = (2 h nu^3 / c^2) (x / T) / (4 sinh^2(x / 2)), x = h nu / k T.
__device__ __forceinline__ double planck_dbdt(double nu, double T) {
    const double x = H_PLANCK * nu / (K_BOLTZ * T);
    if (x > 1400.0) return 0.0;
    const double s = sinh(0.5 * x);
    return 2.0 * H_PLANCK * nu * nu * nu / (C_LIGHT * C_LIGHT) * (x / T) / (4.0 * s * s);
}

}  // namespace hrt
