// A point source's own spectrum (Sect. 2.1.1: every source has a luminosity and a spectrum),
// shared by the device table builder and the host check of the run's inputs.
#pragma once

#include <math.h>

#ifdef __CUDACC__
#define HRT_HD __host__ __device__
#else
#define HRT_HD
#endif

namespace hrt {

// f_nu given at the source's nodes x[0..n-1] (strictly increasing, f >= 0), evaluated at v: a
// power law between two nodes (log-log), a straight line where either value is zero, and zero
// outside the nodes.
HRT_HD inline double user_spectrum(double v, const double* x, const double* f, int n) {
    if (v < x[0] || v > x[n - 1]) return 0.0;
    int lo = 0, hi = n - 1;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (x[mid] <= v) lo = mid; else hi = mid;
    }
    if (f[lo] <= 0.0 || f[lo + 1] <= 0.0) return f[lo] + (f[lo + 1] - f[lo]) * (v - x[lo]) / (x[lo + 1] - x[lo]);
    const double t = log(v / x[lo]) / log(x[lo + 1] / x[lo]);
    return exp((1.0 - t) * log(f[lo]) + t * log(f[lo + 1]));
}

// True when the spectrum has flux at one of the nspec frequencies of the source grid: only
// then does its tabulated in-band part have a luminosity to carry the source's L.
inline bool user_spectrum_has_flux(const double* grid, int nspec, const double* x, const double* f, int n) {
    for (int k = 0; k < nspec; ++k)
        if (user_spectrum(grid[k], x, f, n) > 0.0) return true;
    return false;
}

}  // namespace hrt
