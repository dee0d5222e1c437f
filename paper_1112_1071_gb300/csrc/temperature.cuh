// Per-cell temperature update (FP64), shared by the single-model and batched kernels.
//
// Sect. 2.3, Eq. 2: Adot = acc / (V dt), dt = 1 s.
// Sect. 2.3, Eq. 3: T from E(T) = Adot on the tabulated E(T_m), bisection + log-log
//   interpolation, clamped (and counted) at the table ends.
// Sect. 2.4, Eqs. 4-5: R = delta(prev, new) = max(prev/new, new/prev); its IEEE-754 bit
//   pattern is the sort key of the nearest-rank select (cells without dust get key 0).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

namespace hrt {

__device__ __forceinline__ double invert_E(double A, const double* __restrict__ E, const double* __restrict__ lnE,
                                           const double* __restrict__ lnT, const double* __restrict__ Tn, int nT,
                                           int& clamp) {
    clamp = 0;
    if (!(A > E[0])) { clamp = -1; return Tn[0]; }
    if (A >= E[nT - 1]) { clamp = 1; return Tn[nT - 1]; }
    int lo = 0, hi = nT - 1;   // E[lo] <= A < E[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (E[mid] <= A) lo = mid; else hi = mid;
    }
    const double f = (log(A) - lnE[lo]) / (lnE[lo + 1] - lnE[lo]);
    return exp(lnT[lo] + f * (lnT[lo + 1] - lnT[lo]));
}

// y(x) linear in log-log on the table (lnx nodes ascending), clamped to the end values.
__device__ __forceinline__ double loglog(double x, const double* __restrict__ lnx, const double* __restrict__ lny,
                                         int n) {
    const double lx = log(x);
    if (!(lx > lnx[0])) return exp(lny[0]);
    if (lx >= lnx[n - 1]) return exp(lny[n - 1]);
    int lo = 0, hi = n - 1;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (lnx[mid] <= lx) lo = mid; else hi = mid;
    }
    const double f = (lx - lnx[lo]) / (lnx[lo + 1] - lnx[lo]);
    return exp(lny[lo] + f * (lny[lo + 1] - lny[lo]));
}

// Table row for re-emission: nearest temperature node in log T, ties to the lower node.
__device__ __forceinline__ int32_t nearest_row(double T, const double* __restrict__ lnT, int nT) {
    const double x = log(T);
    if (x <= lnT[0]) return 0;
    if (x >= lnT[nT - 1]) return nT - 1;
    int lo = 0, hi = nT - 1;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (lnT[mid] <= x) lo = mid; else hi = mid;
    }
    return (lnT[lo + 1] - x) < (x - lnT[lo]) ? lo + 1 : lo;
}

// Update one cell; returns its select key and the clamp (-1 low, +1 high, 0 none) through cl.
__device__ __forceinline__ unsigned long long temperature_cell(double acc, double V, bool dust, int quantity,
                                                               bool first, const double* E, const double* lnE,
                                                               const double* lnT, const double* Tn, int nT,
                                                               double& T, double& adot, int32_t& row, int& cl) {
    const double A = acc / V;                               // Eq. 2 with dt = 1 s
    const double Tnew = invert_E(A, E, lnE, lnT, Tn, nT, cl);   // Eq. 3
    unsigned long long key = 0ull;
    if (dust) {
        double R;
        if (quantity == 0) R = fmax(T / Tnew, Tnew / T);
        else R = first ? __longlong_as_double(0x7ff0000000000000ll) : fmax(adot / A, A / adot);
        if (!(R == R)) R = __longlong_as_double(0x7ff0000000000000ll);   // 0/0: treat as infinite change
        key = (unsigned long long)__double_as_longlong(R);
    } else {
        cl = 0;
    }
    T = Tnew;
    adot = A;
    row = nearest_row(Tnew, lnT, nT);
    return key;
}

}  // namespace hrt
