// Internal definition of the library context (hrt_ctx) shared by the host runtime files.
#pragma once
#include <cuda_runtime.h>

#include <cstdarg>
#include <cstdio>
#include <cstdint>
#include <limits>
#include <string>
#include <vector>

#include "../../include/hrt.h"
#include "hrt_internal.h"

namespace hrt {

constexpr double PI = 3.14159265358979323846;
constexpr double C_LIGHT_CGS = 2.99792458e10;
constexpr int NSPEC = 1000;            // source spectrum nodes over the dust band
constexpr int DEFAULT_NSED = 250;

template <class T>
struct DBuf {
    T* p = nullptr;
    size_t n = 0;
    cudaError_t alloc(size_t count) {
        if (count == n && p) return cudaSuccess;
        release();
        if (count == 0) return cudaSuccess;
        cudaError_t e = cudaMalloc(&p, count * sizeof(T));
        if (e != cudaSuccess) { p = nullptr; return e; }
        n = count;
        return cudaSuccess;
    }
    cudaError_t upload(const T* h, size_t count, cudaStream_t s) {
        cudaError_t e = alloc(count);
        if (e != cudaSuccess || count == 0) return e;
        return cudaMemcpyAsync(p, h, count * sizeof(T), cudaMemcpyHostToDevice, s);
    }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        n = 0;
    }
};

struct PointSrc {
    double x[3];
    double L;
    double teff;
    std::vector<double> unu, uf;
};

// External isotropic source (Sect. 2.1.1): a sphere emitting inwards.
struct ExtSrc {
    double c[3];
    double R;
    double L;
    double teff;
};

}  // namespace hrt

using hrt::DBuf;
using hrt::DEFAULT_NSED;
using hrt::DevDust;
using hrt::DevGrid;
using hrt::DevObs;
using hrt::DevSources;
using hrt::PointSrc;
using hrt::ExtSrc;

struct hrt_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    uint64_t seed = 0;
    uint32_t model_id = 0;
    int iteration = 0;
    std::string err;

    // ---- problem (host copies)
    int gtype = -1;
    int n[3] = {0, 0, 0};
    std::vector<double> w[3];
    double L0 = 1.0;
    std::vector<float> rho;
    int64_t n_dust = 0;
    std::vector<double> nu, chi, alb, Tn;
    double g = 0.0;
    std::vector<PointSrc> pts;
    std::vector<hrt::ExtSrc> ext;
    std::vector<double> Lcell;
    double cell_teff = 0.0;
    int nobs = 0, nsed = DEFAULT_NSED, img_nx = 0, img_ny = 0, nimg = 0;
    double lam_min_um = 0.1, lam_max_um = 1000.0, img_half = 0.0;
    std::vector<double> incl, az, img_lam;
    bool dirty_grid = true, dirty_dust = true, dirty_src = true, dirty_obs = true, have_T = false;

    // ---- device problem
    DBuf<float> d_rhoL, d_w1, d_w2, d_w3, d_rw, d_r2w, d_r2wl, d_thw, d_cth, d_sth, d_phw, d_cph, d_sph;
    DBuf<double> d_rwd, d_cthd, d_sthd, d_va, d_vb, d_vc;
    DBuf<float> d_lnu, d_inv_dlnu, d_lchi, d_alb, d_nuf, d_cdf_emit;
    DBuf<double> d_nu, d_kappa, d_Tn, d_lnT, d_E, d_lnE;
    DBuf<double> d_albd, d_mrw_lnchit, d_mrw_lnkp;   // albedo (FP64); MRW node tables
    DBuf<float> d_mrw_k, d_mrw_kp;                   // MRW per-cell coefficients of the current pass
    DBuf<float> d_src_pos, d_spec_nu, d_spec_cdf;
    DBuf<double> d_src_cdf, d_cell_cdf, d_spec_nud, d_teff, d_unu, d_uf;
    DBuf<int> d_uoff, d_un;
    DBuf<float> d_obs_n, d_obs_ex, d_obs_ey, d_src_col, d_ext_c, d_ext_R;
    DBuf<int32_t> d_img_bin;
    // ---- device state
    DBuf<double> d_T, d_adot, d_acc, d_sed, d_img;
    DBuf<int32_t> d_row;
    DBuf<unsigned long long> d_keys, d_esc, d_counters, d_state;
    DBuf<unsigned int> d_hist;
    DBuf<int32_t> d_abort;
    DBuf<unsigned long long> d_work;            // [0] next packet, [1] launch stamp, [2] peel events queued
    DBuf<uint32_t> d_peel_hist, d_peel_sums, d_peel_order;   // its counting sort by cell
    DBuf<hrt::PeelEvent> d_peel_q;                  // peel-off events of an imaging pass (event kernel)
    DBuf<float> d_report;
    DBuf<unsigned> d_report_count;
    // ---- partial diffusion approximation (App. A)
    DBuf<double> d_chid, d_chiR, d_lnchiR, d_pgeo, d_pda, d_Tprev, d_adotprev, d_pda_scal;
    DBuf<uint32_t> d_visits;
    DBuf<uint8_t> d_pda_state;
    DBuf<unsigned long long> d_pda_count;
    DBuf<int> d_pda_flag;
    bool visits_valid = false;
    // ---- raytracing (Sect. 2.6.3)
    DBuf<float> d_rho, d_rt_qd_w, d_rt_qd_chi, d_rt_qs_w, d_rt_qs_chi, d_rt_inv_dnu, d_rt_col;
    DBuf<int32_t> d_rt_qd_off, d_rt_qd_j, d_rt_qd_bin, d_rt_qs_off, d_rt_qs_j, d_rt_qs_bin, d_rt_row;
    DBuf<double> d_rt_cdf, d_rt_sums, d_rt_total, d_src_L;
    unsigned long long* h_stats = nullptr;   // pinned: counters, clamps, Q key
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};   // start, after propagation, end, before propagation
    double Q_prev = std::numeric_limits<double>::infinity();
    bool have_Q = false;
    double L_tot = 0.0;
    double last_eps = 0.0;
    double acc_scale = 0.0;      // eps L0 of the last Lucy iteration (acc holds sum kappa l, scaled)

    DevGrid grid{};
    DevDust dust{};
    DevSources src{};
    DevObs obs{};

    int fail(int code, const char* fmt, ...) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof(buf), fmt, ap);
        va_end(ap);
        err = buf;
        return code;
    }
    int cuda(cudaError_t e, const char* what) {
        if (e == cudaSuccess) return HRT_OK;
        cudaGetLastError();
        return fail(e == cudaErrorMemoryAllocation ? HRT_ENOMEM : HRT_ECUDA, "%s: %s", what, cudaGetErrorString(e));
    }
    int64_t ncells() const { return (int64_t)n[0] * n[1] * n[2]; }
};

#define CK(call, what)                                   \
    do {                                                 \
        int _rc = ctx->cuda((call), what);               \
        if (_rc != HRT_OK) return _rc;                   \
    } while (0)

namespace hrt {
int prepare_ctx(hrt_ctx* ctx);
}  // namespace hrt
