// Host runtime of libhrt: the C ABI of include/hrt.h.  Owns the device memory of a context,
// validates and stages the problem description, builds the device tables and drives one Lucy
// iteration as a stream-ordered sequence of kernels with a single statistics copy at the end.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <limits>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "../../include/hrt.h"
#include "hrt_internal.h"

using namespace hrt;

#include "ctx_internal.h"
#include "user_spectrum.h"


namespace {

bool finite_all(const double* a, int64_t n) {
    for (int64_t i = 0; i < n; ++i)
        if (!std::isfinite(a[i])) return false;
    return true;
}
// First index in [0, n) where ok(i) fails (n when none) and the number of i with count(i),
// over up to 8 host threads for large arrays (the per-cell checks of a 256^3 grid take tens of
// milliseconds on one core).
template <class Ok, class Count>
void scan_cells(int64_t n, Ok ok, Count count, int64_t& first_bad, int64_t& counted) {
    const int64_t big = (int64_t)1 << 20;
    unsigned nt = std::thread::hardware_concurrency();
    nt = nt < 1 ? 1 : (nt > 8 ? 8 : nt);
    if (n < big || nt == 1) nt = 1;
    std::vector<int64_t> bad(nt, n), cnt(nt, 0);
    auto work = [&](unsigned w) {
        const int64_t b = n * w / nt, e = n * (w + 1) / nt;
        int64_t c = 0;
        for (int64_t i = b; i < e; ++i) {
            if (!ok(i)) {
                bad[w] = i;
                break;
            }
            c += count(i) ? 1 : 0;
        }
        cnt[w] = c;
    };
    if (nt == 1) {
        work(0);
    } else {
        std::vector<std::thread> th;
        for (unsigned w = 1; w < nt; ++w) th.emplace_back(work, w);
        work(0);
        for (auto& t : th) t.join();
    }
    first_bad = n;
    counted = 0;
    for (unsigned w = 0; w < nt; ++w) {
        first_bad = std::min(first_bad, bad[w]);
        counted += cnt[w];
    }
}

bool increasing(const double* a, int64_t n) {
    for (int64_t i = 1; i < n; ++i)
        if (!(a[i] > a[i - 1])) return false;
    return true;
}

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};

// ---------------------------------------------------------------- staging
// rho L0 (density times the scaled unit of length), the walk's per-cell factor, formed in FP64
// and rounded once
__global__ void k_density_scaled(const float* __restrict__ rho, float* __restrict__ rhoL, int64_t n, double L0) {
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (int64_t)gridDim.x * blockDim.x)
        rhoL[c] = (float)((double)rho[c] * L0);
}

int stage_grid(hrt_ctx* ctx) {
    const cudaStream_t s = ctx->stream;
    const int64_t nc = ctx->ncells();
    CK(ctx->d_rho.upload(ctx->rho.data(), nc, s), "upload density");
    CK(ctx->d_rhoL.alloc(nc), "upload density");
    {
        const int64_t blocks = std::min<int64_t>((nc + 255) / 256, 65535 * 8);
        k_density_scaled<<<(unsigned)std::max<int64_t>(blocks, 1), 256, 0, s>>>(ctx->d_rho.p, ctx->d_rhoL.p, nc, ctx->L0);
        CK(cudaGetLastError(), "scale density");
    }
    DevGrid& g = ctx->grid;
    g = DevGrid{};
    g.type = ctx->gtype;
    g.n1 = ctx->n[0]; g.n2 = ctx->n[1]; g.n3 = ctx->n[2];
    g.ncells = nc;
    std::vector<double> va(ctx->n[0]), vb(ctx->n[1]), vc(ctx->n[2]);
    if (ctx->gtype == GRID_CARTESIAN) {
        std::vector<float> ws[3];
        for (int a = 0; a < 3; ++a) {
            ws[a].resize(ctx->w[a].size());
            for (size_t i = 0; i < ws[a].size(); ++i) ws[a][i] = (float)(ctx->w[a][i] / ctx->L0);
        }
        CK(ctx->d_w1.upload(ws[0].data(), ws[0].size(), s), "upload walls");
        CK(ctx->d_w2.upload(ws[1].data(), ws[1].size(), s), "upload walls");
        CK(ctx->d_w3.upload(ws[2].data(), ws[2].size(), s), "upload walls");
        g.w1 = ctx->d_w1.p; g.w2 = ctx->d_w2.p; g.w3 = ctx->d_w3.p;
        for (int i = 0; i < ctx->n[0]; ++i) va[i] = ctx->w[0][i + 1] - ctx->w[0][i];
        for (int j = 0; j < ctx->n[1]; ++j) vb[j] = ctx->w[1][j + 1] - ctx->w[1][j];
        for (int k = 0; k < ctx->n[2]; ++k) vc[k] = ctx->w[2][k + 1] - ctx->w[2][k];
    } else if (ctx->gtype == GRID_CYLINDRICAL) {
        const int nR = ctx->n[0], nz = ctx->n[1], np = ctx->n[2];
        std::vector<float> rw(nR + 1), r2w(nR + 1), r2wl(nR + 1), zw(nz + 1), phw(np + 1), cph(np + 1), sph(np + 1);
        std::vector<double> rwd(nR + 1);
        for (int i = 0; i <= nR; ++i) {
            rwd[i] = ctx->w[0][i] / ctx->L0;
            rw[i] = (float)rwd[i];
            r2w[i] = (float)(rwd[i] * rwd[i]);
            r2wl[i] = (float)(rwd[i] * rwd[i] - (double)r2w[i]);
        }
        for (int j = 0; j <= nz; ++j) zw[j] = (float)(ctx->w[1][j] / ctx->L0);
        for (int k = 0; k <= np; ++k) {
            const double p = ctx->w[2][k];
            phw[k] = (float)p;
            cph[k] = (float)std::cos(p);
            sph[k] = (float)std::sin(p);
        }
        CK(ctx->d_rw.upload(rw.data(), rw.size(), s), "walls");
        CK(ctx->d_r2w.upload(r2w.data(), r2w.size(), s), "walls");
        CK(ctx->d_r2wl.upload(r2wl.data(), r2wl.size(), s), "walls");
        CK(ctx->d_rwd.upload(rwd.data(), rwd.size(), s), "walls");
        CK(ctx->d_w2.upload(zw.data(), zw.size(), s), "walls");
        CK(ctx->d_phw.upload(phw.data(), phw.size(), s), "walls");
        CK(ctx->d_cph.upload(cph.data(), cph.size(), s), "walls");
        CK(ctx->d_sph.upload(sph.data(), sph.size(), s), "walls");
        g.rw = ctx->d_rw.p; g.r2w = ctx->d_r2w.p; g.r2wl = ctx->d_r2wl.p; g.rwd = ctx->d_rwd.p;
        g.w2 = ctx->d_w2.p;
        g.phw = ctx->d_phw.p; g.cph = ctx->d_cph.p; g.sph = ctx->d_sph.p;
        g.r0 = rw[0];
        for (int i = 0; i < nR; ++i) va[i] = 0.5 * (ctx->w[0][i + 1] * ctx->w[0][i + 1] - ctx->w[0][i] * ctx->w[0][i]);
        for (int j = 0; j < nz; ++j) vb[j] = ctx->w[1][j + 1] - ctx->w[1][j];
        for (int k = 0; k < np; ++k) vc[k] = ctx->w[2][k + 1] - ctx->w[2][k];
    } else {
        const int nr = ctx->n[0], nt = ctx->n[1], np = ctx->n[2];
        std::vector<float> rw(nr + 1), r2w(nr + 1), r2wl(nr + 1), thw(nt + 1), cth(nt + 1), sth(nt + 1), phw(np + 1), cph(np + 1),
            sph(np + 1);
        std::vector<double> rwd(nr + 1), cthd(nt + 1), sthd(nt + 1);
        for (int i = 0; i <= nr; ++i) {
            rwd[i] = ctx->w[0][i] / ctx->L0;
            rw[i] = (float)rwd[i];
            r2w[i] = (float)(rwd[i] * rwd[i]);
            r2wl[i] = (float)(rwd[i] * rwd[i] - (double)r2w[i]);
        }
        for (int j = 0; j <= nt; ++j) {
            const double t = ctx->w[1][j];
            double c = std::cos(t), sn = std::sin(t);
            if (std::fabs(c) < 1e-12) c = 0.0;      // the midplane wall is the plane z = 0
            thw[j] = (float)t;
            cthd[j] = c; sthd[j] = sn;
            cth[j] = (float)c; sth[j] = (float)sn;
        }
        for (int k = 0; k <= np; ++k) {
            const double p = ctx->w[2][k];
            phw[k] = (float)p;
            cph[k] = (float)std::cos(p);
            sph[k] = (float)std::sin(p);
        }
        // diffusion-approximation geometry (scaled): r centres and widths, radial walls, sin of
        // the polar centres, polar widths, sin of the polar walls, azimuthal widths
        std::vector<double> geo;
        geo.reserve(3 * nr + 3 * nt + np + 2);
        for (int i = 0; i < nr; ++i) geo.push_back(0.5 * (rwd[i] + rwd[i + 1]));
        for (int i = 0; i < nr; ++i) geo.push_back(rwd[i + 1] - rwd[i]);
        for (int i = 0; i <= nr; ++i) geo.push_back(rwd[i]);
        for (int j = 0; j < nt; ++j) geo.push_back(std::sin(0.5 * (ctx->w[1][j] + ctx->w[1][j + 1])));
        for (int j = 0; j < nt; ++j) geo.push_back(ctx->w[1][j + 1] - ctx->w[1][j]);
        for (int j = 0; j <= nt; ++j) geo.push_back(std::sin(ctx->w[1][j]));
        for (int k = 0; k < np; ++k) geo.push_back(ctx->w[2][k + 1] - ctx->w[2][k]);
        CK(ctx->d_pgeo.upload(geo.data(), geo.size(), s), "pda geometry");
        CK(ctx->d_rw.upload(rw.data(), rw.size(), s), "walls");
        CK(ctx->d_r2w.upload(r2w.data(), r2w.size(), s), "walls");
        CK(ctx->d_r2wl.upload(r2wl.data(), r2wl.size(), s), "walls");
        CK(ctx->d_rwd.upload(rwd.data(), rwd.size(), s), "walls");
        CK(ctx->d_thw.upload(thw.data(), thw.size(), s), "walls");
        CK(ctx->d_cth.upload(cth.data(), cth.size(), s), "walls");
        CK(ctx->d_sth.upload(sth.data(), sth.size(), s), "walls");
        CK(ctx->d_cthd.upload(cthd.data(), cthd.size(), s), "walls");
        CK(ctx->d_sthd.upload(sthd.data(), sthd.size(), s), "walls");
        CK(ctx->d_phw.upload(phw.data(), phw.size(), s), "walls");
        CK(ctx->d_cph.upload(cph.data(), cph.size(), s), "walls");
        CK(ctx->d_sph.upload(sph.data(), sph.size(), s), "walls");
        g.rw = ctx->d_rw.p; g.r2w = ctx->d_r2w.p; g.r2wl = ctx->d_r2wl.p; g.rwd = ctx->d_rwd.p;
        g.thw = ctx->d_thw.p; g.cth = ctx->d_cth.p; g.sth = ctx->d_sth.p; g.cthd = ctx->d_cthd.p; g.sthd = ctx->d_sthd.p;
        g.phw = ctx->d_phw.p; g.cph = ctx->d_cph.p; g.sph = ctx->d_sph.p;
        g.r0 = rw[0];
        // FP64 sphere coefficients in the innermost shell (next to the hole, or around the
        // origin without one) and FP64 cone coefficients for walls within sin(theta) < 0.02 of the
        // axis.  Measured on the flared disk: the same in all shells within 1.25 r_in and for
        // sin(theta) < 0.1 cost 1.3x in walk time, with no change in the parity tests.
        g.r_fp64 = (float)(rwd[1] * (1.0 + 1e-6));
        g.sin_fp64 = 0.02f;
        g.poles = (ctx->w[1][0] <= 1e-12 ? 1 : 0) | (ctx->w[1][nt] >= M_PI - 1e-12 ? 2 : 0);
        for (int i = 0; i < nr; ++i) va[i] = (std::pow(ctx->w[0][i + 1], 3) - std::pow(ctx->w[0][i], 3)) / 3.0;
        for (int j = 0; j < nt; ++j) vb[j] = std::cos(ctx->w[1][j]) - std::cos(ctx->w[1][j + 1]);
        for (int k = 0; k < np; ++k) vc[k] = ctx->w[2][k + 1] - ctx->w[2][k];
    }
    CK(ctx->d_va.upload(va.data(), va.size(), s), "volumes");
    CK(ctx->d_vb.upload(vb.data(), vb.size(), s), "volumes");
    CK(ctx->d_vc.upload(vc.data(), vc.size(), s), "volumes");
    g.rhoL = ctx->d_rhoL.p;
    // per-cell state
    CK(ctx->d_acc.alloc(nc), "alloc acc");
    CK(ctx->d_adot.alloc(nc), "alloc adot");
    CK(ctx->d_row.alloc(nc), "alloc rows");
    CK(ctx->d_keys.alloc(nc), "alloc keys");
    if (!ctx->have_T || ctx->d_T.n != (size_t)nc) {
        std::vector<double> T0(nc, 10.0);   // cold start
        CK(ctx->d_T.upload(T0.data(), nc, s), "upload T");
        CK(cudaMemsetAsync(ctx->d_adot.p, 0, nc * sizeof(double), s), "zero adot");
        ctx->have_T = true;
    }
    ctx->dirty_grid = false;
    return HRT_OK;
}

int stage_dust(hrt_ctx* ctx) {
    const cudaStream_t s = ctx->stream;
    const int nnu = (int)ctx->nu.size(), nT = (int)ctx->Tn.size();
    std::vector<float> lnu(nnu), inv(nnu), lchi(nnu), alb(nnu), nuf(nnu);
    std::vector<double> kappa(nnu), lnT(nT);
    for (int k = 0; k < nnu; ++k) {
        lnu[k] = (float)std::log(ctx->nu[k]);
        lchi[k] = (float)std::log(ctx->chi[k]);
        alb[k] = (float)ctx->alb[k];
        nuf[k] = (float)ctx->nu[k];
        kappa[k] = (1.0 - ctx->alb[k]) * ctx->chi[k];
        inv[k] = k + 1 < nnu ? (float)(1.0 / (std::log(ctx->nu[k + 1]) - std::log(ctx->nu[k]))) : 0.f;
    }
    for (int m = 0; m < nT; ++m) lnT[m] = std::log(ctx->Tn[m]);
    CK(ctx->d_lnu.upload(lnu.data(), nnu, s), "dust");
    CK(ctx->d_inv_dlnu.upload(inv.data(), nnu, s), "dust");
    CK(ctx->d_lchi.upload(lchi.data(), nnu, s), "dust");
    CK(ctx->d_alb.upload(alb.data(), nnu, s), "dust");
    CK(ctx->d_nuf.upload(nuf.data(), nnu, s), "dust");
    CK(ctx->d_nu.upload(ctx->nu.data(), nnu, s), "dust");
    CK(ctx->d_kappa.upload(kappa.data(), nnu, s), "dust");
    CK(ctx->d_chid.upload(ctx->chi.data(), nnu, s), "dust");
    CK(ctx->d_Tn.upload(ctx->Tn.data(), nT, s), "dust");
    CK(ctx->d_lnT.upload(lnT.data(), nT, s), "dust");
    CK(ctx->d_E.alloc(nT), "tables");
    CK(ctx->d_lnE.alloc(nT), "tables");
    CK(ctx->d_cdf_emit.alloc((size_t)nT * nnu), "tables");
    CK(launch_emission_tables(nnu, ctx->d_nu.p, ctx->d_kappa.p, nT, ctx->d_Tn.p, ctx->d_E.p, ctx->d_lnE.p,
                              ctx->d_cdf_emit.p, s),
       "emission tables");
    CK(ctx->d_chiR.alloc(nT), "tables");
    CK(ctx->d_lnchiR.alloc(nT), "tables");
    CK(launch_rosseland(nnu, ctx->d_nu.p, ctx->d_chid.p, nT, ctx->d_Tn.p, ctx->d_chiR.p, ctx->d_lnchiR.p, s),
       "rosseland table");
    CK(ctx->d_albd.upload(ctx->alb.data(), nnu, s), "dust");
    CK(ctx->d_mrw_lnchit.alloc(nT), "tables");
    CK(ctx->d_mrw_lnkp.alloc(nT), "tables");
    CK(launch_mrw_tables(nnu, ctx->d_nu.p, ctx->d_chid.p, ctx->d_kappa.p, ctx->d_albd.p, ctx->g, nT, ctx->d_Tn.p,
                         ctx->d_mrw_lnchit.p, ctx->d_mrw_lnkp.p, s),
       "mrw tables");
    DevDust& d = ctx->dust;
    d.nnu = nnu; d.nT = nT;
    d.lnu = ctx->d_lnu.p; d.inv_dlnu = ctx->d_inv_dlnu.p; d.lchi = ctx->d_lchi.p; d.alb = ctx->d_alb.p;
    d.nu = ctx->d_nuf.p; d.cdf_emit = ctx->d_cdf_emit.p; d.g = (float)ctx->g;
    ctx->dirty_dust = false;
    ctx->dirty_src = true;   // source spectra span the dust band
    return HRT_OK;
}

int stage_sources(hrt_ctx* ctx) {
    const cudaStream_t s = ctx->stream;
    // spectrum grid: NSPEC log-spaced frequencies over the dust band
    std::vector<double> snu(NSPEC);
    const double a = ctx->nu.front(), b = ctx->nu.back();
    for (int k = 0; k < NSPEC; ++k) snu[k] = a * std::pow(b / a, (double)k / (NSPEC - 1));
    snu.front() = a;
    snu.back() = b;
    // a spectrum of a source's own must have flux in the band to carry the source's L
    for (size_t i = 0; i < ctx->pts.size(); ++i) {
        const PointSrc& p = ctx->pts[i];
        if (!p.unu.empty() && !user_spectrum_has_flux(snu.data(), NSPEC, p.unu.data(), p.uf.data(), (int)p.unu.size()))
            return ctx->fail(HRT_EINVAL, "source %zu: its spectrum has no flux in the dust band", i);
    }
    const int npt = (int)ctx->pts.size();
    const int next = (int)ctx->ext.size();
    const bool cell = !ctx->Lcell.empty();
    const int nsrc = npt + next + (cell ? 1 : 0);
    std::vector<double> L(nsrc), teff(nsrc), unu, uf;
    std::vector<int> uoff(nsrc, 0), un(nsrc, 0);
    std::vector<float> pos(3 * std::max(npt, 1), 0.f);
    for (int i = 0; i < npt; ++i) {
        L[i] = ctx->pts[i].L;
        teff[i] = ctx->pts[i].teff;
        for (int a = 0; a < 3; ++a) pos[3 * i + a] = (float)(ctx->pts[i].x[a] / ctx->L0);
        uoff[i] = (int)unu.size();
        un[i] = (int)ctx->pts[i].unu.size();
        unu.insert(unu.end(), ctx->pts[i].unu.begin(), ctx->pts[i].unu.end());
        uf.insert(uf.end(), ctx->pts[i].uf.begin(), ctx->pts[i].uf.end());
    }
    std::vector<float> ec(3 * std::max(next, 1), 0.f), eR(std::max(next, 1), 0.f);
    for (int e = 0; e < next; ++e) {
        L[npt + e] = ctx->ext[e].L;
        teff[npt + e] = ctx->ext[e].teff;
        uoff[npt + e] = (int)unu.size();
        un[npt + e] = 0;
        for (int a = 0; a < 3; ++a) ec[3 * e + a] = (float)(ctx->ext[e].c[a] / ctx->L0);
        eR[e] = (float)(ctx->ext[e].R / ctx->L0);
    }
    CK(ctx->d_ext_c.upload(ec.data(), ec.size(), s), "external sources");
    CK(ctx->d_ext_R.upload(eR.data(), eR.size(), s), "external sources");
    if (cell) {
        double tot = 0.0;
        std::vector<double> cc(ctx->Lcell.size());
        for (size_t c = 0; c < cc.size(); ++c) { tot += ctx->Lcell[c]; cc[c] = tot; }
        for (auto& v : cc) v /= tot;
        cc.back() = 1.0;
        CK(ctx->d_cell_cdf.upload(cc.data(), cc.size(), s), "cell source");
        L[npt + next] = tot;
        teff[npt + next] = ctx->cell_teff;
    }
    double cum = 0.0;
    std::vector<double> cdf(nsrc);
    for (int i = 0; i < nsrc; ++i) { cum += L[i]; cdf[i] = cum; }
    ctx->L_tot = cum;
    for (auto& v : cdf) v /= cum;
    cdf.back() = 1.0;
    std::vector<float> snuf(snu.begin(), snu.end());
    if (unu.empty()) { unu.push_back(0.0); uf.push_back(0.0); }
    CK(ctx->d_src_pos.upload(pos.data(), pos.size(), s), "sources");
    CK(ctx->d_src_cdf.upload(cdf.data(), nsrc, s), "sources");
    CK(ctx->d_spec_nud.upload(snu.data(), NSPEC, s), "sources");
    CK(ctx->d_spec_nu.upload(snuf.data(), NSPEC, s), "sources");
    CK(ctx->d_teff.upload(teff.data(), nsrc, s), "sources");
    CK(ctx->d_unu.upload(unu.data(), unu.size(), s), "sources");
    CK(ctx->d_uf.upload(uf.data(), uf.size(), s), "sources");
    CK(ctx->d_uoff.upload(uoff.data(), nsrc, s), "sources");
    CK(ctx->d_un.upload(un.data(), nsrc, s), "sources");
    CK(ctx->d_spec_cdf.alloc((size_t)nsrc * NSPEC), "sources");
    CK(launch_source_spectra(nsrc, NSPEC, ctx->d_spec_nud.p, ctx->d_teff.p, ctx->d_unu.p, ctx->d_uf.p, ctx->d_uoff.p,
                             ctx->d_un.p, ctx->d_spec_cdf.p, s),
       "source spectra");
    DevSources& S = ctx->src;
    S.npoint = npt; S.nsrc = nsrc; S.nspec = NSPEC;
    S.pos = ctx->d_src_pos.p; S.cdf = ctx->d_src_cdf.p; S.spec_nu = ctx->d_spec_nu.p; S.spec_cdf = ctx->d_spec_cdf.p;
    S.cell_cdf = cell ? ctx->d_cell_cdf.p : nullptr;
    S.col = nullptr;            // set per imaging pass
    S.next = next;
    S.ext_c = ctx->d_ext_c.p;
    S.ext_R = ctx->d_ext_R.p;
    ctx->dirty_src = false;
    return HRT_OK;
}

int stage_observers(hrt_ctx* ctx) {
    const cudaStream_t s = ctx->stream;
    const int no = ctx->nobs;
    std::vector<float> n(3 * std::max(no, 1)), ex(3 * std::max(no, 1)), ey(3 * std::max(no, 1));
    for (int o = 0; o < no; ++o) {
        const double i = ctx->incl[o], p = ctx->az[o];
        const double nn[3] = {std::sin(i) * std::cos(p), std::sin(i) * std::sin(p), std::cos(i)};
        const double e1[3] = {-std::sin(p), std::cos(p), 0.0};
        const double e2[3] = {nn[1] * e1[2] - nn[2] * e1[1], nn[2] * e1[0] - nn[0] * e1[2], nn[0] * e1[1] - nn[1] * e1[0]};
        for (int a = 0; a < 3; ++a) { n[3 * o + a] = (float)nn[a]; ex[3 * o + a] = (float)e1[a]; ey[3 * o + a] = (float)e2[a]; }
    }
    const double lmin = ctx->lam_min_um * 1e-4, lmax = ctx->lam_max_um * 1e-4;
    std::vector<int32_t> ib(std::max(ctx->nimg, 1), -1);
    for (int l = 0; l < ctx->nimg; ++l) {
        const double lam = ctx->img_lam[l] * 1e-4;
        const double x = ctx->nsed * std::log(lam / lmin) / std::log(lmax / lmin);
        ib[l] = (x >= 0 && x < ctx->nsed) ? (int)std::floor(x) : -1;
    }
    CK(ctx->d_obs_n.upload(n.data(), n.size(), s), "observers");
    CK(ctx->d_obs_ex.upload(ex.data(), ex.size(), s), "observers");
    CK(ctx->d_obs_ey.upload(ey.data(), ey.size(), s), "observers");
    CK(ctx->d_img_bin.upload(ib.data(), ib.size(), s), "observers");
    DevObs& O = ctx->obs;
    O.nobs = no; O.nsed = ctx->nsed;
    O.img_nx = ctx->img_nx; O.img_ny = ctx->img_ny; O.nimg = ctx->img_nx > 0 ? ctx->nimg : 0;
    O.n = ctx->d_obs_n.p; O.ex = ctx->d_obs_ex.p; O.ey = ctx->d_obs_ey.p;
    // bin = floor(nsed ln(lambda/lmin)/ln(lmax/lmin)), lambda = c/nu
    const double den = std::log(lmax / lmin);
    O.sed_b = ctx->nsed / den;
    O.sed_a = ctx->nsed * (std::log(C_LIGHT_CGS) - std::log(lmin)) / den;
    O.sed_af = (float)O.sed_a;
    O.sed_bf = (float)O.sed_b;
    O.img_half = (float)(ctx->img_half / ctx->L0);
    O.img_scale = ctx->img_half > 0 ? (float)(ctx->img_nx / (2.0 * ctx->img_half / ctx->L0)) : 0.f;
    O.img_bin = ctx->d_img_bin.p;
    CK(ctx->d_sed.alloc(std::max<size_t>(1, (size_t)no * ctx->nsed)), "sed");
    CK(ctx->d_img.alloc(std::max<size_t>(1, (size_t)no * O.nimg * ctx->img_nx * ctx->img_ny)), "image");
    CK(ctx->d_esc.alloc((size_t)N_ESC_MU * ctx->nsed), "escape");
    ctx->dirty_obs = false;
    return HRT_OK;
}

int prepare(hrt_ctx* ctx) {
    if (ctx->gtype < 0) return ctx->fail(HRT_ESTATE, "grid not set");
    if ((int64_t)ctx->rho.size() != ctx->ncells()) return ctx->fail(HRT_ESTATE, "density not set");
    if (ctx->nu.empty()) return ctx->fail(HRT_ESTATE, "dust not set");
    if (ctx->pts.empty() && ctx->ext.empty() && ctx->Lcell.empty()) return ctx->fail(HRT_ESTATE, "no sources");
    int rc;
    if (ctx->dirty_grid && (rc = stage_grid(ctx)) != HRT_OK) return rc;
    if (ctx->dirty_dust && (rc = stage_dust(ctx)) != HRT_OK) return rc;
    if (ctx->dirty_src && (rc = stage_sources(ctx)) != HRT_OK) return rc;
    if (ctx->dirty_obs && (rc = stage_observers(ctx)) != HRT_OK) return rc;
    ctx->dust.emit_row = ctx->d_row.p;
    CK(ctx->d_counters.alloc(N_COUNTERS + 4), "counters");
    CK(ctx->d_state.alloc(4), "select state");
    CK(ctx->d_hist.alloc(256), "select histogram");
    CK(ctx->d_abort.alloc(1), "abort flag");
    CK(ctx->d_work.alloc(3), "work counter");
    CK(ctx->d_report.alloc(WD_REPORTS * WD_FIELDS), "watchdog report");
    CK(ctx->d_report_count.alloc(1), "watchdog report");
    if (!ctx->h_stats) CK(cudaMallocHost(&ctx->h_stats, sizeof(unsigned long long) * (N_COUNTERS + 8)), "pinned stats");
    for (auto& e : ctx->ev)
        if (!e) CK(cudaEventCreate(&e), "event");
    return HRT_OK;
}

}  // namespace

int hrt::prepare_ctx(hrt_ctx* ctx) {
    DeviceGuard dg(ctx->device);
    return prepare(ctx);
}

// ==================================================================== ABI
extern "C" {

const char* hrt_version(void) { return "hrt 0.1 sm_103a"; }

int hrt_create(hrt_ctx** out, int device, uint64_t seed, void* stream) {
    if (!out) return HRT_EINVAL;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return HRT_ECUDA;
    }
    hrt_ctx* ctx = new (std::nothrow) hrt_ctx();
    if (!ctx) return HRT_ENOMEM;
    ctx->device = device;
    ctx->seed = seed;
    ctx->stream = (cudaStream_t)stream;
    *out = ctx;
    return HRT_OK;
}

int hrt_destroy(hrt_ctx* ctx) {
    if (!ctx) return HRT_EINVAL;
    DeviceGuard dg(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    for (auto* b : {&ctx->d_rhoL, &ctx->d_w1, &ctx->d_w2, &ctx->d_w3, &ctx->d_rw, &ctx->d_r2w, &ctx->d_r2wl,
                    &ctx->d_thw, &ctx->d_cth, &ctx->d_sth, &ctx->d_phw, &ctx->d_cph, &ctx->d_sph, &ctx->d_lnu,
                    &ctx->d_inv_dlnu, &ctx->d_lchi, &ctx->d_alb, &ctx->d_nuf, &ctx->d_cdf_emit, &ctx->d_src_pos,
                    &ctx->d_spec_nu, &ctx->d_spec_cdf, &ctx->d_obs_n, &ctx->d_obs_ex, &ctx->d_obs_ey,
                    &ctx->d_src_col, &ctx->d_ext_c, &ctx->d_ext_R})
        b->release();
    for (auto* b : {&ctx->d_rwd, &ctx->d_cthd, &ctx->d_sthd, &ctx->d_va, &ctx->d_vb, &ctx->d_vc, &ctx->d_nu,
                    &ctx->d_kappa, &ctx->d_Tn, &ctx->d_lnT, &ctx->d_E, &ctx->d_lnE, &ctx->d_src_cdf, &ctx->d_cell_cdf,
                    &ctx->d_spec_nud, &ctx->d_teff, &ctx->d_unu, &ctx->d_uf, &ctx->d_T, &ctx->d_adot, &ctx->d_acc,
                    &ctx->d_sed, &ctx->d_img, &ctx->d_chid, &ctx->d_chiR, &ctx->d_lnchiR, &ctx->d_pgeo, &ctx->d_pda,
                    &ctx->d_Tprev, &ctx->d_adotprev, &ctx->d_pda_scal, &ctx->d_albd, &ctx->d_mrw_lnchit,
                    &ctx->d_mrw_lnkp})
        b->release();
    ctx->d_mrw_k.release(); ctx->d_mrw_kp.release();
    ctx->d_visits.release(); ctx->d_pda_state.release(); ctx->d_pda_count.release(); ctx->d_pda_flag.release();
    for (auto* b : {&ctx->d_rho, &ctx->d_rt_qd_w, &ctx->d_rt_qd_chi, &ctx->d_rt_qs_w, &ctx->d_rt_qs_chi,
                    &ctx->d_rt_inv_dnu, &ctx->d_rt_col})
        b->release();
    for (auto* b : {&ctx->d_rt_qd_off, &ctx->d_rt_qd_j, &ctx->d_rt_qd_bin, &ctx->d_rt_qs_off, &ctx->d_rt_qs_j,
                    &ctx->d_rt_qs_bin, &ctx->d_rt_row})
        b->release();
    for (auto* b : {&ctx->d_rt_cdf, &ctx->d_rt_sums, &ctx->d_rt_total, &ctx->d_src_L}) b->release();
    ctx->d_report.release(); ctx->d_report_count.release();
    ctx->d_uoff.release(); ctx->d_un.release(); ctx->d_img_bin.release(); ctx->d_row.release();
    ctx->d_keys.release(); ctx->d_esc.release(); ctx->d_counters.release(); ctx->d_state.release();
    ctx->d_hist.release(); ctx->d_abort.release(); ctx->d_work.release(); ctx->d_peel_q.release();
    ctx->d_peel_hist.release(); ctx->d_peel_sums.release(); ctx->d_peel_order.release();
    if (ctx->h_stats) cudaFreeHost(ctx->h_stats);
    for (auto e : ctx->ev)
        if (e) cudaEventDestroy(e);
    delete ctx;
    return HRT_OK;
}

const char* hrt_last_error(const hrt_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

int hrt_set_stream(hrt_ctx* ctx, void* stream) {
    if (!ctx) return HRT_EINVAL;
    ctx->stream = (cudaStream_t)stream;
    return HRT_OK;
}

static int set_grid(hrt_ctx* ctx, int type, int n1, int n2, int n3, const double* w1, const double* w2, const double* w3) {
    if (!ctx) return HRT_EINVAL;
    if (n1 < 1 || n2 < 1 || n3 < 1 || !w1 || !w2 || !w3) return ctx->fail(HRT_EINVAL, "grid: empty axis");
    if ((int64_t)n1 * n2 * n3 >= (int64_t)1 << 31) return ctx->fail(HRT_EINVAL, "grid: more than 2^31 cells");
    const double* w[3] = {w1, w2, w3};
    const int n[3] = {n1, n2, n3};
    for (int a = 0; a < 3; ++a)
        if (!finite_all(w[a], n[a] + 1) || !increasing(w[a], n[a] + 1))
            return ctx->fail(HRT_EINVAL, "grid: walls of axis %d not finite and strictly increasing", a);
    if (type == GRID_CYLINDRICAL) {
        if (w1[0] < 0) return ctx->fail(HRT_EINVAL, "grid: negative cylinder radius");
        if (w3[0] != 0.0 || std::fabs(w3[n3] - 2 * PI) > 1e-12) return ctx->fail(HRT_EINVAL, "grid: phi walls must span [0, 2 pi]");
        if (n3 > 1)
            for (int k = 0; k < n3; ++k)
                if (w3[k + 1] - w3[k] > PI + 1e-12) return ctx->fail(HRT_EINVAL, "grid: phi cells wider than pi");
    }
    if (type == GRID_SPHERICAL) {
        if (w1[0] < 0) return ctx->fail(HRT_EINVAL, "grid: negative radius");
        if (w2[0] != 0.0 || std::fabs(w2[n2] - PI) > 1e-12) return ctx->fail(HRT_EINVAL, "grid: theta walls must span [0, pi]");
        if (w3[0] != 0.0 || std::fabs(w3[n3] - 2 * PI) > 1e-12) return ctx->fail(HRT_EINVAL, "grid: phi walls must span [0, 2 pi]");
        if (n3 > 1)
            for (int k = 0; k < n3; ++k)
                if (w3[k + 1] - w3[k] > PI + 1e-12) return ctx->fail(HRT_EINVAL, "grid: phi cells wider than pi");
    }
    ctx->gtype = type;
    double L0 = 0.0;
    for (int a = 0; a < 3; ++a) {
        ctx->n[a] = n[a];
        ctx->w[a].assign(w[a], w[a] + n[a] + 1);
        if (type == GRID_CARTESIAN || a == 0 || (type == GRID_CYLINDRICAL && a == 1))
            L0 = std::max(L0, std::max(std::fabs(w[a][0]), std::fabs(w[a][n[a]])));
    }
    if (type == GRID_SPHERICAL) {
        ctx->w[1].back() = PI;
        ctx->w[2].back() = 2 * PI;
    }
    if (type == GRID_CYLINDRICAL) ctx->w[2].back() = 2 * PI;
    ctx->L0 = L0 > 0 ? L0 : 1.0;
    ctx->rho.clear();
    ctx->Lcell.clear();
    ctx->have_T = false;
    ctx->have_Q = false;
    ctx->dirty_grid = ctx->dirty_src = ctx->dirty_obs = true;
    return HRT_OK;
}

int hrt_set_grid_cartesian(hrt_ctx* ctx, int nx, int ny, int nz, const double* xw, const double* yw, const double* zw) {
    return set_grid(ctx, GRID_CARTESIAN, nx, ny, nz, xw, yw, zw);
}

int hrt_set_grid_spherical(hrt_ctx* ctx, int nr, int nt, int np, const double* rw, const double* tw, const double* pw) {
    return set_grid(ctx, GRID_SPHERICAL, nr, nt, np, rw, tw, pw);
}

int hrt_set_grid_cylindrical(hrt_ctx* ctx, int nR, int nz, int np, const double* Rw, const double* zw, const double* pw) {
    return set_grid(ctx, GRID_CYLINDRICAL, nR, nz, np, Rw, zw, pw);
}

int hrt_set_density(hrt_ctx* ctx, const float* rho, int64_t n) {
    if (!ctx) return HRT_EINVAL;
    if (ctx->gtype < 0) return ctx->fail(HRT_ESTATE, "density before grid");
    if (!rho || n != ctx->ncells()) return ctx->fail(HRT_EINVAL, "density: expected %lld cells", (long long)ctx->ncells());
    int64_t nd = 0, bad = n;
    scan_cells(n, [&](int64_t c) { return std::isfinite(rho[c]) && rho[c] >= 0.f; },
               [&](int64_t c) { return rho[c] > 0.f; }, bad, nd);
    if (bad < n) return ctx->fail(HRT_EINVAL, "density: cell %lld not finite and >= 0", (long long)bad);
    ctx->rho.assign(rho, rho + n);
    ctx->n_dust = nd;
    ctx->dirty_grid = true;
    return HRT_OK;
}

int hrt_set_dust(hrt_ctx* ctx, int nnu, const double* nu, const double* chi, const double* albedo, double g, int nT,
                 const double* T) {
    if (!ctx) return HRT_EINVAL;
    if (nnu < 2 || nT < 2 || !nu || !chi || !albedo || !T) return ctx->fail(HRT_EINVAL, "dust: need >= 2 nodes");
    if (!finite_all(nu, nnu) || !increasing(nu, nnu) || nu[0] <= 0) return ctx->fail(HRT_EINVAL, "dust: nu must increase");
    for (int k = 0; k < nnu; ++k)
        if (!(chi[k] > 0) || !std::isfinite(chi[k]) || !(albedo[k] >= 0 && albedo[k] <= 1))
            return ctx->fail(HRT_EINVAL, "dust: chi > 0 and albedo in [0,1] required (node %d)", k);
    if (!(g > -1 && g < 1)) return ctx->fail(HRT_EINVAL, "dust: g outside (-1, 1)");
    if (!finite_all(T, nT) || !increasing(T, nT) || T[0] <= 0) return ctx->fail(HRT_EINVAL, "dust: T nodes must increase");
    ctx->nu.assign(nu, nu + nnu);
    ctx->chi.assign(chi, chi + nnu);
    ctx->alb.assign(albedo, albedo + nnu);
    ctx->Tn.assign(T, T + nT);
    ctx->g = g;
    ctx->dirty_dust = true;
    ctx->dirty_src = true;
    return HRT_OK;
}

static int add_point(hrt_ctx* ctx, const double x[3], double L, double teff, int n, const double* nu, const double* f) {
    if (!ctx) return HRT_EINVAL;
    if (!x || !finite_all(x, 3)) return ctx->fail(HRT_EINVAL, "source: position not finite");
    if (!(L > 0) || !std::isfinite(L)) return ctx->fail(HRT_EINVAL, "source: L must be > 0");
    if (ctx->gtype < 0) return ctx->fail(HRT_ESTATE, "source before grid");
    if (ctx->gtype == GRID_CARTESIAN) {
        for (int a = 0; a < 3; ++a)
            if (x[a] < ctx->w[a].front() || x[a] > ctx->w[a].back()) return ctx->fail(HRT_EINVAL, "source outside the grid");
    } else if (ctx->gtype == GRID_CYLINDRICAL) {       // inside the outer cylinder, between the end planes
        if (std::hypot(x[0], x[1]) >= ctx->w[0].back() || x[2] < ctx->w[1].front() || x[2] > ctx->w[1].back())
            return ctx->fail(HRT_EINVAL, "source outside the grid");
    } else if (std::sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]) >= ctx->w[0].back()) {
        return ctx->fail(HRT_EINVAL, "source outside the grid");
    }
    PointSrc p;
    for (int a = 0; a < 3; ++a) p.x[a] = x[a];
    p.L = L;
    p.teff = teff;
    if (n > 0) {
        if (!nu || !f || n < 2 || !finite_all(nu, n) || !increasing(nu, n) || !(nu[0] > 0) || !finite_all(f, n))
            return ctx->fail(HRT_EINVAL, "source spectrum: frequencies must be finite, > 0 and increasing");
        for (int k = 0; k < n; ++k)
            if (f[k] < 0) return ctx->fail(HRT_EINVAL, "source spectrum negative");
        p.unu.assign(nu, nu + n);
        p.uf.assign(f, f + n);
    } else if (!(teff > 0) || !std::isfinite(teff)) {
        return ctx->fail(HRT_EINVAL, "source: Teff must be finite and > 0");
    }
    ctx->pts.push_back(p);
    ctx->dirty_src = true;
    return HRT_OK;
}

int hrt_add_point_source(hrt_ctx* ctx, const double x[3], double L, double Teff) {
    return add_point(ctx, x, L, Teff, 0, nullptr, nullptr);
}

int hrt_add_point_source_spectrum(hrt_ctx* ctx, const double x[3], double L, int n, const double* nu, const double* fnu) {
    if (n < 2) return ctx ? ctx->fail(HRT_EINVAL, "source spectrum needs >= 2 nodes") : HRT_EINVAL;
    return add_point(ctx, x, L, 0.0, n, nu, fnu);
}

int hrt_set_cell_source(hrt_ctx* ctx, const double* Lcell, int64_t n, double Teff) {
    if (!ctx) return HRT_EINVAL;
    if (ctx->gtype < 0) return ctx->fail(HRT_ESTATE, "cell source before grid");
    if (!Lcell || n != ctx->ncells()) return ctx->fail(HRT_EINVAL, "cell source: expected %lld cells", (long long)ctx->ncells());
    if (!(Teff > 0)) return ctx->fail(HRT_EINVAL, "cell source: Teff must be > 0");
    double tot = 0.0;
    for (int64_t c = 0; c < n; ++c) {
        if (!(Lcell[c] >= 0) || !std::isfinite(Lcell[c])) return ctx->fail(HRT_EINVAL, "cell source: L must be finite >= 0");
        tot += Lcell[c];
    }
    if (!(tot > 0)) return ctx->fail(HRT_EINVAL, "cell source: zero luminosity");
    ctx->Lcell.assign(Lcell, Lcell + n);
    ctx->cell_teff = Teff;
    ctx->dirty_src = true;
    return HRT_OK;
}

int hrt_add_external_source(hrt_ctx* ctx, const double c[3], double radius, double L, double Teff) {
    if (!ctx) return HRT_EINVAL;
    if (ctx->gtype < 0) return ctx->fail(HRT_ESTATE, "external source before grid");
    if (!c || !std::isfinite(c[0]) || !std::isfinite(c[1]) || !std::isfinite(c[2]))
        return ctx->fail(HRT_EINVAL, "external source: centre not finite");
    if (!(radius > 0) || !std::isfinite(radius)) return ctx->fail(HRT_EINVAL, "external source: radius must be > 0");
    if (!(L > 0) || !std::isfinite(L)) return ctx->fail(HRT_EINVAL, "external source: L must be > 0");
    if (!(Teff > 0) || !std::isfinite(Teff)) return ctx->fail(HRT_EINVAL, "external source: Teff must be > 0");
    ExtSrc e;
    for (int a = 0; a < 3; ++a) e.c[a] = c[a];
    e.R = radius;
    e.L = L;
    e.teff = Teff;
    ctx->ext.push_back(e);
    ctx->dirty_src = true;
    return HRT_OK;
}

int hrt_clear_sources(hrt_ctx* ctx) {
    if (!ctx) return HRT_EINVAL;
    ctx->pts.clear();
    ctx->ext.clear();
    ctx->Lcell.clear();
    ctx->dirty_src = true;
    return HRT_OK;
}

int hrt_set_peeloff(hrt_ctx* ctx, int nobs, const double* incl, const double* az, int nsed, double lam_min_um,
                    double lam_max_um, int img_nx, int img_ny, double img_half_extent_cm, int nimg, const double* img_lam_um) {
    if (!ctx) return HRT_EINVAL;
    if (nobs < 0 || (nobs > 0 && (!incl || !az))) return ctx->fail(HRT_EINVAL, "peeloff: observers");
    if (nsed < 1 || !(lam_min_um > 0) || !(lam_max_um > lam_min_um) || !std::isfinite(lam_max_um))
        return ctx->fail(HRT_EINVAL, "peeloff: SED bins");
    if (img_nx < 0 || img_ny < 0 ||
        (img_nx > 0 && (img_ny < 1 || !(img_half_extent_cm > 0) || !std::isfinite(img_half_extent_cm) || nimg < 1 ||
                        !img_lam_um)))
        return ctx->fail(HRT_EINVAL, "peeloff: image");
    if (img_nx > 0)
        for (int l = 0; l < nimg; ++l)
            if (!(img_lam_um[l] > 0) || !std::isfinite(img_lam_um[l]))
                return ctx->fail(HRT_EINVAL, "peeloff: image wavelength %d must be finite and > 0", l);
    if (nobs > 0 && (!finite_all(incl, nobs) || !finite_all(az, nobs))) return ctx->fail(HRT_EINVAL, "peeloff: angles");
    ctx->nobs = nobs;
    ctx->incl.assign(incl, incl + nobs);
    ctx->az.assign(az, az + nobs);
    ctx->nsed = nsed;
    ctx->lam_min_um = lam_min_um;
    ctx->lam_max_um = lam_max_um;
    ctx->img_nx = img_nx;
    ctx->img_ny = img_ny;
    ctx->img_half = img_half_extent_cm;
    ctx->nimg = img_nx > 0 ? nimg : 0;
    ctx->img_lam.assign(img_lam_um, img_lam_um + ctx->nimg);
    ctx->dirty_obs = true;
    return HRT_OK;
}

void hrt_default_params(hrt_run_params* p) {
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->max_interactions = 1000000;
    p->peel = 0;
    p->update_temperature = 1;
    p->terminate_on_absorb = 0;
    p->quantity = 0;
    p->p = 0.99;
    p->q_thres = 1.02;
    p->delta_thres = std::numeric_limits<double>::infinity();
    p->kernel = HRT_KERNEL_EVENT;
    p->watchdog_ms = 0.0;
}

// Quadrature of the SED bins for raytracing (Sect. 2.6.3): each bin (log-spaced in wavelength) is
// cut at the nodes of the emission pdf and of the extinction; 3-point Gauss-Legendre in nu on each
// piece; chi log-log between the dust nodes in FP64.  off[b]..off[b+1] are the nodes of bin b.
static void rt_quadrature(const hrt_ctx* ctx, const std::vector<double>& pnodes, std::vector<int32_t>& off,
                          std::vector<int32_t>& jv, std::vector<int32_t>& bin, std::vector<float>& wv,
                          std::vector<float>& chiv) {
    const int nsed = ctx->nsed;
    const double lmin = ctx->lam_min_um * 1e-4, lmax = ctx->lam_max_um * 1e-4;
    std::vector<double> brk(pnodes);
    brk.insert(brk.end(), ctx->nu.begin(), ctx->nu.end());
    std::sort(brk.begin(), brk.end());
    brk.erase(std::unique(brk.begin(), brk.end()), brk.end());
    const double gx[3] = {-std::sqrt(0.6), 0.0, std::sqrt(0.6)}, gw[3] = {5.0 / 9.0, 8.0 / 9.0, 5.0 / 9.0};
    const int nn = (int)ctx->nu.size(), np = (int)pnodes.size();
    off.assign(nsed + 1, 0);
    jv.clear(); bin.clear(); wv.clear(); chiv.clear();
    for (int b = 0; b < nsed; ++b) {
        const double nu_lo = C_LIGHT_CGS / (lmin * std::pow(lmax / lmin, (double)(b + 1) / nsed));
        const double nu_hi = C_LIGHT_CGS / (lmin * std::pow(lmax / lmin, (double)b / nsed));
        off[b] = (int32_t)wv.size();
        std::vector<double> cuts{nu_lo};
        for (double x : brk)
            if (x > nu_lo && x < nu_hi) cuts.push_back(x);
        cuts.push_back(nu_hi);
        for (size_t c = 0; c + 1 < cuts.size(); ++c) {
            const double mid = 0.5 * (cuts[c] + cuts[c + 1]), half = 0.5 * (cuts[c + 1] - cuts[c]);
            for (int g = 0; g < 3; ++g) {
                const double x = mid + half * gx[g];
                int j = (int)(std::upper_bound(pnodes.begin(), pnodes.end(), x) - pnodes.begin()) - 1;
                j = std::min(std::max(j, 0), np - 2);
                int k = (int)(std::upper_bound(ctx->nu.begin(), ctx->nu.end(), x) - ctx->nu.begin()) - 1;
                k = std::min(std::max(k, 0), nn - 2);
                double t = std::log(x / ctx->nu[k]) / std::log(ctx->nu[k + 1] / ctx->nu[k]);
                t = std::min(std::max(t, 0.0), 1.0);
                const double chi = std::exp((1 - t) * std::log(ctx->chi[k]) + t * std::log(ctx->chi[k + 1]));
                jv.push_back(j);
                bin.push_back(b);
                wv.push_back((float)(half * gw[g]));
                chiv.push_back((float)chi);
            }
        }
    }
    off[nsed] = (int32_t)wv.size();
}

int hrt_run_iteration(hrt_ctx* ctx, int64_t n_packets, const hrt_run_params* params, hrt_iter_stats* out) {
    if (!ctx) return HRT_EINVAL;
    hrt_run_params P;
    if (params) P = *params;
    else hrt_default_params(&P);
    if (n_packets < 1 || n_packets > 0xFFFFFFFFll) return ctx->fail(HRT_EINVAL, "n_packets must be in [1, 2^32)");
    if (!(P.p > 0 && P.p <= 1)) return ctx->fail(HRT_EINVAL, "percentile p must be in (0, 1]");
    if (P.max_interactions < 0) return ctx->fail(HRT_EINVAL, "max_interactions < 0");
    if (P.pda_min_visits < 0 || P.pda_min_visits > 0xFFFFFFFFll)
        return ctx->fail(HRT_EINVAL, "pda_min_visits must be in [0, 2^32)");
    if (P.raytrace_rays < 0 || P.raytrace_rays > 0xFFFFFFFFll)
        return ctx->fail(HRT_EINVAL, "raytrace_rays must be in [0, 2^32)");
    if (!(P.mrw_gamma >= 0) || !std::isfinite(P.mrw_gamma))
        return ctx->fail(HRT_EINVAL, "mrw_gamma must be finite and >= 0");
    if (P.peel_queue_events < 0) return ctx->fail(HRT_EINVAL, "peel_queue_events must be >= 0");
    if (P.kernel != HRT_KERNEL_EVENT && P.kernel != HRT_KERNEL_PLAIN && P.kernel != HRT_KERNEL_REGROUP)
        return ctx->fail(HRT_EINVAL, "unknown kernel");
    if (P.quantity != 0 && P.quantity != 1) return ctx->fail(HRT_EINVAL, "quantity must be 0 (T) or 1 (Adot)");
    if (P.block_size != 0 && P.block_size != 256)
        return ctx->fail(HRT_EINVAL, "block_size must be 0 or 256 (the kernels are compiled for 256 threads)");
    if (P.blocks_per_sm < 0 || P.regroup_threshold < 0 || P.regroup_threshold > 32)
        return ctx->fail(HRT_EINVAL, "blocks_per_sm >= 0 and regroup_threshold in [0, 32] required");
    if (!(P.watchdog_ms >= 0) || !std::isfinite(P.watchdog_ms)) return ctx->fail(HRT_EINVAL, "watchdog_ms must be finite and >= 0");
    if (std::isnan(P.q_thres) || std::isnan(P.delta_thres)) return ctx->fail(HRT_EINVAL, "convergence thresholds are NaN");
    const int64_t n_total = P.n_total > 0 ? P.n_total : n_packets;
    if (P.first_packet < 0 || P.n_total < 0 || n_total > 0x100000000ll || P.first_packet + n_packets > n_total)
        return ctx->fail(HRT_EINVAL, "packet share: need 0 <= first_packet, first_packet + n_packets <= n_total <= 2^32");
    DeviceGuard dg(ctx->device);
    int rc = prepare(ctx);
    if (rc != HRT_OK) return rc;
    const cudaStream_t s = ctx->stream;
    const int64_t nc = ctx->ncells();
    int launched = 0;
    CK(cudaEventRecord(ctx->ev[0], s), "event");
    if (P.update_temperature) CK(cudaMemsetAsync(ctx->d_acc.p, 0, nc * sizeof(double), s), "zero acc");
    // re-emission rows from the temperatures this pass uses (every pass: the temperatures may
    // have been set since the last update)
    CK(launch_emit_rows(ctx->d_T.p, ctx->d_row.p, nc, ctx->d_lnT.p, (int)ctx->Tn.size(), s), "emission rows");
    launched++;
    const bool mrw = P.mrw_gamma > 0;
    if (mrw) {
        // modified random walk coefficients at the same temperatures
        CK(ctx->d_mrw_k.alloc(nc), "alloc mrw");
        CK(ctx->d_mrw_kp.alloc(nc), "alloc mrw");
        CK(launch_mrw_cells(nc, ctx->grid.rhoL, ctx->d_T.p, ctx->d_lnT.p, ctx->d_mrw_lnchit.p, ctx->d_mrw_lnkp.p,
                            (int)ctx->Tn.size(), ctx->d_mrw_k.p, ctx->d_mrw_kp.p, s),
           "mrw coefficients");
        launched++;
    }
    if (P.peel) {
        CK(cudaMemsetAsync(ctx->d_sed.p, 0, ctx->d_sed.n * sizeof(double), s), "zero sed");
        CK(cudaMemsetAsync(ctx->d_img.p, 0, ctx->d_img.n * sizeof(double), s), "zero image");
    }
    CK(cudaMemsetAsync(ctx->d_esc.p, 0, ctx->d_esc.n * sizeof(unsigned long long), s), "zero escape");
    CK(cudaMemsetAsync(ctx->d_counters.p, 0, ctx->d_counters.n * sizeof(unsigned long long), s), "zero counters");
    CK(cudaMemsetAsync(ctx->d_abort.p, 0, sizeof(int32_t), s), "zero abort");
    CK(cudaMemsetAsync(ctx->d_work.p, 0, ctx->d_work.n * sizeof(unsigned long long), s), "zero work");
    CK(cudaMemsetAsync(ctx->d_report_count.p, 0, sizeof(unsigned), s), "zero report");

    PropagateJob job;
    job.grid = ctx->grid;
    job.dust = ctx->dust;
    job.src = ctx->src;
    job.obs = ctx->obs;
    // the acc buffer is written only by Lucy iterations; an imaging pass writes a scratch copy
    job.tal.acc = ctx->d_acc.p;
    job.tal.sed = ctx->d_sed.p;
    job.tal.img = ctx->d_img.p;
    job.tal.esc = ctx->d_esc.p;
    job.tal.counters = ctx->d_counters.p;
    job.tal.abort_flag = ctx->d_abort.p;
    job.tal.report = ctx->d_report.p;
    job.tal.report_count = ctx->d_report_count.p;
    // packet entries per cell, for the diffusion approximation of this Lucy iteration
    const bool pda = P.pda_min_visits > 0 && P.update_temperature && ctx->gtype == GRID_SPHERICAL;
    job.tal.visits = nullptr;
    if (pda) {
        CK(ctx->d_visits.alloc(nc), "alloc visits");
        CK(cudaMemsetAsync(ctx->d_visits.p, 0, nc * sizeof(uint32_t), s), "zero visits");
        job.tal.visits = ctx->d_visits.p;
    }
    RunArgs& A = job.args;
    A = RunArgs{};
    A.n_packets = n_packets;
    A.first_packet = P.first_packet;
    A.key0 = (uint32_t)(ctx->seed & 0xFFFFFFFFu);
    A.key1 = (uint32_t)(ctx->seed >> 32);
    A.iter_key = P.update_temperature ? (uint32_t)ctx->iteration : (0x80000000u | (uint32_t)ctx->iteration);
    A.model_key = ctx->model_id;
    A.eps = ctx->L_tot / (double)n_total;
    ctx->last_eps = A.eps;
    A.epsL0 = A.eps * ctx->L0;
    A.max_interactions = P.max_interactions;
    A.peel = P.peel && ctx->nobs > 0;
    const bool raytrace = A.peel && !P.update_temperature && P.raytrace_rays > 0;
    A.rt = raytrace ? 1 : 0;
    A.terminate_on_absorb = P.terminate_on_absorb;
    A.mrw_gamma = mrw ? (float)P.mrw_gamma : 0.f;
    A.mrw_k = mrw ? ctx->d_mrw_k.p : nullptr;
    A.mrw_kp = mrw ? ctx->d_mrw_kp.p : nullptr;
    A.budget_ns = P.watchdog_ms > 0 ? (uint64_t)(P.watchdog_ms * 1e6) : 0ull;
    A.smem_sed = (size_t)ctx->obs.nobs * ctx->obs.nsed * 8 + (size_t)N_ESC_MU * ctx->obs.nsed * 4 <= 96 * 1024;
    A.work_counter = ctx->d_work.p;
    A.t0 = ctx->d_work.p + 1;
    Launch L;
    L.block = P.block_size > 0 ? P.block_size : 256;
    L.blocks_per_sm = P.blocks_per_sm;
    L.regroup = P.regroup_threshold;
    if (!P.update_temperature) {
        // imaging pass: deposits go to a scratch buffer (the key buffer), the Lucy accumulators are kept
        job.tal.acc = reinterpret_cast<double*>(ctx->d_keys.p);
        CK(cudaMemsetAsync(ctx->d_keys.p, 0, nc * sizeof(double), s), "zero scratch");
    }
    CK(launch_stamp(ctx->d_work.p + 1, s), "stamp");
    launched++;
    const bool columns = A.peel && ctx->src.npoint > 0;
    if (columns) CK(ctx->d_src_col.alloc((size_t)ctx->src.npoint * ctx->obs.nobs), "source columns");
    CK(cudaEventRecord(ctx->ev[3], s), "event");
    job.src.col = nullptr;
    if (columns) {
        CK(launch_source_columns(job.grid, job.src, job.obs, ctx->d_src_col.p, s), "source columns");
        job.src.col = ctx->d_src_col.p;
        launched++;
    }
    if (A.peel && P.kernel != HRT_KERNEL_PLAIN) {
        // queue for the peel pass: two events per packet (an overflow is peeled inline), at most
        // 2^27 events (4 GiB of 32-byte records)
        const int64_t cap = P.peel_queue_events > 0
                                ? std::min<int64_t>(P.peel_queue_events, (int64_t)1 << 27)
                                : std::min<int64_t>(std::max<int64_t>(2 * n_packets, (int64_t)1 << 20), (int64_t)1 << 27);
        if (ctx->d_peel_q.n < (size_t)cap) CK(ctx->d_peel_q.alloc((size_t)cap), "peel queue");
        job.args.peel_q = ctx->d_peel_q.p;
        job.args.peel_n = ctx->d_work.p + 2;
        job.args.peel_cap = cap;
    }
    cudaError_t e = P.kernel == HRT_KERNEL_PLAIN ? launch_propagate_plain(job, L, s, &launched)
                    : (P.kernel == HRT_KERNEL_REGROUP && regroup_supported(job)) ? launch_propagate_regroup(job, L, s, &launched)
                                                                            : launch_propagate_event(job, L, s, &launched);
    CK(e, "propagate");
    if (job.args.peel_q) {
        const size_t nk = (size_t)nc + 1;
        if (ctx->d_peel_hist.n < nk) CK(ctx->d_peel_hist.alloc(nk), "peel sort");
        if (ctx->d_peel_sums.n < nk / 1024 + 1) CK(ctx->d_peel_sums.alloc(nk / 1024 + 1), "peel sort");
        if (ctx->d_peel_order.n < ctx->d_peel_q.n) CK(ctx->d_peel_order.alloc(ctx->d_peel_q.n), "peel sort");
        CK(launch_peel_pass(job, ctx->d_peel_hist.p, ctx->d_peel_sums.p, ctx->d_peel_order.p, s, &launched), "peel pass");
    }
    CK(cudaEventRecord(ctx->ev[1], s), "event");
    if (raytrace) {
        std::vector<int32_t> qd_off, qd_j, qd_bin, qs_off, qs_j, qs_bin;
        std::vector<float> qd_w, qd_chi, qs_w, qs_chi;
        rt_quadrature(ctx, ctx->nu, qd_off, qd_j, qd_bin, qd_w, qd_chi);
        std::vector<double> snu(NSPEC);
        const double a0 = ctx->nu.front(), a1 = ctx->nu.back();
        for (int k = 0; k < NSPEC; ++k) snu[k] = a0 * std::pow(a1 / a0, (double)k / (NSPEC - 1));
        snu.front() = a0;
        snu.back() = a1;
        rt_quadrature(ctx, snu, qs_off, qs_j, qs_bin, qs_w, qs_chi);
        std::vector<float> inv(ctx->nu.size());
        for (size_t k = 0; k + 1 < ctx->nu.size(); ++k) inv[k] = (float)(1.0 / (ctx->nu[k + 1] - ctx->nu[k]));
        const int npt = (int)ctx->pts.size();
        std::vector<double> Ls(std::max(npt, 1), 0.0);
        for (int i = 0; i < npt; ++i) Ls[i] = ctx->pts[i].L;
        CK(ctx->d_rt_qd_off.upload(qd_off.data(), qd_off.size(), s), "raytrace");
        CK(ctx->d_rt_qd_j.upload(qd_j.data(), qd_j.size(), s), "raytrace");
        CK(ctx->d_rt_qd_bin.upload(qd_bin.data(), qd_bin.size(), s), "raytrace");
        CK(ctx->d_rt_qd_w.upload(qd_w.data(), qd_w.size(), s), "raytrace");
        CK(ctx->d_rt_qd_chi.upload(qd_chi.data(), qd_chi.size(), s), "raytrace");
        CK(ctx->d_rt_qs_off.upload(qs_off.data(), qs_off.size(), s), "raytrace");
        CK(ctx->d_rt_qs_j.upload(qs_j.data(), qs_j.size(), s), "raytrace");
        CK(ctx->d_rt_qs_bin.upload(qs_bin.data(), qs_bin.size(), s), "raytrace");
        CK(ctx->d_rt_qs_w.upload(qs_w.data(), qs_w.size(), s), "raytrace");
        CK(ctx->d_rt_qs_chi.upload(qs_chi.data(), qs_chi.size(), s), "raytrace");
        CK(ctx->d_rt_inv_dnu.upload(inv.data(), inv.size(), s), "raytrace");
        CK(ctx->d_src_L.upload(Ls.data(), Ls.size(), s), "raytrace");
        CK(ctx->d_rt_cdf.alloc(nc), "raytrace");
        CK(ctx->d_rt_sums.alloc(nc / 1024 + 2), "raytrace");
        CK(ctx->d_rt_total.alloc(1), "raytrace");
        CK(ctx->d_rt_col.alloc((size_t)P.raytrace_rays * ctx->nobs), "raytrace");
        CK(ctx->d_rt_row.alloc((size_t)P.raytrace_rays), "raytrace");
        RtJob J;
        std::memset(&J, 0, sizeof(J));
        J.n1 = ctx->n[0]; J.n2 = ctx->n[1]; J.n3 = ctx->n[2];
        J.nc = nc;
        J.rho = ctx->d_rho.p;
        J.va = ctx->d_va.p; J.vb = ctx->d_vb.p; J.vc = ctx->d_vc.p;
        J.T = ctx->d_T.p;
        J.lnT = ctx->d_lnT.p; J.lnE = ctx->d_lnE.p;
        J.nT = (int)ctx->Tn.size();
        J.nnu = (int)ctx->nu.size();
        J.emit_row = ctx->d_row.p;
        J.cdf_emit = ctx->d_cdf_emit.p;
        J.inv_dnu = ctx->d_rt_inv_dnu.p;
        J.qd_off = ctx->d_rt_qd_off.p; J.qd_j = ctx->d_rt_qd_j.p; J.qd_bin = ctx->d_rt_qd_bin.p;
        J.qd_w = ctx->d_rt_qd_w.p; J.qd_chi = ctx->d_rt_qd_chi.p; J.nqd = (int)qd_w.size();
        J.qs_off = ctx->d_rt_qs_off.p; J.qs_j = ctx->d_rt_qs_j.p; J.qs_bin = ctx->d_rt_qs_bin.p;
        J.qs_w = ctx->d_rt_qs_w.p; J.qs_chi = ctx->d_rt_qs_chi.p; J.nqs = (int)qs_w.size();
        J.nsed = ctx->nsed;
        J.npoint = npt;
        J.src_col = job.src.col;
        J.src_pos = ctx->d_src_pos.p;
        J.src_L = ctx->d_src_L.p;
        J.spec_cdf = ctx->d_spec_cdf.p;
        J.spec_nu = ctx->d_spec_nud.p;
        J.nspec = NSPEC;
        J.n_rays = P.raytrace_rays;
        J.key0 = A.key0; J.key1 = A.key1;
        J.iter_key = 0x40000000u | (uint32_t)ctx->iteration;
        J.model_key = A.model_key;
        J.cdf = ctx->d_rt_cdf.p; J.scan_sums = ctx->d_rt_sums.p; J.total = ctx->d_rt_total.p;
        J.col = ctx->d_rt_col.p; J.row = ctx->d_rt_row.p;
        J.sed = ctx->d_sed.p; J.img = ctx->d_img.p;
        J.counters = ctx->d_counters.p;
        double Ldust = 0.0;
        CK(run_raytrace(ctx->grid, ctx->obs, J, &Ldust, s, &launched), "raytrace");
    }
    const int64_t k_rank = ctx->n_dust > 0 ? (nc - ctx->n_dust) + (int64_t)std::ceil(P.p * (double)ctx->n_dust) - 1 : 0;
    PdaStats pda_stats{0, 0, 0.0};
    if (P.update_temperature) {
        TemperatureJob tj;
        tj.gtype = ctx->gtype;
        tj.n1 = ctx->n[0]; tj.n2 = ctx->n[1]; tj.n3 = ctx->n[2];
        tj.ncells = nc;
        tj.rhoL = ctx->d_rhoL.p;
        tj.acc = ctx->d_acc.p;
        tj.acc_scale = A.epsL0;
        ctx->acc_scale = A.epsL0;
        tj.va = ctx->d_va.p; tj.vb = ctx->d_vb.p; tj.vc = ctx->d_vc.p;
        tj.E = ctx->d_E.p; tj.lnE = ctx->d_lnE.p; tj.lnT = ctx->d_lnT.p; tj.Tn = ctx->d_Tn.p;
        tj.nT = (int)ctx->Tn.size();
        tj.quantity = P.quantity;
        tj.first = ctx->iteration == 0 ? 1 : 0;
        tj.T = ctx->d_T.p;
        tj.adot = ctx->d_adot.p;
        tj.emit_row = ctx->d_row.p;
        tj.keys = ctx->d_keys.p;
        tj.counters = ctx->d_counters.p + N_COUNTERS;
        if (pda) {
            CK(ctx->d_Tprev.alloc(nc), "alloc pda");
            CK(ctx->d_adotprev.alloc(nc), "alloc pda");
            CK(cudaMemcpyAsync(ctx->d_Tprev.p, ctx->d_T.p, nc * 8, cudaMemcpyDeviceToDevice, s), "pda copy");
            CK(cudaMemcpyAsync(ctx->d_adotprev.p, ctx->d_adot.p, nc * 8, cudaMemcpyDeviceToDevice, s), "pda copy");
        }
        CK(launch_temperature(tj, s, &launched), "temperature");
        if (pda) {
            CK(ctx->d_pda.alloc((size_t)15 * nc), "alloc pda");
            CK(ctx->d_pda_state.alloc(nc), "alloc pda");
            CK(ctx->d_pda_scal.alloc(8), "alloc pda");
            CK(ctx->d_pda_count.alloc(1), "alloc pda");
            CK(ctx->d_pda_flag.alloc(1), "alloc pda");
            PdaJob J;
            J.n1 = ctx->n[0]; J.n2 = ctx->n[1]; J.n3 = ctx->n[2];
            J.nc = nc;
            J.rhoL = ctx->d_rhoL.p;
            const double* gp = ctx->d_pgeo.p;
            J.rc = gp; gp += J.n1;
            J.dr = gp; gp += J.n1;
            J.rface = gp; gp += J.n1 + 1;
            J.stc = gp; gp += J.n2;
            J.dth = gp; gp += J.n2;
            J.stf = gp; gp += J.n2 + 1;
            J.dph = gp;
            J.visits = ctx->d_visits.p;
            J.n_min = (uint32_t)P.pda_min_visits;
            J.T_prev = ctx->d_Tprev.p;
            J.adot_prev = ctx->d_adotprev.p;
            J.T = ctx->d_T.p; J.adot = ctx->d_adot.p; J.row = ctx->d_row.p; J.keys = ctx->d_keys.p;
            J.lnT = ctx->d_lnT.p; J.lnE = ctx->d_lnE.p; J.lnchiR = ctx->d_lnchiR.p;
            J.nT = (int)ctx->Tn.size();
            J.quantity = P.quantity;
            J.first = ctx->iteration == 0 ? 1 : 0;
            J.state = ctx->d_pda_state.p;
            double* w = ctx->d_pda.p;
            J.dtau = w; w += 3 * nc;
            J.W = w; w += 6 * nc;
            J.x = w; w += nc;
            J.r = w; w += nc;
            J.p = w; w += nc;
            J.q = w; w += nc;
            J.b = w; w += nc;
            J.dg = w;
            J.scal = ctx->d_pda_scal.p;
            J.count = ctx->d_pda_count.p;
            J.flag = ctx->d_pda_flag.p;
            int hflag = 0;
            double hscal[8];
            CK(run_pda(J, 1e-12, 100000, &hflag, hscal, &pda_stats, s, &launched), "diffusion approximation");
        }
        if (ctx->n_dust > 0) {
            int kk = std::max<int64_t>(0, std::min<int64_t>(k_rank, nc - 1));
            CK(launch_select_kth(ctx->d_keys.p, nc, (unsigned long long)kk, ctx->d_hist.p, ctx->d_state.p,
                                 ctx->d_counters.p + N_COUNTERS + 2, s, &launched),
               "quantile");
        }
    }
    CK(cudaMemcpyAsync(ctx->h_stats, ctx->d_counters.p, sizeof(unsigned long long) * (N_COUNTERS + 4),
                       cudaMemcpyDeviceToHost, s),
       "stats copy");
    CK(cudaEventRecord(ctx->ev[2], s), "event");
    CK(cudaStreamSynchronize(s), "iteration");
    const unsigned long long* h = ctx->h_stats;
    hrt_iter_stats st;
    std::memset(&st, 0, sizeof(st));
    st.iteration = ctx->iteration;
    st.n_packets = n_packets;
    st.e_emitted = n_total == n_packets ? ctx->L_tot : A.eps * (double)n_packets;
    st.e_escaped = (double)h[C_ESCAPED] * A.eps;
    st.e_killed = (double)h[C_KILLED] * A.eps;
    st.e_absorbed = (double)h[C_ABSORBED_TERM] * A.eps;
    st.n_interactions = (int64_t)h[C_INTERACTIONS];
    st.n_scatter = (int64_t)h[C_SCATTER];
    st.n_absorb = (int64_t)h[C_ABSORB];
    st.n_crossings = (int64_t)h[C_CROSSINGS];
    st.n_peel_crossings = (int64_t)h[C_PEEL_CROSSINGS];
    st.n_killed = (int64_t)h[C_KILLED];
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ctx->ev[3], ctx->ev[1]);
    st.ms_propagate = ms;
    cudaEventElapsedTime(&ms, ctx->ev[0], ctx->ev[2]);
    st.ms_total = ms;
    st.kernel_launches = launched;
    st.n_pda = pda_stats.n_cells;
    st.n_mrw = (int64_t)h[C_MRW];
    st.pda_iterations = pda_stats.iterations;
    st.pda_residual = pda_stats.residual;
    if (P.update_temperature) ctx->visits_valid = pda;
    const double inf = std::numeric_limits<double>::infinity();
    st.Q = inf;
    st.Delta = inf;
    if (P.update_temperature) {
        st.clamp_low = (int64_t)h[N_COUNTERS];
        st.clamp_high = (int64_t)h[N_COUNTERS + 1];
        if (ctx->n_dust > 0) {
            unsigned long long key = h[N_COUNTERS + 2];
            double Q;
            std::memcpy(&Q, &key, sizeof(Q));
            st.Q = Q;
            st.Delta = ctx->have_Q && std::isfinite(ctx->Q_prev) && std::isfinite(Q)
                           ? std::max(ctx->Q_prev / Q, Q / ctx->Q_prev)
                           : inf;
            ctx->Q_prev = Q;
            ctx->have_Q = true;
        }
        st.converged = (st.Q < P.q_thres) && (st.Delta < P.delta_thres || std::isinf(P.delta_thres)) ? 1 : 0;
        ctx->iteration++;
    }
    if (out) *out = st;
    if (h[C_WATCHDOG] > 0) return ctx->fail(HRT_ETIMEDOUT, "propagation watchdog expired after %.3f ms", P.watchdog_ms);
    return HRT_OK;
}

// ---------------------------------------------------------------- read-out / state
static int get_dev(hrt_ctx* ctx, const void* src, size_t bytes_avail, void* dst, size_t bytes, bool to_host) {
    if (!dst) return ctx->fail(HRT_EINVAL, "null output");
    if (bytes > bytes_avail || !src) return ctx->fail(HRT_ESTATE, "nothing to read (run an iteration first)");
    DeviceGuard dg(ctx->device);
    CK(cudaMemcpyAsync(dst, src, bytes, to_host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, ctx->stream), "copy");
    if (to_host) CK(cudaStreamSynchronize(ctx->stream), "copy");
    return HRT_OK;
}

int64_t hrt_num_cells(const hrt_ctx* ctx) { return ctx ? ctx->ncells() : -1; }

int hrt_get_temperature(hrt_ctx* ctx, double* out, int64_t n) {
    if (!ctx) return HRT_EINVAL;
    if (n < ctx->ncells()) return ctx->fail(HRT_EINVAL, "output shorter than the cell count");
    return get_dev(ctx, ctx->d_T.p, ctx->d_T.n * 8, out, ctx->ncells() * 8, true);
}
int hrt_get_temperature_device(hrt_ctx* ctx, double* out, int64_t n) {
    if (!ctx) return HRT_EINVAL;
    if (n < ctx->ncells()) return ctx->fail(HRT_EINVAL, "output shorter than the cell count");
    return get_dev(ctx, ctx->d_T.p, ctx->d_T.n * 8, out, ctx->ncells() * 8, false);
}
int hrt_get_specific_energy(hrt_ctx* ctx, double* out, int64_t n) {
    if (!ctx) return HRT_EINVAL;
    if (n < ctx->ncells()) return ctx->fail(HRT_EINVAL, "output shorter than the cell count");
    return get_dev(ctx, ctx->d_adot.p, ctx->d_adot.n * 8, out, ctx->ncells() * 8, true);
}
int hrt_get_absorbed(hrt_ctx* ctx, double* out, int64_t n) {
    if (!ctx) return HRT_EINVAL;
    if (n < ctx->ncells()) return ctx->fail(HRT_EINVAL, "output shorter than the cell count");
    const int rc = get_dev(ctx, ctx->d_acc.p, ctx->d_acc.n * 8, out, ctx->ncells() * 8, true);
    if (rc != HRT_OK) return rc;
    for (int64_t c = 0; c < ctx->ncells(); ++c) out[c] *= ctx->acc_scale;   // sum eps kappa l in cgs
    return HRT_OK;
}
int hrt_get_sed(hrt_ctx* ctx, double* out, int64_t n) {
    if (!ctx) return HRT_EINVAL;
    const int64_t m = (int64_t)ctx->nobs * ctx->nsed;
    if (n < m) return ctx->fail(HRT_EINVAL, "output shorter than nobs*nsed");
    return get_dev(ctx, ctx->d_sed.p, ctx->d_sed.n * 8, out, m * 8, true);
}
int hrt_get_sed_device(hrt_ctx* ctx, double* out, int64_t n) {
    if (!ctx) return HRT_EINVAL;
    const int64_t m = (int64_t)ctx->nobs * ctx->nsed;
    if (n < m) return ctx->fail(HRT_EINVAL, "output shorter than nobs*nsed");
    return get_dev(ctx, ctx->d_sed.p, ctx->d_sed.n * 8, out, m * 8, false);
}
int hrt_get_image(hrt_ctx* ctx, double* out, int64_t n) {
    if (!ctx) return HRT_EINVAL;
    const int64_t m = (int64_t)ctx->nobs * ctx->nimg * ctx->img_nx * ctx->img_ny;
    if (n < m) return ctx->fail(HRT_EINVAL, "output shorter than the image");
    if (m == 0) return HRT_OK;
    return get_dev(ctx, ctx->d_img.p, ctx->d_img.n * 8, out, m * 8, true);
}
int hrt_get_escape(hrt_ctx* ctx, double* out, int64_t n) {
    if (!ctx) return HRT_EINVAL;
    const int64_t m = (int64_t)N_ESC_MU * ctx->nsed;
    if (n < m) return ctx->fail(HRT_EINVAL, "output shorter than 10*nsed");
    std::vector<unsigned long long> cnt(m);
    int rc = get_dev(ctx, ctx->d_esc.p, ctx->d_esc.n * 8, cnt.data(), m * 8, true);
    if (rc != HRT_OK) return rc;
    // counts of escaping packets times the packet energy of the last call
    for (int64_t i = 0; i < m; ++i) out[i] = (double)cnt[i] * ctx->last_eps;
    return HRT_OK;
}

int hrt_set_temperature(hrt_ctx* ctx, const double* T, int64_t n) {
    if (!ctx) return HRT_EINVAL;
    if (ctx->gtype < 0 || (int64_t)ctx->rho.size() != ctx->ncells()) return ctx->fail(HRT_ESTATE, "set grid and density first");
    if (!T || n != ctx->ncells()) return ctx->fail(HRT_EINVAL, "temperature: expected %lld cells", (long long)ctx->ncells());
    {
        int64_t bad = n, unused = 0;
        scan_cells(n, [&](int64_t c) { return T[c] > 0 && std::isfinite(T[c]); }, [](int64_t) { return false; },
                   bad, unused);
        if (bad < n) return ctx->fail(HRT_EINVAL, "temperature must be finite > 0");
    }
    DeviceGuard dg(ctx->device);
    if (ctx->dirty_grid) {
        int rc = stage_grid(ctx);
        if (rc != HRT_OK) return rc;
    }
    CK(ctx->d_T.upload(T, n, ctx->stream), "upload T");
    CK(cudaStreamSynchronize(ctx->stream), "upload T");
    ctx->have_T = true;
    return HRT_OK;
}

int hrt_set_temperature_device(hrt_ctx* ctx, const double* d_T, int64_t n) {
    if (!ctx) return HRT_EINVAL;
    if (ctx->gtype < 0 || (int64_t)ctx->rho.size() != ctx->ncells()) return ctx->fail(HRT_ESTATE, "set grid and density first");
    if (!d_T || n != ctx->ncells()) return ctx->fail(HRT_EINVAL, "temperature: expected %lld cells", (long long)ctx->ncells());
    DeviceGuard dg(ctx->device);
    if (ctx->dirty_grid) {
        int rc = stage_grid(ctx);
        if (rc != HRT_OK) return rc;
    }
    CK(cudaMemcpyAsync(ctx->d_T.p, d_T, n * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream), "copy T");
    ctx->have_T = true;
    return HRT_OK;
}

int hrt_get_watchdog_report(hrt_ctx* ctx, float* out, int64_t n) {
    if (!ctx || !out) return HRT_EINVAL;
    if (n < (int64_t)WD_REPORTS * WD_FIELDS) return ctx->fail(HRT_EINVAL, "report needs %d floats", WD_REPORTS * WD_FIELDS);
    if (!ctx->d_report.p) return 0;
    DeviceGuard dg(ctx->device);
    unsigned cnt = 0;
    CK(cudaMemcpyAsync(&cnt, ctx->d_report_count.p, sizeof(unsigned), cudaMemcpyDeviceToHost, ctx->stream), "report");
    CK(cudaMemcpyAsync(out, ctx->d_report.p, sizeof(float) * WD_REPORTS * WD_FIELDS, cudaMemcpyDeviceToHost, ctx->stream),
       "report");
    CK(cudaStreamSynchronize(ctx->stream), "report");
    return (int)(cnt < (unsigned)WD_REPORTS ? cnt : (unsigned)WD_REPORTS);
}

int hrt_set_iteration(hrt_ctx* ctx, int iteration) {
    if (!ctx || iteration < 0) return HRT_EINVAL;
    ctx->iteration = iteration;
    return HRT_OK;
}

int hrt_set_specific_energy(hrt_ctx* ctx, const double* adot, int64_t n) {
    if (!ctx) return HRT_EINVAL;
    if (ctx->gtype < 0 || (int64_t)ctx->rho.size() != ctx->ncells()) return ctx->fail(HRT_ESTATE, "set grid and density first");
    if (!adot || n != ctx->ncells())
        return ctx->fail(HRT_EINVAL, "specific energy: expected %lld cells", (long long)ctx->ncells());
    for (int64_t c = 0; c < n; ++c)
        if (!(adot[c] >= 0) || !std::isfinite(adot[c])) return ctx->fail(HRT_EINVAL, "specific energy must be finite >= 0");
    DeviceGuard dg(ctx->device);
    if (ctx->dirty_grid) {
        int rc = stage_grid(ctx);
        if (rc != HRT_OK) return rc;
    }
    CK(ctx->d_adot.upload(adot, n, ctx->stream), "upload adot");
    CK(cudaStreamSynchronize(ctx->stream), "upload adot");
    return HRT_OK;
}

int hrt_set_convergence_state(hrt_ctx* ctx, int have_Q, double Q_prev) {
    if (!ctx) return HRT_EINVAL;
    if (have_Q && !(Q_prev >= 1.0)) return ctx->fail(HRT_EINVAL, "Q_prev must be >= 1 (a ratio max(a/b, b/a)) or +inf");
    ctx->have_Q = have_Q != 0;
    ctx->Q_prev = have_Q ? Q_prev : std::numeric_limits<double>::infinity();
    return HRT_OK;
}

int hrt_get_convergence_state(hrt_ctx* ctx, int* have_Q, double* Q_prev) {
    if (!ctx || !have_Q || !Q_prev) return HRT_EINVAL;
    *have_Q = ctx->have_Q ? 1 : 0;
    *Q_prev = ctx->Q_prev;
    return HRT_OK;
}

int hrt_set_model_id(hrt_ctx* ctx, uint32_t model_id) {
    if (!ctx) return HRT_EINVAL;
    ctx->model_id = model_id;
    return HRT_OK;
}

// ---------------------------------------------------------------- single steps
int hrt_step_philox(int64_t n, const uint32_t* d_ctr, const uint32_t* d_key, uint32_t* d_out, void* stream) {
    if (n < 0 || (n > 0 && (!d_ctr || !d_key || !d_out))) return HRT_EINVAL;
    cudaError_t e = launch_step_philox(n, d_ctr, d_key, d_out, (cudaStream_t)stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
    return e == cudaSuccess ? HRT_OK : HRT_ECUDA;
}

static int step_prepare(hrt_ctx* ctx) {
    if (!ctx) return HRT_EINVAL;
    DeviceGuard dg(ctx->device);
    return prepare(ctx);
}

int hrt_step_cell_exit(hrt_ctx* ctx, int64_t n, const float* d_pos, const float* d_dir, const int32_t* d_cell,
                       float* d_dist, int32_t* d_exit) {
    int rc = step_prepare(ctx);
    if (rc != HRT_OK) return rc;
    DeviceGuard dg(ctx->device);
    CK(launch_step_cell_exit(ctx->grid, n, d_pos, d_dir, d_cell, d_dist, d_exit, (float)(1.0 / ctx->L0), (float)ctx->L0,
                             ctx->stream),
       "cell exit");
    CK(cudaStreamSynchronize(ctx->stream), "cell exit");
    return HRT_OK;
}

int hrt_step_wall_distance(hrt_ctx* ctx, int64_t n, const float* d_pos, const int32_t* d_cell, float* d_dist) {
    int rc = step_prepare(ctx);
    if (rc != HRT_OK) return rc;
    if (n < 0 || (n > 0 && (!d_pos || !d_cell || !d_dist))) return ctx->fail(HRT_EINVAL, "wall distance: bad arguments");
    DeviceGuard dg(ctx->device);
    CK(launch_step_wall_distance(ctx->grid, n, d_pos, d_cell, d_dist, (float)(1.0 / ctx->L0), (float)ctx->L0,
                                 ctx->stream),
       "wall distance");
    CK(cudaStreamSynchronize(ctx->stream), "wall distance");
    return HRT_OK;
}

int hrt_step_mrw_path(int64_t n, const float* d_tau0, const float* d_zeta, float* d_out, void* stream) {
    if (n < 0 || (n > 0 && (!d_tau0 || !d_zeta || !d_out))) return HRT_EINVAL;
    cudaError_t e = launch_step_mrw_path(n, d_tau0, d_zeta, d_out, (cudaStream_t)stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
    return e == cudaSuccess ? HRT_OK : HRT_ECUDA;
}

int hrt_step_tau_to_edge(hrt_ctx* ctx, int64_t n, const float* d_pos, const float* d_dir, const float* d_nu, float* d_tau) {
    int rc = step_prepare(ctx);
    if (rc != HRT_OK) return rc;
    DeviceGuard dg(ctx->device);
    CK(launch_step_tau(ctx->grid, ctx->dust, n, d_pos, d_dir, d_nu, d_tau, (float)(1.0 / ctx->L0), ctx->stream), "tau");
    CK(cudaStreamSynchronize(ctx->stream), "tau");
    return HRT_OK;
}

int hrt_step_hg_scatter(hrt_ctx* ctx, int64_t n, const float* d_dir_in, const float* d_u1, const float* d_u2,
                        float* d_dir_out) {
    if (!ctx) return HRT_EINVAL;
    if (ctx->nu.empty()) return ctx->fail(HRT_ESTATE, "dust not set");
    DeviceGuard dg(ctx->device);
    CK(launch_step_hg((float)ctx->g, n, d_dir_in, d_u1, d_u2, d_dir_out, ctx->stream), "hg");
    CK(cudaStreamSynchronize(ctx->stream), "hg");
    return HRT_OK;
}

int hrt_step_sample_emission(hrt_ctx* ctx, int64_t n, const int32_t* d_row, const float* d_u, float* d_nu) {
    int rc = step_prepare(ctx);
    if (rc != HRT_OK) return rc;
    DeviceGuard dg(ctx->device);
    CK(launch_step_sample(ctx->dust.nu, ctx->dust.cdf_emit, ctx->dust.nnu, n, d_row, d_u, d_nu, ctx->stream), "sample");
    CK(cudaStreamSynchronize(ctx->stream), "sample");
    return HRT_OK;
}

int hrt_step_sample_source(hrt_ctx* ctx, int64_t n, const int32_t* d_src, const float* d_u, float* d_nu) {
    int rc = step_prepare(ctx);
    if (rc != HRT_OK) return rc;
    DeviceGuard dg(ctx->device);
    CK(launch_step_sample(ctx->src.spec_nu, ctx->src.spec_cdf, ctx->src.nspec, n, d_src, d_u, d_nu, ctx->stream), "sample");
    CK(cudaStreamSynchronize(ctx->stream), "sample");
    return HRT_OK;
}

int hrt_step_temperature(hrt_ctx* ctx, int64_t n, const double* d_adot, double* d_T) {
    int rc = step_prepare(ctx);
    if (rc != HRT_OK) return rc;
    DeviceGuard dg(ctx->device);
    CK(launch_invert_temperature(d_adot, d_T, n, ctx->d_E.p, ctx->d_lnE.p, ctx->d_lnT.p, ctx->d_Tn.p,
                                 (int)ctx->Tn.size(), ctx->stream),
       "temperature");
    CK(cudaStreamSynchronize(ctx->stream), "temperature");
    return HRT_OK;
}

int hrt_get_visits(hrt_ctx* ctx, uint32_t* out, int64_t n) {
    if (!ctx || !out) return HRT_EINVAL;
    if (!ctx->visits_valid) return ctx->fail(HRT_ESTATE, "no packet entries counted: run a Lucy iteration with pda_min_visits > 0");
    if (n != ctx->ncells()) return ctx->fail(HRT_EINVAL, "visits: n must equal the number of cells");
    DeviceGuard dg(ctx->device);
    CK(cudaMemcpyAsync(out, ctx->d_visits.p, n * sizeof(uint32_t), cudaMemcpyDeviceToHost, ctx->stream), "visits");
    CK(cudaStreamSynchronize(ctx->stream), "visits");
    return HRT_OK;
}

int hrt_get_rosseland(hrt_ctx* ctx, double* out, int64_t n) {
    int rc = step_prepare(ctx);
    if (rc != HRT_OK) return rc;
    if (!out || n < (int64_t)ctx->Tn.size()) return ctx->fail(HRT_EINVAL, "rosseland: output too short");
    DeviceGuard dg(ctx->device);
    CK(cudaMemcpyAsync(out, ctx->d_chiR.p, ctx->Tn.size() * 8, cudaMemcpyDeviceToHost, ctx->stream), "rosseland");
    CK(cudaStreamSynchronize(ctx->stream), "rosseland");
    return HRT_OK;
}

int hrt_get_tables(hrt_ctx* ctx, double* E, int64_t nE, float* cdf, int64_t ncdf) {
    int rc = step_prepare(ctx);
    if (rc != HRT_OK) return rc;
    const int64_t nT = (int64_t)ctx->Tn.size(), nnu = (int64_t)ctx->nu.size();
    if (nE < nT || ncdf < nT * nnu || !E || !cdf) return ctx->fail(HRT_EINVAL, "table outputs too short");
    DeviceGuard dg(ctx->device);
    CK(cudaMemcpyAsync(E, ctx->d_E.p, nT * 8, cudaMemcpyDeviceToHost, ctx->stream), "tables");
    CK(cudaMemcpyAsync(cdf, ctx->d_cdf_emit.p, nT * nnu * 4, cudaMemcpyDeviceToHost, ctx->stream), "tables");
    CK(cudaStreamSynchronize(ctx->stream), "tables");
    return HRT_OK;
}

}  // extern "C"
