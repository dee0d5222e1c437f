// Host-side declarations shared by the library's translation units (not part of the ABI).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "hrt_types.h"

namespace hrt {

// Launch shape of a propagation kernel.
struct Launch {
    int block = 256;
    int blocks = 0;          // 0: blocks_per_sm * SMs
    int blocks_per_sm = 0;   // 0: occupancy limit
    int regroup = 0;         // event kernel regroup threshold (lanes)
};

// Device-side view of one model plus the launch parameters of one propagation pass.
struct PropagateJob {
    DevGrid grid;
    DevDust dust;
    DevSources src;
    DevObs obs;
    Tallies tal;
    RunArgs args;
};

// propagate.cu
cudaError_t launch_stamp(unsigned long long* t0, cudaStream_t s);
cudaError_t launch_propagate_plain(const PropagateJob& job, const Launch& l, cudaStream_t s, int* launched);
cudaError_t launch_source_columns(const DevGrid& g, const DevSources& src, const DevObs& o, float* col,
                                  cudaStream_t s);
cudaError_t launch_propagate_event(const PropagateJob& job, const Launch& l, cudaStream_t s, int* launched);
// regroup.cu: the event kernel with packets regrouped by state across a block's warps (not for
// modified-random-walk runs; see regroup_supported)
bool regroup_supported(const PropagateJob& job);
cudaError_t launch_propagate_regroup(const PropagateJob& job, const Launch& l, cudaStream_t s, int* launched);
// peel.cu: the peel pass of an imaging pass over the events the event kernel queued in
// job.args.peel_q; hist [ncells + 1], sums [(ncells + 1024) / 1024], order [peel_cap] scratch
cudaError_t launch_peel_pass(const PropagateJob& job, uint32_t* hist, uint32_t* sums, uint32_t* order, cudaStream_t s,
                             int* launched);

// event.cu: one persistent launch over the (model, packet range) chunks of grid type gtype
cudaError_t launch_propagate_batch(int gtype, const BatchModel* models, const BatchChunk* chunks, int nchunks,
                                   unsigned* chunk_counter, const BatchState* state, const Launch& l, cudaStream_t s);

// batch_kernels.cu
cudaError_t launch_batch_begin(const BatchModel* models, BatchState* state, int nmodels, const BatchSeg* segs,
                               int nsegs, unsigned* chunk_counter, unsigned* hist, int nesc_per_model, cudaStream_t s);
cudaError_t launch_batch_temperature(const BatchModel* models, BatchState* state, const BatchSeg* segs, int nsegs,
                                     cudaStream_t s);
cudaError_t launch_batch_select(const BatchModel* models, BatchState* state, int nmodels, const BatchSeg* segs,
                                int nsegs, unsigned* hist, cudaStream_t s);
cudaError_t launch_batch_end(const BatchModel* models, BatchState* state, int nmodels, double q_thres,
                             double delta_thres, cudaStream_t s);

// temperature.cu
struct TemperatureJob {
    int32_t gtype;
    int32_t n1, n2, n3;
    int64_t ncells;
    const float* rhoL;
    const double* acc;   // sum kappa l in the scaled length unit
    double acc_scale;    // eps L0: acc * acc_scale = sum eps kappa l (cgs)
    const double* va;    // per-axis volume factors: V = va[i] vb[j] vc[k] (cm^3)
    const double* vb;
    const double* vc;
    const double* E;     // [nT] emission table
    const double* lnE;   // [nT]
    const double* lnT;   // [nT]
    const double* Tn;    // [nT]
    int32_t nT;
    int32_t quantity;    // 0 T, 1 Adot
    int32_t first;       // first iteration for the Adot quantity (no previous value)
    double* T;           // in: previous, out: new
    double* adot;        // in: previous, out: new
    int32_t* emit_row;   // out
    unsigned long long* keys;       // out: bit pattern of R (0 for cells without dust)
    unsigned long long* counters;   // [2] clamp low/high (cells with dust)
};
cudaError_t launch_temperature(const TemperatureJob& j, cudaStream_t s, int* launched);
// exact nearest-rank select of the k-th smallest key; writes the key to *d_out
cudaError_t launch_select_kth(const unsigned long long* keys, int64_t n, unsigned long long k,
                              unsigned int* d_hist, unsigned long long* d_state, unsigned long long* d_out,
                              cudaStream_t s, int* launched);
cudaError_t launch_invert_temperature(const double* adot, double* T, int64_t n, const double* E, const double* lnE,
                                      const double* lnT, const double* Tn, int nT, cudaStream_t s);
cudaError_t launch_emit_rows(const double* T, int32_t* rows, int64_t n, const double* lnT, int nT, cudaStream_t s);

// pda.cu: partial diffusion approximation (App. A), spherical-polar grids
struct PdaJob {
    int32_t n1, n2, n3;
    int64_t nc;
    const float* rhoL;                       // rho L0
    const double *rc, *dr, *rface;           // [n1] centre, width; [n1+1] walls (scaled)
    const double *stc, *dth, *stf;           // [n2] sin(theta centre), dtheta; [n2+1] sin(theta walls)
    const double* dph;                       // [n3]
    const uint32_t* visits;                  // packet entries per cell in this iteration
    uint32_t n_min;                          // cells with dust and fewer entries are solved
    const double* T_prev;                    // temperatures the iteration started from (chi_R, keys)
    const double* adot_prev;
    double* T;                               // in: Monte-Carlo T of this iteration, out: after the PDA
    double* adot;
    int32_t* row;
    unsigned long long* keys;
    const double *lnT, *lnE, *lnchiR;        // [nT] tables
    int32_t nT;
    int32_t quantity, first;
    uint8_t* state;                          // 0 Monte-Carlo, 1 candidate, 2 solved
    double *dtau, *W, *x, *r, *p, *q, *b, *dg;   // [3][nc], [6][nc], [nc] x 6
    double* scal;                            // [8] CG scalars
    unsigned long long* count;
    int* flag;
};
// raytrace.cu: raytracing of point-source and dust emission (Sect. 2.6.3)
struct RtJob {
    int32_t n1, n2, n3;
    int64_t nc;
    const float* rho;                        // g/cm^3
    const double *va, *vb, *vc;              // per-axis volume factors (cm^3)
    const double* T;
    const double *lnT, *lnE;                 // [nT]
    int32_t nT, nnu;
    const int32_t* emit_row;                 // re-emission rows of this pass
    const float* cdf_emit;                   // [nT][nnu]
    const float* inv_dnu;                    // [nnu-1] 1 / (nu_{j+1} - nu_j)
    // quadrature of the SED bins: dust rows (qd_*) and source spectra (qs_*), sorted by bin
    const int32_t *qd_off, *qd_j, *qd_bin;
    const float *qd_w, *qd_chi;
    int32_t nqd;
    const int32_t *qs_off, *qs_j, *qs_bin;
    const float *qs_w, *qs_chi;
    int32_t nqs;
    int32_t nsed, npoint;
    const float* src_col;                    // [npoint][nobs], -1 outside the grid
    const float* src_pos;                    // [npoint][3] scaled
    const double* src_L;                     // [npoint] erg/s
    const float* spec_cdf;                   // [nsrc][nspec]
    const double* spec_nu;                   // [nspec]
    int32_t nspec;
    // dust rays
    int64_t n_rays;
    uint32_t key0, key1, iter_key, model_key;
    double* cdf;                             // [nc] emission CDF (work)
    double* scan_sums;                       // [nc / 1024 + 1]
    double* total;                           // [1] L_dust
    float* col;                              // [n_rays][nobs]
    int32_t* row;                            // [n_rays]
    double eps4pi;                           // L_dust / n_rays / (4 pi), set by run_raytrace
    double* sed;
    double* img;
    unsigned long long* counters;
};
cudaError_t run_raytrace(const DevGrid& g, const DevObs& o, RtJob J, double* host_total, cudaStream_t s,
                         int* launched);

struct PdaStats {
    int64_t n_cells;
    int64_t iterations;
    double residual;                         // |b - A x| / |b| at exit
};
cudaError_t launch_rosseland(int nnu, const double* nu, const double* chi, int nT, const double* T, double* chiR,
                             double* lnchiR, cudaStream_t s);
// modified random walk (mrw.cu): FP64 node tables of ln chi_t(T) and ln kappa_P(T), then the FP32
// per-cell coefficients rhoL chi_t(T_c) and kappa_P(T_c) a pass reads
cudaError_t launch_mrw_tables(int nnu, const double* nu, const double* chi, const double* kappa, const double* alb,
                              double g, int nT, const double* T, double* ln_chit, double* ln_kp, cudaStream_t s);
cudaError_t launch_mrw_cells(int64_t n, const float* rhoL, const double* T, const double* lnT, const double* ln_chit,
                             const double* ln_kp, int nT, float* k, float* kp, cudaStream_t s);
cudaError_t run_pda(const PdaJob& J, double tol, int max_iter, int* host_flag, double* host_scal, PdaStats* st,
                    cudaStream_t s, int* launched);

// tables.cu (FP64 table construction on the device)
cudaError_t launch_emission_tables(int nnu, const double* nu, const double* kappa, int nT, const double* T,
                                   double* E, double* lnE, float* cdf, cudaStream_t s);
cudaError_t launch_source_spectra(int nsrc, int nspec, const double* spec_nu, const double* teff,
                                  const double* user_nu, const double* user_f, const int* user_off,
                                  const int* user_n, float* spec_cdf, cudaStream_t s);

// steps.cu
cudaError_t launch_step_philox(int64_t n, const uint32_t* ctr, const uint32_t* key, uint32_t* out, cudaStream_t s);
cudaError_t launch_step_cell_exit(const DevGrid& g, int64_t n, const float* pos, const float* dir,
                                  const int32_t* cell, float* dist, int32_t* ex, float inv_L0, float L0, cudaStream_t s);
cudaError_t launch_step_tau(const DevGrid& g, const DevDust& d, int64_t n, const float* pos, const float* dir,
                            const float* nu, float* tau, float inv_L0, cudaStream_t s);
cudaError_t launch_step_wall_distance(const DevGrid& g, int64_t n, const float* pos, const int32_t* cell, float* dist,
                                     float inv_L0, float L0, cudaStream_t s);
cudaError_t launch_step_mrw_path(int64_t n, const float* tau0, const float* zeta, float* out, cudaStream_t s);
cudaError_t launch_step_hg(float g, int64_t n, const float* din, const float* u1, const float* u2, float* dout,
                           cudaStream_t s);
cudaError_t launch_step_sample(const float* x, const float* cdf, int nx, int64_t n, const int32_t* row,
                               const float* u, float* out, cudaStream_t s);

}  // namespace hrt
