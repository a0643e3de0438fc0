// internal.h -- host-side declarations shared by the translation units of libgcmc.
#pragma once
#include <atomic>
#include <cstdint>
#include <cuda_runtime.h>

#include "common.cuh"

namespace gcmc {

struct HostLog {               // device pointers of the per-packet debug outputs
    double *pk_f;
    int64_t *pk_steps;
    double *pk_tau;
    int32_t *tr_cell;
    double *tr_len;
    int32_t *tr_n;
    int32_t n_trace, max_trace;
};

// per-job parameters of the cell-table kernels
struct PrepJob {
    int32_t lam, g;            // wavelength / band index, g-ordinate
    int32_t lam_hint;
    int32_t bslot;             // emission: row of this job's band in the group's 4 pi V B(T) table
    double lam_m;              // wavelength (m) for the Planck function (k-table) or rest wavelength (xsec)
    double c1;                 // Planck prefactor 2 h c^2 / lambda^5 (k-table)
    void *rec;                 // output: albedo records or alpha (march precision)
    long long *cdf;            // emission: cumulative pdf in 2^62 fixed point (first scratch for L_i as FP64)
    void *wcell;               // emission: launch weight (march precision)
    double *info;              // emission: [L_tot, n_incl, cdf_total, Q_tot bits, constants of the pdf] (device)
    double *bsum;              // emission: per-block partial sums [nblk]
    double *bcnt;              // emission: per-block included counts [nblk]
    double *lum;               // emission: optional copy of L_i (debug), or NULL
    const double *vb;          // emission: the group's 4 pi V_i B(T_i) table, [band slot][cell]
    // emission, entry s < number of band slots of the group: wavelength, Planck prefactor of slot s
    double pl_lam, pl_c1;
};

// slots of PrepJob::info
enum : int {
    INFO_LTOT = 0, INFO_NINCL = 1, INFO_CDFTOT = 2, INFO_QTOT = 3,   // QTOT: int64 bits
    INFO_QA = 4, INFO_QB = 5,                                        // Q_i = rint(QA L_i + QB)
    INFO_INVL = 6, INFO_BN = 7,                                      // 1 / L_tot, beta / n_incl
};

struct KtabDev {               // device k-table (natural logs in FP64)
    int nb, ng, nT, np;
    const double *lnk;         // [nb][ng][nT][np]
    // FP32 node records {k_ab, ln k_(a+1)b - ln k_ab, ln k_a(b+1) - ln k_ab, mixed second difference}:
    // k = k_ab exp(wT d1 + wp d2 + wT wp d3) is the bilinear interpolation of ln k with an argument of
    // order one, so FP32 keeps ~1e-7 relative accuracy (ln k itself would lose ~ulp(10))
    const float4 *node_f;      // [nb][ng][nT][np]
    const double *Tg, *pg;     // axes
};

struct XsecDev {
    int nl, nT, np;
    const double *lam;         // [nl]
    const double *lnsig;       // [nl][nT][np] FP64 logs
    const float *lnsig_f;      // FP32 logs
    const double *Tg, *pg;
    double view_theta, view_phi, omega_rot;
};

struct AlbDev {
    int nlam;
    const double *kabs, *kray, *qcld, *wcld, *gcld;
    const float *acld;
};

constexpr int PREP_BLOCK = 256;
constexpr int EMIS_SCAN_BLOCK = 1024;

// cell tables (S1)
cudaError_t prep_albedo(int precision, const DevGrid *dgrid, const DevGrid &hgrid, const AlbDev &op,
                        const PrepJob *djobs, int njobs, cudaStream_t st);
cudaError_t prep_emission(int precision, const DevGrid *dgrid, const DevGrid &hgrid, const KtabDev &kt,
                          const PrepJob *djobs, int njobs, int nslots, double tau_vert_max, double beta, int2 *wk_ab,
                          void *wk_w, cudaStream_t st);
int emis_col_blocks(const DevGrid &g);     // partial-sum blocks of the column kernel
cudaError_t prep_xsec(int precision, const DevGrid *dgrid, const DevGrid &hgrid, const XsecDev &xs,
                      const PrepJob *djobs, int njobs, int2 *wk_ab, double2 *wk_w, double *wk_fac, cudaStream_t st);

// transport
size_t transport_smem(int block);
cudaError_t launch_plain(int precision, bool scatter, const DevGrid *grids, const DevJob *job, int64_t packet0,
                         int64_t n_run, const HostLog *hl, int tab_entries_n, cudaStream_t st);
cudaError_t launch_persistent(int precision, bool scatter, const DevGrid *grids, const DevJob *jobs, int n_jobs,
                              int64_t total_items, int chunk, int block, int blocks_per_sm, int interval, int refill_min,
                              int one_grid, int tab_n, unsigned long long *work, cudaStream_t st);

// process-wide kernel launch counter
extern std::atomic<long long> g_launches;
inline void count_launch(int n = 1) { g_launches.fetch_add(n, std::memory_order_relaxed); }

// random-gather microbenchmark
cudaError_t gather_bench(const void *table, int64_t n_records, int record_bytes, int64_t iters, int blocks, int threads,
                         float *sink, cudaStream_t st);

// self test
cudaError_t selftest_philox(const uint32_t *ctr, const uint32_t *key, int n, uint32_t *out_lib, uint32_t *out_cur,
                            cudaStream_t st);

}  // namespace gcmc
