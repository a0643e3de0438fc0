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

constexpr int XS_LOCAL = 64;   // most table wavelengths an FP32 cross-section job brackets in

// per-job parameters of the cell-table kernels
struct PrepJob {
    int32_t lam, g;            // wavelength / band index, g-ordinate
    int32_t lam_hint, pad;
    double lam_m;              // band centre (k-table) or rest wavelength (xsec), m
    void *rec;                 // output: albedo records or alpha (march precision)
    void *alpha;               // output with albedo records: alpha alone, the table the cell march reads
    long long *cdf;            // emission: cumulative pdf in 2^62 fixed point (first scratch for L_i as FP64)
    void *wcell;               // emission: launch weight (march precision)
    double *info;              // emission: [L_tot, n_incl, cdf_total, Q_tot bits, constants of the pdf] (device)
    double *bsum;              // emission: per-block partial sums [nblk]
    double *bcnt;              // emission: per-block included counts [nblk]
    double *lum;               // emission: optional copy of L_i (debug), or NULL
    // cross sections, FP32 runs: the table wavelengths lambda_l, l = xs_lo .. xs_lo + xs_n - 1, that
    // bracket every Doppler-shifted wavelength of the grid, as FP32 offsets lambda_l / lambda_0 - 1
    // (xs_n = -1: bracket in FP64 instead)
    int32_t xs_lo, xs_n;
    float xs_d[XS_LOCAL];
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
    // per-cell tables of the grid the table is uploaded for, built once at upload:
    const int2 *ab;            // [ncell] (T, p) interpolation cell
    const double2 *w64;        // [ncell] (wT, wp) in FP64
    const float2 *w32;         // [ncell] the same rounded to FP32
    const double *vb;          // [nb][ncell] 4 pi V_i B_lambda(T_i) at each band centre
    const double *gw;          // [ng] g-ordinate weights, or NULL (band jobs need them)
};

struct XsecDev {
    int nl, nT, np;
    const double *lam;         // [nl]
    const double *lnsig;       // [nl][nT][np] FP64 logs
    const float *lnsig_f;      // FP32 logs
    const double *Tg, *pg;
    double view_theta, view_phi, omega_rot;
    // per-cell tables of the grid the table is uploaded for, built once at upload:
    const int2 *ab;            // [ncell] (T, p) interpolation cell
    const double2 *w;          // [ncell] (wT, wp)
    const double *fac;         // [ncell] Doppler factor lambda_eff / lambda_0 = 1 - v_LOS / c
    const float2 *w32;         // [ncell] (wT, wp) in FP32
    const float *dlt_f;        // [ncell] lambda_eff / lambda_0 - 1 in FP32
    double dmin, dmax;         // range of dlt_f over the grid
};

struct AlbDev {
    int nlam;
    const double *kabs, *kray, *qcld, *wcld, *gcld;
    const float *acld;
};

constexpr int PREP_BLOCK = 256;
// cells per block of the emission pdf scan: small blocks, so that the cell-table kernels of a
// newly admitted job fit beside a resident serving kernel
constexpr int EMIS_SCAN_BLOCK = 256;

// cell tables (S1)
cudaError_t prep_albedo(int precision, const DevGrid *dgrid, const DevGrid &hgrid, const AlbDev &op,
                        const PrepJob *djobs, int njobs, cudaStream_t st);
cudaError_t prep_emission(int precision, const DevGrid &hgrid, const KtabDev &kt, const PrepJob *djobs, int njobs,
                          double tau_vert_max, double beta, cudaStream_t st);
int emis_col_blocks(const DevGrid &g);     // partial-sum blocks of the column kernel
cudaError_t prep_emission_xsec(int precision, const DevGrid &hgrid, const XsecDev &xs, const PrepJob *djobs, int njobs,
                               double tau_vert_max, double beta, cudaStream_t st);
cudaError_t prep_xsec(int precision, const DevGrid &hgrid, const XsecDev &xs, const PrepJob *djobs, int njobs,
                      cudaStream_t st);
// per-cell tables of an opacity on its grid (at upload): interpolation cells and weights, and
// 4 pi V B(T) per band (k-table) or the Doppler factors (cross sections); lam_dev: band centres [nb]
cudaError_t ktable_cells(const DevGrid &hgrid, const double *lam_dev, int nb, int2 *ab, double2 *w64, float2 *w32,
                         double *vb, const KtabDev &kt, cudaStream_t st);
cudaError_t xsec_cells(const DevGrid &hgrid, const XsecDev &xs, int2 *ab, double2 *w, double *fac, float2 *w32,
                       float *dlt, float *minmax, cudaStream_t st);

// serving queue (continuous batching): host-mapped control block, job ring and completion records,
// and device-side claim counters
constexpr unsigned SERVE_RING = 65536;      // published jobs addressable at once (ring of segments)
struct ServeCtl {
    unsigned long long published;           // segments published by the host (store-release)
    unsigned int stop;                      // the host asks the kernel to leave when idle
    unsigned int err;                       // set by the kernel: a claim met another job of its slot
};
// A slot's claim counter holds (generation << SERVE_GEN_SHIFT) | items claimed; the generation
// (the job's admission number) is set with the count when the slot is given to a job, so a claim
// can tell whether the counter still belongs to the job it read from the ring.
constexpr int SERVE_GEN_SHIFT = 40;
// upper bound on the polls of an idle warp while other warps still run (about 20 s): past it the
// warp reports an error and the launch leaves
constexpr long long SERVE_IDLE_CAP = 20000000;
struct ServeSeg {
    const DevJob *job;                      // device pointer
    int64_t n_items;                        // work items of `chunk` packets
    uint32_t slot;                          // completion record and counters
    uint32_t gen;                           // admission number of the job (low 24 bits)
};
struct ServeDone {
    unsigned long long acc[ACC_SLOTS];      // the job's accumulators
    double info[4];                         // emission: L_tot, n_incl, cdf_total
    unsigned long long seq;                 // segment index + 1, written last
    unsigned long long pad[3];
};
struct ServeQueue {
    ServeCtl *ctl;                          // host-mapped
    const ServeSeg *ring;                   // host-mapped [SERVE_RING]
    ServeDone *done;                        // host-mapped [slots]
    unsigned long long *cur_seg;            // device: oldest segment with unclaimed items
    unsigned long long *n_idle;             // device: warps of the current launch without work
    unsigned long long *exiting;            // device: the current launch is leaving
    unsigned long long *slot_next;          // device [slots]: next item of the slot's job to claim
    unsigned long long *slot_done;          // device [slots]: items of the slot's job finished
};
cudaError_t launch_serve(bool ext, const DevGrid *grids, const ServeQueue &q, int block, int blocks_per_sm, int chunk,
                         int interval,
                         int refill_min, int tab_n, int idle_polls, int *grid_blocks, cudaStream_t st);

// transport
size_t transport_smem(int block);
// Optional code compiled into a transport-kernel variant (template FEAT): band jobs' per-packet
// g-ordinate tables (FEAT_BAND); the optional physics of scattered packets (FEAT_EXT: surfaces,
// two-term HG clouds, multiple scattering in transmission, stellar limb darkening, forced scattering,
// continuous absorption's weight bookkeeping); and continuous absorption's second optical depth in the
// cell step (FEAT_CABS, with FEAT_EXT).  Batches that use none of them run variants without that code.
constexpr int FEAT_BAND = 1, FEAT_EXT = 2, FEAT_CABS = 4, FEAT_ALL = 7;

cudaError_t launch_plain(int precision, bool scatter, int feat, const DevGrid *grids, const DevJob *job, int64_t packet0,
                         int64_t n_run, const HostLog *hl, int tab_entries_n, cudaStream_t st);
cudaError_t launch_persistent(int precision, bool scatter, int feat, const DevGrid *grids, const DevJob *jobs, int n_jobs,
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
