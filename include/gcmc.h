/*
 * gcmc.h -- C ABI of libgcmc: GB300-native Monte Carlo radiative transfer of photon packets
 * through a 3D spherical (longitude x latitude x pressure-level) exoplanet atmosphere, after
 * the gCMCRT method (Lee et al. 2022, arXiv:2110.15640).
 *
 * The calls follow the paper's statement of the problem (Sect. 2): the host prepares the grid
 * and the opacity structure and hands them to GPU memory ("global GPU modules"), packets are
 * run on the GPU, and the image/spectrum tallies come back to the host.  Three modes:
 *   GCMC_ALBEDO        scattered starlight with peel-off towards the observer (Sect. 4.6, 5.2)
 *   GCMC_EMISSION      thermal emission from the atmospheric volume (Sect. 4.3, 4.6, 5.3)
 *   GCMC_TRANSMISSION  limb chords through the annulus (Sect. 5.1), with per-cell Doppler-shifted
 *                      high-resolution opacity (Sect. 7); or on scattering opacities, optionally with
 *                      multiple scattering after the chord; optional stellar limb darkening
 *
 * Conventions
 *  - Status: every call returns 0 (GCMC_OK) or a negative GCMC_ERR_* code; no exceptions cross
 *    the ABI.  gcmc_last_error() gives a one-line message for the last failure of a context.
 *  - Memory: input pointers are host or device memory as the descriptor's `memory` field says
 *    (GCMC_MEM_HOST / GCMC_MEM_DEVICE).  The library copies what it needs during the call; the
 *    caller keeps ownership of its buffers.  Device memory the library needs (resident grids,
 *    opacity tables, per-job cell tables, work queues) is obtained through the context's
 *    allocator (cudaMalloc unless gcmc_set_allocator installs another) and released by
 *    gcmc_destroy.
 *  - Streams: all work of a context is ordered on its stream (gcmc_set_stream; default: the
 *    legacy default stream).  Calls that return host results synchronise that stream.
 *  - Threads: a context is not thread-safe; use one context per host thread.
 *  - Determinism: tallies depend only on (grid, opacity, source, mode, lambda, g, N, seed, job
 *    key).  Packets draw counter-based Philox4x32-10 numbers keyed by (seed; packet, event, job
 *    key); tallies are accumulated as 64-bit fixed point (2^-32 resolution), so the result of a
 *    job is bit-identical whether it runs alone or batched with other jobs that use the same optional
 *    features.  The transport kernels are compiled in variants with and without the optional physics
 *    (surfaces, two-term HG, transmission scattering, limb darkening, biased flights, continuous
 *    absorption) and band jobs' tables; a batch runs in the variant its jobs need, and a job batched
 *    with jobs that need another variant can differ from its run alone at FP32 rounding.  The server
 *    (gcmc_server_*) runs every request in its own variant, so a served request is bit-identical
 *    alone and in any mix.
 *  - Units: SI (m, m^-1, m^2/kg, kg/m^3, K, Pa, W).  Per-cell arrays are flattened [k][j][i]
 *    with longitude fastest; k = 0 is the bottom shell.
 */
#ifndef GCMC_H
#define GCMC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GCMC_MAX_OBS 8

typedef struct gcmc_ctx gcmc_ctx;
typedef int gcmc_status;

enum {
    GCMC_OK = 0,
    GCMC_ERR_ARG = -1,        /* invalid argument (sizes, ids, NULL, non-monotone edges) */
    GCMC_ERR_OOM = -2,        /* the allocator returned NULL */
    GCMC_ERR_CUDA = -3,       /* a CUDA runtime call failed (message in gcmc_last_error) */
    GCMC_ERR_STEP_CAP = -4,   /* reported in stats: packets stopped by the per-packet step cap */
    GCMC_ERR_TIMEOUT = -5,    /* a bounded wait gave up */
    GCMC_ERR_NOT_READY = -6,  /* gcmc_poll: the ticket's work is still running */
    GCMC_ERR_NAN = -7,        /* NaN, infinite or negative values in an upload */
    GCMC_ERR_RANGE = -8       /* a size exceeds a compiled limit */
};

enum { GCMC_ALBEDO = 0, GCMC_EMISSION = 1, GCMC_TRANSMISSION = 2 };
enum { GCMC_MEM_HOST = 0, GCMC_MEM_DEVICE = 1 };
enum { GCMC_FP32 = 0, GCMC_FP64 = 1 };
enum { GCMC_OPAC_ALBEDO = 0, GCMC_OPAC_KTABLE = 1, GCMC_OPAC_XSEC = 2 };

typedef void *(*gcmc_alloc_fn)(size_t bytes, void *user);
typedef void (*gcmc_free_fn)(void *ptr, void *user);

/* ---------------------------------------------------------------- context */

/* Create a context on CUDA device `device`.  *out receives the handle.  Errors: GCMC_ERR_ARG (out is
   NULL), GCMC_ERR_CUDA (no such device, or it cannot be selected), GCMC_ERR_OOM. */
gcmc_status gcmc_create(int device, gcmc_ctx **out);
/* Release every device buffer of the context and the context itself.  GCMC_ERR_ARG for NULL. */
gcmc_status gcmc_destroy(gcmc_ctx *ctx);
/* Order all later work of the context on `cuda_stream` (a cudaStream_t; NULL = default stream).
   GCMC_ERR_ARG for a NULL context. */
gcmc_status gcmc_set_stream(gcmc_ctx *ctx, void *cuda_stream);
/* Route the context's device allocations through alloc/free (e.g. a framework's caching
   allocator).  Must be called before the first upload.  NULL restores cudaMalloc/cudaFree.
   Errors: GCMC_ERR_ARG (after an upload, or only one of alloc and free_fn given). */
gcmc_status gcmc_set_allocator(gcmc_ctx *ctx, gcmc_alloc_fn alloc, gcmc_free_fn free_fn, void *user);
/* Message of the last failing call on this context ("" if none).  Owned by the context. */
const char *gcmc_last_error(gcmc_ctx *ctx);

/* ---------------------------------------------------------------- grid (Sect. 2, 7) */

typedef struct {
    int32_t nlon, nlat, nr;   /* cells in longitude, latitude, radius; nlon >= 1, nlat >= 1, nr >= 1 */
    int32_t memory;           /* GCMC_MEM_HOST or GCMC_MEM_DEVICE for every pointer below */
    const double *r_edges;    /* [nr+1] shell radii, m, strictly increasing; r_edges[0] = R0 (black bottom) */
    const double *lat_edges;  /* [nlat+1] latitude edges, rad, strictly increasing, -pi/2 .. pi/2 */
    const double *lon_edges;  /* [nlon+1] longitude edges, rad, strictly increasing, span exactly 2 pi */
    const float *T;           /* [ncell] temperature, K (> 0) */
    const float *p;           /* [ncell] pressure, Pa (> 0) */
    const float *rho;         /* [ncell] density, kg/m^3 (>= 0) */
    const float *wind;        /* [3][ncell] (u east, v north, w up), m/s, or NULL */
} gcmc_grid_desc;

/* Copy a grid to the device; *grid_id receives its id.  Errors: GCMC_ERR_ARG (sizes, edges),
   GCMC_ERR_NAN (non-finite or non-positive T, p; negative rho), GCMC_ERR_OOM, GCMC_ERR_CUDA. */
gcmc_status gcmc_upload_grid(gcmc_ctx *ctx, const gcmc_grid_desc *desc, int *grid_id);

/* ---------------------------------------------------------------- opacity (Sect. 3.6, 7) */

typedef struct {
    int32_t kind;             /* GCMC_OPAC_ALBEDO, GCMC_OPAC_KTABLE or GCMC_OPAC_XSEC */
    int32_t memory;           /* where the pointers live */
    /* GCMC_OPAC_ALBEDO: per wavelength l, alpha_ext = rho (kabs + kray) + acld qcld,
       alpha_sca = rho kray + wcld acld qcld, omega = alpha_sca / alpha_ext,
       P_gas = rho kray / alpha_sca (Sect. 3.6), HG asymmetry g = gcld */
    int32_t nlam;
    const double *kabs, *kray, *qcld, *wcld, *gcld;   /* [nlam] each */
    const float *acld;                                /* [ncell] cloud extinction, 1/m, or NULL */
    /* GCMC_OPAC_KTABLE: k[b][g][T][p] (m^2/kg), bilinear in (ln T, ln p) of ln k, clamped */
    int32_t nb, ng, nT, np;
    const double *lam;        /* [nb] band-centre wavelength (m), for the Planck function */
    const double *Tg, *pg;    /* [nT], [np] strictly increasing table axes */
    const float *k;           /* [nb][ng][nT][np] */
    /* GCMC_OPAC_XSEC: sigma[l][T][p] (m^2/kg) on wavelengths xlam[nl]; uses Tg, pg, nT, np above */
    int32_t nl, pad;
    const double *xlam;       /* [nl] strictly increasing, m */
    const float *sigma;       /* [nl][nT][np] > 0 */
    double view_theta;        /* observer polar angle (colatitude), rad, for v_LOS (Sect. 7) */
    double view_phi;          /* observer longitude, rad */
    double omega_rot;         /* planetary rotation rate, rad/s */
    const double *gw;         /* GCMC_OPAC_KTABLE: [ng] g-ordinate weights (sum 1), needed by band jobs
                                 (g_idx = -1); may be NULL */
} gcmc_opacity_desc;

/* Copy an opacity description for grid `grid_id` to the device.  *opac_id receives its id.
   Errors: GCMC_ERR_ARG, GCMC_ERR_NAN (negative or non-finite opacities), GCMC_ERR_OOM, GCMC_ERR_CUDA. */
gcmc_status gcmc_upload_opacity(gcmc_ctx *ctx, int grid_id, const gcmc_opacity_desc *desc, int *opac_id);

/* ---------------------------------------------------------------- source and options (Sect. 4, 5) */

typedef struct {
    double star[3];           /* unit vector from the planet centre towards the star */
    int32_t n_obs;            /* 1 .. GCMC_MAX_OBS observer directions */
    int32_t survival;         /* 1 survival biasing W <- W omega (Sect. 4.4); 0 analog absorb/scatter */
    double obs[GCMC_MAX_OBS][3]; /* unit vectors towards the observer(s) */
    double w_rr;              /* Russian roulette (Sect. 4.5) when W < w_rr * W_launch */
    double p_surv;            /* roulette survival probability (weight / p_surv on survival) */
    double tau_peel_cut;      /* peel-off / chord marches stop beyond this optical depth */
    double tau_vert_max;      /* emission: cells with vertical tau above them >= this do not emit (Sect. 4.6) */
    double beta_emis;         /* emission: hybrid biasing fraction of the uniform-in-cell pdf (Sect. 4.3) */
    double hg_iso_eps;        /* |g| below this samples HG isotropically */
    int32_t scatter_emission; /* emission: 1 = follow packets after the launch peel-off */
    int32_t precision;        /* GCMC_FP32 (FP32 march, FP64 near-tangent roots) or GCMC_FP64 */
    int64_t max_steps;        /* per-packet cap on cell segments (stats count capped packets) */
    int32_t cloud_phase;      /* cloud phase function (Sect. 3): GCMC_CLOUD_HG, or GCMC_CLOUD_TTHG, the two-term
                                 HG of one asymmetry g: a P_HG(g) + (1 - a) P_HG(-g/2), a = 1 - g^2/4; a
                                 scattering picks the term from its gas/cloud uniform u1 rescaled to
                                 (u1 - P_gas) / (1 - P_gas) */
    int32_t pad2;
    double surface_albedo;    /* Lambertian lower boundary of this albedo in [0, 1] (Sect. 3); 0 = black.  A packet
                                 that reaches it peels off towards each observer above the local horizon
                                 with weight A_s mu_o / pi and leaves with cosine sqrt(zeta) about the normal,
                                 weight A_s (survival biasing) or probability A_s (analog).  Albedo mode only:
                                 emission and transmission packets do not fly */
    /* transmission (Sect. 5.1) */
    int32_t trans_scatter;    /* 1 = multiple scattering: after its chord (tally column 0) the packet flies from its
                                 launch point along -star and every scattering peels off towards the transit
                                 observer -star into column 1, weighted by the launch b / R_TOA.  Needs
                                 scattering opacities (GCMC_OPAC_ALBEDO); 0 = chords only */
    int32_t ld_law;           /* stellar limb darkening: GCMC_LD_NONE or a law below; the packet carries
                                 I(mu)/I(disk centre), mu the stellar zenith-angle cosine behind its chord */
    double ld_coef[4];        /* linear u; quadratic c1 c2; square-root c d; logarithmic e f (mu ln mu term);
                                 power-2 c alpha (1 - c (1 - mu^alpha)); four-coefficient a1..a4 */
    double star_radius;       /* m, > 0 when ld_law is set */
    double star_dist;         /* m, planet-star distance: the solid angle of the stellar disk for the scattered
                                 light (gcmc_transit); 0 when unused */
    double transit_xy[2];     /* sky-plane position of the planet centre relative to the stellar disk centre, m,
                                 along the launch basis e1 = star x z / |star x z| (star x x when |star_z| >= 0.9),
                                 e2 = star x e1: a chord launched at (b, psi) sits at transit_xy + b (cos psi, sin psi) */
    /* emission band jobs (g_idx = -1, Sect. 4.7): each packet draws its g-ordinate with probability q(g)
       (fourth word of its event-1 draw) and carries W_g = p(g)/q(g), p(g) = w_g L_g / sum_g w_g L_g; its cell
       then comes from that g's hybrid pdf (launch uniform, no stratification).  stats.l_tot of a band job
       is L_band = sum_g w_g L_g and stats.n_emit_cells the sum over g. */
    int32_t g_bias;           /* GCMC_GBIAS_NONE q = p, GCMC_GBIAS_UNIFORM q = 1/N_g,
                                 GCMC_GBIAS_COMPOSITE q = (1 - g_beta) p + g_beta / N_g */
    int32_t pad3;
    double g_beta;            /* composite fraction in [0, 1] */
    /* variance reduction for scattered packets (albedo; transmission with multiple scattering) */
    int32_t forced_first;     /* forced scattering (Sect. 4.2): 1 = the first flight only (forced first scattering),
                                 2 = every flight.  A march along the flight gives the optical depth tau_m to the
                                 grid boundary; W e^-tau_m leaves unscattered and the packet, weight
                                 W (1 - e^-tau_m), interacts at tau = -ln(1 - zeta (1 - e^-tau_m)).  Not forced
                                 past tau_peel_cut or when the path ends on a reflecting surface */
    int32_t cont_abs;         /* 1 = continuous absorption (Sect. 4.1): flights sample their optical depth in the
                                 scattering opacity omega alpha, the weight decays by e^-tau_abs along the path
                                 (booked as absorbed) and every interaction scatters (peel-offs without omega) */
    int32_t path_bias;        /* how the flights forced_first selects sample tau (Sect. 4.2): 0 forced scattering
                                 (above); 1 path length stretching, not forced: tau from (e^-tau + a e^-a tau) / 2,
                                 a = 1 / (1 + tau_m); 2 hybrid: forced, tau from the mean of the truncated
                                 exponential and the uniform on [0, tau_m].  Both reweight the packet by p/q,
                                 booked with the roulette's gain (ledger[4]) and loss (ledger[5]) */
    int32_t pad4;
} gcmc_source_desc;

#define GCMC_GBIAS_NONE 0
#define GCMC_GBIAS_UNIFORM 1
#define GCMC_GBIAS_COMPOSITE 2

#define GCMC_LD_NONE 0
#define GCMC_LD_LINEAR 1
#define GCMC_LD_QUADRATIC 2
#define GCMC_LD_SQRT 3
#define GCMC_LD_LOG 4
#define GCMC_LD_POWER2 5
#define GCMC_LD_CLARET4 6

#define GCMC_CLOUD_HG 0
#define GCMC_CLOUD_TTHG 1

/* Register a source description; *source_id receives its id.  Errors: GCMC_ERR_ARG (not unit vectors,
   options out of range, unknown cloud_phase, surface_albedo outside [0, 1], unknown ld_law, limb
   darkening without a stellar radius, star_dist neither 0 nor above star_radius). */
gcmc_status gcmc_set_source(gcmc_ctx *ctx, int grid_id, const gcmc_source_desc *desc, int *source_id);

/* ---------------------------------------------------------------- running packets */

typedef struct {
    int64_t packets;          /* packets run */
    int64_t steps;            /* packet-steps: cell segments processed in flights, peel-offs and chords */
    double ledger[8];         /* sum of weights: emitted, escaped, absorbed, bottom, roulette gain,
                                 roulette loss, step-capped, lost (emitted + gain = the rest); the gain and
                                 loss entries also book the p/q reweights of stretched or hybrid flights */
    double l_tot;             /* emission: total luminosity of the emitting cells, W/m (Sect. 5.3) */
    double cdf_total;         /* emission: total of the hybrid pdf (1 up to rounding) */
    int64_t n_emit_cells;     /* emission: cells above the tau_vert cut */
    int64_t flags;            /* GCMC_FLAG_* bits raised by any packet of the job (0: none) */
} gcmc_stats;

/* gcmc_stats.flags: a peel-off or chord contribution that was not a number, negative or at least 1e9
   (left out of the tallies) */
enum { GCMC_FLAG_TALLY_RANGE = 1 };

typedef struct {
    int32_t grid_id, opac_id, source_id, mode;
    int32_t lam_idx;          /* wavelength (albedo, xsec) or band (k-table) index */
    int32_t g_idx;            /* g-ordinate (k-table), or -1: a band job whose packets draw their g-ordinate
                                 (Sect. 4.7, gcmc_source_desc.g_bias); ignored otherwise */
    int32_t obs_idx;          /* -1: tally every observer of the source; else only observer obs_idx */
    uint32_t job_key;         /* 32-bit key of the job in the Philox counter */
    int64_t n_packets;
    uint64_t seed;
} gcmc_job;

/* Plain form (the paper's GPU loop, Sect. 2: one (lambda, g) job at a time): one job, one cell-table
   preparation (S1: extinction and emission tables, Sect. 3.6, 4.3, 7) and one transport launch (one
   thread per packet: launch, tau sampling, cell march, interaction and peel-off, Sect. 3, 4.1-4.6;
   chords, Sect. 5.1).
   tallies_out: one column per observer (albedo, emission); transmission: the chord column, plus the
   scattered-light column when the source sets trans_scatter; sums over packets of f (the host divides by N, see gcmc_postscale), in
   host or device memory per tallies_memory.  stats_out may be NULL.  Synchronises the stream
   when tallies_memory is GCMC_MEM_HOST or stats_out is not NULL. */
gcmc_status gcmc_run_packets(gcmc_ctx *ctx, const gcmc_job *job, double *tallies_out, int tallies_memory,
                             gcmc_stats *stats_out);

typedef struct {
    int32_t block;            /* threads per block (multiple of 32), 0 = default */
    int32_t blocks_per_sm;    /* resident blocks per SM of the persistent grid, 0 = as many as fit; with
                                 128-thread blocks, FP32 kernels compiled for more resident blocks (fewer
                                 registers) run from 6 (absorber-only marches: 6 and 8; scattering: 5 and 6)
                                 and 5 (scattering); a value above what fits is lowered to it */
    int32_t chunk;            /* packets per warp work item (multiple of 32), 0 = default (1024) */
    int32_t interval;         /* march steps between warp refill checks, 0 = default (1) */
    int32_t refill_min;       /* refill a warp's idle lanes only when at least this many (1..32) are idle,
                                 or when its work item has no packets left to start; 0 = default (16) */
    int32_t pad;
} gcmc_launch_cfg;

/* Batched form: the jobs the paper's host loop would run one after another (Sect. 2; each job computes
   what gcmc_run_packets computes, Sect. 3-5) as cell tables of every job, then ONE persistent transport
   launch that drains a device work queue of (job, packet range) items.  tallies_out: [n_jobs][GCMC_MAX_OBS].
   stats_out: [n_jobs] or NULL.  cfg may be NULL (defaults). */
gcmc_status gcmc_run_batch(gcmc_ctx *ctx, const gcmc_job *jobs, int n_jobs, const gcmc_launch_cfg *cfg,
                           double *tallies_out, int tallies_memory, gcmc_stats *stats_out);

/* Captured batches (the host loop of Sect. 2 replayed; each job as in Sect. 3-5): the batched form
   (cell tables of every job, one persistent transport launch, tallies) planned once and captured into a CUDA graph on the context's stream (which must not be the
   default stream), to be replayed step after step without host-side planning or launch overhead.
   The graph owns its workspace; the grids, opacities and sources it uses must stay uploaded.
   gcmc_graph_launch replays it asynchronously and, if tallies_out (device [n_jobs][GCMC_MAX_OBS]) is
   not NULL, copies the tallies there; gcmc_graph_read synchronises and returns the last replay's
   tallies (host [n_jobs][GCMC_MAX_OBS], may be NULL) and stats ([n_jobs] or NULL). */
typedef struct gcmc_graph gcmc_graph;
gcmc_status gcmc_graph_create(gcmc_ctx *ctx, const gcmc_job *jobs, int n_jobs, const gcmc_launch_cfg *cfg,
                              gcmc_graph **out);
gcmc_status gcmc_graph_launch(gcmc_graph *g, double *tallies_out);
gcmc_status gcmc_graph_read(gcmc_graph *g, double *tallies_out, gcmc_stats *stats_out);
gcmc_status gcmc_graph_destroy(gcmc_graph *g);

/* Contribution functions (Sect. 6): one albedo or emission job run with per-cell counters of the
   peel-off contributions, attributed to the cell each peel-off leaves from.  cf_out (host,
   [2][n_obs][ncell], n_obs the job's observer count) receives the sums of f over packets, in the
   units of tallies_out: [0] thermal (emission launch peel-offs), [1] scattered (peel-offs at
   scattering events).  They add up, over cells and both kinds, to the job's tally; the paper's
   contribution function of a cell is its share, CF = cf / tally.  tallies_out [GCMC_MAX_OBS] and
   stats_out may be NULL.  Transmission jobs are refused (GCMC_ERR_ARG).  Synchronises the stream. */
gcmc_status gcmc_run_contrib(gcmc_ctx *ctx, const gcmc_job *job, double *tallies_out, double *cf_out,
                             gcmc_stats *stats_out);

/* Asynchronous batched form for request loops (the host loop of Sect. 2 without waiting; each job as
   in Sect. 3-5): enqueue the work on the context's stream and return a ticket at once; gcmc_poll
   returns GCMC_ERR_NOT_READY until the ticket's work has finished, then fills tallies_out
   [n_jobs][GCMC_MAX_OBS] (host) and stats_out (may be NULL). */
gcmc_status gcmc_submit(gcmc_ctx *ctx, const gcmc_job *jobs, int n_jobs, const gcmc_launch_cfg *cfg,
                        uint64_t *ticket);
gcmc_status gcmc_poll(gcmc_ctx *ctx, uint64_t ticket, double *tallies_out, gcmc_stats *stats_out);

/* The number of tally columns `job` writes (into tallies_out of the run calls, and per packet into
   pk_f of gcmc_run_packets_debug): its observer count (1 when obs_idx >= 0) for albedo and
   emission jobs (Sect. 5.2, 5.3); for transmission jobs 1, or 2 with trans_scatter (the chord
   integral of Sect. 5.1, then the scattered part).  Errors: those of the run calls' job checks
   (GCMC_ERR_ARG). */
gcmc_status gcmc_job_columns(gcmc_ctx *ctx, const gcmc_job *job, int32_t *n_cols);

/* Parity/debug form of gcmc_run_packets: runs packets [packet0, packet0 + n_run) of `job` and
   writes per-packet results to HOST arrays: pk_f [n_run][pk_f_cols] (row-major; its first
   gcmc_job_columns columns receive f per tally column, as in gcmc_run_packets, the rest are left
   untouched), pk_steps [n_run], pk_tau [n_run] (optical depth of the packet's first peel-off or
   chord march), and for the first n_trace packets the segment list: tr_cell [n_trace][max_trace]
   (flat cell index, or -1 before a flight, -2 before a peel-off, -3 before a chord), tr_len,
   tr_n [n_trace].  Any output pointer may be NULL.  A pk_f with fewer columns than the job
   writes is refused (GCMC_ERR_ARG) before any work is queued. */
gcmc_status gcmc_run_packets_debug(gcmc_ctx *ctx, const gcmc_job *job, int64_t packet0, int64_t n_run,
                                   double *pk_f, int32_t pk_f_cols, int64_t *pk_steps, double *pk_tau, int32_t n_trace,
                                   int32_t max_trace, int32_t *tr_cell, double *tr_len, int32_t *tr_n,
                                   double *tallies_out, gcmc_stats *stats_out);

/* S1 only: the cell table of `job` copied to HOST arrays of length ncell (any may be NULL):
   alpha (extinction, 1/m), omega, g, pgas (albedo), lum (emission L_i, W/m), cdf, wcell
   (emission cumulative hybrid pdf and launch weight). */
gcmc_status gcmc_prep_cells(gcmc_ctx *ctx, const gcmc_job *job, double *alpha, double *omega, double *g,
                            double *pgas, double *lum, double *cdf, double *wcell, gcmc_stats *stats_out);

/* ---------------------------------------------------------------- host post-scale (Sect. 5) */

typedef struct {
    double S;                 /* albedo: tally / N (reflected fraction per steradian, flux 1 on R_TOA disk) */
    double A_g;               /* albedo: pi S, referenced to the R_TOA disk (Sect. 5.2) */
    double A_g_R0;            /* albedo: pi S (R_TOA / R0)^2, referenced to the R0 disk */
    double L_p;               /* emission: (L_tot / N) tally, W m^-1 sr^-1 (Sect. 5.3) */
    double I_p;               /* emission: L_p / (pi R_TOA^2); transmission: <I_p> (Sect. 5.1) */
    double F_p;               /* emission: pi I_p */
    double area;              /* transmission: R0^2 + 2 <I_p>  (= (R_p/R_star)^2 R_star^2) */
} gcmc_observables;

typedef struct {
    double I_p_direct;        /* (R_TOA - R0)/N R_TOA tally[0]: the chords, weighted by limb darkening */
    double I_p_scattered;     /* (R_TOA - R0)/N R_TOA tally[1]: scattered light, per steradian */
    double omega_star;        /* solid angle of the stellar disk seen from the planet, 2 pi (1 - sqrt(1 - (R_star / d)^2)) */
    double I_p;               /* I_p_direct - omega_star I_p_scattered */
    double w_core;            /* limb-darkening factor at the planet centre (blocked by the opaque core), 1 without */
    double n_ld;              /* disk-averaged I(mu)/I(centre): 2 int_0^1 mu I(mu) dmu / I(1), 1 without */
    double area;              /* w_core R0^2 + 2 I_p */
    double depth;             /* area / (R_star^2 n_ld), the transit depth (0 when star_radius is 0) */
} gcmc_transit_obs;

/* Transit observables (Sect. 5.1) of one transmission job from its tally columns: tally[0] the chords,
   tally[1] the scattered light (read only when the source sets trans_scatter).  The scattered power per
   steradian counts against the blocked area through omega_star, which needs star_radius and star_dist
   (otherwise omega_star = 0).  Errors: GCMC_ERR_ARG (bad ids, n_packets <= 0, NULL pointers). */
gcmc_status gcmc_transit(gcmc_ctx *ctx, int grid_id, int source_id, const double *tally, int64_t n_packets,
                         gcmc_transit_obs *out);

/* Host post-scale (S9) of one job from its tally sum over N packets (l_tot from the job's stats for
   emission): albedo S = tally/N, A_g = pi S (Sect. 5.2); emission L_p = (L_tot/N) tally, I_p =
   L_p/(pi R_TOA^2), F_p = pi I_p (Sect. 5.3); transmission <I_p> = (R_TOA - R0) R_TOA tally/N and the
   area R0^2 + 2 <I_p> (Sect. 5.1, Eq. trans).  Errors: GCMC_ERR_ARG (bad grid id or mode, n_packets <= 0,
   out NULL). */
gcmc_status gcmc_postscale(gcmc_ctx *ctx, int grid_id, int mode, double tally, int64_t n_packets, double l_tot,
                           gcmc_observables *out);

/* ---------------------------------------------------------------- resources and measurement */

/* Free the device memory of a grid (and of every opacity uploaded for it) or of one opacity.
   The ids are not reused.  Errors: GCMC_ERR_ARG for unknown or already released ids. */
gcmc_status gcmc_release_grid(gcmc_ctx *ctx, int grid_id);
gcmc_status gcmc_release_opacity(gcmc_ctx *ctx, int opac_id);

/* Profiling: when on, every run records CUDA events on the context's stream around its cell-table
   kernels and its transport kernel.  gcmc_get_profile synchronises those events and returns the
   summed milliseconds since profiling was switched on (then starts a new sum). */
gcmc_status gcmc_set_profiling(gcmc_ctx *ctx, int on);
gcmc_status gcmc_get_profile(gcmc_ctx *ctx, double *prep_ms, double *transport_ms, int64_t *transport_launches);

/* Process-wide number of kernels libgcmc has launched so far. */
int64_t gcmc_kernel_launches(void);

/* Random-gather rate of this device: n_gathers loads of record_bytes (4 or 16) from a table of
   n_records records at Philox-random indices, one record per thread per iteration (the access
   pattern of the cell march with no arithmetic).  Writes gathers per second. */
gcmc_status gcmc_gather_bench(gcmc_ctx *ctx, int64_t n_records, int record_bytes, int64_t n_gathers,
                              double *gathers_per_s);

/* ---------------------------------------------------------------- allocation-free variant */

/* Largest cell count gcmc_emission_pdf_noalloc accepts (its scratch: 256 KiB per GPU). */
#define GCMC_NOALLOC_MAX_CELLS 4194304

/* The emission pdf stage (hybrid pdf q_i, cumulative sum and launch weights) without any device
   allocation, for callers that cannot call cudaMalloc/cudaFree: code that must not trigger their
   implicit device-wide synchronisation, or hosts that hand a library only pre-allocated device
   memory.  The paper has no counterpart: this is a calling convention of the library.
   All pointers are DEVICE memory owned by the caller:
     lum     [ncell]  luminosity L_i of each cell, W/m; a negative value marks a cell excluded by the
                      tau_vert cut (as the library's own cell-table kernels mark them)
     cdf     [ncell]  out: cumulative hybrid pdf (the pdf of cell i is cdf[i] - cdf[i-1]); may be lum
                      itself (the pdf then replaces the luminosities in place)
     wcell   [ncell]  out: launch weight (L_i / L_tot) / q_i, 0 for excluded cells
     totals  [3]      out: L_tot, number of emitting cells, cdf total (exactly 3 doubles are written)
   Apart from cdf == lum, the four arrays must not overlap.  beta is the hybrid biasing fraction
   (0..1).  Work is queued on `stream` (a cudaStream_t, NULL = default stream); the call returns
   without waiting.  Scratch lives in a fixed array in the library's device memory, one per GPU, held
   until the process exits; the first call on a device looks up its address (do that first call before
   any stream capture).  That look-up is kept for the process: after cudaDeviceReset on a device the
   library's device memory is gone and this entry point must not be called on that device again.
   Every call shares the array, so calls that overlap on the GPU (e.g. on two streams) race: order
   them on one stream.
   Errors: GCMC_ERR_ARG (NULL pointer, ncell < 1, beta outside [0, 1], overlapping arrays),
   GCMC_ERR_RANGE (ncell > GCMC_NOALLOC_MAX_CELLS), GCMC_ERR_CUDA (a CUDA error was already pending
   when the call began -- it is left pending for its owner and nothing is queued -- or one of the
   call's own launches failed, in which case that error is cleared and reported here). */
gcmc_status gcmc_emission_pdf_noalloc(const double *lum, int64_t ncell, double beta, double *cdf, double *wcell,
                                      double *totals, void *stream);

/* ---------------------------------------------------------------- self tests */

/* Philox4x32-10 of the library and cuRAND's curand_Philox4x32_10 on the device for n
   counters/keys (host arrays ctr [n][4], key [n][2]); results to out_lib, out_curand [n][4]. */
gcmc_status gcmc_selftest_philox(gcmc_ctx *ctx, const uint32_t *ctr, const uint32_t *key, int n,
                                 uint32_t *out_lib, uint32_t *out_curand);

/* ---------------------------------------------------------------- serving (continuous batching)

   A request loop over spectrum jobs that arrive while others run.  The paper runs one (lambda, g)
   job after another from a host loop (Sect. 2); this server keeps grids and opacity tables resident
   and overlaps jobs on the device.  One persistent transport kernel drains a queue of published
   jobs in publication order; a job is admitted in arrival order (its cell tables built on a second
   stream, beside the running kernel) once a completion slot is free and its workspace fits in
   hbm_budget bytes together with the other admitted jobs (admission by HBM footprint); it is
   published to the running kernel through host-mapped memory as soon as its cell tables are ready,
   and warps take its work items once the jobs published before it have none left to claim.
   The warp that finishes a job's last work item writes the job's tallies into host-mapped memory.
   A job's tallies do not depend on what else runs: every packet's random numbers are keyed by
   (seed, packet, event, job key) and the sums are 64-bit fixed point, so a job gives bit-identical
   tallies alone and in any mix.

   Ownership: the server uses its context's grids, opacities and sources, which must stay uploaded
   while jobs that use them are queued; it owns its streams, host-mapped buffers and job workspaces.
   A server and its context are used from one host thread.  Jobs run in FP32 (their source's
   precision must be GCMC_FP32), on grids no larger (in nr + nlat + nlon) than the largest grid
   present when the server was created, with n_packets >= 1. */
typedef struct gcmc_server gcmc_server;

typedef struct {
    int32_t block;            /* threads per block of the serving kernel: 0 or 128 */
    int32_t blocks_per_sm;    /* 0 = one block per SM less than fits (room for cell-table kernels) */
    int32_t chunk;            /* packets per warp work item, multiple of 32; 0 = 256 */
    int32_t interval;         /* march steps between refill checks; 0 = 4 */
    int32_t refill_min;       /* see gcmc_launch_cfg; 0 = 8 */
    int32_t max_jobs;         /* jobs admitted at once (completion slots), 1..32768; 0 = 1024 */
    uint64_t hbm_budget;      /* bytes of job workspace admitted at once; 0 = 8 GiB.  A job larger than
                                 the budget is admitted alone. */
    int32_t idle_us;          /* the serving kernel leaves after about this many microseconds without
                                 published work (it is relaunched when work arrives); 0 = 2000 */
    int32_t pad;
} gcmc_server_cfg;

typedef struct {
    int64_t pending;          /* submitted, waiting for admission */
    int64_t admitted;         /* admitted and not yet complete */
    int64_t completed;        /* completed since creation */
    uint64_t bytes_in_use;    /* workspace of the admitted jobs */
    int64_t kernel_launches;  /* serving-kernel launches since creation */
    int32_t kernel_running;   /* 1 while the serving kernel is resident */
    int32_t grid_blocks;      /* blocks of the last serving-kernel launch */
} gcmc_server_stats;

/* Create the server of a context (cfg may be NULL: all defaults).  Errors: GCMC_ERR_ARG (NULL ctx or
   out, block other than 0 or 128, chunk not a multiple of 32, max_jobs above 32768, no grid uploaded
   yet), GCMC_ERR_OOM, GCMC_ERR_CUDA. */
gcmc_status gcmc_server_create(gcmc_ctx *ctx, const gcmc_server_cfg *cfg, gcmc_server **out);

/* Queue one job (copied); returns its ticket.  Nothing is launched until gcmc_server_progress.
   Errors: GCMC_ERR_ARG for a job that gcmc_run_packets would refuse, or with n_packets < 1, an FP64
   source, a band job (g_idx = -1: submit one job per g-ordinate), or a grid larger than every grid
   present when the server was created. */
gcmc_status gcmc_server_submit(gcmc_server *sv, const gcmc_job *job, uint64_t *ticket);

/* One pass of the request loop, never blocking: collect completed jobs (their tickets are written to
   done_tickets, at most cap of them; *n_done counts all), admit queued jobs that fit, publish those
   whose cell tables are ready, and (re)launch the serving kernel if published work has none. */
gcmc_status gcmc_server_progress(gcmc_server *sv, uint64_t *done_tickets, int cap, int *n_done);

/* Tallies [GCMC_MAX_OBS] (sums of f over packets, as gcmc_run_batch) and stats (may be NULL) of a
   completed job; GCMC_ERR_NOT_READY if the ticket has not completed (or was already taken). */
gcmc_status gcmc_server_result(gcmc_server *sv, uint64_t ticket, double *tallies_out, gcmc_stats *stats_out);

/* Host times of a completed job that gcmc_server_result has not yet taken, in seconds since the
   server was created: t4 = {submitted, admitted (cell tables queued), published, completion seen}. */
gcmc_status gcmc_server_times(gcmc_server *sv, uint64_t ticket, double *t4);

gcmc_status gcmc_server_query(gcmc_server *sv, gcmc_server_stats *stats);

/* Stop the server: published jobs finish first.  Returns GCMC_ERR_TIMEOUT, and frees nothing, if the
   serving kernel has not finished within timeout_s seconds; queued (unadmitted) jobs are dropped. */
gcmc_status gcmc_server_destroy(gcmc_server *sv, double timeout_s);

/* Library version string. */
const char *gcmc_version(void);

#ifdef __cplusplus
}
#endif
#endif /* GCMC_H */
