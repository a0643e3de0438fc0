/*
 * oracle.c -- plain, slow, FP64 CPU Monte Carlo radiative transfer (gCMCRT method).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the independent reference that the CUDA
 * path is checked against.  Only the test suite, the smoke check and the benchmark's
 * CPU-baseline leg may load it; the product path never does.  It shares no code,
 * header, table or constant generator with the CUDA library.
 *
 * What it follows (Lee et al. 2022, "gCMCRT", arXiv:2110.15640):
 *   Sect. 2   packets move through a 3D spherical lon x lat x r grid (sub-grid positions)
 *   Sect. 3   isotropic, Rayleigh and Henyey-Greenstein phase functions and samplers;
 *             gas/cloud scatterer choice with P_gas = k_Ray / (k_Ray + k_sca,cld)
 *   Sect. 4   survival biasing, Russian roulette, next-event (peel-off) estimation
 *             f = W omega Theta exp(-tau_obs), emission hybrid biasing and the tau_vert cut
 *   Sect. 5   transmission estimator <I_p> = (R_TOA - R0)/N sum W (1 - e^-tau) b,
 *             albedo normalisation (incident flux 1), emission L_i = 4 pi V rho kappa B
 *   Sect. 7   line-of-sight velocity and Doppler-shifted opacity lambda_eff = lambda0 (1 - v/c)
 *
 * Readings where the paper is silent or garbled (each one is a choice both sides make):
 *   - Rayleigh sampler: exact inverse CDF of p(mu) = 3/8 (1 + mu^2):  q = 4 zeta - 2,
 *     u = cbrt(q + sqrt(q^2 + 1)), mu = u - 1/u  (the printed formula is garbled).
 *   - HG sampler at |g| < eps: isotropic mu = 2 zeta - 1 (the printed form is 0/0 at g = 0).
 *   - Theta = expected phase function / (4 pi):  (P_gas P_Ray + (1 - P_gas) P_HG) / (4 pi).
 *     Emission launch peel-off: Theta = 1/(4 pi) without omega.
 *   - Survival biasing by default; roulette when W < w_rr W_launch, survive with p_surv.
 *   - Peel-off / chord marches stop once tau > tau_peel_cut (contribution taken as exp(-tau) = 0
 *     for peel-offs and 1 - exp(-tau) = 1 for chords).
 *   - Albedo launch: b = R_TOA sqrt(z1), psi = 2 pi z2 on the TOA disk facing the star,
 *     moving along -star, launch weight 1 (the host divides by N).
 *   - Emission: hybrid pdf q_i = (1 - beta) L_i/L_tot + beta/N'_c over the cells whose vertical
 *     optical depth above them is < tau_vert_max; W = (L_i/L_tot)/q_i; the cell is drawn by
 *     inverse CDF with the stratified uniform (n + z)/N (the per-cell allocation
 *     N_i ~ N q_i of Sect. 4.3); position uniform in r^3, sin(lat), lon.
 *   - Transmission: b ~ U[R0, R_TOA], psi ~ U[0, 2 pi), chord along -star, W = 1, or with stellar
 *     limb darkening W = I(mu)/I(centre) at the chord's position on the stellar disk (0 off the
 *     disk: not traced).  The chord gives column 0, W (1 - e^-tau) b / R_TOA.  With multiple
 *     scattering the packet then flies from its launch point along -star; each scattering peels off
 *     towards -star into column 1 with f b / R_TOA (the host subtracts Omega_star times it).
 *     A packet's weight ends in exactly one ledger entry (a capped chord: "capped" only).
 *   - Doppler: theta, theta_v in the v_LOS formula are polar angles (colatitudes);
 *     v_LOS > 0 is motion away from the observer; opacity interpolated linearly in ln(sigma)
 *     between the bracketing table wavelengths (weight linear in lambda), bilinear in
 *     (ln T, ln p), clamped at the table edges.
 *   - RNG: Philox4x32-10 (Salmon et al. 2011), key = seed, counter = (packet lo, packet hi,
 *     event, job key); event 0 launch, event 1 emission direction, event 2 + n flight n
 *     (words: tau, scatterer, mu, azimuth); event | 2^31: words (analog absorb, roulette).
 *     Uniform = ((w >> 8) + 0.5) 2^-24.
 *
 * Pins: tests/test_oracle_*.py check every function here against something other than itself (known-
 * answer vectors, closed forms, brute-force ray enumeration, an independent adding-doubling solver,
 * limits with analytic answers, exact ledger closure); tests/plant_mistakes.py plants slips in a copy
 * of this file and checks that the pins catch them.
 *
 * Geometry (written plainly): from the current point, every face of the current cell is
 * intersected (two shells, two latitude cones or the equator plane, two longitude
 * half-planes); the nearest root with t > 0 wins, ties in face order (r-, r+, lat-, lat+,
 * lon-, lon+); on the face a packet just entered, the root nearest t = 0 is dropped.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_PI 3.14159265358979323846
#define ORC_C_LIGHT 2.99792458e8
#define ORC_H 6.62607015e-34
#define ORC_KB 1.380649e-23
#define ORC_MAX_OBS 32

/* ------------------------------------------------------------------ public structs */
typedef struct {
    int32_t nlon, nlat, nr, pad;
    const double *r_edges, *lat_edges, *lon_edges;
} orc_grid;

typedef struct {
    const double *alpha;   /* [ncell] extinction, 1/m */
    const double *omega;   /* [ncell] single-scattering albedo or NULL (0) */
    const double *g;       /* [ncell] HG asymmetry or NULL (0) */
    const double *pgas;    /* [ncell] P_gas or NULL (1) */
    const double *cdf;     /* emission: [ncell] cumulative hybrid pdf */
    const double *wcell;   /* emission: [ncell] launch weight */
    double cdf_total;
    double pad;
    /* emission with per-packet g-ordinate sampling (Sect. 4.7): alpha, cdf and wcell hold ng tables
       [g][ncell]; packet g is drawn with probability q(g) and carries W_g = p(g) / q(g) */
    int32_t ng, pad2;
    const double *g_qcdf;  /* [ng] cumulative q(g) */
    const double *g_w;     /* [ng] W_g */
    const double *g_cdftot;/* [ng] total of each g's cumulative hybrid pdf */
} orc_cells;

typedef struct {
    double star[3];
    int32_t n_obs, survival;
    double obs[ORC_MAX_OBS][3];
    double w_rr, p_surv, tau_peel_cut, tau_vert_max, beta_emis, hg_iso_eps;
    int32_t scatter_emission, pad;
    int64_t max_steps;
    int32_t cloud_phase;   /* 0: Henyey-Greenstein; 1: two-term HG with the paper's defaults (Sect. 3) */
    int32_t pad2;
    double surface_albedo; /* Lambertian lower boundary of this albedo (0: black) */
    int32_t trans_scatter; /* transmission: after the chord the packet scatters, with peel-offs towards
                              the transit observer (Sect. 5.1); needs scattering cell records */
    int32_t ld_law;        /* stellar limb-darkening law (Sect. 5.1): 0 none, 1 linear, 2 quadratic,
                              3 square-root, 4 logarithmic, 5 power-2, 6 four-coefficient */
    double ld_coef[4];
    double star_radius;    /* m */
    double star_dist;      /* m (used by the host post-scale only) */
    double transit_xy[2];  /* planet centre on the sky plane relative to the stellar disk centre, along the
                              launch basis (e1, e2), m */
    int32_t g_bias;        /* (the library's band-job options; the oracle reads its g table from orc_cells) */
    int32_t pad3;
    double g_beta;
    int32_t forced_first;  /* biased flights (Sect. 4.2): 1 the first flight only, 2 every flight */
    int32_t cont_abs;      /* continuous absorption (Sect. 4.1) */
    int32_t path_bias;     /* how biased flights sample tau: 0 forced scattering, 1 path length stretching,
                              2 hybrid forced scattering with path length stretching */
    int32_t pad4;
} orc_source;

typedef struct {
    int32_t mode;          /* 0 albedo, 1 emission, 2 transmission */
    uint32_t job_key;
    uint64_t seed;
    int64_t n_packets;     /* N used in the stratified emission draw and in the job */
    int64_t packet0;       /* first packet index to run */
    int64_t n_run;         /* number of packets to run from packet0 */
    int32_t nthreads, n_trace, max_trace, pad;
    double *tally;         /* [n_obs] sum of f */
    double *ledger;        /* [8] emitted, escaped, absorbed, bottom, rr_gain, rr_loss, capped, lost */
    int64_t *steps;        /* [1] packet-steps */
    double *pk_f;          /* [n_run][n_obs] or NULL */
    int64_t *pk_steps;     /* [n_run] or NULL */
    double *pk_tau;        /* [n_run] tau of the packet's first peel-off / chord march, or NULL */
    int32_t *tr_cell;      /* [n_trace][max_trace] flat cell index, or -1 - kind at a march start */
    double *tr_len;        /* [n_trace][max_trace] */
    int32_t *tr_n;         /* [n_trace] entries written */
    double *cf;            /* contribution functions (Sect. 6), or NULL: [2][n_obs][ncell] sums of the
                              peel-off contributions f by the cell they leave from; [0] thermal (the
                              emission launch peel-off), [1] scattered (peel-offs at scattering events) */
    double *tr_pos;        /* [n_trace][max_trace][3] or NULL: the end point of each traced segment (the
                              interaction point, or the crossing point of the face it leaves by); at a
                              march start (cell < 0) the point the march starts from.  Logging only. */
} orc_run_args;

/* ------------------------------------------------------------------ Philox4x32-10 */
/* Counter-based generator of Salmon et al. (2011, SC'11), written from its published definition: ten
   rounds, each two 32 x 32 -> 64-bit products of counter words with the round multipliers, the high
   halves XORed with the other counter words and the key, the key bumped by the Weyl constants between
   rounds.  The paper does not name its generator; a counter keyed by (packet, event, job) makes every
   packet's stream independent of how packets are scheduled. */
static inline uint32_t mulhilo(uint32_t a, uint32_t b, uint32_t *hi)
{
    uint64_t p = (uint64_t)a * (uint64_t)b;
    *hi = (uint32_t)(p >> 32);
    return (uint32_t)p;
}

void orc_philox(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
        uint32_t hi0, hi1;
        uint32_t lo0 = mulhilo(0xD2511F53u, c0, &hi0);
        uint32_t lo1 = mulhilo(0xCD9E8D57u, c2, &hi1);
        uint32_t n0 = hi1 ^ c1 ^ k0, n1 = lo1, n2 = hi0 ^ c3 ^ k1, n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

static inline double u01(uint32_t w) { return ((double)(w >> 8) + 0.5) * (1.0 / 16777216.0); }

static void draw(uint64_t seed, int64_t packet, uint32_t event, uint32_t job, double u[4])
{
    uint32_t ctr[4] = {(uint32_t)(uint64_t)packet, (uint32_t)((uint64_t)packet >> 32), event, job};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t w[4];
    orc_philox(ctr, key, w);
    for (int i = 0; i < 4; ++i) u[i] = u01(w[i]);
}

/* ------------------------------------------------------------------ samplers (Sect. 3) */
double orc_sample_iso(double z) { return 2.0 * z - 1.0; }

double orc_sample_rayleigh(double z)
{
    double q = 4.0 * z - 2.0;
    double u = cbrt(q + sqrt(q * q + 1.0));
    return u - 1.0 / u;
}

double orc_sample_hg(double g, double z, double eps)
{
    if (fabs(g) < eps) return 2.0 * z - 1.0;
    double a = (1.0 - g * g) / (1.0 - g + 2.0 * g * z);
    double mu = (1.0 + g * g - a * a) / (2.0 * g);
    if (mu > 1.0) mu = 1.0;
    if (mu < -1.0) mu = -1.0;
    return mu;
}

double orc_phase_rayleigh(double mu) { return 0.75 * (1.0 + mu * mu); }

double orc_phase_hg(double mu, double g)
{
    double den = 1.0 + g * g - 2.0 * g * mu;
    return (1.0 - g * g) / (den * sqrt(den));
}

/* Theta: probability per steradian of scattering into cos(theta) = mu for the gas/cloud mixture */
double orc_theta(double mu, double pgas, double g)
{
    return (pgas * orc_phase_rayleigh(mu) + (1.0 - pgas) * orc_phase_hg(mu, g)) / (4.0 * ORC_PI);
}

/* two-term HG (Sect. 3): P = a P_HG(g1) + (1 - a) P_HG(g2), with the defaults the paper uses for a
   single asymmetry factor g: g1 = g, g2 = -g/2, a = 1 - g2^2 */
void orc_tthg_params(double g, double *g1, double *g2, double *a)
{
    *g1 = g;
    *g2 = -0.5 * g;
    *a = 1.0 - (*g2) * (*g2);
}

double orc_phase_tthg(double mu, double g)
{
    double g1, g2, a;
    orc_tthg_params(g, &g1, &g2, &a);
    return a * orc_phase_hg(mu, g1) + (1.0 - a) * orc_phase_hg(mu, g2);
}

/* expected phase function per steradian of the gas / cloud mixture, cloud phase function of the kind */
double orc_theta_kind(double mu, double pgas, double g, int kind)
{
    const double pc = kind == 1 ? orc_phase_tthg(mu, g) : orc_phase_hg(mu, g);
    return (pgas * orc_phase_rayleigh(mu) + (1.0 - pgas) * pc) / (4.0 * ORC_PI);
}

/* limb-darkening laws (Sect. 5.1: the stellar intensity at zenith-angle cosine mu relative to the disk
   centre, mu = 1); each of these equals 1 at mu = 1.  Negative values (bad coefficients) count as 0. */
double orc_limb(int law, const double c[4], double mu)
{
    const double x = 1.0 - mu;
    double I;
    switch (law) {
    case 1: I = 1.0 - c[0] * x; break;
    case 2: I = 1.0 - c[0] * x - c[1] * x * x; break;
    case 3: I = 1.0 - c[0] * x - c[1] * (1.0 - sqrt(mu)); break;
    case 4: I = 1.0 - c[0] * x - c[1] * (mu > 0.0 ? mu * log(mu) : 0.0); break;
    case 5: I = 1.0 - c[0] * (1.0 - pow(mu, c[1])); break;
    case 6:
        I = 1.0;
        for (int k = 1; k <= 4; ++k) I -= c[k - 1] * (1.0 - pow(mu, 0.5 * k));
        break;
    default: I = 1.0;
    }
    return I > 0.0 ? I : 0.0;
}

/* cosine of a cloud scattering: HG, or the two-term HG, whose term is chosen by zc < a (zc uniform) */
double orc_sample_cloud(double g, double zc, double z, double eps, int kind)
{
    if (kind != 1) return orc_sample_hg(g, z, eps);
    double g1, g2, a;
    orc_tthg_params(g, &g1, &g2, &a);
    return orc_sample_hg(zc < a ? g1 : g2, z, eps);
}

/* new direction at polar angle acos(mu) and azimuth psi about d; the azimuth origin is the
   unit vector e1 = (dx dz, dy dz, -(1 - dz^2)) / sqrt(1 - dz^2), e2 = (-dy, dx, 0) / sqrt(1 - dz^2) */
void orc_turn(const double d[3], double mu, double psi, double out[3])
{
    double s = sqrt(fmax(0.0, 1.0 - mu * mu));
    double cp = cos(psi), sp = sin(psi);
    if (fabs(d[2]) < 0.99999) {
        double den = sqrt(1.0 - d[2] * d[2]);
        double e1[3] = {d[0] * d[2] / den, d[1] * d[2] / den, -den};
        double e2[3] = {-d[1] / den, d[0] / den, 0.0};
        for (int i = 0; i < 3; ++i) out[i] = mu * d[i] + s * (cp * e1[i] + sp * e2[i]);
    } else {
        out[0] = s * cp;
        out[1] = s * sp;
        out[2] = (d[2] > 0 ? 1.0 : -1.0) * mu;
    }
    double n = sqrt(out[0] * out[0] + out[1] * out[1] + out[2] * out[2]);
    out[0] /= n; out[1] /= n; out[2] /= n;
}

/* ------------------------------------------------------------------ geometry */
enum { F_RIN = 0, F_ROUT = 1, F_LATLO = 2, F_LATHI = 3, F_LONLO = 4, F_LONHI = 5 };
enum { END_INTERACT = 0, END_ESCAPE = 1, END_BOTTOM = 2, END_CUTOFF = 3, END_CAP = 4, END_LOST = 5 };

static inline double dot3(const double a[3], const double b[3]) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

/* Face intersections of the spherical grid (Sect. 2: cells bounded by two radial shells, two latitude
   cones and two longitude half-planes).  The two roots of t^2 + 2 b t + c = 0 (shells), in the stable
   form; returns the count. */
static int shell_roots(const double x[3], const double d[3], double r, double t[2])
{
    double b = dot3(x, d);
    double c = dot3(x, x) - r * r;
    double disc = b * b - c;
    if (disc < 0.0) return 0;
    double sq = sqrt(disc);
    double q = -(b + (b >= 0 ? sq : -sq));
    if (q == 0.0) { t[0] = 0.0; return 1; }
    t[0] = q;
    t[1] = c / q;
    return 2;
}

/* roots of the cone z = r sin(theta) (one nappe, sign of z = sign of theta) or the plane z = 0 */
static int cone_roots(const double x[3], const double d[3], double theta, double t[2])
{
    double s = sin(theta);
    int n = 0;
    if (fabs(theta) < 1e-15) {
        if (d[2] == 0.0) return 0;
        t[0] = -x[2] / d[2];
        return 1;
    }
    double s2 = s * s;
    double A = d[2] * d[2] - s2;
    double B = x[2] * d[2] - s2 * dot3(x, d);
    double C = x[2] * x[2] - s2 * dot3(x, x);
    double cand[2];
    int m = 0;
    if (fabs(A) < 1e-300) {
        if (B == 0.0) return 0;
        cand[m++] = -C / (2.0 * B);
    } else {
        double disc = B * B - A * C;
        if (disc < 0.0) return 0;
        double sq = sqrt(disc);
        double q = -(B + (B >= 0 ? sq : -sq));
        if (q == 0.0) {
            cand[m++] = 0.0;
        } else {
            cand[m++] = q / A;
            cand[m++] = C / q;
        }
    }
    for (int i = 0; i < m; ++i) {
        double z = x[2] + cand[i] * d[2];
        if ((theta > 0 && z > 0) || (theta < 0 && z < 0)) t[n++] = cand[i];
    }
    return n;
}

/* root of the half-plane at longitude phi (points with azimuth phi) */
static int lon_root(const double x[3], const double d[3], double phi, double t[1])
{
    double c = cos(phi), s = sin(phi);
    double nx = -s * x[0] + c * x[1];
    double nd = -s * d[0] + c * d[1];
    if (nd == 0.0) return 0;
    double tt = -nx / nd;
    double along = c * (x[0] + tt * d[0]) + s * (x[1] + tt * d[1]);
    if (!(along > 0.0)) return 0;
    t[0] = tt;
    return 1;
}

typedef struct {
    const orc_grid *G;
    const double *alpha;
    int64_t steps, max_steps;
    /* trace */
    int32_t *tr_cell;
    double *tr_len;
    int32_t tr_n, tr_max;
    /* a second optical depth accumulated along the same path (continuous absorption), or NULL */
    const double *alpha2;
    double tau2;
    double *tr_pos;    /* [tr_max][3] or NULL */
} march_ctx;

static inline int64_t flat(const orc_grid *G, const int c[3]) { return ((int64_t)c[2] * G->nlat + c[1]) * G->nlon + c[0]; }

static void trace_put(march_ctx *M, int32_t cell, double len, const double x[3])
{
    if (M->tr_cell && M->tr_n < M->tr_max) {
        M->tr_cell[M->tr_n] = cell;
        M->tr_len[M->tr_n] = len;
        if (M->tr_pos)
            for (int i = 0; i < 3; ++i) M->tr_pos[3 * M->tr_n + i] = x[i];
        M->tr_n++;
    }
}

/* Locate the latitude / longitude bin of a point (radial index given by the caller). */
static void locate_angles(const orc_grid *G, const double x[3], int c[3])
{
    double lat = atan2(x[2], sqrt(x[0] * x[0] + x[1] * x[1]));
    double lon = atan2(x[1], x[0]);
    double lo0 = G->lon_edges[0];
    while (lon < lo0) lon += 2.0 * ORC_PI;
    while (lon >= lo0 + 2.0 * ORC_PI) lon -= 2.0 * ORC_PI;
    int j = 0;
    while (j < G->nlat - 1 && lat >= G->lat_edges[j + 1]) ++j;
    int i = 0;
    while (i < G->nlon - 1 && lon >= G->lon_edges[i + 1]) ++i;
    c[0] = i;
    c[1] = j;
}

/*
 * March a straight ray from x (inside cell c; on face `entry` if entry >= 0) along d.
 * tau_target >= 0: stop where the accumulated optical depth reaches it (END_INTERACT).
 * tau_target <  0: run to the boundary, or stop once tau exceeds tau_cut (END_CUTOFF).
 * On return x is the end point and c its cell.
 */
static int march(march_ctx *M, double x[3], const double d[3], int c[3], int entry, double tau_target,
                 double tau_cut, double *tau_acc)
{
    const orc_grid *G = M->G;
    for (;;) {
        if (M->steps >= M->max_steps) return END_CAP;
        double best = INFINITY;
        int bestf = -1;
        for (int f = 0; f < 6; ++f) {
            double t[2];
            int n = 0;
            switch (f) {
            case F_RIN: n = shell_roots(x, d, G->r_edges[c[2]], t); break;
            case F_ROUT: n = shell_roots(x, d, G->r_edges[c[2] + 1], t); break;
            case F_LATLO: if (c[1] > 0) n = cone_roots(x, d, G->lat_edges[c[1]], t); break;
            case F_LATHI: if (c[1] < G->nlat - 1) n = cone_roots(x, d, G->lat_edges[c[1] + 1], t); break;
            case F_LONLO: if (G->nlon > 1) n = lon_root(x, d, G->lon_edges[c[0]], t); break;
            case F_LONHI: if (G->nlon > 1) n = lon_root(x, d, G->lon_edges[c[0] + 1], t); break;
            }
            if (f == entry) {
                if (f >= F_LONLO) n = 0;              /* a half-plane is crossed once */
                else if (n == 2) {                    /* drop the root at the entry point */
                    if (fabs(t[0]) <= fabs(t[1])) t[0] = t[1];
                    n = 1;
                } else n = 0;
            }
            for (int q = 0; q < n; ++q)
                if (t[q] > 0.0 && t[q] < best) { best = t[q]; bestf = f; }
        }
        M->steps++;
        int64_t idx = flat(G, c);
        double a = M->alpha[idx];
        if (bestf < 0) return END_LOST;
        if (tau_target >= 0.0 && a > 0.0 && *tau_acc + a * best >= tau_target) {
            double l = (tau_target - *tau_acc) / a;
            for (int i = 0; i < 3; ++i) x[i] += l * d[i];
            *tau_acc = tau_target;
            if (M->alpha2) M->tau2 += M->alpha2[idx] * l;
            trace_put(M, (int32_t)idx, l, x);
            return END_INTERACT;
        }
        *tau_acc += a * best;
        if (M->alpha2) M->tau2 += M->alpha2[idx] * best;
        for (int i = 0; i < 3; ++i) x[i] += best * d[i];
        trace_put(M, (int32_t)idx, best, x);
        switch (bestf) {
        case F_RIN:
            if (c[2] == 0) return END_BOTTOM;
            c[2] -= 1; entry = F_ROUT; break;
        case F_ROUT:
            if (c[2] == G->nr - 1) return END_ESCAPE;
            c[2] += 1; entry = F_RIN; break;
        case F_LATLO: c[1] -= 1; entry = F_LATHI; break;
        case F_LATHI: c[1] += 1; entry = F_LATLO; break;
        case F_LONLO: c[0] = (c[0] + G->nlon - 1) % G->nlon; entry = F_LONHI; break;
        case F_LONHI: c[0] = (c[0] + 1) % G->nlon; entry = F_LONLO; break;
        }
        if (tau_target < 0.0 && *tau_acc > tau_cut) return END_CUTOFF;
    }
}

/* Exported for the brute-force geometry tests: trace one ray, return its segment list. */
int orc_trace_ray(const orc_grid *G, const double *alpha, const double o[3], const double d[3],
                  int32_t start_cell_flat, int32_t entry_face, int32_t max_seg,
                  int32_t *cells, double *lens, int32_t *end_status)
{
    march_ctx M = {G, alpha, 0, (int64_t)1 << 40, cells, lens, 0, max_seg, NULL, 0.0};
    double x[3] = {o[0], o[1], o[2]};
    int c[3];
    c[0] = start_cell_flat % G->nlon;
    c[1] = (start_cell_flat / G->nlon) % G->nlat;
    c[2] = start_cell_flat / (G->nlon * G->nlat);
    double tau = 0.0;
    *end_status = march(&M, x, d, c, entry_face, -1.0, INFINITY, &tau);
    return M.tr_n;
}

/* ------------------------------------------------------------------ S1: cell tables */
static void interp_idx(const double *grid, int n, double v, int *a, double *w)
{
    /* bracket ln(v) on ln(grid) with clamping; grid increasing, n >= 2 */
    if (v <= grid[0]) { *a = 0; *w = 0.0; return; }
    if (v >= grid[n - 1]) { *a = n - 2; *w = 1.0; return; }
    int lo = 0, hi = n - 1;
    while (hi - lo > 1) {
        int mid = (lo + hi) / 2;
        if (grid[mid] <= v) lo = mid; else hi = mid;
    }
    *a = lo;
    *w = (log(v) - log(grid[lo])) / (log(grid[lo + 1]) - log(grid[lo]));
}

/* Albedo cell records: alpha_ext, omega, g, P_gas (Sect. 3.6 mixture) */
void orc_prep_albedo(int64_t ncell, const double *rho, const double *acld, double kabs, double kray,
                     double qcld, double wcld, double gcld, double *alpha, double *omega, double *g,
                     double *pgas)
{
    for (int64_t i = 0; i < ncell; ++i) {
        double ac = acld ? acld[i] * qcld : 0.0;
        double ray = rho[i] * kray;
        double ext = rho[i] * (kabs + kray) + ac;
        double sca = ray + wcld * ac;
        alpha[i] = ext;
        omega[i] = ext > 0.0 ? sca / ext : 0.0;
        pgas[i] = sca > 0.0 ? ray / sca : 1.0;
        g[i] = gcld;
    }
}

static double planck_lambda(double lam, double T)
{
    double x = ORC_H * ORC_C_LIGHT / (lam * ORC_KB * T);
    return 2.0 * ORC_H * ORC_C_LIGHT * ORC_C_LIGHT / pow(lam, 5.0) / expm1(x);
}

double orc_planck(double lam, double T) { return planck_lambda(lam, T); }

/* Emission cell tables for one (band, g): alpha = rho k(T, p); L_i = 4 pi V_i alpha_i B(T_i);
   hybrid pdf over the cells with vertical tau above them < tau_vert_max; cdf and launch weight. */
void orc_emission_tables(const orc_grid *G, const double *T, const double *alpha, double lam, double tau_vert_max,
                         double beta, double *L, double *cdf, double *wcell, double *out_Ltot,
                         double *out_cdf_total, int64_t *out_nincl);

void orc_prep_emission(const orc_grid *G, const double *T, const double *p, const double *rho,
                       const float *ktab /* [nT][np] slice for this (band, g) */, int nT, int np,
                       const double *Tg, const double *pg, double lam, double tau_vert_max, double beta,
                       double *alpha, double *L, double *cdf, double *wcell, double *out_Ltot,
                       double *out_cdf_total, int64_t *out_nincl)
{
    int64_t nl = G->nlon, nt = G->nlat, nr = G->nr;
    int64_t ncell = nl * nt * nr;
    for (int64_t idx = 0; idx < ncell; ++idx) {
        int a, b;
        double wT, wp;
        interp_idx(Tg, nT, T[idx], &a, &wT);
        interp_idx(pg, np, p[idx], &b, &wp);
        double l00 = log((double)ktab[a * np + b]), l10 = log((double)ktab[(a + 1) * np + b]);
        double l01 = log((double)ktab[a * np + b + 1]), l11 = log((double)ktab[(a + 1) * np + b + 1]);
        double lk = (1 - wT) * (1 - wp) * l00 + wT * (1 - wp) * l10 + (1 - wT) * wp * l01 + wT * wp * l11;
        alpha[idx] = rho[idx] * exp(lk);
    }
    orc_emission_tables(G, T, alpha, lam, tau_vert_max, beta, L, cdf, wcell, out_Ltot, out_cdf_total, out_nincl);
}

/* Emission cell tables from the cells' extinction alpha (Sect. 4.3, 4.6): the tau_vert cut (a cell emits
   while the vertical optical depth above it is below tau_vert_max), L_i = 4 pi V_i alpha_i B_lambda(T_i),
   the hybrid pdf q_i = (1 - beta) L_i / L_tot + beta / n_incl, its cumulative sum and the launch weights
   (L_i / L_tot) / q_i.  Used with k-table opacities and with Doppler-shifted cross-sections (Sect. 7). */
void orc_emission_tables(const orc_grid *G, const double *T, const double *alpha, double lam, double tau_vert_max,
                         double beta, double *L, double *cdf, double *wcell, double *out_Ltot,
                         double *out_cdf_total, int64_t *out_nincl)
{
    int64_t nl = G->nlon, nt = G->nlat, nr = G->nr;
    int64_t ncell = nl * nt * nr;
    /* volumes and luminosities */
    char *incl = (char *)calloc((size_t)ncell, 1);
    for (int64_t j = 0; j < nt; ++j)
        for (int64_t i = 0; i < nl; ++i) {
            double tau_above = 0.0;
            for (int64_t k = nr - 1; k >= 0; --k) {
                int64_t idx = (k * nt + j) * nl + i;
                incl[idx] = tau_above < tau_vert_max;
                tau_above += alpha[idx] * (G->r_edges[k + 1] - G->r_edges[k]);
            }
        }
    double Ltot = 0.0;
    int64_t nincl = 0;
    for (int64_t idx = 0; idx < ncell; ++idx) {
        int64_t i = idx % nl, j = (idx / nl) % nt, k = idx / (nl * nt);
        double r1 = G->r_edges[k], r2 = G->r_edges[k + 1];
        double V = (r2 * r2 * r2 - r1 * r1 * r1) / 3.0 * (sin(G->lat_edges[j + 1]) - sin(G->lat_edges[j])) *
                   (G->lon_edges[i + 1] - G->lon_edges[i]);
        L[idx] = 4.0 * ORC_PI * V * alpha[idx] * planck_lambda(lam, T[idx]);
        if (incl[idx]) { Ltot += L[idx]; nincl++; }
    }
    double run = 0.0;
    for (int64_t idx = 0; idx < ncell; ++idx) {
        double q = 0.0, w = 0.0;
        if (incl[idx] && nincl > 0) {
            if (Ltot > 0.0) {
                q = (1.0 - beta) * L[idx] / Ltot + beta / (double)nincl;
                w = q > 0.0 ? (L[idx] / Ltot) / q : 0.0;
            } else {
                q = 1.0 / (double)nincl;
                w = 0.0;
            }
        }
        run += q;
        cdf[idx] = run;
        wcell[idx] = w;
    }
    free(incl);
    *out_Ltot = Ltot;
    *out_cdf_total = run;
    *out_nincl = nincl;
}

/* Transmission cell table at rest wavelength lam0: per-cell v_LOS (Sect. 7), lambda_eff,
   sigma interpolated in ln sigma (linear weight in lambda), bilinear in (ln T, ln p). */
void orc_prep_xsec(const orc_grid *G, const double *T, const double *p, const double *rho,
                   const double *wind /* [3][ncell] or NULL */, const float *sig /* [nl][nT][np] */,
                   int nl, int nT, int np, const double *lamg, const double *Tg, const double *pg,
                   double lam0, double view_theta, double view_phi, double omega_rot, double *alpha,
                   double *vlos_out)
{
    int64_t nlon = G->nlon, nlat = G->nlat, nr = G->nr;
    int64_t ncell = nlon * nlat * nr;
    for (int64_t idx = 0; idx < ncell; ++idx) {
        int64_t i = idx % nlon, j = (idx / nlon) % nlat, k = idx / (nlon * nlat);
        double v = 0.0;
        if (wind) {
            double lat = 0.5 * (G->lat_edges[j] + G->lat_edges[j + 1]);
            double th = 0.5 * ORC_PI - lat;                       /* polar angle of the cell */
            double ph = 0.5 * (G->lon_edges[i] + G->lon_edges[i + 1]);
            double rmid = 0.5 * (G->r_edges[k] + G->r_edges[k + 1]);
            double u = wind[idx], vv = wind[ncell + idx], w = wind[2 * ncell + idx];
            double dph = ph - view_phi;
            v = u * sin(view_theta) * sin(dph) + (vv * cos(th) - w * sin(th)) * sin(view_theta) * cos(dph) -
                (vv * sin(th) + w * cos(th)) * cos(view_theta) +
                omega_rot * rmid * sin(th) * sin(view_theta) * sin(dph);
        }
        if (vlos_out) vlos_out[idx] = v;
        double le = lam0 * (1.0 - v / ORC_C_LIGHT);
        int l;
        double wl;
        if (le <= lamg[0]) { l = 0; wl = 0.0; }
        else if (le >= lamg[nl - 1]) { l = nl - 2; wl = 1.0; }
        else {
            int lo = 0, hi = nl - 1;
            while (hi - lo > 1) {
                int mid = (lo + hi) / 2;
                if (lamg[mid] <= le) lo = mid; else hi = mid;
            }
            l = lo;
            wl = (le - lamg[l]) / (lamg[l + 1] - lamg[l]);
        }
        int a, b;
        double wT, wp;
        interp_idx(Tg, nT, T[idx], &a, &wT);
        interp_idx(pg, np, p[idx], &b, &wp);
        double ls[2];
        for (int e = 0; e < 2; ++e) {
            const float *s = sig + (int64_t)(l + e) * nT * np;
            double l00 = log((double)s[a * np + b]), l10 = log((double)s[(a + 1) * np + b]);
            double l01 = log((double)s[a * np + b + 1]), l11 = log((double)s[(a + 1) * np + b + 1]);
            ls[e] = (1 - wT) * (1 - wp) * l00 + wT * (1 - wp) * l10 + (1 - wT) * wp * l01 + wT * wp * l11;
        }
        alpha[idx] = rho[idx] * exp((1.0 - wl) * ls[0] + wl * ls[1]);
    }
}

/* ------------------------------------------------------------------ packets */
/* one peel-off contribution attributed to the cell it leaves from (contribution functions) */
typedef struct {
    int64_t idx;
    int32_t kind, obs;
    double f;
} cf_rec;

typedef struct {
    double tally[ORC_MAX_OBS], tally_c[ORC_MAX_OBS];
    double ledger[8], ledger_c[8];
    int64_t steps;
    cf_rec *cf;            /* this chunk's contributions in packet order (when requested) */
    int64_t n_cf, cap_cf;
    int cf_oom;
} acc_t;

static void cf_put(acc_t *acc, int64_t idx, int kind, int obs, double f)
{
    if (acc->n_cf == acc->cap_cf) {
        int64_t cap = acc->cap_cf ? 2 * acc->cap_cf : 1024;
        cf_rec *q = (cf_rec *)realloc(acc->cf, (size_t)cap * sizeof(cf_rec));
        if (!q) {
            acc->cf_oom = 1;
            return;
        }
        acc->cf = q;
        acc->cap_cf = cap;
    }
    cf_rec r = {idx, kind, obs, f};
    acc->cf[acc->n_cf++] = r;
}

static inline void kahan(double *s, double *c, double v)
{
    double y = v - *c;
    double t = *s + y;
    *c = (t - *s) - y;
    *s = t;
}

typedef struct {
    const orc_grid *G;
    const orc_cells *C;
    const orc_source *S;
    const orc_run_args *A;
    const double *a_sca, *a_abs;   /* continuous absorption: omega alpha and (1 - omega) alpha per cell */
} job_t;

static void perp_basis(const double s[3], double e1[3], double e2[3])
{
    double a[3] = {0.0, 0.0, 1.0};
    if (fabs(s[2]) >= 0.9) { a[0] = 1.0; a[2] = 0.0; }
    /* e1 = normalize(s x a), e2 = s x e1 */
    e1[0] = s[1] * a[2] - s[2] * a[1];
    e1[1] = s[2] * a[0] - s[0] * a[2];
    e1[2] = s[0] * a[1] - s[1] * a[0];
    double n = sqrt(dot3(e1, e1));
    for (int i = 0; i < 3; ++i) e1[i] /= n;
    e2[0] = s[1] * e1[2] - s[2] * e1[1];
    e2[1] = s[2] * e1[0] - s[0] * e1[2];
    e2[2] = s[0] * e1[1] - s[1] * e1[0];
}

/* peel-off optical depth from x (cell c) towards o; returns exp(-tau) or 0 if occulted / cut */
static double peel(march_ctx *M, const double x0[3], const int c0[3], const double o[3], double cut,
                   double *tau_out, int *status, int entry)
{
    double x[3] = {x0[0], x0[1], x0[2]};
    int c[3] = {c0[0], c0[1], c0[2]};
    double tau = 0.0;
    int st = march(M, x, o, c, entry, -1.0, cut, &tau);
    *tau_out = tau;
    *status = st;
    if (st == END_ESCAPE) return exp(-tau);
    return 0.0;
}

/* a weight change of a biased flight (p/q), booked with the roulette's gain and loss so that the ledger
   closes packet by packet */
static void reweight(acc_t *acc, double *W, double factor)
{
    const double Wn = *W * factor;
    if (Wn > *W) kahan(&acc->ledger[4], &acc->ledger_c[4], Wn - *W);
    else kahan(&acc->ledger[5], &acc->ledger_c[5], *W - Wn);
    *W = Wn;
}

/* tally columns of a job: one per observer (albedo, emission); transmission: the chord (direct)
   column, plus the scattered-light column when packets scatter after their chord */
static int tally_cols(const orc_source *S, int mode)
{
    if (mode == 2) return S->trans_scatter ? 2 : 1;
    return S->n_obs;
}

/* One packet's life: launch (albedo disk, Sect. 5.2; emission cell draw, Sect. 4.3; transmission chord,
   Sect. 5.1), then flights of optical depth -ln(zeta) (with forcing or path biasing, Sect. 4.2), each
   ending in an interaction with its peel-offs f = W omega Theta e^-tau (Sect. 4.6), survival biasing or
   analog scattering and the roulette (Sect. 4.4, 4.5), a new direction (Sect. 3), or at the surface
   (Sect. 3), the top (escape) or the black bottom.  f of each tally column is added to the tallies. */
static void run_packet(const job_t *J, int64_t n, acc_t *acc, double *pk_f, int64_t *pk_steps, double *pk_tau,
                       int32_t *tr_cell, double *tr_len, int32_t *tr_n, int32_t tr_max, double *tr_pos)
{
    const orc_grid *G = J->G;
    const orc_cells *C = J->C;
    const orc_source *S = J->S;
    const orc_run_args *A = J->A;
    march_ctx M = {G, C->alpha, 0, S->max_steps, tr_cell, tr_len, 0, tr_max, NULL, 0.0, tr_pos};
    double Rtoa = G->r_edges[G->nr];
    double R0 = G->r_edges[0];
    double u[4];
    double f_obs[ORC_MAX_OBS];
    for (int o = 0; o < ORC_MAX_OBS; ++o) f_obs[o] = 0.0;
    double first_tau = -1.0;
    double x[3], d[3];
    int c[3], entry = -1;
    double W = 0.0, W0 = 0.0;
    int transport = 0;
    /* peel-off targets: every observer (albedo, emission), or in transmission the transit observer
       -star, whose scattered light goes to column 1 weighted by the launch b / R_TOA (Sect. 5.1) */
    const int trans = A->mode == 2;
    const double antistar[3] = {-S->star[0], -S->star[1], -S->star[2]};
    const int n_peel = trans ? 1 : S->n_obs;
    double peel_scale = 1.0;

    draw(A->seed, n, 0u, A->job_key, u);
    if (A->mode == 0 || A->mode == 2) {
        double e1[3], e2[3];
        perp_basis(S->star, e1, e2);
        double b = (A->mode == 0) ? Rtoa * sqrt(u[0]) : R0 + u[0] * (Rtoa - R0);
        double psi = 2.0 * ORC_PI * u[1];
        double h = sqrt(fmax(0.0, Rtoa * Rtoa - b * b));
        for (int i = 0; i < 3; ++i) {
            x[i] = b * (cos(psi) * e1[i] + sin(psi) * e2[i]) + h * S->star[i];
            d[i] = -S->star[i];
        }
        c[2] = G->nr - 1;
        locate_angles(G, x, c);
        entry = F_ROUT;
        W = W0 = 1.0;
        if (trans && S->ld_law) {
            /* limb darkening (Sect. 5.1): the chord's sky-plane position on the stellar disk gives the
               stellar zenith-angle cosine mu, and the packet carries I(mu) / I(disk centre); a chord
               that misses the stellar disk carries nothing and is not traced */
            const double X = S->transit_xy[0] + b * cos(psi), Y = S->transit_xy[1] + b * sin(psi);
            const double q = (X * X + Y * Y) / (S->star_radius * S->star_radius);
            W = W0 = q < 1.0 ? orc_limb(S->ld_law, S->ld_coef, sqrt(1.0 - q)) : 0.0;
        }
        kahan(&acc->ledger[0], &acc->ledger_c[0], W0);
        if (A->mode == 0) {
            transport = 1;
        } else if (W > 0.0) {
            const double x_l[3] = {x[0], x[1], x[2]};
            const int c_l[3] = {c[0], c[1], c[2]};
            trace_put(&M, -3, 0.0, x);
            double tau = 0.0;
            int st = march(&M, x, d, c, entry, -1.0, S->tau_peel_cut, &tau);
            double contrib;
            if (st == END_ESCAPE) contrib = (1.0 - exp(-tau)) * b / Rtoa;
            else if (st == END_CUTOFF || st == END_BOTTOM) contrib = b / Rtoa;
            else contrib = 0.0;
            first_tau = tau;
            f_obs[0] += W * contrib;
            if (st == END_CAP || st == END_LOST) {
                kahan(&acc->ledger[st == END_CAP ? 6 : 7], &acc->ledger_c[st == END_CAP ? 6 : 7], W);
            } else if (S->trans_scatter) {
                /* multiple scattering (Sect. 5.1): the packet itself starts at the launch point */
                x[0] = x_l[0]; x[1] = x_l[1]; x[2] = x_l[2];
                c[0] = c_l[0]; c[1] = c_l[1]; c[2] = c_l[2];
                peel_scale = b / Rtoa;
                transport = 1;
            } else {
                kahan(&acc->ledger[1], &acc->ledger_c[1], W);
            }
        }
    } else {
        /* emission launch: stratified draw over the hybrid pdf */
        /* stratified draw: packet n takes the point (n + z) / N of the cumulative pdf, i.e.
           (n + z) * (cdf_total / N) on the un-normalised cumulative sum */
        int64_t ncell = (int64_t)G->nlon * G->nlat * G->nr;
        const double *cdf = C->cdf, *wcell = C->wcell;
        double Wg = 1.0;
        double target = ((double)n + u[0]) * (C->cdf_total / (double)A->n_packets);
        if (C->ng > 0) {
            /* per-packet g-ordinate (Sect. 4.7): g with probability q(g) from the fourth word of
               event 1, then the cell from that g's pdf with the launch uniform (no stratification:
               the packets of one g are a random subset) */
            double v[4];
            draw(A->seed, n, 1u, A->job_key, v);
            int g = 0;
            while (g < C->ng - 1 && !(C->g_qcdf[g] > v[3])) ++g;
            cdf = C->cdf + (int64_t)g * ncell;
            wcell = C->wcell + (int64_t)g * ncell;
            M.alpha = C->alpha + (int64_t)g * ncell;
            Wg = C->g_w[g];
            target = u[0] * C->g_cdftot[g];
        }
        int64_t lo = 0, hi = ncell - 1;
        while (lo < hi) {
            int64_t mid = (lo + hi) / 2;
            if (cdf[mid] > target) hi = mid; else lo = mid + 1;
        }
        int64_t idx = lo;
        c[0] = (int)(idx % G->nlon);
        c[1] = (int)((idx / G->nlon) % G->nlat);
        c[2] = (int)(idx / ((int64_t)G->nlon * G->nlat));
        double r1 = G->r_edges[c[2]], r2 = G->r_edges[c[2] + 1];
        double r = cbrt(r1 * r1 * r1 + u[1] * (r2 * r2 * r2 - r1 * r1 * r1));
        double s1 = sin(G->lat_edges[c[1]]), s2 = sin(G->lat_edges[c[1] + 1]);
        double sl = s1 + u[2] * (s2 - s1);
        double cl = sqrt(fmax(0.0, 1.0 - sl * sl));
        double ph = G->lon_edges[c[0]] + u[3] * (G->lon_edges[c[0] + 1] - G->lon_edges[c[0]]);
        x[0] = r * cl * cos(ph);
        x[1] = r * cl * sin(ph);
        x[2] = r * sl;
        W = W0 = Wg * wcell[idx];
        kahan(&acc->ledger[0], &acc->ledger_c[0], W0);
        int capped = 0;
        for (int o = 0; o < S->n_obs; ++o) {
            double tau;
            int st;
            trace_put(&M, -2, 0.0, x);
            double e = peel(&M, x, c, S->obs[o], S->tau_peel_cut, &tau, &st, -1);
            if (first_tau < 0) first_tau = tau;
            if (st == END_CAP) {
                capped = 1;
                break;
            }
            f_obs[o] += W * e / (4.0 * ORC_PI);
            if (A->cf) cf_put(acc, idx, 0, o, W * e / (4.0 * ORC_PI));
        }
        if (S->scatter_emission && M.steps < M.max_steps) {
            double v[4];
            draw(A->seed, n, 1u, A->job_key, v);
            double mu = 2.0 * v[0] - 1.0, psi = 2.0 * ORC_PI * v[1];
            double s = sqrt(fmax(0.0, 1.0 - mu * mu));
            d[0] = s * cos(psi);
            d[1] = s * sin(psi);
            d[2] = mu;
            entry = -1;
            transport = 1;
        } else if (capped || (S->scatter_emission && M.steps >= M.max_steps)) {
            /* stopped by the step cap: a peel-off it cut, or (followed packets) no step left to go on */
            kahan(&acc->ledger[6], &acc->ledger_c[6], W);
        }
    }

    uint32_t ev = 2;
    int first = 1;
    /* continuous absorption (Sect. 4.1): flights sample their optical depth in the scattering opacity
       omega alpha, the weight decays by e^-tau_abs along the path, and every interaction scatters */
    const int ca = S->cont_abs && J->a_sca != NULL;
    while (transport) {
        draw(A->seed, n, ev, A->job_key, u);
        double tau_t = -log(u[0]);
        if ((first && S->forced_first == 1) || S->forced_first == 2) {
            /* forced scattering (Sect. 4.2), on the first flight or on every flight: the optical depth tau_m
               of the flight's path to the grid boundary (in the flight's own opacity); the packet interacts
               before it, carrying
               W (1 - e^-tau_m) with the truncated-exponential tau = -ln(1 - zeta (1 - e^-tau_m)), and
               W e^-tau_m leaves unscattered.  Not forced when the path runs past the cut-off depth or
               ends on a reflecting surface. */
            double tau_m = 0.0;
            int sm = END_ESCAPE;
            trace_put(&M, -4, 0.0, x);
            if (ca) { M.alpha = J->a_sca; M.alpha2 = J->a_abs; M.tau2 = 0.0; }
            (void)peel(&M, x, c, d, S->tau_peel_cut, &tau_m, &sm, entry);
            const double tau2_m = M.tau2;
            if (ca) { M.alpha = C->alpha; M.alpha2 = NULL; }
            if (sm == END_CAP) { kahan(&acc->ledger[6], &acc->ledger_c[6], W); break; }
            if (S->path_bias == 1) {
                /* path length stretching (Sect. 4.2): tau from the composite of the natural exponential and
                   one stretched to the path, q = (e^-tau + a e^-a tau) / 2 with a = 1 / (1 + tau_m); the
                   component is chosen by the third word of the event | 2^31 draw; weight e^-tau / q.  Not
                   applied past the cut-off depth. */
                if (sm != END_CUTOFF) {
                    double v[4];
                    draw(A->seed, n, ev | 0x80000000u, A->job_key, v);
                    const double a = 1.0 / (1.0 + tau_m);
                    tau_t = v[2] < 0.5 ? -log(u[0]) : -log(u[0]) / a;
                    const double q = 0.5 * (exp(-tau_t) + a * exp(-a * tau_t));
                    reweight(acc, &W, exp(-tau_t) / q);
                }
            } else if (sm == END_ESCAPE || (sm == END_BOTTOM && !(S->surface_albedo > 0.0))) {
                const double p = -expm1(-tau_m);
                const double rem = W * exp(-tau_m);
                const int q = sm == END_ESCAPE ? 1 : 3;
                if (ca) {
                    const double kept = rem * exp(-tau2_m);
                    kahan(&acc->ledger[q], &acc->ledger_c[q], kept);
                    kahan(&acc->ledger[2], &acc->ledger_c[2], rem - kept);
                } else {
                    kahan(&acc->ledger[q], &acc->ledger_c[q], rem);
                }
                W *= p;
                tau_t = -log1p(-u[0] * p);
                if (S->path_bias == 2) {
                    /* hybrid (Sect. 4.2): within the path, the composite of the truncated exponential
                       e^-tau / p and the uniform 1 / tau_m; weight (e^-tau / p) / q */
                    double v[4];
                    draw(A->seed, n, ev | 0x80000000u, A->job_key, v);
                    if (!(v[2] < 0.5)) tau_t = u[0] * tau_m;
                    const double ft = exp(-tau_t) / p;
                    reweight(acc, &W, ft / (0.5 * ft + 0.5 / tau_m));
                }
            }
        }
        first = 0;
        double tau = 0.0;
        trace_put(&M, -1, 0.0, x);
        if (ca) { M.alpha = J->a_sca; M.alpha2 = J->a_abs; M.tau2 = 0.0; }
        int st = march(&M, x, d, c, entry, tau_t, INFINITY, &tau);
        if (ca) {
            M.alpha = C->alpha;
            M.alpha2 = NULL;
            const double Wn = W * exp(-M.tau2);
            kahan(&acc->ledger[2], &acc->ledger_c[2], W - Wn);
            W = Wn;
        }
        if (st == END_ESCAPE) { kahan(&acc->ledger[1], &acc->ledger_c[1], W); break; }
        if (st == END_BOTTOM && S->surface_albedo > 0.0) {
            /* Lambertian reflection at the lower boundary (Sect. 3): peel-offs with the Lambert phase
               function mu_o / pi per steradian, then weight A_s (survival) or reflection with
               probability A_s (analog), cosine sqrt(zeta) about the outward normal */
            const double As = S->surface_albedo;
            const double rr = sqrt(dot3(x, x));
            const double nrm[3] = {x[0] / rr, x[1] / rr, x[2] / rr};
            const int64_t sidx = flat(G, c);
            int capped = 0;
            for (int o = 0; o < n_peel; ++o) {
                /* the point lies on the lower boundary: its root there is dropped; directions into
                   the planet contribute nothing and are not traced */
                const double *od = trans ? antistar : S->obs[o];
                const double mo = dot3(nrm, od);
                if (!(mo > 0.0)) continue;
                double tau_o = 0.0;
                int so = END_ESCAPE;
                trace_put(&M, -2, 0.0, x);
                const double e = peel(&M, x, c, od, S->tau_peel_cut, &tau_o, &so, F_RIN);
                if (so == END_CAP) { capped = 1; break; }
                const double fo = W * As * (mo / ORC_PI) * e;
                f_obs[trans ? 1 : o] += fo * peel_scale;
                if (A->cf) cf_put(acc, sidx, 1, o, fo);
            }
            if (capped) { kahan(&acc->ledger[6], &acc->ledger_c[6], W); break; }
            if (S->survival) {
                kahan(&acc->ledger[3], &acc->ledger_c[3], W * (1.0 - As));
                W *= As;
                if (W < S->w_rr * W0) {
                    double v[4];
                    draw(A->seed, n, ev | 0x80000000u, A->job_key, v);
                    if (v[1] < S->p_surv) {
                        double Wn = W / S->p_surv;
                        kahan(&acc->ledger[4], &acc->ledger_c[4], Wn - W);
                        W = Wn;
                    } else {
                        kahan(&acc->ledger[5], &acc->ledger_c[5], W);
                        break;
                    }
                }
            } else {
                double v[4];
                draw(A->seed, n, ev | 0x80000000u, A->job_key, v);
                if (!(v[0] < As)) { kahan(&acc->ledger[3], &acc->ledger_c[3], W); break; }
                if (W < S->w_rr * W0) {
                    /* forcing and continuous absorption change weights in analog mode too */
                    if (v[1] < S->p_surv) {
                        double Wn = W / S->p_surv;
                        kahan(&acc->ledger[4], &acc->ledger_c[4], Wn - W);
                        W = Wn;
                    } else {
                        kahan(&acc->ledger[5], &acc->ledger_c[5], W);
                        break;
                    }
                }
            }
            double nd[3];
            orc_turn(nrm, sqrt(u[2]), 2.0 * ORC_PI * u[3], nd);
            d[0] = nd[0]; d[1] = nd[1]; d[2] = nd[2];
            entry = F_RIN;
            ++ev;
            continue;
        }
        if (st == END_BOTTOM) { kahan(&acc->ledger[3], &acc->ledger_c[3], W); break; }
        if (st != END_INTERACT) { kahan(&acc->ledger[st == END_CAP ? 6 : 7], &acc->ledger_c[st == END_CAP ? 6 : 7], W); break; }
        int64_t idx = flat(G, c);
        double om = ca ? 1.0 : (C->omega ? C->omega[idx] : 0.0);
        double gg = C->g ? C->g[idx] : 0.0;
        double pg = C->pgas ? C->pgas[idx] : 1.0;
        int capped = 0;
        for (int o = 0; o < n_peel; ++o) {
            const double *od = trans ? antistar : S->obs[o];
            double tau_o;
            int so;
            trace_put(&M, -2, 0.0, x);
            double e = peel(&M, x, c, od, S->tau_peel_cut, &tau_o, &so, -1);
            if (so == END_CAP) { capped = 1; break; }
            const double fo = W * om * orc_theta_kind(dot3(d, od), pg, gg, S->cloud_phase) * e;
            f_obs[trans ? 1 : o] += fo * peel_scale;
            if (A->cf) cf_put(acc, idx, 1, o, fo);
        }
        if (capped) { kahan(&acc->ledger[6], &acc->ledger_c[6], W); break; }
        if (W * om == 0.0) { kahan(&acc->ledger[2], &acc->ledger_c[2], W); break; }
        if (S->survival) {
            kahan(&acc->ledger[2], &acc->ledger_c[2], W * (1.0 - om));
            W *= om;
            if (W < S->w_rr * W0) {
                double v[4];
                draw(A->seed, n, ev | 0x80000000u, A->job_key, v);
                if (v[1] < S->p_surv) {
                    double Wn = W / S->p_surv;
                    kahan(&acc->ledger[4], &acc->ledger_c[4], Wn - W);
                    W = Wn;
                } else {
                    kahan(&acc->ledger[5], &acc->ledger_c[5], W);
                    break;
                }
            }
        } else {
            double v[4];
            draw(A->seed, n, ev | 0x80000000u, A->job_key, v);
            if (!(v[0] < om)) { kahan(&acc->ledger[2], &acc->ledger_c[2], W); break; }
            if (W < S->w_rr * W0) {
                /* forcing and continuous absorption change weights in analog mode too */
                if (v[1] < S->p_surv) {
                    double Wn = W / S->p_surv;
                    kahan(&acc->ledger[4], &acc->ledger_c[4], Wn - W);
                    W = Wn;
                } else {
                    kahan(&acc->ledger[5], &acc->ledger_c[5], W);
                    break;
                }
            }
        }
        /* scatterer: gas if u1 < P_gas, else cloud; the cloud's own choice (two-term HG) uses u1's
           remaining uniform (u1 - P_gas) / (1 - P_gas) */
        double mu = (u[1] < pg) ? orc_sample_rayleigh(u[2])
                                : orc_sample_cloud(gg, (u[1] - pg) / (1.0 - pg), u[2], S->hg_iso_eps, S->cloud_phase);
        double nd[3];
        orc_turn(d, mu, 2.0 * ORC_PI * u[3], nd);
        d[0] = nd[0]; d[1] = nd[1]; d[2] = nd[2];
        entry = -1;
        ++ev;
    }

    for (int o = 0; o < tally_cols(S, A->mode); ++o) {
        kahan(&acc->tally[o], &acc->tally_c[o], f_obs[o]);
        if (pk_f) pk_f[o] = f_obs[o];
    }
    acc->steps += M.steps;
    if (pk_steps) *pk_steps = M.steps;
    if (pk_tau) *pk_tau = first_tau;
    if (tr_n) *tr_n = M.tr_n;
}

#define CHUNK 1024

typedef struct {
    const job_t *J;
    acc_t *chunks;
    int64_t nchunks;
    int64_t next;
    pthread_mutex_t mu;
} pool_t;

static void run_chunk(const job_t *J, int64_t ch, acc_t *acc)
{
    const orc_run_args *A = J->A;
    int64_t b = ch * CHUNK, e = b + CHUNK;
    if (e > A->n_run) e = A->n_run;
    for (int64_t q = b; q < e; ++q) {
        int64_t n = A->packet0 + q;
        int32_t *tc = NULL;
        double *tl = NULL;
        int32_t *tn = NULL;
        double *tp = NULL;
        if (A->tr_cell && q < A->n_trace) {
            tc = A->tr_cell + q * A->max_trace;
            tl = A->tr_len + q * A->max_trace;
            tn = A->tr_n + q;
            if (A->tr_pos) tp = A->tr_pos + 3 * q * A->max_trace;
        }
        run_packet(J, n, acc, A->pk_f ? A->pk_f + q * tally_cols(J->S, A->mode) : NULL, A->pk_steps ? A->pk_steps + q : NULL,
                   A->pk_tau ? A->pk_tau + q : NULL, tc, tl, tn, A->max_trace, tp);
    }
}

static void *worker(void *arg)
{
    pool_t *P = (pool_t *)arg;
    for (;;) {
        pthread_mutex_lock(&P->mu);
        int64_t ch = P->next++;
        pthread_mutex_unlock(&P->mu);
        if (ch >= P->nchunks) break;
        run_chunk(P->J, ch, &P->chunks[ch]);
    }
    return NULL;
}

/* Run packets [packet0, packet0 + n_run) of one job; deterministic for any thread count
   (per-chunk Kahan sums combined in chunk order). Returns 0 on success. */
int orc_run(const orc_grid *G, const orc_cells *C, const orc_source *S, orc_run_args *A)
{
    if (S->n_obs < 1 || S->n_obs > ORC_MAX_OBS) return -1;
    job_t J = {G, C, S, A, NULL, NULL};
    double *a_sca = NULL, *a_abs = NULL;
    if (S->cont_abs && C->omega) {
        const int64_t ncell = (int64_t)G->nlon * G->nlat * G->nr;
        a_sca = (double *)malloc(sizeof(double) * (size_t)ncell);
        a_abs = (double *)malloc(sizeof(double) * (size_t)ncell);
        if (!a_sca || !a_abs) { free(a_sca); free(a_abs); return -2; }
        for (int64_t i = 0; i < ncell; ++i) {
            a_sca[i] = C->alpha[i] * C->omega[i];
            a_abs[i] = C->alpha[i] - a_sca[i];
        }
        J.a_sca = a_sca;
        J.a_abs = a_abs;
    }
    int64_t nch = (A->n_run + CHUNK - 1) / CHUNK;
    acc_t *chunks = (acc_t *)calloc((size_t)(nch > 0 ? nch : 1), sizeof(acc_t));
    if (!chunks) return -2;
    pool_t P;
    P.J = &J;
    P.chunks = chunks;
    P.nchunks = nch;
    P.next = 0;
    pthread_mutex_init(&P.mu, NULL);
    int nt = A->nthreads > 0 ? A->nthreads : 1;
    if (nt == 1) {
        worker(&P);
    } else {
        pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)nt);
        for (int t = 0; t < nt; ++t) pthread_create(&th[t], NULL, worker, &P);
        for (int t = 0; t < nt; ++t) pthread_join(th[t], NULL);
        free(th);
    }
    pthread_mutex_destroy(&P.mu);
    double ts[ORC_MAX_OBS] = {0}, tc[ORC_MAX_OBS] = {0}, ls[8] = {0}, lc[8] = {0};
    int64_t steps = 0;
    int cf_oom = 0;
    for (int64_t ch = 0; ch < nch; ++ch) {
        for (int o = 0; o < tally_cols(S, A->mode); ++o) kahan(&ts[o], &tc[o], chunks[ch].tally[o]);
        for (int q = 0; q < 8; ++q) kahan(&ls[q], &lc[q], chunks[ch].ledger[q]);
        steps += chunks[ch].steps;
        /* contributions in packet order: the sums do not depend on the thread count */
        const int64_t ncell = (int64_t)G->nlon * G->nlat * G->nr;
        for (int64_t q = 0; q < chunks[ch].n_cf; ++q) {
            const cf_rec *r = &chunks[ch].cf[q];
            A->cf[((int64_t)r->kind * S->n_obs + r->obs) * ncell + r->idx] += r->f;
        }
        cf_oom |= chunks[ch].cf_oom;
        free(chunks[ch].cf);
    }
    for (int o = 0; o < tally_cols(S, A->mode); ++o) A->tally[o] = ts[o];
    if (A->ledger) for (int q = 0; q < 8; ++q) A->ledger[q] = ls[q];
    if (A->steps) A->steps[0] = steps;
    free(chunks);
    free(a_sca);
    free(a_abs);
    return cf_oom ? -3 : 0;
}

int orc_max_obs(void) { return ORC_MAX_OBS; }
