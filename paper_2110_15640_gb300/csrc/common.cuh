// common.cuh -- device-side data layout and small primitives of libgcmc.
//
// Layout in HBM (one context):
//   DevGrid   per uploaded grid: edge tables in FP64 and FP32 (r, r^2 as an FP32 hi+lo pair,
//             sin(lat), sin^2(lat), cos/sin(lon)), per-cell T, p, rho, wind (FP32) and volume (FP64).
//   DevJob    per job of a launch: mode, Philox key, packet count, pointers to the job's cell table
//             (albedo: 16-byte {alpha, omega, g, P_gas} records in FP32, 32 bytes in FP64; absorber
//             marches: 4/8-byte alpha), emission CDF and launch weights (FP64), source geometry and
//             the job's 64-bit fixed-point accumulators.
// Per-cell arrays are flattened [k][j][i] (longitude fastest), so a warp of packets launched from
// neighbouring cells of one latitude row gathers neighbouring records.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/gcmc.h"

namespace gcmc {

constexpr int MAX_OBS = GCMC_MAX_OBS;
constexpr double PI = 3.14159265358979323846;
constexpr double C_LIGHT = 2.99792458e8;
constexpr double H_PLANCK = 6.62607015e-34;
constexpr double K_BOLTZ = 1.380649e-23;
// tally accumulator slots per job: [0, MAX_OBS) f sums, then 8 ledger sums, steps, packets, flags
constexpr int ACC_LEDGER = MAX_OBS;
constexpr int ACC_STEPS = MAX_OBS + 8;
constexpr int ACC_PACKETS = MAX_OBS + 9;
constexpr int ACC_FLAGS = MAX_OBS + 10;
constexpr int ACC_SLOTS = 32;            // padded (256 bytes per job)
constexpr double FIX_SCALE = 4294967296.0;   // 2^32: fixed-point resolution of tallies and ledger

// ray kinds: a flight to an interaction, a peel-off, a limb chord, and the march that measures a forced
// first flight's optical depth to the grid boundary
enum { K_FLIGHT = 0, K_PEEL = 1, K_CHORD = 2, K_FORCE = 3 };
enum { E_CONT = -1, E_INTERACT = 0, E_ESCAPE = 1, E_BOTTOM = 2, E_CUTOFF = 3, E_CAP = 4, E_LOST = 5 };
enum { FLAG_OVERFLOW = GCMC_FLAG_TALLY_RANGE, FLAG_LOST = 2, FLAG_BAD = 4 };   // reported in gcmc_stats.flags
constexpr int GINFO_STRIDE = 32;    // doubles between the info blocks of a band job's g-ordinates
constexpr int GTAB_ROW = 4;         // doubles per g row of a band job's sampling table

struct DevGrid {
    int32_t nlon, nlat, nr, pad;
    int64_t ncell;
    double R0, Rtoa, lon0;
    const double *r, *r2, *lat, *slat, *s2lat, *lon, *clon, *slon;     // FP64 edge tables
    const float *r_f, *r2hi_f, *r2lo_f, *lat_f, *slat_f, *s2lat_f, *lon_f, *clon_f, *slon_f;
    const float *shA_f;                                                 // [nr] (r_{k+1}/r_k)^3 - 1
    // low parts of the FP32 edges (edge = hi + lo to ~48 bits) and FP32 cell widths, so that
    // positions sampled inside a cell carry no edge rounding that repeats for every packet
    const float *r_lo_f, *slat_lo_f, *lon_lo_f, *dslat_f, *dlon_f;
    // per latitude band j in one hemisphere, 1 - |sin| at its lower edge as FP32 hi + lo: cos(lat) =
    // sqrt(c (2 - c)) from c = 1 - |sin(lat)| keeps full relative precision towards the poles, where
    // sqrt(1 - sin^2) from an FP32 sin(lat) loses it (0 for the band across the equator)
    const float *cb_f, *cb_lo_f;
    // the march's edge tables as pairs (one 8/16-byte load each), staged in shared memory by the kernels:
    // r2p = (r^2 hi, r^2 lo) [nr+1], slp = (sin lat, sin^2 lat) [nlat+1], csp = (cos lon, sin lon) [nlon+1]
    const float2 *r2p_f, *slp_f, *csp_f;
    const double2 *r2p, *slp, *csp;
    uint64_t mag_lon, mag_ll;   // ceil(2^40 / nlon), ceil(2^40 / (nlon nlat)): exact division of cell indices
    const float *T, *p, *rho, *wind;                                    // per cell
    const double *vol;                                                  // per cell
};

struct __align__(16) Rec64 {
    double a, w, g, pg;
};

struct DevJob {
    int32_t mode, n_obs, grid_slot, survival;
    int32_t precision, cloud_phase;   // cloud_phase: GCMC_CLOUD_HG or GCMC_CLOUD_TTHG
    uint32_t key, pad1;
    uint64_t seed;
    int64_t n_packets;
    int64_t chunk_begin;        // first work item of this job (batched launches)
    int64_t max_steps;
    const void *rec;            // albedo records, or alpha for absorber marches
    const long long *cdf;       // emission: cumulative hybrid pdf, 2^62 fixed point
    const void *wcell;          // emission: launch weights (march precision)
    const double *info;         // emission: [L_tot, n_incl, cdf_total, ...] written by the cell-table kernels
    long long cdf_step_fix;     // emission: floor(Q_tot / N), the stratum width in fixed point
    double star[3], e1[3], e2[3];
    double obs[MAX_OBS][3];
    double w_rr, p_surv, tau_cut, hg_eps;
    // the same vectors and constants rounded once to FP32, for FP32 marches
    float star_f[3], e1_f[3], e2_f[3];
    float obs_f[MAX_OBS][3];
    float w_rr_f, p_surv_f, hg_eps_f, pad2;
    unsigned long long *acc;    // [ACC_SLOTS]
    // contribution functions (Sect. 6), or NULL: [2][n_obs][cf_ncell] fixed-point sums of the peel-off
    // contributions by the cell they leave from, [0] thermal (emission launch), [1] scattered
    unsigned long long *cf;
    int64_t cf_ncell;
    // options read outside the march (kept after the fields every packet launch reads)
    int32_t n_tal;              // tally columns: n_obs; transmission: 1, or 2 with multiple scattering
    int32_t rec4;               // cell records are (alpha, omega, g, P_gas) (scattering opacities), else alpha
    int32_t trans_scatter;      // transmission: packets scatter after their chord (column 1)
    int32_t ld_law;             // stellar limb-darkening law (GCMC_LD_*)
    int32_t ng_s, g_bias;       // band job: g-ordinates drawn per packet (0: one g-ordinate); q(g) option
    double g_beta;              // composite fraction of q(g)
    const double *gw;           // [ng] g-ordinate weights (band jobs)
    double *gtab;               // band job: [ng] rows {cumulative q, W_g, w_g L_g, Q_tot(g) as int64 bits}
    const double *ginfo;        // band job: each g-ordinate's info block, GINFO_STRIDE doubles apart
    double surf_as, ld_c[4], star_r, tr_x, tr_y;   // surface albedo; limb darkening, stellar radius, planet offset
    float surf_as_f, ld_c_f[4], star_r_f, tr_x_f, tr_y_f;
    const void *arec;           // scattering records: their alpha as a compact table for the cell march
    int32_t forced_first;       // biased flights: 1 the first, 2 every flight (albedo; transmission scattering)
    int32_t cont_abs;           // continuous absorption (scattering records only)
    int32_t path_bias, pad5;    // biased flights sample tau forced (0), stretched (1) or hybrid (2)
};

// job constants in the march precision (FP32 marches read the copies rounded on the host)
template <typename real> struct JV;
template <> struct JV<double> {
    static __device__ __forceinline__ double star(const DevJob &J, int q) { return J.star[q]; }
    static __device__ __forceinline__ double e1(const DevJob &J, int q) { return J.e1[q]; }
    static __device__ __forceinline__ double e2(const DevJob &J, int q) { return J.e2[q]; }
    static __device__ __forceinline__ double obs(const DevJob &J, int o, int q) { return J.obs[o][q]; }
    static __device__ __forceinline__ double w_rr(const DevJob &J) { return J.w_rr; }
    static __device__ __forceinline__ double p_surv(const DevJob &J) { return J.p_surv; }
    static __device__ __forceinline__ double hg_eps(const DevJob &J) { return J.hg_eps; }
    static __device__ __forceinline__ double surf_as(const DevJob &J) { return J.surf_as; }
    static __device__ __forceinline__ double ld_c(const DevJob &J, int q) { return J.ld_c[q]; }
    static __device__ __forceinline__ double star_r(const DevJob &J) { return J.star_r; }
    static __device__ __forceinline__ double tr_x(const DevJob &J) { return J.tr_x; }
    static __device__ __forceinline__ double tr_y(const DevJob &J) { return J.tr_y; }
};
template <> struct JV<float> {
    static __device__ __forceinline__ float star(const DevJob &J, int q) { return J.star_f[q]; }
    static __device__ __forceinline__ float e1(const DevJob &J, int q) { return J.e1_f[q]; }
    static __device__ __forceinline__ float e2(const DevJob &J, int q) { return J.e2_f[q]; }
    static __device__ __forceinline__ float obs(const DevJob &J, int o, int q) { return J.obs_f[o][q]; }
    static __device__ __forceinline__ float w_rr(const DevJob &J) { return J.w_rr_f; }
    static __device__ __forceinline__ float p_surv(const DevJob &J) { return J.p_surv_f; }
    static __device__ __forceinline__ float hg_eps(const DevJob &J) { return J.hg_eps_f; }
    static __device__ __forceinline__ float surf_as(const DevJob &J) { return J.surf_as_f; }
    static __device__ __forceinline__ float ld_c(const DevJob &J, int q) { return J.ld_c_f[q]; }
    static __device__ __forceinline__ float star_r(const DevJob &J) { return J.star_r_f; }
    static __device__ __forceinline__ float tr_x(const DevJob &J) { return J.tr_x_f; }
    static __device__ __forceinline__ float tr_y(const DevJob &J) { return J.tr_y_f; }
};

// ------------------------------------------------------------------ Philox4x32-10 (Salmon et al. 2011)
__device__ __forceinline__ uint4 philox10(uint4 c, uint2 k)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) {
            k.x += 0x9E3779B9u;
            k.y += 0xBB67AE85u;
        }
        const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    }
    return c;
}

__device__ __forceinline__ uint4 draw_words(uint64_t seed, int64_t packet, uint32_t event, uint32_t key)
{
    return philox10(make_uint4((uint32_t)(uint64_t)packet, (uint32_t)((uint64_t)packet >> 32), event, key),
                    make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
}

// uniform in (0, 1): ((w >> 8) + 1/2) 2^-24, exact in FP64, correctly rounded in FP32
template <typename real> __device__ __forceinline__ real u01(uint32_t w);
template <> __device__ __forceinline__ double u01<double>(uint32_t w)
{
    return ((double)(w >> 8) + 0.5) * (1.0 / 16777216.0);
}
template <> __device__ __forceinline__ float u01<float>(uint32_t w)
{
    return __fmaf_rn((float)(w >> 8), 5.9604644775390625e-8f, 2.98023223876953125e-8f);
}

// ------------------------------------------------------------------ precision-dispatched helpers
template <typename real> struct M;
template <> struct M<float> {
    static __device__ __forceinline__ float sqrt_(float x) { return sqrtf(x); }
    static __device__ __forceinline__ float rsqrt_(float x) { return rsqrtf(x); }
    // accurate expf / logf (a few ulp), not the __expf / __logf intrinsics: these run once per ray end or
    // flight start, where the intrinsics' errors (an absolute 2^-21 in -ln(xi) for xi near 1, a relative
    // 2^-24 |x| in e^-x up to the cut-off depth 50) would exceed the rounding of the march itself
    static __device__ __forceinline__ float exp_(float x) { return expf(x); }
    static __device__ __forceinline__ float log_(float x) { return logf(x); }
    // 1 - e^-x with full relative precision for small x
    static __device__ __forceinline__ float one_minus_exp_neg(float x) { return -expm1f(-x); }
    static __device__ __forceinline__ float cbrt_(float x) { return cbrtf(x); }
    static __device__ __forceinline__ float div_(float a, float b) { return __fdividef(a, b); }
    static __device__ __forceinline__ void sincos_(float x, float *s, float *c) { sincosf(x, s, c); }
    static __device__ __forceinline__ float atan2_(float y, float x) { return atan2f(y, x); }
    static __device__ __forceinline__ float inf() { return __int_as_float(0x7f800000); }
};
template <> struct M<double> {
    static __device__ __forceinline__ double sqrt_(double x) { return sqrt(x); }
    static __device__ __forceinline__ double rsqrt_(double x) { return 1.0 / sqrt(x); }
    static __device__ __forceinline__ double exp_(double x) { return exp(x); }
    static __device__ __forceinline__ double log_(double x) { return log(x); }
    // the FP64 path follows the definition term by term, as the oracle does
    static __device__ __forceinline__ double one_minus_exp_neg(double x) { return 1.0 - exp(-x); }
    static __device__ __forceinline__ double cbrt_(double x) { return cbrt(x); }
    static __device__ __forceinline__ double div_(double a, double b) { return a / b; }
    static __device__ __forceinline__ void sincos_(double x, double *s, double *c) { sincos(x, s, c); }
    static __device__ __forceinline__ double atan2_(double y, double x) { return atan2(y, x); }
    static __device__ __forceinline__ double inf() { return __longlong_as_double(0x7ff0000000000000ll); }
};

template <typename real> __device__ __forceinline__ const real *tab_r(const DevGrid &g);
template <> __device__ __forceinline__ const float *tab_r<float>(const DevGrid &g) { return g.r_f; }
template <> __device__ __forceinline__ const double *tab_r<double>(const DevGrid &g) { return g.r; }
template <typename real> __device__ __forceinline__ const real *tab_slat(const DevGrid &g);
template <> __device__ __forceinline__ const float *tab_slat<float>(const DevGrid &g) { return g.slat_f; }
template <> __device__ __forceinline__ const double *tab_slat<double>(const DevGrid &g) { return g.slat; }
template <typename real> __device__ __forceinline__ const real *tab_s2lat(const DevGrid &g);
template <> __device__ __forceinline__ const float *tab_s2lat<float>(const DevGrid &g) { return g.s2lat_f; }
template <> __device__ __forceinline__ const double *tab_s2lat<double>(const DevGrid &g) { return g.s2lat; }
template <typename real> __device__ __forceinline__ const real *tab_lat(const DevGrid &g);
template <> __device__ __forceinline__ const float *tab_lat<float>(const DevGrid &g) { return g.lat_f; }
template <> __device__ __forceinline__ const double *tab_lat<double>(const DevGrid &g) { return g.lat; }
template <typename real> __device__ __forceinline__ const real *tab_lon(const DevGrid &g);
template <> __device__ __forceinline__ const float *tab_lon<float>(const DevGrid &g) { return g.lon_f; }
template <> __device__ __forceinline__ const double *tab_lon<double>(const DevGrid &g) { return g.lon; }
template <typename real> __device__ __forceinline__ const real *tab_clon(const DevGrid &g);
template <> __device__ __forceinline__ const float *tab_clon<float>(const DevGrid &g) { return g.clon_f; }
template <> __device__ __forceinline__ const double *tab_clon<double>(const DevGrid &g) { return g.clon; }
template <typename real> __device__ __forceinline__ const real *tab_slon(const DevGrid &g);
template <> __device__ __forceinline__ const float *tab_slon<float>(const DevGrid &g) { return g.slon_f; }
template <> __device__ __forceinline__ const double *tab_slon<double>(const DevGrid &g) { return g.slon; }

// r_k^2 as an unevaluated sum hi + lo (exact r^2 in FP64; FP32 pair carries ~48 bits)
template <typename real> __device__ __forceinline__ void r2_pair(const DevGrid &g, int k, real &hi, real &lo);
template <> __device__ __forceinline__ void r2_pair<float>(const DevGrid &g, int k, float &hi, float &lo)
{
    hi = __ldg(g.r2hi_f + k);
    lo = __ldg(g.r2lo_f + k);
}
template <> __device__ __forceinline__ void r2_pair<double>(const DevGrid &g, int k, double &hi, double &lo)
{
    hi = __ldg(g.r2 + k);
    lo = 0.0;
}

template <typename real> struct Pair;
template <> struct Pair<float> { using type = float2; };
template <> struct Pair<double> { using type = double2; };

template <typename real> __device__ __forceinline__ const typename Pair<real>::type *pair_r2(const DevGrid &g);
template <> __device__ __forceinline__ const float2 *pair_r2<float>(const DevGrid &g) { return g.r2p_f; }
template <> __device__ __forceinline__ const double2 *pair_r2<double>(const DevGrid &g) { return g.r2p; }
template <typename real> __device__ __forceinline__ const typename Pair<real>::type *pair_sl(const DevGrid &g);
template <> __device__ __forceinline__ const float2 *pair_sl<float>(const DevGrid &g) { return g.slp_f; }
template <> __device__ __forceinline__ const double2 *pair_sl<double>(const DevGrid &g) { return g.slp; }
template <typename real> __device__ __forceinline__ const typename Pair<real>::type *pair_cs(const DevGrid &g);
template <> __device__ __forceinline__ const float2 *pair_cs<float>(const DevGrid &g) { return g.csp_f; }
template <> __device__ __forceinline__ const double2 *pair_cs<double>(const DevGrid &g) { return g.csp; }

// the march's view of a grid: sizes and edge tables (in shared memory inside the kernels)
template <typename real> struct Tabs {
    const typename Pair<real>::type *r2, *sl, *cs;
    int nlon, nlat, nr;
};

// number of pair entries the march tables of a grid take
__host__ __device__ inline int tab_entries(int nlon, int nlat, int nr) { return (nr + 1) + (nlat + 1) + (nlon + 1); }

// copy a grid's march tables into `dst` (lanes lane0 .. lane0 + nthreads - 1 cooperate)
template <typename real>
__device__ __forceinline__ Tabs<real> stage_tabs(const DevGrid &G, typename Pair<real>::type *dst, int t, int nthreads)
{
    using P = typename Pair<real>::type;
    const int a = G.nr + 1, b = G.nlat + 1, c = G.nlon + 1;
    const P *r2 = pair_r2<real>(G), *sl = pair_sl<real>(G), *cs = pair_cs<real>(G);
    for (int q = t; q < a + b + c; q += nthreads)
        dst[q] = q < a ? r2[q] : q < a + b ? sl[q - a] : cs[q - a - b];
    Tabs<real> T;
    T.r2 = dst;
    T.sl = dst + a;
    T.cs = dst + a + b;
    T.nlon = G.nlon;
    T.nlat = G.nlat;
    T.nr = G.nr;
    return T;
}

// fixed-point conversion of a non-negative contribution
template <typename real> __device__ __forceinline__ long long to_fix(real v);
template <> __device__ __forceinline__ long long to_fix<float>(float v) { return __float2ll_rn(v * 4294967296.0f); }
template <> __device__ __forceinline__ long long to_fix<double>(double v) { return __double2ll_rn(v * FIX_SCALE); }

}  // namespace gcmc
