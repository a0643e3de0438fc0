// transport.cu -- photon-packet transport kernels (launch, tau sampling, cell march, interaction,
// peel-off, limb chord, tally) in two launch forms:
//   plain      one launch per job, one thread per packet (the straightforward GPU form)
//   persistent one launch for a whole batch of jobs: resident warps pull (job, packet range) work
//              items from a device counter; inside an item, lanes whose packets have finished are
//              refilled together once at least `refill_min` of them are idle (ballot/popc), so the
//              long launch code runs convergently instead of one lane at a time.
// Each lane runs a small state machine whose every iteration is ONE cell step of whatever ray the
// packet currently follows (flight with an optical-depth target, peel-off towards an observer, or
// a chord), so lanes stay convergent on the same march code while their packets are in different
// phases.  Kernels are instantiated without the scattering code (SCAT = false) for batches of
// absorber-only marches (emission peel-offs, limb chords), which halves the live packet state.
// Tallies and the energy ledger are 64-bit fixed point: per-thread slots in shared memory,
// warp-reduced and added atomically to the job's accumulators, so sums are order independent.
#include <climits>

#include "internal.h"
#include "march.cuh"

namespace gcmc {

template <typename real> struct Packet {
    Ray<real> ray;
    int kind, obs, stage, alive;
    real W, W0;
    real ix, iy, iz;       // interaction / emission point
    real fx, fy, fz;       // flight direction before scattering
    real om, gg, pg;       // cell record at the interaction
    real bimp;             // chord impact parameter / R_TOA
    int ci, cj, ck;
    int cell0;             // flat index of the cell the current peel-off leaves from
    int steps;
    int hint;              // launch cell of this lane's previous packet of the same work item (-1: none)
    int goff;              // band job: offset of the packet's g-ordinate table (g * ncell), else 0
    int ended, end_e, end_idx;   // the current ray has ended (persistent kernel: processed at the refill point)
    uint32_t ev;
    int64_t n;
};

// per-job constants kept in registers for a work item
template <typename real> struct JobC {
    int max_steps;
    int contabs;           // continuous absorption: flights march in omega alpha and accumulate (1 - omega) alpha
    real tau_cut;
    const real *rec;       // march table: alpha per cell
    const real *recf;      // scattering records (alpha, omega, g, P_gas) per cell, or NULL
};

struct LogOut {
    int64_t packet0;
    double *pk_f;
    int64_t *pk_steps;
    double *pk_tau;
    int32_t *tr_cell;
    double *tr_len;
    int32_t *tr_n;
    int32_t n_trace, max_trace;
};

constexpr int NSLOT = ACC_FLAGS + 1;

template <typename real, bool LOG> struct Sink {
    static constexpr bool is_log = LOG;
    unsigned long long *sm;   // this thread's first slot; slots are blockDim apart
    int stride;
    // this thread's copy of the last three words of its packet's current flight draw (the scatterer,
    // mu and azimuth words of the event whose first word sampled the flight's optical depth), blockDim
    // apart: the interaction at the end of the flight reads them instead of drawing the event again
    uint32_t *wc;
    LogOut lg;

    __device__ __forceinline__ void add(int slot, unsigned long long v) { sm[slot * stride] += v; }
    __device__ __forceinline__ void flag(unsigned long long v) { sm[ACC_FLAGS * stride] |= v; }
    __device__ __forceinline__ void tally(int o, real f, int64_t n, int n_obs)
    {
        if (!(f < (real)1.0e9) || !(f >= (real)0)) {
            flag(FLAG_OVERFLOW);
            return;
        }
        add(o, (unsigned long long)to_fix<real>(f));
        if constexpr (LOG) {
            if (lg.pk_f) lg.pk_f[(n - lg.packet0) * n_obs + o] += (double)f;
        }
    }
    __device__ __forceinline__ void ledger(int q, real w) { add(ACC_LEDGER + q, (unsigned long long)to_fix<real>(w)); }
    __device__ __forceinline__ void trace(int64_t n, int cell, real len)
    {
        if constexpr (LOG) {
            const int64_t q = n - lg.packet0;
            if (lg.tr_cell && q < lg.n_trace) {
                const int t = lg.tr_n[q];
                if (t < lg.max_trace) {
                    lg.tr_cell[q * lg.max_trace + t] = cell;
                    lg.tr_len[q * lg.max_trace + t] = (double)len;
                    lg.tr_n[q] = t + 1;
                }
            }
        }
    }
};

template <typename real>
__device__ __forceinline__ void start_ray(Packet<real> &P, real ox, real oy, real oz, real dx, real dy, real dz, int i,
                                          int j, int k, int kind, real tau_target)
{
    ray_setup<real>(P.ray, ox, oy, oz, dx, dy, dz);
    P.ray.i = i;
    P.ray.j = j;
    P.ray.k = k;
    P.ray.tau = (real)0;
    P.ray.tau2 = (real)0;
    P.ray.tau_target = tau_target;
    P.kind = kind;
}

template <typename real, class SinkT>
__device__ __forceinline__ void start_peel(Packet<real> &P, const DevJob &J, SinkT &S)
{
    S.trace(P.n, -2, (real)0);
    start_ray<real>(P, P.ix, P.iy, P.iz, JV<real>::obs(J, P.obs, 0), JV<real>::obs(J, P.obs, 1), JV<real>::obs(J, P.obs, 2), P.ci,
                    P.cj, P.ck, K_PEEL, (real)-1);
}

// how a flight samples its optical depth (Sect. 4.2): the natural exponential; forced, the exponential
// truncated at the boundary, -ln(1 - zeta p) with p = 1 - e^-tau_m (p may round to 1 on deep paths, where
// the truncated form still applies); path length stretching, the composite (e^-tau + a e^-a tau) / 2 with
// a = 1 / (1 + tau_m); hybrid, forced with the composite of the truncated exponential and the uniform on
// [0, tau_m].  The composites choose their component by the third word of the event | 2^31 draw and
// reweight the packet by p(tau) / q(tau), booked with the roulette's gain and loss.
enum { FL_NATURAL = 0, FL_FORCED = 1, FL_STRETCH = 2, FL_HYBRID = 3 };

template <typename real, class SinkT>
__device__ __noinline__ void reweight(Packet<real> &P, SinkT &S, real factor)
{
    const real Wn = P.W * factor;
    if (Wn > P.W) S.ledger(4, Wn - P.W);
    else S.ledger(5, P.W - Wn);
    P.W = Wn;
}

template <typename real, class SinkT>
__device__ __forceinline__ void start_flight(Packet<real> &P, const DevJob &J, SinkT &S, real dx, real dy, real dz,
                                             int mode = FL_NATURAL, real p = (real)1, real taum = (real)0)
{
    const uint4 w = draw_words(J.seed, P.n, P.ev, J.key);
    S.wc[0] = w.y;
    S.wc[S.stride] = w.z;
    S.wc[2 * S.stride] = w.w;
    real tau;
    if (mode == FL_NATURAL) {
        tau = -M<real>::log_(u01<real>(w.x));
    } else {
        const real u = u01<real>(w.x);
        if (mode == FL_STRETCH) {
            const uint4 v = draw_words(J.seed, P.n, P.ev | 0x80000000u, J.key);
            const real a = (real)1 / ((real)1 + taum);
            tau = -M<real>::log_(u);
            if (!(u01<real>(v.z) < (real)0.5)) tau = tau / a;
            const real q = (real)0.5 * (M<real>::exp_(-tau) + a * M<real>::exp_(-a * tau));
            reweight<real>(P, S, M<real>::exp_(-tau) / q);
        } else {
            if constexpr (sizeof(real) == 8) tau = -log1p(-u * p);
            else tau = -log1pf(-u * p);
            if (mode == FL_HYBRID) {
                const uint4 v = draw_words(J.seed, P.n, P.ev | 0x80000000u, J.key);
                if (!(u01<real>(v.z) < (real)0.5)) tau = u * taum;
                const real ft = M<real>::exp_(-tau) / p;
                reweight<real>(P, S, ft / ((real)0.5 * ft + (real)0.5 / taum));
            }
        }
    }
    S.trace(P.n, -1, (real)0);
    start_ray<real>(P, P.ix, P.iy, P.iz, dx, dy, dz, P.ci, P.cj, P.ck, K_FLIGHT, tau);
}

// a forced flight: the march to the grid boundary along (dx, dy, dz), kept in fx, fy, fz for the flight
template <typename real, class SinkT>
__device__ __forceinline__ void start_force(Packet<real> &P, SinkT &S, real dx, real dy, real dz)
{
    P.fx = dx;
    P.fy = dy;
    P.fz = dz;
    S.trace(P.n, -4, (real)0);
    start_ray<real>(P, P.ix, P.iy, P.iz, dx, dy, dz, P.ci, P.cj, P.ck, K_FORCE, (real)-1);
}

// the first flight from the launch point along -star: forced (forced_first 1 or 2) or plain
template <typename real, class SinkT>
__device__ __forceinline__ void start_first_flight(Packet<real> &P, const DevJob &J, SinkT &S)
{
    if (J.forced_first) start_force<real>(P, S, -JV<real>::star(J, 0), -JV<real>::star(J, 1), -JV<real>::star(J, 2));
    else start_flight<real>(P, J, S, -JV<real>::star(J, 0), -JV<real>::star(J, 1), -JV<real>::star(J, 2));
}

// a flight after a scattering or a surface reflection: forced when every flight is (forced_first 2)
template <typename real, bool EXT, class SinkT>
__device__ __forceinline__ void start_next_flight(Packet<real> &P, const DevJob &J, SinkT &S, real dx, real dy, real dz)
{
    if constexpr (EXT) {
        if (J.forced_first == 2) {
            start_force<real>(P, S, dx, dy, dz);
            return;
        }
    }
    start_flight<real>(P, J, S, dx, dy, dz);
}

template <typename real, class SinkT>
__device__ __forceinline__ void finish(Packet<real> &P, SinkT &S)
{
    S.add(ACC_STEPS, (unsigned long long)P.steps);
    S.add(ACC_PACKETS, 1ull);
    if constexpr (SinkT::is_log) {
        if (S.lg.pk_steps) S.lg.pk_steps[P.n - S.lg.packet0] = P.steps;
    }
    P.alive = 0;
}

// smallest cell index with cdf > target (stratified targets increase along a work item, so the
// search gallops forward from the lane's previous launch cell; identical result to bisection)
__device__ __forceinline__ int cdf_find(const long long *__restrict__ cb, int ncell, long long tbits, int hint)
{
    int lo = 0, hi = ncell - 1;
    if (hint >= 0) {
        if (__ldg(cb + hint) > tbits) return hint;
        int step = 1, base = hint;
        for (;;) {
            const int probe = min(base + step, ncell - 1);
            if (probe == ncell - 1 || __ldg(cb + probe) > tbits) {
                lo = base + 1;
                hi = probe;
                break;
            }
            base = probe;
            step <<= 1;
        }
    }
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(cb + mid) > tbits) hi = mid; else lo = mid + 1;
    }
    return lo;
}

// stellar limb darkening (Sect. 5.1): I(mu) / I(disk centre) for the laws GCMC_LD_*, negative values as 0
template <typename real> __device__ __noinline__ real limb(const DevJob &J, real mu)
{
    const real x = (real)1 - mu;
    const real c0 = JV<real>::ld_c(J, 0), c1 = JV<real>::ld_c(J, 1);
    real I = (real)1;
    switch (J.ld_law) {
    case GCMC_LD_LINEAR: I = (real)1 - c0 * x; break;
    case GCMC_LD_QUADRATIC: I = (real)1 - c0 * x - c1 * x * x; break;
    case GCMC_LD_SQRT: I = (real)1 - c0 * x - c1 * ((real)1 - M<real>::sqrt_(mu)); break;
    case GCMC_LD_LOG: I = (real)1 - c0 * x - c1 * (mu > (real)0 ? mu * log(mu) : (real)0); break;
    case GCMC_LD_POWER2: I = (real)1 - c0 * ((real)1 - pow(mu, c1)); break;
    case GCMC_LD_CLARET4:
        for (int k = 1; k <= 4; ++k) I -= JV<real>::ld_c(J, k - 1) * ((real)1 - pow(mu, (real)(0.5 * k)));
        break;
    default: break;
    }
    return I > (real)0 ? I : (real)0;
}

// band job (Sect. 4.7): g-ordinate with probability q(g) from the fourth word of event 1 (decided in
// FP64), then the cell from that g's pdf with the launch uniform, u Q_tot(g) in exact integers; returns
// the cell, the packet's table offset g ncell and its weight W_g
template <typename real>
__device__ __noinline__ int band_draw(const DevJob &J, const DevGrid &G, int64_t n, uint32_t wx, int &goff, real &Wg)
{
    const uint4 w1 = draw_words(J.seed, n, 1u, J.key);
    const double ug = u01<double>(w1.w);
    int g = 0;
    while (g < J.ng_s - 1 && !(J.gtab[g * GTAB_ROW] > ug)) ++g;
    goff = g * (int)G.ncell;
    Wg = (real)J.gtab[g * GTAB_ROW + 1];
    const unsigned long long qg = (unsigned long long)reinterpret_cast<const long long *>(J.gtab)[g * GTAB_ROW + 3];
    const long long target = (long long)__umul64hi((unsigned long long)(2u * (wx >> 8) + 1u) << 39, qg);
    return cdf_find(J.cdf + goff, (int)G.ncell, target, -1);
}

// S2: packet launch (Sect. 5: albedo disk, emission hybrid pdf, transmission annulus)
template <typename real, bool SCAT, int FEAT, class SinkT>
__device__ void launch(Packet<real> &P, const DevJob &J, const DevGrid &G, int64_t n, SinkT &S)
{
    P.n = n;
    P.steps = 0;
    P.alive = 1;
    P.ended = 0;
    P.ev = 2;
    P.goff = 0;
    if constexpr (SinkT::is_log) {
        if (S.lg.pk_tau) S.lg.pk_tau[n - S.lg.packet0] = -1.0;
        if (S.lg.pk_steps) S.lg.pk_steps[n - S.lg.packet0] = 0;
    }
    const uint4 w = draw_words(J.seed, n, 0u, J.key);
    if (J.mode != GCMC_EMISSION) {
        const real Rt = (real)G.Rtoa, R0 = (real)G.R0;
        const real u0 = u01<real>(w.x), u1 = u01<real>(w.y);
        real b, h;
        if (SCAT && J.mode == GCMC_ALBEDO) b = Rt * M<real>::sqrt_(u0);
        else b = R0 + u0 * (Rt - R0);
        if constexpr (sizeof(real) == 8) h = sqrt(fmax(0.0, Rt * Rt - b * b));
        else h = M<real>::sqrt_(fmaxf(0.0f, (Rt - b) * (Rt + b)));
        real sp, cp;
        M<real>::sincos_((real)(2.0 * PI) * u1, &sp, &cp);
        real x[3], d[3];
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            x[q] = b * (cp * JV<real>::e1(J, q) + sp * JV<real>::e2(J, q)) + h * JV<real>::star(J, q);
            d[q] = -JV<real>::star(J, q);
        }
        int i, j;
        locate_angles<real>(G, x[0], x[1], x[2], i, j);
        P.W = P.W0 = (real)1;
        if constexpr ((FEAT & FEAT_EXT) != 0) {
            if (J.mode == GCMC_TRANSMISSION && J.ld_law != GCMC_LD_NONE) {
                // the chord's sky-plane position on the stellar disk gives the stellar zenith-angle cosine
                const real X = JV<real>::tr_x(J) + b * cp, Y = JV<real>::tr_y(J) + b * sp;
                const real Rs = JV<real>::star_r(J);
                const real q = M<real>::div_(X * X + Y * Y, Rs * Rs);
                P.W = P.W0 = q < (real)1 ? limb<real>(J, M<real>::sqrt_((real)1 - q)) : (real)0;
            }
        }
        S.ledger(0, P.W0);
        P.ix = x[0];
        P.iy = x[1];
        P.iz = x[2];
        P.ci = i;
        P.cj = j;
        P.ck = G.nr - 1;
        if constexpr (SCAT) {
            if (J.mode == GCMC_ALBEDO) {
                if constexpr ((FEAT & FEAT_EXT) != 0) start_first_flight<real>(P, J, S);
                else start_flight<real>(P, J, S, d[0], d[1], d[2]);
                return;
            }
        }
        P.bimp = b / Rt;
        if (P.W == (real)0) {   // a chord off the stellar disk carries nothing and is not traced
            finish<real>(P, S);
            return;
        }
        S.trace(n, -3, (real)0);
        start_ray<real>(P, x[0], x[1], x[2], d[0], d[1], d[2], i, j, G.nr - 1, K_CHORD, (real)-1);
        return;
    }
    // emission: stratified inverse-CDF draw of the cell over the hybrid pdf
    // stratified target (n + u) Q_tot / N in 2^62 fixed point with u = (m + 1/2) 2^-24, m the top 24
    // bits of the word: n step + floor((2m + 1) step / 2^25), exact integer arithmetic (< Q_tot)
    const real *wcell = reinterpret_cast<const real *>(J.wcell);
    real Wg = (real)1;
    int idx;
    if ((FEAT & FEAT_BAND) && J.ng_s > 0) {
        idx = band_draw<real>(J, G, n, w.x, P.goff, Wg);
        wcell += P.goff;
    } else {
        const unsigned long long step = (unsigned long long)J.cdf_step_fix;
        const long long target = (long long)((unsigned long long)n * step +
                                             __umul64hi((unsigned long long)(2u * (w.x >> 8) + 1u) << 39, step));
        idx = cdf_find(J.cdf, (int)G.ncell, target, P.hint);
        P.hint = idx;
    }
    const int nll = G.nlon * G.nlat;
    const int k = (int)(((uint64_t)idx * G.mag_ll) >> 40);
    const int rem = idx - k * nll;
    const int j = (int)(((uint64_t)rem * G.mag_lon) >> 40);
    const int i = rem - j * G.nlon;
    const real u1 = u01<real>(w.y), u2 = u01<real>(w.z), u3 = u01<real>(w.w);
    real r, sl, ph;
    float cl_f = 0.0f;
    if constexpr (sizeof(real) == 8) {
        const double r1 = G.r[k], r2 = G.r[k + 1];
        r = cbrt(r1 * r1 * r1 + u1 * (r2 * r2 * r2 - r1 * r1 * r1));
        const double s1 = G.slat[j], s2 = G.slat[j + 1];
        sl = s1 + u2 * (s2 - s1);
        ph = G.lon[i] + u3 * (G.lon[i + 1] - G.lon[i]);
    } else {
        // r = r1 (1 + u A)^(1/3), A = (r2/r1)^3 - 1, as r1 + (r1_lo + r1 expm1(log1p(u A)/3)); sin(lat) and
        // lon likewise from hi + lo edges: each coordinate is rounded once, so no edge rounding is
        // shared by all packets of a cell
        const float r1 = __ldg(G.r_f + k);
        const float x = u1 * __ldg(G.shA_f + k);
        // (1 + x)^(1/3) - 1: binomial series for thin shells (truncation < 3e-8 relative at x < 0.05)
        const float t = x < 0.05f ? x * (1.0f / 3.0f + x * (-1.0f / 9.0f + x * (5.0f / 81.0f + x * (-10.0f / 243.0f +
                                                                                                 x * (22.0f / 729.0f)))))
                                  : expm1f(log1pf(x) * (1.0f / 3.0f));
        r = r1 + __fmaf_rn(r1, t, __ldg(G.r_lo_f + k));
        ph = __ldg(G.lon_f + i) + __fmaf_rn(u3, __ldg(G.dlon_f + i), __ldg(G.lon_lo_f + i));
        const float s1 = __ldg(G.slat_f + j), s2 = __ldg(G.slat_f + j + 1), ds = __ldg(G.dslat_f + j);
        if (s1 >= 0.0f || s2 <= 0.0f) {
            // a band in one hemisphere: c = 1 - |sin(lat)| is uniform in the band like sin(lat), linear from
            // its value at the lower edge; cos(lat) = sqrt(c (2 - c)) keeps its relative precision at the poles
            // The largest uniform, 1 - 2^-25, rounds to 1 in FP32; at the north pole band's top that would
            // put c at 0 or, through the rounding of the edge, a hair below it (cos(lat) not a number), or
            // the point on the polar axis, where the azimuth and so the longitude cell are undefined.  So
            // the uniform is kept below 1 (1 - 2^-24, its FP32 neighbour) and c at or above 0.
            const bool north = s1 >= 0.0f;
            const float ub = fminf(u2, 0x1.fffffep-1f);
            const float c = fmaxf(__fmaf_rn(north ? -ub : ub, ds, __ldg(G.cb_f + j)) + __ldg(G.cb_lo_f + j), 0.0f);
            sl = north ? 1.0f - c : c - 1.0f;
            cl_f = sqrtf(c * (2.0f - c));
        } else {
            sl = s1 + __fmaf_rn(u2, ds, __ldg(G.slat_lo_f + j));
            cl_f = sqrtf(fmaxf(0.0f, 1.0f - sl * sl));
        }
    }
    real cl;
    if constexpr (sizeof(real) == 8) cl = sqrt(fmax(0.0, 1.0 - sl * sl));
    else cl = cl_f;
    real sp, cp;
    M<real>::sincos_(ph, &sp, &cp);
    P.ix = r * cl * cp;
    P.iy = r * cl * sp;
    P.iz = r * sl;
    P.ci = i;
    P.cj = j;
    P.ck = k;
    P.cell0 = idx;
    P.W = P.W0 = Wg * wcell[idx];
    S.ledger(0, P.W0);
    P.stage = 0;
    P.obs = 0;
    start_peel<real>(P, J, S);
}

template <typename real, int FEAT, class SinkT>
__device__ void after_peels_scatter(Packet<real> &P, const DevJob &J, SinkT &S)
{
    const real om = P.om;
    if (P.W * om == (real)0) {
        S.ledger(2, P.W);
        finish<real>(P, S);
        return;
    }
    if (J.survival) {
        S.ledger(2, P.W * ((real)1 - om));
        P.W *= om;
        if (P.W < JV<real>::w_rr(J) * P.W0) {
            const uint4 v = draw_words(J.seed, P.n, P.ev | 0x80000000u, J.key);
            if (u01<real>(v.y) < JV<real>::p_surv(J)) {
                const real Wn = P.W / JV<real>::p_surv(J);
                S.ledger(4, Wn - P.W);
                P.W = Wn;
            } else {
                S.ledger(5, P.W);
                finish<real>(P, S);
                return;
            }
        }
    } else {
        const uint4 v = draw_words(J.seed, P.n, P.ev | 0x80000000u, J.key);
        if (!(u01<real>(v.x) < om)) {
            S.ledger(2, P.W);
            finish<real>(P, S);
            return;
        }
        if (P.W < JV<real>::w_rr(J) * P.W0) {
            // forcing and continuous absorption change weights in analog mode too: the same roulette
            if (u01<real>(v.y) < JV<real>::p_surv(J)) {
                const real Wn = P.W / JV<real>::p_surv(J);
                S.ledger(4, Wn - P.W);
                P.W = Wn;
            } else {
                S.ledger(5, P.W);
                finish<real>(P, S);
                return;
            }
        }
    }
    // the words of this flight's event, drawn when the flight started
    const real u1 = u01<real>(S.wc[0]), u2 = u01<real>(S.wc[S.stride]), u3 = u01<real>(S.wc[2 * S.stride]);
    real mu;
    if (u1 < P.pg) {
        mu = sample_rayleigh<real>(u2);
    } else {
        // cloud: HG, or the two-term HG whose term is chosen by u1 rescaled to (u1 - P_gas) / (1 - P_gas)
        real gs = P.gg;
        if constexpr ((FEAT & FEAT_EXT) != 0) {
            if (J.cloud_phase == GCMC_CLOUD_TTHG) {
                real g2, a;
                tthg_terms<real>(P.gg, g2, a);
                gs = M<real>::div_(u1 - P.pg, (real)1 - P.pg) < a ? P.gg : g2;
            }
        }
        mu = sample_hg<real>(gs, u2, JV<real>::hg_eps(J));
    }
    real dx = P.fx, dy = P.fy, dz = P.fz;
    turn<real>(dx, dy, dz, mu, (real)(2.0 * PI) * u3);
    ++P.ev;
    start_next_flight<real, (FEAT & FEAT_EXT) != 0>(P, J, S, dx, dy, dz);
}

// first observer, from o on, above the horizon of the surface point (normal in fx, fy, fz)
template <typename real>
__device__ __forceinline__ int surface_obs(const Packet<real> &P, const DevJob &J, int o)
{
    for (; o < J.n_obs; ++o)
        if (P.fx * JV<real>::obs(J, o, 0) + P.fy * JV<real>::obs(J, o, 1) + P.fz * JV<real>::obs(J, o, 2) > (real)0) break;
    return o;
}

// Lambertian reflection after the surface peel-offs (Sect. 3): weight A_s (survival biasing, then
// roulette) or reflection with probability A_s (analog); the absorbed part ends at the lower boundary.
// New direction: cosine sqrt(u2) about the normal, azimuth 2 pi u3, from the flight's own draws.
template <typename real, class SinkT>
__device__ void after_peels_surface(Packet<real> &P, const DevJob &J, SinkT &S)
{
    const real As = JV<real>::surf_as(J);
    if (J.survival) {
        S.ledger(3, P.W * ((real)1 - As));
        P.W *= As;
        if (P.W < JV<real>::w_rr(J) * P.W0) {
            const uint4 v = draw_words(J.seed, P.n, P.ev | 0x80000000u, J.key);
            if (u01<real>(v.y) < JV<real>::p_surv(J)) {
                const real Wn = P.W / JV<real>::p_surv(J);
                S.ledger(4, Wn - P.W);
                P.W = Wn;
            } else {
                S.ledger(5, P.W);
                finish<real>(P, S);
                return;
            }
        }
    } else {
        const uint4 v = draw_words(J.seed, P.n, P.ev | 0x80000000u, J.key);
        if (!(u01<real>(v.x) < As)) {
            S.ledger(3, P.W);
            finish<real>(P, S);
            return;
        }
        if (P.W < JV<real>::w_rr(J) * P.W0) {
            // forcing and continuous absorption change weights in analog mode too: the same roulette
            if (u01<real>(v.y) < JV<real>::p_surv(J)) {
                const real Wn = P.W / JV<real>::p_surv(J);
                S.ledger(4, Wn - P.W);
                P.W = Wn;
            } else {
                S.ledger(5, P.W);
                finish<real>(P, S);
                return;
            }
        }
    }
    // the words of this flight's event, drawn when the flight started
    real dx = P.fx, dy = P.fy, dz = P.fz;
    turn<real>(dx, dy, dz, M<real>::sqrt_(u01<real>(S.wc[S.stride])), (real)(2.0 * PI) * u01<real>(S.wc[2 * S.stride]));
    ++P.ev;
    start_next_flight<real, true>(P, J, S, dx, dy, dz);
}

template <typename real, bool SCAT, int FEAT, class SinkT>
__device__ void on_end(Packet<real> &P, const DevJob &J, SinkT &S, int e, int idx)
{
    constexpr bool EXT = (FEAT & FEAT_EXT) != 0;
    Ray<real> &R = P.ray;
    if constexpr (SCAT && EXT) {
        if (P.kind == K_FORCE) {
            // forced scattering (Sect. 4.2): R.tau is the optical depth of the flight's path to the grid
            // boundary; W e^-tau leaves unscattered, W (1 - e^-tau) interacts before it.  Not forced past
            // the cut-off depth or when the path ends on a reflecting surface.  The flight's direction is
            // in fx, fy, fz.
            if (e == E_CAP) {
                S.ledger(6, P.W);
                finish<real>(P, S);
                return;
            }
            real p = (real)1;
            const bool forced = J.path_bias != 1 &&
                                (e == E_ESCAPE || (e == E_BOTTOM && !(JV<real>::surf_as(J) > (real)0)));
            int mode = forced ? (J.path_bias == 2 ? FL_HYBRID : FL_FORCED) : FL_NATURAL;
            if (J.path_bias == 1 && e != E_CUTOFF) mode = FL_STRETCH;   // stretching does not force
            if (forced) {
                real em;
                if constexpr (sizeof(real) == 8) em = expm1(-R.tau);
                else em = expm1f(-R.tau);
                p = -em;
                const real rem = P.W * M<real>::exp_(-R.tau);
                const int q = e == E_ESCAPE ? 1 : 3;
                if (J.cont_abs) {
                    const real kept = rem * M<real>::exp_(-R.tau2);
                    S.ledger(q, kept);
                    S.ledger(2, rem - kept);
                } else {
                    S.ledger(q, rem);
                }
                P.W *= p;
            }
            start_flight<real>(P, J, S, P.fx, P.fy, P.fz, mode, p, R.tau);
            return;
        }
        if (P.kind == K_FLIGHT && J.cont_abs) {
            // continuous absorption (Sect. 4.1): the weight decays by e^-tau_abs along the flight
            const real Wn = P.W * M<real>::exp_(-R.tau2);
            S.ledger(2, P.W - Wn);
            P.W = Wn;
        }
        if (P.kind == K_FLIGHT && e == E_BOTTOM && JV<real>::surf_as(J) > (real)0) {
                // a reflecting lower boundary: surface point and its outward normal (kept in fx, fy, fz),
                // then the peel-offs towards the observers above its horizon
                P.ix = R.cx + R.s * R.dx;
                P.iy = R.cy + R.s * R.dy;
                P.iz = R.cz + R.s * R.dz;
                const real rr = M<real>::sqrt_(P.ix * P.ix + P.iy * P.iy + P.iz * P.iz);
                P.fx = M<real>::div_(P.ix, rr);
                P.fy = M<real>::div_(P.iy, rr);
                P.fz = M<real>::div_(P.iz, rr);
                P.ci = R.i;
                P.cj = R.j;
                P.ck = R.k;
                P.cell0 = idx;
                P.stage = 2;
                P.obs = surface_obs<real>(P, J, 0);
                if (P.obs < J.n_obs) start_peel<real>(P, J, S);
                else after_peels_surface<real>(P, J, S);
                return;
        }
    }
    if constexpr (SCAT) {
        if (P.kind == K_FLIGHT) {
            if (e != E_INTERACT) {
                S.ledger(e == E_ESCAPE ? 1 : e == E_BOTTOM ? 3 : e == E_CAP ? 6 : 7, P.W);
                finish<real>(P, S);
                return;
            }
            P.fx = R.dx;
            P.fy = R.dy;
            P.fz = R.dz;
            P.ix = R.cx + R.s * R.dx;
            P.iy = R.cy + R.s * R.dy;
            P.iz = R.cz + R.s * R.dz;
            P.ci = R.i;
            P.cj = R.j;
            P.ck = R.k;
            P.cell0 = idx;
            if constexpr (sizeof(real) == 4) {
                const float4 rc = __ldg(reinterpret_cast<const float4 *>(J.rec) + idx);
                P.om = rc.y;
                P.gg = rc.z;
                P.pg = rc.w;
            } else {
                const Rec64 rc = reinterpret_cast<const Rec64 *>(J.rec)[idx];
                P.om = rc.w;
                P.gg = rc.g;
                P.pg = rc.pg;
            }
            if constexpr (EXT) {
                if (J.cont_abs) P.om = (real)1;   // continuous absorption: the interaction is a scattering
            }
            P.stage = 1;
            P.obs = 0;
            start_peel<real>(P, J, S);
            return;
        }
    }
    if (P.kind == K_PEEL) {
        if (e == E_CAP) {
            S.ledger(6, P.W);
            finish<real>(P, S);
            return;
        }
        const real ex = (e == E_ESCAPE) ? M<real>::exp_(-R.tau) : (real)0;
        real f;
        if (!SCAT || P.stage == 0) {
            if constexpr (SinkT::is_log) {
                if (P.obs == 0 && S.lg.pk_tau) S.lg.pk_tau[P.n - S.lg.packet0] = (double)R.tau;
            }
            f = P.W * ex * (real)(1.0 / (4.0 * PI));
        } else {
            const real mu = P.fx * JV<real>::obs(J, P.obs, 0) + P.fy * JV<real>::obs(J, P.obs, 1) + P.fz * JV<real>::obs(J, P.obs, 2);
            if constexpr (EXT) {
                if (P.stage == 2) f = P.W * JV<real>::surf_as(J) * (mu * (real)(1.0 / PI)) * ex;   // Lambert: mu_o / pi
                else f = P.W * P.om * theta_mix<real>(mu, P.pg, P.gg, J.cloud_phase == GCMC_CLOUD_TTHG) * ex;
            } else {
                f = P.W * P.om * theta_mix<real>(mu, P.pg, P.gg) * ex;
            }
        }
        int col = P.obs;
        if constexpr (SCAT && EXT) {
            // transmission: scattered light goes to column 1, weighted by the launch b / R_TOA
            if (J.mode == GCMC_TRANSMISSION) {
                col = 1;
                f = f * P.bimp;
            }
        }
        S.tally(col, f, P.n, J.n_tal);
        if (J.cf && f < (real)1.0e9 && f >= (real)0) {
            // the same fixed-point contribution, by the cell the peel-off left from
            const int kind = (!SCAT || P.stage == 0) ? 0 : 1;
            atomicAdd(J.cf + (int64_t)(kind * J.n_obs + P.obs) * J.cf_ncell + P.cell0,
                      (unsigned long long)to_fix<real>(f));
        }
        ++P.obs;
        if constexpr (SCAT && EXT) {
            if (P.stage == 2) P.obs = surface_obs<real>(P, J, P.obs);
        }
        if (P.obs < J.n_obs) {
            start_peel<real>(P, J, S);
            return;
        }
        if constexpr (SCAT) {
            if (J.mode != GCMC_EMISSION) {
                if constexpr (EXT) {
                    if (P.stage == 2) {
                        after_peels_surface<real>(P, J, S);
                        return;
                    }
                }
                after_peels_scatter<real, FEAT>(P, J, S);
                return;
            }
        }
        finish<real>(P, S);
        return;
    }
    // chord (column 0: W (1 - e^-tau) b / R_TOA)
    const bool through = e == E_ESCAPE || e == E_CUTOFF || e == E_BOTTOM;
    real c = (real)0;
    if (e == E_ESCAPE) c = M<real>::one_minus_exp_neg(R.tau) * P.bimp;
    else if (through) c = P.bimp;
    if constexpr (SinkT::is_log) {
        if (S.lg.pk_tau) S.lg.pk_tau[P.n - S.lg.packet0] = (double)R.tau;
    }
    S.tally(0, P.W * c, P.n, J.n_tal);
    if (!through) {
        S.ledger(e == E_CAP ? 6 : 7, P.W);
        finish<real>(P, S);
        return;
    }
    if constexpr (SCAT && EXT) {
        if (J.trans_scatter) {
            // multiple scattering (Sect. 5.1): the packet itself flies from its launch point along -star
            start_first_flight<real>(P, J, S);
            return;
        }
    }
    S.ledger(1, P.W);
    finish<real>(P, S);
}

// one cell step (S3-S7) of the packet's current ray; FEAT_BAND kernels read the packet's g-ordinate
// table (band jobs), FEAT_CABS kernels carry continuous absorption
template <typename real, bool SCAT, int FEAT, class SinkT>
__device__ __forceinline__ void step(Packet<real> &P, const DevJob &J, const DevGrid &G, const Tabs<real> &T,
                                     const JobC<real> &jc, SinkT &S)
{
    Ray<real> &R = P.ray;
    if (P.steps >= jc.max_steps) {
        P.ended = 1;
        P.end_e = E_CAP;
        P.end_idx = 0;
        return;
    }
    ++P.steps;
    const int idx = (R.k * T.nlat + R.j) * T.nlon + R.i;
    real a;
    const int go = (FEAT & FEAT_BAND) ? P.goff : 0;
    real a2 = (real)0;
    if constexpr (SCAT && (FEAT & FEAT_CABS) != 0) {
        if (jc.contabs) {
            // continuous absorption: flights (and the forcing march) run in the scattering opacity omega alpha
            // and accumulate the absorption (1 - omega) alpha
            const auto aw = __ldg(reinterpret_cast<const typename Pair<real>::type *>(jc.recf + 4 * idx));
            const bool fl = P.kind == K_FLIGHT || P.kind == K_FORCE;
            const real as = aw.x * aw.y;
            a = fl ? as : aw.x;
            a2 = fl ? aw.x - as : (real)0;
        } else {
            a = __ldg(jc.rec + idx + go);
        }
    } else {
        a = __ldg(jc.rec + idx + go);
    }
    bool to_lat, to_lon;
    int dk;
    const real sx = cell_exit<real>(G, T, R, to_lat, to_lon, dk);
    const real seg = sx - R.s;
    if constexpr (SCAT) {
        if (R.tau_target >= (real)0 && a > (real)0 && R.tau + a * seg >= R.tau_target) {
            const real l = M<real>::div_(R.tau_target - R.tau, a);
            if constexpr ((FEAT & FEAT_CABS) != 0) {
                if (jc.contabs) R.tau2 += a2 * l;
            }
            S.trace(P.n, idx, l);
            R.s += l;
            R.tau = R.tau_target;
            P.ended = 1;
            P.end_e = E_INTERACT;
            P.end_idx = idx;
            return;
        }
    }
    R.tau += a * seg;
    if constexpr (SCAT && (FEAT & FEAT_CABS) != 0) {
        if (jc.contabs) R.tau2 += a2 * seg;
    }
    S.trace(P.n, idx, seg);
    R.s = sx;
    int e = cross_face<real>(T, R, to_lat, to_lon, dk);
    // the optical-depth cut-off applies to marches without an interaction target (peel-offs, chords;
    // every march of an absorber-only kernel)
    if (e == E_CONT && (!SCAT || R.tau_target < (real)0) && R.tau > jc.tau_cut) e = E_CUTOFF;
    if (e != E_CONT) {
        P.ended = 1;
        P.end_e = e;
        P.end_idx = idx;
    }
}

// the end of the packet's current ray: tally, next ray, interaction or finish
template <typename real, bool SCAT, int FEAT, class SinkT>
__device__ __forceinline__ void settle(Packet<real> &P, const DevJob &J, SinkT &S)
{
    P.ended = 0;
    on_end<real, SCAT, FEAT>(P, J, S, P.end_e, P.end_idx);
}

// warp-reduce the per-thread accumulators and add them to the job's totals
__device__ __forceinline__ void flush(unsigned long long *sm, int stride, unsigned long long *acc)
{
    const int lane = threadIdx.x & 31;
#pragma unroll 1
    for (int s = 0; s < NSLOT; ++s) {
        unsigned long long v = sm[s * stride];
        sm[s * stride] = 0ull;
        if (s == ACC_FLAGS) {
#pragma unroll
            for (int o = 16; o; o >>= 1) v |= __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0 && v) atomicOr(acc + s, v);
        } else {
#pragma unroll
            for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0 && v) atomicAdd(acc + s, v);
        }
    }
}

template <typename real> __device__ __forceinline__ JobC<real> job_consts(const DevJob &J)
{
    JobC<real> c;
    c.max_steps = (int)min(J.max_steps, (int64_t)INT_MAX);
    c.tau_cut = (real)J.tau_cut;
    c.rec = reinterpret_cast<const real *>(J.arec ? J.arec : J.rec);
    c.recf = J.rec4 ? reinterpret_cast<const real *>(J.rec) : nullptr;
    c.contabs = J.cont_abs;
    return c;
}

template <typename real, bool SCAT, bool LOG, int FEAT>
__global__ void __launch_bounds__(256) k_transport_plain(const DevGrid *__restrict__ grids,
                                                         const DevJob *__restrict__ jobp, int64_t packet0, int64_t n_run,
                                                         LogOut lg)
{
    extern __shared__ __align__(16) unsigned long long sacc[];
    Sink<real, LOG> S;
    S.sm = sacc + threadIdx.x;
    S.stride = blockDim.x;
    S.wc = reinterpret_cast<uint32_t *>(sacc + NSLOT * blockDim.x) + threadIdx.x;
    S.lg = lg;
    for (int s = 0; s < NSLOT; ++s) S.sm[s * S.stride] = 0ull;
    const DevJob &J = *jobp;
    const DevGrid &G = grids[J.grid_slot];
    auto *tab = reinterpret_cast<typename Pair<real>::type *>(reinterpret_cast<uint32_t *>(sacc + NSLOT * blockDim.x) +
                                                              3 * blockDim.x);
    const Tabs<real> T = stage_tabs<real>(G, tab, threadIdx.x, blockDim.x);
    __syncthreads();
    const JobC<real> jc = job_consts<real>(J);
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q < n_run) {
        Packet<real> P;
        P.hint = -1;
        launch<real, SCAT, FEAT>(P, J, G, packet0 + q, S);
        while (P.alive) {
            if (P.ended) settle<real, SCAT, FEAT>(P, J, S);
            else step<real, SCAT, FEAT>(P, J, G, T, jc, S);
        }
    }
    __syncwarp();
    flush(S.sm, S.stride, J.acc);
}

// One work item (packets p0 .. p1-1 of job J) on one warp: lanes whose packets have finished are
// refilled together once at least refill_min of them are idle; rays that ended are settled at
// those points; between them every live lane takes `interval` cell steps.
template <typename real, bool SCAT, int FEAT, class SinkT>
__device__ __forceinline__ void run_item(const DevJob &J, const DevGrid &G, const Tabs<real> &T, int64_t p0, int64_t p1,
                                         int interval, int refill_min, SinkT &S)
{
    const unsigned lt = (1u << (threadIdx.x & 31)) - 1u;
    const JobC<real> jc = job_consts<real>(J);
    const int count = (int)(p1 - p0);          // packets of the item (at most chunk)
    int next = 0;                              // packets of the item started so far
    Packet<real> P;
    P.alive = 0;
    P.hint = -1;
    P.ended = 0;
    for (;;) {
        if (P.alive && P.ended) settle<real, SCAT, FEAT>(P, J, S);
        const unsigned idle = __ballot_sync(0xffffffffu, !P.alive);
        const int left = count - next;
        if (idle && left > 0) {
            const int n_idle = __popc(idle);
            if (n_idle >= min(refill_min, left)) {
                const int mine = next + __popc(idle & lt);
                if (!P.alive && mine < count) launch<real, SCAT, FEAT>(P, J, G, p0 + mine, S);
                next += n_idle;
            }
        }
        if (!__any_sync(0xffffffffu, P.alive)) break;
        for (int t = 0; t < interval; ++t)
            if (P.alive && !P.ended) step<real, SCAT, FEAT>(P, J, G, T, jc, S);
    }
    __syncwarp();
}

// MINB > 0: compiled for MINB resident 128-thread blocks per SM (register cap 65536 / (128 MINB));
// MINB = 0: any block size up to 256, at most 128 registers (two 256-thread blocks per SM)
template <typename real, bool SCAT, int MINB, int FEAT>
__global__ void __launch_bounds__(MINB ? 128 : 256, MINB ? MINB : 2) k_transport_persistent(const DevGrid *__restrict__ grids,
                                                              const DevJob *__restrict__ jobs, int n_jobs,
                                                              int64_t total_items, int chunk, int interval,
                                                              int refill_min, int one_grid, int tab_n,
                                                              unsigned long long *work)
{
    extern __shared__ __align__(16) unsigned long long sacc[];
    Sink<real, false> S;
    S.sm = sacc + threadIdx.x;
    S.stride = blockDim.x;
    S.wc = reinterpret_cast<uint32_t *>(sacc + NSLOT * blockDim.x) + threadIdx.x;
    for (int s = 0; s < NSLOT; ++s) S.sm[s * S.stride] = 0ull;
    const int lane = threadIdx.x & 31;
    // march tables in shared memory: one copy per block when every job uses the same grid, else one
    // per warp, restaged when the warp's work item comes from another grid
    auto *tab0 = reinterpret_cast<typename Pair<real>::type *>(reinterpret_cast<uint32_t *>(sacc + NSLOT * blockDim.x) +
                                                               3 * blockDim.x);
    Tabs<real> T;
    int cur_grid = -1;
    if (one_grid) {
        cur_grid = jobs[0].grid_slot;
        T = stage_tabs<real>(grids[cur_grid], tab0, threadIdx.x, blockDim.x);
        __syncthreads();
    }
    for (;;) {
        unsigned long long item = 0;
        if (lane == 0) item = atomicAdd(work, 1ull);
        item = __shfl_sync(0xffffffffu, item, 0);
        if ((int64_t)item >= total_items) break;
        // job of this item: last job whose first item is <= item
        int lo = 0, hi = n_jobs - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (jobs[mid].chunk_begin <= (int64_t)item) lo = mid; else hi = mid - 1;
        }
        const DevJob &J = jobs[lo];
        const DevGrid &G = grids[J.grid_slot];
        if (J.grid_slot != cur_grid) {
            __syncwarp();
            cur_grid = J.grid_slot;
            T = stage_tabs<real>(G, tab0 + (threadIdx.x >> 5) * tab_n, lane, 32);
            __syncwarp();
        }
        const int64_t p0 = ((int64_t)item - J.chunk_begin) * chunk;
        run_item<real, SCAT, FEAT>(J, G, T, p0, min(p0 + (int64_t)chunk, J.n_packets), interval, refill_min, S);
        flush(S.sm, S.stride, J.acc);
    }
}

// ------------------------------------------------------------------ serving kernel
// A persistent kernel fed by a queue of jobs that the host publishes while it runs (continuous
// batching).  Warps drain the published jobs in publication order: each claims work items of the
// oldest job that has unclaimed items (from the counter of the job's slot), runs them, and adds its
// tallies; the warp that finishes a job's last item
// copies the job's accumulators and emission totals into the job's completion record in host-mapped
// memory and then writes the record's sequence number.  A warp that finds no published work polls
// with a sleep and leaves after `idle_polls` empty polls, or at once when the host sets `stop`; the
// host relaunches the kernel when new work is published after it has left.
__device__ __forceinline__ unsigned long long ld_acquire_sys(const unsigned long long *p)
{
    unsigned long long v;
    asm volatile("ld.acquire.sys.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ unsigned int ld_acquire_sys(const unsigned int *p)
{
    unsigned int v;
    asm volatile("ld.acquire.sys.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ unsigned long long ld_relaxed_gpu(const unsigned long long *p)
{
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_sys(unsigned long long *p, unsigned long long v)
{
    asm volatile("st.release.sys.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

template <typename real, bool SCAT, int FEAT>
__global__ void __launch_bounds__(128, 4) k_transport_serve(const DevGrid *__restrict__ grids, ServeQueue q, int chunk,
                                                         int interval, int refill_min, int tab_n, int idle_polls)
{
    extern __shared__ __align__(16) unsigned long long sacc[];
    Sink<real, false> S;
    S.sm = sacc + threadIdx.x;
    S.stride = blockDim.x;
    S.wc = reinterpret_cast<uint32_t *>(sacc + NSLOT * blockDim.x) + threadIdx.x;
    for (int s = 0; s < NSLOT; ++s) S.sm[s * S.stride] = 0ull;
    const int lane = threadIdx.x & 31;
    auto *tabw = reinterpret_cast<typename Pair<real>::type *>(reinterpret_cast<uint32_t *>(sacc + NSLOT * blockDim.x) +
                                                               3 * blockDim.x) +
                 (threadIdx.x >> 5) * tab_n;
    Tabs<real> T;
    int cur_grid = -1;
    long long empty = 0;
    bool idle = false;
    const unsigned long long n_warps = (unsigned long long)gridDim.x * (blockDim.x >> 5);
    for (;;) {
        // the kernel leaves as a whole: once one warp has seen every warp idle for idle_polls polls it
        // sets `exiting`, and every warp leaves at its next check (work published later is taken by
        // the next launch)
        // lane 0 reads the queue state; the warp takes every decision on the broadcast values
        unsigned long long seg = 0, pub = 0, leaving = 0;
        if (lane == 0) {
            leaving = ld_relaxed_gpu(q.exiting);
            seg = ld_relaxed_gpu(q.cur_seg);
            pub = ld_acquire_sys(&q.ctl->published);
        }
        leaving = __shfl_sync(0xffffffffu, leaving, 0);
        seg = __shfl_sync(0xffffffffu, seg, 0);
        pub = __shfl_sync(0xffffffffu, pub, 0);
        if (leaving) break;
        if (seg >= pub) {
            int quit = 0;
            if (lane == 0) {
                if (!idle) atomicAdd(q.n_idle, 1ull);
                const bool all_idle = ld_relaxed_gpu(q.n_idle) == n_warps;
                if ((all_idle && (empty >= idle_polls || ld_acquire_sys(&q.ctl->stop))) || empty >= SERVE_IDLE_CAP) {
                    if (!all_idle) atomicOr_system(&q.ctl->err, 2u);   // waited SERVE_IDLE_CAP polls
                    atomicExch(q.exiting, 1ull);
                    quit = 1;
                }
            }
            idle = true;
            ++empty;
            if (__shfl_sync(0xffffffffu, quit, 0)) break;
            __nanosleep(1000);
            continue;
        }
        if (idle) {
            idle = false;
            if (lane == 0) atomicAdd(q.n_idle, ~0ull);   // minus one
        }
        empty = 0;
        const unsigned r = (unsigned)(seg % SERVE_RING);
        const ServeSeg sg = q.ring[r];
        unsigned long long w = 0;
        if (lane == 0) w = atomicAdd(q.slot_next + sg.slot, 1ull);
        w = __shfl_sync(0xffffffffu, w, 0);
        const unsigned long long item = w & ((1ull << SERVE_GEN_SHIFT) - 1ull);
        if ((unsigned)(w >> SERVE_GEN_SHIFT) != (sg.gen & 0xFFFFFFu)) {
            // the slot was given to another job after this warp read the ring: report it and move on
            if (lane == 0) atomicOr_system(&q.ctl->err, 1u);
            __syncwarp();
            continue;
        }
        if ((int64_t)item >= sg.n_items) {       // every item of this job is claimed: move on
            if (lane == 0) atomicCAS(q.cur_seg, seg, seg + 1);
            __syncwarp();
            continue;
        }
        const DevJob &J = *sg.job;
        const DevGrid &G = grids[J.grid_slot];
        if (J.grid_slot != cur_grid) {
            __syncwarp();
            cur_grid = J.grid_slot;
            T = stage_tabs<real>(G, tabw, lane, 32);
            __syncwarp();
        }
        const int64_t p0 = (int64_t)item * chunk;
        run_item<real, SCAT, FEAT>(J, G, T, p0, min(p0 + (int64_t)chunk, J.n_packets), interval, refill_min, S);
        flush(S.sm, S.stride, J.acc);
        __threadfence();
        unsigned long long fin = 0;
        if (lane == 0) fin = atomicAdd(q.slot_done + sg.slot, 1ull) + 1ull;
        fin = __shfl_sync(0xffffffffu, fin, 0);
        if ((int64_t)fin == sg.n_items) {        // last item of the job: publish its completion record
            __threadfence();
            ServeDone *d = q.done + sg.slot;
            d->acc[lane] = atomicAdd(J.acc + lane, 0ull);   // ACC_SLOTS == 32: one slot per lane
            if (lane < 3) d->info[lane] = J.mode == GCMC_EMISSION ? J.info[lane] : 0.0;
            __threadfence_system();
            __syncwarp();
            if (lane == 0) st_release_sys(&d->seq, seg + 1ull);
        }
    }
}

// ------------------------------------------------------------------ host launchers
size_t transport_smem(int block) { return (size_t)NSLOT * block * sizeof(unsigned long long) + (size_t)3 * block * 4; }

static size_t tab_bytes(int precision, int entries) { return (size_t)entries * (precision == GCMC_FP64 ? 16 : 8); }

// the logging (parity) kernels carry every optional feature; the others only when the job needs one
template <typename real, bool SCAT>
static void plain_dispatch(unsigned nb, int block, size_t sm, cudaStream_t st, const DevGrid *grids, const DevJob *job,
                           int64_t packet0, int64_t n_run, const LogOut &lg, bool log, int feat)
{
    if (log) k_transport_plain<real, SCAT, true, FEAT_ALL><<<nb, block, sm, st>>>(grids, job, packet0, n_run, lg);
    else if (feat) k_transport_plain<real, SCAT, false, FEAT_ALL><<<nb, block, sm, st>>>(grids, job, packet0, n_run, lg);
    else k_transport_plain<real, SCAT, false, 0><<<nb, block, sm, st>>>(grids, job, packet0, n_run, lg);
}

cudaError_t launch_plain(int precision, bool scatter, int feat, const DevGrid *grids, const DevJob *job, int64_t packet0,
                         int64_t n_run, const HostLog *hl, int tab_entries_n, cudaStream_t st)
{
    const int block = 128;
    const int64_t nb = (n_run + block - 1) / block;
    if (nb == 0) return cudaSuccess;
    LogOut lg{};
    if (hl) {
        lg.packet0 = packet0;
        lg.pk_f = hl->pk_f;
        lg.pk_steps = hl->pk_steps;
        lg.pk_tau = hl->pk_tau;
        lg.tr_cell = hl->tr_cell;
        lg.tr_len = hl->tr_len;
        lg.tr_n = hl->tr_n;
        lg.n_trace = hl->n_trace;
        lg.max_trace = hl->max_trace;
    }
    const size_t sm = transport_smem(block) + tab_bytes(precision, tab_entries_n);
    count_launch(1);
    const unsigned g = (unsigned)nb;
    if (precision == GCMC_FP64) {
        if (scatter) plain_dispatch<double, true>(g, block, sm, st, grids, job, packet0, n_run, lg, hl != nullptr, feat);
        else plain_dispatch<double, false>(g, block, sm, st, grids, job, packet0, n_run, lg, hl != nullptr, feat);
    } else {
        if (scatter) plain_dispatch<float, true>(g, block, sm, st, grids, job, packet0, n_run, lg, hl != nullptr, feat);
        else plain_dispatch<float, false>(g, block, sm, st, grids, job, packet0, n_run, lg, hl != nullptr, feat);
    }
    return cudaGetLastError();
}

template <typename real, bool SCAT, int MINB, int FEAT>
static cudaError_t persistent_run(int block, int blocks_per_sm, int nsm, const DevGrid *grids, const DevJob *jobs,
                                  int n_jobs, int64_t total_items, int chunk, int interval, int refill_min, int one_grid,
                                  int tab_n, unsigned long long *work, cudaStream_t st)
{
    auto kern = k_transport_persistent<real, SCAT, MINB, FEAT>;
    const size_t sm = transport_smem(block) + (size_t)tab_n * sizeof(typename Pair<real>::type) * (one_grid ? 1 : block / 32);
    if (sm > 48 * 1024) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, block, sm);
    if (occ < 1) return cudaErrorInvalidConfiguration;
    if (blocks_per_sm <= 0 || blocks_per_sm > occ) blocks_per_sm = occ;
    const unsigned grid = (unsigned)(nsm * blocks_per_sm);
    kern<<<grid, block, sm, st>>>(grids, jobs, n_jobs, total_items, chunk, interval, refill_min, one_grid, tab_n, work);
    return cudaGetLastError();
}

template <typename real, bool SCAT>
static cudaError_t persistent_dispatch(int block, int blocks_per_sm, int nsm, const DevGrid *grids, const DevJob *jobs,
                                       int n_jobs, int64_t total_items, int chunk, int interval, int refill_min,
                                       int one_grid, int tab_n, unsigned long long *work, int feat, cudaStream_t st)
{
    // batches that need optional features run variants compiled with them.  FP32 absorber-only kernel:
    // band jobs (also in the capped variants) and limb-darkened chords separately; FP32 scattering
    // kernel: the optional physics with and without continuous absorption; all of them otherwise.
    if (feat) {
        if constexpr (sizeof(real) == 4 && !SCAT) {
            if (feat == FEAT_BAND) {
                if (block <= 128 && blocks_per_sm >= 8)
                    return persistent_run<real, SCAT, 8, FEAT_BAND>(block, blocks_per_sm, nsm, grids, jobs, n_jobs,
                                                                    total_items, chunk, interval, refill_min, one_grid,
                                                                    tab_n, work, st);
                if (block <= 128 && blocks_per_sm >= 6)
                    return persistent_run<real, SCAT, 6, FEAT_BAND>(block, blocks_per_sm, nsm, grids, jobs, n_jobs,
                                                                    total_items, chunk, interval, refill_min, one_grid,
                                                                    tab_n, work, st);
                return persistent_run<real, SCAT, 0, FEAT_BAND>(block, blocks_per_sm, nsm, grids, jobs, n_jobs,
                                                                total_items, chunk, interval, refill_min, one_grid,
                                                                tab_n, work, st);
            }
            if (feat == FEAT_EXT)
                return persistent_run<real, SCAT, 0, FEAT_EXT>(block, blocks_per_sm, nsm, grids, jobs, n_jobs, total_items,
                                                               chunk, interval, refill_min, one_grid, tab_n, work, st);
        }
        if constexpr (sizeof(real) == 4 && SCAT) {
            // the optional physics (transit with scattering, surfaces, TTHG, forcing; with and without
            // continuous absorption) also in variants for 5 resident 128-thread blocks per SM
            if (feat == FEAT_EXT && block <= 128 && blocks_per_sm >= 5)
                return persistent_run<real, SCAT, 5, FEAT_EXT>(block, blocks_per_sm, nsm, grids, jobs, n_jobs, total_items,
                                                               chunk, interval, refill_min, one_grid, tab_n, work, st);
            if (feat == FEAT_EXT)
                return persistent_run<real, SCAT, 0, FEAT_EXT>(block, blocks_per_sm, nsm, grids, jobs, n_jobs, total_items,
                                                               chunk, interval, refill_min, one_grid, tab_n, work, st);
            if (feat == (FEAT_EXT | FEAT_CABS) && block <= 128 && blocks_per_sm >= 5)
                return persistent_run<real, SCAT, 5, FEAT_EXT | FEAT_CABS>(block, blocks_per_sm, nsm, grids, jobs, n_jobs,
                                                                           total_items, chunk, interval, refill_min,
                                                                           one_grid, tab_n, work, st);
            if (feat == (FEAT_EXT | FEAT_CABS))
                return persistent_run<real, SCAT, 0, FEAT_EXT | FEAT_CABS>(block, blocks_per_sm, nsm, grids, jobs, n_jobs,
                                                                           total_items, chunk, interval, refill_min,
                                                                           one_grid, tab_n, work, st);
        }
        return persistent_run<real, SCAT, 0, FEAT_ALL>(block, blocks_per_sm, nsm, grids, jobs, n_jobs, total_items, chunk,
                                                       interval, refill_min, one_grid, tab_n, work, st);
    }
    // FP32 absorber-only batches (the emission and limb-chord hot path) have variants compiled for
    // 6 and 8 resident 128-thread blocks per SM (register caps 80 and 64); blocks_per_sm selects them.
    // FP32 scattering batches: 5 and 6 blocks (register caps 102 and 85).
    if constexpr (sizeof(real) == 4 && SCAT) {
        if (block <= 128 && blocks_per_sm >= 6)
            return persistent_run<real, SCAT, 6, 0>(block, blocks_per_sm, nsm, grids, jobs, n_jobs, total_items, chunk,
                                                 interval, refill_min, one_grid, tab_n, work, st);
        if (block <= 128 && blocks_per_sm == 5)
            return persistent_run<real, SCAT, 5, 0>(block, blocks_per_sm, nsm, grids, jobs, n_jobs, total_items, chunk,
                                                 interval, refill_min, one_grid, tab_n, work, st);
    }
    if constexpr (sizeof(real) == 4 && !SCAT) {
        if (block <= 128 && blocks_per_sm >= 8)
            return persistent_run<real, SCAT, 8, 0>(block, blocks_per_sm, nsm, grids, jobs, n_jobs, total_items, chunk,
                                                 interval, refill_min, one_grid, tab_n, work, st);
        if (block <= 128 && blocks_per_sm >= 6)
            return persistent_run<real, SCAT, 6, 0>(block, blocks_per_sm, nsm, grids, jobs, n_jobs, total_items, chunk,
                                                 interval, refill_min, one_grid, tab_n, work, st);
    }
    return persistent_run<real, SCAT, 0, 0>(block, blocks_per_sm, nsm, grids, jobs, n_jobs, total_items, chunk,
                                                interval, refill_min, one_grid, tab_n, work, st);
}

cudaError_t launch_serve(bool ext, const DevGrid *grids, const ServeQueue &q, int block, int blocks_per_sm, int chunk,
                         int interval,
                         int refill_min, int tab_n, int idle_polls, int *grid_blocks, cudaStream_t st)
{
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (block != 128) return cudaErrorInvalidValue;
    if (interval < 1) interval = 1;
    refill_min = refill_min < 1 ? 1 : refill_min > 32 ? 32 : refill_min;
    // the plain variant, or every optional physics (band jobs are not served)
    auto kern = ext ? k_transport_serve<float, true, FEAT_EXT | FEAT_CABS> : k_transport_serve<float, true, 0>;
    const size_t sm = transport_smem(block) + (size_t)tab_n * sizeof(float2) * (block / 32);
    if (sm > 48 * 1024) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, block, sm);
    if (occ < 1) return cudaErrorInvalidConfiguration;
    // default: one block per SM less than fits, so that the cell-table kernels of newly admitted jobs
    // run beside the serving kernel
    if (blocks_per_sm <= 0) blocks_per_sm = occ > 1 ? occ - 1 : 1;
    if (blocks_per_sm > occ) blocks_per_sm = occ;
    *grid_blocks = nsm * blocks_per_sm;
    count_launch(1);
    kern<<<(unsigned)(nsm * blocks_per_sm), block, sm, st>>>(grids, q, chunk, interval, refill_min, tab_n, idle_polls);
    return cudaGetLastError();
}

cudaError_t launch_persistent(int precision, bool scatter, int feat, const DevGrid *grids, const DevJob *jobs, int n_jobs,
                              int64_t total_items, int chunk, int block, int blocks_per_sm, int interval, int refill_min,
                              int one_grid, int tab_n, unsigned long long *work, cudaStream_t st)
{
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (block <= 0) block = 128;
    if (block > 256 || block % 32) return cudaErrorInvalidValue;
    if (interval < 1) interval = 1;
    refill_min = refill_min < 1 ? 1 : refill_min > 32 ? 32 : refill_min;
    count_launch(1);
    if (precision == GCMC_FP64) {
        if (scatter)
            return persistent_dispatch<double, true>(block, blocks_per_sm, nsm, grids, jobs, n_jobs, total_items, chunk,
                                                     interval, refill_min, one_grid, tab_n, work, feat, st);
        return persistent_dispatch<double, false>(block, blocks_per_sm, nsm, grids, jobs, n_jobs, total_items, chunk,
                                                  interval, refill_min, one_grid, tab_n, work, feat, st);
    }
    if (scatter)
        return persistent_dispatch<float, true>(block, blocks_per_sm, nsm, grids, jobs, n_jobs, total_items, chunk,
                                                interval, refill_min, one_grid, tab_n, work, feat, st);
    return persistent_dispatch<float, false>(block, blocks_per_sm, nsm, grids, jobs, n_jobs, total_items, chunk,
                                             interval, refill_min, one_grid, tab_n, work, feat, st);
}

}  // namespace gcmc
