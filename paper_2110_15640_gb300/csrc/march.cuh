// march.cuh -- the cell-by-cell ray march through the spherical grid (hot loops 1-3), the packet
// launch geometry and the scattering samplers, templated on the arithmetic type.
//
// Every straight ray is written x(s) = c0 + s d with c0 its point of closest approach to the planet
// centre (c0 . d = 0, |c0| = p) and s the signed distance from c0.  In that frame
//   radial shell r:          s = -/+ sqrt(r^2 - p^2)
//   latitude cone sin(th)=S: (dz^2 - S^2) s^2 + 2 (zc dz) s + (zc^2 - S^2 p^2) = 0, disc = S^2 p^2 (Q - S^2),
//                            Q = dz^2 + (zc/p)^2, valid on the nappe where z has the sign of S;
//                            for dz = 0 (a ray parallel to the equatorial plane) s = -/+ (p/|S|) sqrt(Q - S^2)
//   equator plane:           s = -zc / dz
//   longitude half-plane:    s = -(n . c0) / (n . d), n = (-sin phi, cos phi, 0), on the phi side
// Along a straight line the radius is convex in s, the azimuth is monotone (sign of (o x d)_z) and
// the latitude has at most one extremum (sign of dz p^2 - zc s), so a cell has one candidate exit
// per face family: one shell, usually one cone, and one half-plane.  Each family's next crossing
// depends only on the ray and the cell index of that family (k, j or i), so it stays valid while
// the ray crosses faces of the other families: the march keeps the cone and half-plane crossings (and
// the cell index after each) and evaluates one again only once the ray has reached it (the family just
// crossed, or an exact tie); the shell crossing is short and is evaluated at every step.  In FP32 the
// impact parameter p^2 is carried as an unevaluated FP32 pair built with error-free products, so
// r^2 - p^2 keeps ~48 bits near grazing incidence; cone roots within TAN_EPS of tangency are recomputed
// in FP64.
#pragma once
#include "common.cuh"

namespace gcmc {

template <typename real> struct Ray {
    real cx, cy, cz;        // closest-approach point c0
    real dx, dy, dz;        // unit direction
    real s;                 // current position along the ray
    real p2hi, p2lo;        // |c0|^2 = p^2 as hi + lo
    real p, chz, Q;         // p, zc / p, dz^2 + chz^2
    real crz;               // (o x d)_z: sign gives the direction of azimuthal motion
    real B, dz2;            // zc dz and dz^2 (cone coefficients that depend on the ray only)
    real tau, tau_target;   // accumulated optical depth; interaction target (< 0: none)
    real tau2;              // continuous absorption: absorption optical depth along a flight
    real tl, tn;            // next crossing of the latitude and longitude family (s); at or behind s:
                            // to be evaluated again (-inf on a new ray)
    int lj, li;             // j after that cone crossing, i after that half-plane crossing (wrapped)
    int i, j, k;            // current cell
};

// error-free product a*b = hi + lo
// (the _rn intrinsics are never contracted into FMAs, which would break the error-free forms)
__device__ __forceinline__ void two_prod(float a, float b, float &hi, float &lo)
{
    hi = __fmul_rn(a, b);
    lo = __fmaf_rn(a, b, -hi);
}
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// (a*b - c*d) as an FP32 pair
__device__ __forceinline__ void diff_prod(float a, float b, float c, float d, float &hi, float &lo)
{
    float p1, e1, p2, e2;
    two_prod(a, b, p1, e1);
    two_prod(c, d, p2, e2);
    float s, e;
    two_sum(p1, -p2, s, e);
    e = __fadd_rn(e, __fsub_rn(e1, e2));
    hi = __fadd_rn(s, e);
    lo = __fsub_rn(e, __fsub_rn(hi, s));
}

// square of a pair, accumulated into (H, L)
__device__ __forceinline__ void add_sq(float hi, float lo, float &H, float &L)
{
    float q, qe;
    two_prod(hi, hi, q, qe);
    qe = __fmaf_rn(2.0f * hi, lo, qe);
    float s, e;
    two_sum(H, q, s, e);
    L = __fadd_rn(L, __fadd_rn(e, qe));
    H = s;
}

template <typename real>
__device__ __forceinline__ void ray_setup(Ray<real> &R, real ox, real oy, real oz, real dx, real dy, real dz)
{
    const real inv = M<real>::rsqrt_(dx * dx + dy * dy + dz * dz);
    dx *= inv;
    dy *= inv;
    dz *= inv;
    const real bo = ox * dx + oy * dy + oz * dz;
    R.dx = dx;
    R.dy = dy;
    R.dz = dz;
    R.cx = ox - bo * dx;
    R.cy = oy - bo * dy;
    R.cz = oz - bo * dz;
    R.s = bo;
    if constexpr (sizeof(real) == 4) {
        // p^2 = |o x d|^2 as an FP32 pair
        float ah, al, bh, bl, ch, cl;
        diff_prod(oy, dz, oz, dy, ah, al);
        diff_prod(oz, dx, ox, dz, bh, bl);
        diff_prod(ox, dy, oy, dx, ch, cl);
        float H = 0.0f, L = 0.0f;
        add_sq(ah, al, H, L);
        add_sq(bh, bl, H, L);
        add_sq(ch, cl, H, L);
        const float hi = __fadd_rn(H, L);
        R.p2hi = hi;
        R.p2lo = __fsub_rn(L, __fsub_rn(hi, H));
        R.crz = ch;
    } else {
        const double ax = oy * dz - oz * dy, ay = oz * dx - ox * dz, az = ox * dy - oy * dx;
        R.p2hi = ax * ax + ay * ay + az * az;
        R.p2lo = 0.0;
        R.crz = az;
    }
    R.p = M<real>::sqrt_(R.p2hi);
    R.chz = R.p > (real)0 ? M<real>::div_(R.cz, R.p) : (real)0;
    R.Q = dz * dz + R.chz * R.chz;
    R.B = R.cz * dz;
    R.dz2 = dz * dz;
    R.tl = -M<real>::inf();
    R.tn = -M<real>::inf();
    R.lj = 0;
    R.li = 0;
}

constexpr double TAN_EPS_CONE = 1e-5;

// the cone roots on the valid nappe in FP64, recomputed from the FP32 ray near tangency;
// returns the number of roots written to r[]
__device__ __noinline__ int cone_roots64(double cx, double cy, double cz, double dx, double dy, double dz, double S,
                                         double S2, double *r)
{
    if (S == 0.0) {   // equator plane z = 0
        if (dz == 0.0) return 0;
        r[0] = -cz / dz;
        return 1;
    }
    const double p2 = cx * cx + cy * cy + cz * cz;
    const double A = dz * dz - S2;
    const double B = cz * dz;
    const double C = cz * cz - S2 * p2;
    const double disc = B * B - A * C;
    if (disc < 0.0) return 0;
    const double sq = sqrt(disc);
    const double q = -(B + copysign(sq, B));
    double t[2];
    int m = 0, n = 0;
    if (q != 0.0) {
        t[m++] = q / A;
        t[m++] = C / q;
    } else {
        t[m++] = 0.0;
    }
    for (int i = 0; i < m; ++i) {
        const double z = cz + t[i] * dz;
        if (S > 0 ? z > 0.0 : z < 0.0) r[n++] = t[i];
    }
    return n;
}

// smallest root > smin of latitude edge e on its valid nappe (the equator edge is the plane z = 0);
// +inf if none.  Straight-line code: every lane of a warp runs the same instructions.
template <typename real>
__device__ __forceinline__ real cone_root(const DevGrid &G, const Tabs<real> &T, const Ray<real> &R, int e, real smin)
{
    const real inf = M<real>::inf();
    const auto sp = T.sl[e];
    const real S = sp.x, S2 = sp.y;
    const real A = R.dz2 - S2;
    const real dn = R.Q - S2;                       // disc = S^2 p^2 (Q - S^2)
    if constexpr (sizeof(real) == 4) {
        if (dn >= (real)0 && (dn < (real)TAN_EPS_CONE || fabsf(A) < (real)TAN_EPS_CONE)) {
            // near tangency: roots in FP64 from the FP32 ray; validity is decided on the rounded
            // root, the same test as every other face, so a face just crossed is never taken again
            double r[2];
            const int m = cone_roots64(R.cx, R.cy, R.cz, R.dx, R.dy, R.dz, __ldg(G.slat + e), __ldg(G.s2lat + e), r);
            real best = inf;
            for (int i = 0; i < m; ++i) {
                const real rf = (real)r[i];
                if (rf > smin && rf < best) best = rf;
            }
            return best;
        }
    }
    const real B = R.B;
    const real C = R.p2hi * ((R.chz - S) * (R.chz + S));
    const real sq = fabs(S) * R.p * M<real>::sqrt_(fmax(dn, (real)0));
    const real q = -(B + copysign(sq, B));
    // the equator edge is the plane z = 0 with the single root -zc/dz (two rounded copies of one root
    // could otherwise re-cross the plane at zero length)
    const bool eq = S == (real)0;
    const real r1 = eq ? M<real>::div_(-R.cz, R.dz) : M<real>::div_(q, A);
    const real r2 = M<real>::div_(C, q);
    const real z1 = R.cz + r1 * R.dz, z2 = R.cz + r2 * R.dz;
    // a root counts on the nappe whose z has the sign of S
    const bool ok = dn >= (real)0 && q != (real)0;
    const bool v1 = (eq ? R.dz != (real)0 : ok && z1 * S > (real)0) && r1 > smin;
    const bool v2 = !eq && ok && z2 * S > (real)0 && r2 > smin;
    const real a1 = v1 ? r1 : inf, a2 = v2 ? r2 : inf;
    return a1 < a2 ? a1 : a2;
}

// Rays parallel to the equatorial plane (dz = 0: every peel-off and limb chord towards an observer in that
// plane) keep z = zc, so |sin(lat)| = |zc| / sqrt(p^2 + s^2), largest at s = 0.  Edge S (on the nappe where
// z has the sign of S) is met where p^2 + s^2 = zc^2 / S^2, at s = -/+ t with t = (p / |S|) sqrt(Q - S^2),
// Q = (zc / p)^2, and not at all when Q <= S^2.  Smallest such root > R.s of edge e, +inf if none; in FP32
// within TAN_EPS of tangency the roots are recomputed in FP64, as for any cone.
template <typename real>
__device__ __forceinline__ real flat_cone_root(const DevGrid &G, const Tabs<real> &T, const Ray<real> &R, int e)
{
    const real inf = M<real>::inf();
    const auto sp = T.sl[e];
    const real S = sp.x, S2 = sp.y;
    const real dn = R.Q - S2;
    if constexpr (sizeof(real) == 4) {
        if (dn >= (real)0 && dn < (real)TAN_EPS_CONE) {
            double r[2];
            const int m = cone_roots64(R.cx, R.cy, R.cz, R.dx, R.dy, R.dz, __ldg(G.slat + e), __ldg(G.s2lat + e), r);
            real best = inf;
            for (int i = 0; i < m; ++i) {
                const real rf = (real)r[i];
                if (rf > R.s && rf < best) best = rf;
            }
            return best;
        }
    }
    const real t = M<real>::div_(R.p * M<real>::sqrt_(fmax(dn, (real)0)), fabs(S));
    const real a = -t > R.s ? -t : t > R.s ? t : inf;
    return dn > (real)0 && R.cz * S > (real)0 ? a : inf;
}

// the closed-form root of flat_cone_root away from tangency, for an edge (S, S^2) with dn = Q - S^2;
// straight-line code
template <typename real>
__device__ __forceinline__ real flat_root(const Ray<real> &R, typename Pair<real>::type sp, real dn, bool has)
{
    const real t = M<real>::div_(R.p * M<real>::sqrt_(fmax(dn, (real)0)), fabs(sp.x));
    const real a = -t > R.s ? -t : t > R.s ? t : M<real>::inf();
    return has && dn > (real)0 && R.cz * sp.x > (real)0 ? a : M<real>::inf();
}

// Latitude exit of a ray parallel to the equatorial plane: the nearer crossing of the band's two edges
// (the poles are not surfaces); dj the change of j there.  Both edges in straight-line code; only when
// one of them lies within TAN_EPS of tangency (FP32) is it evaluated as flat_cone_root does.
template <typename real>
__device__ __forceinline__ real lat_exit_flat(const DevGrid &G, const Tabs<real> &T, const Ray<real> &R, int &dj)
{
    const real inf = M<real>::inf();
    const bool has_lo = R.j > 0, has_hi = R.j + 1 < T.nlat;
    const auto lo = T.sl[R.j], hi = T.sl[R.j + 1];
    const real dnl = R.Q - lo.y, dnh = R.Q - hi.y;
    real tlo, thi;
    if constexpr (sizeof(real) == 4) {
        const bool nl = has_lo && dnl >= (real)0 && dnl < (real)TAN_EPS_CONE;
        const bool nh = has_hi && dnh >= (real)0 && dnh < (real)TAN_EPS_CONE;
        if (nl || nh) {
            tlo = has_lo ? flat_cone_root<real>(G, T, R, R.j) : inf;
            thi = has_hi ? flat_cone_root<real>(G, T, R, R.j + 1) : inf;
            dj = thi < tlo ? 1 : -1;
            return thi < tlo ? thi : tlo;
        }
    }
    tlo = flat_root<real>(R, lo, dnl, has_lo);
    thi = flat_root<real>(R, hi, dnh, has_hi);
    dj = thi < tlo ? 1 : -1;
    return thi < tlo ? thi : tlo;
}

// Latitude exit of the current cell.  Along the line, f(s) = sin(lat) = (zc + s dz) / sqrt(p^2 + s^2)
// has f' of the sign of g(s) = dz p^2 - s zc, so a single extremum, f = sign(zc) sqrt(Q), at
// g = 0, and the limits -dz, +dz at s -> -inf, +inf.  Moving up (g > 0) the ray crosses the upper
// edge S_hi iff the supremum of f ahead exceeds it (sqrt(Q) if the maximum lies ahead, i.e. zc > 0,
// else dz); failing that, after the maximum it crosses the lower edge iff dz < S_lo; the upper
// crossing always comes first.  Moving down mirrors this.  So one cone is evaluated per step, with
// the same root and validity rules as before; when Q or dz lies within TAN_EPS of an edge's S^2 or S
// (the boundaries of the choice, which are also the tangency cases) both cones are evaluated.
template <typename real>
__device__ __forceinline__ real lat_exit(const DevGrid &G, const Tabs<real> &T, const Ray<real> &R, int &dj)
{
    if (R.dz == (real)0) return lat_exit_flat<real>(G, T, R, dj);
    const real inf = M<real>::inf();
    const bool has_lo = R.j > 0, has_hi = R.j + 1 < T.nlat;
    // the poles are not surfaces: sentinels outside [-1, 1] make them unreachable below
    const real Slo = has_lo ? T.sl[R.j].x : (real)-2;
    const real Shi = has_hi ? T.sl[R.j + 1].x : (real)2;
    const real dz = R.dz, Q = R.Q;
    const real eps = sizeof(real) == 4 ? (real)TAN_EPS_CONE : (real)1e-12;
    const bool amb = fabs(Q - Shi * Shi) < eps || fabs(Q - Slo * Slo) < eps || fabs(dz - Shi) < eps ||
                     fabs(dz - Slo) < eps;
    if (amb) {
        const real tlo = has_lo ? cone_root<real>(G, T, R, R.j, R.s) : inf;
        const real thi = has_hi ? cone_root<real>(G, T, R, R.j + 1, R.s) : inf;
        dj = thi < tlo ? 1 : -1;
        return thi < tlo ? thi : tlo;
    }
    const real g = dz * R.p2hi - R.s * R.cz;
    const bool up = g > (real)0 || (g == (real)0 && R.cz < (real)0);
    const bool ext_ahead = up ? R.cz > (real)0 : R.cz < (real)0;
    bool to_hi, to_lo;
    if (up) {
        to_hi = ext_ahead ? (Shi <= (real)0 || Q > Shi * Shi) : dz > Shi;
        to_lo = !to_hi && ext_ahead && dz < Slo;
    } else {
        to_lo = ext_ahead ? (Slo >= (real)0 || Q > Slo * Slo) : dz < Slo;
        to_hi = !to_lo && ext_ahead && dz > Shi;
    }
    const real t = cone_root<real>(G, T, R, to_hi ? R.j + 1 : R.j, R.s);
    dj = to_hi ? 1 : -1;
    return (to_hi || to_lo) ? t : inf;
}

// Radial family: inward (s < 0) and still outside the inner shell -> inner root, else outer root;
// dk the change of k at that crossing.
template <typename real>
__device__ __forceinline__ real radial_exit(const Tabs<real> &T, const Ray<real> &R, int &dk)
{
    const auto ri = T.r2[R.k], ro = T.r2[R.k + 1];
    const real hin = (ri.x - R.p2hi) + (ri.y - R.p2lo);
    const real hout = (ro.x - R.p2hi) + (ro.y - R.p2lo);
    const bool inward = R.s < (real)0 && hin > (real)0;
    const real h = inward ? hin : fmax(hout, (real)0);
    const real rt = M<real>::sqrt_(h);
    dk = inward ? -1 : 1;
    return inward ? -rt : rt;
}

// Longitude family: the azimuth along a line is monotone (sign of (o x d)_z), so only the edge ahead
// counts; +inf if the ray does not reach it; di the change of i at that crossing.
template <typename real>
__device__ __forceinline__ real lon_exit(const Tabs<real> &T, const Ray<real> &R, int &di)
{
    const bool east = R.crz > (real)0;
    const auto cs = T.cs[east ? R.i + 1 : R.i];
    const real nd = R.dy * cs.x - R.dx * cs.y;
    const real sr = M<real>::div_(-(R.cy * cs.x - R.cx * cs.y), nd);
    const bool lon_ok = T.nlon > 1 && R.crz != (real)0 && nd != (real)0 && sr > R.s &&
                        cs.x * (R.cx + sr * R.dx) + cs.y * (R.cy + sr * R.dy) > (real)0;
    di = east ? 1 : -1;
    return lon_ok ? sr : M<real>::inf();
}

// Exit of the current cell: the s of the exit point; to_lat / to_lon tell a cone (j becomes R.lj) or a
// half-plane (i becomes R.li) from a shell (k changes by dk).  A cone or half-plane crossing at or behind
// R.s (the family just crossed, or an exact tie that the order below gave to another family) is
// evaluated again first, its root at R.s no longer counting; ties go to the shell, then the cone, as if
// every family were evaluated at every step.
template <typename real>
__device__ __forceinline__ real cell_exit(const DevGrid &G, const Tabs<real> &T, Ray<real> &R, bool &to_lat,
                                          bool &to_lon, int &dk)
{
    // (not strictly ahead: also true for a ray whose position is not a number, so a family is never
    // taken without having been evaluated for the current ray)
    if (!(R.tl > R.s)) {
        int dj;
        R.tl = lat_exit<real>(G, T, R, dj);
        R.lj = R.j + dj;
    }
    if (!(R.tn > R.s)) {
        int di;
        R.tn = lon_exit<real>(T, R, di);
        const int ni = R.i + di;
        R.li = ni < 0 ? T.nlon - 1 : ni == T.nlon ? 0 : ni;
    }
    const real sr = radial_exit<real>(T, R, dk);
    to_lat = R.tl < sr;
    const real b = to_lat ? R.tl : sr;
    to_lon = R.tn < b;
    return to_lon ? R.tn : b;
}

// Cross the exit that cell_exit chose: update the cell; returns E_CONT, or E_ESCAPE / E_BOTTOM (the cell
// is left unchanged) for a shell crossing out of the grid.
template <typename real, class GT>
__device__ __forceinline__ int cross_face(const GT &G, Ray<real> &R, bool to_lat, bool to_lon, int dk)
{
    const bool shell = !(to_lat || to_lon);
    const int nk = R.k + dk;
    const bool in = (unsigned)nk < (unsigned)G.nr;
    R.k = shell && in ? nk : R.k;
    R.j = to_lat && !to_lon ? R.lj : R.j;
    R.i = to_lon ? R.li : R.i;
    return shell && !in ? (nk < 0 ? E_BOTTOM : E_ESCAPE) : E_CONT;
}

// ------------------------------------------------------------------ samplers (Sect. 3)
template <typename real> __device__ __forceinline__ real sample_rayleigh(real z)
{
    // exact inverse CDF of 3/8 (1 + mu^2): mu^3 + 3 mu = 8 z - 4
    const real q = (real)4 * z - (real)2;
    const real u = M<real>::cbrt_(q + M<real>::sqrt_(q * q + (real)1));
    return u - M<real>::div_((real)1, u);
}

template <typename real> __device__ __forceinline__ real sample_hg(real g, real z, real eps)
{
    if (fabs(g) < eps) return (real)2 * z - (real)1;
    const real a = M<real>::div_((real)1 - g * g, (real)1 - g + (real)2 * g * z);
    real mu = M<real>::div_((real)1 + g * g - a * a, (real)2 * g);
    mu = mu > (real)1 ? (real)1 : mu;
    mu = mu < (real)-1 ? (real)-1 : mu;
    return mu;
}

// Henyey-Greenstein phase function, normalised to 2 over mu in [-1, 1]
template <typename real> __device__ __forceinline__ real phase_hg(real mu, real g)
{
    const real den = (real)1 + g * g - (real)2 * g * mu;
    return ((real)1 - g * g) * M<real>::rsqrt_(den) * M<real>::div_((real)1, den);
}

// two-term HG of one asymmetry g (Sect. 3): terms g1 = g, g2 = -g/2, weight a = 1 - g2^2 on the first
template <typename real> __device__ __forceinline__ void tthg_terms(real g, real &g2, real &a)
{
    g2 = (real)-0.5 * g;
    a = (real)1 - g2 * g2;
}

// probability per steradian of scattering by angle acos(mu): (P_gas P_Ray + (1 - P_gas) P_cloud) / (4 pi),
// P_cloud the HG function, or the two-term HG when tthg is set
template <typename real> __device__ __forceinline__ real theta_mix(real mu, real pg, real g, bool tthg = false)
{
    const real pr = (real)0.75 * ((real)1 + mu * mu);
    real pc = phase_hg<real>(mu, g);
    if (tthg) {
        real g2, a;
        tthg_terms<real>(g, g2, a);
        pc = a * pc + ((real)1 - a) * phase_hg<real>(mu, g2);
    }
    return (pg * pr + ((real)1 - pg) * pc) * (real)(1.0 / (4.0 * PI));
}

// direction at polar angle acos(mu), azimuth psi about d (azimuth origin as in the standard
// e1 = (dx dz, dy dz, -(1 - dz^2)) / sqrt(1 - dz^2), e2 = (-dy, dx, 0) / sqrt(1 - dz^2) frame)
template <typename real>
__device__ __forceinline__ void turn(real &dx, real &dy, real &dz, real mu, real psi)
{
    real sp, cp;
    M<real>::sincos_(psi, &sp, &cp);
    const real s = M<real>::sqrt_(fmax((real)0, (real)1 - mu * mu));
    real nx, ny, nz;
    if (fabs(dz) < (real)0.99999) {
        const real den = M<real>::sqrt_((real)1 - dz * dz);
        const real id = M<real>::div_((real)1, den);
        nx = mu * dx + s * (cp * dx * dz * id - sp * dy * id);
        ny = mu * dy + s * (cp * dy * dz * id + sp * dx * id);
        nz = mu * dz - s * cp * den;
    } else {
        nx = s * cp;
        ny = s * sp;
        nz = (dz > (real)0 ? (real)1 : (real)-1) * mu;
    }
    const real inv = M<real>::rsqrt_(nx * nx + ny * ny + nz * nz);
    dx = nx * inv;
    dy = ny * inv;
    dz = nz * inv;
}

// latitude / longitude bins of a point (radial index known)
template <typename real>
__device__ __forceinline__ void locate_angles(const DevGrid &G, real x, real y, real z, int &i, int &j)
{
    const real lat = M<real>::atan2_(z, M<real>::sqrt_(x * x + y * y));
    real lon = M<real>::atan2_(y, x);
    const real lo0 = (real)G.lon0;
    const real two_pi = (real)(2.0 * PI);
    while (lon < lo0) lon += two_pi;
    while (lon >= lo0 + two_pi) lon -= two_pi;
    const real *lat_t = tab_lat<real>(G);
    const real *lon_t = tab_lon<real>(G);
    int jj = 0;
    while (jj < G.nlat - 1 && lat >= __ldg(lat_t + jj + 1)) ++jj;
    int ii = 0;
    // binary search over longitude edges
    int lo = 0, hi = G.nlon - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(lon_t + mid) <= lon) lo = mid; else hi = mid - 1;
    }
    ii = lo;
    i = ii;
    j = jj;
}

}  // namespace gcmc
