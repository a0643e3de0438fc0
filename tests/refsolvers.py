"""Independent reference solutions used to pin the oracle (no Monte Carlo, no shared code).

* `hfunction`      Chandrasekhar's H-function for isotropic scattering, by iterating
                   1/H(mu) = sqrt(1 - w) + (w/2) int_0^1 mu' H(mu') / (mu + mu') dmu'.
* `AddingDoubling` plane-parallel, homogeneous slab reflection/transmission for a phase
                   function with a short Legendre expansion (isotropic, Rayleigh), azimuthal
                   Fourier modes m = 0..L, Gauss quadrature, thin-layer single scattering
                   initialisation and repeated doubling.
* `brute_segments` all intersections of a straight ray with every shell, latitude cone
                   (or the equator plane) and longitude half-plane of a spherical grid,
                   sorted, with each segment's cell found by binning its midpoint.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import lpmv, expn


def gauss01(n):
    x, w = np.polynomial.legendre.leggauss(n)
    return 0.5 * (x + 1.0), 0.5 * w


def hfunction(omega, n=200, iters=20000, tol=1e-15):
    mu, w = gauss01(n)
    H = np.ones(n)
    K = mu[None, :] * w[None, :] / (mu[:, None] + mu[None, :])
    for _ in range(iters):
        Hn = 1.0 / (math.sqrt(1.0 - omega) + 0.5 * omega * (K @ H))
        if np.max(np.abs(Hn - H)) < tol:
            H = Hn
            break
        H = Hn
    return mu, w, H


def ag_isotropic_semi_infinite(omega, n=200):
    """Geometric albedo of a sphere with a semi-infinite isotropic atmosphere:
    A_g = (w/4) int_0^1 H(mu)^2 mu dmu."""
    mu, w, H = hfunction(omega, n)
    return 0.25 * omega * np.sum(w * H * H * mu)


class AddingDoubling:
    """Reflection R^m(mu, mu0) and transmission T^m of a homogeneous slab.

    Conventions: a collimated beam of flux pi F0 at incidence cosine mu0 gives reflected
    intensity I_r(mu, phi) = mu0 F0 R(mu, mu0, phi - phi0), R = sum_m (2 - delta_m0) R^m cos(m dphi).
    The phase function is P(cos Theta) = sum_l beta_l P_l(cos Theta) with beta_0 = 1.
    """

    def __init__(self, beta, omega, tau, n=40, dtau0=2.0 ** -30):
        self.beta = np.asarray(beta, np.float64)
        self.omega = float(omega)
        self.tau = float(tau)
        self.mu, self.w = gauss01(n)
        self.n = n
        L = len(self.beta) - 1
        self.R = []
        self.T = []
        for m in range(L + 1):
            R, T = self._mode(m, dtau0)
            self.R.append(R)
            self.T.append(T)

    def _pm(self, m, x):
        L = len(self.beta) - 1
        out = np.zeros((L + 1, len(x)))
        for l in range(m, L + 1):
            out[l] = lpmv(m, l, x)
        return out

    def _mode(self, m, dtau0):
        mu, w, om = self.mu, self.w, self.omega
        L = len(self.beta) - 1
        c = np.array([math.factorial(l - m) / math.factorial(l + m) if l >= m else 0.0 for l in range(L + 1)])
        Pp = self._pm(m, mu)
        Pn = self._pm(m, -mu)
        coef = (self.beta * c)[:, None]
        Prefl = (Pp * coef).T @ Pn            # [i, j] : P^m(mu_i, -mu_j)
        Ptran = (Pp * coef).T @ Pp            # [i, j] : P^m(mu_i, mu_j)
        # number of doublings: start below dtau0, end exactly at tau
        nd = max(0, int(math.ceil(math.log2(self.tau / dtau0))))
        dt = self.tau / 2.0 ** nd
        MU, MU0 = np.meshgrid(mu, mu, indexing="ij")
        R1 = 0.25 * om * Prefl / (MU + MU0) * (-np.expm1(-dt * (1.0 / MU + 1.0 / MU0)))
        same = np.abs(MU - MU0) < 1e-14
        with np.errstate(divide="ignore", invalid="ignore"):
            T1 = 0.25 * om * Ptran / (MU - MU0) * (np.exp(-dt / MU) - np.exp(-dt / MU0))
        T1[same] = (0.25 * om * Ptran * dt / MU0 ** 2 * np.exp(-dt / MU0))[same]
        C = np.diag(mu * w)
        E = np.diag(np.exp(-dt / mu))
        Rop = 2.0 * R1 @ C
        Top = E + 2.0 * T1 @ C
        I = np.eye(self.n)
        for _ in range(nd):
            G = np.linalg.inv(I - Rop @ Rop)
            Rn = Rop + Top @ G @ Rop @ Top
            Tn = Top @ G @ Top
            Rop, Top = Rn, Tn
        Rm = Rop / (2.0 * (mu * w)[None, :])
        Td = (Top - np.diag(np.exp(-self.tau / mu))) / (2.0 * (mu * w)[None, :])
        return Rm, Td

    def refl(self, dphi):
        """R(mu_i, mu_j, dphi) on the quadrature nodes."""
        out = np.zeros((self.n, self.n))
        for m, Rm in enumerate(self.R):
            out += (1.0 if m == 0 else 2.0) * Rm * math.cos(m * dphi)
        return out

    def geometric_albedo(self):
        """Zero phase: emergent direction opposite to the incident one (mu = mu0, dphi = pi);
        A_g = 2 int_0^1 R(mu, mu, pi) mu^2 dmu (sphere of locally plane-parallel slabs)."""
        Rd = np.diag(self.refl(math.pi))
        return 2.0 * np.sum(self.w * Rd * self.mu ** 2)

    def plane_albedo(self):
        """Reflected / incident flux per incidence mu0 (m = 0 only)."""
        return 2.0 * (self.R[0] * (self.mu * self.w)[:, None]).sum(axis=0)

    def flux_transmission(self):
        return np.exp(-self.tau / self.mu) + 2.0 * (self.T[0] * (self.mu * self.w)[:, None]).sum(axis=0)


def emission_shell_Lp(B, tau, R):
    """Isothermal slab of vertical optical depth tau over a black, non-emitting sphere of radius R,
    scattering off: L_p = B * 2 pi R^2 int_0^1 (1 - exp(-tau/mu)) mu dmu = B 2 pi R^2 (1/2 - E3(tau))."""
    return B * 2.0 * math.pi * R * R * (0.5 - expn(3, tau))


def transmission_integral_uniform(alpha, R0, Rtoa):
    """2 int_R0^Rtoa (1 - exp(-2 alpha sqrt(Rtoa^2 - b^2))) b db for a uniform absorber."""
    s0 = math.sqrt(Rtoa * Rtoa - R0 * R0)
    a = 2.0 * alpha
    return s0 * s0 - 2.0 * (1.0 / a ** 2 - math.exp(-a * s0) * (s0 / a + 1.0 / a ** 2))


# --------------------------------------------------------------------------- brute force geometry

def _locate(grid, x):
    r = np.linalg.norm(x)
    lat = math.atan2(x[2], math.hypot(x[0], x[1]))
    lon = math.atan2(x[1], x[0])
    lo0 = grid.lon_edges[0]
    lon = (lon - lo0) % (2.0 * math.pi) + lo0
    k = int(np.searchsorted(grid.r_edges, r, side="right") - 1)
    j = int(np.clip(np.searchsorted(grid.lat_edges, lat, side="right") - 1, 0, grid.nlat - 1))
    i = int(np.clip(np.searchsorted(grid.lon_edges, lon, side="right") - 1, 0, grid.nlon - 1))
    return i, j, k


def brute_segments(grid, o, d):
    """Segments (flat cell index, length) of the ray o + t d, t > 0, until it leaves the top
    shell or meets the bottom shell.  Every crossing is enumerated analytically."""
    o = np.asarray(o, np.float64)
    d = np.asarray(d, np.float64)
    ts = []
    b = o @ d
    for r in grid.r_edges:
        disc = b * b - (o @ o - r * r)
        if disc >= 0:
            sq = math.sqrt(disc)
            ts += [-b - sq, -b + sq]
    for th in grid.lat_edges[1:-1]:
        if abs(th) < 1e-15:
            if d[2] != 0:
                ts.append(-o[2] / d[2])
            continue
        s2 = math.sin(th) ** 2
        A = d[2] ** 2 - s2
        B = o[2] * d[2] - s2 * b
        Cc = o[2] ** 2 - s2 * (o @ o)
        roots = []
        if abs(A) < 1e-300:
            roots = [-Cc / (2 * B)]
        else:
            disc = B * B - A * Cc
            if disc >= 0:
                sq = math.sqrt(disc)
                roots = [(-B - sq) / A, (-B + sq) / A]
        for t in roots:
            z = o[2] + t * d[2]
            if z * th > 0:
                ts.append(t)
    if grid.nlon > 1:
        for ph in grid.lon_edges[:-1]:
            c, s = math.cos(ph), math.sin(ph)
            nd = -s * d[0] + c * d[1]
            if nd != 0:
                t = -(-s * o[0] + c * o[1]) / nd
                if c * (o[0] + t * d[0]) + s * (o[1] + t * d[1]) > 0:
                    ts.append(t)
    ts = np.array(sorted(t for t in ts if t > 0.0))
    segs = []
    t0 = 0.0
    R0, Rt = grid.r_edges[0], grid.r_edges[-1]
    for t1 in ts:
        mid = o + 0.5 * (t0 + t1) * d
        rm = np.linalg.norm(mid)
        if rm >= Rt or rm <= R0:
            break
        i, j, k = _locate(grid, mid)
        segs.append(((k * grid.nlat + j) * grid.nlon + i, t1 - t0))
        t0 = t1
        end = o + t1 * d
        re = np.linalg.norm(end)
        if abs(re - R0) <= 1e-9 * R0 and (end @ d) < 0:
            break
    return segs
