"""Seeded synthetic initial conditions (host, numpy).

These generators produce the input particle sets only; they hold none of the
method's arithmetic (no forces, keys, trees or cut-offs), so the CUDA path and
the CPU oracle can both be fed from them.

* ``plummer`` -- Plummer (1911) sphere sampled as in Aarseth, Henon & Wielen
  (1974): radius from the inverted cumulative mass, speed by von Neumann
  rejection on q^2 (1 - q^2)^(7/2), isotropic directions; shifted to the
  centre-of-mass frame and scaled to N-body (Heggie) units, G = M = 1,
  E = -1/4 (length scale 3 pi / 16), equal masses 1/N.  The cumulative mass
  fraction is capped at ``x_max`` (0.999) to keep the extreme tail finite.
* ``king`` -- King (1966) model with central potential W0: the lowered
  isothermal distribution function, the Poisson equation integrated with
  RK4 in FP64; radii from the cumulative mass, speeds by rejection from the
  lowered Maxwellian; scaled to N-body units with the model's own energy.
* ``salpeter_masses`` -- dN/dm ~ m^-2.35 on [m_lo, m_hi] by inverse CDF,
  normalised to total mass 1.
"""
from __future__ import annotations

import math

import numpy as np


def _isotropic(rng, n):
    u = rng.uniform(-1.0, 1.0, n)
    phi = rng.uniform(0.0, 2.0 * math.pi, n)
    s = np.sqrt(1.0 - u * u)
    return np.stack([s * np.cos(phi), s * np.sin(phi), u], axis=0)


def plummer(n: int, seed: int, x_max: float = 0.999):
    """Returns (pos (3, n), vel (3, n), mass (n,)) in N-body units, FP64."""
    rng = np.random.default_rng(seed)
    x = rng.uniform(0.0, x_max, n)
    x = np.where(x == 0.0, x_max * 1e-12, x)
    r = 1.0 / np.sqrt(x ** (-2.0 / 3.0) - 1.0)
    pos = _isotropic(rng, n) * r
    # speed fraction q with density q^2 (1 - q^2)^(7/2): rejection, max 0.1
    q = np.empty(n)
    todo = np.arange(n)
    while todo.size:
        qq = rng.uniform(0.0, 1.0, todo.size)
        gg = rng.uniform(0.0, 0.1, todo.size)
        ok = gg < qq * qq * (1.0 - qq * qq) ** 3.5
        q[todo[ok]] = qq[ok]
        todo = todo[~ok]
    ve = math.sqrt(2.0) * (1.0 + r * r) ** -0.25
    vel = _isotropic(rng, n) * (q * ve)
    mass = np.full(n, 1.0 / n)
    pos -= pos.mean(axis=1, keepdims=True)
    vel -= vel.mean(axis=1, keepdims=True)
    lscale = 3.0 * math.pi / 16.0
    pos *= lscale
    vel /= math.sqrt(lscale)
    return pos, vel, mass


def salpeter_masses(n: int, seed: int, m_lo=0.1, m_hi=10.0, alpha=2.35):
    rng = np.random.default_rng(seed)
    u = rng.uniform(0.0, 1.0, n)
    a = 1.0 - alpha
    m = (m_lo ** a + u * (m_hi ** a - m_lo ** a)) ** (1.0 / a)
    return m / m.sum()


def _king_profile(W0: float):
    """Integrates the King (1966) Poisson equation in King units (core radius
    1, velocity scale sigma = 1, G = 1, central density 9 / (4 pi)):
        W'' + (2 / r) W' = -9 rho(W) / rho(W0),
        rho(W) ~ exp(W) erf(sqrt W) - sqrt(4 W / pi) (1 + 2 W / 3),
    with RK4 steps of 10^-3 in ln r from the centre to the tidal radius
    (W = 0).  Returns r, W(r), M(<r) = -r^2 W'(r)."""
    from math import erf, exp, pi, sqrt

    def rho(W):
        if W <= 0.0:
            return 0.0
        return exp(W) * erf(sqrt(W)) - sqrt(4.0 * W / pi) * (1.0 + 2.0 * W / 3.0)

    rho0 = rho(W0)

    def f(r, y):
        W, dW = y
        return (dW, -9.0 * rho(W) / rho0 - 2.0 * dW / r)

    r = 1e-4
    y = (W0 - 1.5 * r * r, -3.0 * r)  # series about the centre
    rs, Ws, Ms = [0.0, r], [W0, y[0]], [0.0, -r * r * y[1]]
    while y[0] > 0.0 and r < 1e5:
        h = 1e-3 * r
        k1 = f(r, y)
        k2 = f(r + h / 2, (y[0] + h / 2 * k1[0], y[1] + h / 2 * k1[1]))
        k3 = f(r + h / 2, (y[0] + h / 2 * k2[0], y[1] + h / 2 * k2[1]))
        k4 = f(r + h, (y[0] + h * k3[0], y[1] + h * k3[1]))
        yn = (y[0] + h / 6 * (k1[0] + 2 * k2[0] + 2 * k3[0] + k4[0]),
              y[1] + h / 6 * (k1[1] + 2 * k2[1] + 2 * k3[1] + k4[1]))
        rn = r + h
        if yn[0] <= 0.0:
            t = y[0] / (y[0] - yn[0])
            rn = r + t * h
            yn = (0.0, y[1] + t * (yn[1] - y[1]))
        rs.append(rn)
        Ws.append(yn[0])
        Ms.append(-rn * rn * yn[1])
        r, y = rn, yn
    return np.array(rs), np.array(Ws), np.array(Ms)


def king(n: int, seed: int, W0: float = 9.0, masses=None):
    """King (1966) model; returns (pos (3, n), vel (3, n), mass (n,)) in
    N-body units: total mass 1, G = 1 and E = -1/4 with the energy taken from
    the smooth model (virial: E = U / 2, U = -int M(<r) dM / r)."""
    rng = np.random.default_rng(seed)
    r_t, W_t, M_t = _king_profile(W0)
    Mtot = float(M_t[-1])
    u = rng.uniform(0.0, Mtot, n)
    r = np.interp(u, M_t, r_t)
    W = np.interp(r, r_t, W_t)
    pos = _isotropic(rng, n) * r
    # speed density ~ v^2 (exp(W - v^2 / 2) - 1) on [0, sqrt(2W)] (sigma = 1)
    v = np.zeros(n)
    todo = np.nonzero(W > 0.0)[0]
    while todo.size:
        Wt = W[todo]
        vmax = np.sqrt(2.0 * Wt)
        vv = rng.uniform(0.0, 1.0, todo.size) * vmax
        fv = vv * vv * np.expm1(Wt - 0.5 * vv * vv)
        fmax = vmax * vmax * np.expm1(Wt)
        ok = rng.uniform(0.0, 1.0, todo.size) * fmax < fv
        v[todo[ok]] = vv[ok]
        todo = todo[~ok]
    vel = _isotropic(rng, n) * v
    mass = np.full(n, 1.0 / n) if masses is None else np.asarray(masses, float)
    mass = mass / mass.sum()
    pos -= (pos * mass).sum(axis=1, keepdims=True)
    vel -= (vel * mass).sum(axis=1, keepdims=True)
    dM = np.diff(M_t)
    rm = 0.5 * (r_t[1:] + r_t[:-1])
    Mm = 0.5 * (M_t[1:] + M_t[:-1])
    U = -float(np.sum(Mm * dM / rm))
    E = 0.5 * U
    # x' = a x, m' = m / Mtot, v' = v / sqrt(Mtot a): E' = E / (Mtot^2 a)
    a = -4.0 * E / (Mtot * Mtot)
    pos *= a
    vel /= math.sqrt(Mtot * a)
    return pos, vel, mass


def plummer_ensemble(n_clusters: int, seed: int, n_min: int = 1024,
                     n_max: int = 65536):
    """Independent Plummer clusters (each in N-body units, total mass 1,
    centred on the origin) of N_c = round(exp(U[ln n_min, ln n_max]))
    particles, cluster c seeded with seed + c.  Returns (pos (3, N),
    vel (3, N), mass (N,), offsets (n_clusters + 1,))."""
    rng = np.random.default_rng(seed)
    sizes = np.rint(np.exp(rng.uniform(math.log(n_min), math.log(n_max),
                                       n_clusters))).astype(np.int64)
    off = np.zeros(n_clusters + 1, np.int64)
    np.cumsum(sizes, out=off[1:])
    parts = [plummer(int(sz), seed + 1 + c) for c, sz in enumerate(sizes)]
    pos = np.concatenate([p[0] for p in parts], axis=1)
    vel = np.concatenate([p[1] for p in parts], axis=1)
    mass = np.concatenate([p[2] for p in parts])
    return pos, vel, mass, off
