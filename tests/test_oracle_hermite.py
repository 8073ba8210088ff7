"""Pins of the oracle's hard part (Sect. 2.1-2.2): F_hard over neighbour rows
and its jerk, and the fourth-order Hermite integrator with block timesteps.

* The neighbour-row hard force equals the direct hard sum over all pairs
  (rows hold every particle within h >= r_cut; pairs beyond r_cut weigh 0),
  and soft + hard is the Newtonian force (K + (1 - K) = 1, Eq. 7-9).
* The jerk equals central differences of the hard acceleration along the
  particles' straight-line motion.
* A Keplerian binary well inside r_in (K = 0, so the pair is fully hard)
  returns to its initial state after whole periods; the error falls by about
  2^4 when eta halves (fourth order).
* Energy of a compact softened cluster (all pairs hard) is conserved.
* Particles with empty rows drift, x + dt v, and particles whose neighbours
  all lie beyond r_cut move in straight lines.
* The block schedule does not depend on the unit of time: with time scaled
  by 2 (velocities halved, G quartered, dt_soft doubled; all exact in
  binary) the step gives the same positions and half the velocities, bit
  for bit.  This pins the dimension of every term of Eq. 18-20 (Eq. 18's
  denominator as printed, |a^(0)| |a^(3)|, fails it).
* The first level of a binary at pericentre is the one Eq. 20 gives with
  the closed-form acceleration and jerk of a Kepler orbit.
* The fused-order mirror of the GPU kernels stays within the oracle's own
  response to one-ulp input perturbations.
"""
import numpy as np
import pytest

import oracle

GAMMA = 0.1


def _cluster(n, seed, scale):
    rng = np.random.default_rng(seed)
    pos = rng.normal(size=(n, 3)) * scale
    vel = rng.normal(size=(n, 3)) * 0.3
    m = rng.uniform(0.5, 1.5, n) / n
    return pos, vel, m


def test_row_hard_force_equals_direct_hard_sum():
    pos, vel, m = _cluster(400, 1, 0.05)
    r_cut, eps = 0.03, 1e-3
    off, idx = oracle.neighbours(pos, 1.2 * r_cut)
    a, _ = oracle.hard_force(pos, vel, m, off, idx, eps=eps, r_cut=r_cut, gamma=GAMMA)
    d = oracle.direct(pos, m, eps=eps, r_cut=r_cut, gamma=GAMMA, kind="hard")
    scale = np.abs(d).max()
    assert np.abs(a - d).max() <= 1e-12 * scale
    assert np.count_nonzero(np.abs(d).sum(axis=1)) > 100  # most rows interact
    soft = oracle.direct(pos, m, eps=eps, r_cut=r_cut, gamma=GAMMA, kind="soft")
    newton = oracle.direct(pos, m, eps=eps, r_cut=r_cut, gamma=GAMMA, kind="newton")
    assert np.abs(a + soft - newton).max() <= 1e-12 * np.abs(newton).max()


def test_jerk_equals_finite_differences():
    pos, vel, m = _cluster(300, 2, 0.04)
    r_cut, eps = 0.03, 1e-3
    off, idx = oracle.neighbours(pos, 2.0 * r_cut)
    kw = dict(eps=eps, r_cut=r_cut, gamma=GAMMA)
    _, jk = oracle.hard_force(pos, vel, m, off, idx, **kw)
    dt = 1e-6
    ap, _ = oracle.hard_force(pos + dt * vel, vel, m, off, idx, **kw)
    am, _ = oracle.hard_force(pos - dt * vel, vel, m, off, idx, **kw)
    fd = (ap - am) / (2 * dt)
    # pairs crossing r_in or r_cut are included: K is C^3 there (Eq. 12)
    assert np.abs(jk - fd).max() <= 1e-6 * np.abs(jk).max()


def _binary(e, a=0.01, M=1.0):
    # relative orbit at pericentre, centre-of-mass frame, masses M/2 each
    rp = a * (1 - e)
    vp = np.sqrt(M * (1 + e) / rp)
    pos = np.array([[-rp / 2, 0, 0], [rp / 2, 0, 0]])
    vel = np.array([[0, -vp / 2, 0], [0, vp / 2, 0]])
    period = 2 * np.pi * np.sqrt(a ** 3 / M)
    return pos, vel, np.array([M / 2, M / 2]), period


def _kepler_error(eta, periods=2):
    pos, vel, m, period = _binary(0.5)
    off, idx = np.array([0, 1, 2]), np.array([1, 0], dtype=np.int32)
    p, v = pos, vel
    for _ in range(periods):  # one soft step per period
        p, v, st = oracle.hermite(p, v, m, off, idx, dt_soft=period, r_cut=1.0,
                                  gamma=GAMMA, eta=eta)
        assert st[3] == 0
    return np.abs(p - pos).max() / 0.01


def test_kepler_binary_returns_after_whole_periods():
    e1 = _kepler_error(0.1)
    e2 = _kepler_error(0.05)
    assert e1 < 1e-3 and e2 < 1e-4, (e1, e2)
    assert e2 < e1 / 8, (e1, e2)  # fourth order: ~1/16


def test_energy_of_compact_cluster_is_conserved():
    pos, vel, m = _cluster(64, 5, 0.01)
    r_cut, eps = 10.0, 2e-3  # every pair far inside r_in: pure softened Newton
    off, idx = oracle.neighbours(pos, r_cut)

    def energies(p, v):
        ke = 0.5 * np.sum(m[:, None] * v * v)
        d = p[:, None, :] - p[None, :, :]
        s = np.sqrt((d * d).sum(-1) + eps * eps)
        np.fill_diagonal(s, np.inf)
        pe = -0.5 * np.sum(m[:, None] * m[None, :] / s)
        return ke, pe

    vel = vel - np.average(vel, axis=0, weights=m)
    ke, pe = energies(pos, vel)
    vel = vel * np.sqrt(-0.5 * pe / ke)  # virial equilibrium
    e0 = sum(energies(pos, vel))
    t_cross = 0.01 / np.sqrt(2 * (-pe) / 2)  # size / rms speed

    def error(eta):
        p, v = pos, vel
        for _ in range(4):
            p, v, st = oracle.hermite(p, v, m, off, idx, dt_soft=t_cross,
                                      eps=eps, r_cut=r_cut, gamma=GAMMA, eta=eta)
        assert st[1] > st[0] > 4  # individual steps: more particle steps than blocks
        return abs(sum(energies(p, v)) - e0) / abs(e0)

    e1, e2 = error(0.05), error(0.025)
    assert e1 < 1e-7 and e2 < e1 / 8, (e1, e2)  # fourth order: ~1/16


def test_isolated_and_out_of_range_particles_move_straight():
    pos, vel, m = _cluster(50, 7, 1.0)
    r_cut = 1e-3
    # rows: particle 0 lists particle 1 (far beyond r_cut); the rest empty
    n = pos.shape[0]
    off = np.zeros(n + 1, dtype=np.int64)
    off[1:] = 1
    off[2:] = 2
    idx = np.array([1, 0], dtype=np.int32)
    p, v, st = oracle.hermite(pos, vel, m, off, idx, dt_soft=0.5, r_cut=r_cut,
                              gamma=GAMMA)
    assert np.array_equal(p[2:], pos[2:] + 0.5 * vel[2:])  # isolated drift
    assert np.array_equal(v, vel)
    assert np.abs(p[:2] - (pos[:2] + 0.5 * vel[:2])).max() <= 1e-15 * np.abs(pos).max() * 8


def _scaled_run(lam):
    pos, vel, m = _cluster(200, 11, 0.02)
    off, idx = oracle.neighbours(pos, 0.03)
    x, v, st, det = oracle.hermite(pos, vel / lam, m, off, idx, dt_soft=lam / 128,
                                   G=1.0 / lam ** 2, eps=1e-4, r_cut=0.02,
                                   gamma=GAMMA, detail=True)
    return x, v * lam, st, det


def test_schedule_does_not_depend_on_the_time_unit():
    x1, v1, st1, d1 = _scaled_run(1.0)
    for lam in (2.0, 0.25):
        x2, v2, st2, d2 = _scaled_run(lam)
        assert st1 == st2
        assert np.array_equal(d1["nstep"], d2["nstep"])
        assert np.array_equal(x1, x2) and np.array_equal(v1, v2)
    assert st1[1] > 2 * np.count_nonzero(d1["nstep"])  # several steps each


def test_first_level_follows_eq20_for_a_kepler_binary():
    # a binary at pericentre, separation r, relative speed w, far inside r_in
    # (K = 0): |a_i| = G m_j / r^2 and, with q . u = 0, |da_i| = G m_j w / r^3
    eta, alpha, r_cut, dt_soft = 0.1, 0.1, 1.0, 1.0
    for e in (0.0, 0.3, 0.6, 0.9):
        pos, vel, m, _ = _binary(e)
        r = pos[1, 0] - pos[0, 0]
        w = vel[1, 1] - vel[0, 1]
        off, idx = np.array([0, 1, 2]), np.array([1, 0], dtype=np.int32)
        _, _, _, det = oracle.hermite(pos, vel, m, off, idx, dt_soft=dt_soft,
                                      r_cut=r_cut, gamma=GAMMA, eta=eta,
                                      alpha=alpha, detail=True)
        a = m[1] / r ** 2
        j = m[1] * w / r ** 3
        a0 = alpha * m[0] / r_cut ** 2
        dt = (eta / 10) * np.sqrt((a * a + a0 * a0) / (j * j))
        k = int(np.ceil(np.log2(dt_soft / 4 / dt)))  # dt_max = dt_soft / 4
        assert det["lev0"][0] == det["lev0"][1] == k, (e, det["lev0"], k)


def test_mirror_is_within_rounding_of_the_oracle():
    from parity_util import assert_hard_step_close, hermite_sensitivity
    pos, vel, m = _cluster(1500, 4, 0.03)
    off, idx = oracle.neighbours(pos, 0.0125)
    kw = dict(dt_soft=1 / 128, eps=1e-4, r_cut=0.01, gamma=GAMMA)
    x0, v0, sx, sv = hermite_sensitivity(
        lambda p, v: oracle.hermite(p, v, m, off, idx, **kw)[:2], pos, vel)
    xm, vm, stm = oracle.hermite_mirror(pos, vel, m, off, idx, **kw)
    assert_hard_step_close(xm, vm, x0, v0, sx, sv)
    assert stm == oracle.hermite(pos, vel, m, off, idx, **kw)[2]
    a, j = oracle.hard_force(pos, vel, m, off, idx, eps=1e-4, r_cut=0.01, gamma=GAMMA)
    am, jm = oracle.hard_force_mirror(pos, vel, m, off, idx, eps=1e-4, r_cut=0.01,
                                      gamma=GAMMA)
    assert not np.array_equal(a, am)  # the two really round differently
    assert np.abs(am - a).max() <= 1e-12 * np.abs(a).max()
