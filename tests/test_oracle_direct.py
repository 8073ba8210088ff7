"""Pins of the oracle's direct summation (Eq. 2-3, 5-8) and leapfrog pieces
against closed forms, invariants and textbook results."""
import math

import numpy as np
import pytest

import oracle
from paper_1506_04553_b300 import ics

GAMMA = 0.1


def _pair(r, eps, r_cut, kind):
    pos = np.array([[0.0, 0.0, 0.0], [r, 0.0, 0.0]])
    m = np.array([0.25, 0.75])
    return oracle.direct(pos, m, G=2.0, eps=eps, r_cut=r_cut, gamma=GAMMA,
                         kind=kind, potential=True)


def test_two_body_beyond_cutoff_is_newtonian():
    # s >= r_cut: K = 1 (Eq. 12), so the soft force is the softened Newtonian
    # pull G m_j / s^3 q toward the partner and the hard force vanishes
    r, eps, rc = 0.3, 0.05, 0.1
    s = math.hypot(r, eps)
    (a, phi) = _pair(r, eps, rc, "soft")
    assert abs(a[0, 0] - 2.0 * 0.75 * r / s**3) < 1e-14
    assert abs(a[1, 0] + 2.0 * 0.25 * r / s**3) < 1e-14
    assert np.all(a[:, 1:] == 0.0)
    assert abs(phi[0] + 2.0 * 0.75 / s) < 1e-14  # W = 1 beyond r_cut (Eq. 16)
    (ah, phih) = _pair(r, eps, rc, "hard")
    assert np.all(ah == 0.0)
    assert np.all(np.abs(phih) < 1e-15)


def test_two_body_inside_r_in_is_all_hard():
    # s < r_in: K = 0, the whole force is in the hard part (Eq. 7-8)
    r, rc = 0.004, 0.1  # r_in = 0.01
    (a, _) = _pair(r, 0.0, rc, "soft")
    assert np.all(a == 0.0)
    (ah, _) = _pair(r, 0.0, rc, "hard")
    assert abs(ah[0, 0] - 2.0 * 0.75 / r**2) < 1e-9 * (2.0 * 0.75 / r**2)
    # the soft potential inside r_in is W/s = c / r_cut (Eq. 16 first branch)
    (_, phi) = _pair(r, 0.0, rc, "soft")
    c = oracle.W_inner_slope(GAMMA)
    assert abs(phi[0] + 2.0 * 0.75 * c / rc) < 1e-12


def test_soft_plus_hard_is_newton_and_momentum():
    rng = np.random.default_rng(5)
    pos = rng.normal(size=(500, 3)) * 0.05
    m = rng.uniform(0.5, 2.0, 500) / 500
    kw = dict(G=1.0, eps=1e-3, r_cut=0.02, gamma=GAMMA)
    a_s = oracle.direct(pos, m, kind="soft", **kw)
    a_h = oracle.direct(pos, m, kind="hard", **kw)
    a_n = oracle.direct(pos, m, kind="newton", **kw)
    scale = np.abs(a_n).max()
    assert np.abs(a_s + a_h - a_n).max() < 1e-12 * scale
    # Newton's third law pair by pair: sum m_i a_i = 0
    for a in (a_s, a_h, a_n):
        tot = (m[:, None] * a).sum(axis=0)
        assert np.abs(tot).max() < 1e-13 * (m[:, None] * np.abs(a)).sum()
    # both parts are genuinely non-trivial here
    assert np.abs(a_s).max() > 0.1 * scale and np.abs(a_h).max() > 0.1 * scale


def test_force_is_minus_gradient_of_potential():
    # a_i = -grad_i phi_i for the soft and hard parts (Eq. 5-8)
    rng = np.random.default_rng(7)
    pos = rng.normal(size=(40, 3)) * 0.01
    m = rng.uniform(0.5, 2.0, 40) / 40
    kw = dict(G=1.0, eps=2e-4, r_cut=0.02, gamma=GAMMA)
    for kind in ("soft", "hard", "newton"):
        a, _ = oracle.direct(pos, m, kind=kind, potential=True, **kw)
        h = 1e-7
        for i in (0, 7, 23):
            g = np.zeros(3)
            for c in range(3):
                pp = pos.copy(); pp[i, c] += h
                pm = pos.copy(); pm[i, c] -= h
                _, fp = oracle.direct(pp, m, kind=kind, potential=True, rows=[i], **kw)
                _, fm = oracle.direct(pm, m, kind=kind, potential=True, rows=[i], **kw)
                g[c] = (fp[0] - fm[0]) / (2 * h)
            assert np.abs(a[i] + g).max() < 1e-5 * np.abs(a[i]).max() + 1e-9


def test_plummer_potential_energy_nbody_units():
    # Plummer sphere in N-body units: E = -1/4 and the virial theorem give
    # W_pot = -1/2 (= -3 pi / (32 a) with a = 3 pi / 16); the Newtonian direct
    # sum of a sample of N = 8192 lies within a few percent of it
    n = 8192
    pos, vel, m = ics.plummer(n, seed=1)
    _, phi = oracle.direct(pos.T, m, kind="newton", eps=4.0 / n, potential=True)
    W = 0.5 * float((m * phi).sum())
    assert abs(W - (-3.0 * math.pi / (32.0 * (3.0 * math.pi / 16.0)))) < 0.02
    T = 0.5 * float((m * (vel * vel).sum(axis=0)).sum())
    assert abs(2 * T / -W - 1.0) < 0.05


def test_softening_limit():
    rng = np.random.default_rng(9)
    pos = rng.normal(size=(100, 3))
    m = np.full(100, 0.01)
    a0 = oracle.direct(pos, m, kind="newton", eps=0.0)
    a1 = oracle.direct(pos, m, kind="newton", eps=1e-6)
    assert np.abs(a1 - a0).max() < 1e-8 * np.abs(a0).max()


def test_rows_subset_matches_full():
    rng = np.random.default_rng(3)
    pos = rng.normal(size=(300, 3)) * 0.1
    m = np.full(300, 1 / 300)
    full = oracle.direct(pos, m, kind="soft", eps=1e-3, r_cut=0.05)
    rows = np.array([5, 17, 299, 0])
    sub = oracle.direct(pos, m, kind="soft", eps=1e-3, r_cut=0.05, rows=rows)
    assert np.array_equal(sub, full[rows])


def test_kick_and_drift_definition():
    rng = np.random.default_rng(2)
    v = rng.normal(size=(3, 50))
    x = rng.normal(size=(3, 50))
    a = rng.normal(size=(3, 50)).astype(np.float32)
    assert np.array_equal(oracle.kick(v, a, 0.125), v + 0.125 * a.astype(np.float64))
    assert np.array_equal(oracle.drift(x, v, 1 / 256), x + (1 / 256) * v)
