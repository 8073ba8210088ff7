"""Pins of the oracle's two-species path (Sect. 3.2.2: stars and two black
holes, a cut-off per kind of pair, no split and no softening between the
black holes, eta per species) against closed forms: the black hole pair
feels exactly the unsoftened Newtonian force, all of it hard; star pairs
keep the split of Eq. 7-8 with their own cut-off and softening; neighbour
radii apply per pair type; and a black hole binary integrated alone by the
hard part returns to its start after one Kepler period."""
import math

import numpy as np
import pytest

import oracle

INF = math.inf
GAMMA = 0.1


def _weights(s, r_cut):
    y = s / r_cut
    x = (y - GAMMA) / (1 - GAMMA)
    K = 0.0 if x < 0 else (1.0 if x >= 1 else x**4 * (35 - 84 * x + 70 * x**2 - 20 * x**3))
    return K


def test_black_hole_pair_is_unsoftened_newton_and_all_hard():
    # stars far away (beyond every cut-off), black holes 0.3 apart
    pos = np.array([[10.0, 0, 0], [-10.0, 0, 0], [0.1, 0.2, 0.0], [0.4, 0.2, 0.0]])
    m = np.array([1e-3, 1e-3, 0.01, 0.02])
    kw = dict(eps=[1e-2, 1e-2, 0.0], r_cut=[0.05, 0.5, INF])
    soft = oracle.direct_species(pos, m, 2, kind="soft", **kw)
    hard = oracle.direct_species(pos, m, 2, kind="hard", **kw)
    # soft force on a black hole: the stars only (K = 1 at 10 > r_cut[1]),
    # softened with eps[1]; nothing from the other black hole
    for b_ in (2, 3):
        want = np.zeros(3)
        for s_ in (0, 1):
            q = pos[s_] - pos[b_]
            want += m[s_] * q / (q @ q + 1e-4) ** 1.5
        assert np.allclose(soft[b_], want, rtol=1e-14, atol=0)
    # hard force on the black holes: G m_j / d^2 along x, exactly unsoftened
    # (plus the stars, at 10 with K(10/0.5) = 1: no hard part from them)
    assert hard[2, 0] == pytest.approx(0.02 / 0.3**2, rel=1e-14)
    assert hard[3, 0] == pytest.approx(-0.01 / 0.3**2, rel=1e-14)
    assert np.all(hard[2:, 1:] == 0.0)


def test_star_pairs_split_with_their_own_cut_off_and_softening():
    d = 0.03
    pos = np.array([[0.0, 0, 0], [d, 0, 0], [5.0, 0, 0]])
    m = np.array([0.5, 0.25, 0.1])
    eps = [1e-3, 2e-3, 0.0]
    r_cut = [0.04, 0.3, INF]
    # particle 2 is the black hole, far from the stars: K = 1 for its pairs
    soft = oracle.direct_species(pos, m, 1, eps=eps, r_cut=r_cut, kind="soft")
    hard = oracle.direct_species(pos, m, 1, eps=eps, r_cut=r_cut, kind="hard")
    s = math.sqrt(d * d + eps[0] ** 2)
    K = _weights(s, r_cut[0])
    assert 0.0 < K < 1.0
    f01 = 0.25 * d / s**3  # on star 0 from star 1, Newtonian softened
    sb = math.sqrt(25.0 + eps[1] ** 2)
    fbh = 0.1 * 5.0 / sb**3  # from the black hole, K = 1 at 5 > r_cut[1]
    assert soft[0, 0] == pytest.approx(K * f01 + fbh, rel=1e-12)
    assert hard[0, 0] == pytest.approx((1 - K) * f01, rel=1e-12)
    # soft + hard = Newton with the pair's softening, for every particle
    newton = np.zeros_like(soft)
    for i in range(3):
        for j in range(3):
            if i == j:
                continue
            t = (i >= 2) + (j >= 2)
            q = pos[j] - pos[i]
            sij = math.sqrt(q @ q + eps[t] ** 2)
            newton[i] += m[j] * q / sij**3
    assert np.allclose(soft + hard, newton, rtol=1e-13, atol=0)


def test_neighbour_radius_per_pair_type():
    # stars 0, 1, 2; black holes 3, 4 far apart from each other
    pos = np.array([[0.0, 0, 0], [0.05, 0, 0], [0.3, 0, 0],
                    [0.2, 0, 0], [100.0, 0, 0]])
    off, idx = oracle.neighbours_species(pos, 2, h=[0.1, 0.25, INF])
    rows = [idx[off[i]:off[i + 1]].tolist() for i in range(5)]
    assert rows[0] == [1, 3]     # star 1 at 0.05 < 0.1; hole 3 at 0.2 < 0.25
    assert rows[1] == [0, 3]     # hole 3 at 0.15
    assert rows[2] == [3]        # star 1 at 0.25 > 0.1; hole 3 at 0.1
    assert rows[3] == [0, 1, 2, 4]  # holes: always neighbours
    assert rows[4] == [3]
    # symmetric
    for i in range(5):
        for j in rows[i]:
            assert i in rows[j]


def test_species_reduce_to_the_plain_path_with_no_black_holes():
    rng = np.random.default_rng(4)
    pos = rng.normal(size=(300, 3)) * 0.02
    vel = rng.normal(size=(300, 3)) * 0.1
    m = rng.uniform(0.5, 1.5, 300) / 300
    off, idx = oracle.neighbours(pos, 0.0125)
    off2, idx2 = oracle.neighbours_species(pos, 0, h=[0.0125, 1.0, 1.0])
    assert np.array_equal(off, off2) and np.array_equal(idx, idx2)
    a, j = oracle.hard_force(pos, vel, m, off, idx, eps=1e-4, r_cut=0.01)
    a2, j2 = oracle.hard_force_species(pos, vel, m, off, idx, 0, eps=[1e-4, 1, 1],
                                       r_cut=[0.01, 1, 1])
    assert np.array_equal(a, a2) and np.array_equal(j, j2)
    x, v, st = oracle.hermite(pos, vel, m, off, idx, dt_soft=1 / 128, eps=1e-4,
                              r_cut=0.01)
    x2, v2, st2 = oracle.hermite_species(pos, vel, m, off, idx, 0, dt_soft=1 / 128,
                                         eps=[1e-4, 1, 1], r_cut=[0.01, 1, 1],
                                         eta=[0.1, 0.5])
    assert np.array_equal(x, x2) and np.array_equal(v, v2) and st == st2


def test_black_hole_binary_returns_after_one_kepler_period():
    """Two black holes on a circular orbit of separation a (Sect. 3.2.2
    sets them at +-0.5 with speeds +-0.5): the hard part alone integrates
    the unsoftened, unsplit pair; after one period they are back."""
    m1 = m2 = 0.01
    a = 0.02
    mu = m1 + m2
    v_rel = math.sqrt(mu / a)
    pos = np.array([[a / 2, 0.0, 0.0], [-a / 2, 0.0, 0.0]])
    vel = np.array([[0.0, v_rel / 2, 0.0], [0.0, -v_rel / 2, 0.0]])
    m = np.array([m1, m2])
    P = 2 * math.pi * math.sqrt(a**3 / mu)
    off, idx = oracle.neighbours_species(pos, 2, h=[0.01, 0.05, INF])
    assert off.tolist() == [0, 1, 2]
    kw = dict(eps=[1e-4, 1e-4, 0.0], r_cut=[1 / 256, 1 / 32, INF], p=2, kmax=30)
    x, v, st = oracle.hermite_species(pos, vel, m, off, idx, 2, dt_soft=P,
                                      eta=[0.1, 0.03], **kw)
    assert np.abs(x - pos).max() < 1e-6 * a
    assert np.abs(v - vel).max() < 1e-6 * v_rel
    # the black holes' own eta sets their steps: a larger eta takes fewer
    _, _, st_loose = oracle.hermite_species(pos, vel, m, off, idx, 2, dt_soft=P,
                                            eta=[0.03, 0.1], **kw)
    assert st_loose[1] < st[1]
