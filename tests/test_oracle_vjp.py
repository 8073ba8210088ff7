"""Pins of the oracle's gradients of L = sum_i w_i . a_i (tree topology and
interaction lists frozen): central finite differences, translation
invariance, and theta = 0 against an independent direct-summation gradient."""
import numpy as np
import pytest

import oracle
from paper_1506_04553_b300 import ics

GAMMA = 0.1


@pytest.fixture(scope="module")
def setup():
    n = 2048
    pos, _, m = ics.plummer(n, seed=31)
    pos = pos.T.copy()
    m = m * np.random.default_rng(32).uniform(0.5, 1.5, n)
    w = np.random.default_rng(40).normal(size=(n, 3))
    kw = dict(G=1.0, eps=1e-3, r_cut=0.05, gamma=GAMMA)
    t = oracle.Tree(pos, m, n_leaf=8, n_group=32)
    t.walk(0.5, 0.05, 0.05)
    gx, gm = t.vjp(w, **kw)
    return pos, m, w, kw, t, gx, gm


def _loss(t, pos, m, w, kw):
    t.update(pos, m)
    return float((t.force(**kw) * w).sum())


def test_lists_mix_cells_and_particles(setup):
    _, _, _, _, t, _, _ = setup
    L = t.lists()
    assert L["pc"].size > 1000 and L["ppn"].size > 1000 and L["ppf"].size > 1000


def test_gradient_matches_central_differences(setup):
    pos, m, w, kw, t, gx, gm = setup
    h = 1e-6
    rng = np.random.default_rng(5)
    rows = rng.choice(pos.shape[0], 12, replace=False)
    for i in rows:
        for c in range(3):
            pp = pos.copy(); pp[i, c] += h
            pm = pos.copy(); pm[i, c] -= h
            fd = (_loss(t, pp, m, w, kw) - _loss(t, pm, m, w, kw)) / (2 * h)
            assert abs(fd - gx[i, c]) <= 1e-5 * np.abs(gx).max() + 1e-6 * abs(fd), (i, c, fd, gx[i, c])
        hm = 1e-6 * m[i]
        mp = m.copy(); mp[i] += hm
        mm = m.copy(); mm[i] -= hm
        fd = (_loss(t, pos, mp, w, kw) - _loss(t, pos, mm, w, kw)) / (2 * hm)
        assert abs(fd - gm[i]) <= 1e-5 * np.abs(gm).max() + 1e-6 * abs(fd), (i, fd, gm[i])
    t.update(pos, m)


def test_translation_invariance(setup):
    # a_i depends on differences of positions only, so sum_k dL/dx_k = 0
    pos, m, w, kw, t, gx, gm = setup
    assert np.abs(gx.sum(axis=0)).max() <= 1e-10 * np.abs(gx).sum(axis=0).max()


def test_theta_zero_equals_direct_gradient():
    n = 600
    rng = np.random.default_rng(9)
    pos = rng.normal(size=(n, 3)) * 0.05
    m = rng.uniform(0.5, 1.5, n) / n
    w = rng.normal(size=(n, 3))
    kw = dict(G=1.0, eps=5e-4, r_cut=0.03, gamma=GAMMA)
    t = oracle.Tree(pos, m, n_leaf=16, n_group=64)
    t.walk(0.0, 0.03, 0.03)
    gx, gm = t.vjp(w, **kw)
    dx, dm = oracle.direct_vjp(pos, m, w, **kw)
    assert np.abs(gx - dx).max() <= 1e-11 * np.abs(dx).max()
    assert np.abs(gm - dm).max() <= 1e-11 * np.abs(dm).max()
