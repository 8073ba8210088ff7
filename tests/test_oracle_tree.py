"""Pins of the oracle's Barnes-Hut tree (Sect. 2.2): structure invariants,
brute-force key construction, multipole accuracy, theta -> 0 limit, and the
completeness of every interaction list."""
import math

import numpy as np
import pytest

import oracle
from paper_1506_04553_b300 import ics

GAMMA = 0.1


def _brute_key(p, lo, size):
    """Morton key from the bit strings of the three 21-bit integer
    coordinates, interleaved as strings (x bit first in every triple)."""
    q = []
    for a in range(3):
        v = int(math.floor((p[a] - lo[a]) / size * 2**21))
        q.append(min(max(v, 0), 2**21 - 1))
    bits = [format(v, "021b") for v in q]
    return int("".join(bits[0][k] + bits[1][k] + bits[2][k] for k in range(21)), 2)


def test_morton_key_brute_force():
    rng = np.random.default_rng(11)
    pos = rng.normal(size=(400, 3))
    lo, size = oracle.root_box(pos)
    assert np.all(lo == pos.min(axis=0))
    assert size > np.ptp(pos, axis=0).max()
    for p in pos:
        assert oracle.morton_key(p, lo, size) == _brute_key(p, lo, size)
    # the extreme corner lands in the last cell, not outside the cube
    hi = pos.max(axis=0)
    assert oracle.morton_key(hi, lo, size) == _brute_key(hi, lo, size)


def _cell_cube(key, level, lo, size):
    """Geometric cube of the level-`level` ancestor of `key`."""
    q = [0, 0, 0]
    for b in range(level):
        tri = (key >> (3 * (20 - b))) & 7
        q[0] = 2 * q[0] + ((tri >> 2) & 1)
        q[1] = 2 * q[1] + ((tri >> 1) & 1)
        q[2] = 2 * q[2] + (tri & 1)
    side = size / 2**level
    return np.array(lo) + np.array(q) * side, side


@pytest.fixture(scope="module")
def plummer_tree():
    pos, _, m = ics.plummer(8192, seed=1)
    t = oracle.Tree(pos.T, m, n_leaf=16, n_group=64)
    return pos.T.copy(), m, t


def test_tree_structure(plummer_tree):
    pos, m, t = plummer_tree
    key, order = t.particles()
    lo, size = t.root()
    n = pos.shape[0]
    # sorted by (key, original index)
    assert np.all((np.diff(key.astype(object)) > 0)
                  | ((np.diff(key.astype(object)) == 0) & (np.diff(order) > 0)))
    assert np.array_equal(np.sort(order), np.arange(n))
    c = t.cells()
    C = t.ncell
    for k in range(C):
        f, cnt, L = int(c["first"][k]), int(c["count"][k]), int(c["level"][k])
        if c["nchild"][k] == 0:
            assert cnt <= 16 or L == 21
        else:
            assert cnt > 16 and L < 21
            ch = np.arange(c["child_first"][k], c["child_first"][k] + c["nchild"][k])
            assert np.all(c["level"][ch] == L + 1)
            assert c["first"][ch[0]] == f
            assert np.array_equal(c["first"][ch[1:]], c["first"][ch[:-1]] + c["count"][ch[:-1]])
            assert c["count"][ch].sum() == cnt
        # members inside the geometric cube of the cell's key prefix
        corner, side = _cell_cube(int(key[f]), int(L), lo, size)
        mem = pos[order[f:f + cnt]]
        assert np.all(mem >= corner - 1e-12 * size)
        assert np.all(mem <= corner + side + 1e-12 * size)
        # all members share the level-L prefix
        sh = 3 * (21 - L)
        assert len({int(v) >> sh for v in key[f:f + cnt]}) == 1


def test_moments(plummer_tree):
    pos, m, t = plummer_tree
    key, order = t.particles()
    c = t.cells()
    for k in range(0, t.ncell, 7):
        f, cnt = c["first"][k], c["count"][k]
        mem = pos[order[f:f + cnt]]
        mm = m[order[f:f + cnt]]
        M = mm.sum()
        com = (mm[:, None] * mem).sum(axis=0) / M
        assert abs(c["M"][k] - M) < 1e-14 * M
        assert np.abs(c["com"][k] - com).max() < 1e-12 * (1 + np.abs(com).max())
        Q = c["Q"][k]
        assert abs(Q[0] + Q[1] + Q[2]) < 1e-12 * (np.abs(Q).max() + 1e-300)
        if cnt == 1:
            assert np.all(Q == 0.0)
        # FP32 boxes contain the members (outward rounding)
        assert np.all(c["fmin"][k].astype(np.float64) <= mem.min(axis=0))
        assert np.all(c["fmax"][k].astype(np.float64) >= mem.max(axis=0))
    # parallel-axis theorem: a parent's quadrupole equals its children's
    # quadrupoles plus each child's mass shifted to the parent's centre
    for k in np.nonzero(c["nchild"] > 0)[0][:200]:
        ch = np.arange(c["child_first"][k], c["child_first"][k] + c["nchild"][k])
        Q = np.zeros(6)
        for j in ch:
            d = c["com"][j] - c["com"][k]
            d2 = d @ d
            Q += c["Q"][j] + c["M"][j] * np.array([
                3 * d[0] * d[0] - d2, 3 * d[1] * d[1] - d2, 3 * d[2] * d[2] - d2,
                3 * d[0] * d[1], 3 * d[0] * d[2], 3 * d[1] * d[2]])
        assert np.abs(Q - c["Q"][k]).max() < 1e-10 * (np.abs(Q).max() + 1e-300)


def test_groups_partition(plummer_tree):
    pos, m, t = plummer_tree
    g = t.groups()
    o = np.argsort(g["first"])
    first, count = g["first"][o], g["count"][o]
    assert first[0] == 0
    assert np.array_equal(first[1:], first[:-1] + count[:-1])
    assert first[-1] + count[-1] == pos.shape[0]
    assert count.max() <= 64 and count.min() >= 1
    # every group lies inside one container: a cell of at most 16 * 64
    # particles whose parent holds more; inside it groups are chunks of 64
    c = t.cells()
    cont = [k for k in range(t.ncell)
            if (c["count"][k] <= 1024 or c["nchild"][k] == 0)
            and (c["parent"][k] < 0 or c["count"][c["parent"][k]] > 1024)]
    cf = np.sort(c["first"][cont])
    assert cf[0] == 0 and np.sum(c["count"][cont]) == pos.shape[0]
    box = np.searchsorted(cf, first, side="right") - 1
    start = cf[box]
    assert np.all((first - start) % 64 == 0)  # chunks from the container start
    assert count.mean() > 48  # well filled (52 for this input)


def test_quadrupole_expansion_accuracy():
    # a compact cluster seen from afar: monopole + quadrupole leaves an error
    # of order (b/r)^3 relative to the monopole; halving b/r must shrink it
    # about eightfold (a wrong quadrupole term would leave (b/r)^2)
    rng = np.random.default_rng(4)
    src = rng.normal(size=(40, 3)) * np.array([1.0, 0.5, 0.25])
    m = rng.uniform(0.5, 1.5, 40)
    errs = []
    for dist in (20.0, 40.0, 80.0):
        probe = np.array([[dist, 0.3 * dist, -0.2 * dist]])
        pos = np.vstack([src, probe])
        mm = np.concatenate([m, [1e-30]])
        t = oracle.Tree(pos, mm, n_leaf=1, n_group=1)
        t.walk(theta=0.9, h=1e-9, r_cut=1e-9)
        L = t.lists()
        g = t.groups()
        key, order = t.particles()
        k = int(np.nonzero(order == 40)[0][0])
        gi = int(np.nonzero((g["first"] <= k) & (g["first"] + g["count"] > k))[0][0])
        assert L["pc_off"][gi + 1] - L["pc_off"][gi] >= 1  # the cluster is a cell
        a_tree = t.force(r_cut=1e-9, eps=0.0)[40]
        a_dir = oracle.direct(pos, mm, kind="newton", rows=[40])[0]
        mono = m.sum() / np.sum(probe**2)
        errs.append(np.linalg.norm(a_tree - a_dir) / mono)
    assert errs[0] < 1e-3
    assert 5.0 < errs[0] / errs[1] < 12.0
    assert 5.0 < errs[1] / errs[2] < 12.0


def _rel_err(a, ref):
    nr = np.linalg.norm(ref, axis=1)
    floor = 1e-3 * np.sqrt(np.mean(nr**2))
    return np.linalg.norm(a - ref, axis=1) / np.maximum(nr, floor)


def test_theta_zero_is_direct_sum(plummer_tree):
    pos, m, t = plummer_tree
    n = pos.shape[0]
    kw = dict(G=1.0, eps=4.0 / n, r_cut=0.01, gamma=GAMMA)
    t.walk(theta=0.0, h=0.01, r_cut=0.01)
    L = t.lists()
    assert L["pc"].size == 0
    a_t, p_t = t.force(potential=True, **kw)
    a_d, p_d = oracle.direct(pos, m, kind="soft", potential=True, **kw)
    assert np.abs(a_t - a_d).max() < 1e-12 * np.abs(a_d).max()
    assert np.abs(p_t - p_d).max() < 1e-12 * np.abs(p_d).max()


def test_error_shrinks_with_theta(plummer_tree):
    pos, m, t = plummer_tree
    n = pos.shape[0]
    kw = dict(G=1.0, eps=4.0 / n, r_cut=0.01, gamma=GAMMA)
    a_d = oracle.direct(pos, m, kind="soft", **kw)
    med = []
    for th in (0.8, 0.6, 0.4, 0.2):
        t.walk(theta=th, h=0.01, r_cut=0.01)
        med.append(np.median(_rel_err(t.force(**kw), a_d)))
    assert all(med[i + 1] < med[i] for i in range(len(med) - 1)), med
    assert med[2] < 2e-3  # theta = 0.4


def test_lists_complete_and_guarded(plummer_tree):
    pos, m, t = plummer_tree
    h = r_cut = 0.01
    t.walk(theta=0.4, h=h, r_cut=r_cut)
    L = t.lists()
    key, order = t.particles()
    c = t.cells()
    g = t.groups()
    xs = pos[order]
    hg = max(h, r_cut)
    for gi in range(0, t.ngroup, 5):
        cov = np.zeros(pos.shape[0], np.int64)
        for cid in L["pc"][L["pc_off"][gi]:L["pc_off"][gi + 1]]:
            cov[c["first"][cid]:c["first"][cid] + c["count"][cid]] += 1
        near = L["ppn"][L["ppn_off"][gi]:L["ppn_off"][gi + 1]]
        far = L["ppf"][L["ppf_off"][gi]:L["ppf_off"][gi + 1]]
        cov[near] += 1
        cov[far] += 1
        assert np.all(cov == 1)  # every particle exactly once
        mem = xs[g["first"][gi]:g["first"][gi] + g["count"][gi]]
        # cells and far particles: every pair farther apart than max(h, r_cut)
        for cid in L["pc"][L["pc_off"][gi]:L["pc_off"][gi + 1]][:50]:
            src = xs[c["first"][cid]:c["first"][cid] + c["count"][cid]]
            d = np.linalg.norm(mem[:, None, :] - src[None, :, :], axis=2)
            assert d.min() > hg
        if far.size:
            d = np.linalg.norm(mem[:, None, :] - xs[far][None, :, :], axis=2)
            assert d.min() > hg


def test_degenerate_inputs():
    # one particle, a few coincident particles, a tiny cluster
    t = oracle.Tree(np.zeros((1, 3)), np.ones(1))
    assert t.ncell == 1 and t.ngroup == 1
    t.walk(0.4, 0.01, 0.01)
    assert np.all(t.force(r_cut=0.01) == 0.0)
    pos = np.zeros((40, 3))
    t = oracle.Tree(pos, np.full(40, 0.025), n_leaf=16, n_group=16)
    c = t.cells()
    assert c["level"].max() == 21  # a chain down to the finest level
    assert t.ngroup == 3  # the big leaf in chunks of 16
    t.walk(0.4, 0.01, 0.01)
    a = t.force(r_cut=0.01, eps=0.0)
    assert np.all(a == 0.0)  # coincident pairs have K(0) = 0
