"""Pins of the soft-interaction counts behind the cost model of Sect. 3.1.2
(the tree part costs O(theta^-3 N log N) per soft step), on the oracle's
tree: at theta = 0 no cell is accepted and every group meets every
particle, N^2 pair terms; a cell accepted at some theta is, at any smaller
theta, either accepted too or opened into at least one entry, so the count
of every group never rises with theta; and the counts per particle grow
with N at fixed theta."""
import numpy as np

import oracle
from paper_1506_04553_b300 import ics


def _counts(t, theta, r_out):
    """Interactions per group (cells, particles), each list entry taken
    once per particle of the group."""
    t.walk(theta, r_out, r_out)
    L = t.lists()
    cnt = t.groups()["count"].astype(np.int64)
    pc = np.diff(L["pc_off"]) * cnt
    pp = (np.diff(L["ppn_off"]) + np.diff(L["ppf_off"])) * cnt
    return pc, pp


def test_theta_zero_is_the_direct_sum_count():
    pos, _, m = ics.plummer(3000, seed=8)
    t = oracle.Tree(pos.T, m, n_leaf=16, n_group=64)
    pc, pp = _counts(t, 0.0, 0.01)
    assert pc.sum() == 0
    assert pp.sum() == 3000 * 3000


def test_counts_never_rise_with_theta():
    pos, _, m = ics.plummer(16384, seed=9)
    t = oracle.Tree(pos.T, m, n_leaf=16, n_group=64)
    r_out = 0.01 * (16384 / 8192) ** (-1 / 3)
    prev = None
    totals = []
    for theta in (0.2, 0.3, 0.4, 0.5, 0.6, 0.8, 1.0):
        pc, pp = _counts(t, theta, r_out)
        tot = pc + pp
        if prev is not None:
            assert np.all(tot <= prev), theta  # group by group
        prev = tot
        totals.append(tot.sum())
    assert totals[0] > 2 * totals[-1]


def test_counts_per_particle_grow_with_n():
    per = []
    for n in (4096, 16384, 65536):
        pos, _, m = ics.plummer(n, seed=10)
        t = oracle.Tree(pos.T, m, n_leaf=16, n_group=64)
        pc, pp = _counts(t, 0.4, 0.01 * (n / 8192) ** (-1 / 3))
        per.append((pc.sum() + pp.sum()) / n)
    assert per[0] < per[1] < per[2]
