"""Full-size parity on sampled outputs, in the launch configuration bench.py
times: Plummer N = 2^20 (theta 0.4, r_out 0.0025) and a King W0 = 9 model
with Salpeter masses, N = 2^21 (theta 0.5, r_out 0.002).  Forces of randomly
chosen groups against the same-tree FP64 oracle; neighbour rows of sampled
particles (King: drawn from the 4 x 2048 densest) against brute force over
all particles."""
import numpy as np
import pytest

import oracle
from paper_1506_04553_b300 import ics
from parity_util import gpu_run, rel_err

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


def _check(pos, m, params, n_groups=256, n_rows=2048, dense_rows=False):
    ctx, acc, _, ngb = gpu_run(pos, m, params)
    n = pos.shape[0]
    t = oracle.Tree(pos, m, n_leaf=params.n_leaf, n_group=params.n_group)
    h = params.h if params.h > 0 else params.r_out
    t.walk(params.theta, h, params.r_out)
    st = ctx.stats()
    L = t.lists()
    assert st["list_pc"] == L["pc"].size and st["list_pp_near"] == L["ppn"].size
    ctx.lists()  # the inspection walk records the deepest stack
    depth = ctx.stats()["max_walk_stack"]
    print(f"deepest walk stack: {depth} of 768")
    assert 0 < depth <= 768 // 4
    g = t.groups()
    rng = np.random.default_rng(77)
    sel = rng.choice(t.ngroup, n_groups, replace=False)
    a_o = t.force(G=params.G, eps=params.eps, r_cut=params.r_out,
                  gamma=params.gamma, groups=sel)
    key, order = t.particles()
    rows = np.concatenate([order[g["first"][q]:g["first"][q] + g["count"][q]] for q in sel])
    e = rel_err(acc[rows], a_o[rows])
    assert np.median(e) <= 1e-5 and e.max() <= 1e-4, (np.median(e), e.max())
    off, idx = ngb
    if dense_rows:
        cnt = np.diff(off)
        cand = np.argsort(-cnt)[: 4 * n_rows]
        rsel = rng.choice(cand, n_rows, replace=False)
    else:
        rsel = rng.choice(n, n_rows, replace=False)
    off_o, idx_o = oracle.neighbours(pos, h, rows=rsel)
    for r, i in enumerate(rsel):
        assert np.array_equal(idx[off[i]:off[i + 1]], idx_o[off_o[r]:off_o[r + 1]]), i
    return np.diff(off)


def test_plummer_2p20(cuda):
    from paper_1506_04553_b300 import Params
    n = 1 << 20
    pos, _, m = ics.plummer(n, 2)
    cnt = _check(pos.T.copy(), m, Params(theta=0.4, r_out=0.0025, eps=4.0 / n))
    assert cnt.sum() > 0


def test_king_w9_salpeter_2p21(cuda):
    from paper_1506_04553_b300 import Params
    n = 1 << 21
    masses = ics.salpeter_masses(n, seed=3 + 7919)
    pos, _, m = ics.king(n, 3, W0=9.0, masses=masses)
    cnt = _check(pos.T.copy(), m, Params(theta=0.5, r_out=0.002, eps=4.0 / n),
                 dense_rows=True)
    assert cnt.max() >= 8  # dense core (measured maximum: 12 neighbours)


def test_plummer_2p20_sixteen_kdk_steps(cuda):
    """The 16-step workload: Plummer N = 2^20 (seed 2), theta 0.4, r_out
    0.0025, eps 4/N, 16 leapfrog steps of the soft part at dt = 1/256 (kick
    dt/2, drift dt, build, force, neighbour lists, kick dt/2: the Sect. 2.2
    step with the Hermite step replaced by a drift of every particle).  After
    every step the GPU's force on a fixed subsample (the first 4096 of a
    seeded permutation) is compared with the same-tree FP64 oracle built from
    the GPU's own positions of that step: trajectories of an N-body system
    diverge, so the error is measured per step on the GPU's state."""
    import torch
    from paper_1506_04553_b300 import Context, Params, drift, kick
    n, dt = 1 << 20, 1.0 / 256
    pos, vel, m = ics.plummer(n, 2)
    params = Params(theta=0.4, r_out=0.0025, eps=4.0 / n)
    ctx = Context(params)
    pd = torch.tensor(pos, device="cuda")
    vd = torch.tensor(vel, device="cuda")
    md = torch.tensor(m, device="cuda")
    ctx.build_tree(pd, md)
    acc = ctx.long_force()
    sub = np.random.default_rng(2).permutation(n)[:4096]
    worst = []
    for step in range(16):
        kick(vd, acc, dt / 2)
        drift(pd, vd, dt)
        ctx.build_tree(pd, md)
        ctx.long_force(acc)
        ctx.neighbours()
        kick(vd, acc, dt / 2)
        p_h = pd.cpu().numpy().T.copy()
        a_g = acc.cpu().numpy().T.astype(np.float64)[sub]
        t = oracle.Tree(p_h, m, n_leaf=params.n_leaf, n_group=params.n_group)
        t.walk(params.theta, params.r_out, params.r_out)
        a_o = t.force_particles(sub, G=params.G, eps=params.eps,
                                r_cut=params.r_out, gamma=params.gamma)
        e = rel_err(a_g, a_o)
        worst.append((step + 1, float(np.median(e)), float(e.max())))
        assert np.median(e) <= 1e-5 and e.max() <= 1e-4, worst[-1]
    print("per-step error on the subsample (step, median, max):",
          ", ".join(f"({s}, {a:.2e}, {b:.2e})" for s, a, b in worst))
