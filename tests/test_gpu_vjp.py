"""Backward pass (p3t_long_force_vjp, the autograd wrapper) against the FP64
oracle's gradient of L = sum_i w_i . a_i with the tree structure frozen.

Tolerance: the CUDA path evaluates every Jacobian product in FP32
(group-relative coordinates, ~1e-7 relative per term) and sums them into FP64;
per-particle relative error (floor 1e-3 rms): median <= 1e-5 for dL/dx and
dL/dm, max <= 1e-4 for dL/dx and <= 4e-3 for dL/dm, about three times the
largest values measured over these cases (medians ~3e-7; maxima 3.3e-5 for
dL/dx and 1.2e-3 for dL/dm, whose terms cancel more: a particle's mass
gradient sums signed potentials of opposite sign)."""
import numpy as np
import pytest

import oracle
from paper_1506_04553_b300 import ics
from parity_util import rel_err

pytestmark = pytest.mark.gpu

GAMMA = 0.1
MED, MAX_X, MAX_M = 1e-5, 1e-4, 4e-3


def _gpu_vjp(pos, m, w, params):
    import torch
    from paper_1506_04553_b300 import Context
    ctx = Context(params)
    pd = torch.tensor(np.ascontiguousarray(pos.T), device="cuda")
    md = torch.tensor(m, device="cuda")
    ctx.build_tree(pd, md)
    acc = ctx.long_force()
    wd = torch.tensor(np.ascontiguousarray(w.T), dtype=torch.float32, device="cuda")
    gx, gm = ctx.long_force_vjp(wd)
    return ctx, gx.cpu().numpy().T.copy(), gm.cpu().numpy()


def _scalar_err(a, ref):
    floor = 1e-3 * np.sqrt(np.mean(ref ** 2))
    return np.abs(a - ref) / np.maximum(np.abs(ref), floor)


def _case(n, seed, theta, unequal=True):
    pos, _, m = ics.plummer(n, seed)
    pos = pos.T.copy()
    if unequal:
        m = m * np.random.default_rng(seed + 100).uniform(0.5, 1.5, n)
    w = np.random.default_rng(seed + 40).normal(size=(n, 3))
    r_out = 0.01 * (n / 8192) ** (-1.0 / 3.0)
    return pos, m, w, dict(theta=theta, r_out=r_out, eps=4.0 / n)


@pytest.mark.parametrize("n,theta", [(16384, 0.4), (65536, 0.4), (4096, 0.7)])
def test_vjp_matches_oracle(cuda, n, theta):
    from paper_1506_04553_b300 import Params
    pos, m, w, kw = _case(n, 4, theta)
    p = Params(**kw)
    ctx, gx, gm = _gpu_vjp(pos, m, w, p)
    t = oracle.Tree(pos, m, n_leaf=p.n_leaf, n_group=p.n_group)
    t.walk(p.theta, p.r_out, p.r_out)
    ox, om = t.vjp(w, G=p.G, eps=p.eps, r_cut=p.r_out, gamma=p.gamma)
    ex = rel_err(gx, ox)
    em = _scalar_err(gm, om)
    print(f"n={n} theta={theta}: dL/dx median {np.median(ex):.2e} max {ex.max():.2e}; "
          f"dL/dm median {np.median(em):.2e} max {em.max():.2e}")
    assert np.median(ex) <= MED and ex.max() <= MAX_X, (np.median(ex), ex.max())
    assert np.median(em) <= MED and em.max() <= MAX_M, (np.median(em), em.max())


def test_vjp_theta_zero_equals_direct_gradient(cuda):
    from paper_1506_04553_b300 import Params
    n = 2048
    pos, m, w, kw = _case(n, 8, 0.0)
    p = Params(**kw)
    _, gx, gm = _gpu_vjp(pos, m, w, p)
    dx, dm = oracle.direct_vjp(pos, m, w, G=1.0, eps=p.eps, r_cut=p.r_out, gamma=GAMMA)
    ex = rel_err(gx, dx)
    em = _scalar_err(gm, dm)
    assert np.median(ex) <= MED and ex.max() <= MAX_X, (np.median(ex), ex.max())
    assert np.median(em) <= MED and em.max() <= MAX_M, (np.median(em), em.max())


def test_vjp_translation_invariance(cuda):
    from paper_1506_04553_b300 import Params
    pos, m, w, kw = _case(8192, 3, 0.4)
    _, gx, _ = _gpu_vjp(pos, m, w, Params(**kw))
    assert np.abs(gx.sum(axis=0)).max() <= 1e-5 * np.abs(gx).sum(axis=0).max()


def test_autograd_function(cuda):
    import torch
    from paper_1506_04553_b300 import Context, Params
    from paper_1506_04553_b300.autograd import long_range_force
    pos, m, w, kw = _case(8192, 5, 0.4)
    ctx = Context(Params(**kw))
    pd = torch.tensor(np.ascontiguousarray(pos.T), device="cuda", requires_grad=True)
    md = torch.tensor(m, device="cuda", requires_grad=True)
    wd = torch.tensor(np.ascontiguousarray(w.T), dtype=torch.float32, device="cuda")
    acc = long_range_force(pd, md, ctx)
    loss = (acc * wd).sum()
    loss.backward()
    gx, gm = ctx.long_force_vjp(wd)
    assert torch.allclose(pd.grad, gx, rtol=0, atol=0)
    assert torch.allclose(md.grad, gm, rtol=0, atol=0)
    t = oracle.Tree(pos, m)
    t.walk(kw["theta"], kw["r_out"], kw["r_out"])
    ox, _ = t.vjp(w, eps=kw["eps"], r_cut=kw["r_out"])
    ex = rel_err(pd.grad.cpu().numpy().T, ox)
    assert np.median(ex) <= MED


def _vjp_vs_oracle(pos, m, w, p):
    _, gx, gm = _gpu_vjp(pos, m, w, p)
    t = oracle.Tree(pos, m, n_leaf=p.n_leaf, n_group=p.n_group)
    t.walk(p.theta, p.r_out, p.r_out)
    ox, om = t.vjp(w, G=p.G, eps=p.eps, r_cut=p.r_out, gamma=p.gamma)
    return gx, gm, ox, om


@pytest.mark.parametrize("n", [1, 2, 17, 65, 300, 4099])
def test_vjp_small_and_ragged_sizes(cuda, n):
    """Groups, source tiles (64 per lane pair of a warp) and particle sweeps
    (four at a time) all partial: a few particles in a tight clump, every
    pair near, and a size that leaves a ragged tail at every level."""
    from paper_1506_04553_b300 import Params
    rng = np.random.default_rng(500 + n)
    pos = rng.normal(size=(n, 3)) * 0.01
    m = rng.uniform(0.5, 1.5, n) / n
    w = rng.normal(size=(n, 3))
    p = Params(theta=0.5, r_out=0.005, eps=1e-4, gamma=GAMMA)
    gx, gm, ox, om = _vjp_vs_oracle(pos, m, w, p)
    if n == 1:  # no pair at all
        assert np.all(gx == 0.0) and np.all(gm == 0.0)
        assert np.all(ox == 0.0) and np.all(om == 0.0)
        return
    ex = rel_err(gx, ox)
    em = _scalar_err(gm, om)
    assert np.median(ex) <= MED and ex.max() <= MAX_X, (np.median(ex), ex.max())
    assert np.median(em) <= MED and em.max() <= MAX_M, (np.median(em), em.max())


def test_vjp_coincident_particles(cuda):
    """Coincident particles with eps = 0 inside a Plummer sphere: their pairs
    have K(0) = 0, so they add nothing to the force or its derivative (the
    backward's near terms must not form 0 * inf); the rest matches the
    oracle."""
    from paper_1506_04553_b300 import Params
    n = 4096
    pos, _, m = ics.plummer(n, 21)
    pos = pos.T.copy()
    pos[:80] = pos[0]  # a leaf of 80 coincident particles, a chain above it
    w = np.random.default_rng(22).normal(size=(n, 3))
    p = Params(theta=0.4, r_out=0.01, eps=0.0, gamma=GAMMA)
    gx, gm, ox, om = _vjp_vs_oracle(pos, m, w, p)
    assert np.all(np.isfinite(gx)) and np.all(np.isfinite(gm))
    ex = rel_err(gx, ox)
    em = _scalar_err(gm, om)
    assert np.median(ex) <= MED and ex.max() <= MAX_X, (np.median(ex), ex.max())
    assert np.median(em) <= MED and em.max() <= MAX_M, (np.median(em), em.max())
