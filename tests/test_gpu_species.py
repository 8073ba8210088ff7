"""Two species on the GPU (p3t_set_species, Sect. 3.2.2: a star cluster
with black holes, a cut-off per kind of pair) against the oracle: neighbour
rows bit for bit (star pairs within h, black hole-star pairs within h_bh,
black hole pairs always); soft forces of the stars against the oracle's
tree over the stars plus the black holes' direct terms, and of the black
holes against direct sums; whole hard steps bit for bit with pair
constants per type and eta per species."""
import math

import numpy as np
import pytest

import oracle
from paper_1506_04553_b300 import ics
from parity_util import assert_hard_step_close, hermite_sensitivity, rel_err

pytestmark = pytest.mark.gpu

INF = math.inf
GAMMA = 0.1


def _system(n_star, seed, n_bh=2):
    """Plummer stars (N-body units) and n_bh black holes of 1% of the
    cluster's mass each, on a ring of radius 0.5 with speed 0.5 (the
    binary of Sect. 3.2.2 for n_bh = 2)."""
    pos, vel, m = ics.plummer(n_star, seed)
    pos, vel = pos.T.copy(), vel.T.copy()
    ang = 2 * np.pi * np.arange(n_bh) / n_bh
    bp = np.stack([0.5 * np.cos(ang), 0.5 * np.sin(ang), np.zeros(n_bh)], 1)
    bv = np.stack([-0.5 * np.sin(ang), 0.5 * np.cos(ang), np.zeros(n_bh)], 1)
    return (np.concatenate([pos, bp]), np.concatenate([vel, bv]),
            np.concatenate([m, np.full(n_bh, 0.01)]))


P = dict(theta=0.4, r_out=0.01, h=0.0125, eps=1e-4)
SP = dict(r_cut_bh=1 / 32, eps_bh=1e-4, h_bh=1 / 32 + 0.01, eta_bh=0.03)


def _ctx(n, n_bh, **kw):
    from paper_1506_04553_b300 import Context, Params
    ctx = Context(Params(gamma=GAMMA, **{**P, **kw}))
    ctx.set_species(n, n_bh, **SP)
    return ctx


def _dev(a, dtype=None):
    import torch
    t = torch.tensor(np.ascontiguousarray(a))
    return (t.to(dtype) if dtype is not None else t).cuda()


@pytest.mark.parametrize("n_bh", [1, 2, 5])
def test_species_neighbours_bitexact(cuda, n_bh):
    pos, _, m = _system(20000, 21, n_bh)
    # put one black hole in the core so that its row is long
    pos[-1] = [0.01, -0.02, 0.0]
    n = pos.shape[0]
    ctx = _ctx(n, n_bh)
    ctx.build_tree(_dev(pos.T), _dev(m))
    ctx.long_force()
    off, idx = ctx.neighbours()
    off, idx = off.cpu().numpy(), idx.cpu().numpy()
    off_o, idx_o = oracle.neighbours_species(pos, n_bh, h=[P["h"], SP["h_bh"], INF])
    assert np.array_equal(off, off_o)
    assert np.array_equal(idx, idx_o)
    assert off_o[-1] - off_o[-2] > 5  # the core black hole's row


def test_species_soft_force(cuda):
    pos, _, m = _system(30000, 22)
    pos[-1] = [0.02, 0.01, -0.01]
    n, n_bh = pos.shape[0], 2
    nfs = n - n_bh
    ctx = _ctx(n, n_bh)
    ctx.build_tree(_dev(pos.T), _dev(m))
    acc = ctx.long_force().cpu().numpy().astype(np.float64).T
    # stars: the tree over the stars (same lists) plus the black holes
    t = oracle.Tree(pos[:nfs], m[:nfs], n_leaf=16, n_group=64)
    t.walk(P["theta"], P["h"], P["r_out"])
    a_tree = t.force(eps=P["eps"], r_cut=P["r_out"], gamma=GAMMA)
    kw = dict(eps=[P["eps"], SP["eps_bh"], 0.0], r_cut=[P["r_out"], SP["r_cut_bh"], INF],
              gamma=GAMMA, kind="soft")
    m_bh_only = m.copy()
    m_bh_only[:nfs] = 0.0
    a_cross = oracle.direct_species(pos, m_bh_only, n_bh, rows=np.arange(nfs), **kw)
    e = rel_err(acc[:nfs], a_tree + a_cross)
    assert np.median(e) <= 1e-5 and e.max() <= 1e-4, (np.median(e), e.max())
    # black holes: stars only (no soft force between black holes)
    a_bh = oracle.direct_species(pos, m, n_bh, rows=np.arange(nfs, n), **kw)
    assert np.allclose(acc[nfs:], a_bh, rtol=1e-6, atol=0)
    # the core black hole's stars within r_cut_bh are weighted by K < 1
    assert np.linalg.norm(a_cross, axis=1).max() > 0.1


@pytest.mark.parametrize("where", ["core", "far"])
def test_species_hard_step(cuda, where):
    """A tight black hole binary in the core (one component of the binary
    and many stars: the per-component warp path) or far out (the binary
    alone: a packed warp).  Against the plain oracle within 16 times its
    response to one-ulp input perturbations; against the fused-order mirror
    bit for bit."""
    import torch
    from paper_1506_04553_b300 import HermiteParams
    pos, vel, m = _system(6000, 23)
    c = 0.0 if where == "core" else 3.0
    pos[-1] = [c + 0.005, 0.0, 0.0]
    pos[-2] = [c - 0.005, 0.0, 0.0]
    vel[-1] = [0.0, 0.9, 0.0]
    vel[-2] = [0.0, -0.9, 0.0]
    n, n_bh = pos.shape[0], 2
    h = [0.02, 0.15 if where == "core" else 0.05, INF]
    off, idx = oracle.neighbours_species(pos, n_bh, h=h)
    eps = [1e-4, 1e-4, 0.0]
    r_cut = [0.016, 1 / 32, INF]
    hp = HermiteParams(dt_soft=1 / 256, eta=0.1, alpha=0.1)
    okw = dict(dt_soft=hp.dt_soft, eps=eps, r_cut=r_cut, eta=[0.1, 0.03],
               gamma=GAMMA, alpha=0.1, p=hp.log2_soft_over_max, kmax=hp.kmax)
    xm, vm, sm = oracle.hermite_species(pos, vel, m, off, idx, n_bh, mirror=True, **okw)
    _, _, st, det = oracle.hermite_species(pos, vel, m, off, idx, n_bh, detail=True, **okw)
    x0, v0, sx, sv = hermite_sensitivity(
        lambda p, v: oracle.hermite_species(p, v, m, off, idx, n_bh, **okw)[:2],
        pos, vel)
    from paper_1506_04553_b300 import Context, Params
    ctx = Context(Params(r_out=r_cut[0], eps=eps[0], gamma=GAMMA))
    ctx.set_species(n, n_bh, r_cut_bh=r_cut[1], eps_bh=eps[1], h_bh=h[1], eta_bh=0.03)
    pg, vg = _dev(pos.T), _dev(vel.T)
    ctx.hard_step(pg, vg, _dev(m), _dev(off), _dev(idx, torch.int32), hp)
    s = ctx.stats()
    xg, vg = pg.cpu().numpy().T, vg.cpu().numpy().T
    assert det["margin"].min() > 1e-10  # no level decision near a tie
    assert_hard_step_close(xg, vg, x0, v0, sx, sv)
    assert (s["herm_particle_steps"], s["herm_pairs"], s["herm_capped"]) == st[1:]
    assert np.array_equal(xg, xm)
    assert np.array_equal(vg, vm)
    assert (s["herm_particle_steps"], s["herm_pairs"], s["herm_capped"]) == sm[1:]
    comp = s["herm_max_component"]
    assert (comp > 32) if where == "core" else (comp <= 32)


def test_species_argument_checks(cuda):
    import torch
    from paper_1506_04553_b300 import Context, P3TError, Params
    ctx = Context(Params(r_out=0.01))
    for bad in (dict(n=10, n_bh=10), dict(n=10, n_bh=-1), dict(n=100, n_bh=33),
                dict(n=10, n_bh=2, r_cut_bh=0.0), dict(n=10, n_bh=2, eta_bh=0.0),
                dict(n=10, n_bh=2, h_bh=float("nan"))):
        kw = {"r_cut_bh": 0.03, "eps_bh": 0.0, "h_bh": 0.04, "eta_bh": 0.03, **bad}
        with pytest.raises(P3TError):
            ctx.set_species(**kw)
    pos, _, m = _system(500, 24)
    ctx.set_species(pos.shape[0], 2, **SP)
    ctx.build_tree(_dev(pos.T), _dev(m))
    with pytest.raises(P3TError):  # n must be the species layout's
        ctx.build_tree(_dev(pos[:400].T), _dev(m[:400]))
    ctx.build_tree(_dev(pos.T), _dev(m))
    ctx.long_force()
    w = torch.zeros((3, pos.shape[0]), dtype=torch.float32, device="cuda")
    with pytest.raises(P3TError) as ei:
        ctx.long_force_vjp(w)
    assert ei.value.code == 5
    ctx.set_species(0, 0)  # off again: a plain build of any n
    ctx.build_tree(_dev(pos[:400].T), _dev(m[:400]))
    ctx.long_force_vjp(torch.zeros((3, 400), dtype=torch.float32, device="cuda"))


def test_species_coincident_black_hole_and_star(cuda):
    """A black hole exactly on a star with eps_bh = 0: K(0) = 0, so the pair
    adds no force (as for coincident stars); the pair is a neighbour pair
    (distance 0 < h_bh); everything else matches the oracle."""
    from paper_1506_04553_b300 import Context, Params
    pos, _, m = _system(3000, 25, n_bh=1)
    pos[-1] = pos[17]
    n, nfs = pos.shape[0], pos.shape[0] - 1
    ctx = Context(Params(gamma=GAMMA, **P))
    ctx.set_species(n, 1, r_cut_bh=1 / 32, eps_bh=0.0, h_bh=0.04, eta_bh=0.03)
    ctx.build_tree(_dev(pos.T), _dev(m))
    acc = ctx.long_force().cpu().numpy().astype(np.float64).T
    assert np.all(np.isfinite(acc))
    kw = dict(eps=[P["eps"], 0.0, 0.0], r_cut=[P["r_out"], 1 / 32, INF], gamma=GAMMA,
              kind="soft")
    a_bh = oracle.direct_species(pos, m, 1, rows=np.array([n - 1]), **kw)
    assert np.allclose(acc[-1], a_bh[0], rtol=1e-6, atol=0)
    off, idx = ctx.neighbours()
    off_o, idx_o = oracle.neighbours_species(pos, 1, h=[P["h"], 0.04, INF])
    assert np.array_equal(off.cpu().numpy(), off_o)
    assert np.array_equal(idx.cpu().numpy(), idx_o)
    assert 17 in idx_o[off_o[-2]:off_o[-1]]


def test_species_p3t_step_in_a_graph(cuda):
    """A whole P3T step with black holes (half-kick, hard step, build,
    F_soft with the black hole terms, merged neighbour rows, half-kick),
    captured in a CUDA graph with P3T_FLAG_NO_SYNC, replays bit for bit what
    the same step gives uncaptured."""
    import torch
    from paper_1506_04553_b300 import (FLAG_NO_SYNC, Context, HermiteParams,
                                       Params, drift, kick)
    pos_h, vel_h, m_h = _system(8000, 26)
    pos_h[-1] = [0.01, 0.0, 0.0]
    n, n_bh = pos_h.shape[0], 2
    dt = 1 / 512
    mk = lambda flags=0: Params(theta=0.4, r_out=0.01, gamma=GAMMA, eps=1e-4,
                                h=0.0125, flags=flags)
    hp = HermiteParams(dt_soft=dt, eta=0.1, alpha=0.1)

    def state():
        return [_dev(pos_h.T), _dev(vel_h.T), _dev(m_h)]

    def setup(ctx, pos, vel, mass):
        ctx.set_species(n, n_bh, **SP)
        ctx.build_tree(pos, mass)
        acc = ctx.long_force()
        off, idx0 = ctx.neighbours()
        idx = torch.empty(4 * idx0.numel() + 1024, dtype=torch.int32, device="cuda")
        ctx.neighbours_into(off, idx)
        ctx.hard_step(pos.clone(), vel.clone(), mass, off, idx, hp)  # scratch
        return acc, off, idx

    def step(ctx, pos, vel, mass, acc, off, idx):
        kick(vel, acc, 0.5 * dt)
        ctx.hard_step(pos, vel, mass, off, idx, hp, check=False)
        ctx.build_tree(pos, mass)
        ctx.long_force(acc, check=False)
        ctx.neighbours_into(off, idx, sync=False)
        kick(vel, acc, 0.5 * dt)

    # uncaptured
    ca = Context(mk())
    pa, va, ma = state()
    acc_a, off_a, idx_a = setup(ca, pa, va, ma)
    ca.set_params(mk(FLAG_NO_SYNC))
    ca.set_species(n, n_bh, **SP)
    step(ca, pa, va, ma, acc_a, off_a, idx_a)
    torch.cuda.synchronize()
    ca.check()
    # captured
    cb = Context(mk())
    pb, vb, mb = state()
    acc_b, off_b, idx_b = setup(cb, pb, vb, mb)
    cb.set_params(mk(FLAG_NO_SYNC))
    cb.set_species(n, n_bh, **SP)
    p0, v0, a0 = pb.clone(), vb.clone(), acc_b.clone()
    o0, i0 = off_b.clone(), idx_b.clone()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        step(cb, pb, vb, mb, acc_b, off_b, idx_b)  # warm the stream
    torch.cuda.current_stream().wait_stream(s)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        step(cb, pb, vb, mb, acc_b, off_b, idx_b)
    for t, t0 in ((pb, p0), (vb, v0), (acc_b, a0), (off_b, o0), (idx_b, i0)):
        t.copy_(t0)
    g.replay()
    torch.cuda.synchronize()
    cb.check()
    nnz = int(off_a[-1])
    assert torch.equal(pa, pb) and torch.equal(va, vb)
    assert torch.equal(acc_a, acc_b)
    assert torch.equal(off_a, off_b)
    assert torch.equal(idx_a[:nnz], idx_b[:nnz])
    assert off_a[-1] - off_a[-2] > 0  # the core black hole has a row


def test_species_black_hole_binary_full_size(cuda):
    """The bench's black hole binary setup (2^17 stars, two black holes of
    0.01 at (+-0.5, 0, 0); r_cut 1/256 and 1/32, h = r_cut + 3 sigma
    dt_soft, dt_soft 1/1024) in the bench's launch configuration: the black
    hole rows and 2000 sampled star rows of the neighbour lists bit for bit,
    and the soft forces of the same rows, against the oracle."""
    from paper_1506_04553_b300 import Context, Params
    nfs, n_bh = 1 << 17, 2
    n = nfs + n_bh
    dt = 1.0 / 1024
    buf = 3 * dt / np.sqrt(2)
    r_fs, r_bh = 1 / 256, 1 / 32
    ps, _, ms = ics.plummer(nfs, 7000)
    pos = np.concatenate([ps.T, [[0.5, 0.0, 0.0], [-0.5, 0.0, 0.0]]])
    m = np.concatenate([ms, [0.01, 0.01]])
    ctx = Context(Params(theta=0.4, r_out=r_fs, gamma=GAMMA, eps=1e-4, h=r_fs + buf))
    ctx.set_species(n, n_bh, r_cut_bh=r_bh, eps_bh=1e-4, h_bh=r_bh + buf, eta_bh=0.03)
    ctx.build_tree(_dev(pos.T), _dev(m))
    acc = ctx.long_force().cpu().numpy().astype(np.float64).T
    off, idx = ctx.neighbours()
    off, idx = off.cpu().numpy(), idx.cpu().numpy()
    rows = np.sort(np.concatenate([np.random.default_rng(5).choice(nfs, 2000, replace=False),
                                   [nfs, nfs + 1]]))
    off_o, idx_o = oracle.neighbours_species(pos, n_bh, h=[r_fs + buf, r_bh + buf, INF],
                                             rows=rows)
    for q, r in enumerate(rows):
        assert np.array_equal(idx[off[r]:off[r + 1]], idx_o[off_o[q]:off_o[q + 1]]), r
    assert off[n] - off[nfs] > 2  # black hole rows hold stars
    kw = dict(eps=[1e-4, 1e-4, 0.0], r_cut=[r_fs, r_bh, INF], gamma=GAMMA, kind="soft")
    a_bh = oracle.direct_species(pos, m, n_bh, rows=np.arange(nfs, n), **kw)
    assert np.allclose(acc[nfs:], a_bh, rtol=1e-6, atol=0)
    t = oracle.Tree(pos[:nfs], m[:nfs], n_leaf=16, n_group=64)
    t.walk(0.4, r_fs + buf, r_fs)
    a_tree = t.force(eps=1e-4, r_cut=r_fs, gamma=GAMMA)
    srows = rows[rows < nfs]
    m_bh_only = m.copy()
    m_bh_only[:nfs] = 0.0
    a_cross = oracle.direct_species(pos, m_bh_only, n_bh, rows=srows, **kw)
    e = rel_err(acc[srows], a_tree[srows] + a_cross)
    assert np.median(e) <= 1e-5 and e.max() <= 1e-4, (np.median(e), e.max())
