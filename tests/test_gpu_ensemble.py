"""Ensembles of independent clusters (p3t_set_ensemble): every cluster must
give what the oracle gives for that cluster alone (structure and lists
bit-exact, forces within the usual tolerances, gradients within about three
times the largest errors measured, neighbour lists bit-exact), including a
one-particle and a two-particle cluster; and a step captured in a CUDA graph
must replay to the same forces."""
import numpy as np
import pytest

import oracle
from paper_1506_04553_b300 import ics
from parity_util import rel_err

pytestmark = pytest.mark.gpu


def _ensemble():
    pos, vel, m, off = ics.plummer_ensemble(10, seed=900, n_min=64, n_max=4096)
    # add a one-particle and a two-particle cluster
    extra = np.array([[0.3, 0.1, -0.2], [0.0, 0.0, 0.0], [0.001, 0.0, 0.0]]).T
    pos = np.concatenate([pos, extra], axis=1)
    m = np.concatenate([m, [1.0, 0.5, 0.5]])
    off = np.concatenate([off, [off[-1] + 1, off[-1] + 3]])
    nc = off.size - 1
    sizes = np.diff(off)
    r_out = 0.01 * (np.maximum(sizes, 2) / 8192.0) ** (-1.0 / 3.0)
    eps = 4.0 / sizes
    return pos, m, off, r_out, eps


@pytest.fixture(scope="module")
def ens(cuda):
    import torch
    from paper_1506_04553_b300 import Context, Params
    pos, m, off, r_out, eps = _ensemble()
    n = pos.shape[1]
    ctx = Context(Params(theta=0.4))
    ctx.set_ensemble(off, r_out=r_out, eps=eps)
    pd = torch.tensor(pos, device="cuda")
    md = torch.tensor(m, device="cuda")
    ctx.build_tree(pd, md)
    acc = ctx.long_force().cpu().numpy().T.astype(np.float64)
    o, i = ctx.neighbours()
    w = np.random.default_rng(5).normal(size=(n, 3))
    gx, gm = ctx.long_force_vjp(torch.tensor(w.T.copy(), dtype=torch.float32, device="cuda"))
    return dict(ctx=ctx, pos=pos, m=m, off=off, r_out=r_out, eps=eps, acc=acc,
                ngb=(o.cpu().numpy(), i.cpu().numpy()), w=w,
                gx=gx.cpu().numpy().T.copy(), gm=gm.cpu().numpy(), pd=pd, md=md)


def test_each_cluster_matches_its_own_oracle(ens):
    ctx = ens["ctx"]
    key_g, order_g = ctx.order()
    cells = ctx.cells()
    groups = ctx.groups()
    off = ens["off"]
    for k in range(off.size - 1):
        b, e = int(off[k]), int(off[k + 1])
        p = ens["pos"][:, b:e].T.copy()
        mk = ens["m"][b:e]
        t = oracle.Tree(p, mk)
        t.walk(0.4, ens["r_out"][k], ens["r_out"][k])
        key_o, order_o = t.particles()
        assert np.array_equal(key_g[b:e], key_o)
        assert np.array_equal(order_g[b:e].astype(np.int64), order_o + b)
        co = t.cells()
        sel = (cells["first"] >= b) & (cells["first"] < e)
        gset = set(zip(cells["level"][sel].tolist(), (cells["first"][sel] - b).tolist(),
                       cells["count"][sel].tolist()))
        oset = set(zip(co["level"].tolist(), co["first"].tolist(), co["count"].tolist()))
        assert gset == oset
        go = t.groups()
        gsel = (groups["first"] >= b) & (groups["first"] < e)
        assert sorted((groups["first"][gsel] - b).tolist()) == sorted(go["first"].tolist())
        a_o = t.force(eps=ens["eps"][k], r_cut=ens["r_out"][k])
        if e - b > 1:
            err = rel_err(ens["acc"][b:e], a_o)
            assert np.median(err) <= 1e-5 and err.max() <= 1e-4, (k, err.max())
        else:
            assert np.all(ens["acc"][b:e] == 0.0)
        off_g, idx_g = ens["ngb"]
        off_o, idx_o = oracle.neighbours(p, ens["r_out"][k])
        for r in range(e - b):
            row = idx_g[off_g[b + r]:off_g[b + r + 1]]
            assert np.array_equal(row, idx_o[off_o[r]:off_o[r + 1]] + b)
        ox, om = t.vjp(ens["w"][b:e], eps=ens["eps"][k], r_cut=ens["r_out"][k])
        if e - b > 1:
            ex = rel_err(ens["gx"][b:e], ox)
            floor = 1e-3 * np.sqrt(np.mean(om ** 2))
            em = np.abs(ens["gm"][b:e] - om) / np.maximum(np.abs(om), floor)
            print(f"cluster {k} (N = {e - b}): dL/dx max {ex.max():.2e}, "
                  f"dL/dm max {em.max():.2e}")
            # about three times the largest measured (7.3e-5 and 4.4e-4)
            assert np.median(ex) <= 1e-5 and ex.max() <= 2e-4, (k, ex.max())
            assert np.median(em) <= 1e-5 and em.max() <= 1.5e-3, (k, em.max())


def test_graph_capture_replays_the_step(ens):
    import torch
    from paper_1506_04553_b300 import Context, FLAG_NO_SYNC, Params
    pos, m, off, r_out, eps = _ensemble()
    n = pos.shape[1]
    ctx = Context(Params(theta=0.4))
    ctx.set_ensemble(off, r_out=r_out, eps=eps)
    pd = torch.tensor(pos, device="cuda")
    md = torch.tensor(m, device="cuda")
    acc = torch.empty((3, n), dtype=torch.float32, device="cuda")
    w = torch.ones((3, n), dtype=torch.float32, device="cuda")
    gx = torch.empty((3, n), dtype=torch.float64, device="cuda")
    gm = torch.empty((n,), dtype=torch.float64, device="cuda")
    ctx.build_tree(pd, md)          # sizes the buffers
    ctx.long_force(acc)
    ctx.long_force_vjp(w, gx, gm)
    ctx.set_params(Params(theta=0.4, flags=FLAG_NO_SYNC))
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):      # warm-up on the capture stream
        ctx.build_tree(pd, md)
        ctx.long_force(acc, check=False)
    torch.cuda.current_stream().wait_stream(s)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        ctx.build_tree(pd, md)
        ctx.long_force(acc, check=False)
        ctx.long_force_vjp(w, gx, gm, check=False)
    # new positions in the static input, replay, compare with a plain call
    rng = np.random.default_rng(1)
    pos2 = pos + 1e-3 * rng.normal(size=pos.shape)
    pd.copy_(torch.tensor(pos2, device="cuda"))
    g.replay()
    torch.cuda.synchronize()
    ctx.check()
    acc_graph = acc.clone()
    ref = Context(Params(theta=0.4))
    ref.set_ensemble(off, r_out=r_out, eps=eps)
    ref.build_tree(pd, md)
    acc_ref = ref.long_force()
    assert torch.equal(acc_graph, acc_ref)


def test_full_ensemble_sampled_clusters(cuda):
    """The batched workload itself: 256 Plummer clusters with N_c
    log-uniform in [1024, 65536] (3.9 M particles), r_out = 0.01
    (N_c / 8192)^(-1/3), eps 4 / N_c, theta 0.4, in one context and one
    launch per kernel.  Eight clusters spanning the sizes (the smallest and
    the largest included) against the oracle run on each cluster alone:
    forces within the usual tolerances (median 1e-5, max 1e-4), gradients of
    sum w.a with median 1e-5 and maxima three times the measured ones."""
    import torch
    from paper_1506_04553_b300 import Context, Params
    pos, _, m, off = ics.plummer_ensemble(256, seed=5000)
    n = int(off[-1])
    sizes = np.diff(off)
    r_out = 0.01 * (sizes / 8192.0) ** (-1.0 / 3.0)
    eps = 4.0 / sizes
    ctx = Context(Params(theta=0.4))
    ctx.set_ensemble(off, r_out=r_out, eps=eps)
    ctx.build_tree(torch.tensor(pos, device="cuda"), torch.tensor(m, device="cuda"))
    acc = ctx.long_force().cpu().numpy().T.astype(np.float64)
    w = np.random.default_rng(41).normal(size=(n, 3)).astype(np.float32)
    gx, gm = ctx.long_force_vjp(torch.tensor(w.T.copy(), device="cuda"))
    gx, gm = gx.cpu().numpy().T, gm.cpu().numpy()
    order = np.argsort(sizes, kind="stable")
    pick = order[np.round(np.linspace(0, len(sizes) - 1, 8)).astype(int)]
    assert sizes[pick[-1]] == sizes.max() and sizes[pick[0]] == sizes.min()
    for c in pick:
        b, e = int(off[c]), int(off[c + 1])
        t = oracle.Tree(pos[:, b:e].T.copy(), m[b:e])
        t.walk(0.4, r_out[c], r_out[c])
        a_o = t.force(eps=eps[c], r_cut=r_out[c])
        err = rel_err(acc[b:e], a_o)
        assert np.median(err) <= 1e-5 and err.max() <= 1e-4, (c, e - b, err.max())
        ox, om = t.vjp(w[b:e].astype(np.float64), eps=eps[c], r_cut=r_out[c])
        ex = rel_err(gx[b:e], ox)
        em = rel_err(gm[b:e, None], om[:, None])
        # about three times the largest values measured over these clusters
        # (dL/dx 6.4e-5, dL/dm 1.9e-3)
        assert np.median(ex) <= 1e-5 and ex.max() <= 2e-4, (c, ex.max())
        assert np.median(em) <= 1e-5 and em.max() <= 6e-3, (c, em.max())
        print(f"cluster {c} (N = {e - b}): force max {err.max():.1e}, dL/dx max "
              f"{ex.max():.1e}, dL/dm max {em.max():.1e}")
