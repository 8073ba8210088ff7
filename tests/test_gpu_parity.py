"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Bit-exact: Morton keys, sort order, root cube, cell and group structure, FP32
boxes, interaction-list sets, neighbour lists, kick and drift.
Within tolerance: forces against the same-tree FP64 oracle (per-particle
relative error, floor 1e-3 rms: median <= 1e-5, max <= 1e-4), moments.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1506_04553_b300 import ics
from parity_util import compare_lists, compare_structure, gpu_run, rel_err

pytestmark = pytest.mark.gpu

GAMMA = 0.1


def _params(**kw):
    from paper_1506_04553_b300 import Params
    return Params(**kw)


def _plummer(n, seed):
    pos, vel, m = ics.plummer(n, seed)
    return pos.T.copy(), vel, m


CASES = {
    # config 1: Plummer N = 8192, r_out = 0.01, theta = 0.4, eps = 4/N
    "plummer8192": lambda: (*_plummer(8192, 1)[::2], dict(
        theta=0.4, r_out=0.01, eps=4 / 8192)),
    "plummer3000_theta0.6": lambda: (*_plummer(3000, 7)[::2], dict(
        theta=0.6, r_out=0.02, eps=1e-3, n_leaf=8, n_group=32)),
    "gauss_dense": lambda: (np.random.default_rng(3).normal(size=(5000, 3)) * 0.05,
                            np.random.default_rng(4).uniform(0.5, 1.5, 5000) / 5000,
                            dict(theta=0.5, r_out=0.01, eps=0.0, h=0.012)),
}


@pytest.fixture(scope="module", params=sorted(CASES))
def case(request, cuda):
    pos, m, kw = CASES[request.param]()
    p = _params(**kw)
    ctx, acc, pot, ngb = gpu_run(pos, m, p, potential=True)
    t = oracle.Tree(pos, m, n_leaf=p.n_leaf, n_group=p.n_group)
    h = p.h if p.h > 0 else p.r_out
    t.walk(p.theta, h, p.r_out)
    return dict(name=request.param, pos=pos, m=m, p=p, ctx=ctx, acc=acc,
                pot=pot, ngb=ngb, tree=t, h=h)


def test_structure_bitexact(case):
    compare_structure(case["ctx"], case["tree"])


def test_lists_identical(case):
    # the fused walk+force kernel's counts (taken before the inspection walk
    # overwrites them) and the inspection lists both match the oracle
    st = case["ctx"].stats()
    og, gid = compare_structure(case["ctx"], case["tree"])
    compare_lists(case["ctx"], case["tree"], og, gid)
    L = case["tree"].lists()
    assert st["list_pc"] == L["pc"].size
    assert st["list_pp_near"] == L["ppn"].size
    assert st["list_pp_far"] == L["ppf"].size


def test_fused_kernel_lists_identical(case):
    """The sources the timed walk + force kernel itself evaluates (recorded by
    an instantiation of the same kernel) are, group by group, the oracle's
    interaction lists: cells, near-leaf and far-leaf particles."""
    ctx, tree = case["ctx"], case["tree"]
    og, gid = compare_structure(ctx, tree)
    F, Lo = ctx.force_lists(), tree.lists()
    for g in range(tree.ngroup):
        q = gid[g]
        pc_o = og[Lo["pc"][Lo["pc_off"][g]:Lo["pc_off"][g + 1]]]
        pc_g = F["pc"][F["pc_off"][q]:F["pc_off"][q + 1]]
        assert sorted(pc_o.tolist()) == pc_g.tolist(), f"cells of group {g}"
        for name in ("ppn", "ppf"):
            lo_ = Lo[name][Lo[name + "_off"][g]:Lo[name + "_off"][g + 1]]
            lg_ = F[name][F[name + "_off"][q]:F[name + "_off"][q + 1]]
            assert sorted(lo_.tolist()) == lg_.tolist(), f"{name} of group {g}"
    assert F["pc"].size == Lo["pc"].size and F["ppf"].size == Lo["ppf"].size


def test_force_matches_same_tree_oracle(case):
    p = case["p"]
    a_o, p_o = case["tree"].force(G=p.G, eps=p.eps, r_cut=p.r_out,
                                  gamma=p.gamma, potential=True)
    e = rel_err(case["acc"], a_o)
    assert np.median(e) <= 1e-5, np.median(e)
    assert e.max() <= 1e-4, e.max()
    ep = np.abs(case["pot"] - p_o) / np.abs(p_o)
    assert np.median(ep) <= 1e-5 and ep.max() <= 1e-4, (np.median(ep), ep.max())


def test_neighbours_bitexact(case):
    off, idx = case["ngb"]
    off_o, idx_o = oracle.neighbours(case["pos"], case["h"])
    assert np.array_equal(off, off_o)
    assert np.array_equal(idx.astype(np.int64), idx_o.astype(np.int64))
    if case["name"] == "gauss_dense":
        assert off[-1] > 5 * case["pos"].shape[0]  # several neighbours each
        # rows kept by the counting walk (at most 8) and rows filled by the
        # second walk over the listed groups both occur
        rl = np.diff(off)
        assert ((rl > 0) & (rl <= 8)).sum() > 100 and (rl > 8).sum() > 100


def test_theta_zero_equals_direct_sum(cuda):
    pos, _, m = ics.plummer(4096, 12)
    pos = pos.T.copy()
    p = _params(theta=0.0, r_out=0.01, eps=4 / 4096)
    ctx, acc, pot, _ = gpu_run(pos, m, p, potential=True)
    assert ctx.stats()["list_pc"] == 0
    a_d, p_d = oracle.direct(pos, m, G=1.0, eps=p.eps, r_cut=p.r_out,
                             gamma=GAMMA, kind="soft", potential=True)
    e = rel_err(acc, a_d)
    assert np.median(e) <= 1e-5 and e.max() <= 1e-4, (np.median(e), e.max())


def test_error_vs_direct_consistent_with_theta(cuda):
    pos, _, m = ics.plummer(8192, 1)
    pos = pos.T.copy()
    a_d = oracle.direct(pos, m, eps=4 / 8192, r_cut=0.01, gamma=GAMMA)
    meds = []
    for th in (0.8, 0.4, 0.2):
        _, acc, _, _ = gpu_run(pos, m, _params(theta=th, r_out=0.01, eps=4 / 8192),
                               neighbours=False)
        meds.append(np.median(rel_err(acc, a_d)))
    assert meds[0] > meds[1] > meds[2]
    assert meds[1] < 2e-3


def test_kick_drift_bitexact(cuda):
    import torch
    from paper_1506_04553_b300 import drift, kick
    rng = np.random.default_rng(8)
    v = rng.normal(size=(3, 10001))
    x = rng.normal(size=(3, 10001))
    a = rng.normal(size=(3, 10001)).astype(np.float32)
    vd = torch.tensor(v, device="cuda")
    xd = torch.tensor(x, device="cuda")
    ad = torch.tensor(a, device="cuda")
    kick(vd, ad, 1 / 512)
    drift(xd, vd, 1 / 256)
    v1 = oracle.kick(v, a, 1 / 512)
    x1 = oracle.drift(x, v1, 1 / 256)
    assert np.array_equal(vd.cpu().numpy(), v1)
    assert np.array_equal(xd.cpu().numpy(), x1)


def test_energy(cuda):
    import torch
    pos, vel, m = ics.plummer(4096, 5)
    p = _params(theta=0.4, r_out=0.01, eps=4 / 4096)
    ctx, acc, pot, _ = gpu_run(pos.T.copy(), m, p, potential=True,
                               neighbours=False)
    out = ctx.energy(torch.tensor(m, device="cuda"),
                     torch.tensor(vel, device="cuda"),
                     torch.tensor(pot, device="cuda")).cpu().numpy()
    ek = 0.5 * float((m * (vel * vel).sum(axis=0)).sum())
    ep = 0.5 * float((m * pot).sum())
    assert abs(out[0] - ek) <= 1e-12 * abs(ek)
    assert abs(out[1] - ep) <= 1e-12 * abs(ep)


@pytest.mark.parametrize("n", [1, 2, 16, 17, 65, 300])
def test_small_sizes(cuda, n):
    rng = np.random.default_rng(n)
    pos = rng.normal(size=(n, 3)) * 0.01
    m = rng.uniform(0.5, 1.5, n) / n
    p = _params(theta=0.5, r_out=0.005, eps=1e-4)
    ctx, acc, _, ngb = gpu_run(pos, m, p)
    t = oracle.Tree(pos, m)
    t.walk(p.theta, p.r_out, p.r_out)
    og, gid = compare_structure(ctx, t)
    compare_lists(ctx, t, og, gid)
    a_o = t.force(eps=p.eps, r_cut=p.r_out)
    if n > 1:
        e = rel_err(acc, a_o)
        assert e.max() <= 1e-4
    else:
        assert np.all(acc == 0.0)
    off_o, idx_o = oracle.neighbours(pos, p.r_out)
    assert np.array_equal(ngb[0], off_o) and np.array_equal(ngb[1], idx_o)


def test_coincident_particles(cuda):
    # all particles at one point: the tree is a chain down to level 21, every
    # pair has K(0) = 0 (force exactly zero) and every pair is a neighbour
    n = 100
    pos = np.full((n, 3), 0.25)
    m = np.full(n, 1.0 / n)
    p = _params(theta=0.4, r_out=0.01, eps=0.0, n_leaf=16, n_group=32)
    ctx, acc, _, ngb = gpu_run(pos, m, p)
    assert np.all(acc == 0.0)
    t = oracle.Tree(pos, m, n_leaf=16, n_group=32)
    t.walk(p.theta, p.r_out, p.r_out)
    og, gid = compare_structure(ctx, t)
    compare_lists(ctx, t, og, gid)
    off, idx = ngb
    assert off[-1] == n * (n - 1)
    off_o, idx_o = oracle.neighbours(pos, p.r_out)
    assert np.array_equal(off, off_o) and np.array_equal(idx, idx_o)


def test_deep_chain_inside_a_cluster(cuda):
    """A Plummer sphere with 80 coincident particles inside: a chain of
    single-child cells down to level 21 ending in a leaf of 80 particles (more
    than any leaf size bin below it) among ordinary leaves.  The bottom-up
    moments climb the chain; cells, boxes and moments match the oracle."""
    pos, _, m = ics.plummer(4000, 31)
    pos = pos.T.copy()
    pos[:80] = 0.0123
    m = np.full(4000, 1.0 / 4000)
    p = _params(theta=0.5, r_out=0.01, eps=1e-3)
    ctx, acc, _, _ = gpu_run(pos, m, p, neighbours=False)
    t = oracle.Tree(pos, m, n_leaf=p.n_leaf, n_group=p.n_group)
    t.walk(p.theta, p.r_out, p.r_out)
    og, gid = compare_structure(ctx, t)
    compare_lists(ctx, t, og, gid)
    assert ctx.stats()["n_levels"] == 22
    a_o = t.force(G=p.G, eps=p.eps, r_cut=p.r_out, gamma=p.gamma)
    e = rel_err(acc, a_o)
    assert np.median(e) <= 1e-5 and e.max() <= 1e-4, (np.median(e), e.max())


def test_force_and_neighbours_concurrently(cuda):
    """p3t_long_force and p3t_neighbours on two streams after one build (each
    walk has its own work counter) give bit for bit the sequential results,
    also on a dense case with long neighbour rows."""
    import torch
    from paper_1506_04553_b300 import Context
    pos = np.random.default_rng(3).normal(size=(20000, 3)) * 0.05
    m = np.full(20000, 1.0 / 20000)
    ctx = Context(_params(theta=0.5, r_out=0.006, eps=1e-4, h=0.008))
    pd = torch.tensor(pos.T.copy(), device="cuda")
    md = torch.tensor(m, device="cuda")
    ctx.build_tree(pd, md)
    n = pos.shape[0]
    acc_s = torch.empty((3, n), dtype=torch.float32, device="cuda")
    ctx.long_force(acc_s)
    off_s, idx_s = ctx.neighbours()
    nnz = int(off_s[-1])
    assert int((torch.diff(off_s) > 8).sum()) > 1000  # long rows: the second walk runs
    acc_c = torch.empty_like(acc_s)
    off_c = torch.empty_like(off_s)
    idx_c = torch.empty((nnz + 1024,), dtype=torch.int32, device="cuda")
    side = torch.cuda.Stream()
    for _ in range(3):
        side.wait_stream(torch.cuda.current_stream())
        ctx.long_force(acc_c, check=False)
        with torch.cuda.stream(side):
            ctx.neighbours_into(off_c, idx_c, sync=False)
        torch.cuda.current_stream().wait_stream(side)
        torch.cuda.synchronize()
        ctx.check()
        assert torch.equal(acc_c, acc_s)
        assert torch.equal(off_c, off_s)
        assert torch.equal(idx_c[:nnz], idx_s)


def test_exact_distance_ties(cuda):
    # pairs at exactly r = h (excluded) and just inside (included)
    h = 0.5
    pos = np.array([[0.0, 0.0, 0.0], [0.5, 0.0, 0.0], [0.0, 0.3, 0.4],
                    [0.0, -0.3, 0.39999], [0.0, 0.0, 0.0], [0.1, 0.1, 0.1]])
    m = np.full(6, 1 / 6)
    p = _params(theta=0.4, r_out=0.5, h=h, eps=0.0)
    _, _, _, ngb = gpu_run(pos, m, p)
    off_o, idx_o = oracle.neighbours(pos, h)
    assert np.array_equal(ngb[0], off_o) and np.array_equal(ngb[1], idx_o)


def test_keys_on_quantisation_boundaries(cuda):
    """Coordinates on, and up to 3 ulp either side of, the boundaries of the
    2^21 quantisation cells of a cube whose side makes the GPU's product
    (x - lo) (2^21 / side) and the definition's quotient floor differently
    for some of them: the division must decide there.  Keys are compared bit
    for bit with the oracle."""
    rng = np.random.default_rng(21)
    n = 8000
    ext = 1.4376431999070005
    side = ext * (1.0 + 2.0 ** -20)
    pos = rng.uniform(0.0, ext, size=(n, 3))
    pos[0] = 0.0
    pos[1] = ext  # extent ext on every axis, lo = 0
    k = rng.integers(1, 2 ** 21 - 1, size=n - 2)
    x = k * side / 2.0 ** 21
    for _ in range(3):  # move each coordinate by -3 .. +3 ulp
        step = rng.integers(-1, 2, size=n - 2)
        x = np.where(step < 0, np.nextafter(x, -1.0),
                     np.where(step > 0, np.nextafter(x, 2.0), x))
    x = np.clip(x, 0.0, ext)
    pos[2:, 0] = x
    pos[2:, 1] = np.roll(x, 17)
    m = np.full(n, 1.0 / n)
    p = _params(theta=0.5, r_out=0.01, eps=1e-3)
    ctx, _, _, _ = gpu_run(pos, m, p, neighbours=False)
    t = oracle.Tree(pos, m, n_leaf=p.n_leaf, n_group=p.n_group)
    _, size_g = ctx.root()
    assert size_g == side
    key_g, _ = ctx.order()
    key_o, _ = t.particles()
    assert np.array_equal(key_g, key_o)
    # cases where the product and the quotient floor differently do occur
    q_div = np.floor((x / side) * 2.0 ** 21)
    q_mul = np.floor((x * (1.0 / side)) * 2.0 ** 21)
    assert np.count_nonzero(q_div != q_mul) > 20


def test_empty_input(cuda):
    import torch
    from paper_1506_04553_b300 import Context
    ctx = Context(_params())
    e = torch.zeros((3, 0), dtype=torch.float64, device="cuda")
    ctx.build_tree(e, torch.zeros((0,), dtype=torch.float64, device="cuda"))
    acc = ctx.long_force()
    assert acc.shape == (3, 0)
    off, idx = ctx.neighbours()
    assert off.cpu().tolist() == [0] and idx.numel() == 0


def test_errors(cuda):
    import torch
    from paper_1506_04553_b300 import Context, P3TError
    ctx = Context(_params())
    with pytest.raises(P3TError) as ei:
        ctx.long_force(torch.zeros((3, 0), dtype=torch.float32, device="cuda"))
    assert ei.value.code == 5  # force before build
    pos = torch.zeros((3, 10), dtype=torch.float64, device="cuda")
    pos[0, 3] = float("nan")
    with pytest.raises(P3TError) as ei:
        ctx.build_tree(pos, torch.ones(10, dtype=torch.float64, device="cuda"))
    assert ei.value.code == 1
    pos[0, 3] = 0.0
    with pytest.raises(P3TError) as ei:
        ctx.build_tree(pos, -torch.ones(10, dtype=torch.float64, device="cuda"))
    assert ei.value.code == 1
    # valid input after errors works again
    ctx.build_tree(torch.rand((3, 10), dtype=torch.float64, device="cuda"),
                   torch.ones(10, dtype=torch.float64, device="cuda"))
    ctx.long_force()
    # neighbour capacity too small
    off = torch.zeros(11, dtype=torch.int64, device="cuda")
    idx = torch.zeros(1, dtype=torch.int32, device="cuda")
    ctx2 = Context(_params(r_out=10.0))
    ctx2.build_tree(torch.rand((3, 10), dtype=torch.float64, device="cuda"),
                    torch.ones(10, dtype=torch.float64, device="cuda"))
    ctx2.long_force()
    with pytest.raises(P3TError) as ei:
        ctx2.neighbours_into(off, idx)
    assert ei.value.code == 2


def test_group_order_changes_nothing(cuda):
    """The group kernels take the groups most expensive first, estimated from
    the previous force evaluation; the first build of a context has no
    estimate and takes them in index order.  Each group's sums do not depend
    on that order, so forces, potentials, neighbour lists and interaction
    counts are bit-identical across the two; the backward pass adds the
    groups' contributions with FP64 atomics in whatever order they arrive, so
    its gradients agree to FP64 rounding."""
    import torch
    from paper_1506_04553_b300 import Context
    pos, _, m = _plummer(20000, 12)
    ctx = Context(_params(theta=0.4, r_out=0.01, eps=1e-4))
    pd = torch.tensor(np.ascontiguousarray(pos.T), device="cuda")
    md = torch.tensor(m, device="cuda")
    w = torch.randn((3, pos.shape[0]), generator=torch.Generator().manual_seed(5)).float().cuda()
    runs = []
    for _ in range(3):  # index order, then twice with recorded costs
        ctx.build_tree(pd, md)
        acc, pot = ctx.long_force(want_potential=True)
        off, idx = ctx.neighbours()
        gx, gm = ctx.long_force_vjp(w)
        st = ctx.stats()
        runs.append([t.cpu().numpy() for t in (acc, pot, off, idx, gx, gm)]
                    + [st["int_pc"], st["int_pp"], st["int_pp_near"]])
    for r in runs[1:]:
        for a, b in zip(runs[0][:4], r[:4]):
            assert np.array_equal(a, b)
        for a, b in zip(runs[0][4:6], r[4:6]):
            assert np.allclose(a, b, rtol=1e-12, atol=1e-12 * np.abs(a).max())
        assert runs[0][6:] == r[6:]
