"""The hard part on the GPU (p3t_hard_force, p3t_hard_step) against the FP64
oracle: both evaluate every FP64 operation in the same order with one
rounding each, so forces, jerks and whole Hermite steps (block-timestep
schedule included) agree bit for bit.  The component search is checked
against scipy's connected components."""
import numpy as np
import pytest
from scipy.sparse import csr_matrix
from scipy.sparse.csgraph import connected_components

import oracle
from paper_1506_04553_b300 import ics

pytestmark = pytest.mark.gpu

GAMMA = 0.1


def _dev(a, dtype=None):
    import torch
    t = torch.tensor(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def _gauss(n, seed, scale):
    rng = np.random.default_rng(seed)
    pos = rng.normal(size=(n, 3)) * scale
    vel = rng.normal(size=(n, 3)) * 0.3
    m = rng.uniform(0.5, 1.5, n) / n
    return pos, vel, m


def _plummer(n, seed):
    pos, vel, m = ics.plummer(n, seed)
    return pos.T.copy(), vel.T.copy(), m


def test_hard_force_bitwise(cuda):
    import torch
    from paper_1506_04553_b300 import hard_force
    pos, vel, m = _gauss(3000, 1, 0.05)
    r_cut, eps = 0.02, 1e-3
    off, idx = oracle.neighbours(pos, 1.25 * r_cut)
    a_o, j_o = oracle.hard_force(pos, vel, m, off, idx, eps=eps, r_cut=r_cut, gamma=GAMMA)
    a_g, j_g = hard_force(_dev(pos.T), _dev(vel.T), _dev(m), _dev(off),
                          _dev(idx, torch.int32), r_cut=r_cut, eps=eps, gamma=GAMMA)
    assert off[-1] > 10000
    assert np.array_equal(a_g.cpu().numpy().T, a_o)
    assert np.array_equal(j_g.cpu().numpy().T, j_o)


def _clumps(seed):
    """Separated clumps of 2..40 particles, some fully connected (rows up to
    39 long), some split into smaller components: every packing size, rows
    longer than the packed limit, and components of more than 32."""
    rng = np.random.default_rng(seed)
    sizes = np.concatenate([np.arange(2, 33), np.arange(2, 33), [33, 40]])
    pos, vel = [], []
    for c, s in enumerate(sizes):
        scale = rng.uniform(0.003, 0.02)
        pos.append(rng.normal(size=(s, 3)) * scale + [c * 1.0, 0.0, 0.0])
        vel.append(rng.normal(size=(s, 3)) * 0.05)
    pos, vel = np.concatenate(pos), np.concatenate(vel)
    n = pos.shape[0]
    return pos, vel, rng.uniform(0.5, 1.5, n) / n


CASES = {
    # Plummer N = 8192 with a wide neighbour sphere: mostly small components
    "plummer8192": lambda: (*_plummer(8192, 3), dict(r_cut=0.02, h=0.025,
                                                      eps=4 / 8192, dt_soft=1 / 256)),
    # dense Gaussian clump: large components, deep block levels
    "gauss_dense": lambda: (*_gauss(2000, 4, 0.03), dict(r_cut=0.01, h=0.0125,
                                                          eps=1e-4, dt_soft=1 / 128)),
    # clumps of every size up to 40: packed warps of each width, long rows
    "clumps": lambda: (*_clumps(12), dict(r_cut=0.04, h=0.05, eps=1e-4, dt_soft=1 / 128)),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_hard_step_bitwise(cuda, name):
    import torch
    from paper_1506_04553_b300 import Context, HermiteParams, Params
    pos, vel, m, kw = CASES[name]()
    n = pos.shape[0]
    off, idx = oracle.neighbours(pos, kw["h"])
    hp = HermiteParams(dt_soft=kw["dt_soft"], eta=0.1, alpha=0.1)
    xo, vo, st = oracle.hermite(pos, vel, m, off, idx, dt_soft=hp.dt_soft,
                                eps=kw["eps"], r_cut=kw["r_cut"], gamma=GAMMA,
                                eta=hp.eta, alpha=hp.alpha, p=hp.log2_soft_over_max,
                                kmax=hp.kmax)
    ctx = Context(Params(r_out=kw["r_cut"], eps=kw["eps"], gamma=GAMMA))
    pg, vg = _dev(pos.T), _dev(vel.T)
    ctx.hard_step(pg, vg, _dev(m), _dev(off), _dev(idx, torch.int32), hp)
    s = ctx.stats()
    assert np.array_equal(pg.cpu().numpy().T, xo), name
    assert np.array_equal(vg.cpu().numpy().T, vo), name
    assert (s["herm_particle_steps"], s["herm_pairs"], s["herm_capped"]) == st[1:], (s, st)
    # components: scipy on the same graph, non-isolated vertices only
    rows = np.repeat(np.arange(n), np.diff(off))
    g = csr_matrix((np.ones(idx.size), (rows, idx)), shape=(n, n))
    ncomp, lab = connected_components(g, directed=False)
    nonis = np.diff(off) > 0
    sizes = np.bincount(lab[nonis])
    sizes = sizes[sizes > 0]
    assert s["herm_components"] == sizes.size
    assert s["herm_max_component"] == sizes.max()
    assert st[1] > nonis.sum()  # individual steps beyond the first
    print(f"{name}: {nonis.sum()} non-isolated, {sizes.size} components "
          f"(largest {sizes.max()}), {st[1]} particle steps")


def test_hard_step_all_isolated_is_a_drift(cuda):
    import torch
    from paper_1506_04553_b300 import Context, HermiteParams, Params
    pos, vel, m = _gauss(1000, 6, 1.0)
    off = np.zeros(1001, dtype=np.int64)
    idx = np.zeros(0, dtype=np.int32)
    ctx = Context(Params(r_out=1e-3))
    pg, vg = _dev(pos.T), _dev(vel.T)
    ctx.hard_step(pg, vg, _dev(m), _dev(off), _dev(idx, torch.int32),
                  HermiteParams(dt_soft=0.25))
    assert np.array_equal(pg.cpu().numpy().T, pos + 0.25 * vel)
    assert np.array_equal(vg.cpu().numpy().T, vel)
    assert ctx.stats()["herm_components"] == 0


def test_hard_step_capped_levels_bitwise(cuda):
    """A coarse finest level (kmax = 3) caps many steps; the capped schedule
    and its counter agree with the oracle."""
    import torch
    from paper_1506_04553_b300 import Context, HermiteParams, Params
    pos, vel, m = _gauss(800, 9, 0.02)
    off, idx = oracle.neighbours(pos, 0.0125)
    hp = HermiteParams(dt_soft=1 / 64, kmax=3)
    xo, vo, st = oracle.hermite(pos, vel, m, off, idx, dt_soft=hp.dt_soft, eps=1e-4,
                                r_cut=0.01, gamma=GAMMA, kmax=3)
    assert st[3] > 0
    ctx = Context(Params(r_out=0.01, eps=1e-4, gamma=GAMMA))
    pg, vg = _dev(pos.T), _dev(vel.T)
    ctx.hard_step(pg, vg, _dev(m), _dev(off), _dev(idx, torch.int32), hp)
    assert np.array_equal(pg.cpu().numpy().T, xo)
    assert np.array_equal(vg.cpu().numpy().T, vo)
    assert ctx.stats()["herm_capped"] == st[3]


def test_hard_part_argument_checks(cuda):
    import torch
    from paper_1506_04553_b300 import Context, HermiteParams, P3TError, Params, hard_force
    pos, vel, m = _gauss(100, 10, 0.05)
    off = np.zeros(101, dtype=np.int64)
    idx = np.zeros(0, dtype=np.int32)
    args = [_dev(pos.T), _dev(vel.T), _dev(m), _dev(off), _dev(idx, torch.int32)]
    ctx = Context(Params(r_out=0.01))
    for bad in (dict(eta=0.0), dict(eta=float("nan")), dict(alpha=-1.0),
                dict(dt_soft=0.0), dict(kmax=0), dict(log2_soft_over_max=-1),
                dict(log2_soft_over_max=30, kmax=40), dict(dt_soft=1e-300),
                dict(dt_soft=1e301)):
        with pytest.raises(P3TError):
            ctx.hard_step(*args, HermiteParams(**{"dt_soft": 0.01, **bad}))
    with pytest.raises(P3TError):
        hard_force(*args, r_cut=1e-20)
    a, j = hard_force(*args, r_cut=0.01)  # empty rows: no force
    assert not a.any() and not j.any()
    # the ensemble layout is refused
    ctx.set_ensemble(np.array([0, 50, 100], dtype=np.int64))
    with pytest.raises(P3TError):
        ctx.hard_step(*args, HermiteParams(dt_soft=0.01))
    # n = 0 is a no-op
    e = [torch.zeros((3, 0), dtype=torch.float64, device="cuda"),
         torch.zeros((3, 0), dtype=torch.float64, device="cuda"),
         torch.zeros((0,), dtype=torch.float64, device="cuda"),
         torch.zeros((1,), dtype=torch.int64, device="cuda"), _dev(idx, torch.int32)]
    Context(Params(r_out=0.01)).hard_step(*e, HermiteParams(dt_soft=0.01))
