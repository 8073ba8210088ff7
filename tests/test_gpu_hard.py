"""The hard part on the GPU (p3t_hard_force, p3t_hard_step) against the FP64
oracle, which evaluates Eq. 7 and the timestep criteria of Eq. 18-20 as
printed (plain operations, criteria as dt <= eta sqrt(num / den)):

* forces and jerks within 1e-13 of the per-particle magnitude of their pair
  sums (the GPU fuses products into FMAs, the oracle does not);
* whole Hermite steps within 16 times the oracle's own response to one-ulp
  perturbations of its input (hard steps in dense clumps are chaotic, so
  rounding differences grow), with the same number of particle steps, and
  the particles whose level decision lies within 1e-10 of a tie counted and
  reported.

Separately, the oracle's fused-order mirror (same formulas, the GPU's order
of operations) must agree with the GPU bit for bit: that checks the block
schedule and the component bookkeeping exactly.  The component search is
checked against scipy's connected components."""
import numpy as np
import pytest
from scipy.sparse import csr_matrix
from scipy.sparse.csgraph import connected_components

import oracle
from paper_1506_04553_b300 import ics
from parity_util import (assert_hard_step_close, hard_force_scales,
                         hermite_sensitivity)

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


FORCE_CASES = {
    "gauss3000": lambda: (*_gauss(3000, 1, 0.05), 0.02, 1e-3, 0.025),
    "plummer8192": lambda: (*_plummer(8192, 3), 0.02, 4 / 8192, 0.025),
    "gauss_dense": lambda: (*_gauss(2000, 4, 0.03), 0.01, 1e-4, 0.0125),
}

FORCE_TOL = 1e-13  # of the per-particle magnitude of the pair sums


@pytest.mark.parametrize("name", sorted(FORCE_CASES))
def test_hard_force_vs_plain_oracle(cuda, name):
    import torch
    from paper_1506_04553_b300 import hard_force
    pos, vel, m, r_cut, eps, h = FORCE_CASES[name]()
    off, idx = oracle.neighbours(pos, h)
    a_o, j_o = oracle.hard_force(pos, vel, m, off, idx, eps=eps, r_cut=r_cut, gamma=GAMMA)
    a_g, j_g = hard_force(_dev(pos.T), _dev(vel.T), _dev(m), _dev(off),
                          _dev(idx, torch.int32), r_cut=r_cut, eps=eps, gamma=GAMMA)
    a_g, j_g = a_g.cpu().numpy().T, j_g.cpu().numpy().T
    sa, sj = hard_force_scales(pos, vel, m, off, idx, eps, r_cut)
    ea = np.linalg.norm(a_g - a_o, axis=1)
    ej = np.linalg.norm(j_g - j_o, axis=1)
    assert np.all(ea <= FORCE_TOL * sa), (ea / np.maximum(sa, 1e-300)).max()
    assert np.all(ej <= FORCE_TOL * sj), (ej / np.maximum(sj, 1e-300)).max()
    assert np.count_nonzero(np.abs(a_o).sum(axis=1)) > 300  # rows that interact
    print(f"{name}: |da|/scale max {(ea / np.maximum(sa, 1e-300)).max():.2e}, "
          f"|dj|/scale max {(ej / np.maximum(sj, 1e-300)).max():.2e}")


def test_hard_force_mirror_bitwise(cuda):
    """The fused-order mirror reproduces the GPU's hard force bit for bit."""
    import torch
    from paper_1506_04553_b300 import hard_force
    pos, vel, m = _gauss(3000, 1, 0.05)
    r_cut, eps = 0.02, 1e-3
    off, idx = oracle.neighbours(pos, 1.25 * r_cut)
    a_o, j_o = oracle.hard_force_mirror(pos, vel, m, off, idx, eps=eps,
                                        r_cut=r_cut, gamma=GAMMA)
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


TIE = 1e-10  # level decisions closer than this to a tie may flip on rounding


def _gpu_hard_step(pos, vel, m, off, idx, kw, hp):
    import torch
    from paper_1506_04553_b300 import Context, Params
    ctx = Context(Params(r_out=kw["r_cut"], eps=kw["eps"], gamma=GAMMA))
    pg, vg = _dev(pos.T), _dev(vel.T)
    ctx.hard_step(pg, vg, _dev(m), _dev(off), _dev(idx, torch.int32), hp)
    return pg.cpu().numpy().T, vg.cpu().numpy().T, ctx.stats()


@pytest.mark.parametrize("name", sorted(CASES))
def test_hard_step_vs_plain_oracle(cuda, name):
    from paper_1506_04553_b300 import HermiteParams
    pos, vel, m, kw = CASES[name]()
    n = pos.shape[0]
    off, idx = oracle.neighbours(pos, kw["h"])
    hp = HermiteParams(dt_soft=kw["dt_soft"], eta=0.1, alpha=0.1)
    okw = dict(dt_soft=hp.dt_soft, eps=kw["eps"], r_cut=kw["r_cut"], gamma=GAMMA,
               eta=hp.eta, alpha=hp.alpha, p=hp.log2_soft_over_max, kmax=hp.kmax)
    _, _, st, det = oracle.hermite(pos, vel, m, off, idx, detail=True, **okw)
    x0, v0, sx, sv = hermite_sensitivity(
        lambda p, v: oracle.hermite(p, v, m, off, idx, **okw)[:2], pos, vel)
    xg, vg, s = _gpu_hard_step(pos, vel, m, off, idx, kw, hp)
    # particles in a component with a decision near a tie: counted, reported
    rows = np.repeat(np.arange(n), np.diff(off))
    g = csr_matrix((np.ones(idx.size), (rows, idx)), shape=(n, n))
    _, lab = connected_components(g, directed=False)
    tie = np.isin(lab, lab[det["margin"] < TIE])
    keep = ~tie
    rx, rv = assert_hard_step_close(xg[keep], vg[keep], x0[keep], v0[keep],
                                    sx[keep], sv[keep])
    if not tie.any():
        assert (s["herm_particle_steps"], s["herm_pairs"], s["herm_capped"]) == st[1:], (s, st)
    assert tie.sum() <= 0.001 * n
    print(f"{name}: ratio to the oracle's rounding response x {rx:.2f} v {rv:.2f}; "
          f"particles near a level tie {int(tie.sum())}; least margin "
          f"{det['margin'].min():.1e}")


@pytest.mark.parametrize("name", sorted(CASES))
def test_hard_step_mirror_bitwise(cuda, name):
    """The fused-order mirror reproduces the GPU's hard step bit for bit:
    the same block schedule, components and counters."""
    from paper_1506_04553_b300 import HermiteParams
    pos, vel, m, kw = CASES[name]()
    n = pos.shape[0]
    off, idx = oracle.neighbours(pos, kw["h"])
    hp = HermiteParams(dt_soft=kw["dt_soft"], eta=0.1, alpha=0.1)
    xo, vo, st = oracle.hermite_mirror(pos, vel, m, off, idx, dt_soft=hp.dt_soft,
                                       eps=kw["eps"], r_cut=kw["r_cut"], gamma=GAMMA,
                                       eta=hp.eta, alpha=hp.alpha,
                                       p=hp.log2_soft_over_max, kmax=hp.kmax)
    xg, vg, s = _gpu_hard_step(pos, vel, m, off, idx, kw, hp)
    assert np.array_equal(xg, xo), name
    assert np.array_equal(vg, vo), name
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


def test_hard_step_capped_levels(cuda):
    """A coarse finest level (kmax = 3) caps many steps; the capped schedule
    and its counter agree with the oracle (plain: within the rounding
    tolerance; mirror: bit for bit)."""
    from paper_1506_04553_b300 import HermiteParams
    pos, vel, m = _gauss(800, 9, 0.02)
    off, idx = oracle.neighbours(pos, 0.0125)
    hp = HermiteParams(dt_soft=1 / 64, kmax=3)
    okw = dict(dt_soft=hp.dt_soft, eps=1e-4, r_cut=0.01, gamma=GAMMA, kmax=3)
    xm, vm, sm = oracle.hermite_mirror(pos, vel, m, off, idx, **okw)
    _, _, st = oracle.hermite(pos, vel, m, off, idx, **okw)
    assert st[3] > 0
    x0, v0, sx, sv = hermite_sensitivity(
        lambda p, v: oracle.hermite(p, v, m, off, idx, **okw)[:2], pos, vel)
    xg, vg, s = _gpu_hard_step(pos, vel, m, off, idx,
                               dict(r_cut=0.01, eps=1e-4), hp)
    assert_hard_step_close(xg, vg, x0, v0, sx, sv)
    assert s["herm_capped"] == st[3]
    assert np.array_equal(xg, xm)
    assert np.array_equal(vg, vm)
    assert s["herm_capped"] == sm[3]


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
