"""Failure paths of the kernels' bounded loops and waits, and of the cell
capacity, driven by small bounds (p3t_set_limits): no GPU fault is caused.
A kernel that reaches a bound stops that work item, latches a status and
returns; the host reads P3T_ERR_TIMEOUT (or P3T_ERR_CAPACITY) from p3t_check
or the synchronising call, and the same context then works again once the
bounds are restored."""
import numpy as np
import pytest

import oracle
from paper_1506_04553_b300 import ics

pytestmark = pytest.mark.gpu

TIMEOUT, CAPACITY = 4, 2


def _tensors(pos, m):
    import torch
    return (torch.tensor(np.ascontiguousarray(pos.T), device="cuda"),
            torch.tensor(m, device="cuda"))


def _raises(code, fn):
    from paper_1506_04553_b300 import P3TError
    with pytest.raises(P3TError) as e:
        fn()
    assert e.value.code == code, e.value


def test_walk_iteration_bound_times_out_then_recovers(cuda):
    import torch
    from paper_1506_04553_b300 import Context, Params
    pos, _, m = ics.plummer(4096, 11)
    pd, md = _tensors(pos.T.copy(), m)
    ctx = Context(Params(theta=0.4, r_out=0.01, eps=4 / 4096))
    ctx.build_tree(pd, md)
    ref = ctx.long_force().clone()
    w = torch.randn((3, 4096), dtype=torch.float32, device="cuda")
    gref = ctx.long_force_vjp(w)[0].clone()
    ctx.set_limits(walk_iters=3)  # a walk needs far more iterations
    _raises(TIMEOUT, lambda: ctx.long_force())        # fused walk + force
    _raises(TIMEOUT, lambda: ctx.neighbours())        # neighbour walk
    _raises(TIMEOUT, lambda: ctx.long_force_vjp(w))   # backward walk
    _raises(TIMEOUT, lambda: ctx.lists())             # inspection walk
    ctx.set_limits()
    ctx.check()  # nothing left latched
    assert torch.equal(ctx.long_force(), ref)
    assert torch.equal(ctx.long_force_vjp(w)[0], gref)
    off, idx = ctx.neighbours()
    off_o, idx_o = oracle.neighbours(pos.T.copy(), 0.01)
    assert np.array_equal(off.cpu().numpy(), off_o)


def _clump():
    rng = np.random.default_rng(4)
    pos = rng.normal(size=(2000, 3)) * 0.03
    vel = rng.normal(size=(2000, 3)) * 0.3
    return pos, vel, rng.uniform(0.5, 1.5, 2000) / 2000


@pytest.mark.parametrize("bound", ["uf_rounds", "block_steps"])
def test_hard_step_bounds_time_out_then_recover(cuda, bound):
    """The union-find of the component search (a dense clump: one component
    of ~1800 particles needs lookups of several rounds) and the block steps
    of a component (hundreds needed) stop at their bounds."""
    import torch
    from paper_1506_04553_b300 import Context, HermiteParams, Params
    pos, vel, m = _clump()
    off, idx = oracle.neighbours(pos, 0.0125)
    kw = dict(dt_soft=1 / 128, eps=1e-4, r_cut=0.01, gamma=0.1)
    xm, vm, _ = oracle.hermite_mirror(pos, vel, m, off, idx, **kw)
    ctx = Context(Params(r_out=0.01, eps=1e-4, gamma=0.1))
    hp = HermiteParams(dt_soft=1 / 128)
    dev = lambda a, t=None: torch.tensor(np.ascontiguousarray(a), dtype=t).cuda()
    args = lambda: (dev(pos.T), dev(vel.T), dev(m), dev(off),
                    dev(idx, torch.int32))
    ctx.set_limits(**{bound: 1 if bound == "uf_rounds" else 2})
    a = args()
    _raises(TIMEOUT, lambda: ctx.hard_step(*a, hp))
    ctx.set_limits()
    ctx.check()
    a = args()
    ctx.hard_step(*a, hp)
    assert np.array_equal(a[0].cpu().numpy().T, xm)
    assert np.array_equal(a[1].cpu().numpy().T, vm)


def test_cell_bound_reports_the_needed_cells(cuda):
    from paper_1506_04553_b300 import Context, Params
    pos, _, m = ics.plummer(8192, 1)
    pd, md = _tensors(pos.T.copy(), m)
    ctx = Context(Params(theta=0.4, r_out=0.01))
    ctx.set_limits(max_cells=100)
    _raises(CAPACITY, lambda: ctx.build_tree(pd, md))
    need = ctx.stats()["need_cells"]
    assert need > 100
    ctx.set_limits()
    ctx.build_tree(pd, md)
    st = ctx.stats()
    assert st["need_cells"] == st["n_cells"] >= need
    t = oracle.Tree(pos.T.copy(), m)
    assert st["n_cells"] == t.ncell
