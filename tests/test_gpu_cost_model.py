"""The force kernel's own interaction counters (the cost-model figures of
Sect. 3.1.2 that the bench reports) equal the oracle's counts: every list
entry taken once per particle of its group, cells and particles apart, at
several theta including 0 (N^2 pair terms)."""
import numpy as np
import pytest

import oracle
from paper_1506_04553_b300 import ics

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("theta", [0.0, 0.3, 0.5, 0.8])
def test_interaction_counters_match_oracle(cuda, theta):
    import torch
    from paper_1506_04553_b300 import Context, Params
    n = 20000
    pos, _, m = ics.plummer(n, seed=14)
    r_out = 0.01 * (n / 8192) ** (-1 / 3)
    ctx = Context(Params(theta=theta, r_out=r_out, gamma=0.1, eps=4.0 / n,
                         h=r_out, n_leaf=16, n_group=64))
    ctx.build_tree(torch.tensor(pos, device="cuda"), torch.tensor(m, device="cuda"))
    ctx.long_force()
    st = ctx.stats()
    t = oracle.Tree(pos.T, m, n_leaf=16, n_group=64)
    t.walk(theta, r_out, r_out)
    L = t.lists()
    cnt = t.groups()["count"].astype(np.int64)
    pc = int((np.diff(L["pc_off"]) * cnt).sum())
    ppn = int((np.diff(L["ppn_off"]) * cnt).sum())
    ppf = int((np.diff(L["ppf_off"]) * cnt).sum())
    assert st["int_pc"] == pc
    assert st["int_pp"] == ppn + ppf
    assert st["int_pp_near"] == ppn
    if theta == 0.0:
        assert pc == 0 and ppn + ppf == n * n
