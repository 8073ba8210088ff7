"""The autotuner (p3t_autotune) on an ensemble of uneven clusters, through the
C ABI: the objective is build + force + backward, the (n_group, n_leaf) pairs
are checked against the theta/2 reference as the header states, and the
configuration it keeps gives forces and gradients that match the FP64 oracle
run with the same group and leaf sizes, cluster by cluster."""
import numpy as np
import pytest

import oracle
from paper_1506_04553_b300 import ics
from parity_util import rel_err

pytestmark = pytest.mark.gpu


def test_autotune_keeps_an_accurate_fast_configuration(cuda):
    import torch
    from paper_1506_04553_b300 import Context, Params
    pos, _, m, off = ics.plummer_ensemble(12, seed=700, n_min=1024, n_max=8192)
    n = int(off[-1])
    sizes = np.diff(off)
    r_out = 0.01 * (sizes / 8192.0) ** (-1.0 / 3.0)
    eps = 4.0 / sizes
    ctx = Context(Params(theta=0.4))
    ctx.set_ensemble(off, r_out=r_out, eps=eps)
    pd = torch.tensor(pos, device="cuda")
    md = torch.tensor(m, device="cuda")
    w = np.random.default_rng(9).normal(size=(n, 3)).astype(np.float32)
    wd = torch.tensor(w.T.copy(), device="cuda")
    t = ctx.autotune(pd, md, w=wd, reps=1)
    assert t["n_group"] in (32, 48, 64) and t["n_leaf"] in (8, 16, 32)
    assert t["force_warps"] in (2, 4, 8) and t["vjp_warps"] in (2, 4)
    assert t["evaluated"] == 9 + 3 * 2
    # the accuracy check as stated (the start, n_group 64 / n_leaf 16, is kept)
    med, mx = np.array(t["cand_err_median"]), np.array(t["cand_err_max"])
    kept = (med <= 1.25 * t["base_err_median"]) & (mx <= 2.0 * t["base_err_max"])
    kept[2 * 3 + 1] = True
    assert t["rejected"] == int((~kept).sum())
    q = [32, 48, 64].index(t["n_group"]) * 3 + [8, 16, 32].index(t["n_leaf"])
    assert kept[q]
    assert 0 < t["ms"] <= t["cand_ms"][q]  # the block shapes only lower it
    assert t["err_median"] == med[q] and t["err_max"] == mx[q]
    assert t["base_err_median"] < 1e-4  # theta 0.4 against theta 0.2
    # the context keeps it: forces and gradients against the oracle with the
    # same sizes, every cluster on its own
    p = ctx.params
    assert (p.n_group, p.n_leaf) == (t["n_group"], t["n_leaf"])
    ctx.build_tree(pd, md)
    acc = ctx.long_force().cpu().numpy().T.astype(np.float64)
    gx, gm = ctx.long_force_vjp(wd)
    gx, gm = gx.cpu().numpy().T, gm.cpu().numpy()
    for c in range(len(sizes)):
        b, e = int(off[c]), int(off[c + 1])
        tr = oracle.Tree(pos[:, b:e].T.copy(), m[b:e], n_leaf=p.n_leaf,
                         n_group=p.n_group)
        tr.walk(0.4, r_out[c], r_out[c])
        err = rel_err(acc[b:e], tr.force(eps=eps[c], r_cut=r_out[c]))
        assert np.median(err) <= 1e-5 and err.max() <= 1e-4, (c, err.max())
        if c % 4 == 0:
            ox, om = tr.vjp(w[b:e].astype(np.float64), eps=eps[c], r_cut=r_out[c])
            ex = rel_err(gx[b:e], ox)
            assert np.median(ex) <= 1e-5 and ex.max() <= 1e-4, (c, ex.max())
    print(f"chose n_group {t['n_group']}, n_leaf {t['n_leaf']}, warps "
          f"{t['force_warps']}/{t['vjp_warps']}: {t['ms']:.2f} ms; error "
          f"{t['err_median']:.1e} / {t['err_max']:.1e} (start "
          f"{t['base_err_median']:.1e} / {t['base_err_max']:.1e}), rejected "
          f"{t['rejected']}")
