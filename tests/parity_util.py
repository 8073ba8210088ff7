"""Helpers shared by the GPU parity tests: run the CUDA path and the oracle on
the same seeded input and compare what must be identical."""
from __future__ import annotations

import numpy as np

import oracle


def rel_err(a, ref):
    """Per-particle relative error |a - ref| / max(|ref|, 1e-3 rms|ref|)."""
    nr = np.linalg.norm(ref, axis=1)
    floor = 1e-3 * np.sqrt(np.mean(nr ** 2)) if nr.size else 0.0
    return np.linalg.norm(a - ref, axis=1) / np.maximum(nr, floor)


def gpu_run(pos, mass, params, potential=False, neighbours=True):
    """pos (n, 3) FP64 host array; returns (ctx, acc (n,3) FP64, pot or None,
    (offsets, idx) or None)."""
    import torch
    from paper_1506_04553_b300 import Context
    ctx = Context(params)
    n = pos.shape[0]
    pd = torch.tensor(np.ascontiguousarray(pos.T), dtype=torch.float64,
                      device="cuda")
    md = torch.tensor(mass, dtype=torch.float64, device="cuda")
    ctx.build_tree(pd, md)
    out = ctx.long_force(want_potential=potential)
    acc, pot = (out if potential else (out, None))
    ngb = None
    if neighbours:
        off, idx = ctx.neighbours()
        ngb = (off.cpu().numpy(), idx.cpu().numpy())
    torch.cuda.synchronize()
    a = acc.cpu().numpy().astype(np.float64).T.copy()
    p = pot.cpu().numpy() if pot is not None else None
    return ctx, a, p, ngb


def cell_keys(cells):
    return list(zip(cells["level"].tolist(), cells["first"].tolist()))


def compare_structure(ctx, tree):
    """Asserts identical keys, order, cells, groups; returns id maps."""
    key_g, order_g = ctx.order()
    key_o, order_o = tree.particles()
    assert np.array_equal(key_g, key_o), "Morton keys differ"
    assert np.array_equal(order_g.astype(np.int64), order_o), "sort order differs"
    lo_g, size_g = ctx.root()
    lo_o, size_o = tree.root()
    assert np.array_equal(lo_g, lo_o) and size_g == size_o, "root cube differs"
    cg, co = ctx.cells(), tree.cells()
    kg, ko = cell_keys(cg), cell_keys(co)
    assert len(kg) == len(ko), f"cell count {len(kg)} != {len(ko)}"
    mg = {k: i for i, k in enumerate(kg)}
    mo = {k: i for i, k in enumerate(ko)}
    assert set(mg) == set(mo), "cell sets differ"
    og = np.array([mg[k] for k in ko])  # oracle cell id -> gpu cell id
    assert np.array_equal(cg["count"][og], co["count"])
    assert np.array_equal(cg["nchild"][og], co["nchild"])
    assert np.array_equal(cg["fmin"][og], co["fmin"]), "FP32 cell boxes differ"
    assert np.array_equal(cg["fmax"][og], co["fmax"]), "FP32 cell boxes differ"
    M = co["M"]
    assert np.all(np.abs(cg["M"][og] - M) <= 1e-12 * M)
    scale = np.abs(co["com"]).max() + 1.0
    assert np.abs(cg["com"][og] - co["com"]).max() <= 1e-12 * scale
    qs = np.abs(co["Q"]).max(axis=1, keepdims=True) + 1e-300
    assert np.all(np.abs(cg["Q"][og] - co["Q"]) <= 1e-9 * qs + 1e-18)
    gg, go = ctx.groups(), tree.groups()
    assert sorted(gg["first"].tolist()) == sorted(go["first"].tolist())
    pg = {f: i for i, f in enumerate(gg["first"].tolist())}
    gid = np.array([pg[f] for f in go["first"].tolist()])  # oracle -> gpu
    assert np.array_equal(gg["count"][gid], go["count"])
    assert np.array_equal(gg["fmin"][gid], go["fmin"])
    assert np.array_equal(gg["fmax"][gid], go["fmax"])
    return og, gid


def compare_lists(ctx, tree, og, gid, groups=None):
    """Asserts identical interaction-list sets for every (or the listed)
    oracle group."""
    Lg, Lo = ctx.lists(), tree.lists()
    cg = ctx.cells()
    go_to_key = {}
    kg = cell_keys(cg)
    sel = range(tree.ngroup) if groups is None else groups
    for g in sel:
        q = gid[g]
        pc_o = Lo["pc"][Lo["pc_off"][g]:Lo["pc_off"][g + 1]]
        pc_g = Lg["pc"][Lg["pc_off"][q]:Lg["pc_off"][q + 1]]
        assert sorted(og[pc_o].tolist()) == sorted(pc_g.tolist()), f"cell list of group {g}"
        for name in ("ppn", "ppf"):
            lo_ = Lo[name][Lo[name + "_off"][g]:Lo[name + "_off"][g + 1]]
            lg_ = Lg[name][Lg[name + "_off"][q]:Lg[name + "_off"][q + 1]]
            assert sorted(lo_.tolist()) == sorted(lg_.tolist()), f"{name} list of group {g}"


# --------------------------------------------------------------------------
# Tolerances of the hard part (GPU against the plain FP64 oracle)
# --------------------------------------------------------------------------

U64 = 2.0 ** -53  # unit roundoff of FP64


def hard_force_scales(pos, vel, m, off, idx, eps, r_cut, G=1.0):
    """Per-particle bounds of the terms of the hard sums (Eq. 7): sum_j G m_j
    / s^2 for the acceleration and sum_j G m_j |u| (4 / s^3 + 2.5 / (r_cut
    s^2)) for the jerk (1 - K <= 1, |dK/dx| <= 35/16).  Rounding in the sums
    is of order U64 times these, however much the terms cancel."""
    n = len(m)
    rows = np.repeat(np.arange(n), np.diff(off))
    q = pos[rows] - pos[idx]
    u = vel[rows] - vel[idx]
    s2 = (q * q).sum(1) + eps * eps
    un = np.sqrt((u * u).sum(1))
    sa = np.bincount(rows, G * m[idx] / s2, minlength=n)
    sj = np.bincount(rows, G * m[idx] * un * (4 / s2 ** 1.5 + 2.5 / (r_cut * s2)),
                     minlength=n)
    return sa, sj


def hermite_sensitivity(run, pos, vel, reps=4, seed=0):
    """How far rounding alone can move the result of a hard step: the
    per-particle largest change of the plain oracle's final positions and
    velocities when its input positions and velocities are perturbed by one
    unit in the last place (random signs), over `reps` perturbations.
    run(pos, vel) -> (x, v).  Returns (x0, v0, dx, dv)."""
    x0, v0 = run(pos, vel)
    rng = np.random.default_rng(seed)
    dx = np.zeros(len(pos))
    dv = np.zeros(len(pos))
    for _ in range(reps):
        pp = pos * (1 + rng.choice([-1.0, 1.0], pos.shape) * 2.0 * U64)
        vp = vel * (1 + rng.choice([-1.0, 1.0], vel.shape) * 2.0 * U64)
        x1, v1 = run(pp, vp)
        dx = np.maximum(dx, np.abs(x1 - x0).max(axis=1))
        dv = np.maximum(dv, np.abs(v1 - v0).max(axis=1))
    return x0, v0, dx, dv


def assert_hard_step_close(xg, vg, x0, v0, sx, sv, factor=16.0):
    """GPU hard step against the plain oracle: every particle within
    `factor` times the oracle's own response to one-ulp input perturbations
    (hermite_sensitivity), and never tighter than 4 ulp of its coordinates.
    Returns the largest ratios (x, v) for reporting."""
    fx = 4 * 2 * U64 * np.abs(x0).max(axis=1)
    fv = 4 * 2 * U64 * np.maximum(np.abs(v0).max(axis=1), np.abs(v0).max() * 1e-3)
    rx = np.abs(xg - x0).max(axis=1) / np.maximum(sx, fx)
    rv = np.abs(vg - v0).max(axis=1) / np.maximum(sv, fv)
    assert rx.max() <= factor, (rx.max(), int(rx.argmax()))
    assert rv.max() <= factor, (rv.max(), int(rv.argmax()))
    return float(rx.max()), float(rv.max())
