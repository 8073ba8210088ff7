"""Whole P3T steps (Sect. 2.2): half-kick by F_soft, the hard step (isolated
particles drift, the others are Hermite-integrated over dt_soft on the
neighbour lists), new tree, F_soft and neighbour lists, half-kick.

The split of the potential is exact (W + (1 - W) = 1, Eq. 5-6), so the
energy of the scheme is the softened Newtonian energy, computed here by the
oracle's direct sum.  With the paper's standard parameters (Table 1:
dt_soft = (1/256)(N/16K)^(-1/3), r_cut = 4 dt_soft, buffer 3 sigma dt_soft
with sigma = 1/sqrt(2), eps = 4/N, eta = 0.1, dt_max = dt_soft/4) the
energy error after 32 steps must be small, and far below that of plain
leapfrog steps of the same dt_soft with the whole force from the tree
(r_cut -> 0: no hard part)."""
import numpy as np
import pytest

import oracle
from paper_1506_04553_b300 import ics

pytestmark = pytest.mark.gpu


def _energy(pos, vel, m, eps):
    ke = 0.5 * np.sum(m[None, :] * vel * vel)
    _, pot = oracle.direct(pos.T.copy(), m, eps=eps, kind="newton", potential=True)
    return ke + 0.5 * np.sum(m * pot)


def _run(n, steps, p3t):
    import torch
    import paper_1506_04553_b300 as P
    pos_h, vel_h, m = ics.plummer(n, 11)
    dt = (1 / 256) * (n / 16384) ** (-1 / 3)
    eps = 4.0 / n
    r_cut = 4 * dt if p3t else 1e-9
    h = r_cut + 3 * dt / np.sqrt(2) if p3t else 1e-9
    ctx = P.Context(P.Params(theta=0.4, r_out=r_cut, eps=eps, h=h))
    pos = torch.tensor(pos_h, device="cuda")
    vel = torch.tensor(vel_h, device="cuda")
    mass = torch.tensor(m, device="cuda")
    acc = torch.empty((3, n), dtype=torch.float32, device="cuda")
    hp = P.HermiteParams(dt_soft=dt)
    ctx.build_tree(pos, mass)
    ctx.long_force(acc)
    off, idx = ctx.neighbours()
    e0 = _energy(pos_h, vel_h, m, eps)
    for _ in range(steps):
        P.kick(vel, acc, 0.5 * dt)
        if p3t:
            ctx.hard_step(pos, vel, mass, off, idx, hp)
            assert ctx.stats()["herm_capped"] == 0
        else:
            P.drift(pos, vel, dt)
        ctx.build_tree(pos, mass)
        ctx.long_force(acc)
        off, idx = ctx.neighbours()
        P.kick(vel, acc, 0.5 * dt)
    e1 = _energy(pos.cpu().numpy(), vel.cpu().numpy(), m, eps)
    return abs(e1 - e0) / abs(e0), ctx.stats()


def test_p3t_steps_conserve_energy(cuda):
    err_p3t, st = _run(4096, 32, True)
    err_lf, _ = _run(4096, 32, False)
    print(f"|dE/E| after 32 steps: P3T {err_p3t:.2e}, leapfrog {err_lf:.2e}; "
          f"last hard step: {st['herm_components']} components, "
          f"{st['herm_particle_steps']} particle steps")
    assert st["herm_components"] > 100  # the hard part does work
    assert err_p3t < 2e-5
    assert err_p3t < err_lf / 100
