"""Parity at the full throughput workload: 512x256x256 cells, 8 ppc (268,435,456
electrons), FP32 cell-offset form in the library's default tile launch (8x8x8
tiles, the kernel bench.py times), ids tracked.

The oracle cannot advance 268M particles in test time, so it checks outputs it
can compute one by one:
* 20,000 randomly sampled particles: gather + Boris + move through the same
  full-size fields, compared particle by particle (by id);
* the current of a 4x4x4-cell block: every particle that can reach the block
  is advanced and deposited by the oracle on a small shifted grid, compared
  node by node with the library's J;
* properties at any size: the particle count, and the continuity equation
  (rho^{n+1} - rho^n)/dt + div J^{n+1/2} = 0 on the library's own outputs.
The species is hotter than the throughput workload (u_th = 0.5 instead of
0.05) so that the single step crosses cell and tile faces; everything else
(sizes, ppc, dx, dt, tile shape) is the throughput workload's.
Tolerances as in the one-step FP32 parity tests: 2e-5 of a cell, 2e-5 (1 + |u|),
and 2e-5 of the block's largest current.
"""
import dataclasses

import numpy as np
import pytest

import oracle
import workload

pytestmark = pytest.mark.gpu


def test_fp32_full_size_sampled_vs_oracle():
    import paper_1503_00276_gb300 as pg

    g, sps, _ = workload.config3(8)
    sp = dataclasses.replace(sps[0], uth=(0.5, 0.5, 0.5))
    n = workload.n_particles(g, sp)
    assert n == 268435456
    f = workload.random_fields(g, seed=31, amp=0.05)
    sim = pg.Simulation(g, [sp], precision="fp32", track_ids=True)
    for c, name in enumerate(["E1", "E2", "E3", "B1", "B2", "B3"]):
        sim.set_field(name, f[c])
    rho0 = sim.fields("RHO")
    sim.step(1)
    assert sim.diag()["error_flags"] == 0
    rho1 = sim.fields("RHO")
    J = [sim.fields(nm) for nm in ("J1", "J2", "J3")]
    x, u = sim.particles()
    ids = sim.ids()
    sim.close()
    assert x.shape[0] == n
    inv = np.full(n, -1, dtype=np.int64)
    inv[ids] = np.arange(n, dtype=np.int64)
    assert (inv >= 0).all()  # every id exactly once

    # sampled particles, one by one through the full-size fields
    rng = np.random.default_rng(5)
    samp = np.sort(rng.choice(n, 20000, replace=False))
    x0, u0 = workload.load_particles(g, sp, samp)
    xr, ur = oracle.advance_particles(g, f, sp.rqm, x0, u0)
    xg, ug = x[inv[samp]], u[inv[samp]]
    L = np.array([g.nx[d] * g.dx[d] for d in range(3)])
    d = xg - xr
    d = d - L * np.round(d / L)
    ex = np.max(np.abs(d / np.array(g.dx)))
    eu = np.max(np.abs(ug - ur) / (1.0 + np.abs(ur)))
    assert ex < 2e-5 and eu < 2e-5, (ex, eu)

    # current of one block of cells, rebuilt by the oracle from every particle
    # that starts within two cells of it
    nxc, nyc, nzc = (int(v) for v in g.nx)
    b0 = np.array([301, 117, 45])  # block origin (cells), away from the box faces
    nb, margin = 4, 2
    lo = b0 - margin
    cells = [np.arange(lo[k], lo[k] + nb + 2 * margin) for k in range(3)]
    cz, cy, cx = np.meshgrid(cells[2], cells[1], cells[0], indexing="ij")
    cid = (cz * nyc + cy) * nxc + cx
    ppc = sp.ppc_total
    pidx = (cid.reshape(-1)[:, None] * ppc + np.arange(ppc)[None, :]).reshape(-1)
    xa, ua = workload.load_particles(g, sp, pidx)
    xb, _ = oracle.advance_particles(g, f, sp.rqm, xa, ua, wrap=False)
    # small grid whose cell 0 is global cell b0 - 6 in every direction
    sub = dataclasses.replace(g, nx=(16, 16, 16))
    shift = (b0 - 6) * np.array(g.dx)
    q = workload.macro_charge(g, sp)
    jref = [np.zeros((16, 16, 16)) for _ in range(3)]
    for p in range(pidx.size):
        cur = oracle.deposit_vb(sub, xa[p] - shift, xb[p] - shift, 0.0, q)
        for c in range(3):
            jref[c] += cur[c]
    sl_sub = (slice(6, 6 + nb),) * 3
    sl_glob = (slice(b0[2], b0[2] + nb), slice(b0[1], b0[1] + nb), slice(b0[0], b0[0] + nb))
    for c in range(3):
        a = J[c][sl_glob]
        r = jref[c][sl_sub]
        scale = np.max(np.abs(r))
        assert scale > 0
        assert np.max(np.abs(a - r)) < 2e-5 * scale, (c, np.max(np.abs(a - r)) / scale)

    # continuity on the library's own full-size outputs
    dx = g.dx
    div = ((J[0] - np.roll(J[0], 1, 2)) / dx[0] + (J[1] - np.roll(J[1], 1, 1)) / dx[1]
           + (J[2] - np.roll(J[2], 1, 0)) / dx[2])
    res = np.max(np.abs((rho1 - rho0) / g.dt + div))
    assert res < 2e-5 * np.max(np.abs(rho0)) / g.dt, res
