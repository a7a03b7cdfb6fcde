"""GPU tests of the autotuner: every candidate is timed, the choice is the
fastest that ran, and a simulation built with the choice advances like the
oracle (one-step FP32 tolerances)."""
import numpy as np
import pytest

import oracle
import workload

pytestmark = pytest.mark.gpu


def test_autotune_picks_the_fastest_candidate_and_it_is_correct():
    import paper_1503_00276_gb300 as pg
    dx = (0.1, 0.1, 0.1)
    g = workload.Grid(ndim=3, nx=(32, 16, 16), dx=dx, dt=workload.courant_dt(dx, 3))
    sp = workload.Species(ppc=(2, 1, 1), uth=(0.3,) * 3, seed=77)
    best, tried = pg.autotune(g, [sp], warmup=1, steps=2)
    shapes = {t["tile"] for t in tried}
    assert (8, 8, 8) in shapes and (16, 8, 4) in shapes and (4, 4, 4) in shapes
    ran = [t for t in tried if t["ms_per_step"] > 0]
    assert ran and best["ms_per_step"] == min(t["ms_per_step"] for t in ran)
    tile = best["tile"]
    f = workload.random_fields(g, seed=3, amp=0.2)
    x0, u0 = workload.load_particles(g, sp)
    sim = pg.Simulation(g, [sp], precision="fp32", explicit=[(x0, u0, workload.macro_charge(g, sp))], tile=tile,
                        track_ids=True, sort_period=best["sort_period"], ctas_per_sm=best["ctas_per_sm"])
    for c, name in enumerate(["E1", "E2", "E3", "B1", "B2", "B3"]):
        sim.set_field(name, f[c])
    ref = oracle.from_workload(g, [sp], fields=f)
    ref.step(1)
    sim.step(1)
    x, u = sim.particles()
    ids = sim.ids()
    L = np.array([g.nx[d] * dx[d] for d in range(3)])
    d = x - ref.x[0][ids]
    d = d - L * np.round(d / L)
    assert np.max(np.abs(d / np.array(dx))) < 2e-5
    assert np.max(np.abs(u - ref.u[0][ids]) / (1 + np.abs(ref.u[0][ids]))) < 2e-5
    sim.close()


def test_batch_autotune_over_members():
    import paper_1503_00276_gb300 as pg
    dx = (0.1, 0.1, 1.0)
    mem = []
    for i, nx in enumerate(((64, 32, 1), (128, 64, 1), (32, 32, 1))):
        g = workload.Grid(ndim=2, nx=nx, dx=dx, dt=workload.courant_dt(dx, 2))
        mem.append((g, [workload.Species(ppc=(2, 2, 1), uth=(0.2,) * 3, seed=90 + i)]))
    best, tried = pg.batch_autotune(mem, warmup=1, steps=2)
    assert {t["tile"] for t in tried} == {(32, 16, 1), (16, 16, 1), (8, 8, 1)}
    assert {t["ctas_per_sm"] for t in tried} == {2, 4}
    ran = [t for t in tried if t["ms_per_step"] > 0]
    assert len(ran) == len(tried) and best["ms_per_step"] == min(t["ms_per_step"] for t in ran)
    b = pg.Batch(mem, tile=best["tile"], ctas_per_sm=best["ctas_per_sm"])
    b.step(3)
    assert b.info()["tile"] == best["tile"]
    for i in range(len(mem)):
        assert b.sim(i).diag()["error_flags"] == 0
    b.close()
