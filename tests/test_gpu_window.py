"""GPU parity of the moving window and the laser set-up against the oracle.

* pic_laser_add: the fields of pulses moving in x1 and x2, with and without a
  focal plane, in 2D and 3D, equal the oracle's laser_fields (FP64 form to
  1e-12, FP32 form to 1e-6 of the peak: one rounding).
* A 2D run with the window moving at c, a laser pulse and a warm plasma: after
  20 steps (about 14 one-cell shifts) the shift count, the set of surviving
  particles (ids: the back columns dropped, the injected ones continuing the
  loader's sequence), their positions and momenta (1e-4 of a cell / of u: FP32
  against FP64 over 20 steps, as the many-step parity test) and the fields
  (1e-4 of their maxima) match the oracle.
"""
import numpy as np
import pytest

import oracle
import workload

pytestmark = pytest.mark.gpu

NAMES = ["E1", "E2", "E3", "B1", "B2", "B3"]


@pytest.mark.parametrize("ndim", [2, 3])
@pytest.mark.parametrize("wavetype,focus", [(1, None), (2, None), (1, 3.0), (2, -4.0)])
@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 1e-6)])
def test_laser_setup_matches_oracle(prec, tol, wavetype, focus, ndim):
    import paper_1503_00276_gb300 as pg
    if ndim == 2:
        dx = (0.1, 0.2, 1.0)
        g = workload.Grid(ndim=2, nx=(128, 32, 1), dx=dx, dt=workload.courant_dt(dx, 2))
        tile = (32, 16)
    else:
        dx = (0.1, 0.2, 0.2)
        g = workload.Grid(ndim=3, nx=(64, 32, 16), dx=dx, dt=workload.courant_dt(dx, 3))
        tile = (8, 8, 8)
    las = workload.Laser(vosc=2.0, rkkp=10.0, w0=1.5, rise=1.5, length=0.5, fall=1.5, start=2.0, pol=30.0,
                         phase=0.3, offset=(0.4, -0.2), wavetype=wavetype, focus=focus)
    sim = pg.Simulation(g, [], precision=prec, tile=tile if prec == "fp32" else None)
    sim.add_laser(las)
    ref = oracle.laser_fields(g, las)
    assert max(np.max(np.abs(r)) for r in ref) > 1.0  # the pulse lies in the box
    for c, name in enumerate(NAMES):
        m = max(np.max(np.abs(ref[c])), 1e-300)
        assert np.max(np.abs(sim.fields(name) - ref[c])) <= tol * max(m, 1.0), name
    sim.close()


@pytest.mark.parametrize("smooth", [0, 2])
def test_moving_window_with_laser_matches_oracle(smooth):
    """20 steps of a window moving at c with a laser, FP32, against the oracle;
    with smooth = 2 the current is smoothed by two (1, 2, 1) passes per
    direction, which reach across the open x1 side (values beyond it read 0)."""
    import paper_1503_00276_gb300 as pg
    dx = (0.1, 0.2, 1.0)
    g = workload.Grid(ndim=2, nx=(64, 32, 1), dx=dx, dt=workload.courant_dt(dx, 2), move_window=True,
                      smooth_level=(smooth, smooth, 0))
    sp = workload.Species(ppc=(2, 2, 1), uth=(0.1, 0.1, 0.1), ufl=(0.3, 0.0, 0.0), seed=17)
    las = workload.Laser(vosc=0.5, rkkp=8.0, w0=2.0, rise=1.0, fall=1.0, start=1.0)
    ref = oracle.from_workload(g, [sp])
    for c, f in enumerate(oracle.laser_fields(g, las)):
        ref.fld[c] += f
    sim = pg.Simulation(g, [sp], precision="fp32", tile=(32, 16), track_ids=True)
    sim.add_laser(las)
    n = 20
    ref.step(n)
    sim.step(n)
    assert ref.shifts >= 10
    ids = sim.ids()
    x, u = sim.particles()
    assert np.array_equal(np.sort(ids), np.sort(ref.ids[0]))
    pos = {int(i): k for k, i in enumerate(ref.ids[0])}
    order = np.array([pos[int(i)] for i in ids])
    L2 = g.nx[1] * dx[1]
    d = x - ref.x[0][order]
    d[:, 1] -= L2 * np.round(d[:, 1] / L2)
    assert np.max(np.abs(d[:, 0] / dx[0])) < 1e-4 and np.max(np.abs(d[:, 1] / dx[1])) < 1e-4
    assert np.max(np.abs(u - ref.u[0][order])) < 1e-4
    for c, name in enumerate(NAMES):
        m = np.max(np.abs(ref.fld[c]))
        if m == 0:
            continue
        assert np.max(np.abs(sim.fields(name) - ref.fld[c])) < 1e-4 * m, name
    assert sim.diag()["n_particles"] == ref.x[0].shape[0]
    sim.close()


def test_beam_driver_in_moving_window_matches_oracle():
    """A plasma plus a bi-Gaussian relativistic driver (explicit species, no
    injection) in a 3D moving window: both species against the oracle after
    10 steps."""
    import paper_1503_00276_gb300 as pg
    dx = (0.05, 0.1, 0.1)
    g = workload.Grid(ndim=3, nx=(64, 16, 16), dx=dx, dt=workload.courant_dt(dx, 3), move_window=True)
    plasma = workload.Species(ppc=(1, 1, 2), uth=(0.02, 0.02, 0.02), seed=41)
    beam = workload.Species(rqm=-1.0, ppc=(0, 0, 0), seed=42)
    bx, bu, bq = workload.beam_particles(g, 3000, (2.2, 0.8, 0.8), 0.3, 0.15, 100.0, 2.0, 42)
    px, pu = workload.load_particles(g, plasma)
    ref = oracle.State(g, [plasma, beam], [px, bx], [pu, bu], [workload.macro_charge(g, plasma), bq])
    sim = pg.Simulation(g, [plasma, beam], precision="fp32", explicit=[None, (bx, bu, bq)], tile=(16, 8, 4),
                        track_ids=True)
    ref.step(10)
    sim.step(10)
    assert ref.shifts >= 5
    for s in range(2):
        ids = sim.ids(s)
        x, u = sim.particles(s)
        assert np.array_equal(np.sort(ids), np.sort(ref.ids[s]))
        pos = {int(i): k for k, i in enumerate(ref.ids[s])}
        order = np.array([pos[int(i)] for i in ids])
        L = np.array([1e300, g.nx[1] * dx[1], g.nx[2] * dx[2]])
        d = x - ref.x[s][order]
        d[:, 1:] -= L[1:] * np.round(d[:, 1:] / L[1:])
        assert np.max(np.abs(d / np.array(dx))) < 1e-4, s
        assert np.max(np.abs(u - ref.u[s][order]) / (1 + np.abs(ref.u[s][order]))) < 1e-4, s
    for c, name in enumerate(NAMES):
        m = np.max(np.abs(ref.fld[c]))
        if m > 0:
            assert np.max(np.abs(sim.fields(name) - ref.fld[c])) < 1e-4 * m, name
    sim.close()


def test_antenna_and_window_start_match_oracle():
    """A pulse driven through the lower x1 boundary into a warm plasma while
    the window is still; the window starts moving at window_start: fields,
    shift count and particles against the oracle after 40 steps."""
    import paper_1503_00276_gb300 as pg
    dx = (0.05, 0.2, 1.0)
    g = workload.Grid(ndim=2, nx=(128, 16, 1), dx=dx, dt=workload.courant_dt(dx, 2), move_window=True,
                      window_start=1.0)
    sp = workload.Species(ppc=(2, 1, 1), uth=(0.02, 0.02, 0.02), seed=61)
    las = workload.Laser(vosc=0.5, rkkp=8.0, w0=1.2, rise=0.6, length=0.0, fall=0.6, start=0.1, antenna=True,
                         focus=2.0)
    x, u = workload.load_particles(g, sp)
    ref = oracle.State(g, [sp], [x], [u], [workload.macro_charge(g, sp)])
    ref.add_antenna(las)
    sim = pg.Simulation(g, [sp], precision="fp32", tile=(32, 16), track_ids=True)
    sim.add_laser(las)
    n = 40
    ref.step(n)
    sim.step(n)
    assert ref.shifts == int(np.floor((n * g.dt - 1.0) / dx[0])) and ref.shifts > 0
    for c, name in enumerate(NAMES):
        m = np.max(np.abs(ref.fld[c]))
        if m > 0:
            assert np.max(np.abs(sim.fields(name) - ref.fld[c])) < 1e-4 * m, name
    assert np.max(np.abs(ref.fld[1])) > 0.5  # the pulse is in
    ids = sim.ids()
    assert np.array_equal(np.sort(ids), np.sort(ref.ids[0]))
    sim.close()
