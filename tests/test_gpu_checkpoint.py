"""Checkpoint / restart on the GPU: the restored state equals the saved one
bit for bit (particles by id, E/B, step count), in both forms, and the
restored run continues like the uninterrupted one (FP32: 1e-4 of a cell / of
u after 5 steps, the order-dependent FP32 current sums being the only
difference; FP64: 1e-12)."""
import numpy as np
import pytest

import workload

pytestmark = pytest.mark.gpu

NAMES = ["E1", "E2", "E3", "B1", "B2", "B3"]


def _state(sim):
    x, u = sim.particles()
    ids = sim.ids()
    o = np.argsort(ids)
    return ids[o], x[o], u[o], [sim.fields(n) for n in NAMES]


@pytest.mark.parametrize("prec,tol", [("fp32", 1e-4), ("fp64", 1e-12)])
def test_checkpoint_roundtrip_and_continuation(tmp_path, prec, tol):
    import paper_1503_00276_gb300 as pg
    dx = (0.1, 0.1, 0.1)
    g = workload.Grid(ndim=3, nx=(32, 16, 16), dx=dx, dt=workload.courant_dt(dx, 3), b0=(0.0, 0.0, 0.2))
    sps = [workload.Species(ppc=(2, 1, 1), uth=(0.3,) * 3, seed=5),
           workload.Species(rqm=100.0, ppc=(1, 1, 1), uth=(0.01,) * 3, seed=6)]
    a = pg.Simulation(g, sps, precision=prec, tile=(8, 8, 8) if prec == "fp32" else None, track_ids=True)
    a.step(7)
    path = tmp_path / "run.ckpt"
    a.save(path)
    b = pg.Simulation.load(path)
    assert b.info()["step"] == 7 and b.nspecies == 2
    sa, sb = _state(a), _state(b)
    np.testing.assert_array_equal(sa[0], sb[0])
    np.testing.assert_array_equal(sa[1], sb[1])
    np.testing.assert_array_equal(sa[2], sb[2])
    for fa, fb in zip(sa[3], sb[3]):
        np.testing.assert_array_equal(fa, fb)
    # the second species too
    xa, ua = a.particles(1)
    xb, ub = b.particles(1)
    oa, ob = np.argsort(a.ids(1)), np.argsort(b.ids(1))
    np.testing.assert_array_equal(xa[oa], xb[ob])
    np.testing.assert_array_equal(ua[oa], ub[ob])
    a.step(5)
    b.step(5)
    sa, sb = _state(a), _state(b)
    np.testing.assert_array_equal(sa[0], sb[0])
    L = np.array([g.nx[d] * dx[d] for d in range(3)])
    d = sa[1] - sb[1]
    d = d - L * np.round(d / L)
    assert np.max(np.abs(d / np.array(dx))) < tol
    assert np.max(np.abs(sa[2] - sb[2])) < tol
    assert a.diag()["step"] == b.diag()["step"] == 12
    a.close()
    b.close()


def test_checkpoint_mid_antenna_pulse_in_moving_window(tmp_path):
    """A pulse driven through the lower x1 boundary of a moving-window run
    (window still until t = 1, then moving at c): the run is saved at step 20,
    while the pulse is half way in, restored, and continued to step 40, past
    the start of the window's motion.  The restored run matches the
    uninterrupted one and the oracle (same antenna, State.window_step) to 1e-4:
    the restored state carries the pulse table, the shift count, the x1 origin
    and the injection counter."""
    import oracle
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
    a = pg.Simulation(g, [sp], precision="fp32", tile=(32, 16), track_ids=True)
    a.add_laser(las)
    a.step(20)
    assert 0.1 < 20 * g.dt < 0.1 + 1.2  # mid-entry: the pulse front is in, its tail is not
    path = tmp_path / "antenna.ckpt"
    a.save(path)
    b = pg.Simulation.load(path)
    assert b.info()["step"] == 20
    a.step(20)
    b.step(20)
    ref.step(40)
    assert ref.shifts > 0
    ia, ib = a.ids(), b.ids()
    assert np.array_equal(np.sort(ia), np.sort(ib)) and np.array_equal(np.sort(ib), np.sort(ref.ids[0]))
    xa, ua = a.particles()
    xb, ub = b.particles()
    oa, ob = np.argsort(ia), np.argsort(ib)
    L2 = g.nx[1] * dx[1]
    d = xa[oa] - xb[ob]
    d[:, 1] -= L2 * np.round(d[:, 1] / L2)
    assert np.max(np.abs(d[:, 0] / dx[0])) < 1e-4 and np.max(np.abs(d[:, 1] / dx[1])) < 1e-4
    assert np.max(np.abs(ua[oa] - ub[ob])) < 1e-4
    for c, name in enumerate(NAMES):
        m = np.max(np.abs(ref.fld[c]))
        if m == 0:
            continue
        fb = b.fields(name)
        assert np.max(np.abs(fb - a.fields(name))) < 1e-4 * m, name
        assert np.max(np.abs(fb - ref.fld[c])) < 1e-4 * m, name
    assert np.max(np.abs(ref.fld[1])) > 0.5  # the pulse got in after the restart too
    a.close()
    b.close()
