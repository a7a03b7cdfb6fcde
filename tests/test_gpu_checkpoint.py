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
