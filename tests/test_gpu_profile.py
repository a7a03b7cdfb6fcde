"""GPU parity of density profiles (per-particle charge weights) against the
oracle on the same seeded inputs: which lattice places get a particle (ids),
their weights, and the orbits, currents and fields they produce, in the FP64
plain form (1e-10 after 20 steps) and the FP32 tiled form (one step at 2e-5,
ten steps at 1e-4); explicit per-particle weights; a moving window whose front
reaches the plasma edge (injection with the profile at lab-frame positions);
checkpoint and restart with weights."""
import dataclasses

import numpy as np
import pytest

import oracle
import workload

pytestmark = pytest.mark.gpu

NAMES = ["E1", "E2", "E3", "B1", "B2", "B3"]
DX2 = (0.1, 0.1, 1.0)
# a vacuum gap below x1 = 0.8, then a linear ramp up to x1 = 2.4, then flat;
# in x2 a dip to 0.4 in the middle
PROF2 = (((0.0, 0.8, 0.8 + 1e-9, 2.4, 10.0), (0.0, 0.0, 0.2, 1.0, 1.0)), ((0.0, 0.8, 1.6), (1.0, 0.4, 1.0)))


def _setup2(uth=0.3):
    g = workload.Grid(ndim=2, nx=(32, 16, 1), dx=DX2, dt=workload.courant_dt(DX2, 2), rho_bg=0.0,
                      b0=(0.0, 0.0, 0.2))
    sp = workload.Species(ppc=(2, 2, 1), uth=(uth,) * 3, seed=71, density=1.3, profile=PROF2, den_min=1e-6)
    f = workload.random_fields(g, seed=72, amp=0.1)
    return g, sp, f


def _sim(g, sps, prec, f=None, tile=None, explicit=None):
    import paper_1503_00276_gb300 as pg
    sim = pg.Simulation(g, sps, precision=prec, tile=tile, track_ids=True, explicit=explicit)
    if f is not None:
        for c, name in enumerate(NAMES):
            sim.set_field(name, f[c])
    return sim


def _match(sim, ref, s=0):
    ids = sim.ids(s)
    assert np.array_equal(np.sort(ids), np.sort(ref.ids[s]))
    pos = {int(i): k for k, i in enumerate(ref.ids[s])}
    return np.array([pos[int(i)] for i in ids])


def _perr(g, xa, xb):
    L = np.array([g.nx[0] * g.dx[0], g.nx[1] * g.dx[1], g.nx[2] * g.dx[2] if g.ndim == 3 else 1.0])
    d = xa - xb
    d = d - L * np.round(d / L)
    return np.max(np.abs(d[:, :g.ndim] / np.array(g.dx[:g.ndim])))


def test_profile_fp64_plain_20_steps_matches_oracle():
    g, sp, f = _setup2()
    ref = oracle.from_workload(g, [sp], fields=f)
    sim = _sim(g, [sp], "fp64", f)
    order = _match(sim, ref)
    np.testing.assert_allclose(sim.weights(), ref.w[0][order], rtol=0, atol=1e-15)
    ref.step(20)
    sim.step(20)
    order = _match(sim, ref)
    x, u = sim.particles()
    assert _perr(g, x, ref.x[0][order]) < 1e-10
    assert np.max(np.abs(u - ref.u[0][order])) < 1e-10
    for c, name in enumerate(NAMES):
        assert np.max(np.abs(sim.fields(name) - ref.fld[c])) < 1e-9 * np.max(np.abs(ref.fld[c])), name
    d = sim.diag()
    assert abs(d["kinetic_energy"] - ref.kinetic_energy()) < 1e-9 * abs(ref.kinetic_energy())
    sim.close()


@pytest.mark.parametrize("ndim", [2, 3])
def test_profile_fp32_one_and_ten_steps_match_oracle(ndim):
    if ndim == 2:
        g, sp, f = _setup2()
        tile = (16, 16)
    else:
        dx = (0.1, 0.1, 0.1)
        g = workload.Grid(ndim=3, nx=(32, 16, 16), dx=dx, dt=workload.courant_dt(dx, 3), rho_bg=0.0)
        prof = (PROF2[0], None, ((0.0, 1.6), (0.5, 1.5)))
        sp = workload.Species(ppc=(2, 1, 1), uth=(0.3,) * 3, seed=73, profile=prof, den_min=1e-6)
        f = workload.random_fields(g, seed=74, amp=0.1)
        tile = (8, 8, 8)
    ref = oracle.from_workload(g, [sp], fields=f)
    sim = _sim(g, [sp], "fp32", f, tile=tile)
    order = _match(sim, ref)
    np.testing.assert_allclose(sim.weights(), ref.w[0][order], rtol=1e-7, atol=0)
    ref.particle_phase()
    jref = [c.copy() for c in ref.cur]
    ref.field_solve()
    sim.step(1)
    order = _match(sim, ref)
    x, u = sim.particles()
    assert _perr(g, x, ref.x[0][order]) < 2e-5
    assert np.max(np.abs(u - ref.u[0][order]) / (1 + np.abs(ref.u[0][order]))) < 2e-5
    for c, name in enumerate(["J1", "J2", "J3"]):
        jm = np.max(np.abs(jref[c]))
        assert np.max(np.abs(sim.fields(name) - jref[c])) < 2e-5 * jm, name
    ref.step(9)
    sim.step(9)
    order = _match(sim, ref)
    x, u = sim.particles()
    assert _perr(g, x, ref.x[0][order]) < 1e-4
    assert np.max(np.abs(u - ref.u[0][order])) < 1e-4
    np.testing.assert_allclose(sim.fields("RHO"), ref.rho(), rtol=0, atol=2e-5 * np.max(np.abs(ref.rho())))
    sim.close()


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("fp32", 2e-5)])
def test_explicit_weights_match_oracle(prec, tol):
    g, sp, f = _setup2()
    sp = dataclasses.replace(sp, profile=None)
    x, u = workload.load_particles(g, sp)
    w = 0.5 + np.random.default_rng(5).random(x.shape[0])
    q = workload.macro_charge(g, sp)
    ref = oracle.State(g, [sp], [x], [u], [q], fields=f, weights=[w])
    sim = _sim(g, [sp], prec, f, tile=(16, 16) if prec == "fp32" else None, explicit=[(x, u, q, w)])
    ref.particle_phase()
    jref = [c.copy() for c in ref.cur]
    sim.step(1)
    for c, name in enumerate(["J1", "J2", "J3"]):
        jm = np.max(np.abs(jref[c]))
        assert np.max(np.abs(sim.fields(name) - jref[c])) < tol * jm, name
    sim.close()


def test_moving_window_reaches_a_profiled_plasma():
    """The window starts in vacuum; the plasma begins 0.6 beyond its front.
    After the front passes the edge, the injected particles carry the profile
    (a ramp) at their lab-frame positions, as in the oracle."""
    dx = (0.1, 0.2, 1.0)
    g = workload.Grid(ndim=2, nx=(40, 8, 1), dx=dx, dt=workload.courant_dt(dx, 2), move_window=True, rho_bg=0.0)
    edge = 4.6
    prof = (((0.0, edge, edge + 1e-9, edge + 2.0, 100.0), (0.0, 0.0, 0.1, 1.0, 1.0)), None)
    sp = workload.Species(ppc=(2, 2, 1), uth=(0.05,) * 3, profile=prof, den_min=1e-6, seed=9)
    ref = oracle.from_workload(g, [sp])
    sim = _sim(g, [sp], "fp32")
    assert sim.n_particles() == 0 and ref.x[0].shape[0] == 0
    ref.step(20)
    sim.step(20)
    assert ref.x[0].shape[0] > 0
    assert sim.n_particles() == ref.x[0].shape[0]
    order = _match(sim, ref)
    np.testing.assert_allclose(sim.weights(), ref.w[0][order], rtol=1e-7, atol=0)
    x, u = sim.particles()
    d = x - ref.x[0][order]
    d[:, 1] -= g.nx[1] * dx[1] * np.round(d[:, 1] / (g.nx[1] * dx[1]))
    assert np.max(np.abs(d[:, :2] / np.array(dx[:2]))) < 1e-4
    sim.close()


def test_checkpoint_keeps_weights(tmp_path):
    import paper_1503_00276_gb300 as pg
    g, sp, f = _setup2()
    a = _sim(g, [sp], "fp32", f, tile=(16, 16))
    a.step(3)
    a.save(tmp_path / "w.ckpt")
    b = pg.Simulation.load(tmp_path / "w.ckpt")
    oa, ob = np.argsort(a.ids()), np.argsort(b.ids())
    np.testing.assert_array_equal(a.weights()[oa], b.weights()[ob])
    a.step(4)
    b.step(4)
    oa, ob = np.argsort(a.ids()), np.argsort(b.ids())
    xa, _ = a.particles()
    xb, _ = b.particles()
    assert np.max(np.abs(xa[oa] - xb[ob])) < 1e-5
    a.close()
    b.close()


def test_tile_shapes_without_a_usable_kernel_are_rejected():
    """A tile shape built only for the small-tile kernel cannot hold a species
    with charge weights or run a moving window: pic_init says so instead of
    stepping nothing."""
    import paper_1503_00276_gb300 as pg
    g, sp, f = _setup2()
    with pytest.raises(RuntimeError, match="small-tile kernel"):
        pg.Simulation(g, [sp], precision="fp32", tile=(16, 8))
    gw = dataclasses.replace(g, move_window=True)
    with pytest.raises(RuntimeError, match="small-tile kernel"):
        pg.Simulation(gw, [dataclasses.replace(sp, profile=None)], precision="fp32", tile=(8, 4))
