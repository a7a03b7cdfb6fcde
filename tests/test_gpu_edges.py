"""Edge cases of the GPU path against the oracle: a species with no particles
(the fields evolve as in vacuum), particles exactly on cell nodes, faces and
box corners and one ulp below the upper face (the FP32 offset rounds to 1
and carries into the next cell), and r-z rings on the axis, on the first
face and at node radii.  Tolerances as in the parity tests: FP64 1e-12 of a
cell after 3 steps, FP32 2e-5."""
import dataclasses

import numpy as np
import pytest

import oracle
import workload
from oracle.cyl import CylState

pytestmark = pytest.mark.gpu

NAMES = ["E1", "E2", "E3", "B1", "B2", "B3"]
DX = (0.1, 0.1, 0.1)


def _grid():
    return workload.Grid(ndim=3, nx=(16, 16, 8), dx=DX, dt=workload.courant_dt(DX, 3), b0=(0.0, 0.0, 0.1),
                         rho_bg=0.0)


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 2e-5)])
def test_empty_species_leaves_a_vacuum_field_solve(prec, tol):
    import paper_1503_00276_gb300 as pg
    g = _grid()
    zero = (np.array([0.0, 1.6]), np.array([0.0, 0.0]))
    sp = workload.Species(ppc=(2, 1, 1), uth=(0.1,) * 3, seed=3, profile=(zero, None, None), den_min=0.0)
    f = workload.random_fields(g, seed=11, amp=0.2)
    ref = oracle.from_workload(g, [sp], fields=f)
    assert ref.x[0].shape[0] == 0
    sim = pg.Simulation(g, [sp], precision=prec, tile=(8, 8, 8) if prec == "fp32" else None)
    for c, name in enumerate(NAMES):
        sim.set_field(name, f[c])
    assert sim.n_particles() == 0
    for _ in range(3):
        ref.particle_phase()
        ref.field_solve()
    sim.step(3)
    for c, name in enumerate(NAMES):
        assert np.max(np.abs(sim.fields(name) - ref.fld[c])) <= tol * np.max(np.abs(ref.fld[c])), name
    d = sim.diag()
    assert d["n_particles"] == 0 and d["kinetic_energy"] == 0.0 and d["total_charge"] == 0.0
    sim.close()


def _degenerate_particles(g):
    L = np.array([g.nx[d] * g.dx[d] for d in range(3)])
    pts = [
        [0.0, 0.0, 0.0],                        # the box's lower corner
        [0.3, 0.5, 0.2],                        # a node
        [0.3, 0.55, 0.25],                      # on an x1 face
        [0.35, 0.5, 0.25],                      # on an x2 face
        [0.35, 0.55, 0.2],                      # on an x3 face
        [0.8, 0.8, 0.4],                        # a tile corner
        [np.nextafter(L[0], 0.0), 0.75, 0.35],  # one ulp below the upper x1 face
        [0.45, np.nextafter(L[1], 0.0), 0.05],  # one ulp below the upper x2 face
        [1.15, 0.95, np.nextafter(L[2], 0.0)],  # one ulp below the upper x3 face
    ]
    x = np.array(pts * 3, dtype=np.float64)
    rng = np.random.default_rng(17)
    u = np.zeros_like(x)
    u[len(pts):2 * len(pts)] = rng.normal(0.0, 0.3, (len(pts), 3))
    u[2 * len(pts):] = rng.normal(0.0, 2.0, (len(pts), 3))  # face crossings in every direction
    return x, u


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 2e-5)])
def test_particles_on_nodes_faces_and_the_upper_edge(prec, tol):
    import paper_1503_00276_gb300 as pg
    g = _grid()
    x, u = _degenerate_particles(g)
    f = workload.random_fields(g, seed=21, amp=0.2)
    sp = workload.Species()
    q = -0.05
    ref = oracle.State(g, [sp], [x], [u], [q], fields=f)
    sim = pg.Simulation(g, [sp], precision=prec, explicit=[(x, u, q)], tile=(8, 8, 8) if prec == "fp32" else None,
                        track_ids=True)
    for c, name in enumerate(NAMES):
        sim.set_field(name, f[c])
    for _ in range(3):
        ref.particle_phase()
        ref.field_solve()
    sim.step(3)
    xs, us = sim.particles()
    ids = sim.ids()
    L = np.array([g.nx[d] * g.dx[d] for d in range(3)])
    d = xs - ref.x[0][ids]
    d = d - L * np.round(d / L)
    assert np.max(np.abs(d) / np.array(DX)) <= tol
    assert np.max(np.abs(us - ref.u[0][ids]) / (1 + np.abs(ref.u[0][ids]))) <= tol
    assert np.all(xs >= 0.0) and np.all(xs < L)
    for c, name in enumerate(NAMES):
        assert np.max(np.abs(sim.fields(name) - ref.fld[c])) <= tol * np.max(np.abs(ref.fld[c])), name
    if prec == "fp32":  # every particle in the tile region its (returned) position says
        _, cref, _ = oracle.tile_bin(g, (8, 8, 8), xs)
        np.testing.assert_array_equal(sim.tile_counts(), cref)
    sim.close()


def test_rings_on_the_axis_faces_and_nodes():
    """r-z: rings exactly on the axis (r = 0), on the face r = dr/2 between the
    first two cells and at node radii, at rest and moving."""
    import paper_1503_00276_gb300 as pg
    g = workload.cyl_grid(16, 12, 0.1, 0.1, rho_bg=0.0, b0=(0.3, 0.0, 0.0))
    r = [0.0, 0.0, 0.05, 0.05, 0.15, 0.25, 0.65]
    z = [0.0, 0.35, 0.4, 0.45, 0.5, 0.1, 1.55]
    x = np.c_[z, r, np.zeros(len(r))]
    u = np.array([[0.0, 0.0, 0.0], [0.2, 0.3, 0.4], [0.0, -0.5, 0.1], [0.1, 0.5, -0.3], [0.3, -1.2, 0.2],
                  [-0.4, 0.0, 0.9], [1.0, 0.5, 0.5]])
    q = -0.02
    ref = CylState(g.nx[0], g.nx[1], g.dx[0], g.dx[1], g.dt, b0=g.b0)
    ref.add_species(x, u, q, -1.0)
    sim = pg.Simulation(g, [workload.Species(rqm=-1.0)], precision="fp64", explicit=[(x, u, q)], track_ids=True)
    ref.step(6)
    sim.step(6)
    xs, us = sim.particles(0)
    ids = sim.ids(0)
    assert np.all(xs[:, 1] >= 0.0)
    assert np.max(np.abs(xs[:, 1] - ref.species[0]["x"][ids, 1])) <= 1e-12
    assert np.max(np.abs(us - ref.species[0]["u"][ids]) / (1 + np.abs(ref.species[0]["u"][ids]))) <= 1e-12
    for c, name in enumerate(NAMES):
        m = np.max(np.abs(ref.F[c][:12]))
        assert np.max(np.abs(sim.fields(name)[0] - ref.F[c][:12])) <= 1e-11 * max(m, 1e-300), name
    sim.close()
