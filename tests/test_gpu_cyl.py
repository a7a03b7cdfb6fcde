"""GPU parity of the 2D cylindrically symmetric (r-z) mode against the r-z
oracle on the same seeded inputs (FP64 plain form both sides: positions and
momenta 1e-10, fields and current densities 1e-10 of their largest value,
diagnostics 1e-10 relative), and the discrete invariants on the library's own
outputs."""
import math

import numpy as np
import pytest

import workload
from oracle.cyl import CylState

pytestmark = pytest.mark.gpu

NAMES = ["E1", "E2", "E3", "B1", "B2", "B3"]


def _grid(nz=32, nr=16, rho_bg=1.0, b0=(0.0, 0.0, 0.0), e0=(0.0, 0.0, 0.0)):
    return workload.cyl_grid(nz, nr, 0.1, 0.1, rho_bg=rho_bg, b0=b0, e0=e0)


def _oracle(g, parts, fields=None):
    s = CylState(g.nx[0], g.nx[1], g.dx[0], g.dx[1], g.dt, zmin=g.xmin[0], e0=g.e0, b0=g.b0, rho_bg=g.rho_bg)
    for x, u, q, rqm, w in parts:
        s.add_species(x, u, q, rqm, w)
    if fields is not None:
        for c in range(6):
            s.F[c][: g.nx[1]] = fields[c]
        s.boundary_fields()
    return s


def _sim(g, sps, parts, fields=None):
    import paper_1503_00276_gb300 as pg
    sim = pg.Simulation(g, sps, precision="fp64", explicit=[(x, u, q, w) for x, u, q, rqm, w in parts],
                        track_ids=True)
    if fields is not None:
        for c, name in enumerate(NAMES):
            sim.set_field(name, fields[c][None])
    return sim


def _column(seed=61, uth=0.2, nz=32, nr=16):
    g = _grid(nz, nr)
    sp = workload.Species(rqm=-1.0, ppc=(2, 2, 1), uth=(uth,) * 3, density=1.0, seed=seed)
    x, u = workload.load_cylindrical(g, sp)
    rng = np.random.default_rng(seed + 1)
    f = [rng.normal(0.0, 0.05, (nr, nz)) for _ in range(6)]
    return g, sp, [(x, u, workload.macro_charge(g, sp), sp.rqm, None)], f


def _close(a, b, tol, scale=None):
    s = np.max(np.abs(b)) if scale is None else scale
    assert np.max(np.abs(a - b)) <= tol * max(s, 1e-300), (np.max(np.abs(a - b)), s)


def test_parity_with_the_oracle_fp64():
    g, sp, parts, f = _column()
    ref = _oracle(g, parts, f)
    sim = _sim(g, [sp], parts, f)
    for _ in range(10):
        ref.step(1)
        sim.step(1)
    x, u = sim.particles(0)
    ids = sim.ids(0)
    rx, ru = ref.species[0]["x"][ids], ref.species[0]["u"][ids]
    L = g.nx[0] * g.dx[0]
    dz = x[:, 0] - rx[:, 0]
    dz = dz - L * np.round(dz / L)
    assert np.max(np.abs(dz)) <= 1e-10 * g.dx[0]
    assert np.max(np.abs(x[:, 1] - rx[:, 1])) <= 1e-10 * g.dx[1]
    assert np.max(np.abs(u - ru) / (1.0 + np.abs(ru))) <= 1e-10
    nr = g.nx[1]
    for c, name in enumerate(NAMES):
        _close(sim.fields(name)[0], ref.F[c][:nr], 1e-10)
    for c, name in enumerate(["J1", "J2", "J3"]):
        _close(sim.fields(name)[0], ref.J[c][:nr], 1e-10)
    d = sim.diag()
    assert abs(d["field_energy"] - ref.field_energy()) <= 1e-10 * ref.field_energy()
    assert abs(d["kinetic_energy"] - ref.kinetic_energy()) <= 1e-10 * ref.kinetic_energy()
    assert abs(d["total_charge"] - ref.total_charge()) <= 1e-12 * abs(ref.total_charge())
    rho = ref.rho()
    assert abs(d["rho_particles_abs_max"] - np.abs(rho[1:nr]).max()) <= 1e-10 * np.abs(rho[1:nr]).max()
    assert abs(d["gauss_resid_max"] - np.abs(ref.gauss_residual()).max()) <= 1e-10 * np.abs(rho[1:nr]).max()
    _close(sim.fields("RHO")[0][1:nr], rho[1:nr], 1e-12)
    sim.close()


def test_device_lattice_matches_the_input_recipe():
    """The device lattice loader with the reflection of the first cell and the
    ring weights w = r equals workload.load_cylindrical."""
    import paper_1503_00276_gb300 as pg
    g = _grid(16, 12)
    sp = workload.Species(rqm=-1.0, ppc=(2, 3, 1), uth=(0.1,) * 3, density=1.0, seed=5)
    sim = pg.Simulation(g, [sp], precision="fp64", track_ids=True)
    x, u = sim.particles(0)
    ids = sim.ids(0)
    rx, ru = workload.load_cylindrical(g, sp)
    np.testing.assert_array_equal(x[:, :2], rx[ids, :2])
    np.testing.assert_allclose(u, ru[ids], rtol=1e-14, atol=1e-16)
    np.testing.assert_array_equal(sim.weights(0), rx[ids, 1])
    # uniform column: rho = -1 exactly at the node rows off the axis
    np.testing.assert_allclose(sim.fields("RHO")[0][2:12], -1.0, rtol=0, atol=1e-13)
    sim.close()


def test_absorption_at_the_wall_matches_the_oracle():
    g = _grid(16, 12, rho_bg=0.0)
    rng = np.random.default_rng(4)
    n = 64
    x = np.c_[rng.uniform(0, 1.6, n), rng.uniform(0.6, 1.1, n), np.zeros(n)]
    u = np.c_[rng.normal(0, 0.3, n), rng.uniform(0.5, 4.0, n), rng.normal(0, 1.0, n)]
    parts = [(x, u, -0.01, -1.0, None)]
    sp = workload.Species(rqm=-1.0)
    ref = _oracle(g, parts)
    sim = _sim(g, [sp], parts)
    ref.step(8)
    sim.step(8)
    xs, us = sim.particles(0)
    ids = sim.ids(0)
    dead_ref = ref.species[0]["x"][ids, 1] < 0
    assert dead_ref.sum() > n // 4
    np.testing.assert_array_equal(xs[:, 1] < 0, dead_ref)
    np.testing.assert_array_equal(xs[dead_ref, 1], -1.0)
    np.testing.assert_array_equal(us[dead_ref], 0.0)
    live = ~dead_ref
    assert np.max(np.abs(xs[live, 1] - ref.species[0]["x"][ids[live], 1])) <= 1e-10
    d = sim.diag()
    assert abs(d["total_charge"] - ref.total_charge()) <= 1e-12 * abs(ref.total_charge())
    sim.close()


def _div_e_minus_rho(sim, g):
    Ez, Er, rho = sim.fields("E1")[0], sim.fields("E2")[0], sim.fields("RHO")[0]
    nr, dz, dr = g.nx[1], g.dx[0], g.dx[1]
    j = np.arange(1, nr)
    rn, rh = (j - 0.5) * dr, j * dr
    div = (Ez[j] - np.roll(Ez, 1, axis=1)[j]) / dz + (rh[:, None] * Er[j] - (rh - dr)[:, None] * Er[j - 1]) / (
        rn[:, None] * dr)
    return div - rho[j] - g.rho_bg


def _div_b(sim, g):
    Bz, Br = sim.fields("B1")[0], sim.fields("B2")[0]
    nr, dz, dr = g.nx[1], g.dx[0], g.dx[1]
    dBz = (np.roll(Bz, -1, axis=1) - Bz) / dz
    out = [4.0 * Br[1] / dr + dBz[0]]
    for j in range(1, nr - 1):
        out.append(((j + 0.5) * Br[j + 1] - (j - 0.5) * Br[j]) / (j * dr) + dBz[j])
    return np.array(out)


def test_gauss_and_div_b_invariants_on_the_device():
    """div E - rho constant at every node and div B = 0 in every cell (axis disc
    included), computed here from the library's exported fields."""
    g, sp, parts, f = _column(seed=9, uth=0.3)
    for c in range(3, 6):
        f[c][:] = 0.0
    sim = _sim(g, [sp], parts, f)
    r0 = _div_e_minus_rho(sim, g)
    sim.step(20)
    r1 = _div_e_minus_rho(sim, g)
    assert np.max(np.abs(r1 - r0)) <= 1e-11 * np.max(np.abs(r0))
    bmax = max(np.abs(sim.fields(n)[0]).max() for n in ("B1", "B2", "B3"))
    assert bmax > 1e-4
    assert np.max(np.abs(_div_b(sim, g))) <= 1e-11 * bmax / g.dx[1]
    sim.close()


def test_axis_centred_gyration_on_the_device():
    """The closed-form pin of the oracle, through the C ABI: a ring on the
    discrete Boris circle about the axis keeps r = R (uniform axial b0, charge
    too small to raise fields)."""
    B, rqm = 2.0, -1.0
    g = _grid(16, 40, rho_bg=0.0, b0=(B, 0.0, 0.0))
    umag = 0.6
    gam = math.sqrt(1 + umag * umag)
    theta = 2.0 * math.atan(abs(g.dt * B / (2.0 * rqm)) / gam)
    R = (umag / gam) * g.dt / (2.0 * math.sin(theta / 2))
    sgn = 1.0 if B / rqm < 0 else -1.0
    u = np.array([[0.0, umag * math.sin(theta / 2), sgn * umag * math.cos(theta / 2)]])
    sim = _sim(g, [workload.Species(rqm=rqm)], [(np.array([[0.8, R, 0.0]]), u, -1e-30, rqm, None)])
    for _ in range(5):
        sim.step(10)
        x, _ = sim.particles(0)
        assert abs(x[0, 1] - R) <= 1e-12 * R
    sim.close()


@pytest.mark.parametrize("case", ["batch", "xmin", "courant", "smooth"])
def test_unsupported_r_z_options_are_refused(case):
    import dataclasses

    import paper_1503_00276_gb300 as pg
    g = _grid(16, 8)
    sps = [workload.Species(rqm=-1.0, ppc=(1, 1, 1))]
    if case == "batch":
        with pytest.raises(pg.PicError) as e:
            pg.Batch([(g, sps), (g, sps)], tile=(16, 8))
        assert e.value.code == -8  # PIC_EUNSUPPORTED: the batched step has no r-z solve
        return
    if case == "xmin":
        g = dataclasses.replace(g, xmin=(0.0, 0.0, 0.0))
    elif case == "courant":
        g = dataclasses.replace(g, dt=workload.courant_dt(g.dx, 2, 0.99))
    elif case == "smooth":
        g = dataclasses.replace(g, smooth_level=(1, 0, 0))
    with pytest.raises(pg.PicError) as e:
        pg.Simulation(g, sps, precision="fp64")
    assert e.value.code == {"xmin": -1, "courant": -4, "smooth": -8}[case]


def test_checkpoint_roundtrip_in_the_r_z_mode(tmp_path):
    """Save / load keeps the mode, the ring weights and the absorbed slots bit
    for bit, and the restored run continues like the uninterrupted one."""
    import paper_1503_00276_gb300 as pg
    g = _grid(16, 12, rho_bg=0.0)
    rng = np.random.default_rng(8)
    n = 96
    x = np.c_[rng.uniform(0, 1.6, n), rng.uniform(0.0, 1.1, n), np.zeros(n)]
    u = np.c_[rng.normal(0, 0.3, n), rng.normal(0.5, 1.5, n), rng.normal(0, 1.0, n)]
    a = _sim(g, [workload.Species(rqm=-1.0)], [(x, u, -0.01, -1.0, None)])
    a.step(6)
    path = tmp_path / "rz.ckpt"
    a.save(path)
    b = pg.Simulation.load(path)
    assert b.info()["coords"] == 1
    for s in (a, b):
        assert (s.particles(0)[0][:, 1] < 0).any()  # some rings were absorbed
    np.testing.assert_array_equal(a.particles(0)[0], b.particles(0)[0])
    np.testing.assert_array_equal(a.weights(0), b.weights(0))
    for name in NAMES:
        np.testing.assert_array_equal(a.fields(name), b.fields(name))
    a.step(4)
    b.step(4)
    np.testing.assert_allclose(b.particles(0)[0], a.particles(0)[0], rtol=0, atol=1e-12)
    assert abs(a.diag()["field_energy"] - b.diag()["field_energy"]) <= 1e-12 * a.diag()["field_energy"]
    a.close()
    b.close()


# ---------------------------------------------------------------- FP32 tiled form
def _sim32(g, sps, parts, fields=None, tile=(16, 16)):
    import paper_1503_00276_gb300 as pg
    sim = pg.Simulation(g, sps, precision="fp32", tile=tile, track_ids=True,
                        explicit=[(x, u, q, w) for x, u, q, rqm, w in parts])
    if fields is not None:
        for c, name in enumerate(NAMES):
            sim.set_field(name, fields[c][None])
    return sim


@pytest.mark.parametrize("tile", [(16, 16), (32, 16)])
def test_fp32_one_step_matches_the_oracle(tile):
    """The tile kernel's ring move (pseudo-3D move and rotation in FP32, the
    radial step without cancellation) against the FP64 oracle: positions 2e-5
    of a cell, momenta 2e-5 (1 + |u|), currents and fields 2e-5 of their
    largest value."""
    g, sp, parts, f = _column(seed=33, uth=0.3)
    ref = _oracle(g, parts, f)
    sim = _sim32(g, [sp], parts, f, tile)
    ref.step(1)
    sim.step(1)
    x, u = sim.particles(0)
    ids = sim.ids(0)
    rx, ru = ref.species[0]["x"][ids], ref.species[0]["u"][ids]
    L = g.nx[0] * g.dx[0]
    dz = x[:, 0] - rx[:, 0]
    dz = dz - L * np.round(dz / L)
    assert np.max(np.abs(dz)) <= 2e-5 * g.dx[0]
    assert np.max(np.abs(x[:, 1] - rx[:, 1])) <= 2e-5 * g.dx[1]
    assert np.max(np.abs(u - ru) / (1.0 + np.abs(ru))) <= 2e-5
    nr = g.nx[1]
    for c, name in enumerate(["J1", "J2", "J3"]):
        _close(sim.fields(name)[0], ref.J[c][:nr], 2e-5)
    for c, name in enumerate(NAMES):
        _close(sim.fields(name)[0], ref.F[c][:nr], 2e-5)
    d = sim.diag()
    assert abs(d["kinetic_energy"] - ref.kinetic_energy()) <= 1e-5 * ref.kinetic_energy()
    assert abs(d["field_energy"] - ref.field_energy()) <= 1e-5 * ref.field_energy()
    assert abs(d["total_charge"] - ref.total_charge()) <= 1e-6 * abs(ref.total_charge())
    sim.close()


def test_fp32_gauss_invariant_and_drift_over_ten_steps():
    g, sp, parts, f = _column(seed=35, uth=0.3)
    ref = _oracle(g, parts, f)
    sim = _sim32(g, [sp], parts, f)
    r0 = _div_e_minus_rho(sim, g)
    rho_scale = np.abs(sim.fields("RHO")[0][1:g.nx[1]]).max()
    ref.step(10)
    sim.step(10)
    r1 = _div_e_minus_rho(sim, g)
    assert np.max(np.abs(r1 - r0)) <= 1e-5 * rho_scale
    x, _ = sim.particles(0)
    ids = sim.ids(0)
    assert np.max(np.abs(x[:, 1] - ref.species[0]["x"][ids, 1])) <= 1e-3 * g.dx[1]
    sim.close()


def test_fp32_absorption_removes_the_same_rings():
    g = _grid(16, 16, rho_bg=0.0)
    rng = np.random.default_rng(4)
    n = 64
    x = np.c_[rng.uniform(0, 1.6, n), rng.uniform(1.0, 1.5, n), np.zeros(n)]
    u = np.c_[rng.normal(0, 0.3, n), rng.uniform(0.5, 4.0, n), rng.normal(0, 1.0, n)]
    parts = [(x, u, -0.01, -1.0, None)]
    ref = _oracle(g, parts)
    sim = _sim32(g, [workload.Species(rqm=-1.0)], parts)
    ref.step(8)
    sim.step(8)
    live_ref = np.nonzero(ref.species[0]["x"][:, 1] >= 0)[0]
    ids = np.sort(sim.ids(0))
    assert n // 4 < n - live_ref.size
    np.testing.assert_array_equal(ids, live_ref)
    assert sim.n_particles(0) == live_ref.size
    xs, _ = sim.particles(0)
    o = np.argsort(sim.ids(0))
    assert np.max(np.abs(xs[o, 1] - ref.species[0]["x"][live_ref, 1])) <= 1e-4
    sim.close()


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_uniform_column_residual_sits_on_the_first_row_and_stays(prec):
    """The r-z benchmark column (uniform lattice-loaded electrons, fixed ion
    background 1, no initial E): the particles' density is -1 exactly on node
    rows 2 .. nr-1, but -1.375 on row 1 (the fold of the mirror row below the
    axis, whose rings all land on the first node row), so div E - rho - rho_bg
    starts at +0.375 there and nowhere else.  The scheme conserves charge, so
    that residual stays as it is: pic_diag's maximum after 20 steps equals the
    initial one to 1e-5 of the particles' largest |rho| (FP32; 1e-10 FP64)."""
    import paper_1503_00276_gb300 as pg
    g, sps, _ = workload.config_cyl(nz=64, nr=32)
    sim = pg.Simulation(g, sps, precision=prec)
    r0 = _div_e_minus_rho(sim, g)
    np.testing.assert_allclose(r0[0], 0.375, atol=1e-6)
    assert np.max(np.abs(r0[1:])) < 1e-6
    d0 = sim.diag()
    assert abs(d0["gauss_resid_max"] - 0.375) < 1e-6
    sim.step(20)
    d1 = sim.diag()
    tol = 1e-5 if prec == "fp32" else 1e-10
    assert abs(d1["gauss_resid_max"] - d0["gauss_resid_max"]) <= tol * d1["rho_particles_abs_max"]
    r1 = _div_e_minus_rho(sim, g)
    assert np.max(np.abs(r1 - r0)) <= tol * d1["rho_particles_abs_max"]
    sim.close()
