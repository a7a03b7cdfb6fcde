"""GPU parity: the CUDA path (through the C ABI) against the FP64 CPU oracle on the
same seeded inputs.

Tolerances:
* FP64 plain form: the per-particle arithmetic matches the oracle operation by
  operation; only the order of the FP64 atomic current sums differs, so after
  100 steps of the 64x64 workload positions agree to 1e-10 of a cell and momenta
  to 1e-10 of the thermal spread.
* FP32 cell-offset form: one step is compared particle by particle (by id) with
  |dx| <= 2e-5 cells, |du| <= 2e-5 (1 + |u|) -- a few hundred FP32 ulps of the
  in-cell offset, covering rsqrtf/__fdividef (2 ulp) and the FP32 accumulation
  of current; grid quantities to 2e-5 of their maximum.
"""
import math

import numpy as np
import pytest

import oracle
import workload

pytestmark = pytest.mark.gpu


def _pg():
    import paper_1503_00276_gb300 as pg
    return pg


def _sim(g, sps, prec, fields=None, tile=None, ids=True, explicit=True, sort_period=0):
    pg = _pg()
    ex = None
    if explicit:
        ex = []
        for s in sps:
            x, u = workload.load_particles(g, s)
            ex.append((x, u, workload.macro_charge(g, s)))
    sim = pg.Simulation(g, sps, precision=prec, explicit=ex, tile=tile, track_ids=ids, sort_period=sort_period)
    if fields is not None:
        for c, name in enumerate(["E1", "E2", "E3", "B1", "B2", "B3"]):
            sim.set_field(name, fields[c])
    return sim


def _box(g):
    return np.array([g.nx[d] * g.dx[d] if d < g.ndim else 1.0 for d in range(3)])


def _pos_err_cells(g, xa, xb):
    L = _box(g)
    d = xa - xb
    d = d - L * np.round(d / L)
    return np.max(np.abs(d[:, :g.ndim] / np.array(g.dx[:g.ndim])))


# ---------------------------------------------------------------- FP64 plain

def test_fp64_plain_config0_100_steps_matches_oracle():
    g, sps, nsteps = workload.config0()
    ref = oracle.from_workload(g, sps)
    sim = _sim(g, sps, "fp64")
    d0 = sim.diag()
    assert abs(d0["gauss_resid_max"] - ref.gauss_residual()) < 1e-12
    ref.step(nsteps)
    sim.step(nsteps)
    x, u = sim.particles()
    ids = sim.ids()
    np.testing.assert_array_equal(ids, np.arange(x.shape[0]))
    ex = _pos_err_cells(g, x, ref.x[0])
    eu = np.max(np.abs(u - ref.u[0])) / 0.01
    assert ex < 1e-10 and eu < 1e-10, (ex, eu)
    for c, name in enumerate(["E1", "E2", "E3", "B1", "B2", "B3"]):
        f = sim.fields(name)
        scale = max(np.max(np.abs(ref.fld[c])), 1e-300)
        assert np.max(np.abs(f - ref.fld[c])) <= 1e-9 * scale + 1e-18, name
    d = sim.diag()
    assert d["step"] == nsteps and d["error_flags"] == 0
    assert abs(d["field_energy"] - ref.field_energy()) < 1e-9 * ref.field_energy()
    assert abs(d["kinetic_energy"] - ref.kinetic_energy()) < 1e-9 * ref.kinetic_energy()
    assert d["gauss_resid_max"] < 1e-11
    sim.close()


@pytest.mark.parametrize("smooth", [0, 2])
def test_fp64_plain_3d_random_fields_matches_oracle(smooth):
    dx = (0.1, 0.12, 0.09)
    g = workload.Grid(ndim=3, nx=(12, 8, 10), dx=dx, dt=workload.courant_dt(dx, 3), smooth_level=(smooth,) * 3,
                      e0=(0.01, -0.02, 0.0), b0=(0.0, 0.05, 0.1))
    sp = workload.Species(ppc=(2, 1, 2), uth=(0.2, 0.1, 0.15), ufl=(0.05, 0.0, 0.0), seed=77)
    f = workload.random_fields(g, seed=5, amp=0.05)
    ref = oracle.from_workload(g, [sp], fields=f)
    sim = _sim(g, [sp], "fp64", fields=f)
    ref.step(20)
    sim.step(20)
    x, u = sim.particles()
    assert _pos_err_cells(g, x, ref.x[0]) < 1e-10
    assert np.max(np.abs(u - ref.u[0])) < 1e-10
    for c, name in enumerate(["J1", "J2", "J3"]):
        assert np.max(np.abs(sim.fields(name) - ref.cur[c])) < 1e-10 * np.max(np.abs(ref.cur[c]))
    sim.close()


# ---------------------------------------------------------------- FP32 tiled

CASES_32 = {
    # ndim, nx, tile, ppc lattice (ragged totals), thermal spread
    "3d_8x8x8": (3, (32, 16, 16), (8, 8, 8), (3, 1, 1), 0.3),
    "3d_16x8x4": (3, (32, 16, 8), (16, 8, 4), (1, 2, 1), 0.3),
    "2d_32x16": (2, (64, 32, 1), (32, 16), (3, 2, 1), 0.4),
    "2d_8x8": (2, (16, 8, 1), (8, 8), (2, 2, 1), 0.6),
    # small-tile kernel (whole tile staged in shared memory)
    "3d_4x4x4_small": (3, (16, 8, 12), (4, 4, 4), (3, 1, 1), 0.4),
    "3d_8x4x4_small": (3, (16, 16, 8), (8, 4, 4), (2, 1, 1), 0.4),
    "3d_4x4x2_small": (3, (8, 8, 8), (4, 4, 2), (1, 3, 1), 0.4),
    "2d_8x4_small": (2, (32, 16, 1), (8, 4), (3, 3, 1), 0.5),
    # small-tile kernel with tiles above its stage capacity (chunks from global memory)
    "3d_4x4x4_overfull": (3, (8, 8, 8), (4, 4, 4), (4, 2, 2), 0.4),
}


# sort_period 1: the cell-sorting kernel runs every step; 2: the first step of
# each period is the streaming (compacting) kernel
@pytest.mark.parametrize("sort_period", [1, 2])
@pytest.mark.parametrize("case", sorted(CASES_32))
def test_fp32_tiled_one_step_matches_oracle(case, sort_period):
    ndim, nx, tile, ppc, uth = CASES_32[case]
    dx = (0.1, 0.1, 0.1)
    g = workload.Grid(ndim=ndim, nx=nx, dx=dx, dt=workload.courant_dt(dx, ndim), e0=(0.0, 0.01, 0.0),
                      b0=(0.02, 0.0, 0.05))
    sp = workload.Species(ppc=ppc, uth=(uth,) * 3, seed=1234)
    f = workload.random_fields(g, seed=9, amp=0.2)
    ref = oracle.from_workload(g, [sp], fields=f)
    sim = _sim(g, [sp], "fp32", fields=f, tile=tile, sort_period=sort_period)
    # binning of the loaded particles is bit-exact
    _, counts, _ = oracle.tile_bin(g, tile if ndim == 3 else tuple(tile) + (1,), ref.x[0])
    np.testing.assert_array_equal(sim.tile_counts(), counts)
    ref.particle_phase()
    jref = [c.copy() for c in ref.cur]
    ref.field_solve()
    sim.step(1)
    x, u = sim.particles()
    ids = sim.ids()
    assert x.shape[0] == ref.x[0].shape[0]
    np.testing.assert_array_equal(np.sort(ids), np.arange(x.shape[0]))
    # the oracle wraps x after the deposit as the GPU does
    ex = _pos_err_cells(g, x, ref.x[0][ids])
    eu = np.max(np.abs(u - ref.u[0][ids]) / (1 + np.abs(ref.u[0][ids])))
    assert ex < 2e-5 and eu < 2e-5, (ex, eu)
    for c, name in enumerate(["J1", "J2", "J3"]):
        jm = np.max(np.abs(jref[c]))
        if jm == 0:
            continue
        assert np.max(np.abs(sim.fields(name) - jref[c])) < 2e-5 * jm, name
    for c, name in enumerate(["E1", "E2", "E3", "B1", "B2", "B3"]):
        assert np.max(np.abs(sim.fields(name) - ref.fld[c])) < 2e-5 * np.max(np.abs(ref.fld[c])), name
    # every particle sits in the tile region its cell says
    counts2 = sim.tile_counts()
    _, cref, _ = oracle.tile_bin(g, tile if ndim == 3 else tuple(tile) + (1,), x)
    np.testing.assert_array_equal(counts2, cref)
    sim.close()


# Current smoothing in the FP32 form (appendix nl_smooth: smooth_level passes
# of (w0, w1, w2) / sum per direction): J after the smoothing of one step,
# and the fields it drives, against the oracle's ora_smooth.  The weights are
# the default (1, 2, 1) or, per pass, a binomial pass followed by the
# compensator (-1, 6, -1) (a per-pass weight table).
SMOOTH_CASES = {
    "3d_8x8x8": ((2, 2, 2), None),
    "3d_8x8x8_compensated": ((2, 2, 2), [(1.0, 2.0, 1.0), (-1.0, 6.0, -1.0)]),
    "2d_32x16": ((2, 2, 0), None),
    "3d_4x4x4_small": ((1, 2, 1), None),
}


@pytest.mark.parametrize("sort_period", [1, 2])
@pytest.mark.parametrize("case", sorted(SMOOTH_CASES))
def test_fp32_tiled_smoothing_matches_oracle(case, sort_period):
    level, per_pass = SMOOTH_CASES[case]
    base = case.replace("_compensated", "")
    ndim, nx, tile, ppc, uth = CASES_32[base]
    dx = (0.1, 0.1, 0.1)
    sw = tuple(per_pass if per_pass else (1.0, 2.0, 1.0) for _ in range(3))
    g = workload.Grid(ndim=ndim, nx=nx, dx=dx, dt=workload.courant_dt(dx, ndim), smooth_level=level,
                      smooth_w=sw)
    sp = workload.Species(ppc=ppc, uth=(uth,) * 3, seed=4242)
    f = workload.random_fields(g, seed=19, amp=0.2)
    ref = oracle.from_workload(g, [sp], fields=f)
    sim = _sim(g, [sp], "fp32", fields=f, tile=tile, sort_period=sort_period)
    ref.particle_phase()
    raw = [c.copy() for c in ref.cur]
    ref.smooth_current()
    jref = [c.copy() for c in ref.cur]
    ref.field_solve()
    sim.step(1)
    for c, name in enumerate(["J1", "J2", "J3"]):
        jm = np.max(np.abs(jref[c]))
        assert jm > 0, name
        assert np.max(np.abs(raw[c] - jref[c])) > 0.05 * jm, name  # the smoothing is not a no-op here
        assert np.max(np.abs(sim.fields(name) - jref[c])) < 2e-5 * jm, name
    for c, name in enumerate(["E1", "E2", "E3", "B1", "B2", "B3"]):
        assert np.max(np.abs(sim.fields(name) - ref.fld[c])) < 2e-5 * np.max(np.abs(ref.fld[c])), name
    x, u = sim.particles()
    ids = sim.ids()
    assert _pos_err_cells(g, x, ref.x[0][ids]) < 2e-5
    sim.close()


@pytest.mark.parametrize("sort_period", [1, 3, 8])
def test_fp32_tiled_many_steps_close_to_oracle(sort_period):
    ndim, nx, tile, ppc, uth = CASES_32["3d_8x8x8"]
    dx = (0.1, 0.1, 0.1)
    g = workload.Grid(ndim=3, nx=nx, dx=dx, dt=workload.courant_dt(dx, 3))
    sp = workload.Species(ppc=ppc, uth=(uth,) * 3, seed=4321)
    ref = oracle.from_workload(g, [sp])
    sim = _sim(g, [sp], "fp32", tile=tile, sort_period=sort_period)
    ref.step(20)
    sim.step(20)
    x, u = sim.particles()
    ids = sim.ids()
    assert _pos_err_cells(g, x, ref.x[0][ids]) < 1e-4
    assert np.max(np.abs(u - ref.u[0][ids])) < 1e-4
    assert sim.diag()["error_flags"] == 0
    sim.close()


@pytest.mark.parametrize("sort_period", [1, 2])
def test_fp32_heavy_tiles_split_over_blocks_match_oracle(sort_period):
    """A dense drifting clump (60,000 particles, sigma = 3 cells) over a thin
    thermal background: the clump's tiles hold several slices of 8 chunks, so
    the tile kernel splits them over blocks.  Both species against the oracle
    after 6 steps, and the binning of the result bit-exact."""
    pg = _pg()
    dx = (0.1, 0.1, 0.1)
    g = workload.Grid(ndim=3, nx=(32, 16, 16), dx=dx, dt=workload.courant_dt(dx, 3))
    bg = workload.Species(ppc=(1, 1, 1), uth=(0.3, 0.3, 0.3), seed=808)
    clump = workload.Species(rqm=-1.0, ppc=(0, 0, 0), seed=809)
    cx, cu, cq = workload.beam_particles(g, 60000, (1.2, 0.4, 0.4), 0.3, 0.3, 1.5, 1.0, 809)
    bx, bu = workload.load_particles(g, bg)
    ref = oracle.State(g, [bg, clump], [bx, cx], [bu, cu], [workload.macro_charge(g, bg), cq])
    sim = pg.Simulation(g, [bg, clump], precision="fp32", explicit=[None, (cx, cu, cq)], tile=(8, 8, 8),
                        track_ids=True, sort_period=sort_period)
    counts = sim.tile_counts(1)
    assert counts.max() > 3 * 8192  # the heaviest tile is split into several slices
    ref.step(6)
    sim.step(6)
    # bit 1 (a region overflowed into the spill list, then re-binned) may be
    # set: the clump drifts into tiles sized for the background
    assert sim.diag()["error_flags"] & 1 == 0
    for s in range(2):
        x, u = sim.particles(s)
        ids = sim.ids(s)
        np.testing.assert_array_equal(np.sort(ids), np.arange(ref.x[s].shape[0]))
        assert _pos_err_cells(g, x, ref.x[s][ids]) < 1e-4, s
        assert np.max(np.abs(u - ref.u[s][ids]) / (1 + np.abs(ref.u[s][ids]))) < 1e-4, s
        _, cref, _ = oracle.tile_bin(g, (8, 8, 8), x)
        np.testing.assert_array_equal(sim.tile_counts(s), cref)
    for c, name in enumerate(["E1", "E2", "E3", "B1", "B2", "B3"]):
        m = np.max(np.abs(ref.fld[c]))
        assert np.max(np.abs(sim.fields(name) - ref.fld[c])) < 1e-4 * m, name
    sim.close()


def _energy_gate(fe32, fe64):
    """The FP32 field-energy gate against FP64 (reading of "within 1e-3
    relative of FP64"): at every step |fe32 - fe64| <= 1e-3 fe64[t] where the
    FP64 energy is at least 1e-2 of its history's maximum, and <= 1e-3 of that
    maximum elsewhere (early steps whose energy is near zero, where a relative
    bound would measure rounding only)."""
    fe32, fe64 = np.asarray(fe32), np.asarray(fe64)
    top = np.max(fe64)
    assert top > 0
    big = fe64 >= 1e-2 * top
    assert big.sum() >= len(fe64) // 2
    rel = np.abs(fe32 - fe64)[big] / fe64[big]
    assert np.max(rel) <= 1e-3, np.max(rel)
    assert np.max(np.abs(fe32 - fe64)) <= 1e-3 * top


def test_fp32_gauss_law_and_energy_history_vs_fp64():
    """The FP32 gates on the 64x64 workload: Gauss residual <= 1e-5 max|rho| at
    every step (net density, stricter than the particles' density), and the
    field-energy history against the FP64 plain form (_energy_gate)."""
    g, sps, nsteps = workload.config0()
    s64 = _sim(g, sps, "fp64", ids=False)
    s32 = _sim(g, sps, "fp32", ids=False)
    fe64, fe32 = [], []
    for _ in range(nsteps):
        s64.step(1)
        s32.step(1)
        d64, d32 = s64.diag(), s32.diag()
        fe64.append(d64["field_energy"])
        fe32.append(d32["field_energy"])
        assert d32["gauss_resid_max"] <= 1e-5 * d32["rho_abs_max"], d32
        assert d32["error_flags"] == 0
    _energy_gate(fe32, fe64)
    s64.close()
    s32.close()


def test_fp32_gates_on_3d_thermal_sub_box():
    """The same gates on a sub-box of the 3D throughput workload (64x32x32
    cells, 8 ppc = 524,288 electrons, u_th = 0.05, dx = 0.1, 8x8x8 tiles),
    100 steps: FP32 Gauss residual <= 1e-5 of the particles' max |rho| at every
    step, and the field-energy history (grown from zero by the thermal noise)
    against the FP64 plain form on the same particles."""
    g, sps, _ = workload.config3(8, seed=20004, nx=(64, 32, 32))
    s64 = _sim(g, sps, "fp64", ids=False)
    s32 = _sim(g, sps, "fp32", ids=False, tile=(8, 8, 8))
    fe64, fe32 = [], []
    for _ in range(100):
        s64.step(1)
        s32.step(1)
        d64, d32 = s64.diag(), s32.diag()
        fe64.append(d64["field_energy"])
        fe32.append(d32["field_energy"])
        assert d32["gauss_resid_max"] <= 1e-5 * d32["rho_particles_abs_max"], d32
        assert d32["error_flags"] == 0
        assert d32["n_particles"] == d64["n_particles"] == 524288
    _energy_gate(fe32, fe64)
    s64.close()
    s32.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_continuity_holds_on_gpu_outputs(prec):
    """(rho^{n+1} - rho^n)/dt + div J^{n+1/2} = 0 from the library's own rho, J."""
    dx = (0.1, 0.1, 0.1)
    g = workload.Grid(ndim=3, nx=(16, 16, 8), dx=dx, dt=workload.courant_dt(dx, 3))
    sp = workload.Species(ppc=(2, 2, 1), uth=(0.3,) * 3, seed=8)
    f = workload.random_fields(g, seed=2, amp=0.1)
    sim = _sim(g, [sp], prec, fields=f, tile=(8, 8, 8), ids=False)
    r0 = sim.fields("RHO")
    sim.step(1)
    r1 = sim.fields("RHO")
    J = [sim.fields(n) for n in ("J1", "J2", "J3")]
    div = ((J[0] - np.roll(J[0], 1, 2)) / dx[0] + (J[1] - np.roll(J[1], 1, 1)) / dx[1]
           + (J[2] - np.roll(J[2], 1, 0)) / dx[2])
    res = np.max(np.abs((r1 - r0) / g.dt + div))
    scale = np.max(np.abs(r0)) / g.dt
    assert res < (1e-12 if prec == "fp64" else 2e-5) * scale, res / scale
    sim.close()


def test_bin_tiles_matches_oracle_binning():
    import torch
    pg = _pg()
    rng = np.random.default_rng(0)
    nx, tile = (64, 32, 16), (8, 8, 4)
    n = 100003
    cells = np.stack([rng.integers(0, nx[d], n) for d in range(3)], axis=1).astype(np.int32)
    cnt, start, perm = pg.bin_tiles(nx, tile, torch.from_numpy(cells).cuda())
    g = workload.Grid(ndim=3, nx=nx, dx=(1.0, 1.0, 1.0), dt=0.1)
    _, counts, order = oracle.tile_bin(g, tile, cells.astype(np.float64) + 0.5)
    np.testing.assert_array_equal(cnt.cpu().numpy(), counts)
    np.testing.assert_array_equal(start.cpu().numpy(), np.concatenate([[0], np.cumsum(counts)[:-1]]))
    # the permutation is the oracle's stable order: tile by tile, increasing
    # particle index within each tile (bit-exact index work)
    np.testing.assert_array_equal(perm.cpu().numpy(), order)
    # more than 2^16 tiles (three 8-bit passes over the tile key), and one tile
    for nx2, tile2, n2 in (((512, 256, 8), (2, 2, 2), 300007), ((16, 8, 8), (16, 8, 8), 5003)):
        c2 = np.stack([rng.integers(0, nx2[d], n2) for d in range(3)], axis=1).astype(np.int32)
        cn, sn, pn = pg.bin_tiles(nx2, tile2, torch.from_numpy(c2).cuda())
        g2 = workload.Grid(ndim=3, nx=nx2, dx=(1.0, 1.0, 1.0), dt=0.1)
        _, counts2, order2 = oracle.tile_bin(g2, tile2, c2.astype(np.float64) + 0.5)
        np.testing.assert_array_equal(cn.cpu().numpy(), counts2)
        np.testing.assert_array_equal(pn.cpu().numpy(), order2)
    # empty input
    c0, s0, p0 = pg.bin_tiles(nx, tile, torch.zeros((0, 3), dtype=torch.int32, device="cuda"))
    assert int(c0.sum()) == 0 and int(s0.max()) == 0 and p0.numel() == 0


def test_device_lattice_loader_matches_generator():
    """The CUDA loader draws the same seeded lattice as the shared generator."""
    dx = (0.1, 0.1, 0.1)
    g = workload.Grid(ndim=3, nx=(16, 8, 8), dx=dx, dt=workload.courant_dt(dx, 3))
    sp = workload.Species(ppc=(2, 2, 1), uth=(0.05, 0.05, 0.05), ufl=(0.0, 0.1, 0.0), seed=20004)
    sim = _sim(g, [sp], "fp64", explicit=False)
    x, u = sim.particles()
    ids = sim.ids()
    xr, ur = workload.load_particles(g, sp, ids)
    np.testing.assert_array_equal(x, xr)
    np.testing.assert_allclose(u, ur, rtol=1e-14, atol=1e-16)
    sim.close()
    s32 = _sim(g, [sp], "fp32", explicit=False, tile=(8, 8, 8))
    _, cref, _ = oracle.tile_bin(g, (8, 8, 8), xr)
    np.testing.assert_array_equal(s32.tile_counts(), cref)
    x32, _ = s32.particles()
    i32 = s32.ids()
    assert _pos_err_cells(g, x32, workload.load_particles(g, sp, i32)[0]) < 1e-7
    s32.close()


def test_error_paths_on_gpu():
    pg = _pg()
    dx = (0.1, 0.1, 0.1)
    g = workload.Grid(ndim=3, nx=(12, 8, 8), dx=dx, dt=workload.courant_dt(dx, 3))
    sp = workload.Species(ppc=(1, 1, 1))
    with pytest.raises(pg.PicError) as e:
        pg.Simulation(g, [sp], precision="fp32", tile=(8, 8, 8))  # 12 not a multiple of 8
    assert e.value.code == -1
    with pytest.raises(pg.PicError) as e:
        pg.Simulation(g, [sp], precision="fp64", np_max=100)
    assert e.value.code == -5
    g2 = workload.Grid(ndim=3, nx=(16, 8, 8), dx=dx, dt=workload.courant_dt(dx, 3))
    x = np.full((4, 3), np.nan)
    for prec in ("fp32", "fp64"):
        with pytest.raises(pg.PicError) as e:
            pg.Simulation(g2, [sp], precision=prec, tile=(8, 8, 8), explicit=[(x, np.zeros((4, 3)), -1.0)])
        assert e.value.code == -1
    x = np.full((4, 3), 0.05)
    x[2, 1] = 0.8  # on the upper face of the box: outside [xmin, xmax)
    with pytest.raises(pg.PicError) as e:
        pg.Simulation(g2, [sp], precision="fp64", explicit=[(x, np.zeros((4, 3)), -1.0)])
    assert e.value.code == -1
    with pytest.raises(pg.PicError) as e:
        pg.Simulation(g2, [sp], precision="fp32", tile=(2, 2, 2))
    assert e.value.code == -8
