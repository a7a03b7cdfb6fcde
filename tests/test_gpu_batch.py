"""GPU tests of the batched scan (pic_batch_*): members of uneven size and
particle count advanced by one persistent tile-kernel launch per step and one
CUDA graph launch per step.

* against the same simulations run one by one (pic_step): after 10 steps,
  particles (by id) within 1e-4 of a cell / of u -- FP32 shared-memory current
  sums are order dependent, and those differences feed back through the fields;
* one step of each member against the FP64 oracle with the one-step FP32
  tolerances (2e-5 of a cell, 2e-5 (1 + |u|), grid values 2e-5 of their max);
* re-binning: a member whose tile storage overflows is re-binned between steps
  and keeps every particle;
* graph replay and direct launches give the same run (same tolerance as above),
  with and without moving windows;
* wakefield members (windows moving at c that shift on different steps, open
  x1, front injection, in-box pulses and one antenna) against the same members
  run alone and, for one member, the FP64 oracle, after 30 steps at 1e-4;
* a mixed batch (moving and periodic members, one with current smoothing)
  against its members run alone;
* wakefield members that spill and are re-binned inside the batch, and a
  batch whose second species is empty, against their members run alone.
"""
import os

import numpy as np
import pytest

import oracle
import workload

pytestmark = pytest.mark.gpu

DX = (0.1, 0.1, 1.0)


def _members(uth=0.3):
    out = []
    for i, (nx, ppc) in enumerate((((64, 32, 1), (2, 1, 1)), ((96, 48, 1), (1, 3, 1)), ((128, 16, 1), (2, 2, 1)),
                                   ((32, 64, 1), (3, 1, 1)), ((64, 64, 1), (1, 1, 1)))):
        g = workload.Grid(ndim=2, nx=nx, dx=DX, dt=workload.courant_dt(DX, 2), b0=(0.0, 0.0, 0.1 * i))
        s = workload.Species(ppc=ppc, uth=(uth,) * 3, ufl=(0.05 * i, 0.0, 0.0), seed=700 + i)
        out.append((g, [s]))
    return out


def _compare(a, b, tol):
    xa, ua = a.particles()
    ia = a.ids()
    xb, ub = b.particles()
    ib = b.ids()
    assert xa.shape == xb.shape
    pa, pb = np.argsort(ia), np.argsort(ib)
    np.testing.assert_array_equal(ia[pa], ib[pb])
    L = np.array([a.shape[2] * DX[0], a.shape[1] * DX[1], 1.0])
    d = xa[pa] - xb[pb]
    d = d - L * np.round(d / L)
    assert np.max(np.abs(d[:, :2] / np.array(DX[:2]))) < tol
    assert np.max(np.abs(ua[pa] - ub[pb])) < tol


def test_batch_matches_members_run_one_by_one():
    import paper_1503_00276_gb300 as pg
    mem = _members()
    batch = pg.Batch(mem, track_ids=True)
    assert batch.info()["tile"] == (32, 16, 1)
    batch.step(10)
    info = batch.info()
    # per step, for all members together: clear, tile kernel, fold, B half, E, B half, guards
    assert info["steps"] == 10 and info["launches"] == 10 * 7
    for i, (g, sps) in enumerate(mem):
        solo = pg.Simulation(g, sps, precision="fp32", tile=(32, 16), track_ids=True)
        solo.step(10)
        m = batch.sim(i)
        _compare(m, solo, 1e-4)
        d = m.diag()
        assert d["step"] == 10 and d["error_flags"] == 0
        assert d["gauss_resid_max"] <= 1e-5 * d["rho_abs_max"]
        solo.close()
    with pytest.raises(RuntimeError):
        batch.sim(0).step(1)
    batch.close()


def test_batch_one_step_matches_oracle():
    import paper_1503_00276_gb300 as pg
    mem = _members(uth=0.5)[:3]
    batch = pg.Batch(mem, track_ids=True)
    refs = []
    for i, (g, sps) in enumerate(mem):
        f = workload.random_fields(g, seed=50 + i, amp=0.2)
        m = batch.sim(i)
        for c, name in enumerate(["E1", "E2", "E3", "B1", "B2", "B3"]):
            m.set_field(name, f[c])
        ref = oracle.from_workload(g, sps, fields=f)
        ref.particle_phase()
        jref = [c.copy() for c in ref.cur]
        ref.field_solve()
        refs.append((ref, jref))
    batch.step(1)
    for i, (g, sps) in enumerate(mem):
        ref, jref = refs[i]
        m = batch.sim(i)
        x, u = m.particles()
        ids = m.ids()
        L = np.array([g.nx[0] * DX[0], g.nx[1] * DX[1], 1.0])
        d = x - ref.x[0][ids]
        d = d - L * np.round(d / L)
        assert np.max(np.abs(d[:, :2] / np.array(DX[:2]))) < 2e-5
        assert np.max(np.abs(u - ref.u[0][ids]) / (1 + np.abs(ref.u[0][ids]))) < 2e-5
        for c, name in enumerate(["J1", "J2", "J3"]):
            jm = np.max(np.abs(jref[c]))
            assert np.max(np.abs(m.fields(name) - jref[c])) < 2e-5 * jm, (i, name)
        for c, name in enumerate(["E1", "E2", "E3", "B1", "B2", "B3"]):
            assert np.max(np.abs(m.fields(name) - ref.fld[c])) < 2e-5 * np.max(np.abs(ref.fld[c])), (i, name)
    batch.close()


def test_batch_rebins_a_member_whose_tiles_overflow():
    import paper_1503_00276_gb300 as pg
    mem = _members(uth=0.8)
    batch = pg.Batch(mem, track_ids=True, slack=1e-3)
    n0 = [batch.sim(i).n_particles() for i in range(len(mem))]
    batch.step(8)
    # bit 1 of error_flags: some tile storage spilled (and was re-binned)
    assert any(batch.sim(i).diag()["error_flags"] & 2 for i in range(len(mem)))
    for i, (g, sps) in enumerate(mem):
        m = batch.sim(i)
        assert m.n_particles() == n0[i]
        assert np.array_equal(np.sort(m.ids()), np.arange(n0[i]))
        assert m.diag()["error_flags"] & 1 == 0
        solo = pg.Simulation(g, sps, precision="fp32", tile=(32, 16), track_ids=True, slack=1e-3)
        solo.step(8)
        _compare(m, solo, 1e-4)
        solo.close()
    batch.close()


@pytest.mark.parametrize("wake", [False, True])
def test_batch_graph_and_direct_launches_agree(wake):
    import paper_1503_00276_gb300 as pg
    mem = _wake_members() if wake else _members()
    a = pg.Batch(mem, track_ids=True)
    os.environ["PICGB_BATCH_GRAPH"] = "0"
    try:
        b = pg.Batch(mem, track_ids=True)
    finally:
        del os.environ["PICGB_BATCH_GRAPH"]
    a.step(6)
    b.step(6)
    for i in range(len(mem)):
        if wake:
            _compare_window(a.sim(i), b.sim(i), mem[i][0].dx, 1e-4)
        else:
            _compare(a.sim(i), b.sim(i), 1e-4)
    a.close()
    b.close()


def _wake_members():
    """Four small wakefield members: windows moving at c from different times
    and with different cell sizes (so they shift on different steps), warm
    plasmas of different densities, in-box pulses of different a0 and one
    pulse driven in through the lower x1 boundary."""
    spec = (  # nx, dx, ppc, density, window_start, laser
        ((128, 16, 1), (0.05, 0.2, 1.0), (2, 2, 1), 1.0, 0.0,
         workload.Laser(vosc=1.0, rkkp=10.0, w0=1.2, rise=0.6, fall=0.6, start=1.0)),
        ((64, 32, 1), (0.1, 0.2, 1.0), (2, 1, 1), 0.7, 0.5,
         workload.Laser(vosc=2.0, rkkp=8.0, w0=2.0, rise=1.0, fall=1.0, start=1.0)),
        ((96, 16, 1), (0.05, 0.2, 1.0), (1, 2, 1), 1.5, 0.3,
         workload.Laser(vosc=0.5, rkkp=8.0, w0=1.2, rise=0.6, fall=0.6, start=0.1, antenna=True, focus=2.0)),
        ((128, 32, 1), (0.05, 0.2, 1.0), (2, 2, 1), 0.5, 0.0,
         workload.Laser(vosc=3.0, rkkp=10.0, w0=2.0, rise=0.8, fall=0.8, start=1.0)),
    )
    out = []
    for i, (nx, dx, ppc, dens, t0, las) in enumerate(spec):
        g = workload.Grid(ndim=2, nx=nx, dx=dx, dt=workload.courant_dt(dx, 2), rho_bg=dens, move_window=True,
                          window_start=t0)
        s = workload.Species(ppc=ppc, uth=(0.02, 0.02, 0.02), density=dens, seed=800 + i)
        out.append((g, [s], las))
    return out


def _compare_window(a, b, dx, tol):
    """Same surviving particles (ids), positions in cells and momenta within
    tol; every field within tol of its maximum."""
    ia, ib = a.ids(), b.ids()
    assert np.array_equal(np.sort(ia), np.sort(ib))
    (xa, ua), (xb, ub) = a.particles(), b.particles()
    pa, pb = np.argsort(ia), np.argsort(ib)
    L2 = a.shape[1] * dx[1]
    d = xa[pa] - xb[pb]
    d[:, 1] -= L2 * np.round(d[:, 1] / L2)
    assert np.max(np.abs(d[:, 0] / dx[0])) < tol and np.max(np.abs(d[:, 1] / dx[1])) < tol
    assert np.max(np.abs(ua[pa] - ub[pb]) / (1 + np.abs(ub[pb]))) < tol
    for name in ("E1", "E2", "E3", "B1", "B2", "B3"):
        fb = b.fields(name)
        m = np.max(np.abs(fb))
        if m > 0:
            assert np.max(np.abs(a.fields(name) - fb)) < tol * m, name


def test_batch_of_wakefield_members_with_windows_matches_members_alone_and_oracle():
    """Four members with moving windows and lasers, 30 steps as one batch: each
    member equals the same member run alone through pic_step (ids, positions,
    momenta, fields at 1e-4; shift counts and particle counts exactly), and
    member 0 equals the FP64 oracle at 1e-4 (FP32 against FP64 over 30 steps,
    the tolerance of the single moving-window parity test)."""
    import paper_1503_00276_gb300 as pg
    mem = _wake_members()
    n = 30
    batch = pg.Batch(mem, track_ids=True)
    assert batch.info()["tile"] == (32, 16, 1)
    g0, sps0, las0 = mem[0]
    ref = oracle.from_workload(g0, sps0)
    for c, f in enumerate(oracle.laser_fields(g0, las0)):
        ref.fld[c] += f
    batch.step(n)
    info = batch.info()
    # per step: the 7 stages, fresh columns, window shift, counter gather, one antenna plane
    assert info["steps"] == n and info["launches"] == n * 11
    shifts = []
    for i, (g, sps, las) in enumerate(mem):
        solo = pg.Simulation(g, sps, precision="fp32", tile=(32, 16), track_ids=True)
        solo.add_laser(las)
        solo.step(n)
        m = batch.sim(i)
        dm, ds = m.diag(), solo.diag()
        assert dm["step"] == n and dm["error_flags"] & ~2 == 0
        assert dm["n_particles"] == ds["n_particles"] == m.n_particles()
        # one-cell shifts so far: the window moves at c from window_start on
        shifts.append(max(0, int(np.floor((n * g.dt - g.window_start) / g.dx[0]))))
        # fields are stored window-relative: a member shifted a different
        # number of times would differ from its solo run by whole cells
        _compare_window(m, solo, g.dx, 1e-4)
        solo.close()
    # the members shift on different steps and by different counts
    assert len(set(shifts)) >= 3 and min(shifts) >= 10, shifts
    ref.step(n)
    assert ref.shifts == shifts[0]
    m0 = batch.sim(0)
    ids = m0.ids()
    x, u = m0.particles()
    assert np.array_equal(np.sort(ids), np.sort(ref.ids[0]))
    pos = {int(i): k for k, i in enumerate(ref.ids[0])}
    order = np.array([pos[int(i)] for i in ids])
    d = x - ref.x[0][order]
    L2 = g0.nx[1] * g0.dx[1]
    d[:, 1] -= L2 * np.round(d[:, 1] / L2)
    assert np.max(np.abs(d[:, 0] / g0.dx[0])) < 1e-4 and np.max(np.abs(d[:, 1] / g0.dx[1])) < 1e-4
    assert np.max(np.abs(u - ref.u[0][order]) / (1 + np.abs(ref.u[0][order]))) < 1e-4
    for c, name in enumerate(("E1", "E2", "E3", "B1", "B2", "B3")):
        mref = np.max(np.abs(ref.fld[c]))
        if mref > 0:
            assert np.max(np.abs(m0.fields(name) - ref.fld[c])) < 1e-4 * mref, name
    batch.close()


def test_mixed_batch_of_windows_periodic_and_smoothed_members_matches_members_alone():
    """One batch holding two wakefield members (one with an antenna pulse),
    a periodic member and a periodic member whose current is smoothed (two
    passes along x1, one along x2, launched per member inside the step's
    graph): after 20 steps every member equals the same member run alone."""
    import dataclasses

    import paper_1503_00276_gb300 as pg
    wake = _wake_members()
    per = _members()
    g_s, s_s = per[1]
    g_s = dataclasses.replace(g_s, smooth_level=(2, 1, 0))
    mem = [wake[0], per[0], wake[2], (g_s, s_s)]
    n = 20
    batch = pg.Batch(mem, track_ids=True)
    batch.step(n)
    # stages + fresh columns, shift, gather + one antenna + 3 smoothing passes x 3 components
    assert batch.info()["launches"] == n * (7 + 3 + 1 + 9)
    for i, m in enumerate(mem):
        g, sps = m[0], m[1]
        solo = pg.Simulation(g, sps, precision="fp32", tile=(32, 16), track_ids=True)
        if len(m) > 2:
            solo.add_laser(m[2])
        solo.step(n)
        b = batch.sim(i)
        assert b.diag()["n_particles"] == solo.diag()["n_particles"]
        if g.move_window:
            _compare_window(b, solo, g.dx, 1e-4)
        else:
            _compare(b, solo, 1e-4)
            for name in ("E1", "E2", "E3", "B1", "B2", "B3", "J1", "J2", "J3"):
                f = solo.fields(name)
                top = np.max(np.abs(f))
                if top > 0:
                    assert np.max(np.abs(b.fields(name) - f)) < 1e-4 * top, (i, name)
        solo.close()
    batch.close()


def test_batch_rebins_wakefield_members_and_keeps_windows():
    """Wakefield members with almost no spare slots in their tile regions
    spill and are re-binned between steps inside the batch (re-sized regions,
    tables and graph rebuilt); after 20 steps every member equals the same
    member run alone with the same regions."""
    import paper_1503_00276_gb300 as pg
    mem = _wake_members()[:3]
    n = 20
    batch = pg.Batch(mem, track_ids=True, slack=1e-3)
    batch.step(n)
    assert any(batch.sim(i).diag()["error_flags"] & 2 for i in range(len(mem)))  # some member spilled
    for i, (g, sps, las) in enumerate(mem):
        solo = pg.Simulation(g, sps, precision="fp32", tile=(32, 16), track_ids=True, slack=1e-3)
        solo.add_laser(las)
        solo.step(n)
        m = batch.sim(i)
        assert m.diag()["error_flags"] & 1 == 0
        assert m.n_particles() == solo.n_particles()
        _compare_window(m, solo, g.dx, 1e-4)
        solo.close()
    batch.close()


def test_batch_with_an_empty_species():
    """Two species per member, the second one empty (a density profile that
    is zero everywhere): the batch steps and equals the members run alone."""
    import paper_1503_00276_gb300 as pg
    zero = (np.array([0.0, 1.0]), np.array([0.0, 0.0]))
    empty = workload.Species(rqm=1.0, ppc=(1, 1, 1), seed=5, profile=(zero, None, None), den_min=0.0)
    mem = [(g, [s, empty]) for g, (s,) in _members()[:3]]
    batch = pg.Batch(mem, track_ids=True)
    batch.step(5)
    for i, (g, sps) in enumerate(mem):
        solo = pg.Simulation(g, sps, precision="fp32", tile=(32, 16), track_ids=True)
        solo.step(5)
        m = batch.sim(i)
        assert m.n_particles(1) == 0
        _compare(m, solo, 1e-4)
        solo.close()
    batch.close()
