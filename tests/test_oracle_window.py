"""Pins of the oracle's moving window and laser set-up (thesis: dynamic
simulation spaces; the pulse input section).

* A vacuum pulse from laser_fields moves in +x1 at the group velocity of the
  discrete Yee scheme (computed from its dispersion relation; a wrong B sign
  splits the pulse into two halves moving both ways, a wrong stagger or
  direction moves the centroid the wrong way).
* In a window moving at c the same pulse stays where it was up to the lag
  (c - v_g) t -- which pins the direction and the timing of the shifts.
* A cold plasma at rest keeps its particle count across shifts (a back column
  discarded, a front column injected each time), every particle stays inside
  the window, and injected particles continue the id sequence and sit on the
  loader's sub-lattice of the new front column.
"""
import dataclasses
import math

import numpy as np

import oracle
import workload


def _vacuum(grid):
    return oracle.State(grid, [], [], [], [])


def _centroid(st, dx1, xmin1):
    e2 = st.fld[1][0] ** 2
    w = e2.sum(axis=0)
    x = xmin1 + np.arange(w.size) * dx1
    return float((w * x).sum() / w.sum())


def _group_velocity(k, dx, dt):
    # 1D Yee: sin(w dt / 2) = (dt / dx) sin(k dx / 2)  ->  v_g = dw/dk
    s = dt / dx * math.sin(0.5 * k * dx)
    return math.cos(0.5 * k * dx) / math.sqrt(1.0 - s * s)


def _grid(move):
    dx = (0.05, 0.4, 1.0)
    return workload.Grid(ndim=2, nx=(400, 16, 1), dx=dx, dt=workload.courant_dt(dx, 2), move_window=move)


LASER = workload.Laser(vosc=0.1, rkkp=6.0, w0=1e3, rise=2.0, length=0.0, fall=2.0, start=8.0)


def test_vacuum_pulse_moves_forward_at_the_discrete_group_velocity():
    g = _grid(False)
    st = _vacuum(g)
    for c, f in enumerate(oracle.laser_fields(g, LASER)):
        st.fld[c][...] = f
    x0 = _centroid(st, g.dx[0], 0.0)
    n = 80
    st.step(n)
    x1 = _centroid(st, g.dx[0], 0.0)
    vg = _group_velocity(LASER.rkkp, g.dx[0], g.dt)
    assert abs((x1 - x0) - vg * n * g.dt) < 0.02 * n * g.dt, (x1 - x0, vg * n * g.dt)
    # the pulse moves forward as a whole (a wrong B sign would leave half of it
    # behind); the slowly varying envelope and the discrete E/B ratio leave <1%
    assert np.abs(st.fld[1][0][:, : int(x0 / g.dx[0]) - 40]).max() < 0.02 * 0.1 * 6.0


def test_window_keeps_a_vacuum_pulse_in_place_up_to_the_dispersion_lag():
    g = _grid(True)
    st = _vacuum(g)
    for c, f in enumerate(oracle.laser_fields(g, LASER)):
        st.fld[c][...] = f
    x0 = _centroid(st, g.dx[0], 0.0)
    n = 120
    st.step(n)
    t = n * g.dt
    assert st.shifts == int(math.floor(t / g.dx[0]))
    x1 = _centroid(st, g.dx[0], st.og.xmin[0])  # lab frame
    vg = _group_velocity(LASER.rkkp, g.dx[0], g.dt)
    assert abs((x1 - x0) - vg * t) < 0.02 * t
    # in the window frame the pulse lags by (1 - v_g) t plus the shift granularity
    xw = x1 - st.og.xmin[0]
    assert abs(xw - (x0 - (1.0 - vg) * t - (t - st.shifts * g.dx[0]))) < 0.03 * t + g.dx[0]


def test_window_removes_the_back_column_and_injects_the_front_column():
    g = dataclasses.replace(_grid(True), nx=(40, 8, 1))
    sp = workload.Species(ppc=(2, 2, 1), uth=(0.0, 0.0, 0.0), seed=3)
    st = oracle.from_workload(g, [sp])
    n0 = st.x[0].shape[0]
    steps = 25
    st.step(steps)
    m = st.shifts
    assert m == int(math.floor(steps * g.dt / g.dx[0])) and m > 5
    assert st.x[0].shape[0] == n0  # cold plasma at rest: one column out, one in per shift
    lo = st.og.xmin[0]
    assert abs(lo - m * g.dx[0]) < 1e-12
    assert (st.x[0][:, 0] >= lo).all() and (st.x[0][:, 0] < lo + g.nx[0] * g.dx[0]).all()
    ids = np.sort(st.ids[0])
    # survivors: the initial particles of columns >= m (index = cell * ppc + sub,
    # x1 fastest), then every injected one
    init = np.arange(n0)
    expect = np.concatenate([init[(init // 4) % g.nx[0] >= m], np.arange(n0, n0 + m * g.nx[1] * 4)])
    np.testing.assert_array_equal(ids, expect)
    # the last injection sits on the sub-lattice of the front column
    last = st.ids[0] >= n0 + (m - 1) * g.nx[1] * 4
    off = (st.x[0][last, 0] - lo) / g.dx[0] - (g.nx[0] - 1)
    np.testing.assert_allclose(np.sort(np.unique(np.round(off, 12))), [0.25, 0.75])
    # net charge density (electrons + ion background) of the window: zero away
    # from the open x1 edges (cold plasma at rest, uniform after the shifts)
    r = st.rho()
    assert np.abs(r[0][:, 1:-1]).max() < 1e-12
