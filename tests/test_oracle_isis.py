"""Pins of the oracle's ISIS current deposit (thesis ch. 3, the comparison of
the ISIS and TRISTAN methods): for a 2D path the ISIS current is the average of
the two orders of orthogonal moves over the whole path (no split at cell
faces).  What fixes it:
* a particle that stays in its cell gets the same current from both methods;
* both conserve charge exactly, so the ISIS current satisfies the discrete
  continuity equation and differs from the TRISTAN current by a divergence-free
  field;
* a worked crossing example, computed by hand from the definition
  (tests/golden/isis_crossing.json);
* J3 (out of plane) is the time integral along the straight path, the same for
  both methods."""
import json
import os

import numpy as np
import pytest

import oracle
import workload

DX = (0.1, 0.1, 1.0)


def _grid(deposit="isis", nx=(8, 8, 1)):
    return workload.Grid(ndim=2, nx=nx, dx=DX, dt=workload.courant_dt(DX, 2), deposit=deposit)


def _div(g, cur):
    j1, j2 = cur[0][0], cur[1][0]
    return (j1 - np.roll(j1, 1, 1)) / g.dx[0] + (j2 - np.roll(j2, 1, 0)) / g.dx[1]


def test_isis_equals_tristan_for_in_cell_moves():
    g = _grid()
    rng = np.random.default_rng(3)
    for _ in range(200):
        c = rng.integers(0, 8, 2)
        a = (c + rng.uniform(0.0, 1.0, 2)) * 0.1
        b = (c + rng.uniform(0.0, 1.0, 2)) * 0.1
        xo, xn = np.array([a[0], a[1], 0.0]), np.array([b[0], b[1], 0.0])
        ji = oracle.deposit_isis(g, xo, xn, 0.3, -0.7)
        jv = oracle.deposit_vb(g, xo, xn, 0.3, -0.7)
        for k in range(3):
            np.testing.assert_allclose(ji[k], jv[k], rtol=0, atol=1e-13)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_isis_continuity_and_curl_only_difference(seed):
    g = _grid()
    rng = np.random.default_rng(seed)
    q = -0.37
    worst = 0.0
    for _ in range(100):
        a = rng.uniform(0.0, 0.8, 2)
        d = rng.uniform(-0.095, 0.095, 2)  # up to 0.95 cell: face and corner crossings
        b = a + d
        xo, xn = np.array([a[0], a[1], 0.0]), np.array([b[0], b[1], 0.0])
        ji = oracle.deposit_isis(g, xo, xn, 0.0, q)
        jv = oracle.deposit_vb(g, xo, xn, 0.0, q)
        r0 = oracle.deposit_rho(g, xo[None, :], q)[0]
        r1 = oracle.deposit_rho(g, np.mod(xn, 0.8)[None, :], q)[0]
        res = (r1 - r0) / g.dt + _div(g, ji)
        scale = abs(q) / g.dvol / g.dt
        worst = max(worst, np.max(np.abs(res)) / scale)
        # the two methods differ by a divergence-free current only
        assert np.max(np.abs(_div(g, [ji[0] - jv[0], ji[1] - jv[1]]))) < 1e-12 * scale
    assert worst < 1e-13, worst


def test_isis_hand_worked_crossing_example():
    path = os.path.join(os.path.dirname(__file__), "golden", "isis_crossing.json")
    with open(path) as f:
        case = json.load(f)
    g = _grid(nx=(4, 4, 1))
    a, b = np.array(case["x_old_cells"] + [0.0]), np.array(case["x_new_cells"] + [0.0])
    q = 1.0
    ji = oracle.deposit_isis(g, a * 0.1, b * 0.1, 0.0, q)
    f1 = q * g.dx[0] / (g.dt * g.dvol)
    f2 = q * g.dx[1] / (g.dt * g.dvol)
    exp1 = np.zeros((4, 4))
    exp2 = np.zeros((4, 4))
    for i, j, v in case["j1_cell_units"]:
        exp1[j, i] = v * f1
    for i, j, v in case["j2_cell_units"]:
        exp2[j, i] = v * f2
    np.testing.assert_allclose(ji[0][0], exp1, rtol=0, atol=1e-12 * f1)
    np.testing.assert_allclose(ji[1][0], exp2, rtol=0, atol=1e-12 * f2)
    # and TRISTAN differs here (it splits the path at the face x1 = 1)
    jv = oracle.deposit_vb(g, a * 0.1, b * 0.1, 0.0, q)
    assert np.max(np.abs(jv[0][0] - exp1)) > 0.01 * f1


def test_isis_out_of_plane_current_is_tristans():
    g = _grid()
    xo, xn = np.array([0.275, 0.333, 0.0]), np.array([0.352, 0.281, 0.0])
    ji = oracle.deposit_isis(g, xo, xn, 0.42, -1.0)
    jv = oracle.deposit_vb(g, xo, xn, 0.42, -1.0)
    np.testing.assert_allclose(ji[2], jv[2], rtol=0, atol=1e-14)


def test_isis_rejected_in_3d():
    g = workload.Grid(ndim=3, nx=(4, 4, 4), dx=(0.1,) * 3, dt=0.05, deposit="isis")
    with pytest.raises(ValueError):
        oracle.State(g, [], [], [], [])
