"""Pins of the r-z (2D cylindrically symmetric) oracle against what the thesis'
equations and the mathematics fix: discrete conservation laws of the field
solve and deposit, closed-form orbits, exact densities of a lattice-loaded
column, a closed-form field energy."""
import math

import numpy as np
import pytest

import workload
from oracle.cyl import CylState

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def _random_state(seed=1, n=120, nz=16, nr=10, u_sd=0.3, q=-0.01):
    g = workload.cyl_grid(nz, nr, 0.1, 0.1)
    s = CylState(nz, nr, 0.1, 0.1, g.dt)
    rng = np.random.default_rng(seed)
    x = np.c_[rng.uniform(0, nz * 0.1, n), rng.uniform(0, 0.7 * s.rmax, n), np.zeros(n)]
    u = rng.normal(0, u_sd, (n, 3))
    s.add_species(x, u, q, -1.0)
    return s


def test_div_b_stays_zero_including_the_axis_cell():
    """Faraday's law in flux form keeps div B = 0 in every cell; on the axis
    the disc of radius dr/2 (eq. 2d-field-solve-cyl-b1-axis: the factor 4 is
    its circumference over its area times dr)."""
    s = _random_state()
    rng = np.random.default_rng(5)
    for c in range(3):  # random E, B = 0
        s.F[c][:] = rng.normal(0, 1, s.F[c].shape)
    s.boundary_fields()
    s.step(15)
    bmax = max(np.abs(s.F[c]).max() for c in range(3, 6))
    assert bmax > 1e-2
    assert np.abs(s.div_b()).max() <= 1e-12 * bmax / s.dr


def test_gauss_residual_is_invariant():
    """Yee + a charge-conserving deposit keep div E - rho constant at every
    node (cylindrical divergence with the radius weights of the z components)."""
    s = _random_state()
    g0 = s.gauss_residual().copy()
    assert np.abs(g0).max() > 0.1
    s.step(12)
    assert np.abs(s.gauss_residual() - g0).max() <= 1e-12 * np.abs(g0).max()


def test_continuity_node_by_node():
    """(rho^{n+1} - rho^n)/dt + div j^{n+1/2} = 0 with j = I / V(r) and
    rho = Q / V(r) at every node row off the axis, the row at r = dr/2
    included (it holds the folded mirror row)."""
    s = _random_state(seed=3)
    s.step(2)
    r0 = s.rho()[1:s.nr].copy()
    s.step(1)
    r1 = s.rho()[1:s.nr]
    res = (r1 - r0) / s.dt + s.div_j()
    assert np.abs(res).max() <= 1e-12 * np.abs(r0).max() / s.dt


def test_gauss_invariant_through_absorption_at_the_wall():
    """A particle driven into the wall is absorbed there; the residual at the
    node rows inside (1 .. nr-1) does not change."""
    s = _random_state(seed=7, n=40)
    x = np.array([[0.55, s.rmax - 0.03, 0.0], [0.85, s.rmax - 0.02, 0.0]])
    u = np.array([[0.1, 3.0, 0.5], [-0.2, 5.0, -1.0]])
    s.add_species(x, u, -0.02, -1.0)
    g0 = s.gauss_residual().copy()
    s.step(3)
    assert np.all(s.species[1]["x"][:, 1] == -1.0)
    assert np.abs(s.gauss_residual() - g0).max() <= 1e-12 * np.abs(g0).max()


def test_lattice_column_has_exact_uniform_density():
    """Ring charge q r (reading C2) on a lattice symmetric about each node row
    gives rho = -density exactly at the node rows off the axis (2 .. nr-1):
    the first moments of the hat weights cancel, and V = r_j dr dz."""
    g = workload.cyl_grid(8, 10, 0.1, 0.1)
    sp = workload.Species(rqm=-1.0, ppc=(2, 3, 1), density=1.0, seed=1)
    x, u = workload.load_cylindrical(g, sp)
    s = CylState(8, 10, 0.1, 0.1, g.dt)
    s.add_species(x, u, workload.macro_charge(g, sp), -1.0)
    rho = s.rho()
    np.testing.assert_allclose(rho[2:10], -1.0, rtol=0, atol=1e-13)
    # the wrong volume (at the half row above) is off by (j - 1/2) / j
    assert abs(rho[2, 0] * (1.5 / 2.0) + 1.0) > 0.2


@pytest.mark.parametrize("u0", [(0.3, 0.0, 0.8), (-0.2, 0.5, 0.4), (0.1, -0.3, 0.0)])
def test_free_ring_follows_the_straight_line_in_3d(u0):
    """No fields, no charge: the pseudo-3D move + rotation is exact for a
    straight line, so r_n = |(r0, 0) + n dt (v_r, v_theta)| and z moves
    uniformly; r p_theta (angular momentum) is conserved (eq.
    2d-cyl-position-update-3)."""
    g = workload.cyl_grid(16, 40, 0.1, 0.1)
    s = CylState(16, 40, 0.1, 0.1, g.dt)
    r0, z0 = 1.3, 0.4
    s.add_species([[z0, r0, 0.0]], [u0], 0.0, -1.0)
    u = np.array(u0)
    gam = math.sqrt(1 + u @ u)
    v = u / gam
    for n in range(1, 25):
        s.step(1)
        x = s.species[0]["x"][0]
        uu = s.species[0]["u"][0]
        rn = math.hypot(r0 + n * s.dt * v[1], n * s.dt * v[2])
        assert abs(x[1] - rn) <= 1e-13 * r0
        L = 16 * 0.1
        assert abs(((x[0] - z0 - n * s.dt * v[0]) + L / 2) % L - L / 2) <= 1e-13
        assert abs(x[1] * uu[2] - r0 * u[2]) <= 1e-13 * (1 + abs(r0 * u[2]))
        assert abs(uu @ uu - u @ u) <= 1e-13 * (u @ u)


def test_axis_centred_gyration_keeps_its_radius():
    """Uniform axial B: Boris rotates (p_r, p_theta) by theta = 2 atan(|t|) each
    step and the Cartesian positions lie on a circle of radius
    R = |v| dt / (2 sin(theta/2)).  A ring on that circle about the axis keeps
    r = R at every step, to rounding."""
    B, rqm = 2.0, -1.0
    g = workload.cyl_grid(16, 40, 0.1, 0.1, b0=(B, 0.0, 0.0))
    s = CylState(16, 40, 0.1, 0.1, g.dt, b0=(B, 0.0, 0.0))
    umag = 0.6
    gam = math.sqrt(1 + umag * umag)
    theta = 2.0 * math.atan(abs(s.dt * B / (2.0 * rqm)) / gam)
    R = (umag / gam) * s.dt / (2.0 * math.sin(theta / 2))
    # B/rqm < 0: the momentum turns counter-clockwise in the (r, theta) plane;
    # u^{-1/2} is the chord from the previous point of the circle
    sgn = 1.0 if B / rqm < 0 else -1.0
    u = np.array([0.0, umag * math.sin(theta / 2), sgn * umag * math.cos(theta / 2)])
    s.add_species([[0.8, R, 0.0]], [u], 0.0, rqm)
    for _ in range(60):
        s.step(1)
        x = s.species[0]["x"][0]
        assert abs(x[1] - R) <= 1e-12 * R
    uu = s.species[0]["u"][0]
    assert abs(math.sqrt(uu @ uu) - umag) <= 1e-13


def test_theta_current_of_a_ring_vanishes_on_the_axis():
    """A ring of radius eps -> 0 carries no azimuthal current: with the odd
    fold of the mirror row (reading C4) jtheta at r = dr/2 is proportional to
    eps (an even fold would leave it finite)."""
    out = []
    for eps in (0.01, 0.02):
        g = workload.cyl_grid(16, 10, 0.1, 0.1)
        s = CylState(16, 10, 0.1, 0.1, g.dt)
        s.add_species([[0.55, eps * s.dr, 0.0]], [[0.0, 0.0, 1e-7]], -1.0, -1.0, w=[1.0 / (eps * s.dr)])
        s.step(1)
        out.append(s.J[2][1].sum())
    assert out[0] != 0.0
    assert abs(out[1] / out[0] - 2.0) <= 1e-4


def test_field_energy_of_a_uniform_axial_field():
    """Bz = B0 everywhere inside the wall: the half rows' volumes (axis disc
    included) tile the cylinder of radius r_max exactly, so the energy is
    B0^2 / 2 * pi r_max^2 * L."""
    s = CylState(12, 9, 0.1, 0.2, 0.01)
    s.F[3][:] = 1.7
    s.boundary_fields()
    L = 12 * 0.1
    assert abs(s.field_energy() - 0.5 * 1.7 ** 2 * math.pi * s.rmax ** 2 * L) <= 1e-12 * s.field_energy()


def _radial_te_eig(n, dr=1.0):
    """Largest eigenvalue of the radial part of the r-z solve for the Etheta,
    Bz family (Etheta on node rows 1..n-1 with Etheta_n = 0 at the wall, Bz on
    half rows 0..n-1 with the axis rule), from the discrete stencils."""
    rn = lambda j: (j - 0.5) * dr
    rh = lambda j: j * dr
    D = np.zeros((n - 1, n))  # d Etheta_j / dt = -(Bz_j - Bz_{j-1}) / dr
    G = np.zeros((n, n - 1))  # d Bz_j / dt from Etheta
    for j in range(1, n):
        D[j - 1, j] = -1.0 / dr
        D[j - 1, j - 1] = 1.0 / dr
    G[0, 0] = -4.0 / dr
    for j in range(1, n):
        if j + 1 <= n - 1:
            G[j, j] -= rn(j + 1) / (rh(j) * dr)
        G[j, j - 1] += rn(j) / (rh(j) * dr)
    return float(np.max(np.real(np.linalg.eigvals(-G @ D))))


def test_time_step_bound_of_the_r_z_solve():
    """The leapfrog is stable while dt^2 (4/dz^2 + lambda_r) / 4 < 1, lambda_r
    the largest radial eigenvalue: 1.2105 x 4/dr^2 with the axis rule (a mode
    bound to the axis, the same for every nr >= 10).  Vacuum fields stay
    bounded over 4000 steps at 0.99 of that bound and blow up at 0.99 of the
    Cartesian one, which lies above it."""
    lam = [_radial_te_eig(n) / 4.0 for n in (12, 40, 160)]
    assert max(lam) - min(lam) < 1e-8 and abs(lam[0] - workload.CYL_RADIAL_EIG) < 1e-4
    for dt, grows in ((workload.cyl_courant_dt(0.1, 0.1), False), (workload.courant_dt((0.1, 0.1, 1.0), 2), True)):
        s = CylState(16, 12, 0.1, 0.1, dt)
        rng = np.random.default_rng(0)
        for c in range(6):
            s.F[c][:] = rng.normal(0, 1, s.F[c].shape)
        s.boundary_fields()
        e0 = s.field_energy()
        s.step(4000 if not grows else 600)
        ratio = s.field_energy() / e0
        assert (not np.isfinite(ratio) or ratio > 1e3) == grows, (dt, ratio)
